// Tables of the tensor-core A^T (tcs_adjoint_pool, tc_stream.cuh): the first
// record of every tile, the per-pixel fixed-point accumulators and the bound
// that sets their scale, the table operand, and the launch: max |e| of the
// residual, the pool (one integer addition per record into its pixel's sum),
// then the sums turned into FP32.  Integer addition is associative, so the
// result does not depend on which CTA adds what when: it is reproducible bit
// for bit.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "tc_stream.cuh"

namespace mbir {

// *emax = bits of max |e| over n values (non-negative floats order as their bits; a non-finite value
// gives bits >= 0x7f800000).
template <typename T>
__global__ void tc_emax_kernel(const T* __restrict__ e, long long n, unsigned int* __restrict__ emax)
{
    unsigned int m = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        float v;
        if constexpr (sizeof(T) == 2) v = __bfloat162float(e[i]);
        else v = e[i];
        m = max(m, __float_as_uint(fabsf(v)));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m) atomicMax(emax, m);
}

// The residual's pending MAP update e -= alpha q (alpha = sc[alpha_slot], the previous iteration's step),
// its BF16 copy when there is one, and *emax = bits of max |e| over the values the adjoint then reads (the
// BF16 copy in the BF16 form): the update and the scale's pass over e in one.
__global__ void tc_emax_update_kernel(float* __restrict__ e, __nv_bfloat16* __restrict__ ebf,
                                      const float* __restrict__ q, const double* __restrict__ sc, int alpha_slot,
                                      long long n, unsigned int* __restrict__ emax)
{
    const float a = (float)sc[alpha_slot];
    unsigned int m = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        float v = fmaf(-a, q[i], e[i]);
        e[i] = v;
        if (ebf) {
            const __nv_bfloat16 h = __float2bfloat16_rn(v);
            ebf[i] = h;
            v = __bfloat162float(h);
        }
        m = max(m, __float_as_uint(fabsf(v)));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m) atomicMax(emax, m);
}

// b[v] from the fixed-point sums (tcs_finish_pixel)
__global__ void tc_finish_kernel(int N, const unsigned long long* __restrict__ acc,
                                 const unsigned int* __restrict__ emax, float bound, float* __restrict__ b)
{
    const unsigned int eb = *emax;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < N; v += gridDim.x * blockDim.x)
        b[v] = tcs_finish_pixel(acc[v], eb, bound);
}

// *wmax = bits of the largest record weight w (the four bilinear corners are non-negative and sum to w)
template <typename WT>
__global__ void tc_wmax_kernel(const WT* __restrict__ rw, long long n, unsigned int* __restrict__ wmax)
{
    unsigned int m = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        m = max(m, __float_as_uint(fabsf(tc_rec_w(rw[i]))));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m) atomicMax(wmax, m);
}

// first record of every 128-sample tile of every A-scan (records grouped by tile, n0 ascending from tile to
// tile)
__global__ void tc_tile_off_kernel(GeomParams P, int ntile, const long long* __restrict__ rec_off,
                                   const uint2* __restrict__ rkey, int* __restrict__ tile_off)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (long long)P.K * (ntile + 1)) return;
    const int k = (int)(i / (ntile + 1)), t = (int)(i - (long long)k * (ntile + 1));
    const long long base = rec_off[k];
    int lo = 0, hi = (int)(rec_off[k + 1] - base);
    const int target = t * kTsTile;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (tc_rec_n0(rkey[base + mid]) < target) lo = mid + 1;
        else hi = mid;
    }
    tile_off[i] = lo;
}

// First record of every tile, the per-pixel accumulators (N sums and the max |e| word after them, zeroed)
// and the bound of the fixed-point scale: K x the largest record weight w x (the largest table row sum
// of |T| + the largest |T|, for the tau = t0 tap), doubled for the rounding of the products;
// cudaErrorNotSupported keeps the CUDA-core adjoint.
cudaError_t build_tc_adjoint(mbir_geometry* g, cudaStream_t st)
{
    const GeomParams& P = g->P;
    if (!g->d_tc_key || g->n_records <= 0) return cudaErrorNotSupported;
    const int N = P.W * P.H;
    const int ntile = (P.M + kTsTile - 1) / kTsTile;
    int* d_tile = nullptr;
    unsigned long long* d_acc = nullptr;
    int* d_ctr = nullptr;
    cudaError_t e = cudaMalloc((void**)&d_tile, sizeof(int) * (size_t)P.K * (ntile + 1));
    if (e == cudaSuccess) e = cudaMalloc((void**)&d_acc, sizeof(unsigned long long) * ((size_t)N + 1));
    if (e == cudaSuccess) e = cudaMalloc((void**)&d_ctr, sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(d_acc, 0, sizeof(unsigned long long) * ((size_t)N + 1), st);
    if (e == cudaSuccess) {
        const long long items = (long long)P.K * (ntile + 1);
        tc_tile_off_kernel<<<(int)((items + 255) / 256), 256, 0, st>>>(P, ntile, g->d_rec_off, g->d_tc_key, d_tile);
        e = cudaGetLastError();
    }
    unsigned int wbits = 0;
    if (e == cudaSuccess) {
        unsigned int* d_wmax = reinterpret_cast<unsigned int*>(d_acc + N);
        if (P.precision == MBIR_PREC_BF16)
            tc_wmax_kernel<<<std::max(1, g->n_sm * 8), 256, 0, st>>>(reinterpret_cast<const uint32_t*>(g->d_tc_w),
                                                                     g->n_records, d_wmax);
        else
            tc_wmax_kernel<<<std::max(1, g->n_sm * 8), 256, 0, st>>>(reinterpret_cast<const uint2*>(g->d_tc_w),
                                                                     g->n_records, d_wmax);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(&wbits, d_wmax, sizeof(wbits), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(d_wmax, 0, sizeof(unsigned long long), st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    double tsum = 0.0, tmax = 0.0;
    const int nq = P.Q * P.Tw + 1;
    for (int gpl = 0; gpl < P.G; ++gpl)
        for (int ph = 0; ph <= P.Q; ++ph) {
            double rs = 0.0;
            for (int m = 0; m < P.Tw; ++m) {
                const double t = std::fabs((double)g->tab_host[(size_t)gpl * nq + m * P.Q + ph]);
                rs += t;
                tmax = std::max(tmax, t);
            }
            tsum = std::max(tsum, rs);
        }
    float wmax = 0.0f;
    std::memcpy(&wmax, &wbits, sizeof(wmax));
    const double bound = 2.0 * P.K * (double)wmax * (tsum + tmax);
    if (e == cudaSuccess && !(bound > 0.0 && bound < 1e30)) e = cudaErrorNotSupported;
    if (e != cudaSuccess) {
        void* ptrs[] = {d_tile, d_acc, d_ctr};
        for (void* p : ptrs) cudaFree(p);
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? cudaErrorNotSupported : e;
    }
    g->d_tc_tile = d_tile;
    g->w_tc_acc = d_acc;
    g->d_tc_counter = d_ctr;
    g->tc_bound = (float)bound;
    g->bytes += sizeof(int) * ((size_t)P.K * (ntile + 1) + 1) + sizeof(unsigned long long) * ((size_t)N + 1);
    return cudaSuccess;
}

// The tables above, freed when the tensor-core A^T is not used after all.
void free_tc_adjoint(mbir_geometry* g)
{
    void* ptrs[] = {g->d_tc_tile, g->w_tc_acc, g->d_tc_counter};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    g->d_tc_tile = nullptr;
    g->w_tc_acc = nullptr;
    g->d_tc_counter = nullptr;
}

// ---------------------------------------------------------------------------
// Streamed tensor-core A^T (tcs_adjoint_pool): layout, table operand, launch.
// ---------------------------------------------------------------------------
Tb4Layout tb4_layout(const GeomParams& P, int kwmax)
{
    Tb4Layout L{};
    const bool bf = P.precision == MBIR_PREC_BF16;
    L.parts = bf ? 1 : 2;
    L.R = P.Q + 1;
    L.kb = (P.G * L.R + 15) & ~15;
    L.ntap = (P.Tw + 15) & ~15;
    L.kwmax = std::min(std::min(kwmax, 256), L.kb);
    L.cstride = ((L.kwmax + 31) & ~31) + 4;            // 4 mod 32: the read-back rows hit distinct banks
    L.ewin = (kTsTile + L.ntap + 31) & ~31;
    L.bbytes = (size_t)L.parts * L.kb * L.ntap * 2;
    L.off_e = 256;                                     // after the header and the warps' maxima
    L.off_b = (L.off_e + (size_t)2 * L.ewin * 4 + 1023) & ~(size_t)1023;
    L.off_c = (L.off_b + L.bbytes + 1023) & ~(size_t)1023;
    L.smem = L.off_c + (size_t)kTsTile * L.cstride * 4;
    L.ok = L.R >= 2 && L.ntap <= 128 && L.kwmax >= 16 && L.kwmax % 16 == 0 && 128 + L.kwmax <= (int)kTsCols &&
           kTsTile + L.ntap <= 32 * tb_warps(bf) && L.smem <= 227 * 1024 && L.bbytes < (1u << 20) &&
           P.G * L.R <= 4096;
    return L;
}

// The view is read from device memory (written at set-up) with the residual as a parameter, as for the
// tensor-core A x (fwd_tcs_kernel).
template <bool BF16, int BV>
__global__ void __launch_bounds__(TbShape<BF16>::threads, 1)
    bwd_tcs_kernel(const TbView* __restrict__ base, const void* e, int* __restrict__ status)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    tc_header_init(smem, kTsCols);
    const uint32_t tmem = *reinterpret_cast<volatile uint32_t*>(smem + 8);
    uint32_t mphase = 0, bphase = 0;
    TbView V = *base;
    asm volatile("" : "+l"(e));
    V.e = e;
    tcs_adjoint_pool<BF16, BV>(V, smem, tmem, mphase, bphase, status);
    tc_header_release(smem, tmem, kTsCols);
}

// Table operand of the streamed A^T (rows plane * (Q + 1) + phase, columns taps; FP32 form: the table times
// 2^texp split into two FP16 parts, BF16 form: the stored BF16 table), for a geometry whose records, tile
// offsets and accumulators (build_tc_adjoint) and per-tile column ranges (build_tc_forward_stream) are
// present; cudaErrorNotSupported keeps the other adjoints.
cudaError_t build_tc_adjoint_stream(mbir_geometry* g, cudaStream_t st)
{
    (void)st;
    const GeomParams& P = g->P;
    if (!g->d_tc_tile || !g->w_tc_acc || !g->d_tf4_crange || !g->d_tc_counter)
        return cudaErrorNotSupported;
    Tb4Layout L{};
    for (int kw : {256, 224, 192, 160, 128, 96, 64}) {
        L = tb4_layout(P, kw);
        if (L.ok) break;
    }
    if (!L.ok || g->tf4_wmax > L.kwmax) return cudaErrorNotSupported;
    {
        const Tb4Layout Lt = tb4_layout(P, std::max(g->tf4_wmax, 16));   // no wider than the widest tile
        if (Lt.ok) L = Lt;
    }
    const int nq = P.Q * P.Tw + 1;
    const size_t part = (size_t)L.kb * L.ntap;
    std::vector<uint16_t> img((size_t)L.parts * part, 0);
    if (P.precision == MBIR_PREC_BF16) {
        L.texp = 0;
        for (int gpl = 0; gpl < P.G; ++gpl)
            for (int ph = 0; ph < L.R; ++ph)
                for (int m = 0; m < P.Tw; ++m) {
                    const __nv_bfloat16 v = __float2bfloat16_rn((float)g->tab_host[(size_t)gpl * nq + m * P.Q + ph]);
                    img[kmajor_offset(gpl * L.R + ph, m, L.ntap) / 2] = *reinterpret_cast<const uint16_t*>(&v);
                }
    } else {
        float tmax = 0.0f;
        for (size_t i = 0; i < (size_t)P.G * nq; ++i) tmax = std::max(tmax, std::fabs((float)g->tab_host[i]));
        int ex = 0;
        std::frexp(tmax, &ex);
        L.texp = tmax > 0.0f ? std::min(15 - ex, 126) : 0;
        for (int gpl = 0; gpl < P.G; ++gpl)
            for (int ph = 0; ph < L.R; ++ph)
                for (int m = 0; m < P.Tw; ++m) {
                    const float t = std::ldexp((float)g->tab_host[(size_t)gpl * nq + m * P.Q + ph], L.texp);
                    const __half p1 = __float2half_rn(t);
                    const __half p2 = __float2half_rn(t - __half2float(p1));
                    const size_t o = kmajor_offset(gpl * L.R + ph, m, L.ntap) / 2;
                    img[o] = *reinterpret_cast<const uint16_t*>(&p1);
                    img[part + o] = *reinterpret_cast<const uint16_t*>(&p2);
                }
    }
    uint4* d_b = nullptr;
    TbView* d_view = nullptr;
    cudaError_t e = cudaMalloc((void**)&d_b, L.bbytes);
    if (e == cudaSuccess) e = cudaMemcpy(d_b, img.data(), L.bbytes, cudaMemcpyHostToDevice);
    // the kernel's view without the residual
    if (e == cudaSuccess) {
        const int N = P.W * P.H;
        const void* tab = P.precision == MBIR_PREC_BF16 ? (const void*)g->d_tab_bf16 : (const void*)g->d_tab;
        const TbView V{P, L, d_b, tab, nullptr, g->d_rec_off, g->d_tc_tile, g->d_tf4_crange, g->d_tc_key,
                       g->d_tc_w, g->w_tc_acc, reinterpret_cast<const unsigned int*>(g->w_tc_acc + N),
                       g->tc_bound, g->d_tc_counter};
        e = cudaMalloc((void**)&d_view, sizeof(TbView));
        if (e == cudaSuccess) e = cudaMemcpy(d_view, &V, sizeof(TbView), cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
        cudaFree(d_b);
        cudaFree(d_view);
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? cudaErrorNotSupported : e;
    }
    g->tb4 = L;
    g->d_tb4_bop = d_b;
    g->d_tb_view = d_view;
    g->bytes += L.bbytes;
    return cudaSuccess;
}

static cudaError_t launch_backproject_tcs_impl(const mbir_geometry* g, const float* e_pad, const __nv_bfloat16* e_bf,
                                               float* b, float* e_upd, __nv_bfloat16* ebf_upd, const float* q,
                                               const double* sc, int alpha_slot, cudaStream_t st)
{
    const GeomParams& P = g->P;
    const Tb4Layout& L = g->tb4;
    const bool bf = P.precision == MBIR_PREC_BF16;
    auto kern = bf ? (g->tc_bvar ? bwd_tcs_kernel<true, 1> : bwd_tcs_kernel<true, 0>)
                   : (g->tc_bvar ? bwd_tcs_kernel<false, 1> : bwd_tcs_kernel<false, 0>);
    cudaError_t ce = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(g->d_tc_counter, 0, sizeof(int), st);
    if (ce != cudaSuccess) return ce;
    const int ntile = (P.M + kTsTile - 1) / kTsTile;
    const int grid = std::max(1, std::min(g->n_sm, P.K * ntile));
    const void* e = bf ? (const void*)e_bf : (const void*)e_pad;
    const int N = P.W * P.H;
    unsigned int* emax = reinterpret_cast<unsigned int*>(g->w_tc_acc + N);
    ce = cudaMemsetAsync(g->w_tc_acc, 0, sizeof(unsigned long long) * ((size_t)N + 1), st);
    if (ce != cudaSuccess) return ce;
    const long long ne = (long long)P.K * P.Mp;
    const int eg = (int)std::max(1LL, std::min((ne + 255) / 256, (long long)g->n_sm * 8));
    if (e_upd) tc_emax_update_kernel<<<eg, 256, 0, st>>>(e_upd, bf ? ebf_upd : nullptr, q, sc, alpha_slot, ne, emax);
    else if (bf) tc_emax_kernel<__nv_bfloat16><<<eg, 256, 0, st>>>(e_bf, ne, emax);
    else tc_emax_kernel<float><<<eg, 256, 0, st>>>(e_pad, ne, emax);
    ce = cudaGetLastError();
    if (ce != cudaSuccess) return ce;
    kern<<<grid, 32 * tb_warps(bf), L.smem, st>>>(g->d_tb_view, e, g->d_status);
    ce = cudaGetLastError();
    if (ce != cudaSuccess) return ce;
    tc_finish_kernel<<<std::max(1, std::min((N + 255) / 256, g->n_sm * 8)), 256, 0, st>>>(N, g->w_tc_acc, emax,
                                                                                           g->tc_bound, b);
    return cudaGetLastError();
}

cudaError_t launch_backproject_tcs(const mbir_geometry* g, const float* e_pad, const __nv_bfloat16* e_bf, float* b,
                                   cudaStream_t st)
{
    return launch_backproject_tcs_impl(g, e_pad, e_bf, b, nullptr, nullptr, nullptr, nullptr, 0, st);
}

// A^T e after the residual's pending update e -= alpha q (e: K x Mp FP32, with its BF16 copy ebf in the BF16
// form), the update done in the pass that finds max |e|.
cudaError_t launch_backproject_tcs_update(const mbir_geometry* g, float* e, __nv_bfloat16* ebf, const float* q,
                                          const double* sc, int alpha_slot, float* b, cudaStream_t st)
{
    return launch_backproject_tcs_impl(g, e, ebf, b, e, ebf, q, sc, alpha_slot, st);
}

}  // namespace mbir
