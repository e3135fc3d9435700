// Tables of the tensor-core A^T (tcs_adjoint_pool, tc_stream.cuh): the first
// record of every tile, each record's slot for its contribution, the
// per-pixel reduction of the contributions, the table operand and the launch.
// Slots are grouped by transmitter position (the n_rx A-scans of one position
// are consecutive) and pixel-major inside a group, A-scans in order: the
// contributions of one group, written close together in time, fill whole
// sectors before they leave L2, and a pixel's contributions are summed group
// after group in A-scan order, so the result is reproducible.
#include <algorithm>
#include <cmath>
#include <vector>

#include "tc_stream.cuh"

namespace mbir {

// b = each pixel's contributions summed (tcs_reduce_pixels), one pixel per lane.
__global__ void bwd_tc_reduce_kernel(int N, int n_tx, int n_rx, const long long* __restrict__ rec_off,
                                     const int* __restrict__ goff, const float* __restrict__ contrib,
                                     float* __restrict__ b)
{
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w * 32 < N; w += nw)
        tcs_reduce_pixels(w * 32, N, n_tx, n_rx, rec_off, goff, contrib, b);
}

// cnt[v] += 1 for the records [a, z) of one A-scan (a pixel has at most one record per A-scan)
__global__ void tc_gcount_kernel(long long a, long long z, const int2* __restrict__ rkey, int* __restrict__ cnt)
{
    const long long r = a + blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (r < z) cnt[rkey[r].x] += 1;
}

// off[v] = cnt[0] + ... + cnt[v - 1] for v = 0 .. N (one block): chunks of consecutive pixels per thread, the
// chunk sums scanned across the block
__global__ void tc_gscan_kernel(const int* __restrict__ cnt, int N, int* __restrict__ off)
{
    __shared__ int ws[32];
    const int nt = blockDim.x, tid = threadIdx.x;
    const int chunk = (N + nt - 1) / nt, v0 = min(tid * chunk, N), v1 = min(v0 + chunk, N);
    int sum = 0;
    for (int v = v0; v < v1; ++v) sum += cnt[v];
    // exclusive scan of the chunk sums: warp inclusive scan, then the warps' totals
    int inc = sum;
    for (int d = 1; d < 32; d <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, inc, d);
        if ((tid & 31) >= d) inc += t;
    }
    if ((tid & 31) == 31) ws[tid >> 5] = inc;
    __syncthreads();
    if (tid < 32) {
        int x = tid < (nt >> 5) ? ws[tid] : 0;
        for (int d = 1; d < 32; d <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, x, d);
            if (tid >= d) x += t;
        }
        ws[tid] = x;
    }
    __syncthreads();
    int run = inc - sum + ((tid >> 5) > 0 ? ws[(tid >> 5) - 1] : 0);
    for (int v = v0; v < v1; ++v) {
        off[v] = run;
        run += cnt[v];
    }
    if (tid == nt - 1) off[N] = run;
}

// slot of each record of one A-scan of group g: the group's pixel-major offset of its pixel plus the
// pixel's records already placed in the group (A-scans in order)
__global__ void tc_gdest_kernel(long long a, long long z, long long gbase, const int2* __restrict__ rkey,
                                const int* __restrict__ off, int* __restrict__ cursor, uint32_t* __restrict__ dest)
{
    const long long r = a + blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (r < z) {
        const int v = rkey[r].x;
        const int c = cursor[v];
        dest[r] = (uint32_t)(gbase + off[v] + c);
        cursor[v] = c + 1;
    }
}

// first record of every 128-sample tile of every A-scan (records sorted by n0)
__global__ void tc_tile_off_kernel(GeomParams P, int ntile, const long long* __restrict__ rec_off,
                                   const int2* __restrict__ rkey, int* __restrict__ tile_off)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (long long)P.K * (ntile + 1)) return;
    const int k = (int)(i / (ntile + 1)), t = (int)(i - (long long)k * (ntile + 1));
    const long long base = rec_off[k];
    int lo = 0, hi = (int)(rec_off[k + 1] - base);
    const int target = t * kTsTile;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if ((rkey[base + mid].y >> kRecShift) < target) lo = mid + 1;
        else hi = mid;
    }
    tile_off[i] = lo;
}

// First record of every tile, each record's slot (per transmitter position, pixel-major, A-scans in order)
// and the contribution buffer of the tensor-core A^T; cudaErrorNotSupported keeps the CUDA-core adjoint.
cudaError_t build_tc_adjoint(mbir_geometry* g, cudaStream_t st)
{
    const GeomParams& P = g->P;
    if (!g->d_rec_key || g->n_records <= 0 || g->n_records >= (1LL << 32)) return cudaErrorNotSupported;
    const int N = P.W * P.H;
    const int ntile = (P.M + kTsTile - 1) / kTsTile;
    int* d_cnt = nullptr;
    int* d_tile = nullptr;
    int* d_goff = nullptr;
    uint32_t* d_dest = nullptr;
    float* d_contrib = nullptr;
    int* d_ctr = nullptr;
    const size_t gstride = (size_t)N + 1;
    cudaError_t e = cudaMalloc((void**)&d_cnt, sizeof(int) * (size_t)N);
    if (e == cudaSuccess) e = cudaMalloc((void**)&d_tile, sizeof(int) * (size_t)P.K * (ntile + 1));
    if (e == cudaSuccess) e = cudaMalloc((void**)&d_goff, sizeof(int) * gstride * P.n_tx);
    if (e == cudaSuccess) e = cudaMalloc((void**)&d_dest, sizeof(uint32_t) * (size_t)g->n_records);
    if (e == cudaSuccess) e = cudaMalloc((void**)&d_contrib, sizeof(float) * (size_t)g->n_records);
    if (e == cudaSuccess) e = cudaMalloc((void**)&d_ctr, sizeof(int));
    if (e == cudaSuccess) {
        const long long items = (long long)P.K * (ntile + 1);
        tc_tile_off_kernel<<<(int)((items + 255) / 256), 256, 0, st>>>(P, ntile, g->d_rec_off, g->d_rec_key, d_tile);
        e = cudaGetLastError();
    }
    std::vector<long long> roff((size_t)P.K + 1);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(roff.data(), g->d_rec_off, sizeof(long long) * (P.K + 1), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    // per transmitter position: pixel counts, their offsets, then the slots with a cursor per pixel
    for (int gi = 0; gi < P.n_tx && e == cudaSuccess; ++gi) {
        int* off = d_goff + gstride * gi;
        const int k0 = gi * P.n_rx, k1 = k0 + P.n_rx;
        e = cudaMemsetAsync(d_cnt, 0, sizeof(int) * (size_t)N, st);
        for (int k = k0; k < k1 && e == cudaSuccess; ++k)
            if (roff[k + 1] > roff[k]) {
                tc_gcount_kernel<<<(int)((roff[k + 1] - roff[k] + 255) / 256), 256, 0, st>>>(roff[k], roff[k + 1],
                                                                                            g->d_rec_key, d_cnt);
                e = cudaGetLastError();
            }
        if (e == cudaSuccess) {
            tc_gscan_kernel<<<1, 1024, 0, st>>>(d_cnt, N, off);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaMemsetAsync(d_cnt, 0, sizeof(int) * (size_t)N, st);
        for (int k = k0; k < k1 && e == cudaSuccess; ++k)
            if (roff[k + 1] > roff[k]) {
                tc_gdest_kernel<<<(int)((roff[k + 1] - roff[k] + 255) / 256), 256, 0, st>>>(
                    roff[k], roff[k + 1], roff[k0], g->d_rec_key, off, d_cnt, d_dest);
                e = cudaGetLastError();
            }
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(d_cnt);
    if (e != cudaSuccess) {
        void* ptrs[] = {d_tile, d_goff, d_dest, d_contrib, d_ctr};
        for (void* p : ptrs) cudaFree(p);
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? cudaErrorNotSupported : e;
    }
    g->d_tc_tile = d_tile;
    g->d_tc_goff = d_goff;
    g->d_tc_dest = d_dest;
    g->w_tc_contrib = d_contrib;
    g->d_tc_counter = d_ctr;
    g->bytes += sizeof(int) * ((size_t)P.K * (ntile + 1) + 1 + gstride * P.n_tx) +
                (sizeof(uint32_t) + sizeof(float)) * (size_t)g->n_records;
    return cudaSuccess;
}

// The tables above, freed when the tensor-core A^T is not used after all.
void free_tc_adjoint(mbir_geometry* g)
{
    void* ptrs[] = {g->d_tc_tile, g->d_tc_goff, g->d_tc_dest, g->w_tc_contrib, g->d_tc_counter};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    g->d_tc_tile = nullptr;
    g->d_tc_goff = nullptr;
    g->d_tc_dest = nullptr;
    g->w_tc_contrib = nullptr;
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
    L.off_e = 128;
    L.off_b = (L.off_e + (size_t)2 * L.ewin * 4 + 1023) & ~(size_t)1023;
    L.off_c = (L.off_b + L.bbytes + 1023) & ~(size_t)1023;
    L.smem = L.off_c + (size_t)kTsTile * L.cstride * 4;
    L.ok = L.R >= 2 && L.ntap <= 128 && L.kwmax >= 16 && L.kwmax % 16 == 0 && 128 + L.kwmax <= (int)kTsCols &&
           kTsTile + L.ntap <= kTsThreads && L.smem <= 227 * 1024 && L.bbytes < (1u << 20) &&
           P.G * L.R <= 4096;
    return L;
}

template <bool BF16>
__global__ void __launch_bounds__(kTsThreads, 1) bwd_tcs_kernel(TbView V, int* __restrict__ status)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    tc_header_init(smem, kTsCols);
    const uint32_t tmem = *reinterpret_cast<volatile uint32_t*>(smem + 8);
    uint32_t mphase = 0, bphase = 0;
    tcs_adjoint_pool<BF16>(V, smem, tmem, mphase, bphase, status);
    tc_header_release(smem, tmem, kTsCols);
}

// Table operand of the streamed A^T (rows plane * (Q + 1) + phase, columns taps; FP32 form: the table times
// 2^texp split into two FP16 parts, BF16 form: the stored BF16 table), for a geometry whose records, tile
// offsets and contribution slots (build_tc_adjoint) and per-tile column ranges (build_tc_forward_stream) are
// present; cudaErrorNotSupported keeps the other adjoints.
cudaError_t build_tc_adjoint_stream(mbir_geometry* g, cudaStream_t st)
{
    (void)st;
    const GeomParams& P = g->P;
    if (!g->d_tc_tile || !g->d_tc_dest || !g->w_tc_contrib || !g->d_tf4_crange || !g->d_tc_counter)
        return cudaErrorNotSupported;
    Tb4Layout L{};
    for (int kw : {256, 224, 192, 160, 128, 96, 64}) {
        L = tb4_layout(P, kw);
        if (L.ok) break;
    }
    if (!L.ok || g->tf4_wmax > L.kwmax) return cudaErrorNotSupported;
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
    cudaError_t e = cudaMalloc((void**)&d_b, L.bbytes);
    if (e == cudaSuccess) e = cudaMemcpy(d_b, img.data(), L.bbytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(d_b);
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? cudaErrorNotSupported : e;
    }
    g->tb4 = L;
    g->d_tb4_bop = d_b;
    g->bytes += L.bbytes;
    return cudaSuccess;
}

cudaError_t launch_backproject_tcs(const mbir_geometry* g, const float* e_pad, const __nv_bfloat16* e_bf, float* b,
                                   cudaStream_t st)
{
    const GeomParams& P = g->P;
    const Tb4Layout& L = g->tb4;
    const bool bf = P.precision == MBIR_PREC_BF16;
    auto kern = bf ? bwd_tcs_kernel<true> : bwd_tcs_kernel<false>;
    cudaError_t ce = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(g->d_tc_counter, 0, sizeof(int), st);
    if (ce != cudaSuccess) return ce;
    const int ntile = (P.M + kTsTile - 1) / kTsTile;
    const int grid = std::max(1, std::min(g->n_sm, P.K * ntile));
    const void* tab = bf ? (const void*)g->d_tab_bf16 : (const void*)g->d_tab;
    const void* e = bf ? (const void*)e_bf : (const void*)e_pad;
    TbView V{P, L, g->d_tb4_bop, tab, e, g->d_rec_off, g->d_tc_tile, g->d_tf4_crange, g->d_rec_key, g->d_rec_w,
             g->d_tc_dest, g->w_tc_contrib, g->d_tc_counter};
    kern<<<grid, kTsThreads, L.smem, st>>>(V, g->d_status);
    ce = cudaGetLastError();
    if (ce != cudaSuccess) return ce;
    const int N = P.W * P.H;
    bwd_tc_reduce_kernel<<<std::max(1, std::min((N + 255) / 256, g->n_sm * 16)), 256, 0, st>>>(
        N, P.n_tx, P.n_rx, g->d_rec_off, g->d_tc_goff, g->w_tc_contrib, b);
    return cudaGetLastError();
}

}  // namespace mbir
