// A^T r of the BF16 storage form on the tensor cores.
//
// Every tap of a pair shares one table phase (eq. 13 with the bilinear pulse
// table), so the pair's taps against a residual row are, for each of its four
// table rows, one value of that row's correlation with the residual:
//     C[row][n] = sum_m T[row][m] e[n + 1 + m].
// For one A-scan and a tile of 128 samples n, all G (Q + 1) table rows at once
// are one matrix product  C^T (128 x rows) = H (128 x taps) T^T (taps x rows),
// where H[n][m] = e[n_tile + n + 1 + m] is a Hankel matrix of the residual.
// The product runs on the 5th-generation tensor cores (tcgen05.mma, BF16
// operands, FP32 accumulators in tensor memory): the operands are exactly the
// stored BF16 residual and table, whose products FP32 represents exactly.
// The tile's pairs are the A-scan's sorted records whose first tap falls in
// it; each combines four correlation values with its bilinear weights (less
// the tau = t0 tap, outside the open window of eq. 10) into one contribution,
// stored at the record's place in pixel-major order.  A second kernel sums
// every pixel's contributions in A-scan order, so the result is reproducible.
#include <algorithm>
#include <cmath>
#include <vector>

#include "tc_apply.cuh"
#include "tc_stream.cuh"

namespace mbir {

TcLayout tc_layout(const GeomParams& P)
{
    TcLayout L{};
    L.kpad = (P.Tw + 15) & ~15;
    L.ncols = P.G * (P.Q + 1);
    L.npad = (L.ncols + 15) & ~15;
    L.nchunk0 = std::min(L.npad, ((L.npad / 2) + 15) & ~15);
    L.nchunk1 = L.npad - L.nchunk0;
    L.cstride = L.npad + 1;
    L.off_h = 1024;
    L.off_b = L.off_h + (size_t)kTcTile * L.kpad * 2;
    L.off_e = (L.off_b + (size_t)L.npad * L.kpad * 2 + 127) & ~(size_t)127;
    L.off_c = (L.off_e + (size_t)(kTcTile + L.kpad + 16) * 2 + 127) & ~(size_t)127;
    L.smem = L.off_c + (size_t)kTcTile * L.cstride * 4;
    L.ok = L.npad <= 512 && L.nchunk0 <= 256 && L.nchunk1 <= 256 && L.smem <= 227 * 1024 && P.K <= 65535 &&
           P.Q + 1 <= 4096 && kTcTile + L.kpad <= kTcThreads;
    return L;
}

Tc3Layout tc3_layout(const GeomParams& P)
{
    Tc3Layout L{};
    const int R = P.Q + 1;
    L.kpad = (P.Tw + 15) & ~15;
    L.phsplit = R / 2;
    L.pstride = std::max(L.phsplit + 1, R - L.phsplit);
    L.nrows[0] = L.nrows[1] = (L.pstride * P.G + 15) & ~15;
    L.nmax = std::max(L.nrows[0], L.nrows[1]);
    L.cstride = L.nmax + 1;
    L.bhalf[0] = (size_t)2 * L.nrows[0] * L.kpad * 2;
    L.bhalf[1] = (size_t)2 * L.nrows[1] * L.kpad * 2;
    L.off_h = 1024;
    L.off_b = L.off_h + (size_t)2 * kTcTile * L.kpad * 2;
    L.off_e = (L.off_b + L.bhalf[0] + L.bhalf[1] + 127) & ~(size_t)127;
    L.off_c = (L.off_e + (size_t)(kTcTile + L.kpad + 16) * 4 + 127) & ~(size_t)127;
    L.smem = L.off_c + (size_t)kTcTile * L.cstride * 4;
    L.ok = R >= 2 && L.nmax <= 256 && L.smem <= 227 * 1024 && P.K <= 65535 && kTcTile + L.kpad <= kTcThreads;
    return L;
}

__global__ void __launch_bounds__(kTcThreads, 1) bwd_tc32_kernel(Tc3View V, int* __restrict__ status)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    tc_header_init(smem, 256);
    const uint32_t tmem = *reinterpret_cast<volatile uint32_t*>(smem + 8);
    uint32_t phase = 0, bphase = 0;
    tc_adjoint32_pool(V, smem, tmem, phase, bphase, status);
    tc_header_release(smem, tmem, 256);
}

__global__ void __launch_bounds__(kTcThreads, 1) bwd_tc_kernel(TcAdjView V, int* __restrict__ status)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    tc_header_init(smem, kTcCols);
    const uint32_t tmem = *reinterpret_cast<volatile uint32_t*>(smem + 8);
    uint32_t phase = 0;
    tc_adjoint_pool(V, smem, tmem, phase, status);
    tc_header_release(smem, tmem, kTcCols);
}

// b_v = sum of pixel v's contributions in A-scan order: one warp per pixel,
// lanes sum strided subsets (Neumaier), combined by a fixed shuffle tree.
__global__ void bwd_tc_reduce_kernel(int N, const long long* __restrict__ pix_off, const float* __restrict__ contrib,
                                     float* __restrict__ b)
{
    const int lane = threadIdx.x & 31;
    const int w0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    for (int v = w0; v < N; v += nw) {
        const long long a = __ldg(pix_off + v), z = __ldg(pix_off + v + 1);
        float s = 0.0f, c = 0.0f;
        for (long long j = a + lane; j < z; j += 32) neumaier_add(s, c, __ldg(contrib + j));
        s += c;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) b[v] = s;
    }
}

// per-pixel record counts (integer atomics: order-independent)
__global__ void tc_pix_count_kernel(long long nrec, const int2* __restrict__ rkey, int* __restrict__ cnt)
{
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < nrec; r += (long long)gridDim.x * blockDim.x)
        atomicAdd(cnt + rkey[r].x, 1);
}

// place of each record of A-scan k in pixel-major order (A-scans one after
// the other: a pixel has at most one record per A-scan, so no collisions)
__global__ void tc_dest_kernel(long long a, long long z, const int2* __restrict__ rkey,
                               const long long* __restrict__ pix_off, int* __restrict__ cursor,
                               uint32_t* __restrict__ dest)
{
    const long long r = a + blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (r < z) {
        const int v = rkey[r].x;
        const int c = cursor[v];
        dest[r] = (uint32_t)(pix_off[v] + c);
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
    const int target = t * kTcTile;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if ((rkey[base + mid].y >> kRecShift) < target) lo = mid + 1;
        else hi = mid;
    }
    tile_off[i] = lo;
}

// per (A-scan, tile) and row half: the lowest and highest attenuation plane
// that the tile's records reach (lo | hi << 16; lo > hi when the half has no
// record).  One warp per item.
__global__ void tc3_prange_kernel(GeomParams P, int ntile, int phsplit, const long long* __restrict__ rec_off,
                                  const int2* __restrict__ rkey, const int* __restrict__ tile_off,
                                  uint2* __restrict__ prange)
{
    const long long item = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (item >= (long long)P.K * ntile) return;
    const int k = (int)(item / ntile), t = (int)(item - (long long)k * ntile);
    const long long base = rec_off[k];
    const int a = tile_off[(size_t)k * (ntile + 1) + t], z = tile_off[(size_t)k * (ntile + 1) + t + 1];
    const int R = P.Q + 1;
    int lo[2] = {0xffff, 0xffff}, hi[2] = {0, 0};
    for (int r = a + lane; r < z; r += 32) {
        const int trow = (rkey[base + r].y >> 1) & 0xfff;
        const int gi = trow / R, ph = trow - gi * R, h = ph >= phsplit ? 1 : 0;
        lo[h] = min(lo[h], gi);
        hi[h] = max(hi[h], min(gi + 1, P.G - 1));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            lo[h] = min(lo[h], __shfl_xor_sync(0xffffffffu, lo[h], o));
            hi[h] = max(hi[h], __shfl_xor_sync(0xffffffffu, hi[h], o));
        }
    if (lane == 0) prange[item] = make_uint2((uint32_t)lo[0] | (uint32_t)hi[0] << 16, (uint32_t)lo[1] | (uint32_t)hi[1] << 16);
}

// Builds the tensor-core adjoint's tables for a BF16 geometry with records.
// Returns cudaErrorNotSupported (the caller keeps the other adjoint) when the
// layout does not fit or memory is short.
cudaError_t build_tc_adjoint(mbir_geometry* g, cudaStream_t st)
{
    const GeomParams& P = g->P;
    if (!g->d_rec_key || g->n_records <= 0 || g->n_records >= (1LL << 32)) return cudaErrorNotSupported;
    const bool bf = P.precision == MBIR_PREC_BF16;
    const TcLayout L = tc_layout(P);
    Tc3Layout L3 = tc3_layout(P);
    if (bf ? !L.ok : !L3.ok) return cudaErrorNotSupported;
    const int N = P.W * P.H;
    const int ntile = (P.M + kTcTile - 1) / kTcTile;
    const int R = P.Q + 1, nq = P.Q * P.Tw + 1;
    std::vector<__nv_bfloat16> bimg;
    if (bf) {
        // table operand: row plane * (Q + 1) + phase (plane-major, so that the planes a tile's records reach
        // are one row range), column m = tap, BF16 as in the stored table
        bimg.assign((size_t)L.npad * L.kpad, __float2bfloat16_rn(0.0f));
        for (int gpl = 0; gpl < P.G; ++gpl)
            for (int ph = 0; ph < R; ++ph)
                for (int m = 0; m < P.Tw; ++m)
                    bimg[kmajor_offset(gpl * R + ph, m, L.kpad) / 2] =
                        __float2bfloat16_rn((float)g->tab_host[(size_t)gpl * nq + m * P.Q + ph]);
    } else {
        // FP32 form: per row half, the FP32 table (as the CUDA-core kernels read it) times 2^texp
        // (largest magnitude into [2^14, 2^15)), split into two FP16 parts t = t1 + t2; half h holds
        // phases [h ? phsplit : 0, h ? Q : phsplit] in plane-major rows plane * pstride + (phase - first)
        float tmax = 0.0f;
        for (size_t i = 0; i < (size_t)P.G * nq; ++i) tmax = std::max(tmax, std::fabs((float)g->tab_host[i]));
        int ex = 0;
        std::frexp(tmax, &ex);
        L3.texp = tmax > 0.0f ? std::min(15 - ex, 126) : 0;
        bimg.assign((L3.bhalf[0] + L3.bhalf[1]) / 2, __float2bfloat16_rn(0.0f));
        __half* himg = reinterpret_cast<__half*>(bimg.data());
        size_t base = 0;
        for (int h = 0; h < 2; ++h) {
            const int phb = h ? L3.phsplit : 0, phe = h ? R - 1 : L3.phsplit;
            const size_t part = (size_t)L3.nrows[h] * L3.kpad;
            for (int ph = phb; ph <= phe; ++ph)
                for (int gpl = 0; gpl < P.G; ++gpl)
                    for (int m = 0; m < P.Tw; ++m) {
                        const float t = std::ldexp((float)g->tab_host[(size_t)gpl * nq + m * P.Q + ph], L3.texp);
                        const __half p1 = __float2half_rn(t);
                        const __half p2 = __float2half_rn(t - __half2float(p1));
                        const size_t o = kmajor_offset(gpl * L3.pstride + (ph - phb), m, L3.kpad) / 2;
                        himg[base + o] = p1;
                        himg[base + part + o] = p2;
                    }
            base += 2 * part;
        }
    }
    int* d_cnt = nullptr;
    int* d_tile = nullptr;
    long long* d_poff = nullptr;
    uint32_t* d_dest = nullptr;
    float* d_contrib = nullptr;
    uint4* d_b = nullptr;
    uint2* d_prange = nullptr;
    cudaError_t e = cudaMalloc((void**)&d_cnt, sizeof(int) * (size_t)N);
    if (e == cudaSuccess) e = cudaMalloc((void**)&d_prange, sizeof(uint2) * (size_t)P.K * ntile);
    if (e == cudaSuccess) e = cudaMalloc((void**)&d_tile, sizeof(int) * (size_t)P.K * (ntile + 1));
    if (e == cudaSuccess) e = cudaMalloc((void**)&d_poff, sizeof(long long) * ((size_t)N + 1));
    if (e == cudaSuccess) e = cudaMalloc((void**)&d_dest, sizeof(uint32_t) * (size_t)g->n_records);
    if (e == cudaSuccess) e = cudaMalloc((void**)&d_contrib, sizeof(float) * (size_t)g->n_records);
    if (e == cudaSuccess) e = cudaMalloc((void**)&d_b, bimg.size() * 2);
    if (e == cudaSuccess) e = cudaMemcpy(d_b, bimg.data(), bimg.size() * 2, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_cnt, 0, sizeof(int) * (size_t)N, st);
    if (e == cudaSuccess) {
        const long long nrec = g->n_records;
        tc_pix_count_kernel<<<(int)std::min<long long>((nrec + 255) / 256, 152LL * 64), 256, 0, st>>>(nrec, g->d_rec_key,
                                                                                                      d_cnt);
        const long long items = (long long)P.K * (ntile + 1);
        tc_tile_off_kernel<<<(int)((items + 255) / 256), 256, 0, st>>>(P, ntile, g->d_rec_off, g->d_rec_key, d_tile);
        {
            // plane ranges per tile: per row half (FP32 form) or of the whole tile (BF16 form: no phase
            // reaches the split R, every record counts as half 0)
            const long long warps = (long long)P.K * ntile;
            tc3_prange_kernel<<<(int)((warps * 32 + 255) / 256), 256, 0, st>>>(P, ntile, bf ? R : L3.phsplit,
                                                                              g->d_rec_off, g->d_rec_key, d_tile,
                                                                              d_prange);
        }
        e = cudaGetLastError();
    }
    std::vector<int> cnt(N);
    std::vector<long long> poff((size_t)N + 1, 0), roff((size_t)P.K + 1);
    if (e == cudaSuccess) e = cudaMemcpyAsync(cnt.data(), d_cnt, sizeof(int) * (size_t)N, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(roff.data(), g->d_rec_off, sizeof(long long) * (P.K + 1), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) {
        for (int v = 0; v < N; ++v) poff[v + 1] = poff[v] + cnt[v];
        e = cudaMemcpy(d_poff, poff.data(), sizeof(long long) * ((size_t)N + 1), cudaMemcpyHostToDevice);
    }
    // destinations: A-scans one after the other, a cursor per pixel
    if (e == cudaSuccess) e = cudaMemsetAsync(d_cnt, 0, sizeof(int) * (size_t)N, st);
    for (int k = 0; k < P.K && e == cudaSuccess; ++k) {
        const long long a = roff[k], z = roff[k + 1];
        if (z > a) {
            tc_dest_kernel<<<(int)((z - a + 255) / 256), 256, 0, st>>>(a, z, g->d_rec_key, d_poff, d_cnt, d_dest);
            e = cudaGetLastError();
        }
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(d_cnt);
    if (e != cudaSuccess) {
        cudaFree(d_tile);
        cudaFree(d_poff);
        cudaFree(d_dest);
        cudaFree(d_contrib);
        cudaFree(d_b);
        cudaFree(d_prange);
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? cudaErrorNotSupported : e;
    }
    if (bf) {
        g->tc = L;
        g->d_tc_bop = d_b;
    } else {
        g->tc3 = L3;
        g->d_tc3_bop = d_b;
    }
    g->d_tc3_prange = d_prange;
    g->d_tc_tile = d_tile;
    g->d_tc_pixoff = d_poff;
    g->d_tc_dest = d_dest;
    g->w_tc_contrib = d_contrib;
    g->bytes += bimg.size() * 2 + sizeof(int) * (size_t)P.K * (ntile + 1) + sizeof(long long) * ((size_t)N + 1) +
                sizeof(uint2) * (size_t)P.K * ntile +
                (sizeof(uint32_t) + sizeof(float)) * (size_t)g->n_records;
    return cudaMalloc((void**)&g->d_tc_counter, sizeof(int));
}

cudaError_t launch_backproject_tc(const mbir_geometry* g, const __nv_bfloat16* e_bf, float* b, cudaStream_t st)
{
    const GeomParams& P = g->P;
    const TcLayout& L = g->tc;
    cudaError_t ce = cudaFuncSetAttribute(bwd_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(g->d_tc_counter, 0, sizeof(int), st);
    if (ce != cudaSuccess) return ce;
    const int ntile = (P.M + kTcTile - 1) / kTcTile;
    const int grid = std::max(1, std::min(g->n_sm, P.K * ntile));
    TcAdjView V{P, L, g->d_tc_bop, g->d_tab_bf16, e_bf, g->d_rec_off, g->d_rec_key, g->d_rec_w, g->d_tc_tile,
                 g->d_tc3_prange, g->d_tc_dest, g->w_tc_contrib, g->d_tc_counter};
    bwd_tc_kernel<<<grid, kTcThreads, L.smem, st>>>(V, g->d_status);
    ce = cudaGetLastError();
    if (ce != cudaSuccess) return ce;
    const int N = P.W * P.H;
    bwd_tc_reduce_kernel<<<std::max(1, std::min((N + 7) / 8, 152 * 16)), 256, 0, st>>>(N, g->d_tc_pixoff,
                                                                                     g->w_tc_contrib, b);
    return cudaGetLastError();
}

cudaError_t launch_backproject_tc32(const mbir_geometry* g, const float* e_pad, float* b, cudaStream_t st)
{
    const GeomParams& P = g->P;
    const Tc3Layout& L = g->tc3;
    cudaError_t ce = cudaFuncSetAttribute(bwd_tc32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(g->d_tc_counter, 0, sizeof(int), st);
    if (ce != cudaSuccess) return ce;
    const int ntile = (P.M + kTcTile - 1) / kTcTile;
    const int grid = std::max(1, std::min(g->n_sm, P.K * ntile));
    Tc3View V{P, L, g->d_tc3_bop, g->d_tab, e_pad, g->d_rec_off, g->d_rec_key, g->d_rec_w, g->d_tc_tile, g->d_tc3_prange,
              g->d_tc_dest, g->w_tc_contrib, g->d_tc_counter};
    bwd_tc32_kernel<<<grid, kTcThreads, L.smem, st>>>(V, g->d_status);
    ce = cudaGetLastError();
    if (ce != cudaSuccess) return ce;
    const int N = P.W * P.H;
    bwd_tc_reduce_kernel<<<std::max(1, std::min((N + 7) / 8, 152 * 16)), 256, 0, st>>>(N, g->d_tc_pixoff,
                                                                                     g->w_tc_contrib, b);
    return cudaGetLastError();
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
    bwd_tc_reduce_kernel<<<std::max(1, std::min((N + 7) / 8, 152 * 16)), 256, 0, st>>>(N, g->d_tc_pixoff,
                                                                                     g->w_tc_contrib, b);
    return cudaGetLastError();
}

}  // namespace mbir
