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
#include <vector>

#include "apply_common.cuh"
#include "tc_common.cuh"

namespace mbir {

constexpr int kTcTile = 128;         // samples per MMA tile (M)
constexpr int kTcThreads = 512;      // 16 warps: four per tensor-memory lane quarter
constexpr int kTcUnroll = 4;         // records in flight per thread
constexpr uint32_t kTcCols = 512;    // tensor-memory columns allocated

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

// A batch of records held in registers (kTcUnroll per thread).
struct TcBatch {
    int2 key[kTcUnroll];
    float4 w[kTcUnroll];
    uint32_t dst[kTcUnroll];
};

__device__ __forceinline__ void tc_load_batch(TcBatch& b, const int2* __restrict__ rkey, const float4* __restrict__ rw,
                                              const uint32_t* __restrict__ dest, long long base, int rb, int r1,
                                              int tid)
{
#pragma unroll
    for (int u = 0; u < kTcUnroll; ++u) {
        const int r = rb + u * kTcThreads + tid;
        if (r < r1) {
            b.key[u] = __ldg(rkey + base + r);
            b.w[u] = __ldg(rw + base + r);
            b.dst[u] = __ldg(dest + base + r);
        }
    }
}

// Contributions of a batch: four correlation values per record, less the
// tau = t0 tap of the upper phase row for flagged records.
__device__ __forceinline__ void tc_run_batch(const TcBatch& b, const GeomParams& P, const TcLayout& T,
                                             const float* sC, const __nv_bfloat16* sE,
                                             const __nv_bfloat162* __restrict__ tab, int ts, int rb, int r1, int tid,
                                             float* __restrict__ contrib)
{
    const int R = P.Q + 1, S = table_stride(P.Tw4);
#pragma unroll
    for (int u = 0; u < kTcUnroll; ++u) {
        const int r = rb + u * kTcThreads + tid;
        if (r >= r1) continue;
        const int n0 = b.key[u].y >> kRecShift, trow = (b.key[u].y >> 1) & 0xfff;
        const int gi = trow / R, ph = trow - gi * R;
        const int g1 = min(gi + 1, P.G - 1);
        const float* cr = sC + (n0 - ts) * T.cstride;
        float v = b.w[u].x * cr[ph * P.G + gi];
        v = fmaf(b.w[u].y, cr[ph * P.G + g1], v);
        v = fmaf(b.w[u].z, cr[(ph + 1) * P.G + gi], v);
        v = fmaf(b.w[u].w, cr[(ph + 1) * P.G + g1], v);
        if (b.key[u].y & 1) {
            const float2 tl = __bfloat1622float2(__ldg(tab + ((size_t)gi * R + ph + 1) * S + P.Tw - 1));
            const float ev = __bfloat162float(sE[n0 - ts + P.Tw - 1]);
            v -= (b.w[u].z * tl.x + b.w[u].w * tl.y) * ev;
        }
        contrib[b.dst[u]] = v;
    }
}

// Persistent: items = (A-scan, 128-sample tile) from a counter.  The next
// item's residual window and first record batch are loaded into registers
// while the current item's products and records are processed.
__global__ void __launch_bounds__(kTcThreads, 1)
    bwd_tc_kernel(GeomParams P, TcLayout T, const uint4* __restrict__ bop, const __nv_bfloat162* __restrict__ tab,
                  const __nv_bfloat16* __restrict__ e, const long long* __restrict__ rec_off,
                  const int2* __restrict__ rkey, const float4* __restrict__ rw, const int* __restrict__ tile_off,
                  const uint32_t* __restrict__ dest, float* __restrict__ contrib, int* __restrict__ counter,
                  int* __restrict__ status)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + 8);
    volatile int* next = reinterpret_cast<volatile int*>(smem + 16);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + 20);
    unsigned char* sH = smem + T.off_h;
    unsigned char* sB = smem + T.off_b;
    __nv_bfloat16* sE = reinterpret_cast<__nv_bfloat16*>(smem + T.off_e);
    float* sC = reinterpret_cast<float*>(smem + T.off_c);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    // the table operand T^T (rows x taps, K-major), the same for every item
    const int nb16 = (int)((size_t)T.npad * T.kpad * 2 / 16);
    for (int i = tid; i < nb16; i += blockDim.x) reinterpret_cast<uint4*>(sB)[i] = __ldg(bop + i);
    if (tid == 0) {
        mbar_init(smem_u32(bar), 1);
        *abort_flag = 0;
        *next = atomicAdd(counter, 1);
        fence_mbar_init();
    }
    if (warp == 0) tmem_alloc(smem_u32(tslot), kTcCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    const int ntile = (P.M + kTcTile - 1) / kTcTile;
    const int nitems = P.K * ntile;
    const int W = kTcTile + T.kpad;                  // residual window length (<= kTcThreads)
    const uint32_t lbo = 128, sbo = (uint32_t)(T.kpad / 8) * 128;
    const uint32_t id0 = umma_idesc_bf16(kTcTile, T.nchunk0), id1 = umma_idesc_bf16(kTcTile, T.nchunk1 ? T.nchunk1 : 16);
    const int kc = T.kpad / 8;
    const __nv_bfloat16 zero = __float2bfloat16_rn(0.0f);

    // prefetch of item `it`: window value, record range and first batch
    int it = *next;
    __nv_bfloat16 ew = zero;
    long long pbase = 0;
    int pr0 = 0, pr1 = 0;
    TcBatch pb;
    auto prefetch = [&](int item) {
        const int k = item / ntile, t = item - k * ntile;
        const int n = t * kTcTile + 1 + tid;
        ew = (tid < W && n < P.Mp) ? e[(size_t)k * P.Mp + n] : zero;
        pbase = __ldg(rec_off + k);
        pr0 = __ldg(tile_off + (size_t)k * (ntile + 1) + t);
        pr1 = __ldg(tile_off + (size_t)k * (ntile + 1) + t + 1);
        tc_load_batch(pb, rkey, rw, dest, pbase, pr0, pr1, tid);
    };
    if (it < nitems) prefetch(it);
    uint32_t phase = 0;
    while (it < nitems) {
        const int t = it % ntile, ts = t * kTcTile;
        const long long base = pbase;
        const int r0 = pr0, r1 = pr1;
        if (tid < W) sE[tid] = ew;
        __syncthreads();                             // window visible; every thread has read *next
        if (tid == 0) *next = atomicAdd(counter, 1);
        // Hankel tile H[n][m] = e[ts + n + 1 + m], 8 taps (16 bytes) per store
        const unsigned short* sEu = reinterpret_cast<const unsigned short*>(sE);
        for (int c = tid; c < kTcTile * kc; c += blockDim.x) {
            const int n = c / kc, j = c - n * kc;
            const unsigned short* src = sEu + n + 8 * j;
            uint4 w;
            w.x = (uint32_t)src[0] | ((uint32_t)src[1] << 16);
            w.y = (uint32_t)src[2] | ((uint32_t)src[3] << 16);
            w.z = (uint32_t)src[4] | ((uint32_t)src[5] << 16);
            w.w = (uint32_t)src[6] | ((uint32_t)src[7] << 16);
            *reinterpret_cast<uint4*>(sH + kmajor_offset(n, 8 * j, T.kpad)) = w;
        }
        fence_async_smem();
        __syncthreads();                             // H complete; *next holds the following item
        const int it_next = *next;
        if (tid == 0) {
            tc_fence_after();
            const uint32_t a0 = smem_u32(sH), b0 = smem_u32(sB);
            for (int s = 0; s < T.kpad / 16; ++s) {
                const uint64_t da = umma_desc(a0 + 256 * s, lbo, sbo);
                umma_bf16(tmem, da, umma_desc(b0 + 256 * s, lbo, sbo), id0, s > 0);
                if (T.nchunk1)
                    umma_bf16(tmem + T.nchunk0, da, umma_desc(b0 + (T.nchunk0 / 8) * sbo + 256 * s, lbo, sbo), id1,
                              s > 0);
            }
            umma_commit(smem_u32(bar));
        }
        if (!mbar_wait_bounded(smem_u32(bar), phase, status)) *abort_flag = 1;
        phase ^= 1u;
        __syncthreads();                             // the flag is read uniformly: tensor-memory loads are warp-collective
        tc_fence_after();
        if (!*abort_flag) {
            // tensor memory -> shared C tile: warp = (lane quarter, column quarter)
            const int q = warp & 3, part = warp >> 2;
            const int row = q * 32 + lane;
            const int cw = T.npad / 4;
            for (int c = part * cw; c < part * cw + cw; c += 4) {
                float v[4];
                tmem_ld4(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c, v);
#pragma unroll
                for (int j = 0; j < 4; ++j) sC[row * T.cstride + c + j] = v[j];
            }
        }
        tc_fence_before();
        __syncthreads();
        if (*abort_flag) break;
        // records: the prefetched first batch, then the next item's prefetch, then the rest
        tc_run_batch(pb, P, T, sC, sE, tab, ts, r0, r1, tid, contrib);
        if (it_next < nitems) prefetch(it_next);
        for (int rb = r0 + kTcUnroll * kTcThreads; rb < r1; rb += kTcUnroll * kTcThreads) {
            TcBatch b;
            tc_load_batch(b, rkey, rw, dest, base, rb, r1, tid);
            tc_run_batch(b, P, T, sC, sE, tab, ts, rb, r1, tid, contrib);
        }
        __syncthreads();                             // sC / sE are rewritten by the next item
        it = it_next;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, kTcCols);
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

// Builds the tensor-core adjoint's tables for a BF16 geometry with records.
// Returns cudaErrorNotSupported (the caller keeps the other adjoint) when the
// layout does not fit or memory is short.
cudaError_t build_tc_adjoint(mbir_geometry* g, cudaStream_t st)
{
    const GeomParams& P = g->P;
    if (P.precision != MBIR_PREC_BF16 || !g->d_rec_key || g->n_records <= 0 || g->n_records >= (1LL << 32))
        return cudaErrorNotSupported;
    const TcLayout L = tc_layout(P);
    if (!L.ok) return cudaErrorNotSupported;
    const int N = P.W * P.H;
    const int ntile = (P.M + kTcTile - 1) / kTcTile;
    const int R = P.Q + 1, nq = P.Q * P.Tw + 1;
    // table operand: row c = phase * G + plane, column m = tap, BF16 as in the stored table
    std::vector<__nv_bfloat16> bimg((size_t)L.npad * L.kpad, __float2bfloat16_rn(0.0f));
    for (int c = 0; c < L.ncols; ++c) {
        const int gpl = c % P.G, ph = c / P.G;
        for (int m = 0; m < P.Tw; ++m)
            bimg[kmajor_offset(c, m, L.kpad) / 2] = __float2bfloat16_rn((float)g->tab_host[(size_t)gpl * nq + m * P.Q + ph]);
    }
    (void)R;
    int* d_cnt = nullptr;
    int* d_tile = nullptr;
    long long* d_poff = nullptr;
    uint32_t* d_dest = nullptr;
    float* d_contrib = nullptr;
    uint4* d_b = nullptr;
    cudaError_t e = cudaMalloc((void**)&d_cnt, sizeof(int) * (size_t)N);
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
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? cudaErrorNotSupported : e;
    }
    g->tc = L;
    g->d_tc_bop = d_b;
    g->d_tc_tile = d_tile;
    g->d_tc_pixoff = d_poff;
    g->d_tc_dest = d_dest;
    g->w_tc_contrib = d_contrib;
    g->bytes += bimg.size() * 2 + sizeof(int) * (size_t)P.K * (ntile + 1) + sizeof(long long) * ((size_t)N + 1) +
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
    bwd_tc_kernel<<<grid, kTcThreads, L.smem, st>>>(P, L, g->d_tc_bop, g->d_tab_bf16, e_bf, g->d_rec_off,
                                                    g->d_rec_key, g->d_rec_w, g->d_tc_tile, g->d_tc_dest,
                                                    g->w_tc_contrib, g->d_tc_counter, g->d_status);
    ce = cudaGetLastError();
    if (ce != cudaSuccess) return ce;
    const int N = P.W * P.H;
    bwd_tc_reduce_kernel<<<std::max(1, std::min((N + 7) / 8, 152 * 16)), 256, 0, st>>>(N, g->d_tc_pixoff,
                                                                                     g->w_tc_contrib, b);
    return cudaGetLastError();
}

}  // namespace mbir
