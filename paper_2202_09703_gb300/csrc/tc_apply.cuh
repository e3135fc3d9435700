// Tensor-core adjoint pools, shared by the single-request kernels
// (tc_adjoint.cu) and the batched engine (engine.cu).
// A pool function drains one geometry's (or request's) work counter; every
// thread of the CTA calls it, with the tensor memory already allocated and
// the header of the dynamic shared memory (offset 0: mbarrier, tensor-memory
// address, item slot, abort flag) initialised.  It returns false when a
// bounded wait gave up (the status word is then set).
#pragma once

#include "apply_common.cuh"
#include <cuda_fp16.h>

#include "tc_common.cuh"

namespace mbir {

constexpr int kTcTile = 128;         // A^T: samples per MMA tile (M)
constexpr int kTcThreads = 512;      // 16 warps: four per tensor-memory lane quarter
constexpr int kTcUnroll = 4;         // records in flight per thread
constexpr uint32_t kTcCols = 512;    // tensor-memory columns of the A^T kernels

// A^T of one geometry / request.
struct TcAdjView {
    GeomParams P;
    TcLayout T;
    const uint4* bop;                // table operand image (rows x taps, K-major)
    const __nv_bfloat162* tab;       // BF16 kernel table (for the tau = t0 tap)
    const __nv_bfloat16* e;          // residual, K x Mp
    const long long* rec_off;
    const int2* rkey;
    const float4* rw;
    const int* tile_off;
    const uint2* prange;             // per (A-scan, tile): lowest | highest plane << 16 (.x)
    const uint32_t* dest;            // record -> pixel-major place
    float* contrib;                  // one contribution per record
    int* counter;                    // item counter (zeroed before the launch)
};

// FP32 A^T of one geometry / request (two-part FP16 split, two row halves).
struct Tc3View {
    GeomParams P;
    Tc3Layout T;
    const uint4* bop;                // half 0 image then half 1 image (two parts each)
    const float2* tab;               // FP32 kernel table (for the tau = t0 tap)
    const float* e;                  // residual, K x Mp
    const long long* rec_off;
    const int2* rkey;
    const float4* rw;
    const int* tile_off;
    const uint2* prange;             // per (A-scan, tile): each half's lowest | highest plane << 16
    const uint32_t* dest;
    float* contrib;
    int* counter;
};

// Shared-memory header of the tensor-core kernels.
__device__ __forceinline__ void tc_header_init(unsigned char* smem, uint32_t ncols)
{
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
    if (threadIdx.x == 0) {
        mbar_init(smem_u32(bar), 1);
        mbar_init(smem_u32(smem + 32), 1);          // operand copies of the FP32 kernels
        mbar_init(smem_u32(smem + 40), 1);          // second MMA buffer of the FP32 A x
        *reinterpret_cast<volatile int*>(smem + 20) = 0;
        fence_mbar_init();
    }
    if ((threadIdx.x >> 5) == 0) tmem_alloc(smem_u32(smem + 8), ncols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
}

__device__ __forceinline__ void tc_header_release(unsigned char* smem, uint32_t tmem, uint32_t ncols)
{
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if ((threadIdx.x >> 5) == 0) tmem_dealloc(tmem, ncols);
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
        const float* cr = sC + (n0 - ts) * T.cstride + ph;      // plane-major rows: plane * (Q + 1) + phase
        float v = b.w[u].x * cr[gi * R];
        v = fmaf(b.w[u].y, cr[g1 * R], v);
        v = fmaf(b.w[u].z, cr[gi * R + 1], v);
        v = fmaf(b.w[u].w, cr[g1 * R + 1], v);
        if (b.key[u].y & 1) {
            const float2 tl = __bfloat1622float2(__ldg(tab + ((size_t)gi * R + ph + 1) * S + P.Tw - 1));
            const float ev = __bfloat162float(sE[n0 - ts + P.Tw - 1]);
            v -= (b.w[u].z * tl.x + b.w[u].w * tl.y) * ev;
        }
        contrib[b.dst[u]] = v;
    }
}


// Drains the A^T items (A-scan, 128-sample tile) of V.  The next item's
// residual window and first record batch are loaded into registers while the
// current item's products and records are processed.  Table rows are
// plane-major (plane * (Q + 1) + phase): only the rows of the attenuation
// planes that the tile's records reach (precomputed per tile) are multiplied
// and read back, and a tile without records is skipped.
__device__ __forceinline__ bool tc_adjoint_pool(const TcAdjView& V, unsigned char* smem, uint32_t tmem,
                                                uint32_t& phase, int* status)
{
    const GeomParams& P = V.P;
    const TcLayout& T = V.T;
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
    volatile int* next = reinterpret_cast<volatile int*>(smem + 16);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + 20);
    unsigned char* sH = smem + T.off_h;
    unsigned char* sB = smem + T.off_b;
    __nv_bfloat16* sE = reinterpret_cast<__nv_bfloat16*>(smem + T.off_e);
    float* sC = reinterpret_cast<float*>(smem + T.off_c);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const __nv_bfloat162* __restrict__ tab = V.tab;
    const __nv_bfloat16* __restrict__ e = V.e;
    const long long* __restrict__ rec_off = V.rec_off;
    const int2* __restrict__ rkey = V.rkey;
    const float4* __restrict__ rw = V.rw;
    const int* __restrict__ tile_off = V.tile_off;
    const uint32_t* __restrict__ dest = V.dest;
    float* __restrict__ contrib = V.contrib;
    int* counter = V.counter;

    // the table operand T^T (rows x taps, K-major), the same for every item
    const int nb16 = (int)((size_t)T.npad * T.kpad * 2 / 16);
    for (int i = tid; i < nb16; i += blockDim.x) reinterpret_cast<uint4*>(sB)[i] = __ldg(V.bop + i);
    if (tid == 0) *next = atomicAdd(counter, 1);
    __syncthreads();
    const int ntile = (P.M + kTcTile - 1) / kTcTile;
    const int nitems = P.K * ntile;
    const int W = kTcTile + T.kpad;                  // residual window length (<= kTcThreads)
    const uint32_t lbo = 128, sbo = (uint32_t)(T.kpad / 8) * 128;
    const int kc = T.kpad / 8;
    const __nv_bfloat16 zero = __float2bfloat16_rn(0.0f);

    // prefetch of item `it`: window value, record range and first batch
    int it = *next;
    __nv_bfloat16 ew = zero;
    long long pbase = 0;
    int pr0 = 0, pr1 = 0;
    uint32_t ppl = 0;
    TcBatch pb;
    auto prefetch = [&](int item) {
        const int k = item / ntile, t = item - k * ntile;
        const int n = t * kTcTile + 1 + tid;
        ew = (tid < W && n < P.Mp) ? e[(size_t)k * P.Mp + n] : zero;
        pbase = __ldg(rec_off + k);
        pr0 = __ldg(tile_off + (size_t)k * (ntile + 1) + t);
        pr1 = __ldg(tile_off + (size_t)k * (ntile + 1) + t + 1);
        ppl = __ldg(&V.prange[item].x);
        tc_load_batch(pb, rkey, rw, dest, pbase, pr0, pr1, tid);
    };
    if (it < nitems) prefetch(it);
    while (it < nitems) {
        const int t = it % ntile, ts = t * kTcTile;
        const long long base = pbase;
        const int r0 = pr0, r1 = pr1;
        // the table rows (plane-major) of the planes the tile's records reach, in whole 16-row steps
        const int glo = (int)(ppl & 0xffffu), ghi = (int)(ppl >> 16);
        const int n_lo = glo <= ghi ? (glo * (P.Q + 1)) & ~15 : 0;
        const int nr = glo <= ghi ? min(T.npad, ((ghi + 1) * (P.Q + 1) + 15) & ~15) - n_lo : 0;
        const int nr0 = nr > 256 ? ((nr / 2) + 15) & ~15 : nr, nr1 = nr - nr0;
        if (tid < W) sE[tid] = ew;
        __syncthreads();                             // window visible; every thread has read *next
        if (tid == 0) *next = atomicAdd(counter, 1);
        // Hankel tile H[n][m] = e[ts + n + 1 + m], 8 taps (16 bytes) per store
        const unsigned short* sEu = reinterpret_cast<const unsigned short*>(sE);
        for (int c = tid; c < kTcTile * kc; c += blockDim.x) {
            const int n8 = c >> 3, j = n8 % kc, n = (n8 / kc) * 8 + (c & 7);   // lanes along a core matrix's rows
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
        if (nr > 0) {                                // a tile without records has nothing to correlate
            if (tid == 0) {
                tc_fence_after();
                const uint32_t a0 = smem_u32(sH), b0 = smem_u32(sB) + (uint32_t)(n_lo / 8) * sbo;
                const uint32_t id0 = umma_idesc_bf16(kTcTile, nr0), id1 = umma_idesc_bf16(kTcTile, nr1 ? nr1 : 16);
                for (int s = 0; s < T.kpad / 16; ++s) {
                    const uint64_t da = umma_desc(a0 + 256 * s, lbo, sbo);
                    umma_bf16(tmem, da, umma_desc(b0 + 256 * s, lbo, sbo), id0, s > 0);
                    if (nr1)
                        umma_bf16(tmem + nr0, da, umma_desc(b0 + (nr0 / 8) * sbo + 256 * s, lbo, sbo), id1, s > 0);
                }
                umma_commit(smem_u32(bar));
            }
            if (!mbar_wait_bounded(smem_u32(bar), phase, status)) *abort_flag = 1;
            phase ^= 1u;
            __syncthreads();                         // the flag is read uniformly: tensor-memory loads are warp-collective
            tc_fence_after();
            if (!*abort_flag) {
                // tensor memory -> shared C tile (the range's rows only): warp = (lane quarter, column quarter)
                const int q = warp & 3, part = warp >> 2;
                const int row = q * 32 + lane;
                const int cw = nr / 4;
                for (int c = part * cw; c < part * cw + cw; c += 4) {
                    float v[4];
                    tmem_ld4(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c, v);
#pragma unroll
                    for (int j = 0; j < 4; ++j) sC[row * T.cstride + n_lo + c + j] = v[j];
                }
            }
            tc_fence_before();
            __syncthreads();
            if (*abort_flag) break;
        }
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
    return !*abort_flag;
}

// x = b1 + b2 + b3 with BF16 parts (exact for FP32 x away from underflow).
__device__ __forceinline__ void split3(float x, unsigned short& a, unsigned short& b, unsigned short& c)
{
    const __nv_bfloat16 p1 = __float2bfloat16_rn(x);
    const float r1 = x - __bfloat162float(p1);
    const __nv_bfloat16 p2 = __float2bfloat16_rn(r1);
    const __nv_bfloat16 p3 = __float2bfloat16_rn(r1 - __bfloat162float(p2));
    a = __bfloat16_as_ushort(p1);
    b = __bfloat16_as_ushort(p2);
    c = __bfloat16_as_ushort(p3);
}

// Two values into packed FP16 high and low parts: hi = x rounded to 11 significant bits by Veltkamp's
// splitting, (x (2^13 + 1)) - ((x (2^13 + 1)) - x) (exact in FP16 for |x| in [2^-14, 2^15]), and
// lo = x - hi (exact in FP32) rounded to FP16; x = hi + lo to 2^-23 relative.  No packed conversion
// is spent on the high part's remainder.
__device__ __forceinline__ void split2h_pair(float x0, float x1, uint32_t& hi, uint32_t& lo)
{
    const float t0 = __fmul_rn(x0, 8193.0f), t1 = __fmul_rn(x1, 8193.0f);
    const float h0 = __fsub_rn(t0, __fsub_rn(t0, x0)), h1 = __fsub_rn(t1, __fsub_rn(t1, x1));
    const __half2 H = __floats2half2_rn(h0, h1);
    const __half2 L = __floats2half2_rn(__fsub_rn(x0, h0), __fsub_rn(x1, h1));
    hi = *reinterpret_cast<const uint32_t*>(&H);
    lo = *reinterpret_cast<const uint32_t*>(&L);
}

// Contributions of a batch's records whose phase falls in `half`, from that
// half's correlation tile (columns plane * pstride + phase - first phase of the half).
__device__ __forceinline__ void tc3_run_batch(const TcBatch& b, const GeomParams& P, const Tc3Layout& T, int half,
                                              const float* sC, const float* sE, const float2* __restrict__ tab,
                                              int ts, int rb, int r1, int tid, float* __restrict__ contrib)
{
    const int R = P.Q + 1, S = table_stride(P.Tw4);
    const int phb = half ? T.phsplit : 0;
#pragma unroll
    for (int u = 0; u < kTcUnroll; ++u) {
        const int r = rb + u * kTcThreads + tid;
        if (r >= r1) continue;
        const int n0 = b.key[u].y >> kRecShift, trow = (b.key[u].y >> 1) & 0xfff;
        const int gi = trow / R, ph = trow - gi * R;
        if ((ph >= T.phsplit) != (half == 1)) continue;
        const int g1 = min(gi + 1, P.G - 1);
        const float* cr = sC + (n0 - ts) * T.cstride + (ph - phb);     // plane-major rows
        float v = b.w[u].x * cr[gi * T.pstride];
        v = fmaf(b.w[u].y, cr[g1 * T.pstride], v);
        v = fmaf(b.w[u].z, cr[gi * T.pstride + 1], v);
        v = fmaf(b.w[u].w, cr[g1 * T.pstride + 1], v);
        if (b.key[u].y & 1) {
            const float2 tl = __ldg(tab + ((size_t)gi * R + ph + 1) * S + P.Tw - 1);
            v -= (b.w[u].z * tl.x + b.w[u].w * tl.y) * sE[n0 - ts + P.Tw - 1];
        }
        contrib[b.dst[u]] = v;
    }
}

// Drains the FP32 A^T items (A-scan, 128-sample tile) of V.  Per item: the
// residual window, scaled by a power of two that brings its largest magnitude
// into [2^14, 2^15), split into two FP16 Hankel tiles; for each row half the
// three products H_1 T_1 + H_1 T_2 + H_2 T_1 with the two-part table (scaled
// on the host; the dropped H_2 T_2 is below 2^-22 of the result) accumulate in
// tensor memory and are scaled back as they are read.  The table rows are
// plane-major (plane * pstride + phase offset): per half only the rows of the
// attenuation planes that the tile's records reach (precomputed per tile) are
// multiplied and read back, and a half without records is skipped.  Both
// halves' table operands stay resident (one bulk copy per pool, mbarrier at
// smem + 32); smem + 64 holds the warps' window maxima.
__device__ __forceinline__ bool tc_adjoint32_pool(const Tc3View& V, unsigned char* smem, uint32_t tmem,
                                                  uint32_t& phase, uint32_t& bphase, int* status)
{
    const GeomParams& P = V.P;
    const Tc3Layout& T = V.T;
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
    uint64_t* bbar = reinterpret_cast<uint64_t*>(smem + 32);
    volatile int* next = reinterpret_cast<volatile int*>(smem + 16);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + 20);
    unsigned char* sH = smem + T.off_h;
    unsigned char* sB = smem + T.off_b;
    float* sE = reinterpret_cast<float*>(smem + T.off_e);
    float* sC = reinterpret_cast<float*>(smem + T.off_c);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const float* __restrict__ e = V.e;
    const long long* __restrict__ rec_off = V.rec_off;
    const int2* __restrict__ rkey = V.rkey;
    const float4* __restrict__ rw = V.rw;
    const int* __restrict__ tile_off = V.tile_off;
    const uint32_t* __restrict__ dest = V.dest;
    float* __restrict__ contrib = V.contrib;
    int* counter = V.counter;
    const unsigned char* bimg = reinterpret_cast<const unsigned char*>(V.bop);
    const size_t hbytes = (size_t)kTcTile * T.kpad * 2;     // one part of the Hankel tile
    float* wmax = reinterpret_cast<float*>(smem + 64);
    // both halves' table operands, once
    int copies = 1, waits = 0;                   // the same on every thread
    if (tid == 0) {
        mbar_arrive_expect_tx(smem_u32(bbar), (uint32_t)(T.bhalf[0] + T.bhalf[1]));
        bulk_g2s(smem_u32(sB), bimg, (uint32_t)(T.bhalf[0] + T.bhalf[1]), smem_u32(bbar));
        *next = atomicAdd(counter, 1);
    }
    __syncthreads();
    const float it_scale = __int_as_float((127 - T.texp) << 23);
    const int ntile = (P.M + kTcTile - 1) / kTcTile;
    const int nitems = P.K * ntile;
    const int W = kTcTile + T.kpad;
    const uint32_t lbo = 128, sbo = (uint32_t)(T.kpad / 8) * 128;
    const int kc = T.kpad / 8;
    int it = *next;
    float ew = 0.0f;
    long long pbase = 0;
    int pr0 = 0, pr1 = 0;
    uint2 ppl = make_uint2(0u, 0u);
    TcBatch pb;
    auto prefetch = [&](int item) {
        const int k = item / ntile, t = item - k * ntile;
        const int n = t * kTcTile + 1 + tid;
        ew = (tid < W && n < P.Mp) ? e[(size_t)k * P.Mp + n] : 0.0f;
        pbase = __ldg(rec_off + k);
        pr0 = __ldg(tile_off + (size_t)k * (ntile + 1) + t);
        pr1 = __ldg(tile_off + (size_t)k * (ntile + 1) + t + 1);
        ppl = __ldg(V.prange + item);
        tc_load_batch(pb, rkey, rw, dest, pbase, pr0, pr1, tid);
    };
    if (it < nitems) prefetch(it);
    while (it < nitems) {
        const int t = it % ntile, ts = t * kTcTile;
        const long long base = pbase;
        const int r0 = pr0, r1 = pr1;
        const uint2 planes = ppl;
        if (tid < W) sE[tid] = ew;
        {
            // the window's largest magnitude, one value per warp
            float mx = fabsf(ew);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            if (lane == 0) wmax[warp] = mx;
        }
        __syncthreads();
        if (tid == 0) *next = atomicAdd(counter, 1);
        int se = 0;
        {
            float m = 0.0f;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, wmax[w]);
            int ex = 0;
            frexpf(m, &ex);
            se = m > 0.0f ? min(15 - ex, 126) : 0;
        }
        const float scl = __int_as_float((se + 127) << 23);
        const float unscale = __int_as_float((127 - se) << 23);       // then 2^-texp: two normal factors
        // two FP16 Hankel tiles H_i[n][m] = part i of 2^se e[ts + n + 1 + m]
        for (int c = tid; c < kTcTile * kc; c += blockDim.x) {
            const int n8 = c >> 3, j = n8 % kc, n = (n8 / kc) * 8 + (c & 7);   // lanes along a core matrix's rows
            uint4 hv, lv;
            const float* src = sE + n + 8 * j;
            split2h_pair(src[0] * scl, src[1] * scl, hv.x, lv.x);
            split2h_pair(src[2] * scl, src[3] * scl, hv.y, lv.y);
            split2h_pair(src[4] * scl, src[5] * scl, hv.z, lv.z);
            split2h_pair(src[6] * scl, src[7] * scl, hv.w, lv.w);
            const uint32_t off = kmajor_offset(n, 8 * j, T.kpad);
            *reinterpret_cast<uint4*>(sH + off) = hv;
            *reinterpret_cast<uint4*>(sH + hbytes + off) = lv;
        }
        fence_async_smem();
        __syncthreads();
        const int it_next = *next;
        if (waits < copies) {
            // the table operands have landed (once per pool)
            if (!mbar_wait_bounded(smem_u32(bbar), bphase, status)) *abort_flag = 1;
            bphase ^= 1u;
            ++waits;
            __syncthreads();
        }
        for (int h = 0; h < 2; ++h) {
            // the rows of the planes this half's records reach, in whole 16-row steps (uniform)
            const uint32_t pw = h ? planes.y : planes.x;
            const int glo = (int)(pw & 0xffffu), ghi = (int)(pw >> 16);
            if (glo > ghi) continue;                 // no record of the tile in this half
            const int n_lo = (glo * T.pstride) & ~15;
            const int nr = min(T.nrows[h], ((ghi + 1) * T.pstride + 15) & ~15) - n_lo;
            if (tid == 0 && !*abort_flag) {
                tc_fence_after();
                const uint32_t idesc = umma_idesc_f16(kTcTile, nr);
                const uint32_t a0 = smem_u32(sH);
                const uint32_t b0 = smem_u32(sB) + (uint32_t)(h ? T.bhalf[0] : 0) + (uint32_t)(n_lo / 8) * sbo;
                const uint32_t bpart = (uint32_t)((size_t)T.nrows[h] * T.kpad * 2);
                const int terms[3][2] = {{0, 0}, {0, 1}, {1, 0}};
                for (int s = 0; s < T.kpad / 16; ++s)
                    for (int q = 0; q < 3; ++q)
                        umma_bf16(tmem, umma_desc(a0 + (uint32_t)(terms[q][0] * hbytes) + 256 * s, lbo, sbo),
                                  umma_desc(b0 + terms[q][1] * bpart + 256 * s, lbo, sbo), idesc, s > 0 || q > 0);
                umma_commit(smem_u32(bar));
            }
            __syncthreads();
            if (*abort_flag) break;
            if (!mbar_wait_bounded(smem_u32(bar), phase, status)) *abort_flag = 1;
            phase ^= 1u;
            __syncthreads();                         // uniform flag
            tc_fence_after();
            if (*abort_flag) break;
            {
                const int q = warp & 3, part = warp >> 2;
                const int row = q * 32 + lane;
                const int cw = nr / 4;
                for (int c = part * cw; c < part * cw + cw; c += 4) {
                    float v[4];
                    tmem_ld4(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c, v);
#pragma unroll
                    for (int j = 0; j < 4; ++j) sC[row * T.cstride + n_lo + c + j] = (v[j] * unscale) * it_scale;
                }
            }
            tc_fence_before();
            __syncthreads();
            tc3_run_batch(pb, P, T, h, sC, sE, V.tab, ts, r0, r1, tid, contrib);
            for (int rb = r0 + kTcUnroll * kTcThreads; rb < r1; rb += kTcUnroll * kTcThreads) {
                TcBatch b;
                tc_load_batch(b, rkey, rw, dest, base, rb, r1, tid);
                tc3_run_batch(b, P, T, h, sC, sE, V.tab, ts, rb, r1, tid, contrib);
            }
            __syncthreads();                         // sC is rewritten by the next half
        }
        if (*abort_flag) break;
        if (it_next < nitems) prefetch(it_next);
        it = it_next;
    }
    // no operand copy may outlive the pool (bounded)
    while (waits < copies) {
        mbar_wait_bounded(smem_u32(bbar), bphase, status);
        bphase ^= 1u;
        ++waits;
    }
    __syncthreads();
    return !*abort_flag;
}

}  // namespace mbir
