// Tensor-core apply pools of the BF16 form, shared by the single-request
// kernels (tc_adjoint.cu, tc_forward.cu) and the batched engine (engine.cu).
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
constexpr int kTfTile = 128;         // A x: values of n0 per MMA tile (M)
constexpr int kTfThreads = 512;      // scatter: 4 threads per n0 (phase classes mod 4)
constexpr int kTfUnroll = 8;         // records in flight per scatter thread
constexpr int kTfStage = 6;          // 8-column groups per thread held in registers while converting
constexpr uint32_t kTfCols = 128;    // tensor-memory columns of the A x kernels
constexpr uint32_t kTf3Cols = 256;   // FP32 A x: one 128-column tile per row half
constexpr int kTf3HalfCols = 128;
constexpr int kTf3Unroll = 4;        // FP32 A x: records of each of the two groups in flight per thread
static_assert(kTcThreads == kTfThreads, "the engine runs both pools with one block size");

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

// A x of one geometry / request.
struct TcFwdView {
    GeomParams P;
    TfLayout T;
    const uint4* bop;                // table operand image (taps x table rows, K-major)
    const __nv_bfloat162* tab;
    const long long* rec_off;
    const int* n0_off;
    const ushort4* grp_off;          // per (A-scan, n0): starts of phase classes 1..3 in the bucket
    const int2* rkey;
    const float4* rw;
    const int* order;                // A-scans by decreasing record count
    const float* xr;                 // x gathered per record (record order), see tc_gather_x
    float* y_f32;
    __nv_bfloat16* y_bf16;
    int out_stride;
    int* counter;
};

// FP32 A x of one geometry / request (two-part FP16 split, two phase-aligned halves).
struct TcFwd32View {
    GeomParams P;
    Tf3Layout T;
    const uint4* bop;                // half 0 image then half 1 image (three parts each)
    const float2* tab;               // FP32 kernel table (for the tau = t0 tap)
    const long long* rec_off;
    const int* n0_off;
    const uint4* grp_off;            // per (A-scan, n0): starts of the (half, class) groups 1..7 (16 bits each)
    const int2* rkey;
    const float4* rw;
    const int* order;
    const float* xr;
    float* y;
    int out_stride;
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

// FP32 sums of one column half (cw valid columns, kh padded) -> BF16 pairs in registers.
__device__ __forceinline__ void tf_stage_half(uint4 (&pk)[kTfStage], const float* src, int astr, int cw, int kh, int tid)
{
    const int kc = kh / 8;
#pragma unroll
    for (int q = 0; q < kTfStage; ++q) {
        const int c = tid + q * kTfThreads;
        if (c < kTfTile * kc) {
            const int i8 = c >> 3, j = i8 % kc, i = (i8 / kc) * 8 + (c & 7);   // lanes along a core matrix's rows
            const float* sp = src + i * astr + 8 * j;
            uint32_t w[4];
#pragma unroll
            for (int e2 = 0; e2 < 4; ++e2) {
                const int cc = 8 * j + 2 * e2;
                const float a = cc < cw ? sp[2 * e2] : 0.0f, b = cc + 1 < cw ? sp[2 * e2 + 1] : 0.0f;
                const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
                w[e2] = *reinterpret_cast<const uint32_t*>(&v);
            }
            pk[q] = make_uint4(w[0], w[1], w[2], w[3]);
        }
    }
}

// The staged BF16 pairs -> an operand buffer (K-major core matrices, ka columns).
__device__ __forceinline__ void tf_write_half(const uint4 (&pk)[kTfStage], unsigned char* dst, int kh, int ka, int tid)
{
    const int kc = kh / 8;
#pragma unroll
    for (int q = 0; q < kTfStage; ++q) {
        const int c = tid + q * kTfThreads;
        if (c < kTfTile * kc) {
            const int i8 = c >> 3, j = i8 % kc, i = (i8 / kc) * 8 + (c & 7);   // lanes along a core matrix's rows
            *reinterpret_cast<uint4*>(dst + kmajor_offset(i, 8 * j, ka)) = pk[q];
        }
    }
}

// xr[r] = x[pixel of record r] for records [0, nrec) (grid-stride, all blocks).
__device__ __forceinline__ void tc_gather_x(long long nrec, const int2* __restrict__ rkey, const float* __restrict__ x,
                                            float* __restrict__ xr)
{
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < nrec;
         r += (long long)gridDim.x * blockDim.x)
        xr[r] = __ldg(x + __ldg(&rkey[r].x));
}

// Drains the A x items (A-scans, largest first) of V.
__device__ __forceinline__ bool tc_forward_pool(const TcFwdView& V, unsigned char* smem, uint32_t tmem,
                                                uint32_t& phase, int* status)
{
    const GeomParams& P = V.P;
    const TfLayout& T = V.T;
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
    volatile int* next = reinterpret_cast<volatile int*>(smem + 16);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + 20);
    unsigned char* sB = smem + T.off_b;
    unsigned char* sA = smem + T.off_a;
    float* sAcc = reinterpret_cast<float*>(smem + T.off_acc);
    float* sAcc1 = reinterpret_cast<float*>(smem + T.off_acc1);
    float* sY = reinterpret_cast<float*>(smem + T.off_y);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int R = P.Q + 1, S = table_stride(P.Tw4);
    const __nv_bfloat162* __restrict__ tab = V.tab;
    const long long* __restrict__ rec_off = V.rec_off;
    const int* __restrict__ n0_off = V.n0_off;
    const ushort4* __restrict__ grp_off = V.grp_off;
    const int2* __restrict__ rkey = V.rkey;
    const float4* __restrict__ rw = V.rw;
    const int* __restrict__ order = V.order;
    const float* __restrict__ xr = V.xr;
    float* __restrict__ y_f32 = V.y_f32;
    __nv_bfloat16* __restrict__ y_bf16 = V.y_bf16;
    const int out_stride = V.out_stride;
    int* counter = V.counter;

    // table operand: rows = taps, columns = table rows (plane * (Q + 1) + phase, plane-major), K-major
    const int nb16 = (int)((size_t)T.ntap * T.kb * 2 / 16);
    for (int i = tid; i < nb16; i += blockDim.x) reinterpret_cast<uint4*>(sB)[i] = __ldg(V.bop + i);
    __syncthreads();
    const int ntile = (P.M + kTfTile - 1) / kTfTile;
    const uint32_t lbo = 128, sboA = (uint32_t)(T.ka / 8) * 128, sboB = (uint32_t)(T.kb / 8) * 128;
    const uint32_t idesc = umma_idesc_bf16(kTfTile, T.ntap);
    const int si = tid >> 2, pj = tid & 3;            // scatter role: n0 row and phase class
    int* wlo = reinterpret_cast<int*>(smem + 128);
    int* whi = reinterpret_cast<int*>(smem + 192);
    for (;;) {
        if (tid == 0) *next = atomicAdd(counter, 1);
        __syncthreads();
        const int idx = *next;
        if (idx >= P.K) break;
        const int k = __ldg(order + idx);
        const long long base = __ldg(rec_off + k);
        const int* no = n0_off + (size_t)k * (P.M + 1);
        for (int i = tid; i < T.ylen; i += blockDim.x) sY[i] = 0.0f;
        for (int t = 0; t < ntile; ++t) {
            const int ts = t * kTfTile;
            const int n0 = ts + si;
            const int ra = n0 < P.M ? __ldg(no + n0) : 0, rz = n0 < P.M ? __ldg(no + n0 + 1) : 0;
            for (int i = tid; i < kTfTile * T.astride; i += blockDim.x) sAcc[i] = 0.0f;
            for (int i = tid; i < kTfTile * T.astride1; i += blockDim.x) sAcc1[i] = 0.0f;
            __syncthreads();
            // scatter: thread (n0 row si, phase class pj) owns the cells of the phases = pj (mod 4).  The
            // bucket is ordered by phase class: records of class pj - 1 bring their upper-row corners
            // (z, w), then records of class pj their lower-row corners (x, y), each in record order.
            float* arow0 = sAcc + si * T.astride;
            float* arow1 = sAcc1 + si * T.astride1 - T.c0;
            float flag_corr = 0.0f;
            int glo = P.G, ghi = -1;                 // planes this thread's records reach
            if (ra < rz) {
                const ushort4 go = __ldg(grp_off + (size_t)k * P.M + n0);
                const int gs[5] = {0, go.x, go.y, go.z, rz - ra};
                for (int pass = 0; pass < 2; ++pass) {
                    const int grp = pass == 0 ? ((pj + 3) & 3) : pj;
                    const int qa = ra + gs[grp], qz = ra + gs[grp + 1];
                    for (int rb = qa; rb < qz; rb += kTfUnroll) {
                        int2 key[kTfUnroll];
                        float4 w4[kTfUnroll];
                        float xv[kTfUnroll];
#pragma unroll
                        for (int u = 0; u < kTfUnroll; ++u)
                            if (rb + u < qz) {
                                key[u] = __ldg(rkey + base + rb + u);
                                w4[u] = __ldg(rw + base + rb + u);
                                xv[u] = __ldg(xr + base + rb + u);
                            }
#pragma unroll
                        for (int u = 0; u < kTfUnroll; ++u) {
                            if (rb + u >= qz) break;
                            const int trow = (key[u].y >> 1) & 0xfff;
                            const int gi = trow / R, ph = trow - gi * R;
                            const int g1 = min(gi + 1, P.G - 1);
                            glo = min(glo, gi);
                            ghi = max(ghi, g1);
                            if (pass == 0) {
                                const int c0 = gi * R + ph + 1, c1 = g1 * R + ph + 1;
                                (c0 < T.c0 ? arow0 : arow1)[c0] += w4[u].z * xv[u];
                                (c1 < T.c0 ? arow0 : arow1)[c1] += w4[u].w * xv[u];
                                if (key[u].y & 1) {
                                    // tau = t0 exactly: the last tap of the upper phase row lies outside
                                    const float2 tl =
                                        __bfloat1622float2(__ldg(tab + ((size_t)gi * R + ph + 1) * S + P.Tw - 1));
                                    flag_corr += xv[u] * (w4[u].z * tl.x + w4[u].w * tl.y);
                                }
                            } else {
                                const int c0 = gi * R + ph, c1 = g1 * R + ph;
                                (c0 < T.c0 ? arow0 : arow1)[c0] += w4[u].x * xv[u];
                                (c1 < T.c0 ? arow0 : arow1)[c1] += w4[u].y * xv[u];
                            }
                        }
                    }
                }
            }
            // the four class threads of a sample are adjacent lanes: their flag corrections in class order
            {
                const float f1 = __shfl_down_sync(0xffffffffu, flag_corr, 1);
                const float f2 = __shfl_down_sync(0xffffffffu, flag_corr, 2);
                const float f3 = __shfl_down_sync(0xffffffffu, flag_corr, 3);
                if (pj == 0 && n0 < P.M) sY[n0 + P.Tw] -= ((flag_corr + f1) + f2) + f3;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                glo = min(glo, __shfl_xor_sync(0xffffffffu, glo, o));
                ghi = max(ghi, __shfl_xor_sync(0xffffffffu, ghi, o));
            }
            if (lane == 0) {
                wlo[warp] = glo;
                whi[warp] = ghi;
            }
            __syncthreads();
            // the columns of the planes reached (plane-major), in whole 16-column K steps, split at the
            // halves' boundary c0; every other sum is zero (a tile without records multiplies one zero step)
            int c_lo = 0, c_hi = 16;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
                glo = min(glo, wlo[w]);
                ghi = max(ghi, whi[w]);
            }
            if (ghi >= glo) {
                c_lo = (glo * R) & ~15;
                c_hi = min(T.c0 + T.k1, ((ghi + 1) * R + 15) & ~15);
            }
            const int a0c = c_lo, z0c = min(c_hi, T.c0);                 // first half: [a0c, z0c)
            const int a1c = max(c_lo, T.c0), z1c = c_hi;                 // second half: [a1c, z1c)
            // FP32 sums -> registers -> BF16 operands (K-major, 8 columns per 16-byte store): the first
            // half's operand goes over the start of its own sums, the second half's right after it
            {
                const int ncols = P.G * R;
                unsigned char* sA1 = sA + (size_t)kTfTile * T.ka * 2;
                uint4 pk[kTfStage];
                if (z0c > a0c) tf_stage_half(pk, sAcc + a0c, T.astride, z0c - a0c, z0c - a0c, tid);
                __syncthreads();                     // every first-half sum is in registers
                if (z0c > a0c) tf_write_half(pk, sA, z0c - a0c, T.ka, tid);
                if (z1c > a1c) {
                    tf_stage_half(pk, sAcc1 + (a1c - T.c0), T.astride1, min(z1c, ncols) - a1c, z1c - a1c, tid);
                    tf_write_half(pk, sA1, z1c - a1c, T.ka, tid);
                }
                fence_async_smem();
                __syncthreads();
                if (tid == 0) {
                    tc_fence_after();
                    const uint32_t b0 = smem_u32(sB) + (uint32_t)(a0c / 8) * 128;
                    const uint32_t b1 = smem_u32(sB) + (uint32_t)(a1c / 8) * 128;
                    const uint32_t a0 = smem_u32(sA), a1 = smem_u32(sA1);
                    for (int s = 0; s < (z0c - a0c) / 16; ++s)
                        umma_bf16(tmem, umma_desc(a0 + 256 * s, lbo, sboA), umma_desc(b0 + 256 * s, lbo, sboB), idesc,
                                  s > 0);
                    for (int s = 0; s < (z1c - a1c) / 16; ++s)
                        umma_bf16(tmem, umma_desc(a1 + 256 * s, lbo, sboA), umma_desc(b1 + 256 * s, lbo, sboB),
                                  idesc, z0c > a0c || s > 0);
                    umma_commit(smem_u32(bar));
                }
            }
            if (*abort_flag) break;
            if (!mbar_wait_bounded(smem_u32(bar), phase, status)) *abort_flag = 1;
            phase ^= 1u;
            __syncthreads();
            tc_fence_after();
            if (*abort_flag) break;
            // U (tensor memory) -> shared, rows = n0 - ts, columns = taps
            {
                const int q = warp & 3, part = warp >> 2;        // 16 warps: lane quarter x column quarter
                const int row = q * 32 + lane;
                const int cwid = T.ntap / 4;
                for (int c = part * cwid; c < part * cwid + cwid; c += 4) {
                    float v[4];
                    tmem_ld4(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c, v);
#pragma unroll
                    for (int j = 0; j < 4; ++j) sAcc1[row * T.ustride + c + j] = v[j];
                }
            }
            tc_fence_before();
            __syncthreads();
            // anti-diagonals: y[ts + 1 + j] += sum_i U[i][j - i]
            for (int j = tid; j < kTfTile + T.ntap - 1; j += blockDim.x) {
                float acc = 0.0f;
                const int i0 = max(0, j - T.ntap + 1), i1 = min(kTfTile - 1, j);
                for (int i = i0; i <= i1; ++i) acc += sAcc1[i * T.ustride + j - i];
                sY[ts + 1 + j] += acc;
            }
            __syncthreads();
        }
        if (*abort_flag) break;
        float* yo = y_f32 ? y_f32 + (size_t)k * out_stride : nullptr;
        __nv_bfloat16* yb = y_f32 ? nullptr : y_bf16 + (size_t)k * out_stride;
        for (int n = tid; n < out_stride; n += blockDim.x) {
            const float v = n < P.M ? sY[n] : 0.0f;
            if (yo) yo[n] = v;
            else yb[n] = __float2bfloat16_rn(v);
        }
        __syncthreads();
    }
    return !*abort_flag;
}

// Drains the FP32 A x items (A-scans, largest first) of V.  Per tile of 128
// first-tap samples and per row half (phases [0, phsplit] and [phsplit, Q]):
// the sums S[n0][row] of the half's records are accumulated in FP32 (four
// threads per n0, one per phase class, buckets ordered by (half, class)),
// scaled by a power of two that brings their largest magnitude into
// [2^14, 2^15), converted chunk by chunk into two FP16 parts (22 significant
// bits) and multiplied by the half's two-part table operand (scaled the same
// way on the host): the three products S_1 T_1 + S_1 T_2 + S_2 T_1 (the
// dropped S_2 T_2 is below 2^-22 of the result) accumulate in the half's own
// tensor-memory tile.  The columns are plane-major (plane * pstride + phase
// offset), so the attenuation planes that a tile's records reach (a few of G)
// are one column range: only that range is converted and multiplied, the
// other sums being zero.  U = U_0 / (s_0 t) + U_1 / (s_1 t) then gives the
// anti-diagonal sums added to y.  The other half's table operand is
// bulk-copied while a half's records are scattered (mbarrier at smem + 32);
// smem + 48 holds the halves' scale exponents, smem + 64 the warp maxima,
// smem + 128 / 192 the warps' lowest / highest plane.
__device__ __forceinline__ bool tc_forward32_pool(const TcFwd32View& V, unsigned char* smem, uint32_t tmem,
                                                  uint32_t& phase, uint32_t& bphase, int* status)
{
    // phase bit 0: the MMA barrier of chunk buffer 0 (smem + 0), bit 1: of buffer 1 (smem + 40)
    const GeomParams& P = V.P;
    const Tf3Layout& T = V.T;
    uint64_t* bbar = reinterpret_cast<uint64_t*>(smem + 32);
    volatile int* next = reinterpret_cast<volatile int*>(smem + 16);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + 20);
    unsigned char* sB = smem + T.off_b;
    unsigned char* sA = smem + T.off_a;
    float* sS = reinterpret_cast<float*>(smem + T.off_s);
    float* sY = reinterpret_cast<float*>(smem + T.off_y);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int R = P.Q + 1, S = table_stride(P.Tw4);
    const float2* __restrict__ tab = V.tab;
    const long long* __restrict__ rec_off = V.rec_off;
    const int* __restrict__ n0_off = V.n0_off;
    const uint4* __restrict__ grp_off = V.grp_off;
    const int2* __restrict__ rkey = V.rkey;
    const float4* __restrict__ rw = V.rw;
    const int* __restrict__ order = V.order;
    const float* __restrict__ xr = V.xr;
    const unsigned char* bimg = reinterpret_cast<const unsigned char*>(V.bop);

    auto copy_half = [&](int h) {               // tid 0: bulk copy of half h's operand image
        mbar_arrive_expect_tx(smem_u32(bbar), (uint32_t)T.bhalf);
        bulk_g2s(smem_u32(sB), bimg + (h ? T.bhalf : 0), (uint32_t)T.bhalf, smem_u32(bbar));
    };
    int copies = 1, waits = 0;                   // the same on every thread
    if (tid == 0) copy_half(0);
    const int ntile = (P.M + kTfTile - 1) / kTfTile;
    const uint32_t lbo = 128, sboA = (uint32_t)(T.kc / 8) * 128, sboB = (uint32_t)(T.kb / 8) * 128;
    const uint32_t idesc = umma_idesc_f16(kTfTile, T.ntap);
    const uint32_t apart = (uint32_t)(kTfTile * T.kc * 2), bpart = (uint32_t)(T.ntap * T.kb * 2);
    const int si = tid >> 2, pj = tid & 3;            // scatter role: n0 row and phase class
    volatile int* sexp = reinterpret_cast<volatile int*>(smem + 48);
    float* wmax = reinterpret_cast<float*>(smem + 64);
    int* wlo = reinterpret_cast<int*>(smem + 128);
    int* whi = reinterpret_cast<int*>(smem + 192);
    // the sums start at zero; every later pass that reads them (conversion, anti-diagonals) clears them
    for (int i = tid; i < kTfTile * max(T.astride, T.ustride); i += blockDim.x) sS[i] = 0.0f;
    __syncthreads();
    for (;;) {
        if (tid == 0) *next = atomicAdd(V.counter, 1);
        __syncthreads();
        const int idx = *next;
        if (idx >= P.K) break;
        const int k = __ldg(order + idx);
        const long long base = __ldg(rec_off + k);
        const int* no = n0_off + (size_t)k * (P.M + 1);
        for (int i = tid; i < T.ylen; i += blockDim.x) sY[i] = 0.0f;
        // bucket bounds and group starts of this thread's n0, one tile ahead of their use
        int ra_n = 0, rz_n = 0;
        uint4 go_n = make_uint4(0u, 0u, 0u, 0u);
        if (si < P.M) {
            ra_n = __ldg(no + si);
            rz_n = __ldg(no + si + 1);
            go_n = __ldg(grp_off + (size_t)k * P.M + si);
        }
        for (int t = 0; t < ntile; ++t) {
            const int ts = t * kTfTile;
            const int n0 = ts + si;
            const int ra = ra_n, rz = rz_n;
            int gs[9];
            {
                const uint4 go = go_n;
                const int n1 = n0 + kTfTile;
                ra_n = rz_n = 0;
                go_n = make_uint4(0u, 0u, 0u, 0u);
                if (t + 1 < ntile && n1 < P.M) {
                    ra_n = __ldg(no + n1);
                    rz_n = __ldg(no + n1 + 1);
                    go_n = __ldg(grp_off + (size_t)k * P.M + n1);
                }
                gs[0] = 0;
                gs[1] = (int)(go.x & 0xffffu); gs[2] = (int)(go.x >> 16);
                gs[3] = (int)(go.y & 0xffffu); gs[4] = (int)(go.y >> 16);
                gs[5] = (int)(go.z & 0xffffu); gs[6] = (int)(go.z >> 16);
                gs[7] = (int)(go.w & 0xffffu); gs[8] = rz - ra;
            }
            float flag_corr = 0.0f;
            for (int h = 0; h < 2; ++h) {
                const int phb = h ? T.phsplit : 0;
                float bound = 0.0f;                  // sum of |contributions| of this thread: >= its |S| cells
                int glo = P.G, ghi = -1;              // planes this thread's records reach
                // scatter: thread (n0 row si, phase class pj) owns the cells of this half whose phase is pj
                // (mod 4): upper-row corners of class pj - 1 records, then lower-row corners of class pj
                float* arow = sS + si * T.astride;
                // both groups' records are fetched together, kTf3Unroll of each per round (usually one round)
                int qa0 = ra + gs[4 * h + ((pj + 3) & 3)], qz0 = ra + gs[4 * h + ((pj + 3) & 3) + 1];
                int qa1 = ra + gs[4 * h + pj], qz1 = ra + gs[4 * h + pj + 1];
                while (qa0 < qz0 || qa1 < qz1) {
                    const int n0c = min(qz0 - qa0, kTf3Unroll), n1c = min(qz1 - qa1, kTf3Unroll);
                    int2 k0[kTf3Unroll], k1[kTf3Unroll];
                    float4 w0[kTf3Unroll], w1[kTf3Unroll];
                    float x0[kTf3Unroll], x1[kTf3Unroll];
#pragma unroll
                    for (int u = 0; u < kTf3Unroll; ++u) {
                        if (u < n0c) {
                            k0[u] = __ldg(rkey + base + qa0 + u);
                            w0[u] = __ldg(rw + base + qa0 + u);
                            x0[u] = __ldg(xr + base + qa0 + u);
                        }
                        if (u < n1c) {
                            k1[u] = __ldg(rkey + base + qa1 + u);
                            w1[u] = __ldg(rw + base + qa1 + u);
                            x1[u] = __ldg(xr + base + qa1 + u);
                        }
                    }
                    // class pj - 1: upper-row corners (record order)
#pragma unroll
                    for (int u = 0; u < kTf3Unroll; ++u) {
                        if (u >= n0c) break;
                        const int trow = (k0[u].y >> 1) & 0xfff;
                        const int gi = trow / R, ph = trow - gi * R;
                        const int g1 = min(gi + 1, P.G - 1);
                        const int pc = ph + 1 - phb;
                        arow[gi * T.pstride + pc] += w0[u].z * x0[u];
                        arow[g1 * T.pstride + pc] += w0[u].w * x0[u];
                        bound += (fabsf(w0[u].z) + fabsf(w0[u].w)) * fabsf(x0[u]);
                        glo = min(glo, gi);
                        ghi = max(ghi, g1);
                        if (k0[u].y & 1) {
                            // tau = t0 exactly: the last tap of the upper phase row lies outside
                            const float2 tl = __ldg(tab + ((size_t)gi * R + ph + 1) * S + P.Tw - 1);
                            flag_corr += x0[u] * (w0[u].z * tl.x + w0[u].w * tl.y);
                        }
                    }
                    // class pj: lower-row corners (record order)
#pragma unroll
                    for (int u = 0; u < kTf3Unroll; ++u) {
                        if (u >= n1c) break;
                        const int trow = (k1[u].y >> 1) & 0xfff;
                        const int gi = trow / R, ph = trow - gi * R;
                        const int g1 = min(gi + 1, P.G - 1);
                        const int pc = ph - phb;
                        arow[gi * T.pstride + pc] += w1[u].x * x1[u];
                        arow[g1 * T.pstride + pc] += w1[u].y * x1[u];
                        bound += (fabsf(w1[u].x) + fabsf(w1[u].y)) * fabsf(x1[u]);
                        glo = min(glo, gi);
                        ghi = max(ghi, g1);
                    }
                    qa0 += n0c;
                    qa1 += n1c;
                }
                // the half's scale: a bound of the largest |S| into [2^14, 2^15) (a power of two: exact)
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    bound = fmaxf(bound, __shfl_xor_sync(0xffffffffu, bound, o));
                    glo = min(glo, __shfl_xor_sync(0xffffffffu, glo, o));
                    ghi = max(ghi, __shfl_xor_sync(0xffffffffu, ghi, o));
                }
                if (lane == 0) {
                    wmax[warp] = bound;
                    wlo[warp] = glo;
                    whi[warp] = ghi;
                }
                __syncthreads();                     // every record of the half is in S
                int se = 0, c_lo = 0, c_hi = 16;     // a half without records multiplies one chunk of zeros
                {
                    float m = 0.0f;
                    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
                        m = fmaxf(m, wmax[w]);
                        glo = min(glo, wlo[w]);
                        ghi = max(ghi, whi[w]);
                    }
                    int ex = 0;
                    frexpf(m, &ex);
                    se = m > 0.0f ? min(15 - ex, 126) : 0;
                    // the columns of the planes reached (plane-major), widened to whole 16-column K steps:
                    // every other sum is zero and stays so
                    if (ghi >= glo) {
                        c_lo = (glo * T.pstride) & ~15;
                        c_hi = min(T.kb, ((ghi + 1) * T.pstride + 15) & ~15);
                    }
                }
                if (tid == 0) sexp[h] = se;
                const float scl = __int_as_float((se + 127) << 23);
                // this half's table operand has landed (copied during the scatter)
                if (!mbar_wait_bounded(smem_u32(bbar), bphase, status)) *abort_flag = 1;
                bphase ^= 1u;
                ++waits;
                __syncthreads();                     // uniform flag
                // chunks of kc columns: two FP16 parts of the scaled sums, then the three products; with two chunk
                // buffers a chunk is converted while the previous chunk's products run
                int pending = 0;                     // bit b: products reading buffer b not yet waited for
                for (int c0 = c_lo, q = 0; c0 < c_hi; c0 += T.kc, ++q) {
                    const int b = T.nbuf == 2 ? (q & 1) : 0;
                    if (pending & (1 << b)) {
                        if (!mbar_wait_bounded(smem_u32(smem + (b ? 40 : 0)), (phase >> b) & 1u, status))
                            *abort_flag = 1;
                        phase ^= 1u << b;
                        pending &= ~(1 << b);
                        __syncthreads();
                        if (*abort_flag) break;
                    }
                    unsigned char* sAb = sA + (size_t)b * 2 * apart;
                    const int cw = min(T.kc, c_hi - c0), kc8 = cw / 8;
                    // with two buffers warp 0 only issues the products, so they overlap the next conversion
                    const int cthr = T.nbuf == 2 ? (int)blockDim.x - 32 : (int)blockDim.x;
                    for (int c = T.nbuf == 2 ? tid - 32 : tid; c < kTfTile * kc8; c += cthr) {
                        if (c < 0) break;
                        // eight consecutive items = the eight rows of one core matrix: their 16-byte stores
                        // are contiguous and their row reads (stride astride, not a multiple of 32) hit
                        // distinct banks
                        const int i8 = c >> 3, j = i8 % kc8, i = (i8 / kc8) * 8 + (c & 7);
                        float4* sp = reinterpret_cast<float4*>(sS + i * T.astride + c0 + 8 * j);
                        const float4 v0 = sp[0], v1 = sp[1];
                        sp[0] = make_float4(0.f, 0.f, 0.f, 0.f);
                        sp[1] = make_float4(0.f, 0.f, 0.f, 0.f);
                        uint4 hv, lv;
                        split2h_pair(v0.x * scl, v0.y * scl, hv.x, lv.x);
                        split2h_pair(v0.z * scl, v0.w * scl, hv.y, lv.y);
                        split2h_pair(v1.x * scl, v1.y * scl, hv.z, lv.z);
                        split2h_pair(v1.z * scl, v1.w * scl, hv.w, lv.w);
                        const uint32_t off = kmajor_offset(i, 8 * j, T.kc);
                        *reinterpret_cast<uint4*>(sAb + off) = hv;
                        *reinterpret_cast<uint4*>(sAb + apart + off) = lv;
                    }
                    fence_async_smem();
                    __syncthreads();
                    if (tid == 0) {
                        tc_fence_after();
                        const uint32_t a0 = smem_u32(sAb), b0 = smem_u32(sB) + (uint32_t)(c0 / 8) * 128;
                        const int terms[3][2] = {{0, 0}, {0, 1}, {1, 0}};
                        for (int s = 0; s < cw / 16; ++s)
                            for (int tq = 0; tq < 3; ++tq)
                                umma_bf16(tmem + (uint32_t)(h * kTf3HalfCols),
                                          umma_desc(a0 + terms[tq][0] * apart + 256 * s, lbo, sboA),
                                          umma_desc(b0 + terms[tq][1] * bpart + 256 * s, lbo, sboB), idesc,
                                          c0 > c_lo || s > 0 || tq > 0);
                        umma_commit(smem_u32(smem + (b ? 40 : 0)));
                    }
                    pending |= 1 << b;
                }
                // every product of this half done: the table buffer and the chunk buffers are free
                for (int b = 0; b < 2; ++b)
                    if (pending & (1 << b)) {
                        if (!mbar_wait_bounded(smem_u32(smem + (b ? 40 : 0)), (phase >> b) & 1u, status))
                            *abort_flag = 1;
                        phase ^= 1u << b;
                    }
                __syncthreads();
                tc_fence_after();
                if (*abort_flag) break;
                // the table buffer is free: the other half next (or half 0 of the next tile / item)
                if (tid == 0) copy_half(1 - h);
                ++copies;
            }
            if (*abort_flag) break;
            // the four class threads of a sample are adjacent lanes: their flag corrections in class order
            {
                const float f1 = __shfl_down_sync(0xffffffffu, flag_corr, 1);
                const float f2 = __shfl_down_sync(0xffffffffu, flag_corr, 2);
                const float f3 = __shfl_down_sync(0xffffffffu, flag_corr, 3);
                if (pj == 0 && n0 < P.M) sY[n0 + P.Tw] -= ((flag_corr + f1) + f2) + f3;
            }
            // U = U_0 / (s_0 t) + U_1 / (s_1 t) (tensor memory) -> shared (over the sums), rows = n0 - ts
            {
                const int q = warp & 3, part = warp >> 2;
                const int row = q * 32 + lane;
                const int cwid = T.ntap / 4;
                const float i0 = __int_as_float((127 - sexp[0]) << 23), i1 = __int_as_float((127 - sexp[1]) << 23);
                const float it = __int_as_float((127 - T.texp) << 23);
                for (int c = part * cwid; c < part * cwid + cwid; c += 4) {
                    float v0[4], v1[4];
                    tmem_ld4(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c, v0);
                    tmem_ld4(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(kTf3HalfCols + c), v1);
#pragma unroll
                    for (int j = 0; j < 4; ++j) sS[row * T.ustride + c + j] = (v0[j] * i0) * it + (v1[j] * i1) * it;
                }
            }
            tc_fence_before();
            __syncthreads();
            // anti-diagonals: y[ts + 1 + j] += sum_i U[i][j - i]
            for (int j = tid; j < kTfTile + T.ntap - 1; j += blockDim.x) {
                float acc = 0.0f;
                const int i0 = max(0, j - T.ntap + 1), i1 = min(kTfTile - 1, j);
                for (int i = i0; i <= i1; ++i) {
                    acc += sS[i * T.ustride + j - i];
                    sS[i * T.ustride + j - i] = 0.0f;    // each product is read once: the sums are clear again
                }
                sY[ts + 1 + j] += acc;
            }
            __syncthreads();
        }
        if (*abort_flag) break;
        float* yo = V.y + (size_t)k * V.out_stride;
        for (int n = tid; n < V.out_stride; n += blockDim.x) yo[n] = n < P.M ? sY[n] : 0.0f;
        __syncthreads();
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
