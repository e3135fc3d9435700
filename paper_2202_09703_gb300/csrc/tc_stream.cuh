// A x on the tensor cores, streaming each tile's records (FP32 and BF16
// storage forms), shared by the single-request kernel (tc_fwd_stream.cu)
// and the batched engine (engine.cu).
//
// Eq. 13 with the bilinear pulse table, grouped by first tap n0: for a tile of
// 128 values of n0 of one A-scan,
//     S[n0][col] = sum over the tile's pairs of their weight on table column col times x_v,
//     U (128 x taps) = S T,   y[n0 + 1 + m] += U[n0][m],
// with columns col = plane * (Q + 1) + phase (every tap of a pair shares one
// table phase, so this regrouping is exact).
//
// Records: an A-scan's records are sorted by n0 and, within an n0, by table
// row (plane * (Q + 1) + lower phase) and pixel, so a tile's records are one
// contiguous range and records of one S cell are adjacent.  At set-up each
// tile's range is cut at n0 boundaries into 16 parts of about equal record
// count, one per warp, so no two warps add into the same row of S.  A warp
// streams its part 32 records at a time (coalesced, four loads in flight, the
// next tile's first loads issued while the current tile is multiplied), sums
// the contributions of equal (n0, table row) with a segmented warp scan, and
// the last record of each run adds its four bilinear corners into S with plain
// read-modify-writes: within one instruction the cells are distinct, the four
// corners go in four steps, and each row of S belongs to one warp.  No
// atomics: every cell's additions happen in a fixed order and every output bit
// is reproducible.
//
// The records of a tile reach a few neighbouring attenuation planes, one
// column range [c_lo, c_hi) found per tile at set-up: only that range is held,
// converted and multiplied.  S goes to tensor memory as the MMA's A operand
// (row n0 in lane n0).  FP32 form: S scaled by the power of two that brings
// the sum of the tile's absolute corner contributions (a bound of every |S|)
// below 2^15 and split into two FP16 parts, the table likewise (scale fixed
// per geometry): the three products S1 T1 + S1 T2 + S2 T1 (the dropped S2 T2
// is below 2^-22 of the result).  BF16 form: S rounded once to BF16 against
// the BF16 table, one product.  The table operand stays resident in shared
// memory.  A tile's products are read back after the next tile's records have
// been scattered, so they overlap the scatter; each warp sums the
// anti-diagonals of its 32-row x (taps / 4)-column block of U with shuffles,
// and the sixteen blocks are added per output sample in a fixed order.
#pragma once

#include "tc_apply.cuh"

namespace mbir {

#ifndef MBIR_TS_WARPS_F32
#define MBIR_TS_WARPS_F32 20
#endif
#ifndef MBIR_TS_WARPS_BF16
#define MBIR_TS_WARPS_BF16 24
#endif
// A x: warps per CTA, one part of every tile each, by storage form (512x1024 A x with 16 / 20 / 24 / 28
// warps: FP32 11.1 / 10.4 / 10.8 / 10.8 ms, BF16 10.5 / - / 9.1 / - ms)
__host__ __device__ constexpr int ts_warps(bool bf16) { return bf16 ? MBIR_TS_WARPS_BF16 : MBIR_TS_WARPS_F32; }
template <bool BF16>
struct TsShape {
    static constexpr int warps = ts_warps(BF16);
    static constexpr int threads = 32 * warps;
    static constexpr int split = warps + 1;         // record offsets per tile: the warps' part boundaries
};
constexpr int kTsEpiWarps = 16;     // A x epilogue: four warps per tensor-memory lane quarter read the product
#ifndef MBIR_TB_WARPS_F32
#define MBIR_TB_WARPS_F32 20
#endif
#ifndef MBIR_TB_WARPS_BF16
#define MBIR_TB_WARPS_BF16 20
#endif
// A^T: warps per CTA by storage form (the record pass runs on all of them, the tensor-memory work on 16;
// 512x1024 A^T with 16 / 20 / 24 warps: FP32 7.77 / 7.56 / 7.58 ms, BF16 7.14 / 7.08 / 7.11 ms)
__host__ __device__ constexpr int tb_warps(bool bf16) { return bf16 ? MBIR_TB_WARPS_BF16 : MBIR_TB_WARPS_F32; }
template <bool BF16>
struct TbShape {
    static constexpr int warps = tb_warps(BF16);
    static constexpr int threads = 32 * warps;
};
static_assert(tb_warps(false) % 4 == 0 && tb_warps(false) >= 16 && tb_warps(false) <= 28 &&
              tb_warps(true) % 4 == 0 && tb_warps(true) >= 16 && tb_warps(true) <= 28, "A^T warps: 16..28");
constexpr int kTsTile = 128;        // n0 values per tile (MMA M)
static_assert(ts_warps(false) % 4 == 0 && ts_warps(false) >= kTsEpiWarps && ts_warps(false) < 32 &&
              ts_warps(true) % 4 == 0 && ts_warps(true) >= kTsEpiWarps && ts_warps(true) < 32,
              "A x warps: 16..28, multiples of 4");
constexpr uint32_t kTsCols = 512;   // tensor memory: A operand in [0, 256), the product at 256
constexpr uint32_t kTsDCol = 256;
constexpr int kTsPart = 64;         // anti-diagonal sums per warp block (32 + taps / 4 - 1 <= 63)
constexpr int kTsYRing = 512;       // output samples held in shared memory, a ring indexed by sample mod 512
#ifndef MBIR_TS_RING
#define MBIR_TS_RING 4
#endif
#ifndef MBIR_TS_XAHEAD
#define MBIR_TS_XAHEAD 2
#endif
constexpr int kTsRing = MBIR_TS_RING;      // record batches of a warp in flight (A x)

// Variants of the two pools, chosen per geometry by timing each once at set-up (tune_tc_applies):
// A x: 0 plain read-only loads, 1 the records bypass the L1 and the gathered x is kept there (512x1024 FP32:
// 12.6 against 11.5 ms; 256x512: 0.596 against 0.605 ms); A^T: 0 four, 1 six records per thread and batch
// (512x1024: 8.5 against 8.3 ms).
constexpr int kTcVariants = 2;
template <int FV, typename T>
__device__ __forceinline__ T ld_rec(const T* p)
{
    if constexpr (FV == 1) return ldg_stream(p);
    else return __ldg(p);
}
template <int FV>
__device__ __forceinline__ float ld_x(const float* p)
{
    if constexpr (FV == 1) return ldg_keep(p);
    else return __ldg(p);
}
// batches between an x gather and its use (< kTsRing): with 20 and 24 warps per CTA two batches took the
// 512x1024 A x from 10.35 to 9.04 ms (FP32) and from 9.12 to 8.21 ms (BF16); with 16 warps one was better
constexpr int kTsXAhead = MBIR_TS_XAHEAD;
static_assert(kTsXAhead >= 1 && kTsXAhead < kTsRing, "x is gathered from records already in the ring");

struct TsView {
    GeomParams P;
    Tf4Layout T;
    const uint4* bop;            // table operand image
    const void* tab;             // kernel table, float2 (FP32) or __nv_bfloat162 (BF16): the tau = t0 tap
    const long long* rec_off;
    const uint32_t* crange;      // per (A-scan, tile): c_lo | c_hi << 16
    const int* split;            // per (A-scan, tile): warps + 1 record offsets from the A-scan's first record
    const uint2* rkey;           // packed records (tc_apply.cuh): keys
    const void* rw;              // and weights, uint2 (FP32 form) or uint32 (BF16 form)
    const int* order;            // A-scans by decreasing record count
    const float* x;
    void* y;                     // float, or __nv_bfloat16 when y_bf16; row stride out_stride
    int y_bf16;
    int out_stride;
    int* counter;
};

__device__ __forceinline__ float ts_pow2(int e) { return __int_as_float((e + 127) << 23); }

// Power-of-two exponent that brings a bound m below 2^15 (0 for m = 0).
__device__ __forceinline__ int ts_bound_exponent(float m)
{
    if (!(m > 0.0f)) return 0;
    int ex = 0;
    frexpf(m, &ex);
    return min(15 - ex, 126);
}

// Drains the A x items (A-scans, largest first) of V.  The shared-memory
// header (offset 0: MMA barrier, 8: tensor-memory address, 16: item slot, 20:
// abort flag, 32: table copy barrier) is initialised and kTsCols columns of
// tensor memory are allocated by the caller; mphase / bphase are the parities
// of the two barriers.  Returns false when a bounded wait gave up.
template <bool BF16, int FV>
__device__ __forceinline__ bool tcs_forward_pool(const TsView& V, unsigned char* smem, uint32_t tmem,
                                                 uint32_t& mphase, uint32_t& bphase, int* status)
{
    constexpr int kTsWarps = TsShape<BF16>::warps;
    constexpr int kTsSplit = TsShape<BF16>::split;
    const GeomParams& P = V.P;
    const Tf4Layout& T = V.T;
    const int ntile = (P.M + kTsTile - 1) / kTsTile;
    volatile int* next = reinterpret_cast<volatile int*>(smem + 16);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + 20);
    float* wsum = reinterpret_cast<float*>(smem + 64);
    int* tsp = reinterpret_cast<int*>(smem + T.off_rs);             // this A-scan's part boundaries
    uint32_t* tcr = reinterpret_cast<uint32_t*>(tsp + ntile * kTsSplit);
    float* part = reinterpret_cast<float*>(smem + T.off_part);
    unsigned char* sB = smem + T.off_b;
    float* sS = reinterpret_cast<float*>(smem + T.off_s);
    float* sY = reinterpret_cast<float*>(smem + T.off_y);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    using WT = typename TcW<BF16>::type;
    const int R = T.R, S = table_stride(P.Tw4);
    const int dR = P.G > 1 ? R : 0;                    // columns from a table row to the next plane's
    const uint2* __restrict__ rkey = V.rkey;
    const WT* __restrict__ rw = reinterpret_cast<const WT*>(V.rw);
    const float* __restrict__ xg = V.x;
    const uint32_t tA = tmem, tD = tmem + kTsDCol;
    const int KA = T.kwmax / 2;                        // tensor-memory columns of one part of A
    const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
    const uint32_t full = 0xffffffffu;

    // the table operand; S cleared (a previous pool may have used another row stride)
    if (tid == 0) {
        mbar_arrive_expect_tx(smem_u32(smem + 32), (uint32_t)T.bbytes);
        bulk_g2s(smem_u32(sB), V.bop, (uint32_t)T.bbytes, smem_u32(smem + 32));
    }
    for (int i = tid; i < kTsTile * T.astride; i += blockDim.x) sS[i] = 0.0f;
    if (!mbar_wait_bounded(smem_u32(smem + 32), bphase, status)) *abort_flag = 1;
    bphase ^= 1u;
    __syncthreads();

    const uint32_t idesc = BF16 ? umma_idesc_bf16(kTsTile, T.ntap) : umma_idesc_f16(kTsTile, T.ntap);
    const uint32_t bpart = (uint32_t)(T.ntap * T.kb * 2), sboB = (uint32_t)(T.kb / 8) * 128;
    const int cq = T.ntap / 4;                          // columns of a warp's block of U
    const int qd = warp & 3, pb = warp >> 2;            // lane quarter and column block of this warp
    const float it = ts_pow2(-T.texp);

    // record batches in flight: slot s holds batch b = s (mod kTsRing) of this warp's part of the tile
    uint2 kq[kTsRing];
    WT wq[kTsRing];
    float xq[kTsRing];

    // Products of tile tp (scale exponent se) in tensor memory -> y: wait for them, sum the anti-diagonals of
    // each warp's block with shuffles (lane l: block offsets l and l + 32), then the blocks in a fixed order.
    auto epilogue = [&](int tp, int se) {
        if (!mbar_wait_bounded(smem_u32(smem), mphase, status)) *abort_flag = 1;
        mphase ^= 1u;
        tc_fence_after();
        const float i0 = ts_pow2(-se);
        if (warp < kTsEpiWarps) {
            float lo = 0.0f, hi = 0.0f;
            for (int c = 0; c < cq; c += 4) {
                float v[4];
                tmem_ld4(tD + lane_base + (uint32_t)(pb * cq + c), v);
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int d = c + j;                              // column within the block
                    const float u = __shfl_sync(full, (v[j] * i0) * it, (lane - d) & 31);
                    if (lane >= d) lo += u;
                    else hi += u;
                }
            }
            part[warp * kTsPart + lane] = lo;
            part[warp * kTsPart + 32 + lane] = hi;
        }
        tc_fence_before();
        __syncthreads();
        for (int o = tid; o < kTsTile + T.ntap - 1; o += blockDim.x) {
            float acc = 0.0f;
            for (int w = 0; w < kTsEpiWarps; ++w) {
                const int r = o - ((w & 3) * 32 + (w >> 2) * cq);
                if (r >= 0 && r < 32 + cq - 1) acc += part[w * kTsPart + r];
            }
            sY[(tp * kTsTile + 1 + o) & (kTsYRing - 1)] += acc;
        }
    };
    // Output samples [flushed, upto) are final: written to y and their ring slots cleared.  Every sample not
    // yet flushed lies in [clo, clo + 383] (a tile's products reach 127 + taps samples past its start, the
    // tau = t0 taps of the next tile 255 + Tw), so a ring of 512 holds them without overlap; samples outside
    // that range are zero.
    size_t yrow = 0;                                    // this A-scan's first output element
    int flushed = 0;
    auto flush = [&](int upto, int clo) {
        const int hi = min(upto, V.out_stride);
        for (int n = flushed + tid; n < hi; n += blockDim.x) {
            float v = 0.0f;
            if (n >= clo && n < clo + kTsYRing) {
                v = sY[n & (kTsYRing - 1)];
                sY[n & (kTsYRing - 1)] = 0.0f;
            }
            if (n >= P.M) v = 0.0f;
            if (V.y_bf16) reinterpret_cast<__nv_bfloat16*>(V.y)[yrow + n] = __float2bfloat16_rn(v);
            else reinterpret_cast<float*>(V.y)[yrow + n] = v;
        }
        flushed = max(flushed, upto);
    };

    while (!*abort_flag) {
        if (tid == 0) *next = atomicAdd(V.counter, 1);
        __syncthreads();
        const int idx = *next;
        if (idx >= P.K) break;
        const int k = __ldg(V.order + idx);
        const long long base = __ldg(V.rec_off + k);
        {
            const int* sp = V.split + (size_t)k * ntile * kTsSplit;
            const uint32_t* cr = V.crange + (size_t)k * ntile;
            for (int i = tid; i < ntile * kTsSplit; i += blockDim.x) tsp[i] = __ldg(sp + i);
            for (int i = tid; i < ntile; i += blockDim.x) tcr[i] = __ldg(cr + i);
            for (int i = tid; i < kTsYRing; i += blockDim.x) sY[i] = 0.0f;
        }
        yrow = (size_t)k * V.out_stride;
        flushed = 0;
        __syncthreads();

        // this warp's part [wa, wb) of tile t's records and its batches of 32
        int wa = 0, wb = 0, nb = 0;
        auto warp_range = [&](int t) {
            wa = tsp[t * kTsSplit + warp];
            wb = tsp[t * kTsSplit + warp + 1];
            nb = (wb - wa + 31) >> 5;
        };
        auto issue = [&](uint2& kk, WT& ww, int b) {
            const int rec = wa + 32 * b + lane;
            if (b < nb && rec < wb) {
                kk = ld_rec<FV>(rkey + base + rec);
                ww = ld_rec<FV>(rw + base + rec);
            } else {
                kk = make_uint2(0u, kTcNone);            // not a record: weight zero
                ww = WT{};
            }
        };
        warp_range(0);
#pragma unroll
        for (int s = 0; s < kTsRing; ++s) issue(kq[s], wq[s], s);

        int pend = -1, pend_se = 0;                      // tile whose products wait in tensor memory
        for (int t = 0; t < ntile; ++t) {
            const int ts = t * kTsTile;
            const bool live = tsp[t * kTsSplit + kTsWarps] > tsp[t * kTsSplit];
            if (t + 1 < ntile) {
                // this warp's part of the next tile into L2 while this tile is scattered
                const int pa = tsp[(t + 1) * kTsSplit + warp], pz = tsp[(t + 1) * kTsSplit + warp + 1];
                prefetch_l2_range(rkey + base + pa, (size_t)(pz - pa) * sizeof(int2), lane);
                prefetch_l2_range(rw + base + pa, (size_t)(pz - pa) * sizeof(WT), lane);
            }
            if (live && pend >= 0 && t > pend + 1) {
                // tiles without records lie between the pending tile and this one: finish the pending tile and
                // flush every sample before this tile's first, so that this tile's writes cannot meet older
                // samples in the ring
                __syncthreads();
                epilogue(pend, pend_se);
                __syncthreads();
                flush(t * kTsTile + 1, pend * kTsTile + 1);
                __syncthreads();
                pend = -1;
                if (*abort_flag) break;
            }
            if (live) {
                // ---- scatter: batches b = 0 .. nb-1, slot b mod kTsRing
                float* Sb = sS - (int)(tcr[t] & 0xffffu);
                float bsum = 0.0f;
                // x gathered kTsXAhead batches ahead of its use, the records kTsRing batches ahead
#pragma unroll
                for (int s = 0; s < kTsXAhead; ++s)
                    xq[s] = kq[s].y != kTcNone ? ld_x<FV>(xg + (kq[s].x & kTcPixelMask)) : 0.0f;
                for (int b0 = 0; b0 < nb; b0 += kTsRing) {
#pragma unroll
                    for (int u = 0; u < kTsRing; ++u) {
                        const int b = b0 + u;
                        if (b >= nb) break;
                        if (b + kTsXAhead < nb) {
                            const int sn = (u + kTsXAhead) % kTsRing;
                            xq[sn] = kq[sn].y != kTcNone ? ld_x<FV>(xg + (kq[sn].x & kTcPixelMask)) : 0.0f;
                        }
                        const uint2 kk = kq[u];
                        const bool valid = kk.y != kTcNone;
                        const int n0r = valid ? tc_rec_n0(kk) - ts : 0;
                        const int trow = valid ? tc_rec_row(kk) : 0;
                        // the four bilinear corners times x (zero for a lane without a record)
                        const float wx = tc_rec_w(wq[u]) * xq[u], psi = tc_rec_psi(wq[u]);
                        const float ca = wx * tc_rec_fa(kk), cb = wx - ca;
                        float c1 = ca * psi, c3 = cb * psi;
                        float c0 = ca - c1, c2 = cb - c3;
                        bsum += fabsf(wx);                       // the corners' magnitudes sum to |w x|
                        const int c1col = trow + dR;
                        float* row = Sb + n0r * T.astride;
                        // a marked batch (first record's key.x with bit 31 set): every corner cell is its lane's
                        // alone, so the four read-modify-writes are independent (with one attenuation plane the
                        // two pairs of equal cells are merged first)
                        const bool one_step = (int)__shfl_sync(full, kk.x, 0) < 0;
                        if (one_step) {
                            if (valid) {
                                if (dR == 0) {
                                    row[trow] += c0 + c1;
                                    row[trow + 1] += c2 + c3;
                                } else {
                                    const float s0 = row[trow], s2 = row[trow + 1];
                                    const float s1 = row[c1col], s3 = row[c1col + 1];
                                    row[trow] = s0 + c0;
                                    row[trow + 1] = s2 + c2;
                                    row[c1col] = s1 + c1;
                                    row[c1col + 1] = s3 + c3;
                                }
                            }
                            __syncwarp();
                        } else {
                        // equal (n0, table row) are adjacent lanes: segmented inclusive sums over them (one_step
                        // is the same for the whole warp, so every lane takes part in every shuffle)
                        const int key = valid ? (n0r << 12) | trow : 0x40000000 + lane;
                        const int kup = __shfl_up_sync(full, key, 1);
                        const int kdn = __shfl_down_sync(full, key, 1);
                        if (__any_sync(full, lane > 0 && kup == key)) {
                            // Hillis-Steele steps until no run reaches further back (runs are short)
                            for (int d = 1; d < 32; d <<= 1) {
                                const int kd = __shfl_up_sync(full, key, d);
                                const float a0 = __shfl_up_sync(full, c0, d), a1 = __shfl_up_sync(full, c1, d);
                                const float a2 = __shfl_up_sync(full, c2, d), a3 = __shfl_up_sync(full, c3, d);
                                if (lane >= d && kd == key) {
                                    c0 += a0;
                                    c1 += a1;
                                    c2 += a2;
                                    c3 += a3;
                                }
                                const int k2 = __shfl_up_sync(full, key, min(2 * d, 31));
                                if (!__any_sync(full, lane >= 2 * d && k2 == key)) break;
                            }
                        }
                        // the last record of each run adds its corners, one corner per step: within a step the
                        // writers' cells are distinct and the rows belong to this warp alone
                        const bool writer = valid && (lane == 31 || kdn != key);
                        if (writer) row[trow] += c0;
                        __syncwarp();
                        if (writer) row[c1col] += c1;
                        __syncwarp();
                        if (writer) row[trow + 1] += c2;
                        __syncwarp();
                        if (writer) row[c1col + 1] += c3;
                        __syncwarp();
                        }
                        // tau = t0 exactly (rare): the last tap of the upper phase row lies outside the window;
                        // one lane after another
                        uint32_t fm = __ballot_sync(full, valid && (kk.y & kTcFlag0));
                        while (fm) {
                            if (lane == __ffs(fm) - 1) {
                                const size_t ti = (size_t)(trow + 1) * S + P.Tw - 1;
                                float2 tl;
                                if (BF16) tl = __bfloat1622float2(__ldg(reinterpret_cast<const __nv_bfloat162*>(V.tab) + ti));
                                else tl = __ldg(reinterpret_cast<const float2*>(V.tab) + ti);
                                sY[(ts + n0r + P.Tw) & (kTsYRing - 1)] -= cb * fmaf(psi, tl.y - tl.x, tl.x);
                            }
                            __syncwarp();
                            fm &= fm - 1;
                        }
                        issue(kq[u], wq[u], b + kTsRing);
                    }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) bsum += __shfl_xor_sync(full, bsum, o);
                if (lane == 0) wsum[warp] = bsum;
            }
            // the next tile's first batches load while this tile is converted and multiplied
            if (t + 1 < ntile) {
                warp_range(t + 1);
#pragma unroll
                for (int s = 0; s < kTsRing; ++s) issue(kq[s], wq[s], s);
            }
            if (!live) continue;
            __syncthreads();                             // every record of the tile is in S
            // ---- the previous tile's products -> y (they ran during this tile's scatter); the samples before
            // this tile's first are then final
            if (pend >= 0) {
                epilogue(pend, pend_se);
                __syncthreads();
                flush((pend + 1) * kTsTile + 1, pend * kTsTile + 1);
            }
            if (*abort_flag) break;
            // ---- S -> A operand in tensor memory, S cleared as read
            int se = 0;
            if (!BF16) {
                float tb = 0.0f;
                for (int w = 0; w < kTsWarps; ++w) tb += wsum[w];
                se = ts_bound_exponent(tb);
            }
            const float scl = ts_pow2(se);
            const uint32_t crt = tcr[t];
            const int c_lo = (int)(crt & 0xffffu), kw = (int)(crt >> 16) - c_lo;
            {
                float* srow = sS + (qd * 32 + lane) * T.astride;
                for (int g8 = pb; g8 < kw / 8; g8 += kTsWarps / 4) {
                    float4* sp = reinterpret_cast<float4*>(srow + 8 * g8);
                    const float4 v0 = sp[0], v1 = sp[1];
                    sp[0] = make_float4(0.f, 0.f, 0.f, 0.f);
                    sp[1] = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (BF16) {
                        const __nv_bfloat162 p0 = __floats2bfloat162_rn(v0.x, v0.y), p1 = __floats2bfloat162_rn(v0.z, v0.w);
                        const __nv_bfloat162 p2 = __floats2bfloat162_rn(v1.x, v1.y), p3 = __floats2bfloat162_rn(v1.z, v1.w);
                        const uint4 hv = make_uint4(*reinterpret_cast<const uint32_t*>(&p0),
                                                    *reinterpret_cast<const uint32_t*>(&p1),
                                                    *reinterpret_cast<const uint32_t*>(&p2),
                                                    *reinterpret_cast<const uint32_t*>(&p3));
                        tmem_st4(tA + lane_base + (uint32_t)(4 * g8), hv);
                    } else {
                        uint4 hv, lv;
                        split2h_pair(v0.x * scl, v0.y * scl, hv.x, lv.x);
                        split2h_pair(v0.z * scl, v0.w * scl, hv.y, lv.y);
                        split2h_pair(v1.x * scl, v1.y * scl, hv.z, lv.z);
                        split2h_pair(v1.z * scl, v1.w * scl, hv.w, lv.w);
                        tmem_st4(tA + lane_base + (uint32_t)(4 * g8), hv);
                        tmem_st4(tA + lane_base + (uint32_t)(KA + 4 * g8), lv);
                    }
                }
                tmem_wait_st();
            }
            tc_fence_before();
            __syncthreads();
            if (tid == 0) {
                tc_fence_after();
                const uint32_t b0 = smem_u32(sB) + (uint32_t)(c_lo / 8) * 128;
                for (int s = 0; s < kw / 16; ++s) {
                    umma_f16_ta(tD, tA + 8 * s, umma_desc(b0 + 256 * s, 128, sboB), idesc, s > 0);
                    if (!BF16) {
                        // hi x lo, lo x hi
                        umma_f16_ta(tD, tA + 8 * s, umma_desc(b0 + bpart + 256 * s, 128, sboB), idesc, true);
                        umma_f16_ta(tD, tA + KA + 8 * s, umma_desc(b0 + 256 * s, 128, sboB), idesc, true);
                    }
                }
                umma_commit(smem_u32(smem));
            }
            pend = t;
            pend_se = se;
        }
        if (pend >= 0 && !*abort_flag) epilogue(pend, pend_se);
        __syncthreads();
        if (*abort_flag) break;
        flush(V.out_stride, pend >= 0 ? pend * kTsTile + 1 : V.out_stride);
        __syncthreads();
    }
    return !*abort_flag;
}

// ---------------------------------------------------------------------------
// A^T r on the tensor cores (adjoint of eq. 13): per item (A-scan, tile of 128
// first-tap samples n0), every tap of a pair shares one table phase, so
//     C[n0][row] = sum_m e[n0 + 1 + m] T[row][m]
// is one matrix product of the residual's Hankel tile H[n][m] = e[ts + 1 + n + m]
// (128 x taps, in tensor memory as the A operand) and the table rows the tile's
// records reach (one column range, the B operand resident in shared memory);
// each record then combines four values of C with its bilinear weights (less
// the tau = t0 tap of flagged records) into one contribution v and adds it to
// its pixel's 64-bit fixed-point accumulator: round(v 2^s) by an integer atomic
// (one scale 2^s per apply, tc_fixed_exponent), so the sum is exact and its
// value does not depend on the order of the additions; a last kernel turns the
// sums into FP32 (tcs_finish_pixel).  FP32 form: the window scaled by the power
// of two that brings its largest magnitude into [2^14, 2^15) and split into two
// FP16 parts, the table likewise: three products.  BF16 form: the stored BF16
// residual and table, one product.  The products of the next item run while the
// current item's records are processed.
struct TbView {
    GeomParams P;
    Tb4Layout T;
    const uint4* bop;            // table operand image
    const void* tab;             // kernel table, float2 (FP32) or __nv_bfloat162 (BF16): the tau = t0 tap
    const void* e;               // residual K x Mp: float (FP32) or __nv_bfloat16 (BF16), zero tail
    const long long* rec_off;
    const int* tile_off;         // first record of every tile, K x (ntile + 1)
    const uint32_t* crange;      // per (A-scan, tile): c_lo | c_hi << 16
    const uint2* rkey;           // packed records (tc_apply.cuh): keys
    const void* rw;              // and weights, uint2 (FP32 form) or uint32 (BF16 form)
    unsigned long long* acc;     // per pixel: the fixed-point sum (zero on entry)
    const unsigned int* emax;    // bits of max |e| over the residual (tc_emax)
    float bound;                 // K x max record weight x (max table row sum of |T| + max |T|), doubled
    int* counter;
};

// records per thread in one batch of the A^T pool (two batches in flight), per variant
template <int BV> struct TbUnroll { static constexpr int value = BV == 1 ? 6 : 4; };

// Scale exponent s of the adjoint's fixed-point sums: every contribution is at most bound / K x max|e| in
// magnitude and a pixel has at most one per A-scan, so with s = 61 - (exponents of bound and max|e|) no
// partial sum reaches 2^61.  Clamped to [-126, 126] (2^s and 2^-s normal floats); 0 for a zero residual.
__device__ __forceinline__ int tc_fixed_exponent(unsigned int emax_bits, float bound)
{
    const float em = __uint_as_float(emax_bits);
    if (!(em > 0.0f) || !(em <= 3.4e38f)) return 0;
    int e1 = 0, e2 = 0;
    frexpf(em, &e1);
    frexpf(bound, &e2);
    return min(max(61 - e1 - e2, -126), 126);
}

// b[v] from its fixed-point sum (one rounding to FP32); NaN when the residual held a non-finite value.
__device__ __forceinline__ float tcs_finish_pixel(unsigned long long a, unsigned int emax_bits, float bound)
{
    if (emax_bits >= 0x7f800000u) return __uint_as_float(0x7fc00000u);
    return __ll2float_rn((long long)a) * ts_pow2(-tc_fixed_exponent(emax_bits, bound));
}

// A batch of records held in registers: records rb + u * NT + tid, u < U (NT threads per CTA).
template <int U, typename WT>
struct TbBatch {
    uint2 key[U];
    WT w[U];
};

template <int NT, int U, typename WT>
__device__ __forceinline__ void tb_load(TbBatch<U, WT>& b, const uint2* __restrict__ rkey, const WT* __restrict__ rw,
                                        long long base, int rb, int r1, int tid)
{
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const int r = rb + u * NT + tid;
        if (r < r1) {
            b.key[u] = __ldg(rkey + base + r);
            b.w[u] = __ldg(rw + base + r);
        }
    }
}

// Drains the A^T items of V (header as for tcs_forward_pool; kTsCols tensor-memory columns).
template <bool BF16, int BV, int U = TbUnroll<BV>::value>
__device__ __forceinline__ bool tcs_adjoint_pool(const TbView& V, unsigned char* smem, uint32_t tmem,
                                                 uint32_t& mphase, uint32_t& bphase, int* status)
{
    constexpr int NWB = TbShape<BF16>::warps, NTB = TbShape<BF16>::threads;
    const GeomParams& P = V.P;
    const Tb4Layout& T = V.T;
    const int ntile = (P.M + kTsTile - 1) / kTsTile;
    const int nitems = P.K * ntile;
    volatile int* next = reinterpret_cast<volatile int*>(smem + 16);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + 20);
    float* wmax = reinterpret_cast<float*>(smem + 64);
    float* sE0 = reinterpret_cast<float*>(smem + T.off_e);
    unsigned char* sB = smem + T.off_b;
    float* sC = reinterpret_cast<float*>(smem + T.off_c);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    using WT = typename TcW<BF16>::type;
    const int R = T.R, S = table_stride(P.Tw4);
    const int dR = P.G > 1 ? R : 0;                    // columns from a table row to the next plane's
    const uint2* __restrict__ rkey = V.rkey;
    const WT* __restrict__ rw = reinterpret_cast<const WT*>(V.rw);
    unsigned long long* __restrict__ acc = V.acc;
    const float fsc = ts_pow2(tc_fixed_exponent(*V.emax, V.bound));
    const uint32_t tA = tmem, tD = tmem + 128;
    const int HA = T.ntap / 2;                          // tensor-memory columns of one part of H
    const int qd = warp & 3, pb = warp >> 2;
    const int cq = T.ntap / 4;                          // taps of H converted per thread
    const uint32_t lane_base = (uint32_t)(qd * 32) << 16;
    const uint32_t full = 0xffffffffu;
    const int W = kTsTile + T.ntap;                     // window samples e[ts + 1 .. ts + W]
    const uint32_t sboB = (uint32_t)(T.ntap / 8) * 128, bpart = (uint32_t)(T.kb * T.ntap * 2);
    const float it = ts_pow2(-T.texp);

    if (tid == 0) {
        mbar_arrive_expect_tx(smem_u32(smem + 32), (uint32_t)T.bbytes);
        bulk_g2s(smem_u32(sB), V.bop, (uint32_t)T.bbytes, smem_u32(smem + 32));
        *next = atomicAdd(V.counter, 1);
    }
    if (!mbar_wait_bounded(smem_u32(smem + 32), bphase, status)) *abort_flag = 1;
    bphase ^= 1u;
    __syncthreads();

    auto load_e = [&](int item) -> float {
        const int k = item / ntile, t = item - k * ntile;
        const int n = t * kTsTile + 1 + tid;
        if (tid >= W || n >= P.Mp) return 0.0f;
        if (BF16) return __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(V.e)[(size_t)k * P.Mp + n]);
        return reinterpret_cast<const float*>(V.e)[(size_t)k * P.Mp + n];
    };
    // the window of an item: staged, its warps' maxima published (the scale needs a barrier)
    auto stage = [&](float ew, float* sE) {
        if (tid < W) sE[tid] = ew;
        float mx = fabsf(ew);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(full, mx, o));
        if (lane == 0) wmax[warp] = mx;
    };
    auto window_exponent = [&]() -> int {
        if (BF16) return 0;
        float m = 0.0f;
        for (int w = 0; w < NWB; ++w) m = fmaxf(m, wmax[w]);
        return ts_bound_exponent(m);
    };
    // H of an item into tensor memory: row n (lane), taps [pb cq, pb cq + cq), H[n][m] = 2^se e[ts + 1 + n + m]
    auto convert_h = [&](const float* sE, int se) {
        const float scl = ts_pow2(se);
        const int n = qd * 32 + lane;
        for (int m = pb * cq; m < pb * cq + cq && warp < 16; m += 4) {
            const float a0 = sE[n + m] * scl, a1 = sE[n + m + 1] * scl, a2 = sE[n + m + 2] * scl,
                        a3 = sE[n + m + 3] * scl;
            if (BF16) {
                const __nv_bfloat162 p0 = __floats2bfloat162_rn(a0, a1), p1 = __floats2bfloat162_rn(a2, a3);
                tmem_st2(tA + lane_base + (uint32_t)(m / 2), *reinterpret_cast<const uint32_t*>(&p0),
                         *reinterpret_cast<const uint32_t*>(&p1));
            } else {
                uint32_t h0, l0, h1, l1;
                split2h_pair(a0, a1, h0, l0);
                split2h_pair(a2, a3, h1, l1);
                tmem_st2(tA + lane_base + (uint32_t)(m / 2), h0, h1);
                tmem_st2(tA + lane_base + (uint32_t)(HA + m / 2), l0, l1);
            }
        }
        tmem_wait_st();
    };
    auto crange_of = [&](int item) -> uint32_t { return __ldg(V.crange + item); };
    auto issue_mma = [&](int item) {
        const uint32_t cr = crange_of(item);
        const int c_lo = (int)(cr & 0xffffu), kw = (int)(cr >> 16) - c_lo;
        tc_fence_after();
        const uint32_t idesc = BF16 ? umma_idesc_bf16(kTsTile, kw) : umma_idesc_f16(kTsTile, kw);
        const uint32_t b0 = smem_u32(sB) + (uint32_t)(c_lo / 8) * sboB;
        for (int s = 0; s < T.ntap / 16; ++s) {
            umma_f16_ta(tD, tA + 8 * s, umma_desc(b0 + 256 * s, 128, sboB), idesc, s > 0);
            if (!BF16) {
                umma_f16_ta(tD, tA + 8 * s, umma_desc(b0 + bpart + 256 * s, 128, sboB), idesc, true);
                umma_f16_ta(tD, tA + HA + 8 * s, umma_desc(b0 + 256 * s, 128, sboB), idesc, true);
            }
        }
        umma_commit(smem_u32(smem));
    };

    int cur = *next;
    if (cur >= nitems) return !*abort_flag;
    // first item: window, scale, H, products
    int cbuf = 0;
    stage(load_e(cur), sE0);
    __syncthreads();
    if (tid == 0) *next = atomicAdd(V.counter, 1);
    int cse = window_exponent();
    uint32_t live_cur = crange_of(cur);                  // a tile without records has an empty range
    if (live_cur) convert_h(sE0, cse);
    tc_fence_before();
    __syncthreads();
    int nxt = *next;
    if (tid == 0 && live_cur) issue_mma(cur);
    while (!*abort_flag) {
        const int kc = cur / ntile, tc = cur - kc * ntile;
        const long long base = __ldg(V.rec_off + kc);
        const int r0 = __ldg(V.tile_off + (size_t)kc * (ntile + 1) + tc);
        const int r1 = __ldg(V.tile_off + (size_t)kc * (ntile + 1) + tc + 1);
        // the first records of this item and the next item's window load during the products
        TbBatch<U, WT> ba, bb;
        tb_load<NTB>(ba, rkey, rw, base, r0, r1, tid);
        const float ew = nxt < nitems ? load_e(nxt) : 0.0f;
        float* sEc = sE0 + cbuf * T.ewin;
        float* sEn = sE0 + (cbuf ^ 1) * T.ewin;
        // ---- C of the current item -> shared memory (scaled back)
        const int c_lo = (int)(live_cur & 0xffffu), kw = (int)(live_cur >> 16) - c_lo;
        if (live_cur) {
            if (!mbar_wait_bounded(smem_u32(smem), mphase, status)) *abort_flag = 1;
            mphase ^= 1u;
            tc_fence_after();
            const float i0 = ts_pow2(-cse);
            const int cw = kw / 4, row = qd * 32 + lane;
            float* crow = sC + row * T.cstride;
            for (int c = pb * cw; c < pb * cw + cw && warp < 16; c += 4) {
                float v[4];
                tmem_ld4(tD + lane_base + (uint32_t)c, v);
                *reinterpret_cast<float4*>(crow + c) =
                    make_float4((v[0] * i0) * it, (v[1] * i0) * it, (v[2] * i0) * it, (v[3] * i0) * it);
            }
        }
        if (nxt < nitems) stage(ew, sEn);
        tc_fence_before();
        __syncthreads();                                  // C ready; the next window staged
        if (tid == 0) *next = atomicAdd(V.counter, 1);
        // ---- the next item's H and products, issued before this item's records
        int nse = 0;
        uint32_t live_nxt = 0;
        if (nxt < nitems) {
            nse = window_exponent();
            live_nxt = crange_of(nxt);
            if (live_nxt) convert_h(sEn, nse);
        }
        tc_fence_before();
        __syncthreads();                                  // H of the next item in tensor memory
        const int nn = *next;
        if (tid == 0 && live_nxt) issue_mma(nxt);
        // ---- the current item's records: four values of C each, one fixed-point addition per record; the
        // next batch loads while one is combined
        if (live_cur) {
            const int ts = tc * kTsTile;
            const float* Cb = sC - c_lo;
            auto run = [&](const TbBatch<U, WT>& bt, int rb) {
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int r = rb + u * NTB + tid;
                    if (r >= r1) continue;
                    const uint2 kk = bt.key[u];
                    const int n0r = tc_rec_n0(kk) - ts, trow = tc_rec_row(kk);
                    const float* cr = Cb + n0r * T.cstride;
                    const float fa = tc_rec_fa(kk), psi = tc_rec_psi(bt.w[u]);
                    // bilinear in the attenuation plane (psi), then in the phase (fa)
                    const float c00 = cr[trow], c10 = cr[trow + dR], c01 = cr[trow + 1], c11 = cr[trow + dR + 1];
                    const float a0 = fmaf(psi, c10 - c00, c00), a1 = fmaf(psi, c11 - c01, c01);
                    float v = fmaf(fa, a0 - a1, a1);
                    if (kk.y & kTcFlag0) {
                        // tau = t0 exactly: the last tap of the upper phase row lies outside the window
                        const size_t ti = (size_t)(trow + 1) * S + P.Tw - 1;
                        float2 tl;
                        if (BF16) tl = __bfloat1622float2(__ldg(reinterpret_cast<const __nv_bfloat162*>(V.tab) + ti));
                        else tl = __ldg(reinterpret_cast<const float2*>(V.tab) + ti);
                        v -= (1.0f - fa) * fmaf(psi, tl.y - tl.x, tl.x) * sEc[n0r + P.Tw - 1];
                    }
                    v *= tc_rec_w(bt.w[u]);
                    red_add_global_u64(acc + (kk.x & kTcPixelMask), (unsigned long long)__float2ll_rn(v * fsc));
                }
            };
            constexpr int kStep = U * NTB;
            for (int rb = r0; rb < r1; rb += 2 * kStep) {
                if (rb + kStep < r1) tb_load<NTB>(bb, rkey, rw, base, rb + kStep, r1, tid);
                run(ba, rb);
                if (rb + kStep >= r1) break;
                if (rb + 2 * kStep < r1) tb_load<NTB>(ba, rkey, rw, base, rb + 2 * kStep, r1, tid);
                run(bb, rb + kStep);
            }
        }
        __syncthreads();                                  // C and this window are free
        if (nxt >= nitems) break;
        cur = nxt;
        nxt = nn;
        cbuf ^= 1;
        cse = nse;
        live_cur = live_nxt;
    }
    return !*abort_flag;
}

}  // namespace mbir
