// Device building blocks of the apply kernels, shared by the single-request
// kernels and the batched engine's grouped kernels.
#pragma once

#include "device_common.cuh"

namespace mbir {

constexpr int kRecShift = 13;                     // record key: n0 << 13 | table row << 1 | flag0
constexpr int kRecPixel = 0x7fffffff;             // record pixel field: pixel index (bit 31: a batch mark of the
                                                  // tensor-core A x, set at its set-up)

// The pair of A-scan k and pixel v in TAB mode (legs from the table, eq. 4-6 and 12): true when it is
// active, i.e. its weight is non-zero and its first tap n0 + 1 lies inside the record.
__device__ __forceinline__ bool tab_pair(const GeomParams& P, const DevPtrs& D, int k, int v, Pair& pr)
{
    const int row = v / P.W, col = v - row * P.W;
    const RowInfo ri = load_row(D.rows, row);
    if (!(ri.tvert < (float)(P.M - 1))) return false;
    const int i = k / P.n_rx;
    const Leg tx = get_leg<1, kModeTAB>(P, D, ri, row, col, __ldg(D.txpos + i));
    const Leg rx = get_leg<1, kModeTAB>(P, D, ri, row, col, __ldg(D.rxpos + k));
    pr = make_pair(P, tx, rx, ri.tau);
    return pr.w != 0.0f && pr.n0 >= 0 && pr.n0 + 1 < P.M;
}

// Copies a pulse table (tab_bytes, a multiple of 16) into shared memory.
__device__ __forceinline__ void load_table_smem(void* dst, const void* src, size_t tab_bytes, int tid, int nthreads)
{
    const int4* s = reinterpret_cast<const int4*>(src);
    int4* d = reinterpret_cast<int4*>(dst);
    const int n16 = (int)(tab_bytes / 16);
    for (int t = tid; t < n16; t += nthreads) d[t] = __ldg(s + t);
}

// One pair of A^T r: the taps of the pair against a residual row in shared
// memory (ev points at sample n0 + 1), weighted by the bilinear corners of
// the table.  Returns the pair's contribution w * sum_m H(m) e[n0 + 1 + m].
template <bool BF16>
__device__ __forceinline__ float pair_taps(const typename TabT<BF16>::type* __restrict__ A, int S, int Tw, int Tw4,
                                           const typename ET<BF16>::type* __restrict__ ev, const Pair& pr)
{
    float2 sa = make_float2(0.f, 0.f), sb = make_float2(0.f, 0.f);
    const typename TabT<BF16>::type* B = A + S;
    for (int m = 0; m < Tw4; m += 4) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const float e = ET<BF16>::ld(ev + m + u);
            const float2 ee = make_float2(e, e);
            sa = __ffma2_rn(TabT<BF16>::ld(A + m + u), ee, sa);
            sb = __ffma2_rn(TabT<BF16>::ld(B + m + u), ee, sb);
        }
    }
    const float p1 = pr.psi, p0 = 1.0f - pr.psi;
    float hv = pr.w0 * (p0 * sa.x + p1 * sa.y) + pr.w1 * (p0 * sb.x + p1 * sb.y);
    if (pr.flag0) {
        // tau = t0 exactly: outside the open window of eq. 10
        const float2 bl = TabT<BF16>::ld(B + Tw - 1);
        hv -= pr.w1 * (p0 * bl.x + p1 * bl.y) * ET<BF16>::ld(ev + Tw - 1);
    }
    return pr.w * hv;
}

__device__ __forceinline__ void neumaier_add(float& sum, float& comp, float v)
{
    const float t = sum + v;
    comp += (fabsf(sum) >= fabsf(v)) ? (sum - t) + v : (v - t) + sum;
    sum = t;
}

// One window of A x from the sorted record list: SUB sub-spans of 32 samples,
// the lane's samples being n + 32 s (s < SUB), over the records [r_lo, r_hi)
// of A-scan base `base` that reach the window.  sr / sw are this warp's
// 32-entry staging slots.  Records are staged 32 at a time in batches aligned
// to multiples of 32 in the A-scan's record list, and each lane adds a batch's
// taps in record order before compensating the batch sum into its total, so a
// sample's value does not depend on the window size (records of a batch that
// miss the sample add nothing).
template <bool BF16, int SUB>
__device__ __forceinline__ void span_gather(const typename TabT<BF16>::type* __restrict__ tab, int S, int Tw,
                                            const int2* __restrict__ rkey, const float4* __restrict__ rw,
                                            long long base, int r_lo, int r_hi, const float* __restrict__ x, int n,
                                            int lane, int4* sr, float4* sw, float (&out)[SUB])
{
    using Tab = typename TabT<BF16>::type;
    float sum[SUB], comp[SUB];
#pragma unroll
    for (int s = 0; s < SUB; ++s) sum[s] = comp[s] = 0.0f;
    const int r_first = r_lo & ~31;
    int2 kv = make_int2(0, 0);
    float4 wv = make_float4(0.f, 0.f, 0.f, 0.f);
    float xv = 0.0f;
    if (r_first + lane >= r_lo && r_first + lane < r_hi) {
        kv = __ldg(rkey + base + r_first + lane);
        wv = __ldg(rw + base + r_first + lane);
        xv = __ldg(x + kv.x);
    }
    for (int r0 = r_first; r0 < r_hi; r0 += 32) {
        const int j0 = max(0, r_lo - r0), j1 = min(32, r_hi - r0);
        if (lane >= j0 && lane < j1) {
            const int key = kv.y;
            const int lo = (key >> kRecShift) + 1;
            const int len = Tw - (key & 1);                 // tau = t0 exactly lies outside
            sr[lane] = make_int4(lo, len, ((key >> 1) & 0xfff) * S - lo, 0);
            sw[lane] = make_float4(wv.x * xv, wv.y * xv, wv.z * xv, wv.w * xv);
        }
        __syncwarp();
        if (r0 + 32 + lane < r_hi) {
            kv = __ldg(rkey + base + r0 + 32 + lane);
            wv = __ldg(rw + base + r0 + 32 + lane);
            xv = __ldg(x + kv.x);
        }
        float2 acc[SUB];
#pragma unroll
        for (int s = 0; s < SUB; ++s) acc[s] = make_float2(0.f, 0.f);
#pragma unroll 4
        for (int j = j0; j < j1; ++j) {
            const int4 d = sr[j];
            const int m = n - d.x;                           // tap of the lane's first sample
            if (m < d.y && m + 32 * (SUB - 1) >= 0) {
                const float4 w4 = sw[j];
#pragma unroll
                for (int s = 0; s < SUB; ++s) {
                    if ((unsigned)(m + 32 * s) < (unsigned)d.y) {
                        const Tab* A = tab + (d.z + n + 32 * s);
                        acc[s] = __ffma2_rn(TabT<BF16>::ld(A), make_float2(w4.x, w4.y), acc[s]);
                        acc[s] = __ffma2_rn(TabT<BF16>::ld(A + S), make_float2(w4.z, w4.w), acc[s]);
                    }
                }
            }
        }
        __syncwarp();
#pragma unroll
        for (int s = 0; s < SUB; ++s) neumaier_add(sum[s], comp[s], acc[s].x + acc[s].y);
    }
#pragma unroll
    for (int s = 0; s < SUB; ++s) out[s] = sum[s] + comp[s];
}

// Record range of window w (sub-spans w SUB .. w SUB + SUB - 1) of A-scan k
// from the per-span runs (both run bounds grow with the span, so the union of
// consecutive runs is one range).
__device__ __forceinline__ int2 window_runs(const int2* __restrict__ runs, int k, int nspan, int w, int sub)
{
    const int sp0 = w * sub, sp1 = min(sp0 + sub, nspan) - 1;
    return make_int2(__ldg(&runs[(size_t)k * nspan + sp0].x), __ldg(&runs[(size_t)k * nspan + sp1].y));
}

// Writes the window's outputs to row y (stride `stride`: samples >= M are
// zero), and zeroes the row's tail beyond the last span.
template <int SUB>
__device__ __forceinline__ void window_store(float* yf, __nv_bfloat16* yb, int M, int nspan, int stride, int sp0,
                                             int lane, const float (&v)[SUB])
{
#pragma unroll
    for (int s = 0; s < SUB; ++s) {
        if (sp0 + s >= nspan) break;
        const int n = (sp0 + s) * 32 + lane;
        if (n < stride) {
            const float val = n < M ? v[s] : 0.0f;
            if (yf) yf[n] = val;
            else yb[n] = __float2bfloat16_rn(val);
        }
    }
    if (sp0 + SUB >= nspan)
        for (int t = nspan * 32 + lane; t < stride; t += 32) {
            if (yf) yf[t] = 0.0f;
            else yb[t] = __float2bfloat16_rn(0.0f);
        }
}

constexpr int kBwdTileRows = 16;                       // A^T r tile: 16 rows (one warp each) x 32 columns
constexpr int kBwdWorkerThreads = kBwdTileRows * 32;   // threads of one tile worker

// Named barrier of tile worker h (ids 1 and 2; id 0 is __syncthreads).
__device__ __forceinline__ void worker_barrier(int h)
{
    asm volatile("bar.sync %0, %1;" ::"r"(1 + h), "n"(kBwdWorkerThreads) : "memory");
}

// One A^T r work item {tile row, tile column, ka | kb << 16, group} for tile
// worker h: every pixel of the tile sums its pairs with the A-scans [ka, kb)
// (transmitter outer, receiver inner, the transmit leg kept while the
// receiver changes) and writes the sum to its partial image `grp`.  Residual
// rows stream through the worker's nst-stage ring `ering` (rows of ebytes)
// guarded by the mbarriers at bar0.  A wait that gives up sets *abort_flag
// and the function drains the copies still in flight (bounded) and returns
// false; every thread of the worker returns the same value.
template <int NL, int MODE, bool BF16>
__device__ __forceinline__ bool backproject_item(const GeomParams& P, const DevPtrs& D,
                                                 const typename TabT<BF16>::type* __restrict__ tab,
                                                 const typename ET<BF16>::type* __restrict__ e_g, const int4 item,
                                                 float* __restrict__ partial, typename ET<BF16>::type* ering,
                                                 uint32_t bar0, int nst, size_t ebytes, volatile int* abort_flag,
                                                 uint32_t& par, int h, int hw, int lane, int ht, int3 lat)
{
    using Tab = typename TabT<BF16>::type;
    using E = typename ET<BF16>::type;
    const int S = table_stride(P.Tw4);
    const int R = P.Q + 1;
    const uint32_t rowbytes = (uint32_t)((size_t)P.Mp * sizeof(E));
    const size_t estride = ebytes / sizeof(E);
    // lat = (spacing, first row, first column) of the pixel lattice the tiles cover ((1, 0, 0): the image)
    const int row = (item.x * kBwdTileRows + hw) * lat.x + lat.y, col = (item.y * 32 + lane) * lat.x + lat.z;
    const int ka = item.z & 0xffff, kb = item.z >> 16, grp = item.w;     // A-scans [ka, kb)
    const bool pix_ok = col < P.W && row < P.H;
    const RowInfo ri = load_row(D.rows, min(row, P.H - 1));
    const bool row_ok = pix_ok && ri.tvert < (float)(P.M - 1);
    const int colc = min(col, P.W - 1);
    if (ht == 0) {
        for (int s = 0; s < nst && ka + s < kb; ++s) {
            mbar_arrive_expect_tx(bar0 + 8 * s, rowbytes);
            bulk_g2s(smem_u32(ering + (size_t)s * estride), e_g + (size_t)(ka + s) * P.Mp, rowbytes, bar0 + 8 * s);
        }
    }
    float sum = 0.0f, comp = 0.0f;
    Leg tx = {0.f, 0.f, 0.f, 0.f}, rx_cur = tx, rx_nxt = tx;
    int hx_nxt = 0;
    if constexpr (MODE == kModeTAB) {
        if (row_ok) {
            rx_cur = get_leg<NL, MODE>(P, D, ri, row, colc, __ldg(D.rxpos + ka));
            if (ka + 1 < kb) hx_nxt = __ldg(D.hidx + (size_t)__ldg(D.rxpos + ka + 1) * P.W + colc);
        }
    }
    int i = ka / P.n_rx, j = ka - i * P.n_rx, stage = 0, k = ka;
    bool aborted = false;
    for (; k < kb; ++k) {
        if constexpr (MODE == kModeTAB) {
            // legs of the next A-scan stream in while this one is consumed
            if (row_ok && k + 1 < kb) {
                float4 v = __ldg(D.legs + (size_t)row * P.nh + hx_nxt);
                rx_nxt = Leg{v.x, v.y, v.z, v.w};
                if (k + 2 < kb) hx_nxt = __ldg(D.hidx + (size_t)__ldg(D.rxpos + k + 2) * P.W + colc);
            }
        }
        if (row_ok) {
            if (j == 0 || k == ka) tx = get_leg<NL, MODE>(P, D, ri, row, colc, __ldg(D.txpos + i));
            if constexpr (MODE != kModeTAB) rx_cur = get_leg<NL, MODE>(P, D, ri, row, colc, __ldg(D.rxpos + k));
        }
        const Pair pr = make_pair(P, tx, rx_cur, ri.tau);
        const bool act = row_ok && pr.w != 0.0f && pr.n0 >= 0 && pr.n0 + 1 < P.M;
        const bool ok = mbar_wait_bounded(bar0 + 8 * stage, (par >> stage) & 1u, D.status);
        par ^= 1u << stage;
        if (!ok) *abort_flag = 1;
        if (act && ok) {
            const E* ev = ering + (size_t)stage * estride + pr.n0 + 1;
            const Tab* A = tab + (size_t)(pr.gi * R + pr.r) * S;
            neumaier_add(sum, comp, pair_taps<BF16>(A, S, P.Tw, P.Tw4, ev, pr));
        }
        worker_barrier(h);
        if (*abort_flag) {
            aborted = true;
            break;
        }
        if (ht == 0 && k + nst < kb) {
            mbar_arrive_expect_tx(bar0 + 8 * stage, rowbytes);
            bulk_g2s(smem_u32(ering + (size_t)stage * estride), e_g + (size_t)(k + nst) * P.Mp, rowbytes,
                     bar0 + 8 * stage);
        }
        if constexpr (MODE == kModeTAB) rx_cur = rx_nxt;
        if (++stage == nst) stage = 0;
        if (++j == P.n_rx) { j = 0; ++i; }
    }
    if (aborted) {
        // drain this item's copies still in flight (bounded) before leaving
        if (ht == 0) {
            for (int q = k + 1; q < kb && q < k + nst; ++q) {
                const int s = (q - ka) % nst;
                mbar_wait_bounded(bar0 + 8 * s, (par >> s) & 1u, D.status);
                par ^= 1u << s;
            }
        }
        return false;
    }
    if (pix_ok) partial[(size_t)grp * P.W * P.H + (size_t)row * P.W + col] = sum + comp;
    return true;
}

}  // namespace mbir
