// A x (eq. 11-13 summed over voxels) as a gather: one CTA per A-scan.  The CTA
// walks the image in blocks of columns.  For each block it writes one record
// per (column, row) pair - first tap sample, table row, bilinear weights times
// x - into shared memory.  Inside one layer the travel time grows with depth,
// so each (column, layer) segment of records is sorted by first sample; for
// every 32-sample span of the A-scan the rows whose 68-tap window reaches the
// span form one contiguous run.  The run bounds of every (segment, span) are
// written by a conflict-free scatter (each bound is owned by exactly one row),
// then each warp produces its spans with counted loops over those runs.
// Every output sample is owned by one lane: no atomics, a fixed summation
// order, bitwise reproducible results.
#include <algorithm>

#include "device_common.cuh"

namespace mbir {

constexpr int kKeyShift = 13;                  // record key: n0 << 13 | table row << 1 | flag0
constexpr int kKeyBeyond = (1 << 18) - 1;      // n0 of rows that cannot reach the record

__device__ __forceinline__ int key_n0(int key) { return key >> kKeyShift; }

template <int NL, int MODE, bool BF16, int THREADS>
__global__ void __launch_bounds__(THREADS, 1)
    forward_kernel(GeomParams P, DevPtrs D, const typename TabT<BF16>::type* __restrict__ tab_g,
                   const float* __restrict__ x, float* __restrict__ y_f32, __nv_bfloat16* __restrict__ y_bf16,
                   int out_stride, int CB)
{
    using Tab = typename TabT<BF16>::type;
    constexpr int WARPS = THREADS / 32;
    extern __shared__ __align__(128) unsigned char smem[];
    const int S = table_stride(P.Tw4);
    const int R = P.Q + 1;
    const int nspan = (P.M + 31) >> 5;
    const int nseg = P.n_seg;
    const int ncs = CB * nseg;                        // (column, segment) runs per block
    const size_t tab_bytes = ((size_t)P.Gt * R * S * sizeof(Tab) + 127) & ~(size_t)127;
    const size_t ybytes = ((size_t)P.Mp * 4 + 127) & ~(size_t)127;
    const int nrec = CB * P.H;
    Tab* tab = reinterpret_cast<Tab*>(smem);
    float* yacc = reinterpret_cast<float*>(smem + tab_bytes);
    float* ycomp = reinterpret_cast<float*>(smem + tab_bytes + ybytes);
    float4* wrec = reinterpret_cast<float4*>(smem + tab_bytes + 2 * ybytes);
    int* keys = reinterpret_cast<int*>(wrec + nrec);
    short* fb = reinterpret_cast<short*>(keys + nrec);   // run bounds [first, end) per (run, span)
    short* eb = fb + (size_t)ncs * nspan;
    int* cs_start = reinterpret_cast<int*>(eb + (size_t)ncs * nspan + 2);   // ncs + 1 offsets
    int* wsum = cs_start + ncs + 2;                                            // WARPS partial counts

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int k = blockIdx.x;
    const int i = k / P.n_rx;
    const int txp = __ldg(D.txpos + i), rxp = __ldg(D.rxpos + k);

    {
        const int4* src = reinterpret_cast<const int4*>(tab_g);
        int4* dst = reinterpret_cast<int4*>(tab);
        const int n16 = (int)(tab_bytes / 16);
        for (int t = tid; t < n16; t += THREADS) dst[t] = __ldg(src + t);
    }
    for (int t = tid; t < P.Mp; t += THREADS) {
        yacc[t] = 0.0f;
        ycomp[t] = 0.0f;
    }

    for (int c0 = 0; c0 < P.W; c0 += CB) {
        __syncthreads();
        // ---- records of this column block, in (column, row) order
        for (int idx = tid; idx < nrec; idx += THREADS) {
            const int cl = idx / P.H, row = idx - cl * P.H;
            const int col = c0 + cl;
            int key = -1;
            float4 wv = make_float4(0.f, 0.f, 0.f, 0.f);
            if (col < P.W) {
                RowInfo ri = load_row(D.rows, row);
                if (ri.tvert < (float)(P.M - 1)) {
                    Leg tx = get_leg<NL, MODE>(P, D, ri, row, col, txp);
                    Leg rx = get_leg<NL, MODE>(P, D, ri, row, col, rxp);
                    Pair pr = make_pair(P, tx, rx, ri.tau);
                    const float wx = pr.w * __ldg(x + (size_t)row * P.W + col);
                    if (wx != 0.0f && pr.n0 >= 0 && pr.n0 + 1 < P.M) {
                        key = (pr.n0 << kKeyShift) | ((pr.gi * R + pr.r) << 1) | (pr.flag0 ? 1 : 0);
                        const float p1 = pr.psi, p0 = 1.0f - pr.psi;
                        wv = make_float4(wx * pr.w0 * p0, wx * pr.w0 * p1, wx * pr.w1 * p0, wx * pr.w1 * p1);
                    }
                }
            }
            keys[idx] = key;
            wrec[idx] = wv;
        }
        __syncthreads();
        // ---- stable in-place compaction of the contributing records (key >= 0).
        // A sub-sequence of a sorted run stays sorted, so each (column, segment)
        // run keeps its order by first sample.
        int base = 0;
        for (int c = 0; c * THREADS < nrec; ++c) {
            const int idx = c * THREADS + tid;
            int key = -1;
            float4 wv;
            if (idx < nrec) {
                key = keys[idx];
                wv = wrec[idx];
            }
            const bool act = key >= 0;
            const unsigned bal = __ballot_sync(0xffffffffu, act);
            const int before = __popc(bal & ((1u << lane) - 1u));
            if (lane == 0) wsum[warp] = __popc(bal);
            __syncthreads();
            int off = base;
            for (int w = 0; w < warp; ++w) off += wsum[w];
            int tot = 0;
            for (int w = 0; w < WARPS; ++w) tot += wsum[w];
            const int dst = off + before;
            if (idx < nrec) {
                const int cl = idx / P.H, row = idx - cl * P.H;
                for (int sg = 0; sg < nseg; ++sg)
                    if (row == P.seg_row[sg]) cs_start[cl * nseg + sg] = dst;
            }
            if (act) {
                keys[dst] = key;
                wrec[dst] = wv;
            }
            base += tot;
            __syncthreads();
        }
        if (tid == 0) cs_start[ncs] = base;
        __syncthreads();
        // ---- run bounds by scatter: span s needs records with s*32-Tw <= n0 <= s*32+30.
        // Inside a run n0 is non-decreasing, so record t is the first record of
        // span s for exactly the spans whose threshold falls in (n0[t-1], n0[t]];
        // the run's last record also closes every later span.
        for (int cs = warp; cs < ncs; cs += WARPS) {
            const int a = cs_start[cs], b = cs_start[cs + 1];
            short* F = fb + (size_t)cs * nspan;
            short* E = eb + (size_t)cs * nspan;
            if (a == b) {
                for (int s = lane; s < nspan; s += 32) { F[s] = (short)a; E[s] = (short)a; }
                continue;
            }
            for (int t = a + lane; t < b; t += 32) {
                const int n0 = key_n0(keys[t]);
                const int prev = (t > a) ? key_n0(keys[t - 1]) : -(1 << 20);
                const int s_lo = (prev + P.Tw < 0) ? 0 : (prev + P.Tw) / 32 + 1;
                const int s_hi = min((n0 + P.Tw) >> 5, nspan - 1);
                for (int s = s_lo; s <= s_hi; ++s) F[s] = (short)t;
                const int e_lo = (prev - 31 < 0) ? 0 : (prev - 31) / 32 + 1;
                const int e_hi = (n0 - 31 < 0) ? -1 : min((n0 - 31) >> 5, nspan - 1);
                for (int s = e_lo; s <= e_hi; ++s) E[s] = (short)t;
                if (t == b - 1) {
                    const int s_f = ((n0 + P.Tw) >> 5) + 1;
                    for (int s = s_f; s < nspan; ++s) F[s] = (short)b;
                    const int s_e = (n0 - 31 < 0) ? 0 : ((n0 - 31) >> 5) + 1;
                    for (int s = s_e; s < nspan; ++s) E[s] = (short)b;
                }
            }
        }
        __syncthreads();
        // ---- gather: warp-owned spans of 32 samples, counted loops over runs
        for (int sp = warp; sp < nspan; sp += WARPS) {
            const int n = sp * 32 + lane;
            float2 acc = make_float2(0.f, 0.f);
            for (int cs = 0; cs < ncs; ++cs) {
                const size_t o = (size_t)cs * nspan + sp;
                const int r0 = fb[o], r1 = eb[o];
#pragma unroll 4
                for (int rr = r0; rr < r1; ++rr) {
                    const int key = keys[rr];
                    const int m = n - key_n0(key) - 1;
                    const bool edge = (key & 1) && m == P.Tw - 1;   // tau = t0 exactly: outside
                    if ((unsigned)m < (unsigned)P.Tw && !edge) {
                        const float4 wv = wrec[rr];
                        const Tab* A = tab + (size_t)((key >> 1) & 0xfff) * S + m;
                        acc = __ffma2_rn(TabT<BF16>::ld(A), make_float2(wv.x, wv.y), acc);
                        acc = __ffma2_rn(TabT<BF16>::ld(A + S), make_float2(wv.z, wv.w), acc);
                    }
                }
            }
            if (n < P.M) {
                // Neumaier-compensated accumulation across column blocks
                const float v = acc.x + acc.y;
                const float yv = yacc[n];
                const float t = yv + v;
                ycomp[n] += (fabsf(yv) >= fabsf(v)) ? (yv - t) + v : (v - t) + yv;
                yacc[n] = t;
            }
        }
    }
    __syncthreads();
    if (y_f32) {
        float* yo = y_f32 + (size_t)k * out_stride;
        for (int t = tid; t < out_stride; t += THREADS) yo[t] = (t < P.M) ? yacc[t] + ycomp[t] : 0.0f;
    } else {
        __nv_bfloat16* yo = y_bf16 + (size_t)k * out_stride;
        for (int t = tid; t < out_stride; t += THREADS)
            yo[t] = __float2bfloat16_rn((t < P.M) ? yacc[t] + ycomp[t] : 0.0f);
    }
}

// shared memory: table + accumulator and its compensation + CB columns of
// records (20 B per row) + run bounds (2 x 2 B per (column, segment, span))
// + run offsets and warp counts
size_t forward_smem(const mbir_geometry* g, int* cb_out)
{
    const GeomParams& P = g->P;
    size_t tsz = P.precision == MBIR_PREC_BF16 ? 4 : 8;
    size_t tab = ((size_t)P.Gt * (P.Q + 1) * table_stride(P.Tw4) * tsz + 127) & ~(size_t)127;
    size_t yb = ((size_t)P.Mp * 4 + 127) & ~(size_t)127;
    const size_t nspan = (P.M + 31) / 32;
    const size_t per_col = (size_t)P.H * 20 + (size_t)P.n_seg * nspan * 4 + (size_t)P.n_seg * 4;
    const size_t fixed = tab + 2 * yb + 4 + 8 + 8 + 32 * 4 + 64;
    const size_t budget = 222 * 1024;
    long avail = (long)budget - (long)fixed;
    int cb = avail > 0 ? (int)(avail / per_col) : 0;
    cb = std::min(cb, 16);
    // compacted positions are stored as 16-bit run bounds
    while (cb > 1 && (size_t)cb * P.H > 32767) --cb;
    if (cb_out) *cb_out = cb;
    return fixed + (size_t)std::max(cb, 1) * per_col;
}

template <int NL, int MODE, bool BF16, int THREADS>
static cudaError_t launch_fwd_t(const mbir_geometry* g, const float* x, float* yf, __nv_bfloat16* yb, int stride,
                                cudaStream_t st)
{
    int cb = 0;
    size_t sm = forward_smem(g, &cb);
    if (cb < 1) return cudaErrorInvalidConfiguration;
    auto kern = forward_kernel<NL, MODE, BF16, THREADS>;
    cudaError_t ce = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (ce != cudaSuccess) return ce;
    using Tab = typename TabT<BF16>::type;
    const Tab* tab = BF16 ? (const Tab*)(const void*)g->d_tab_bf16 : (const Tab*)(const void*)g->d_tab;
    kern<<<g->P.K, THREADS, sm, st>>>(g->P, dev_ptrs(g), tab, x, yf, yb, stride, cb);
    return cudaGetLastError();
}

template <int MODE, bool BF16>
static cudaError_t launch_fwd_nl(const mbir_geometry* g, const float* x, float* yf, __nv_bfloat16* yb, int stride,
                                 cudaStream_t st)
{
    if constexpr (MODE == kModeTAB) {
        return launch_fwd_t<1, MODE, BF16, 1024>(g, x, yf, yb, stride, st);
    } else {
        if (g->P.L <= 2) return launch_fwd_t<2, MODE, BF16, 512>(g, x, yf, yb, stride, st);
        if (g->P.L <= 4) return launch_fwd_t<4, MODE, BF16, 512>(g, x, yf, yb, stride, st);
        return launch_fwd_t<8, MODE, BF16, 512>(g, x, yf, yb, stride, st);
    }
}

cudaError_t launch_forward(const mbir_geometry* g, const float* x, float* y_f32, __nv_bfloat16* y_bf16,
                           int out_stride, cudaStream_t st)
{
    if (g->d_tf4_bop) return launch_forward_tcs(g, x, y_f32, y_bf16, out_stride, st);
    if (g->d_rec_key) return launch_forward_sorted(g, x, y_f32, y_bf16, out_stride, st);
    const bool bf = g->P.precision == MBIR_PREC_BF16;
    if (g->P.mode == MBIR_MODE_TAB)
        return bf ? launch_fwd_nl<kModeTAB, true>(g, x, y_f32, y_bf16, out_stride, st)
                  : launch_fwd_nl<kModeTAB, false>(g, x, y_f32, y_bf16, out_stride, st);
    return bf ? launch_fwd_nl<kModeOTF, true>(g, x, y_f32, y_bf16, out_stride, st)
              : launch_fwd_nl<kModeOTF, false>(g, x, y_f32, y_bf16, out_stride, st);
}

}  // namespace mbir
