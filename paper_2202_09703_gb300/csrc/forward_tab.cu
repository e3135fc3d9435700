// TAB-mode A x from a precomputed, sorted record list.
//
// The geometry is fixed, so once per geometry (the paper's "compute the
// system matrix once", Section 3) every A-scan's active pairs are written as
// records {pixel, first tap sample n0 | table row | tau = t0 flag, bilinear
// weights times w} sorted by n0 (ties by pixel index, so the order is
// deterministic).  For each 32-sample span of an A-scan the records whose tap
// window reaches the span are then one contiguous range, stored as run bounds.
//
// The apply kernel is a persistent, barrier-free gather: every warp takes
// whole spans (largest first, from a counter), decodes 32 records at a time
// into its own shared-memory slot (first tap, tap count, table offset, and
// weights times x) while the next 32 stream into registers, and each lane
// accumulates the taps that land on its sample.  Output samples are owned by
// one lane and summed in record order: no atomics on data, fixed order.
#include <algorithm>
#include <vector>

#include "apply_common.cuh"

namespace mbir {

constexpr int kSortThreads = 512;
constexpr int kFwdSortedThreads = 1024;

struct RecPair {
    int n0, trow, flag;
    float4 w;
    bool act;
};

__device__ __forceinline__ RecPair tab_record(const GeomParams& P, const DevPtrs& D, int k, int v)
{
    RecPair o;
    o.act = false;
    const int row = v / P.W, col = v - row * P.W;
    const RowInfo ri = load_row(D.rows, row);
    if (!(ri.tvert < (float)(P.M - 1))) return o;
    const int i = k / P.n_rx;
    const Leg tx = get_leg<1, kModeTAB>(P, D, ri, row, col, __ldg(D.txpos + i));
    const Leg rx = get_leg<1, kModeTAB>(P, D, ri, row, col, __ldg(D.rxpos + k));
    const Pair pr = make_pair(P, tx, rx, ri.tau);
    if (!(pr.w != 0.0f && pr.n0 >= 0 && pr.n0 + 1 < P.M)) return o;
    o.act = true;
    o.n0 = pr.n0;
    o.trow = pr.gi * (P.Q + 1) + pr.r;
    o.flag = pr.flag0 ? 1 : 0;
    const float p1 = pr.psi, p0 = 1.0f - pr.psi;
    o.w = make_float4(pr.w * pr.w0 * p0, pr.w * pr.w0 * p1, pr.w * pr.w1 * p0, pr.w * pr.w1 * p1);
    return o;
}

// active-pair count per A-scan (integer sums: order-independent)
__global__ void rec_count_kernel(GeomParams P, DevPtrs D, long long* __restrict__ counts)
{
    __shared__ int sh[32];
    const int k = blockIdx.x;
    const int N = P.W * P.H;
    int c = 0;
    for (int v = threadIdx.x; v < N; v += blockDim.x) c += tab_record(P, D, k, v).act ? 1 : 0;
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
        counts[k] = t;
    }
}

// Counting sort of one A-scan's records by n0, then each bucket ordered by
// pixel index; run bounds per 32-sample span from the bucket starts.
__global__ void __launch_bounds__(kSortThreads)
    rec_fill_kernel(GeomParams P, DevPtrs D, const long long* __restrict__ off, int2* __restrict__ rkey,
                    float4* __restrict__ rw, int2* __restrict__ runs)
{
    extern __shared__ int hs[];                    // hist[M], start[M + 1]
    int* hist = hs;
    int* start = hs + P.M;
    const int k = blockIdx.x;
    const int N = P.W * P.H;
    const long long base = off[k];
    for (int t = threadIdx.x; t < P.M; t += blockDim.x) hist[t] = 0;
    __syncthreads();
    for (int v = threadIdx.x; v < N; v += blockDim.x) {
        RecPair r = tab_record(P, D, k, v);
        if (r.act) atomicAdd(&hist[r.n0], 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int s = 0;
        for (int t = 0; t < P.M; ++t) {
            start[t] = s;
            s += hist[t];
        }
        start[P.M] = s;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < P.M; t += blockDim.x) hist[t] = 0;    // now the per-bucket cursor
    const int nspan = (P.M + 31) >> 5;
    for (int s = threadIdx.x; s < nspan; s += blockDim.x) {
        // span s needs n0 in [32 s - Tw, 32 s + 30]
        const int lo = max(32 * s - P.Tw, 0), hi = min(32 * s + 31, P.M);
        runs[(size_t)k * nspan + s] = make_int2(start[lo], start[hi]);
    }
    __syncthreads();
    for (int v = threadIdx.x; v < N; v += blockDim.x) {
        RecPair r = tab_record(P, D, k, v);
        if (!r.act) continue;
        const long long p = base + start[r.n0] + atomicAdd(&hist[r.n0], 1);
        rkey[p] = make_int2(v, (r.n0 << kRecShift) | (r.trow << 1) | r.flag);
        rw[p] = r.w;
    }
    __syncthreads();
    __threadfence_block();
    // order each bucket by pixel index (insertion sort; buckets hold a few dozen records)
    for (int t = threadIdx.x; t < P.M; t += blockDim.x) {
        const long long a = base + start[t], b = base + start[t + 1];
        for (long long q = a + 1; q < b; ++q) {
            const int2 kq = rkey[q];
            const float4 wq = rw[q];
            long long p = q - 1;
            while (p >= a && rkey[p].x > kq.x) {
                rkey[p + 1] = rkey[p];
                rw[p + 1] = rw[p];
                --p;
            }
            rkey[p + 1] = kq;
            rw[p + 1] = wq;
        }
    }
}

template <bool BF16>
__global__ void __launch_bounds__(kFwdSortedThreads, 1)
    forward_sorted_kernel(GeomParams P, const typename TabT<BF16>::type* __restrict__ tab_g,
                          const long long* __restrict__ off, const int2* __restrict__ rkey,
                          const float4* __restrict__ rw, const int2* __restrict__ runs,
                          const int* __restrict__ order, int* __restrict__ next_span, const float* __restrict__ x,
                          float* __restrict__ y_f32, __nv_bfloat16* __restrict__ y_bf16, int out_stride)
{
    using Tab = typename TabT<BF16>::type;
    constexpr int WARPS = kFwdSortedThreads / 32;
    extern __shared__ __align__(128) unsigned char smem[];
    const int S = table_stride(P.Tw4);
    const size_t tab_bytes = ((size_t)P.Gt * (P.Q + 1) * S * sizeof(Tab) + 127) & ~(size_t)127;
    Tab* tab = reinterpret_cast<Tab*>(smem);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // per-warp staging of 32 decoded records: {first tap, tap count, table offset - first tap} and weights * x
    int4* sr = reinterpret_cast<int4*>(smem + tab_bytes) + warp * 32;
    float4* sw = reinterpret_cast<float4*>(smem + tab_bytes) + WARPS * 32 + warp * 32;
    load_table_smem(tab, tab_g, tab_bytes, tid, kFwdSortedThreads);
    __syncthreads();
    const int nspan = (P.M + 31) >> 5;
    const int total = P.K * nspan;
    for (;;) {
        // spans are handed out largest-first through a counter, one per warp
        int idx = 0;
        if (lane == 0) idx = atomicAdd(next_span, 1);
        idx = __shfl_sync(0xffffffffu, idx, 0);
        if (idx >= total) break;
        const int gs = __ldg(order + idx);
        const int k = gs / nspan, sp = gs - k * nspan;
        const int n = sp * 32 + lane;
        const long long base = __ldg(off + k);
        const int2 rb = __ldg(runs + gs);
        const float acc = span_gather<BF16>(tab, S, P.Tw, rkey, rw, base, rb.x, rb.y, x, n, lane, sr, sw);
        const float yv = (n < P.M) ? acc : 0.0f;
        if (n < out_stride) {
            if (y_f32) y_f32[(size_t)k * out_stride + n] = yv;
            else y_bf16[(size_t)k * out_stride + n] = __float2bfloat16_rn(yv);
        }
        if (sp == nspan - 1) {
            for (int t = nspan * 32 + lane; t < out_stride; t += 32) {
                if (y_f32) y_f32[(size_t)k * out_stride + t] = 0.0f;
                else y_bf16[(size_t)k * out_stride + t] = __float2bfloat16_rn(0.0f);
            }
        }
    }
}

// Builds the sorted records; returns cudaErrorNotSupported when the record
// list would not fit the byte cap (the caller then keeps the on-the-fly
// record path).
cudaError_t build_sorted_records(mbir_geometry* g, cudaStream_t st, size_t cap_bytes)
{
    const GeomParams& P = g->P;
    if (P.mode != MBIR_MODE_TAB || P.M > 16384) return cudaErrorNotSupported;
    DevPtrs D = dev_ptrs(g);
    long long* d_cnt = nullptr;
    cudaError_t e = cudaMalloc(&d_cnt, sizeof(long long) * (P.K + 1));
    if (e != cudaSuccess) return e;
    rec_count_kernel<<<P.K, 256, 0, st>>>(P, D, d_cnt);
    std::vector<long long> cnt(P.K), off(P.K + 1, 0);
    e = cudaMemcpyAsync(cnt.data(), d_cnt, sizeof(long long) * P.K, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) { cudaFree(d_cnt); return e; }
    for (int k = 0; k < P.K; ++k) off[k + 1] = off[k] + cnt[k];
    const long long R = off[P.K];
    const int nspan = (P.M + 31) / 32;
    const size_t need = (size_t)R * (sizeof(int2) + sizeof(float4)) + (size_t)P.K * nspan * sizeof(int2);
    if (need > cap_bytes) { cudaFree(d_cnt); return cudaErrorNotSupported; }
    e = cudaMemcpyAsync(d_cnt, off.data(), sizeof(long long) * (P.K + 1), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMalloc((void**)&g->d_rec_key, sizeof(int2) * std::max<long long>(R, 1));
    if (e == cudaSuccess) e = cudaMalloc((void**)&g->d_rec_w, sizeof(float4) * std::max<long long>(R, 1));
    if (e == cudaSuccess) e = cudaMalloc((void**)&g->d_runs, sizeof(int2) * (size_t)P.K * nspan);
    if (e != cudaSuccess) { cudaFree(d_cnt); return e; }
    g->d_rec_off = d_cnt;
    g->n_records = R;
    g->bytes += need + sizeof(long long) * (P.K + 1);
    const size_t sm = sizeof(int) * (2 * (size_t)P.M + 1);
    e = cudaFuncSetAttribute(rec_fill_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    rec_fill_kernel<<<P.K, kSortThreads, sm, st>>>(P, D, g->d_rec_off, g->d_rec_key, g->d_rec_w, g->d_runs);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    // spans in decreasing order of work, so the last spans handed out are short
    std::vector<int2> runs((size_t)P.K * nspan);
    e = cudaMemcpy(runs.data(), g->d_runs, sizeof(int2) * runs.size(), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return e;
    g->h_span_cost = (int*)malloc(sizeof(int) * runs.size());
    if (g->h_span_cost)
        for (size_t t = 0; t < runs.size(); ++t) g->h_span_cost[t] = runs[t].y - runs[t].x;
    std::vector<int> order(runs.size());
    for (size_t t = 0; t < order.size(); ++t) order[t] = (int)t;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        return runs[a].y - runs[a].x > runs[b].y - runs[b].x;
    });
    e = cudaMalloc((void**)&g->d_span_order, sizeof(int) * order.size());
    if (e == cudaSuccess) e = cudaMemcpy(g->d_span_order, order.data(), sizeof(int) * order.size(),
                                         cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc((void**)&g->d_span_counter, sizeof(int));
    if (e == cudaSuccess) g->bytes += sizeof(int) * (order.size() + 1);
    return e;
}

size_t forward_sorted_smem(const mbir_geometry* g)
{
    const GeomParams& P = g->P;
    size_t tsz = P.precision == MBIR_PREC_BF16 ? 4 : 8;
    size_t tab = ((size_t)P.Gt * (P.Q + 1) * table_stride(P.Tw4) * tsz + 127) & ~(size_t)127;
    return tab + (size_t)kFwdSortedThreads * (sizeof(float4) + sizeof(int4));
}

cudaError_t launch_forward_sorted(const mbir_geometry* g, const float* x, float* yf, __nv_bfloat16* yb, int stride,
                                  cudaStream_t st)
{
    const size_t sm = forward_sorted_smem(g);
    const int nspan = (g->P.M + 31) / 32;
    const long long spans = (long long)g->P.K * nspan;
    const int grid = (int)std::max<long long>(1, std::min<long long>(g->n_sm, (spans + 31) / 32));
    cudaError_t me = cudaMemsetAsync(g->d_span_counter, 0, sizeof(int), st);
    if (me != cudaSuccess) return me;
    if (g->P.precision == MBIR_PREC_BF16) {
        auto kern = forward_sorted_kernel<true>;
        cudaError_t ce = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (ce != cudaSuccess) return ce;
        kern<<<grid, kFwdSortedThreads, sm, st>>>(g->P, g->d_tab_bf16, g->d_rec_off, g->d_rec_key, g->d_rec_w,
                                                  g->d_runs, g->d_span_order, g->d_span_counter, x, yf, yb, stride);
    } else {
        auto kern = forward_sorted_kernel<false>;
        cudaError_t ce = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (ce != cudaSuccess) return ce;
        kern<<<grid, kFwdSortedThreads, sm, st>>>(g->P, g->d_tab, g->d_rec_off, g->d_rec_key, g->d_rec_w,
                                                  g->d_runs, g->d_span_order, g->d_span_counter, x, yf, yb, stride);
    }
    return cudaGetLastError();
}

}  // namespace mbir
