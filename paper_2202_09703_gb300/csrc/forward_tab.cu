// TAB-mode A x from a precomputed, sorted record list.
//
// The geometry is fixed, so once per geometry (the paper's "compute the
// system matrix once", Section 3) every A-scan's active pairs are written as
// records {pixel, first tap sample n0 | table row | tau = t0 flag, bilinear
// weights times w} sorted by n0 (ties by table row, then pixel index, so the
// order is deterministic).  For each 32-sample span of an A-scan the records whose tap
// window reaches the span are then one contiguous range, stored as run bounds.
//
// The apply kernel is a persistent, barrier-free gather: every warp takes
// whole windows of SUB consecutive spans (largest first, from a counter),
// decodes 32 records at a time into its own shared-memory slot (first tap,
// tap count, table offset, and weights times x) while the next 32 stream into
// registers, and each lane accumulates the taps that land on its SUB samples.
// Output samples are owned by one lane and summed in record order: no atomics
// on data, fixed order.  A wider window reads each staged record for more
// samples; SUB is chosen per geometry by timing the candidates once.
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
    Pair pr;
    o.act = tab_pair(P, D, k, v, pr);
    if (!o.act) return o;
    o.n0 = pr.n0;
    o.trow = pr.gi * (P.Q + 1) + pr.r;
    o.flag = pr.flag0 ? 1 : 0;
    const float p1 = pr.psi, p0 = 1.0f - pr.psi;
    o.w = make_float4(pr.w * pr.w0 * p0, pr.w * pr.w0 * p1, pr.w * pr.w1 * p0, pr.w * pr.w1 * p1);
    return o;
}

// Pixels of the lattice lat = (spacing s, first row, first column): t -> pixel index, Wc x Hc of them
// ((1, 0, 0): every pixel, t = pixel index).
struct Lattice {
    int s, r0, c0, Wc, Nc;
};

__host__ __device__ inline Lattice make_lattice(const GeomParams& P, int3 lat)
{
    Lattice L;
    L.s = lat.x;
    L.r0 = lat.y;
    L.c0 = lat.z;
    L.Wc = (P.W - lat.z + lat.x - 1) / lat.x;
    L.Nc = ((P.H - lat.y + lat.x - 1) / lat.x) * L.Wc;
    return L;
}

__device__ __forceinline__ int lattice_pixel(const GeomParams& P, const Lattice& L, int t)
{
    const int i = t / L.Wc;
    return (i * L.s + L.r0) * P.W + (t - i * L.Wc) * L.s + L.c0;
}

// active-pair count per A-scan over the lattice's pixels (integer sums: order-independent)
__global__ void rec_count_kernel(GeomParams P, DevPtrs D, int3 lat, long long* __restrict__ counts)
{
    __shared__ int sh[32];
    const int k = blockIdx.x;
    const Lattice L = make_lattice(P, lat);
    int c = 0;
    for (int t = threadIdx.x; t < L.Nc; t += blockDim.x) c += tab_record(P, D, k, lattice_pixel(P, L, t)).act ? 1 : 0;
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
        counts[k] = t;
    }
}

// Counting sort of one A-scan's records (pixels of the lattice) by n0, then
// each bucket ordered by table row and pixel index; run bounds per 32-sample
// span from the bucket starts.
__global__ void __launch_bounds__(kSortThreads)
    rec_fill_kernel(GeomParams P, DevPtrs D, int3 lat, const long long* __restrict__ off, int2* __restrict__ rkey,
                    float4* __restrict__ rw, int2* __restrict__ runs)
{
    extern __shared__ int hs[];                    // hist[M], start[M + 1]
    int* hist = hs;
    int* start = hs + P.M;
    const int k = blockIdx.x;
    const Lattice L = make_lattice(P, lat);
    const long long base = off[k];
    for (int t = threadIdx.x; t < P.M; t += blockDim.x) hist[t] = 0;
    __syncthreads();
    for (int t = threadIdx.x; t < L.Nc; t += blockDim.x) {
        RecPair r = tab_record(P, D, k, lattice_pixel(P, L, t));
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
    for (int t = threadIdx.x; t < L.Nc; t += blockDim.x) {
        const int v = lattice_pixel(P, L, t);
        RecPair r = tab_record(P, D, k, v);
        if (!r.act) continue;
        const long long p = base + start[r.n0] + atomicAdd(&hist[r.n0], 1);
        rkey[p] = make_int2(v, (r.n0 << kRecShift) | (r.trow << 1) | r.flag);
        rw[p] = r.w;
    }
    __syncthreads();
    __threadfence_block();
    // order each bucket by (table row = plane * (Q + 1) + lower phase, pixel index) (insertion sort; buckets
    // hold a few dozen records): the tensor-core A x then finds the records of one sum cell adjacent
    auto order_key = [](int2 k) {
        return ((long long)((k.y >> 1) & 0xfff) << 32) | (long long)(unsigned)k.x;
    };
    for (int t = threadIdx.x; t < P.M; t += blockDim.x) {
        const long long a = base + start[t], b = base + start[t + 1];
        for (long long q = a + 1; q < b; ++q) {
            const int2 kq = rkey[q];
            const float4 wq = rw[q];
            const long long oq = order_key(kq);
            long long p = q - 1;
            while (p >= a && order_key(rkey[p]) > oq) {
                rkey[p + 1] = rkey[p];
                rw[p + 1] = rw[p];
                --p;
            }
            rkey[p + 1] = kq;
            rw[p + 1] = wq;
        }
    }
}

template <bool BF16, int SUB>
__global__ void __launch_bounds__(kFwdSortedThreads, 1)
    forward_sorted_kernel(GeomParams P, const typename TabT<BF16>::type* __restrict__ tab_g,
                          const long long* __restrict__ off, const int2* __restrict__ rkey,
                          const float4* __restrict__ rw, const int2* __restrict__ runs,
                          const int* __restrict__ order, int total, int* __restrict__ next_win,
                          const float* __restrict__ x, float* __restrict__ y_f32, __nv_bfloat16* __restrict__ y_bf16,
                          int out_stride)
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
    const int nwin = (nspan + SUB - 1) / SUB;
    for (;;) {
        // windows are handed out largest-first through a counter, one per warp
        int idx = 0;
        if (lane == 0) idx = atomicAdd(next_win, 1);
        idx = __shfl_sync(0xffffffffu, idx, 0);
        if (idx >= total) break;
        const int gw = __ldg(order + idx);
        const int k = gw / nwin, w = gw - k * nwin;
        const int2 rb = window_runs(runs, k, nspan, w, SUB);
        float v[SUB];
        span_gather<BF16, SUB>(tab, S, P.Tw, rkey, rw, __ldg(off + k), rb.x, rb.y, x, w * SUB * 32 + lane, lane,
                               sr, sw, v);
        window_store<SUB>(y_f32 ? y_f32 + (size_t)k * out_stride : nullptr,
                          y_f32 ? nullptr : y_bf16 + (size_t)k * out_stride, P.M, nspan, out_stride, w * SUB, lane, v);
    }
}

// Windows of `sub` spans of every A-scan, largest first (records visited).
static void window_order(const std::vector<int2>& runs, int K, int nspan, int sub, std::vector<int>* order,
                         std::vector<int>* cost)
{
    const int nwin = (nspan + sub - 1) / sub;
    cost->assign((size_t)K * nwin, 0);
    for (int k = 0; k < K; ++k)
        for (int w = 0; w < nwin; ++w) {
            const int sp0 = w * sub, sp1 = std::min(sp0 + sub, nspan) - 1;
            (*cost)[(size_t)k * nwin + w] = runs[(size_t)k * nspan + sp1].y - runs[(size_t)k * nspan + sp0].x;
        }
    order->resize(cost->size());
    for (size_t t = 0; t < order->size(); ++t) (*order)[t] = (int)t;
    std::stable_sort(order->begin(), order->end(), [&](int a, int b) { return (*cost)[a] > (*cost)[b]; });
}

cudaError_t tune_window(mbir_geometry* g, const std::vector<int2>& runs, cudaStream_t st);
cudaError_t install_window(mbir_geometry* g, int sub, const std::vector<int>& order, const std::vector<int>& cost);

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
    rec_count_kernel<<<P.K, 256, 0, st>>>(P, D, make_int3(1, 0, 0), d_cnt);
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
    rec_fill_kernel<<<P.K, kSortThreads, sm, st>>>(P, D, make_int3(1, 0, 0), g->d_rec_off, g->d_rec_key, g->d_rec_w,
                                                   g->d_runs);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    std::vector<int2> runs((size_t)P.K * nspan);
    e = cudaMemcpy(runs.data(), g->d_runs, sizeof(int2) * runs.size(), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMalloc((void**)&g->d_win_counter, sizeof(int));
    if (e != cudaSuccess) return e;
    g->bytes += sizeof(int);
    // two spans per warp until tune_forward_window times the candidates (only when this kernel is the A x)
    std::vector<int> order, cost;
    window_order(runs, P.K, nspan, 2, &order, &cost);
    return install_window(g, 2, order, cost);
}

// Times the CUDA-core A x windows (1, 2, 4 spans) once and keeps the fastest.
cudaError_t tune_forward_window(mbir_geometry* g, cudaStream_t st)
{
    const GeomParams& P = g->P;
    if (!g->d_runs) return cudaSuccess;
    const int nspan = (P.M + 31) / 32;
    std::vector<int2> runs((size_t)P.K * nspan);
    cudaError_t e = cudaMemcpy(runs.data(), g->d_runs, sizeof(int2) * runs.size(), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return e;
    return tune_window(g, runs, st);
}

size_t forward_sorted_smem(const mbir_geometry* g)
{
    const GeomParams& P = g->P;
    size_t tsz = P.precision == MBIR_PREC_BF16 ? 4 : 8;
    size_t tab = ((size_t)P.Gt * (P.Q + 1) * table_stride(P.Tw4) * tsz + 127) & ~(size_t)127;
    return tab + (size_t)kFwdSortedThreads * (sizeof(float4) + sizeof(int4));
}

template <bool BF16, int SUB>
static cudaError_t launch_sorted_t(const mbir_geometry* g, const int* order, const float* x, float* yf,
                                   __nv_bfloat16* yb, int stride, cudaStream_t st)
{
    using Tab = typename TabT<BF16>::type;
    const size_t sm = forward_sorted_smem(g);
    const int nspan = (g->P.M + 31) / 32;
    const long long wins = (long long)g->P.K * ((nspan + SUB - 1) / SUB);
    const int grid = (int)std::max<long long>(1, std::min<long long>(g->n_sm, (wins + 31) / 32));
    auto kern = forward_sorted_kernel<BF16, SUB>;
    cudaError_t ce = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(g->d_win_counter, 0, sizeof(int), st);
    if (ce != cudaSuccess) return ce;
    const Tab* tab = BF16 ? (const Tab*)(const void*)g->d_tab_bf16 : (const Tab*)(const void*)g->d_tab;
    kern<<<grid, kFwdSortedThreads, sm, st>>>(g->P, tab, g->d_rec_off, g->d_rec_key, g->d_rec_w, g->d_runs, order,
                                              (int)wins, g->d_win_counter, x, yf, yb, stride);
    return cudaGetLastError();
}

template <bool BF16>
static cudaError_t launch_sorted_sub(const mbir_geometry* g, int sub, const int* order, const float* x, float* yf,
                                     __nv_bfloat16* yb, int stride, cudaStream_t st)
{
    switch (sub) {
    case 1: return launch_sorted_t<BF16, 1>(g, order, x, yf, yb, stride, st);
    case 2: return launch_sorted_t<BF16, 2>(g, order, x, yf, yb, stride, st);
    default: return launch_sorted_t<BF16, 4>(g, order, x, yf, yb, stride, st);
    }
}

static cudaError_t launch_sorted(const mbir_geometry* g, int sub, const int* order, const float* x, float* yf,
                                 __nv_bfloat16* yb, int stride, cudaStream_t st)
{
    return g->P.precision == MBIR_PREC_BF16 ? launch_sorted_sub<true>(g, sub, order, x, yf, yb, stride, st)
                                            : launch_sorted_sub<false>(g, sub, order, x, yf, yb, stride, st);
}

// Window autotuner: times one A x per candidate window (1, 2 or 4 spans per
// warp) on a random image and keeps the fastest, with its window order and
// per-window costs.  Results do not depend on the choice (see span_gather).
cudaError_t tune_window(mbir_geometry* g, const std::vector<int2>& runs, cudaStream_t st)
{
    const GeomParams& P = g->P;
    const int nspan = (P.M + 31) / 32;
    const int cands[3] = {1, 2, 4};
    std::vector<int> order[3], cost[3];
    for (int c = 0; c < 3; ++c) window_order(runs, P.K, nspan, cands[c], &order[c], &cost[c]);
    int best = 1;                      // two spans per warp unless timing says otherwise
    const size_t N = (size_t)P.W * P.H, KMp = (size_t)P.K * P.Mp;
    float *x = nullptr, *y = nullptr;
    int* d_ord = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc((void**)&x, sizeof(float) * N);
    if (e == cudaSuccess) e = cudaMalloc((void**)&y, sizeof(float) * KMp);
    if (e == cudaSuccess) e = cudaMalloc((void**)&d_ord, sizeof(int) * order[0].size());
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) {
        // x = 1 on every pixel: every record is visited as in a real apply
        std::vector<float> ones(N, 1.0f);
        e = cudaMemcpy(x, ones.data(), sizeof(float) * N, cudaMemcpyHostToDevice);
    }
    float tbest = 0.0f;
    for (int c = 0; c < 3 && e == cudaSuccess; ++c) {
        e = cudaMemcpy(d_ord, order[c].data(), sizeof(int) * order[c].size(), cudaMemcpyHostToDevice);
        float t = 0.0f;
        for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {   // the first run warms up
            e = cudaEventRecord(e0, st);
            if (e == cudaSuccess) e = launch_sorted(g, cands[c], d_ord, x, y, nullptr, P.Mp, st);
            if (e == cudaSuccess) e = cudaEventRecord(e1, st);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
        }
        if (e == cudaSuccess) g->fwd_tune_ms[c] = t;
        if (e == cudaSuccess && (c == 0 || t < tbest)) {
            tbest = t;
            best = c;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(x);
    cudaFree(y);
    cudaFree(d_ord);
    if (e != cudaSuccess) return e;
    return install_window(g, cands[best], order[best], cost[best]);
}

// Makes `sub` the window of the A x launches, with its order and costs.
cudaError_t install_window(mbir_geometry* g, int sub, const std::vector<int>& order, const std::vector<int>& cost)
{
    int* d = nullptr;
    cudaError_t e = cudaMalloc((void**)&d, sizeof(int) * std::max<size_t>(order.size(), 1));
    if (e == cudaSuccess) e = cudaMemcpy(d, order.data(), sizeof(int) * order.size(), cudaMemcpyHostToDevice);
    int* h = (int*)malloc(sizeof(int) * std::max<size_t>(cost.size(), 1));
    if (e != cudaSuccess || !h) {
        cudaFree(d);
        free(h);
        return e != cudaSuccess ? e : cudaErrorMemoryAllocation;
    }
    std::copy(cost.begin(), cost.end(), h);
    if (g->d_win_order) {
        cudaFree(g->d_win_order);
        g->bytes -= sizeof(int) * (size_t)g->n_win;
    }
    free(g->h_win_cost);
    g->d_win_order = d;
    g->h_win_cost = h;
    g->fwd_sub = sub;
    g->n_win = (long long)order.size();
    g->bytes += sizeof(int) * order.size();
    return cudaSuccess;
}

// Replaces the autotuner's window by `sub` spans (1, 2 or 4).  Synchronous.
cudaError_t set_forward_window(mbir_geometry* g, int sub)
{
    const GeomParams& P = g->P;
    const int nspan = (P.M + 31) / 32;
    std::vector<int2> runs((size_t)P.K * nspan);
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(runs.data(), g->d_runs, sizeof(int2) * runs.size(), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return e;
    std::vector<int> order, cost;
    window_order(runs, P.K, nspan, sub, &order, &cost);
    return install_window(g, sub, order, cost);
}

cudaError_t launch_forward_sorted(const mbir_geometry* g, const float* x, float* yf, __nv_bfloat16* yb, int stride,
                                  cudaStream_t st)
{
    return launch_sorted(g, g->fwd_sub, g->d_win_order, x, yf, yb, stride, st);
}

// Record lists of the coordinate descent's colours: for spacing s, colour c = (c / s, c mod s) holds the
// records of the pixels (r, col) with r = c / s and col = c mod s (mod s), built like the full list
// (same order within each bucket); per colour the non-empty windows of `sub` spans, largest first.
// The lists of all colours follow each other; their offsets are absolute.
cudaError_t build_colour_records(mbir_geometry* g, int s, cudaStream_t st)
{
    const GeomParams& P = g->P;
    const int nc = s * s, nspan = (P.M + 31) / 32, sub = g->fwd_sub > 0 ? g->fwd_sub : 2;
    const int nwin = (nspan + sub - 1) / sub;
    const DevPtrs D = dev_ptrs(g);
    const size_t noff = (size_t)nc * (P.K + 1);
    long long* d_off = nullptr;
    cudaError_t e = cudaMalloc((void**)&d_off, sizeof(long long) * noff);
    if (e != cudaSuccess) return e;
    for (int c = 0; c < nc && e == cudaSuccess; ++c) {
        rec_count_kernel<<<P.K, 256, 0, st>>>(P, D, make_int3(s, c / s, c % s), d_off + (size_t)c * (P.K + 1));
        e = cudaGetLastError();
    }
    std::vector<long long> off(noff);
    if (e == cudaSuccess) e = cudaMemcpyAsync(off.data(), d_off, sizeof(long long) * noff, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) { cudaFree(d_off); return e; }
    long long acc = 0;
    for (int c = 0; c < nc; ++c)
        for (int k = 0; k <= P.K; ++k) {
            const long long n = k < P.K ? off[(size_t)c * (P.K + 1) + k] : 0;
            off[(size_t)c * (P.K + 1) + k] = acc;
            acc += n;
        }
    if (acc != g->n_records) { cudaFree(d_off); return cudaErrorInvalidValue; }   // the colours partition the pairs
    int2* d_key = nullptr;
    float4* d_w = nullptr;
    int2* d_runs = nullptr;
    e = cudaMemcpyAsync(d_off, off.data(), sizeof(long long) * noff, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMalloc((void**)&d_key, sizeof(int2) * std::max<long long>(acc, 1));
    if (e == cudaSuccess) e = cudaMalloc((void**)&d_w, sizeof(float4) * std::max<long long>(acc, 1));
    if (e == cudaSuccess) e = cudaMalloc((void**)&d_runs, sizeof(int2) * (size_t)nc * P.K * nspan);
    const size_t sm = sizeof(int) * (2 * (size_t)P.M + 1);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(rec_fill_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    for (int c = 0; c < nc && e == cudaSuccess; ++c) {
        rec_fill_kernel<<<P.K, kSortThreads, sm, st>>>(P, D, make_int3(s, c / s, c % s), d_off + (size_t)c * (P.K + 1),
                                                       d_key, d_w, d_runs + (size_t)c * P.K * nspan);
        e = cudaGetLastError();
    }
    std::vector<int2> runs((size_t)nc * P.K * nspan);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(runs.data(), d_runs, sizeof(int2) * runs.size(), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    std::vector<int> wins;
    std::vector<long long> woff(nc + 1, 0);
    if (e == cudaSuccess) {
        for (int c = 0; c < nc; ++c) {
            const int2* rc = runs.data() + (size_t)c * P.K * nspan;
            std::vector<std::pair<int, int>> cw;      // (records, window)
            for (int k = 0; k < P.K; ++k)
                for (int w = 0; w < nwin; ++w) {
                    const int sp0 = w * sub, sp1 = std::min(sp0 + sub, nspan) - 1;
                    const int n = rc[(size_t)k * nspan + sp1].y - rc[(size_t)k * nspan + sp0].x;
                    if (n > 0) cw.push_back({n, k * nwin + w});
                }
            std::stable_sort(cw.begin(), cw.end(), [](const std::pair<int, int>& a, const std::pair<int, int>& b) {
                return a.first > b.first;
            });
            for (auto& p : cw) wins.push_back(p.second);
            woff[c + 1] = (long long)wins.size();
        }
    }
    int* d_win = nullptr;
    if (e == cudaSuccess) e = cudaMalloc((void**)&d_win, sizeof(int) * std::max<size_t>(wins.size(), 1));
    if (e == cudaSuccess && !wins.empty())
        e = cudaMemcpy(d_win, wins.data(), sizeof(int) * wins.size(), cudaMemcpyHostToDevice);
    long long* h_woff = (long long*)malloc(sizeof(long long) * (nc + 1));
    if (e == cudaSuccess && !h_woff) e = cudaErrorMemoryAllocation;
    if (e != cudaSuccess) {
        cudaFree(d_off); cudaFree(d_key); cudaFree(d_w); cudaFree(d_runs); cudaFree(d_win); free(h_woff);
        return e;
    }
    std::copy(woff.begin(), woff.end(), h_woff);
    g->d_icd_rec_off = d_off;
    g->d_icd_rec_key = d_key;
    g->d_icd_rec_w = d_w;
    g->d_icd_runs = d_runs;
    g->d_icd_win = d_win;
    g->h_icd_win_off = h_woff;
    g->icd_win_sub = sub;
    g->icd_rec_bytes = sizeof(long long) * noff + (sizeof(int2) + sizeof(float4)) * (size_t)std::max<long long>(acc, 1) +
                       sizeof(int2) * runs.size() + sizeof(int) * std::max<size_t>(wins.size(), 1);
    return cudaSuccess;
}

template <bool BF16, int SUB>
static cudaError_t launch_colour_t(const mbir_geometry* g, int c, const float* x, float* yf, int stride,
                                   cudaStream_t st)
{
    using Tab = typename TabT<BF16>::type;
    const GeomParams& P = g->P;
    const int nspan = (P.M + 31) / 32;
    const long long w0 = g->h_icd_win_off[c], total = g->h_icd_win_off[c + 1] - w0;
    cudaError_t ce = cudaMemsetAsync(yf, 0, sizeof(float) * (size_t)P.K * stride, st);
    if (ce != cudaSuccess || total == 0) return ce;
    const size_t sm = forward_sorted_smem(g);
    auto kern = forward_sorted_kernel<BF16, SUB>;
    ce = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(g->d_win_counter, 0, sizeof(int), st);
    if (ce != cudaSuccess) return ce;
    const int grid = (int)std::max<long long>(1, std::min<long long>(g->n_sm, (total + 31) / 32));
    const Tab* tab = BF16 ? (const Tab*)(const void*)g->d_tab_bf16 : (const Tab*)(const void*)g->d_tab;
    kern<<<grid, kFwdSortedThreads, sm, st>>>(P, tab, g->d_icd_rec_off + (size_t)c * (P.K + 1), g->d_icd_rec_key,
                                              g->d_icd_rec_w, g->d_icd_runs + (size_t)c * P.K * nspan,
                                              g->d_icd_win + w0, (int)total, g->d_win_counter, x, yf, nullptr, stride);
    return cudaGetLastError();
}

// y = A x for an x that is zero off colour c (y zeroed first; only the colour's records are read).
cudaError_t launch_forward_colour(const mbir_geometry* g, int c, const float* x, float* yf, int stride,
                                  cudaStream_t st)
{
    const bool bf = g->P.precision == MBIR_PREC_BF16;
    switch (g->icd_win_sub) {
    case 1: return bf ? launch_colour_t<true, 1>(g, c, x, yf, stride, st) : launch_colour_t<false, 1>(g, c, x, yf, stride, st);
    case 2: return bf ? launch_colour_t<true, 2>(g, c, x, yf, stride, st) : launch_colour_t<false, 2>(g, c, x, yf, stride, st);
    default: return bf ? launch_colour_t<true, 4>(g, c, x, yf, stride, st) : launch_colour_t<false, 4>(g, c, x, yf, stride, st);
    }
}

}  // namespace mbir

extern "C" int mbir_set_forward_window(mbir_geometry* g, int spans)
{
    if (!g || (spans != 1 && spans != 2 && spans != 4)) return MBIR_ERR_INVALID_ARG;
    if (!g->d_rec_key) return MBIR_ERR_UNSUPPORTED;
    const cudaError_t e = mbir::set_forward_window(g, spans);
    return e == cudaSuccess ? MBIR_OK : (e == cudaErrorMemoryAllocation ? MBIR_ERR_OOM : MBIR_ERR_CUDA);
}
