// Batched and served reconstructions: many independent MAP problems of
// uneven size advance together, one iteration per engine step.
//
// Every step is one captured CUDA graph of grouped kernels.  Their grids are
// fixed (persistent or grid-stride), and they read the current set of active
// requests from device-side work lists that the host rewrites between steps,
// so the graph is captured once and replayed as requests come and go
// (continuous batching):
//   A^T e   persistent; each request's own work items form a pool drained
//           through a per-request counter (tensor cores: max |e| per request,
//           the (A-scan, tile) items of tcs_adjoint_pool into fixed-point
//           sums, then the sums into b; CUDA cores: pixel tile x
//           transmitter group, longest first; a step with both kinds of
//           request launches both, each taking its own).  A CTA starts at
//           the request its share of the total cost falls on and walks on
//           through the others until every pool is empty, loading a request's
//           table only when it joins that request's pool
//   grad    prior gradient + FP64 partials per (request, pixel block)
//   dir     Polak-Ribiere+ scalars per request, then directions + curvature
//   A d     persistent over each request's records (tensor cores: A-scans
//           of tcs_forward_pool, largest first; CUDA cores: span windows,
//           largest first; a step with both kinds of request launches both
//           kernels, each taking its own), pools and CTA placement as for A^T e
//   P q     direct-arrival projection per (request, A-scan) with FP64 norms
//   step    majorize-minimize step per request; x and e updated
// The apply kernels run the same per-item and per-span code as the
// single-request kernels, on the geometry's own work decomposition.
// Each request's arithmetic depends only on its own data and its own fixed
// work decomposition (the tensor-core A^T sums are integer, so their order
// does not matter), so a result is bitwise the same alone and in any mix.
// Admission is by device memory: a request is admitted when its state fits
// the engine's byte budget; state is allocated with stream-ordered
// cudaMallocAsync and released with cudaFreeAsync when the request retires.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <deque>
#include <map>
#include <memory>
#include <vector>

#include "apply_common.cuh"
#include "map_common.cuh"
#include "tc_apply.cuh"
#include "tc_stream.cuh"

namespace mbir {
PriorParams make_prior_params(const mbir_prior* pr);
bool prior_is_valid(const mbir_prior* pr);
}  // namespace mbir

using namespace mbir;

namespace {

constexpr int kEngThreads = 1024;          // apply kernels: 32 warps (A^T e: two tile workers)
constexpr int kEngStages = 3;              // residual-row ring of A^T e, per worker (2 if 3 do not fit)
constexpr size_t kEngHdr = 128;            // mbarriers and flags at the start of shared memory
constexpr size_t kEngSmem = 227 * 1024;
constexpr int kUpdChunk = 4096;            // elements per update item
constexpr size_t kTableMaxBytes = 160 * 1024;
constexpr int kMpMax = 4224;

// Per-request view used on the device (rewritten by the host every step).
struct ReqDesc {
    GeomParams P;
    DevPtrs D;
    const float2* tab;
    const __nv_bfloat162* tab_bf;
    const long long* rec_off;
    const int2* rkey;      // sorted records (CUDA-core A d)
    const float4* rw;
    const uint2* tkey;     // packed records (tensor-core applies)
    const void* tw;
    int fvar, bvar;        // the geometry's variants of the tensor-core A x and A^T pools
    const int2* runs;
    const float* direct;
    const float* dinv;
    float* x;
    float* e;
    __nv_bfloat16* ebf;
    float* q;
    float* b;
    float* grad;
    float* gprev;
    float* d0;
    float* d1;
    float* bpart;
    const float* msq;
    double* sc;
    double* part;          // [3 nblk grad | nblk curvature | K projection]
    const int* win_order;  // A d windows, largest first
    const int4* items;     // A^T e work items, longest first
    PriorParams pr;
    int it;                // iteration index of this step
    int ngroups;           // transmitter groups (partial images) of the A^T e items
    int n_items;
    int nwin;              // K x windows of `sub` 32-sample spans
    int sub;
    int nblk;              // pixel blocks of kRedThreads
    // tensor-core A^T tables (tc != 0: the accumulators are allocated)
    int tc;
    const int* tc_tile;
    unsigned long long* tc_acc;   // this request's per-pixel fixed-point sums (zero between steps)
    float tc_bound;        // the geometry's scale bound of those sums
    // tensor-core A^T and A x of tc_stream.cuh (tcb, tcs != 0)
    int tcb;
    Tb4Layout tb4l;
    const uint4* tb4_bop;
    int tcs;
    Tf4Layout tf4l;
    const uint4* tf4_bop;
    const uint32_t* tf4_crange;
    const int* tf4_split;
    const int* tf_order;
    long long nrec;        // records of the geometry
};

struct EngLists {
    ReqDesc* desc;
    int* pool;             // per request: next A d span, next A^T e item, bits of max |e| (zeroed every step)
    int* start;            // per CTA: first request of A^T e [0, G), of A d [G, 2G)
    int2* pixblk;          // {req, pixel block}
    int2* rowblk;          // {req, A-scan}
    int4* upd;             // {req, kind (0 x, 1 e), start, 0}
    int* counts;           // n_req, n_pixblk, n_rowblk, n_upd
};

__device__ __forceinline__ const float* dprev_of(const ReqDesc& R) { return (R.it & 1) ? R.d1 : R.d0; }
__device__ __forceinline__ float* dnew_of(const ReqDesc& R) { return (R.it & 1) ? R.d0 : R.d1; }

// ---------------------------------------------------------------------------
// A^T e over every active request
// ---------------------------------------------------------------------------
// Shared-memory geometry of one request in the apply kernels.
template <typename Tab, typename E>
__device__ __forceinline__ void eng_layout(const GeomParams& P, size_t* tab_bytes, size_t* ebytes, int* nst)
{
    *tab_bytes = ((size_t)P.Gt * (P.Q + 1) * table_stride(P.Tw4) * sizeof(Tab) + 127) & ~(size_t)127;
    *ebytes = ((size_t)P.Mp * sizeof(E) + 127) & ~(size_t)127;
    *nst = (kEngHdr + *tab_bytes + 2 * kEngStages * *ebytes <= kEngSmem) ? kEngStages : 2;
}

// Whether request rq's pool (slot 0: A d spans, 1: A^T e items) still has
// work; the answer is the same for every thread of the CTA.
__device__ __forceinline__ bool eng_pool_live(const int* pool, int rq, int slot, int total, volatile int* flag)
{
    if (threadIdx.x == 0) *flag = *reinterpret_cast<const volatile int*>(pool + 3 * rq + slot) < total;
    __syncthreads();
    const bool live = *flag != 0;
    __syncthreads();
    return live;
}

template <bool BF16>
__global__ void __launch_bounds__(kEngThreads, 1) eng_bwd_kernel(EngLists L)
{
    using Tab = typename TabT<BF16>::type;
    using E = typename ET<BF16>::type;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem);                               // [2][kEngStages]
    volatile int* flags = reinterpret_cast<volatile int*>(bars + 2 * kEngStages);     // abort[2], next[2], live
    Tab* tab = reinterpret_cast<Tab*>(smem + kEngHdr);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int h = warp / kBwdTileRows, hw = warp % kBwdTileRows, ht = tid % kBwdWorkerThreads;
    if (tid == 0) {
        for (int b = 0; b < 2 * kEngStages; ++b) mbar_init(smem_u32(bars + b), 1);
        flags[0] = flags[1] = 0;
        fence_mbar_init();
    }
    __syncthreads();
    const uint32_t bar0 = smem_u32(bars + h * kEngStages);
    uint32_t par = 0;
    const int nreq = L.counts[0];
    if (nreq <= 0) return;
    const int r0 = L.start[blockIdx.x] % nreq;
    int cur = -1;
    for (int t = 0; t < nreq; ++t) {
        const int rq = (r0 + t) % nreq;
        const ReqDesc& R = L.desc[rq];
        // requests with the tensor-core A^T are eng_bwd_tcs_kernel's
        if (R.tc || !eng_pool_live(L.pool, rq, 1, R.n_items, flags + 4)) continue;
        const GeomParams& P = R.P;
        size_t tab_bytes, ebytes;
        int nst;
        eng_layout<Tab, E>(P, &tab_bytes, &ebytes, &nst);
        if (rq != cur) {
            load_table_smem(tab, BF16 ? (const void*)R.tab_bf : (const void*)R.tab, tab_bytes, tid, kEngThreads);
            cur = rq;
            __syncthreads();
        }
        E* ering = reinterpret_cast<E*>(smem + kEngHdr + tab_bytes + (size_t)h * nst * ebytes);
        const E* e_g = BF16 ? (const E*)(const void*)R.ebf : (const E*)(const void*)R.e;
        for (;;) {
            if (ht == 0) flags[2 + h] = atomicAdd(L.pool + 3 * rq + 1, 1);
            worker_barrier(h);
            const int it = flags[2 + h];
            worker_barrier(h);
            if (it >= R.n_items) break;
            if (!backproject_item<1, kModeTAB, BF16>(P, R.D, tab, e_g, __ldg(R.items + it), R.bpart, ering, bar0, nst,
                                                     ebytes, flags + h, par, h, hw, lane, ht, make_int3(1, 0, 0)))
                break;
        }
        __syncthreads();                 // both workers are done before the table is replaced
        if (flags[0] | flags[1]) return; // a residual copy never landed (status set)
    }
}

// b = sum of the group partials (fixed order); zero where the pixel's tile
// cannot reach the record.  Grid-stride over (request, pixel block).
__global__ void eng_bwd_reduce_kernel(EngLists L)
{
    const int nb = L.counts[1];
    for (int bb = blockIdx.x; bb < nb; bb += gridDim.x) {
        const int2 rb = L.pixblk[bb];
        const ReqDesc& R = L.desc[rb.x];
        if (R.tc) continue;
        const GeomParams& P = R.P;
        const int N = P.W * P.H;
        const int v = rb.y * kRedThreads + threadIdx.x;
        if (v >= N) continue;
        const int row = v / P.W;
        const int row0 = (row / kBwdTileRows) * kBwdTileRows;
        float s = 0.0f, c = 0.0f;
        if (R.D.rows[row0].tvert < (float)(P.M - 1))
            for (int g = 0; g < R.ngroups; ++g) neumaier_add(s, c, R.bpart[(size_t)g * N + v]);
        R.b[v] = s + c;
    }
}

// grad = -b / sigma^2 + grad R(x); FP64 partials of <g,g>, <g,gprev>, <g,dprev>
__global__ void eng_grad_kernel(EngLists L)
{
    __shared__ double sh[32];
    const int nb = L.counts[1];
    for (int bb = blockIdx.x; bb < nb; bb += gridDim.x) {
        const int2 rb = L.pixblk[bb];
        const ReqDesc& R = L.desc[rb.x];
        const GeomParams& P = R.P;
        const int N = P.W * P.H;
        const int v = rb.y * kRedThreads + threadIdx.x;
        const float* dprev = dprev_of(R);
        double a0 = 0, a1 = 0, a2 = 0;
        if (v < N) {
            const int r = v / P.W, c = v - r * P.W;
            const float xs = R.x[v], ms = R.msq[r];
            float gr = 0.0f;
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                const int r2 = r + c_nb_dr[t], c2 = c + c_nb_dc[t];
                if (r2 < 0 || r2 >= P.H || c2 < 0 || c2 >= P.W) continue;
                float dr;
                qggmrf(R.pr, xs - R.x[r2 * P.W + c2], R.pr.sigma0 * ms * R.msq[r2], &dr, nullptr, nullptr);
                gr += nb_weight(c_nb_dr[t], c_nb_dc[t]) * dr;
            }
            const float g = -R.b[v] * R.pr.inv_s2 + gr;
            R.grad[v] = g;
            a0 = (double)g * g;
            a1 = (double)g * R.gprev[v];
            a2 = (double)g * dprev[v];
        }
        const double s0 = block_sum(a0, sh), s1 = block_sum(a1, sh), s2 = block_sum(a2, sh);
        if (threadIdx.x == 0) {
            R.part[3 * rb.y] = s0;
            R.part[3 * rb.y + 1] = s1;
            R.part[3 * rb.y + 2] = s2;
        }
    }
}

// Polak-Ribiere+ coefficient with a descent restart, one block per request
__global__ void eng_findir_kernel(EngLists L)
{
    __shared__ double sh[32];
    const int nr = L.counts[0];
    for (int r = blockIdx.x; r < nr; r += gridDim.x) {
        const ReqDesc& R = L.desc[r];
        double a0 = 0, a1 = 0, a2 = 0;
        for (int t = threadIdx.x; t < R.nblk; t += blockDim.x) {
            a0 += R.part[3 * t];
            a1 += R.part[3 * t + 1];
            a2 += R.part[3 * t + 2];
        }
        const double gg = block_sum(a0, sh), ggp = block_sum(a1, sh), gdp = block_sum(a2, sh);
        if (threadIdx.x == 0) {
            double* sc = R.sc;
            double beta = 0.0;
            if (R.it > 0 && sc[S_GGPREV] > 0.0) beta = fmax((gg - ggp) / sc[S_GGPREV], 0.0);
            double gd = -gg + beta * gdp;
            if (!(gd < 0.0)) { beta = 0.0; gd = -gg; }
            sc[S_GG] = gg;
            sc[S_BETA] = beta;
            sc[S_GD] = gd;
            sc[S_GGPREV] = gg;
            if (!isfinite(gg)) sc[S_BAD] = 1.0;
        }
    }
}

// d = -grad + beta dprev; gprev = grad; curvature partial over forward cliques
__global__ void eng_dir_kernel(EngLists L)
{
    __shared__ double sh[32];
    const int nb = L.counts[1];
    for (int bb = blockIdx.x; bb < nb; bb += gridDim.x) {
        const int2 rb = L.pixblk[bb];
        const ReqDesc& R = L.desc[rb.x];
        const GeomParams& P = R.P;
        const int N = P.W * P.H;
        const int v = rb.y * kRedThreads + threadIdx.x;
        const float* dprev = dprev_of(R);
        float* dnew = dnew_of(R);
        const float beta = (float)R.sc[S_BETA];
        double acc = 0.0;
        if (v < N) {
            const int r = v / P.W, c = v - r * P.W;
            const float gv = R.grad[v];
            const float dv = -gv + beta * dprev[v];
            dnew[v] = dv;
            R.gprev[v] = gv;
            const float xs = R.x[v], ms = R.msq[r];
            const int dr4[4] = {0, 1, 1, 1}, dc4[4] = {1, -1, 0, 1};
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const int r2 = r + dr4[t], c2 = c + dc4[t];
                if (r2 >= P.H || c2 < 0 || c2 >= P.W) continue;
                const int v2 = r2 * P.W + c2;
                const float d2 = -R.grad[v2] + beta * dprev[v2];
                float kap;
                qggmrf(R.pr, xs - R.x[v2], R.pr.sigma0 * ms * R.msq[r2], nullptr, &kap, nullptr);
                const float dd = dv - d2;
                acc += (double)(nb_weight(dr4[t], dc4[t]) * kap) * (double)dd * (double)dd;
            }
        }
        const double s = block_sum(acc, sh);
        if (threadIdx.x == 0) R.part[3 * R.nblk + rb.y] = s;
    }
}

// Warps of the CTA drain request R's A d pool of windows (SUB spans each).
template <bool BF16, int SUB>
__device__ __forceinline__ void eng_fwd_pool(const ReqDesc& R, int* pool, const typename TabT<BF16>::type* tab,
                                             int lane, int4* sr, float4* sw)
{
    const GeomParams& P = R.P;
    const int S = table_stride(P.Tw4);
    const int nspan = (P.M + 31) >> 5;
    const int nwin = (nspan + SUB - 1) / SUB;
    const float* x = dnew_of(R);
    for (;;) {
        int idx = 0;
        if (lane == 0) idx = atomicAdd(pool, 1);
        idx = __shfl_sync(0xffffffffu, idx, 0);
        if (idx >= R.nwin) break;
        const int gw = __ldg(R.win_order + idx);
        const int k = gw / nwin, w = gw - k * nwin;
        const int2 rb = window_runs(R.runs, k, nspan, w, SUB);
        float v[SUB];
        span_gather<BF16, SUB>(tab, S, P.Tw, R.rkey, R.rw, __ldg(R.rec_off + k), rb.x, rb.y, x, w * SUB * 32 + lane,
                               lane, sr, sw, v);
        window_store<SUB>(R.q + (size_t)k * P.Mp, nullptr, P.M, nspan, P.Mp, w * SUB, lane, v);
    }
}

// q = A d over every active request: warps take windows of a request's pool,
// largest first; the CTA moves on when the pool is empty
template <bool BF16>
__global__ void __launch_bounds__(kEngThreads, 1) eng_fwd_kernel(EngLists L)
{
    using Tab = typename TabT<BF16>::type;
    constexpr int WARPS = kEngThreads / 32;
    extern __shared__ __align__(128) unsigned char smem[];
    volatile int* flag = reinterpret_cast<volatile int*>(smem);
    Tab* tab = reinterpret_cast<Tab*>(smem + kEngHdr);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int4* sr = reinterpret_cast<int4*>(smem + kEngHdr + kTableMaxBytes) + warp * 32;
    float4* sw = reinterpret_cast<float4*>(smem + kEngHdr + kTableMaxBytes) + WARPS * 32 + warp * 32;
    const int nreq = L.counts[0];
    if (nreq <= 0) return;
    const int r0 = L.start[gridDim.x + blockIdx.x] % nreq;
    int cur = -1;
    for (int t = 0; t < nreq; ++t) {
        const int rq = (r0 + t) % nreq;
        const ReqDesc& R = L.desc[rq];
        // requests with the tensor-core A x (their records are in that kernel's order) are eng_fwd_tcs_kernel's
        if (R.tcs || !eng_pool_live(L.pool, rq, 0, R.nwin, flag)) continue;
        const GeomParams& P = R.P;
        if (rq != cur) {
            const size_t tab_bytes =
                ((size_t)P.Gt * (P.Q + 1) * table_stride(P.Tw4) * sizeof(Tab) + 127) & ~(size_t)127;
            load_table_smem(tab, BF16 ? (const void*)R.tab_bf : (const void*)R.tab, tab_bytes, tid, kEngThreads);
            cur = rq;
            __syncthreads();
        }
        if (R.sub == 1) eng_fwd_pool<BF16, 1>(R, L.pool + 3 * rq, tab, lane, sr, sw);
        else if (R.sub == 2) eng_fwd_pool<BF16, 2>(R, L.pool + 3 * rq, tab, lane, sr, sw);
        else eng_fwd_pool<BF16, 4>(R, L.pool + 3 * rq, tab, lane, sr, sw);
        __syncthreads();                 // every warp is done before the table is replaced
    }
}

// A^T e on the tensor cores (FP32 or BF16 form, tc_stream.cuh) over every active request
template <bool BF16>
__global__ void __launch_bounds__(TbShape<BF16>::threads, 1) eng_bwd_tcs_kernel(EngLists L)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    tc_header_init(smem, kTsCols);
    const uint32_t tmem = *reinterpret_cast<volatile uint32_t*>(smem + 8);
    volatile int* flag = reinterpret_cast<volatile int*>(smem + 24);
    uint32_t mphase = 0, bphase = 0;
    const int nreq = L.counts[0];
    if (nreq > 0) {
        const int r0 = L.start[blockIdx.x] % nreq;
        for (int t = 0; t < nreq; ++t) {
            const int rq = (r0 + t) % nreq;
            const ReqDesc& R = L.desc[rq];
            const int nitems = R.P.K * ((R.P.M + kTsTile - 1) / kTsTile);
            if (!R.tc || !eng_pool_live(L.pool, rq, 1, nitems, flag)) continue;
            const void* tab = BF16 ? (const void*)R.tab_bf : (const void*)R.tab;
            const void* e = BF16 ? (const void*)R.ebf : (const void*)R.e;
            const TbView V{R.P, R.tb4l, R.tb4_bop, tab, e, R.rec_off, R.tc_tile, R.tf4_crange, R.tkey, R.tw,
                           R.tc_acc, reinterpret_cast<const unsigned int*>(L.pool + 3 * rq + 2), R.tc_bound,
                           L.pool + 3 * rq + 1};
            const bool ok = R.bvar ? tcs_adjoint_pool<BF16, 1>(V, smem, tmem, mphase, bphase, R.D.status)
                                   : tcs_adjoint_pool<BF16, 0>(V, smem, tmem, mphase, bphase, R.D.status);
            if (!ok) break;
            __syncthreads();
        }
    }
    tc_header_release(smem, tmem, kTsCols);
}

// bits of max |e| of every active request (the scale of its fixed-point A^T sums): block per (request,
// A-scan) row, atomically into the request's pool word
template <bool BF16>
__global__ void eng_emax_kernel(EngLists L)
{
    const int nb = L.counts[2];
    for (int bb = blockIdx.x; bb < nb; bb += gridDim.x) {
        const int2 rk = L.rowblk[bb];
        const ReqDesc& R = L.desc[rk.x];
        if (!R.tc) continue;
        const int Mp = R.P.Mp;
        unsigned int m = 0;
        for (int n = threadIdx.x; n < Mp; n += blockDim.x) {
            const float v = BF16 ? __bfloat162float(R.ebf[(size_t)rk.y * Mp + n]) : R.e[(size_t)rk.y * Mp + n];
            m = max(m, __float_as_uint(fabsf(v)));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
        if ((threadIdx.x & 31) == 0 && m) atomicMax(reinterpret_cast<unsigned int*>(L.pool + 3 * rk.x + 2), m);
    }
}

// b of every active request from its fixed-point sums (tcs_finish_pixel), which are cleared for the next
// step; block per (request, pixel block)
__global__ void eng_bwd_tc_finish_kernel(EngLists L)
{
    const int nb = L.counts[1];
    for (int bb = blockIdx.x; bb < nb; bb += gridDim.x) {
        const int2 rb = L.pixblk[bb];
        const ReqDesc& R = L.desc[rb.x];
        const int v = rb.y * kRedThreads + threadIdx.x;
        if (R.tc && v < R.P.W * R.P.H) {
            const unsigned int eb = *reinterpret_cast<const unsigned int*>(L.pool + 3 * rb.x + 2);
            R.b[v] = tcs_finish_pixel(R.tc_acc[v], eb, R.tc_bound);
            R.tc_acc[v] = 0ull;
        }
    }
}

// q = A d on the tensor cores over every active request (FP32 or BF16 form)
template <bool BF16>
__global__ void __launch_bounds__(TsShape<BF16>::threads, 1) eng_fwd_tcs_kernel(EngLists L)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    tc_header_init(smem, kTsCols);
    const uint32_t tmem = *reinterpret_cast<volatile uint32_t*>(smem + 8);
    volatile int* flag = reinterpret_cast<volatile int*>(smem + 24);
    uint32_t mphase = 0, bphase = 0;
    const int nreq = L.counts[0];
    if (nreq > 0) {
        const int r0 = L.start[gridDim.x + blockIdx.x] % nreq;
        for (int t = 0; t < nreq; ++t) {
            const int rq = (r0 + t) % nreq;
            const ReqDesc& R = L.desc[rq];
            if (!R.tcs || !eng_pool_live(L.pool, rq, 0, R.P.K, flag)) continue;
            const void* tab = BF16 ? (const void*)R.tab_bf : (const void*)R.tab;
            const TsView V{R.P, R.tf4l, R.tf4_bop, tab, R.rec_off, R.tf4_crange, R.tf4_split, R.tkey, R.tw,
                           R.tf_order, dnew_of(R), R.q, 0, R.P.Mp, L.pool + 3 * rq};
            const bool ok = R.fvar ? tcs_forward_pool<BF16, 1>(V, smem, tmem, mphase, bphase, R.D.status)
                                   : tcs_forward_pool<BF16, 0>(V, smem, tmem, mphase, bphase, R.D.status);
            if (!ok) break;
            __syncthreads();
        }
    }
    tc_header_release(smem, tmem, kTsCols);
}

// in-place direct-arrival projection of q per (request, A-scan), FP64 |q|^2
__global__ void eng_proj_kernel(EngLists L)
{
    __shared__ double sh[32];
    __shared__ float gsh;
    const int nb = L.counts[2];
    for (int bb = blockIdx.x; bb < nb; bb += gridDim.x) {
        const int2 rk = L.rowblk[bb];
        const ReqDesc& R = L.desc[rk.x];
        const GeomParams& P = R.P;
        const int k = rk.y, j = k % P.n_rx;
        const float* dj = R.direct + (size_t)j * P.Mp;
        float* qk = R.q + (size_t)k * P.Mp;
        double dr = 0.0;
        for (int n = threadIdx.x; n < P.M; n += blockDim.x) dr += (double)dj[n] * (double)qk[n];
        const double tot = block_sum(dr, sh);
        if (threadIdx.x == 0) gsh = (float)(tot * (double)R.dinv[j]);
        __syncthreads();
        const float g = gsh;
        double ee = 0.0;
        for (int n = threadIdx.x; n < P.M; n += blockDim.x) {
            const float o = qk[n] - g * dj[n];
            qk[n] = o;
            ee += (double)o * o;
        }
        const double e2 = block_sum(ee, sh);
        if (threadIdx.x == 0) R.part[4 * R.nblk + k] = e2;
        __syncthreads();
    }
}

// majorize-minimize step per request
__global__ void eng_finstep_kernel(EngLists L)
{
    __shared__ double sh[32];
    const int nr = L.counts[0];
    for (int r = blockIdx.x; r < nr; r += gridDim.x) {
        const ReqDesc& R = L.desc[r];
        double a = 0, b = 0;
        for (int t = threadIdx.x; t < R.P.K; t += blockDim.x) a += R.part[4 * R.nblk + t];
        for (int t = threadIdx.x; t < R.nblk; t += blockDim.x) b += R.part[3 * R.nblk + t];
        const double qq = block_sum(a, sh), cv = block_sum(b, sh);
        if (threadIdx.x == 0) {
            double* sc = R.sc;
            const double den = qq * (double)R.pr.inv_s2 + cv;
            double alpha = den > 0.0 ? -sc[S_GD] / den : 0.0;
            if (!isfinite(alpha)) { alpha = 0.0; sc[S_BAD] = 1.0; }
            sc[S_QQ] = qq;
            sc[S_CURV] = cv;
            sc[S_ALPHA] = alpha;
        }
    }
}

// x += alpha d and e -= alpha q (BF16 copy of e when stored in BF16)
__global__ void eng_update_kernel(EngLists L)
{
    const int nu = L.counts[3];
    for (int bb = blockIdx.x; bb < nu; bb += gridDim.x) {
        const int4 u = L.upd[bb];
        const ReqDesc& R = L.desc[u.x];
        const float a = (float)R.sc[S_ALPHA];
        if (u.y == 0) {
            const int N = R.P.W * R.P.H;
            const float* d = dnew_of(R);
            for (int t = u.z + threadIdx.x; t < min(N, u.z + kUpdChunk); t += blockDim.x) R.x[t] = fmaf(a, d[t], R.x[t]);
        } else {
            const long long KM = (long long)R.P.K * R.P.Mp;
            const long long end = min(KM, (long long)u.z + kUpdChunk);
            for (long long t = u.z + threadIdx.x; t < end; t += blockDim.x) {
                const float ev = fmaf(-a, R.q[t], R.e[t]);
                R.e[t] = ev;
                if (R.ebf) R.ebf[t] = __float2bfloat16_rn(ev);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct Request {
    int64_t ticket = 0;
    const mbir_geometry* g = nullptr;
    const void* y = nullptr;
    mbir_prior prior{};
    int n_iter = 0, it = 0;
    float* x = nullptr;
    float* gout = nullptr;
    int state = 0;          // 0 queued, 1 active, 2 retiring, 3 done, < 0 error code
    int ngroups = 1, nblk = 0;
    size_t bytes = 0;
    double cost = 0;        // estimated work of one iteration (A^T e estimate, twice)
    double waited = 0;      // work of the steps that ran while this request was passed over
    double bwd_est = -1, fwd_est = -1;   // the geometry's A^T e and A d cost estimates (summed once)
    float *e = nullptr, *q = nullptr, *b = nullptr, *grad = nullptr, *gprev = nullptr, *d0 = nullptr,
          *d1 = nullptr, *bpart = nullptr, *msq = nullptr;
    unsigned long long* acc = nullptr;   // tensor-core A^T: per-pixel fixed-point sums
    __nv_bfloat16* ebf = nullptr;
    double *sc = nullptr, *part = nullptr;
    std::vector<float> msq_host;
    cudaEvent_t done_ev = nullptr;
};

size_t request_bytes(const mbir_geometry* g, int ngroups)
{
    const GeomParams& P = g->P;
    const size_t N = (size_t)P.W * P.H, KMp = (size_t)P.K * P.Mp;
    const size_t nblk = (N + kRedThreads - 1) / kRedThreads;
    size_t b = 2 * KMp * 4 + 6 * N * 4 + (size_t)ngroups * N * 4 + (size_t)P.H * 4 + S_COUNT * 8 +
               (4 * nblk + P.K + 8) * 8;
    if (P.precision == MBIR_PREC_BF16) b += KMp * 2;
    if (g->d_tb4_bop) b += N * 8;   // tensor-core adjoint accumulators
    return b;
}


}  // namespace

struct mbir_engine {
    int device = 0, n_sm = 1;
    size_t budget = 0, used = 0;
    int max_active = 64;
    int64_t next_ticket = 1;
    std::deque<Request*> queue;
    std::vector<Request*> active;        // admitted: state on the device
    std::vector<Request*> sel;           // run in the current step (see select_step)
    std::map<int64_t, std::unique_ptr<Request>> all;
    bool dirty = true;                   // work lists must be rebuilt
    // device work lists (fixed capacity; growing them re-captures the graph)
    EngLists L{};
    size_t cap_desc = 0, cap_pool = 0, cap_pix = 0, cap_row = 0, cap_upd = 0;
    cudaGraphExec_t graph = nullptr;
    int graph_bf16 = -1, graph_tc = -1;
    size_t smem_bwd = 0, smem_fwd = 0;
    // dynamic shared memory of the tensor-core kernels as captured: the largest layout among the
    // admitted requests, not the 227 KB maximum, so that the rest of each SM's 256 KB stays L1
    size_t smem_tc[2] = {0, 0};          // tensor-core A x, A^T
    // host mirrors
    std::vector<ReqDesc> h_desc;
};

namespace {

template <typename T>
cudaError_t ensure_cap(T** p, size_t* cap, size_t need, bool* grew)
{
    if (need <= *cap && *p) return cudaSuccess;
    size_t n = std::max<size_t>(need * 2, 64);
    if (*p) cudaFree(*p);
    cudaError_t e = cudaMalloc((void**)p, sizeof(T) * n);
    if (e == cudaSuccess) {
        *cap = n;
        *grew = true;
    }
    return e;
}

// contiguous, cost-balanced split of `cost` into `parts` ranges
std::vector<int> balance(const std::vector<double>& cost, int parts)
{
    std::vector<int> cut(parts + 1, (int)cost.size());
    cut[0] = 0;
    double total = 0;
    for (double c : cost) total += c;
    double acc = 0;
    int p = 1;
    for (size_t i = 0; i < cost.size() && p < parts; ++i) {
        acc += cost[i];
        while (p < parts && acc >= total * p / parts) cut[p++] = (int)i + 1;
    }
    for (; p < parts; ++p) cut[p] = (int)cost.size();
    return cut;
}

void free_request_state(Request* r, cudaStream_t st)
{
    void* ptrs[] = {r->e, r->q, r->b, r->grad, r->gprev, r->d0, r->d1, r->bpart, r->msq, r->ebf, r->sc, r->part,
                    r->acc};
    for (void* p : ptrs)
        if (p) cudaFreeAsync(p, st);
    r->e = r->q = r->b = r->grad = r->gprev = r->d0 = r->d1 = r->bpart = r->msq = nullptr;
    r->acc = nullptr;
    r->ebf = nullptr;
    r->sc = r->part = nullptr;
}

int admit(mbir_engine* E, Request* r, cudaStream_t st)
{
    const mbir_geometry* g = r->g;
    const GeomParams& P = g->P;
    const size_t N = (size_t)P.W * P.H, KMp = (size_t)P.K * P.Mp;
    r->ngroups = g->n_groups;
    r->nblk = (int)((N + kRedThreads - 1) / kRedThreads);
    cudaError_t e = cudaSuccess;
#define AL(ptr, n) if (e == cudaSuccess) e = cudaMallocAsync((void**)&(ptr), sizeof(*(ptr)) * std::max<size_t>((n), 1), st)
    AL(r->e, KMp);
    AL(r->q, KMp);
    AL(r->b, N);
    AL(r->grad, N);
    AL(r->gprev, N);
    AL(r->d0, N);
    AL(r->d1, N);
    AL(r->bpart, (size_t)r->ngroups * N);
    AL(r->msq, (size_t)P.H);
    AL(r->sc, (size_t)S_COUNT);
    AL(r->part, (size_t)4 * r->nblk + P.K + 8);
    if (P.precision == MBIR_PREC_BF16) AL(r->ebf, KMp);
    if (g->d_tb4_bop) AL(r->acc, N);
#undef AL
    if (e != cudaSuccess) { free_request_state(r, st); return e == cudaErrorMemoryAllocation ? MBIR_ERR_OOM : MBIR_ERR_CUDA; }
    r->msq_host.resize(P.H);
    mbir::compute_msq(g, &r->prior, r->msq_host.data());
    e = cudaMemcpyAsync(r->msq, r->msq_host.data(), sizeof(float) * P.H, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(r->sc, 0, sizeof(double) * S_COUNT, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(r->gprev, 0, sizeof(float) * N, st);
    if (e == cudaSuccess && r->acc) e = cudaMemsetAsync(r->acc, 0, sizeof(unsigned long long) * N, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(r->d0, 0, sizeof(float) * N, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(r->d1, 0, sizeof(float) * N, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(r->x, 0, sizeof(float) * N, st);
    // e = P y (x starts at zero)
    if (e == cudaSuccess)
        e = mbir::launch_project_rows(g, r->y, P.precision == MBIR_PREC_BF16 ? 1 : 0, P.M, nullptr, 0, r->e, P.Mp,
                                      nullptr, nullptr, st);
    if (e == cudaSuccess && r->ebf) e = mbir::launch_to_bf16(r->e, r->ebf, (long long)KMp, st);
    if (e != cudaSuccess) { free_request_state(r, st); return MBIR_ERR_CUDA; }
    r->it = 0;
    r->waited = 0;
    r->cost = 0;
    const int TR = backproject_tile_rows(), ntr = (P.H + TR - 1) / TR;
    for (int tr = 0; tr < ntr; ++tr)
        if (g->h_tvert[tr * TR] < (float)(P.M - 1))
            for (size_t t = (size_t)tr * g->bwd_ntc * P.n_tx; t < (size_t)(tr + 1) * g->bwd_ntc * P.n_tx; ++t)
                r->cost += 2.0 * g->h_bwd_cost[t];
    r->state = 1;
    return MBIR_OK;
}

void fill_desc(ReqDesc& d, const Request* r)
{
    const mbir_geometry* g = r->g;
    d.P = g->P;
    d.D = dev_ptrs(g);
    d.tab = g->d_tab;
    d.tab_bf = g->d_tab_bf16;
    d.rec_off = g->d_rec_off;
    d.rkey = g->d_rec_key;
    d.rw = g->d_rec_w;
    d.tkey = g->d_tc_key;
    d.tw = g->d_tc_w;
    d.fvar = g->tc_fvar;
    d.bvar = g->tc_bvar;
    d.runs = g->d_runs;
    d.direct = g->d_direct;
    d.dinv = g->d_dinv;
    d.x = r->x;
    d.e = r->e;
    d.ebf = r->ebf;
    d.q = r->q;
    d.b = r->b;
    d.grad = r->grad;
    d.gprev = r->gprev;
    d.d0 = r->d0;
    d.d1 = r->d1;
    d.bpart = r->bpart;
    d.msq = r->msq;
    d.sc = r->sc;
    d.part = r->part;
    d.pr = make_prior_params(&r->prior);
    d.it = r->it;
    d.win_order = g->d_win_order;
    d.items = g->d_items;
    d.ngroups = r->ngroups;
    d.n_items = g->n_items;
    d.nwin = (int)g->n_win;
    d.sub = g->fwd_sub;
    d.nblk = r->nblk;
    d.tc = g->d_tb4_bop ? 1 : 0;
    d.tc_tile = g->d_tc_tile;
    d.tc_acc = r->acc;
    d.tc_bound = g->tc_bound;
    d.tcb = g->d_tb4_bop ? 1 : 0;
    d.tb4l = g->tb4;
    d.tb4_bop = g->d_tb4_bop;
    d.tcs = g->d_tf4_bop ? 1 : 0;
    d.tf4l = g->tf4;
    d.tf4_bop = g->d_tf4_bop;
    d.tf4_crange = g->d_tf4_crange;
    d.tf4_split = g->d_tf4_split;
    d.tf_order = g->d_tf_order;
    d.nrec = g->n_records;
}

// First request of each CTA: the requests' costs laid end to end and cut into
// G equal shares; CTA c starts at the request its share begins in.
std::vector<int> start_requests(const std::vector<double>& cost, int G)
{
    std::vector<int> st(G, 0);
    double total = 0;
    for (double c : cost) total += c;
    double acc = 0;
    size_t r = 0;
    for (int c = 0; c < G; ++c) {
        const double at = total * c / G;
        while (r + 1 < cost.size() && acc + cost[r] <= at) acc += cost[r++];
        st[c] = (int)r;
    }
    return st;
}

// Requests run in this step.  All admitted requests hold their state on the
// device, but a step runs one iteration of only some of them, so that small
// requests are not paced by the long iterations of large ones: in order of
// remaining work (estimated iteration cost x iterations left) less half the
// work a request has waited through while passed over (aging, so large
// requests are not starved), a request joins the step if the step's A^T e
// items stay within four per tile worker of the GPU (the first always joins).
constexpr double kAging = 0.5;

void select_step(mbir_engine* E)
{
    std::vector<Request*> order(E->active.begin(), E->active.end());
    auto prio = [](const Request* r) { return r->cost * (r->n_iter - r->it) - kAging * r->waited; };
    std::stable_sort(order.begin(), order.end(), [&](const Request* a, const Request* b) { return prio(a) < prio(b); });
    const long long budget = 4LL * 2 * E->n_sm;
    std::vector<Request*> sel;
    long long items = 0;
    double step_cost = 0;
    for (Request* r : order) {
        if (!sel.empty() && items + r->g->n_items > budget) continue;
        sel.push_back(r);
        items += r->g->n_items;
        step_cost += r->cost;
    }
    for (Request* r : E->active)
        if (std::find(sel.begin(), sel.end(), r) == sel.end()) r->waited += step_cost;
    if (sel != E->sel) {
        E->sel = sel;
        E->dirty = true;
    }
}

// Rebuilds the per-step work lists for the requests run in the step.
int rebuild_lists(mbir_engine* E, cudaStream_t st, bool* grew)
{
    const int G = E->n_sm;
    std::vector<double> bwd_cost, fwd_cost;
    std::vector<int2> pix, rows;
    std::vector<int4> upd;
    for (size_t ri = 0; ri < E->sel.size(); ++ri) {
        const Request* r = E->sel[ri];
        const mbir_geometry* g = r->g;
        const GeomParams& P = g->P;
        // A^T e: the geometry's estimates of its items (tile x transmitter group); A d: records visited per
        // window plus a fixed cost per window.  Summed on the request's first step only.
        Request* rw = E->sel[ri];
        if (rw->bwd_est < 0) {
            const int TR = backproject_tile_rows(), ntr = (P.H + TR - 1) / TR;
            double cb = 0;
            for (int tr = 0; tr < ntr; ++tr) {
                if (!(g->h_tvert[tr * TR] < (float)(P.M - 1))) continue;
                for (size_t t = (size_t)tr * g->bwd_ntc * P.n_tx; t < (size_t)(tr + 1) * g->bwd_ntc * P.n_tx; ++t)
                    cb += g->h_bwd_cost[t];
            }
            double cf = 0;
            for (long long w = 0; w < g->n_win; ++w) cf += g->h_win_cost[w] + 8;
            rw->bwd_est = cb;
            rw->fwd_est = cf;
        }
        bwd_cost.push_back(rw->bwd_est);
        fwd_cost.push_back(rw->fwd_est);
        for (int b = 0; b < r->nblk; ++b) pix.push_back(make_int2((int)ri, b));
        for (int k = 0; k < P.K; ++k) rows.push_back(make_int2((int)ri, k));
        const long long N = (long long)P.W * P.H, KMp = (long long)P.K * P.Mp;
        for (long long t = 0; t < N; t += kUpdChunk) upd.push_back(make_int4((int)ri, 0, (int)t, 0));
        for (long long t = 0; t < KMp; t += kUpdChunk) upd.push_back(make_int4((int)ri, 1, (int)t, 0));
    }
    std::vector<int> start = start_requests(bwd_cost, G), fstart = start_requests(fwd_cost, G);
    start.insert(start.end(), fstart.begin(), fstart.end());
    cudaError_t e = cudaSuccess;
    e = ensure_cap(&E->L.desc, &E->cap_desc, E->sel.size(), grew);
    if (e == cudaSuccess) e = ensure_cap(&E->L.pool, &E->cap_pool, 3 * E->cap_desc, grew);
    if (e == cudaSuccess) e = ensure_cap(&E->L.pixblk, &E->cap_pix, pix.size(), grew);
    if (e == cudaSuccess) e = ensure_cap(&E->L.rowblk, &E->cap_row, rows.size(), grew);
    if (e == cudaSuccess) e = ensure_cap(&E->L.upd, &E->cap_upd, upd.size(), grew);
    if (e != cudaSuccess) return MBIR_ERR_OOM;
    if (!E->L.start) {
        e = cudaMalloc((void**)&E->L.start, sizeof(int) * 2 * G);
        if (e == cudaSuccess) e = cudaMalloc((void**)&E->L.counts, sizeof(int) * 8);
        if (e != cudaSuccess) return MBIR_ERR_OOM;
        *grew = true;
    }
    int counts[8] = {(int)E->sel.size(), (int)pix.size(), (int)rows.size(), (int)upd.size(), 0, 0, 0, 0};
    // pageable copies are staged before cudaMemcpyAsync returns, so the host vectors may go away
    if (!pix.empty())
        e = cudaMemcpyAsync(E->L.pixblk, pix.data(), sizeof(int2) * pix.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && !rows.empty())
        e = cudaMemcpyAsync(E->L.rowblk, rows.data(), sizeof(int2) * rows.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && !upd.empty())
        e = cudaMemcpyAsync(E->L.upd, upd.data(), sizeof(int4) * upd.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(E->L.start, start.data(), sizeof(int) * 2 * G, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(E->L.counts, counts, sizeof(counts), cudaMemcpyHostToDevice, st);
    return e == cudaSuccess ? MBIR_OK : MBIR_ERR_CUDA;
}

// One MAP iteration of every active request, as launched inside the graph.
// tcb / ccb: some requests have the tensor-core A^T / some do not; tcf / ccf likewise for A x.  Each kernel
// takes only the requests of its kind, so a request runs the same kernels alone and in any mix.
cudaError_t enqueue_iteration(mbir_engine* E, bool bf16, bool tcb, bool ccb, bool tcf, bool ccf, cudaStream_t st)
{
    const int G = E->n_sm, SG = E->n_sm * 8;
    cudaError_t e = cudaMemsetAsync(E->L.pool, 0, sizeof(int) * E->cap_pool, st);
    if (e != cudaSuccess) return e;
    if (tcb) {
        if (bf16) eng_emax_kernel<true><<<SG, kRedThreads, 0, st>>>(E->L);
        else eng_emax_kernel<false><<<SG, kRedThreads, 0, st>>>(E->L);
        if (bf16) eng_bwd_tcs_kernel<true><<<G, TbShape<true>::threads, E->smem_tc[1], st>>>(E->L);
        else eng_bwd_tcs_kernel<false><<<G, TbShape<false>::threads, E->smem_tc[1], st>>>(E->L);
        eng_bwd_tc_finish_kernel<<<SG, kRedThreads, 0, st>>>(E->L);
    }
    if (ccb) {
        if (bf16) eng_bwd_kernel<true><<<G, kEngThreads, E->smem_bwd, st>>>(E->L);
        else eng_bwd_kernel<false><<<G, kEngThreads, E->smem_bwd, st>>>(E->L);
        eng_bwd_reduce_kernel<<<SG, kRedThreads, 0, st>>>(E->L);
    }
    eng_grad_kernel<<<SG, kRedThreads, 0, st>>>(E->L);
    eng_findir_kernel<<<G, kRedThreads, 0, st>>>(E->L);
    eng_dir_kernel<<<SG, kRedThreads, 0, st>>>(E->L);
    if (tcf && bf16) eng_fwd_tcs_kernel<true><<<G, TsShape<true>::threads, E->smem_tc[0], st>>>(E->L);
    else if (tcf) eng_fwd_tcs_kernel<false><<<G, TsShape<false>::threads, E->smem_tc[0], st>>>(E->L);
    if (ccf && bf16) eng_fwd_kernel<true><<<G, kEngThreads, E->smem_fwd, st>>>(E->L);
    else if (ccf) eng_fwd_kernel<false><<<G, kEngThreads, E->smem_fwd, st>>>(E->L);
    eng_proj_kernel<<<SG, kRedThreads, 0, st>>>(E->L);
    eng_finstep_kernel<<<G, kRedThreads, 0, st>>>(E->L);
    eng_update_kernel<<<SG, kRedThreads, 0, st>>>(E->L);
    return cudaGetLastError();
}

}  // namespace

extern "C" {

int mbir_engine_create(size_t budget_bytes, int max_active, mbir_engine** out)
{
    if (!out || budget_bytes == 0 || max_active < 1) return MBIR_ERR_INVALID_ARG;
    mbir_engine* E = new mbir_engine();
    cudaGetDevice(&E->device);
    cudaDeviceGetAttribute(&E->n_sm, cudaDevAttrMultiProcessorCount, E->device);
    if (E->n_sm < 1) E->n_sm = 1;
    E->budget = budget_bytes;
    E->max_active = max_active;
    E->smem_bwd = kEngSmem;
    E->smem_fwd = kEngHdr + kTableMaxBytes + (size_t)kEngThreads * (sizeof(int4) + sizeof(float4));
    cudaError_t e = cudaFuncSetAttribute(eng_bwd_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)E->smem_bwd);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(eng_bwd_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)E->smem_bwd);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(eng_fwd_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)E->smem_fwd);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(eng_fwd_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)E->smem_fwd);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(eng_fwd_tcs_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kEngSmem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(eng_bwd_tcs_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kEngSmem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(eng_bwd_tcs_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kEngSmem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(eng_fwd_tcs_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kEngSmem);
    if (e != cudaSuccess) { delete E; return MBIR_ERR_CUDA; }
    *out = E;
    return MBIR_OK;
}

int mbir_engine_destroy(mbir_engine* E)
{
    if (!E) return MBIR_OK;
    cudaDeviceSynchronize();
    for (auto& kv : E->all) {
        free_request_state(kv.second.get(), 0);
        if (kv.second->done_ev) cudaEventDestroy(kv.second->done_ev);
    }
    cudaDeviceSynchronize();
    void* ptrs[] = {E->L.desc, E->L.pool, E->L.start, E->L.pixblk, E->L.rowblk, E->L.upd, E->L.counts};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (E->graph) cudaGraphExecDestroy(E->graph);
    delete E;
    return MBIR_OK;
}

int mbir_engine_submit(mbir_engine* E, const mbir_geometry* g, const void* y_dev, const mbir_prior* pr, int n_iter,
                       float* x_dev, float* g_dev, int64_t* ticket)
{
    if (!E || !g || !y_dev || !x_dev || !ticket || n_iter < 1 || !prior_is_valid(pr)) return MBIR_ERR_INVALID_ARG;
    if (g->P.mode != MBIR_MODE_TAB || !(g->d_rec_key || g->d_tc_key) || !g->h_win_cost) return MBIR_ERR_UNSUPPORTED;
    const size_t tsz = g->P.precision == MBIR_PREC_BF16 ? 4 : 8;
    const size_t tab = ((size_t)g->P.Gt * (g->P.Q + 1) * table_stride(g->P.Tw4) * tsz + 127) & ~(size_t)127;
    const size_t eb = ((size_t)g->P.Mp * (g->P.precision == MBIR_PREC_BF16 ? 2 : 4) + 127) & ~(size_t)127;
    if (tab > kTableMaxBytes || g->P.Mp > kMpMax || kEngHdr + tab + 2 * 2 * eb > kEngSmem || g->device != E->device)
        return MBIR_ERR_UNSUPPORTED;
    const size_t need = request_bytes(g, g->n_groups);
    if (need > E->budget) return MBIR_ERR_BUSY;
    auto r = std::make_unique<Request>();
    r->ticket = E->next_ticket++;
    r->g = g;
    r->y = y_dev;
    r->prior = *pr;
    r->n_iter = n_iter;
    r->x = x_dev;
    r->gout = g_dev;
    r->bytes = need;
    *ticket = r->ticket;
    E->queue.push_back(r.get());
    E->all[r->ticket] = std::move(r);
    return MBIR_OK;
}

int mbir_engine_step(mbir_engine* E, void* stream, int* n_active, int* n_queued)
{
    if (!E) return MBIR_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int rc = MBIR_OK;
    // retire requests that completed their iterations in the previous step
    for (size_t i = 0; i < E->active.size();) {
        Request* r = E->active[i];
        if (r->it < r->n_iter) { ++i; continue; }
        const GeomParams& P = r->g->P;
        if (r->gout) {
            // g = gains of y - A x (eq. 1), through the single-request operators
            cudaError_t e = mbir::launch_forward(r->g, r->x, r->q, nullptr, P.Mp, st);
            if (e == cudaSuccess)
                e = mbir::launch_project_rows(r->g, r->y, P.precision == MBIR_PREC_BF16 ? 1 : 0, P.M, r->q, P.Mp,
                                              r->q, P.Mp, r->gout, nullptr, st);
            if (e != cudaSuccess) rc = MBIR_ERR_CUDA;
        }
        double bad = 0.0;
        cudaMemcpyAsync(&bad, r->sc + S_BAD, sizeof(double), cudaMemcpyDeviceToHost, st);
        cudaStreamSynchronize(st);
        r->state = bad != 0.0 ? MBIR_ERR_NONFINITE : 3;
        free_request_state(r, st);
        E->used -= r->bytes;
        E->active.erase(E->active.begin() + i);
        E->sel.erase(std::remove(E->sel.begin(), E->sel.end(), r), E->sel.end());
        E->dirty = true;
    }
    // admit queued requests that fit the budget (in arrival order)
    while (!E->queue.empty() && (int)E->active.size() < E->max_active && E->used + E->queue.front()->bytes <= E->budget) {
        Request* r = E->queue.front();
        int arc = admit(E, r, st);
        E->queue.pop_front();
        if (arc != MBIR_OK) { r->state = arc; continue; }
        E->used += r->bytes;
        E->active.push_back(r);
        E->dirty = true;
    }
    if (n_queued) *n_queued = (int)E->queue.size();
    if (n_active) *n_active = (int)E->active.size();
    if (E->active.empty()) return rc;
    select_step(E);
    // the graph is specialised to one table precision; mixed precisions run in two passes
    bool grew = false;
    if (E->dirty) {
        int lrc = rebuild_lists(E, st, &grew);
        if (lrc != MBIR_OK) return lrc;
        E->dirty = false;
    }
    E->h_desc.resize(E->sel.size());
    for (size_t i = 0; i < E->sel.size(); ++i) fill_desc(E->h_desc[i], E->sel[i]);
    cudaError_t e = cudaMemcpyAsync(E->L.desc, E->h_desc.data(), sizeof(ReqDesc) * E->h_desc.size(),
                                    cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return MBIR_ERR_CUDA;
    const bool bf16 = E->sel[0]->g->P.precision == MBIR_PREC_BF16;
    for (Request* r : E->active)
        if ((r->g->P.precision == MBIR_PREC_BF16) != bf16) return MBIR_ERR_UNSUPPORTED;
    bool tcb = false, ccb = false, tcf = false, ccf = false;   // requests with / without each tensor-core apply
    for (Request* r : E->sel) {
        if (r->acc) tcb = true;
        else ccb = true;
        if (r->g->d_tf4_bop) tcf = true;
        else ccf = true;
    }
    const int gtc = (int)tcb + 2 * (int)ccb + 4 * (int)tcf + 8 * (int)ccf;
    size_t smem_tc[2] = {1024, 1024};
    for (Request* r : E->active) {
        const mbir_geometry* g = r->g;
        if (g->d_tf4_bop) smem_tc[0] = std::max(smem_tc[0], g->tf4.smem);
        if (g->d_tb4_bop) smem_tc[1] = std::max(smem_tc[1], g->tb4.smem);
    }
    const bool smem_changed = !std::equal(smem_tc, smem_tc + 2, E->smem_tc);
    if (grew || smem_changed || !E->graph || E->graph_bf16 != (int)bf16 || E->graph_tc != gtc) {
        std::copy(smem_tc, smem_tc + 2, E->smem_tc);
        if (E->graph) { cudaGraphExecDestroy(E->graph); E->graph = nullptr; }
        cudaStream_t cs;
        cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
        cudaGraph_t graph;
        e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) e = enqueue_iteration(E, bf16, tcb, ccb, tcf, ccf, cs);
        cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&E->graph, graph, 0);
        if (e2 == cudaSuccess) cudaGraphDestroy(graph);
        cudaStreamDestroy(cs);
        if (e != cudaSuccess) return MBIR_ERR_CUDA;
        E->graph_bf16 = (int)bf16;
        E->graph_tc = gtc;
    }
    e = cudaGraphLaunch(E->graph, st);
    if (e != cudaSuccess) return MBIR_ERR_CUDA;
    for (Request* r : E->sel) ++r->it;
    return rc;
}

int mbir_engine_poll(mbir_engine* E, int64_t ticket, int* state)
{
    if (!E || !state) return MBIR_ERR_INVALID_ARG;
    auto it = E->all.find(ticket);
    if (it == E->all.end()) return MBIR_ERR_INVALID_ARG;
    const Request* r = it->second.get();
    *state = r->state;
    return r->state < 0 ? r->state : MBIR_OK;
}

// Steps the engine until the request is done or `timeout_ms` of host time passes.
int mbir_engine_wait(mbir_engine* E, int64_t ticket, int timeout_ms, void* stream)
{
    if (!E) return MBIR_ERR_INVALID_ARG;
    auto it = E->all.find(ticket);
    if (it == E->all.end()) return MBIR_ERR_INVALID_ARG;
    Request* r = it->second.get();
    cudaEvent_t t0;
    cudaEventCreate(&t0);
    auto start = std::chrono::steady_clock::now();
    while (r->state == 0 || r->state == 1) {
        int na = 0, nq = 0;
        int rc = mbir_engine_step(E, stream, &na, &nq);
        if (rc != MBIR_OK) { cudaEventDestroy(t0); return rc; }
        auto ms = std::chrono::duration_cast<std::chrono::milliseconds>(std::chrono::steady_clock::now() - start).count();
        if (ms > timeout_ms && (r->state == 0 || r->state == 1)) { cudaEventDestroy(t0); return MBIR_ERR_TIMEOUT; }
        if (na == 0 && nq == 0 && r->state <= 1) break;
    }
    cudaEventDestroy(t0);
    return r->state < 0 ? r->state : MBIR_OK;
}

// Cancels a request that has not finished; its outputs are left as they are.
int mbir_engine_cancel(mbir_engine* E, int64_t ticket, void* stream)
{
    if (!E) return MBIR_ERR_INVALID_ARG;
    auto it = E->all.find(ticket);
    if (it == E->all.end()) return MBIR_ERR_INVALID_ARG;
    Request* r = it->second.get();
    if (r->state == 0) {
        E->queue.erase(std::remove(E->queue.begin(), E->queue.end(), r), E->queue.end());
        r->state = MBIR_ERR_CANCELLED;
    } else if (r->state == 1) {
        free_request_state(r, (cudaStream_t)stream);
        E->used -= r->bytes;
        E->active.erase(std::remove(E->active.begin(), E->active.end(), r), E->active.end());
        E->sel.erase(std::remove(E->sel.begin(), E->sel.end(), r), E->sel.end());
        E->dirty = true;
        r->state = MBIR_ERR_CANCELLED;
    }
    return MBIR_OK;
}

size_t mbir_engine_bytes_in_use(const mbir_engine* E) { return E ? E->used : 0; }

}  // extern "C"
