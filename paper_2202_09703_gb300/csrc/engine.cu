// Batched and served reconstructions: many independent MAP problems of
// uneven size advance together, one iteration per engine step.
//
// Every step is one captured CUDA graph of eight grouped kernels.  Their grids
// are fixed (persistent or grid-stride), and they read the current set of
// active requests from device-side work lists that the host rewrites between
// steps, so the graph is captured once and replayed as requests come and go
// (continuous batching):
//   A^T e   persistent, 32 x 32 pixel tiles x transmitter groups of every
//           request, split into contiguous cost-balanced ranges per CTA; a CTA
//           reloads the pulse table only when its next item belongs to
//           another request
//   grad    prior gradient + FP64 partials per (request, pixel block)
//   dir     Polak-Ribiere+ scalars per request, then directions + curvature
//   A d     persistent span gather over each request's sorted records, in
//           chunks of spans assigned to CTAs by cost; warps share a chunk
//   P q     direct-arrival projection per (request, A-scan) with FP64 norms
//   step    majorize-minimize step per request; x and e updated
// Each request's arithmetic depends only on its own data and its own fixed
// work decomposition, so a result is bitwise the same alone and in any mix.
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

namespace mbir {
PriorParams make_prior_params(const mbir_prior* pr);
bool prior_is_valid(const mbir_prior* pr);
}  // namespace mbir

using namespace mbir;

namespace {

constexpr int kEngThreads = 1024;          // apply kernels: 32 warps
constexpr int kEngStages = 3;              // residual-row ring of A^T e
constexpr int kEngTile = 32;               // 32 x 32 pixel tiles
constexpr int kSpanChunk = 64;             // spans per A d work chunk
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
    const int2* rkey;
    const float4* rw;
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
    PriorParams pr;
    int it;                // iteration index of this step
    int ngroups;
    int nblk;              // pixel blocks of kRedThreads
};

struct EngLists {
    ReqDesc* desc;
    int4* bwd_items;       // {req, tile_r << 16 | tile_c, tx0 | tx1 << 16, group}
    int* bwd_cta;          // per-CTA item ranges (gridDim + 1)
    int4* fwd_chunks;      // {req, first span, end span, 0}
    int* fwd_cta;
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
template <bool BF16>
__global__ void __launch_bounds__(kEngThreads, 1) eng_bwd_kernel(EngLists L)
{
    using Tab = typename TabT<BF16>::type;
    using E = typename ET<BF16>::type;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(bars + kEngStages);
    Tab* tab = reinterpret_cast<Tab*>(smem + 128);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        for (int s = 0; s < kEngStages; ++s) mbar_init(smem_u32(bars + s), 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    __syncthreads();
    const uint32_t bar0 = smem_u32(bars);
    uint32_t par = 0;
    int cur = -1;
    size_t tab_bytes = 0, ebytes = 0;
    E* ring = nullptr;
    const int i0 = L.bwd_cta[blockIdx.x], i1 = L.bwd_cta[blockIdx.x + 1];
    for (int it = i0; it < i1; ++it) {
        const int4 item = L.bwd_items[it];
        const ReqDesc& R = L.desc[item.x];
        const GeomParams& P = R.P;
        const int S = table_stride(P.Tw4), Q1 = P.Q + 1;
        if (item.x != cur) {
            __syncthreads();
            tab_bytes = ((size_t)P.Gt * Q1 * S * sizeof(Tab) + 127) & ~(size_t)127;
            ebytes = ((size_t)P.Mp * sizeof(E) + 127) & ~(size_t)127;
            ring = reinterpret_cast<E*>(smem + 128 + tab_bytes);
            load_table_smem(tab, BF16 ? (const void*)R.tab_bf : (const void*)R.tab, tab_bytes, tid, kEngThreads);
            cur = item.x;
            __syncthreads();
        }
        const E* e_g = BF16 ? (const E*)(const void*)R.ebf : (const E*)(const void*)R.e;
        const int row = (item.y >> 16) * kEngTile + warp, col = (item.y & 0xffff) * kEngTile + lane;
        const int tx0 = item.z & 0xffff, tx1 = item.z >> 16, grp = item.w;
        const bool pix_ok = col < P.W && row < P.H;
        const RowInfo ri = load_row(R.D.rows, min(row, P.H - 1));
        const bool row_ok = pix_ok && ri.tvert < (float)(P.M - 1);
        const int colc = min(col, P.W - 1);
        const int ka = tx0 * P.n_rx, kb = tx1 * P.n_rx;
        const uint32_t rowbytes = (uint32_t)((size_t)P.Mp * sizeof(E));
        if (tid == 0) {
            for (int s = 0; s < kEngStages && ka + s < kb; ++s) {
                mbar_arrive_expect_tx(bar0 + 8 * s, rowbytes);
                bulk_g2s(smem_u32(ring + (size_t)s * (ebytes / sizeof(E))), e_g + (size_t)(ka + s) * P.Mp,
                         rowbytes, bar0 + 8 * s);
            }
        }
        float sum = 0.0f, comp = 0.0f;
        Leg tx = {0.f, 0.f, 0.f, 0.f};
        int i = tx0, j = 0, stage = 0;
        bool aborted = false;
        int k = ka;
        for (; k < kb; ++k) {
            Leg rx = tx;
            if (row_ok) {
                if (j == 0) tx = get_leg<1, kModeTAB>(P, R.D, ri, row, colc, __ldg(R.D.txpos + i));
                rx = get_leg<1, kModeTAB>(P, R.D, ri, row, colc, __ldg(R.D.rxpos + k));
            }
            const Pair pr = make_pair(P, tx, rx, ri.tau);
            const bool act = row_ok && pr.w != 0.0f && pr.n0 >= 0 && pr.n0 + 1 < P.M;
            const bool ok = mbar_wait_bounded(bar0 + 8 * stage, (par >> stage) & 1u, R.D.status);
            par ^= 1u << stage;
            if (!ok) *abort_flag = 1;
            if (act && ok) {
                const E* ev = ring + (size_t)stage * (ebytes / sizeof(E)) + pr.n0 + 1;
                const Tab* A = tab + (size_t)(pr.gi * Q1 + pr.r) * S;
                neumaier_add(sum, comp, pair_taps<BF16>(A, S, P.Tw, P.Tw4, ev, pr));
            }
            __syncthreads();
            if (*abort_flag) { aborted = true; break; }
            if (tid == 0 && k + kEngStages < kb) {
                mbar_arrive_expect_tx(bar0 + 8 * stage, rowbytes);
                bulk_g2s(smem_u32(ring + (size_t)stage * (ebytes / sizeof(E))),
                         e_g + (size_t)(k + kEngStages) * P.Mp, rowbytes, bar0 + 8 * stage);
            }
            if (++stage == kEngStages) stage = 0;
            if (++j == P.n_rx) { j = 0; ++i; }
        }
        if (aborted) {
            if (tid == 0)
                for (int q = k + 1; q < kb && q < k + kEngStages; ++q) {
                    const int s = (q - ka) % kEngStages;
                    mbar_wait_bounded(bar0 + 8 * s, (par >> s) & 1u, R.D.status);
                    par ^= 1u << s;
                }
            return;
        }
        if (pix_ok) R.bpart[(size_t)grp * P.W * P.H + (size_t)row * P.W + col] = sum + comp;
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
        const GeomParams& P = R.P;
        const int N = P.W * P.H;
        const int v = rb.y * kRedThreads + threadIdx.x;
        if (v >= N) continue;
        const int row = v / P.W;
        const int row0 = (row / kEngTile) * kEngTile;
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

// q = A d over every active request (span chunks, table reloaded per request)
template <bool BF16>
__global__ void __launch_bounds__(kEngThreads, 1) eng_fwd_kernel(EngLists L)
{
    using Tab = typename TabT<BF16>::type;
    constexpr int WARPS = kEngThreads / 32;
    extern __shared__ __align__(128) unsigned char smem[];
    int* counter = reinterpret_cast<int*>(smem);
    Tab* tab = reinterpret_cast<Tab*>(smem + 128);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int4* sr = reinterpret_cast<int4*>(smem + 128 + kTableMaxBytes) + warp * 32;
    float4* sw = reinterpret_cast<float4*>(smem + 128 + kTableMaxBytes) + WARPS * 32 + warp * 32;
    int cur = -1;
    const int c0 = L.fwd_cta[blockIdx.x], c1 = L.fwd_cta[blockIdx.x + 1];
    for (int ch = c0; ch < c1; ++ch) {
        const int4 cd = L.fwd_chunks[ch];
        const ReqDesc& R = L.desc[cd.x];
        const GeomParams& P = R.P;
        const int S = table_stride(P.Tw4);
        __syncthreads();
        if (cd.x != cur) {
            const size_t tab_bytes = ((size_t)P.Gt * (P.Q + 1) * S * sizeof(Tab) + 127) & ~(size_t)127;
            load_table_smem(tab, BF16 ? (const void*)R.tab_bf : (const void*)R.tab, tab_bytes, tid, kEngThreads);
            cur = cd.x;
        }
        if (tid == 0) *counter = cd.y;
        __syncthreads();
        const int nspan = (P.M + 31) >> 5;
        const float* x = dnew_of(R);
        for (;;) {
            int s = 0;
            if (lane == 0) s = atomicAdd(counter, 1);
            s = __shfl_sync(0xffffffffu, s, 0);
            if (s >= cd.z) break;
            const int k = s / nspan, sp = s - k * nspan;
            const int n = sp * 32 + lane;
            const int2 rb = __ldg(R.runs + s);
            const float acc = span_gather<BF16>(tab, S, P.Tw, R.rkey, R.rw, __ldg(R.rec_off + k), rb.x, rb.y, x, n,
                                                lane, sr, sw);
            float* qo = R.q + (size_t)k * P.Mp;
            if (n < P.Mp) qo[n] = (n < P.M) ? acc : 0.0f;
            if (sp == nspan - 1)
                for (int t = nspan * 32 + lane; t < P.Mp; t += 32) qo[t] = 0.0f;
        }
    }
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
    float *e = nullptr, *q = nullptr, *b = nullptr, *grad = nullptr, *gprev = nullptr, *d0 = nullptr,
          *d1 = nullptr, *bpart = nullptr, *msq = nullptr;
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
    return b;
}

int groups_for(const mbir_geometry* g)
{
    // about 64 A-scans per work item
    const int txg = std::max(1, std::min(g->P.n_tx, 64 / std::max(1, g->P.n_rx)));
    return (g->P.n_tx + txg - 1) / txg;
}

}  // namespace

struct mbir_engine {
    int device = 0, n_sm = 1;
    size_t budget = 0, used = 0;
    int max_active = 64;
    int64_t next_ticket = 1;
    std::deque<Request*> queue;
    std::vector<Request*> active;
    std::map<int64_t, std::unique_ptr<Request>> all;
    bool dirty = true;                   // work lists must be rebuilt
    // device work lists (fixed capacity; growing them re-captures the graph)
    EngLists L{};
    size_t cap_desc = 0, cap_bwd = 0, cap_fwd = 0, cap_pix = 0, cap_row = 0, cap_upd = 0;
    cudaGraphExec_t graph = nullptr;
    int graph_bf16 = -1;
    size_t smem_bwd = 0, smem_fwd = 0;
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
    void* ptrs[] = {r->e, r->q, r->b, r->grad, r->gprev, r->d0, r->d1, r->bpart, r->msq, r->ebf, r->sc, r->part};
    for (void* p : ptrs)
        if (p) cudaFreeAsync(p, st);
    r->e = r->q = r->b = r->grad = r->gprev = r->d0 = r->d1 = r->bpart = r->msq = nullptr;
    r->ebf = nullptr;
    r->sc = r->part = nullptr;
}

int admit(mbir_engine* E, Request* r, cudaStream_t st)
{
    const mbir_geometry* g = r->g;
    const GeomParams& P = g->P;
    const size_t N = (size_t)P.W * P.H, KMp = (size_t)P.K * P.Mp;
    r->ngroups = groups_for(g);
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
#undef AL
    if (e != cudaSuccess) { free_request_state(r, st); return e == cudaErrorMemoryAllocation ? MBIR_ERR_OOM : MBIR_ERR_CUDA; }
    r->msq_host.resize(P.H);
    mbir::compute_msq(g, &r->prior, r->msq_host.data());
    e = cudaMemcpyAsync(r->msq, r->msq_host.data(), sizeof(float) * P.H, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(r->sc, 0, sizeof(double) * S_COUNT, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(r->gprev, 0, sizeof(float) * N, st);
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
    d.ngroups = r->ngroups;
    d.nblk = r->nblk;
}

// Rebuilds the per-epoch work lists for the active set.
int rebuild_lists(mbir_engine* E, cudaStream_t st, bool* grew)
{
    const int G = E->n_sm;
    std::vector<int4> bwd;
    std::vector<double> bwd_cost;
    std::vector<int4> fwd;
    std::vector<double> fwd_cost;
    std::vector<int2> pix, rows;
    std::vector<int4> upd;
    for (size_t ri = 0; ri < E->active.size(); ++ri) {
        const Request* r = E->active[ri];
        const GeomParams& P = r->g->P;
        const int ntr = (P.H + kEngTile - 1) / kEngTile, ntc = (P.W + kEngTile - 1) / kEngTile;
        const int txg = (P.n_tx + r->ngroups - 1) / r->ngroups;
        for (int tr = 0; tr < ntr; ++tr) {
            if (!(r->g->h_tvert[tr * kEngTile] < (float)(P.M - 1))) continue;
            for (int tc = 0; tc < ntc; ++tc)
                for (int gi = 0; gi < r->ngroups; ++gi) {
                    const int t0 = gi * txg, t1 = std::min(P.n_tx, t0 + txg);
                    if (t0 >= t1) continue;
                    bwd.push_back(make_int4((int)ri, (tr << 16) | tc, t0 | (t1 << 16), gi));
                    // the geometry's estimates per 16-row tile and transmitter position
                    const int TR = backproject_tile_rows(), ntr16 = (P.H + TR - 1) / TR;
                    double c = 0;
                    for (int r16 = tr * kEngTile / TR; r16 < std::min(ntr16, (tr + 1) * kEngTile / TR); ++r16)
                        for (int t = t0; t < t1; ++t)
                            c += r->g->h_bwd_cost[((size_t)r16 * r->g->bwd_ntc + tc) * P.n_tx + t];
                    bwd_cost.push_back(c);
                }
        }
        const int nspan = (P.M + 31) / 32;
        const long long nsp = (long long)P.K * nspan;
        for (long long s0 = 0; s0 < nsp; s0 += kSpanChunk) {
            const long long s1 = std::min(nsp, s0 + kSpanChunk);
            double c = 0;
            for (long long s = s0; s < s1; ++s) c += r->g->h_span_cost[s] + 8;
            fwd.push_back(make_int4((int)ri, (int)s0, (int)s1, 0));
            fwd_cost.push_back(c * 32.0);
        }
        for (int b = 0; b < r->nblk; ++b) pix.push_back(make_int2((int)ri, b));
        for (int k = 0; k < P.K; ++k) rows.push_back(make_int2((int)ri, k));
        const long long N = (long long)P.W * P.H, KMp = (long long)P.K * P.Mp;
        for (long long t = 0; t < N; t += kUpdChunk) upd.push_back(make_int4((int)ri, 0, (int)t, 0));
        for (long long t = 0; t < KMp; t += kUpdChunk) upd.push_back(make_int4((int)ri, 1, (int)t, 0));
    }
    std::vector<int> bcut = balance(bwd_cost, G), fcut = balance(fwd_cost, G);
    cudaError_t e = cudaSuccess;
    e = ensure_cap(&E->L.desc, &E->cap_desc, E->active.size(), grew);
    if (e == cudaSuccess) e = ensure_cap(&E->L.bwd_items, &E->cap_bwd, bwd.size(), grew);
    if (e == cudaSuccess) e = ensure_cap(&E->L.fwd_chunks, &E->cap_fwd, fwd.size(), grew);
    if (e == cudaSuccess) e = ensure_cap(&E->L.pixblk, &E->cap_pix, pix.size(), grew);
    if (e == cudaSuccess) e = ensure_cap(&E->L.rowblk, &E->cap_row, rows.size(), grew);
    if (e == cudaSuccess) e = ensure_cap(&E->L.upd, &E->cap_upd, upd.size(), grew);
    if (e != cudaSuccess) return MBIR_ERR_OOM;
    if (!E->L.bwd_cta) {
        e = cudaMalloc((void**)&E->L.bwd_cta, sizeof(int) * (G + 1));
        if (e == cudaSuccess) e = cudaMalloc((void**)&E->L.fwd_cta, sizeof(int) * (G + 1));
        if (e == cudaSuccess) e = cudaMalloc((void**)&E->L.counts, sizeof(int) * 8);
        if (e != cudaSuccess) return MBIR_ERR_OOM;
        *grew = true;
    }
    int counts[8] = {(int)E->active.size(), (int)pix.size(), (int)rows.size(), (int)upd.size(), 0, 0, 0, 0};
    // pageable copies are staged before cudaMemcpyAsync returns, so the host vectors may go away
    if (!bwd.empty()) e = cudaMemcpyAsync(E->L.bwd_items, bwd.data(), sizeof(int4) * bwd.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && !fwd.empty())
        e = cudaMemcpyAsync(E->L.fwd_chunks, fwd.data(), sizeof(int4) * fwd.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && !pix.empty())
        e = cudaMemcpyAsync(E->L.pixblk, pix.data(), sizeof(int2) * pix.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && !rows.empty())
        e = cudaMemcpyAsync(E->L.rowblk, rows.data(), sizeof(int2) * rows.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && !upd.empty())
        e = cudaMemcpyAsync(E->L.upd, upd.data(), sizeof(int4) * upd.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(E->L.bwd_cta, bcut.data(), sizeof(int) * (G + 1), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(E->L.fwd_cta, fcut.data(), sizeof(int) * (G + 1), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(E->L.counts, counts, sizeof(counts), cudaMemcpyHostToDevice, st);
    return e == cudaSuccess ? MBIR_OK : MBIR_ERR_CUDA;
}

// One MAP iteration of every active request, as launched inside the graph.
cudaError_t enqueue_iteration(mbir_engine* E, bool bf16, cudaStream_t st)
{
    const int G = E->n_sm, SG = E->n_sm * 8;
    if (bf16) eng_bwd_kernel<true><<<G, kEngThreads, E->smem_bwd, st>>>(E->L);
    else eng_bwd_kernel<false><<<G, kEngThreads, E->smem_bwd, st>>>(E->L);
    eng_bwd_reduce_kernel<<<SG, kRedThreads, 0, st>>>(E->L);
    eng_grad_kernel<<<SG, kRedThreads, 0, st>>>(E->L);
    eng_findir_kernel<<<G, kRedThreads, 0, st>>>(E->L);
    eng_dir_kernel<<<SG, kRedThreads, 0, st>>>(E->L);
    if (bf16) eng_fwd_kernel<true><<<G, kEngThreads, E->smem_fwd, st>>>(E->L);
    else eng_fwd_kernel<false><<<G, kEngThreads, E->smem_fwd, st>>>(E->L);
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
    E->smem_bwd = 128 + kTableMaxBytes + (size_t)kEngStages * (((size_t)kMpMax * 4 + 127) & ~(size_t)127);
    E->smem_fwd = 128 + kTableMaxBytes + (size_t)kEngThreads * (sizeof(int4) + sizeof(float4));
    cudaError_t e = cudaFuncSetAttribute(eng_bwd_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)E->smem_bwd);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(eng_bwd_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)E->smem_bwd);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(eng_fwd_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)E->smem_fwd);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(eng_fwd_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)E->smem_fwd);
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
    void* ptrs[] = {E->L.desc, E->L.bwd_items, E->L.bwd_cta, E->L.fwd_chunks, E->L.fwd_cta, E->L.pixblk,
                    E->L.rowblk, E->L.upd, E->L.counts};
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
    if (g->P.mode != MBIR_MODE_TAB || !g->d_rec_key || !g->h_span_cost) return MBIR_ERR_UNSUPPORTED;
    const size_t tsz = g->P.precision == MBIR_PREC_BF16 ? 4 : 8;
    const size_t tab = ((size_t)g->P.Gt * (g->P.Q + 1) * table_stride(g->P.Tw4) * tsz + 127) & ~(size_t)127;
    if (tab > kTableMaxBytes || g->P.Mp > kMpMax || g->device != E->device) return MBIR_ERR_UNSUPPORTED;
    const size_t need = request_bytes(g, groups_for(g));
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
    // the graph is specialised to one table precision; mixed precisions run in two passes
    bool grew = false;
    if (E->dirty) {
        int lrc = rebuild_lists(E, st, &grew);
        if (lrc != MBIR_OK) return lrc;
        E->dirty = false;
    }
    E->h_desc.resize(E->active.size());
    for (size_t i = 0; i < E->active.size(); ++i) fill_desc(E->h_desc[i], E->active[i]);
    cudaError_t e = cudaMemcpyAsync(E->L.desc, E->h_desc.data(), sizeof(ReqDesc) * E->h_desc.size(),
                                    cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return MBIR_ERR_CUDA;
    const bool bf16 = E->active[0]->g->P.precision == MBIR_PREC_BF16;
    for (Request* r : E->active)
        if ((r->g->P.precision == MBIR_PREC_BF16) != bf16) return MBIR_ERR_UNSUPPORTED;
    if (grew || !E->graph || E->graph_bf16 != (int)bf16) {
        if (E->graph) { cudaGraphExecDestroy(E->graph); E->graph = nullptr; }
        cudaStream_t cs;
        cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
        cudaGraph_t graph;
        e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) e = enqueue_iteration(E, bf16, cs);
        cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&E->graph, graph, 0);
        if (e2 == cudaSuccess) cudaGraphDestroy(graph);
        cudaStreamDestroy(cs);
        if (e != cudaSuccess) return MBIR_ERR_CUDA;
        E->graph_bf16 = (int)bf16;
    }
    e = cudaGraphLaunch(E->graph, st);
    if (e != cudaSuccess) return MBIR_ERR_CUDA;
    for (Request* r : E->active) ++r->it;
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
        E->dirty = true;
        r->state = MBIR_ERR_CANCELLED;
    }
    return MBIR_OK;
}

size_t mbir_engine_bytes_in_use(const mbir_engine* E) { return E ? E->used : 0; }

}  // extern "C"
