// Column norms |A_v|^2 of the system matrix, the data-term curvature theta2
// of the iterative coordinate descent (Section 2 "Optimization").
//
// One thread per pixel walks every A-scan (transmit leg kept across its
// receivers), forms the pair of eq. 12-13 exactly as the apply kernels do and
// adds w^2 sum_m H(m)^2 over the pair's taps inside the record, the tau = t0
// tap of a flagged pair taking only its lower table row (eq. 10's open
// window).  The sum per pixel runs in A-scan order: deterministic.
//
// It also builds the per-colour work lists of the descent: the A^T items of
// each colour's pixel lattice and, with TAB records, each colour's records.
#include <algorithm>
#include <vector>

#include "apply_common.cuh"

namespace mbir {

constexpr int kColnormThreads = 256;

template <int NL, int MODE>
__global__ void __launch_bounds__(kColnormThreads)
    colnorm_kernel(GeomParams P, DevPtrs D, const float2* __restrict__ tab, float* __restrict__ out)
{
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= P.W * P.H) return;
    const int row = v / P.W, col = v - row * P.W;
    const RowInfo ri = load_row(D.rows, row);
    const int S = table_stride(P.Tw4), R = P.Q + 1;
    float acc = 0.0f;
    if (ri.tvert < (float)(P.M - 1)) {
        Leg tx = {0.f, 0.f, 0.f, 0.f};
        for (int k = 0; k < P.K; ++k) {
            const int i = k / P.n_rx;
            if (k == i * P.n_rx) tx = get_leg<NL, MODE>(P, D, ri, row, col, __ldg(D.txpos + i));
            const Leg rx = get_leg<NL, MODE>(P, D, ri, row, col, __ldg(D.rxpos + k));
            const Pair pr = make_pair(P, tx, rx, ri.tau);
            if (!(pr.w != 0.0f && pr.n0 >= 0 && pr.n0 + 1 < P.M)) continue;
            const float2* A = tab + (size_t)(pr.gi * R + pr.r) * S;
            const float2* B = A + S;
            const float p1 = pr.psi, p0 = 1.0f - pr.psi;
            const int mz = min(P.Tw, P.M - 1 - pr.n0);          // taps n0 + 1 + m inside the record
            float s = 0.0f;
            for (int m = 0; m < mz; ++m) {
                const float2 a = __ldg(A + m), b = __ldg(B + m);
                float h = pr.w0 * (p0 * a.x + p1 * a.y);
                if (!(pr.flag0 && m == P.Tw - 1)) h = fmaf(pr.w1, p0 * b.x + p1 * b.y, h);
                s = fmaf(h, h, s);
            }
            acc = fmaf(pr.w * pr.w, s, acc);
        }
    }
    out[v] = acc;
}

template <int NL, int MODE>
static cudaError_t launch_colnorm_t(const mbir_geometry* g, float* out, cudaStream_t st)
{
    const int N = g->P.W * g->P.H;
    colnorm_kernel<NL, MODE><<<(N + kColnormThreads - 1) / kColnormThreads, kColnormThreads, 0, st>>>(
        g->P, dev_ptrs(g), g->d_tab, out);
    return cudaGetLastError();
}

cudaError_t launch_column_norms(const mbir_geometry* g, float* out, cudaStream_t st)
{
    if (g->P.mode == MBIR_MODE_TAB) return launch_colnorm_t<1, kModeTAB>(g, out, st);
    if (g->P.L <= 2) return launch_colnorm_t<2, kModeOTF>(g, out, st);
    if (g->P.L <= 4) return launch_colnorm_t<4, kModeOTF>(g, out, st);
    return launch_colnorm_t<8, kModeOTF>(g, out, st);
}

void free_icd_lists(mbir_geometry* g)
{
    void* ptrs[] = {g->d_icd_items, g->w_icd_bpart, g->d_icd_rec_off, g->d_icd_rec_key, g->d_icd_rec_w,
                    g->d_icd_runs, g->d_icd_win};
    for (void* p : ptrs) if (p) cudaFree(p);
    free(g->h_icd_item_off);
    free(g->h_icd_win_off);
    g->bytes -= g->icd_bytes + g->icd_rec_bytes;
    g->d_icd_items = nullptr;
    g->w_icd_bpart = nullptr;
    g->d_icd_rec_off = nullptr;
    g->d_icd_rec_key = nullptr;
    g->d_icd_rec_w = nullptr;
    g->d_icd_runs = nullptr;
    g->d_icd_win = nullptr;
    g->h_icd_item_off = nullptr;
    g->h_icd_win_off = nullptr;
    g->icd_bytes = g->icd_rec_bytes = 0;
    g->icd_s = 0;
    if (g->icd_exec) cudaGraphExecDestroy((cudaGraphExec_t)g->icd_exec);
    g->icd_exec = nullptr;
}

// Work lists for colour spacing s.  A^T: per colour the 16 x 32 tiles of its pixel lattice (those whose
// first row can reach the record) times chunks of A-scans, the same chunks for every colour, about four
// items per tile worker so that dynamic fetching evens out the SMs.  A x: per-colour record lists when the geometry has
// records (the colours partition the pairs) and s <= 64; otherwise (or if they do not fit) the full A x.
cudaError_t build_icd_lists(mbir_geometry* g, int s, cudaStream_t st)
{
    free_icd_lists(g);
    const GeomParams& P = g->P;
    const int nc = s * s, TR = backproject_tile_rows();
    int min_tiles = 0;
    for (int c = 0; c < nc; ++c) {
        const int r0 = c / s, c0 = c % s;
        if (r0 >= P.H || c0 >= P.W) continue;
        const int Hc = (P.H - r0 + s - 1) / s, Wc = (P.W - c0 + s - 1) / s;
        int tiles = 0;
        for (int tr = 0; tr * TR < Hc; ++tr)
            if (g->h_tvert[tr * TR * s + r0] < (float)(P.M - 1)) tiles += (Wc + 31) / 32;
        if (tiles > 0) min_tiles = min_tiles == 0 ? tiles : std::min(min_tiles, tiles);
    }
    // A-scan chunks of at least 4 (the residual ring's depth plus one), about four items per tile worker
    int ng = 1;
    if (min_tiles > 0)
        ng = std::max(1, std::min(std::max(P.K / 4, 1), (4 * g->bwd_halves * g->n_sm + min_tiles - 1) / min_tiles));
    const int kg = (P.K + ng - 1) / ng;
    ng = (P.K + kg - 1) / kg;
    std::vector<int4> items;
    std::vector<int> ioff(nc + 1, 0);
    for (int c = 0; c < nc; ++c) {
        const int r0 = c / s, c0 = c % s;
        if (r0 < P.H && c0 < P.W) {
            const int Hc = (P.H - r0 + s - 1) / s, Wc = (P.W - c0 + s - 1) / s;
            for (int tr = 0; tr * TR < Hc; ++tr) {
                if (!(g->h_tvert[tr * TR * s + r0] < (float)(P.M - 1))) continue;
                for (int tc = 0; tc * 32 < Wc; ++tc)
                    for (int gi = 0; gi < ng; ++gi) {
                        const int k0 = gi * kg, k1 = std::min(P.K, k0 + kg);
                        items.push_back(make_int4(tr, tc, k0 | (k1 << 16), gi));
                    }
            }
        }
        ioff[c + 1] = (int)items.size();
    }
    const size_t N = (size_t)P.W * P.H;
    cudaError_t e = cudaMalloc((void**)&g->d_icd_items, sizeof(int4) * std::max<size_t>(items.size(), 1));
    if (e == cudaSuccess && !items.empty())
        e = cudaMemcpy(g->d_icd_items, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc((void**)&g->w_icd_bpart, sizeof(float) * N * ng);
    g->h_icd_item_off = (int*)malloc(sizeof(int) * (nc + 1));
    if (e == cudaSuccess && !g->h_icd_item_off) e = cudaErrorMemoryAllocation;
    if (e != cudaSuccess) {
        free_icd_lists(g);
        return e;
    }
    std::copy(ioff.begin(), ioff.end(), g->h_icd_item_off);
    g->icd_groups = ng;
    g->icd_bytes = sizeof(int4) * std::max<size_t>(items.size(), 1) + sizeof(float) * N * ng;
    g->bytes += g->icd_bytes;
    g->icd_s = s;
    // per-colour record lists up to 64 x 64 colours (their span bounds grow with the colour count)
    if ((g->d_rec_key || g->d_tc_key) && nc <= 4096) {
        e = build_colour_records(g, s, st);
        if (e == cudaSuccess) g->bytes += g->icd_rec_bytes;
        else if (e == cudaErrorMemoryAllocation) {
            cudaGetLastError();                  // no room for a second copy of the records: full A x
            e = cudaSuccess;
        }
    }
    return e;
}

}  // namespace mbir
