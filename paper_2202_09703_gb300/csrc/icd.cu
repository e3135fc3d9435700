// Column norms |A_v|^2 of the system matrix, the data-term curvature theta2
// of the iterative coordinate descent (Section 2 "Optimization").
//
// One thread per pixel walks every A-scan (transmit leg kept across its
// receivers), forms the pair of eq. 12-13 exactly as the apply kernels do and
// adds w^2 sum_m H(m)^2 over the pair's taps inside the record, the tau = t0
// tap of a flagged pair taking only its lower table row (eq. 10's open
// window).  The sum per pixel runs in A-scan order: deterministic.
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

}  // namespace mbir
