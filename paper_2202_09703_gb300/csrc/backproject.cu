// A^T r (adjoint of eq. 13): one thread per pixel, one CTA per tile of
// kRows x 32 pixels.  The CTA walks the A-scans in (Tx, receiver) order,
// keeping the pixel's transmit leg while the receiver changes.  Each A-scan's
// residual row is staged in shared memory by a 1-D bulk copy (TMA engine)
// into a double buffer guarded by mbarriers, so the next row streams in while
// the current one is consumed.  The pulse table sits in shared memory.
// Every tap of a pair shares one table phase, so a pair costs two packed FP32
// FMAs per tap (four dot products, combined once per pair); per-pair partial
// sums are added across A-scans with Neumaier compensation.
#include "device_common.cuh"

namespace mbir {

constexpr int kBwdRows = 16;
constexpr int kBwdThreads = kBwdRows * 32;

__device__ __forceinline__ uint32_t bar_of(int k, uint32_t b0, uint32_t b1) { return (k & 1) ? b1 : b0; }

template <int NL, int MODE, bool BF16>
__global__ void __launch_bounds__(kBwdThreads, 1)
    backproject_kernel(GeomParams P, DevPtrs D, const typename TabT<BF16>::type* __restrict__ tab_g,
                       const typename ET<BF16>::type* __restrict__ e_g, float* __restrict__ b_out)
{
    using Tab = typename TabT<BF16>::type;
    using E = typename ET<BF16>::type;
    extern __shared__ __align__(128) unsigned char smem[];
    const int S = table_stride(P.Tw4);
    const int R = P.Q + 1;
    const size_t tab_elems = (size_t)P.Gt * R * S;
    const size_t tab_bytes = (tab_elems * sizeof(Tab) + 127) & ~(size_t)127;
    const size_t ebytes = ((size_t)P.Mp * sizeof(E) + 127) & ~(size_t)127;
    Tab* tab = reinterpret_cast<Tab*>(smem);
    E* ebuf0 = reinterpret_cast<E*>(smem + tab_bytes);
    E* ebuf1 = reinterpret_cast<E*>(smem + tab_bytes + ebytes);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + tab_bytes + 2 * ebytes);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(bars + 2);

    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int col = blockIdx.x * 32 + lane;
    const int row = blockIdx.y * kBwdRows + warp;
    const int row0 = blockIdx.y * kBwdRows;

    // rows are ordered by depth, so the vertical time grows with the row:
    // a tile whose first row cannot reach the record has nothing to do
    if (__ldg(&D.rows[row0].tvert) >= (float)(P.M - 1)) {
        if (col < P.W && row < P.H) b_out[(size_t)row * P.W + col] = 0.0f;
        return;
    }
    const bool pix_ok = col < P.W && row < P.H;
    RowInfo ri = load_row(D.rows, pix_ok ? row : row0);
    const bool row_ok = pix_ok && ri.tvert < (float)(P.M - 1);

    // pulse table -> shared
    {
        const int4* src = reinterpret_cast<const int4*>(tab_g);
        int4* dst = reinterpret_cast<int4*>(tab);
        const int n16 = (int)(tab_bytes / 16);
        for (int t = tid; t < n16; t += blockDim.x) dst[t] = __ldg(src + t);
    }
    const uint32_t bar0 = smem_u32(&bars[0]), bar1 = smem_u32(&bars[1]);
    const uint32_t rowbytes = (uint32_t)((size_t)P.Mp * sizeof(E));
    if (tid == 0) {
        mbar_init(bar0, 1);
        mbar_init(bar1, 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0) {
        mbar_arrive_expect_tx(bar0, rowbytes);
        bulk_g2s(smem_u32(ebuf0), e_g, rowbytes, bar0);
        if (P.K > 1) {
            mbar_arrive_expect_tx(bar1, rowbytes);
            bulk_g2s(smem_u32(ebuf1), e_g + (size_t)P.Mp, rowbytes, bar1);
        }
    }

    float sum = 0.0f, comp = 0.0f;
    Leg tx = {0.f, 0.f, 0.f, 0.f};
    int i = 0, j = 0;
    for (int k = 0; k < P.K; ++k) {
        if (row_ok) {
            if (j == 0) tx = get_leg<NL, MODE>(P, D, ri, row, col, __ldg(D.txpos + i));
            Leg rx = get_leg<NL, MODE>(P, D, ri, row, col, __ldg(D.rxpos + k));
            Pair pr = make_pair(P, tx, rx, ri.tau);
            const bool act = pr.w != 0.0f && pr.n0 >= 0 && pr.n0 + 1 < P.M;
            const uint32_t bar = (k & 1) ? bar1 : bar0;
            bool ok = mbar_wait_bounded(bar, (uint32_t)((k >> 1) & 1), D.status);
            if (!ok) *abort_flag = 1;
            if (act && ok) {
                const E* ev = ((k & 1) ? ebuf1 : ebuf0) + pr.n0 + 1;
                const Tab* A = tab + (size_t)(pr.gi * R + pr.r) * S;
                const Tab* B = A + S;
                float2 sa = make_float2(0.f, 0.f), sb = make_float2(0.f, 0.f);
                for (int m = 0; m < P.Tw4; m += 4) {
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        float e = ET<BF16>::ld(ev + m + u);
                        float2 ee = make_float2(e, e);
                        sa = __ffma2_rn(TabT<BF16>::ld(A + m + u), ee, sa);
                        sb = __ffma2_rn(TabT<BF16>::ld(B + m + u), ee, sb);
                    }
                }
                const float p1 = pr.psi, p0 = 1.0f - pr.psi;
                float h = pr.w0 * (p0 * sa.x + p1 * sa.y) + pr.w1 * (p0 * sb.x + p1 * sb.y);
                if (pr.flag0) {
                    // tau = t0 exactly: outside the open window of eq. 10
                    float2 bl = TabT<BF16>::ld(B + P.Tw - 1);
                    h -= pr.w1 * (p0 * bl.x + p1 * bl.y) * ET<BF16>::ld(ev + P.Tw - 1);
                }
                float val = pr.w * h;
                float t = sum + val;
                comp += (fabsf(sum) >= fabsf(val)) ? (sum - t) + val : (val - t) + sum;
                sum = t;
            }
        } else {
            const uint32_t bar = (k & 1) ? bar1 : bar0;
            if (!mbar_wait_bounded(bar, (uint32_t)((k >> 1) & 1), D.status)) *abort_flag = 1;
        }
        __syncthreads();
        if (*abort_flag) {
            if (tid == 0) {
                // drain the copies still in flight (rows k and k+1) before exiting
                mbar_wait_bounded(bar_of(k, bar0, bar1), (uint32_t)((k >> 1) & 1), D.status);
                if (k + 1 < P.K)
                    mbar_wait_bounded(bar_of(k + 1, bar0, bar1), (uint32_t)(((k + 1) >> 1) & 1), D.status);
            }
            break;
        }
        if (tid == 0 && k + 2 < P.K) {
            const uint32_t bar = (k & 1) ? bar1 : bar0;
            mbar_arrive_expect_tx(bar, rowbytes);
            bulk_g2s(smem_u32((k & 1) ? ebuf1 : ebuf0), e_g + (size_t)(k + 2) * P.Mp, rowbytes, bar);
        }
        if (++j == P.n_rx) { j = 0; ++i; }
    }
    if (pix_ok) b_out[(size_t)row * P.W + col] = sum + comp;
}

size_t backproject_smem(const mbir_geometry* g)
{
    const GeomParams& P = g->P;
    size_t esz = P.precision == MBIR_PREC_BF16 ? 2 : 4;
    size_t tsz = P.precision == MBIR_PREC_BF16 ? 4 : 8;
    size_t tab = ((size_t)P.Gt * (P.Q + 1) * table_stride(P.Tw4) * tsz + 127) & ~(size_t)127;
    size_t eb = ((size_t)P.Mp * esz + 127) & ~(size_t)127;
    return tab + 2 * eb + 64;
}

template <int NL, int MODE, bool BF16>
static cudaError_t launch_bwd_t(const mbir_geometry* g, const DevPtrs& D, const void* e, float* b, cudaStream_t st)
{
    const GeomParams& P = g->P;
    size_t sm = backproject_smem(g);
    auto kern = backproject_kernel<NL, MODE, BF16>;
    cudaError_t ce = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (ce != cudaSuccess) return ce;
    dim3 grid((P.W + 31) / 32, (P.H + kBwdRows - 1) / kBwdRows);
    using Tab = typename TabT<BF16>::type;
    const Tab* tab = BF16 ? (const Tab*)(const void*)g->d_tab_bf16 : (const Tab*)(const void*)g->d_tab;
    kern<<<grid, kBwdThreads, sm, st>>>(P, D, tab, (const typename ET<BF16>::type*)e, b);
    return cudaGetLastError();
}

DevPtrs dev_ptrs(const mbir_geometry* g)
{
    DevPtrs D;
    D.rows = g->d_rows;
    D.colx = g->d_colx;
    D.pos = g->d_pos;
    D.txpos = g->d_txpos;
    D.rxpos = g->d_rxpos;
    D.legs = g->d_legs;
    D.hidx = g->d_hidx;
    D.status = g->d_status;
    return D;
}

template <int MODE, bool BF16>
static cudaError_t launch_bwd_nl(const mbir_geometry* g, const void* e, float* b, cudaStream_t st)
{
    DevPtrs D = dev_ptrs(g);
    if constexpr (MODE == kModeTAB) {
        return launch_bwd_t<1, MODE, BF16>(g, D, e, b, st);
    } else {
        if (g->P.L <= 2) return launch_bwd_t<2, MODE, BF16>(g, D, e, b, st);
        if (g->P.L <= 4) return launch_bwd_t<4, MODE, BF16>(g, D, e, b, st);
        return launch_bwd_t<8, MODE, BF16>(g, D, e, b, st);
    }
}

cudaError_t launch_backproject(const mbir_geometry* g, const float* e_pad, const __nv_bfloat16* e_bf, float* b,
                               cudaStream_t st)
{
    const bool bf = g->P.precision == MBIR_PREC_BF16;
    if (g->P.mode == MBIR_MODE_TAB)
        return bf ? launch_bwd_nl<kModeTAB, true>(g, e_bf, b, st) : launch_bwd_nl<kModeTAB, false>(g, e_pad, b, st);
    return bf ? launch_bwd_nl<kModeOTF, true>(g, e_bf, b, st) : launch_bwd_nl<kModeOTF, false>(g, e_pad, b, st);
}

}  // namespace mbir
