// Small kernels: the TAB-mode leg table (every leg solved once per geometry,
// the paper's "compute only once"), per-pair diagnostics for parity tests,
// and residual-row padding / BF16 conversion.
#include <algorithm>

#include "device_common.cuh"

namespace mbir {

// one TAB leg per (row, distinct offset); hsign != 0 marks a tilted transmitter's
// signed offset (its eq. 12 factor depends on the side of the ray)
template <int NL>
__global__ void build_legs_kernel(GeomParams P, const RowInfo* __restrict__ rows, const float2* __restrict__ hv,
                                  const int* __restrict__ hsign, float4* __restrict__ legs)
{
    const long long total = (long long)P.H * P.nh;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int row = (int)(t / P.nh), hix = (int)(t - (long long)row * P.nh);
        RowInfo ri = load_row(rows, row);
        float2 h = hv[hix];
        Leg L = solve_leg<NL>(P, ri, df{h.x, h.y}, hsign[hix]);
        legs[t] = make_float4(L.Th, L.Tl, L.g, L.phi);
    }
}

cudaError_t launch_build_legs(const mbir_geometry* g, const int* d_hsign, const float2* d_hvals, cudaStream_t st)
{
    const GeomParams& P = g->P;
    long long total = (long long)P.H * P.nh;
    int blocks = (int)std::min<long long>((total + 255) / 256, 152LL * 16);
    if (P.L <= 2)
        build_legs_kernel<2><<<blocks, 256, 0, st>>>(P, g->d_rows, d_hvals, d_hsign, g->d_legs);
    else if (P.L <= 4)
        build_legs_kernel<4><<<blocks, 256, 0, st>>>(P, g->d_rows, d_hvals, d_hsign, g->d_legs);
    else
        build_legs_kernel<8><<<blocks, 256, 0, st>>>(P, g->d_rows, d_hvals, d_hsign, g->d_legs);
    return cudaGetLastError();
}

template <int NL, int MODE>
__global__ void pair_quantities_kernel(GeomParams P, DevPtrs D, const int* __restrict__ pix, const int* __restrict__ ks,
                                       int n, double* __restrict__ T, float* __restrict__ gam, float* __restrict__ w)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int v = pix[t], k = ks[t];
    const int row = v / P.W, col = v - row * P.W;
    const int i = k / P.n_rx;
    RowInfo ri = load_row(D.rows, row);
    Leg tx = get_leg<NL, MODE>(P, D, ri, row, col, D.txpos[i]);
    Leg rx = get_leg<NL, MODE>(P, D, ri, row, col, D.rxpos[k]);
    df s = df_add({tx.Th, tx.Tl}, {rx.Th, rx.Tl});
    T[t] = (double)s.hi + (double)s.lo;
    gam[t] = (tx.g + rx.g) * P.inv_gscale;
    w[t] = ri.tau * tx.phi * rx.phi;
}

cudaError_t launch_pair_quantities(const mbir_geometry* g, const int* pix, const int* k, int n, double* T,
                                   float* gam, float* w, cudaStream_t st)
{
    const GeomParams& P = g->P;
    DevPtrs D = dev_ptrs(g);
    int blocks = (n + 127) / 128;
    if (P.mode == MBIR_MODE_TAB)
        pair_quantities_kernel<1, kModeTAB><<<blocks, 128, 0, st>>>(P, D, pix, k, n, T, gam, w);
    else if (P.L <= 2)
        pair_quantities_kernel<2, kModeOTF><<<blocks, 128, 0, st>>>(P, D, pix, k, n, T, gam, w);
    else if (P.L <= 4)
        pair_quantities_kernel<4, kModeOTF><<<blocks, 128, 0, st>>>(P, D, pix, k, n, T, gam, w);
    else
        pair_quantities_kernel<8, kModeOTF><<<blocks, 128, 0, st>>>(P, D, pix, k, n, T, gam, w);
    return cudaGetLastError();
}

// active pairs and in-record taps of one apply (geometry only)
template <int NL, int MODE>
__global__ void count_taps_kernel(GeomParams P, DevPtrs D, unsigned long long* __restrict__ out)
{
    const int N = P.W * P.H;
    unsigned long long np = 0, nt = 0;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < N; v += gridDim.x * blockDim.x) {
        const int row = v / P.W, col = v - row * P.W;
        RowInfo ri = load_row(D.rows, row);
        if (ri.tvert >= (float)(P.M - 1)) continue;
        Leg tx = {0.f, 0.f, 0.f, 0.f};
        for (int k = 0, i = 0, j = 0; k < P.K; ++k) {
            if (j == 0) tx = get_leg<NL, MODE>(P, D, ri, row, col, D.txpos[i]);
            Leg rx = get_leg<NL, MODE>(P, D, ri, row, col, D.rxpos[k]);
            Pair pr = make_pair(P, tx, rx, ri.tau);
            if (pr.w != 0.0f && pr.n0 >= 0 && pr.n0 + 1 < P.M) {
                int last = min(pr.n0 + P.Tw, P.M - 1);         // taps n0+1 .. n0+Tw inside the record
                int t = last - pr.n0;
                if (pr.flag0 && last == pr.n0 + P.Tw) --t;      // tau = t0 is outside the window
                ++np;
                nt += t;
            }
            if (++j == P.n_rx) { j = 0; ++i; }
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        np += __shfl_xor_sync(0xffffffffu, np, o);
        nt += __shfl_xor_sync(0xffffffffu, nt, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(out, np);        // integer sums: order-independent
        atomicAdd(out + 1, nt);
    }
}

cudaError_t launch_count_taps(const mbir_geometry* g, unsigned long long* d_out, cudaStream_t st)
{
    const GeomParams& P = g->P;
    DevPtrs D = dev_ptrs(g);
    int N = P.W * P.H;
    int blocks = std::min((N + 127) / 128, 152 * 8);
    if (P.mode == MBIR_MODE_TAB)
        count_taps_kernel<1, kModeTAB><<<blocks, 128, 0, st>>>(P, D, d_out);
    else if (P.L <= 2)
        count_taps_kernel<2, kModeOTF><<<blocks, 128, 0, st>>>(P, D, d_out);
    else if (P.L <= 4)
        count_taps_kernel<4, kModeOTF><<<blocks, 128, 0, st>>>(P, D, d_out);
    else
        count_taps_kernel<8, kModeOTF><<<blocks, 128, 0, st>>>(P, D, d_out);
    return cudaGetLastError();
}

// K x M (float or bfloat16) -> K x Mp float with zeros in [M, Mp)
__global__ void pad_rows_kernel(GeomParams P, const void* __restrict__ src, int src_bf16, float* __restrict__ dst)
{
    const int k = blockIdx.x;
    for (int n = threadIdx.x; n < P.Mp; n += blockDim.x) {
        float v = 0.0f;
        if (n < P.M) {
            size_t s = (size_t)k * P.M + n;
            v = src_bf16 ? __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(src)[s])
                         : reinterpret_cast<const float*>(src)[s];
        }
        dst[(size_t)k * P.Mp + n] = v;
    }
}

// Loads pad_rows_kernel (see load_backproject_partials).
cudaError_t load_pad_rows()
{
    cudaFuncAttributes a;
    return cudaFuncGetAttributes(&a, pad_rows_kernel);
}

cudaError_t launch_pad_rows(const mbir_geometry* g, const void* src, int src_bf16, float* dst, cudaStream_t st)
{
    pad_rows_kernel<<<g->P.K, 256, 0, st>>>(g->P, src, src_bf16, dst);
    return cudaGetLastError();
}

// A wait that nothing completes: the mbarrier expects one arrival that never
// comes.  The bounded wait gives up after max_cycles, records the failure and
// returns, exactly as the apply kernels do when a bulk copy never lands.
__global__ void bounded_wait_selftest_kernel(long long max_cycles, int* status)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(smem_u32(&bar), 1);
        fence_mbar_init();
    }
    __syncthreads();
    const uint32_t b = smem_u32(&bar);
    long long start = clock64();
    bool ok = false;
    while (!(ok = mbar_try_wait(b, 0))) {
        if (clock64() - start > max_cycles) break;
    }
    if (!ok && threadIdx.x == 0) atomicExch(status, 1);
}

}  // namespace mbir

extern "C" int mbir_selftest_bounded_wait(long long max_cycles)
{
    if (max_cycles <= 0 || max_cycles > 4000000000LL) return MBIR_ERR_INVALID_ARG;
    int* d = nullptr;
    if (cudaMalloc(&d, sizeof(int)) != cudaSuccess) return MBIR_ERR_OOM;
    int h = 0;
    cudaError_t e = cudaMemset(d, 0, sizeof(int));
    if (e == cudaSuccess) {
        mbir::bounded_wait_selftest_kernel<<<1, 32>>>(max_cycles, d);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(&h, d, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return MBIR_ERR_CUDA;
    return h ? MBIR_ERR_TIMEOUT : MBIR_OK;
}
