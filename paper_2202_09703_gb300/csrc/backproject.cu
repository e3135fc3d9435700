// A^T r (adjoint of eq. 13).  Thread = pixel.  A persistent grid of one CTA
// per SM holds the pulse table in shared memory once; each CTA runs two
// independent tile workers (16 x 32 pixels each, synchronised by their own
// named barrier) that take work items = (pixel tile, range of A-scans: whole
// transmitter groups for the full image) from a shared counter, longest
// estimated item first.  A worker walks its A-scans in (Tx, receiver) order, keeping
// the pixel's transmit leg while the receiver changes.  Residual rows are
// staged in shared memory by 1-D bulk copies (TMA engine) into a 3-stage ring
// guarded by mbarriers with bounded waits.  Every tap of a pair shares one
// table phase, so the tap loop is two packed FP32 FMAs over four dot products,
// combined once per pair; per-pair sums are added across A-scans with
// Neumaier compensation.  Each item writes its own partial image; a second
// kernel adds the groups in a fixed order, so results are reproducible.
#include <algorithm>

#include "apply_common.cuh"

namespace mbir {

constexpr int kBwdRows = kBwdTileRows;
constexpr int kBwdHalfThreads = kBwdWorkerThreads;   // threads per tile worker
constexpr int kBwdThreads = 2 * kBwdHalfThreads;     // at most two workers per CTA
constexpr int kBwdMaxStages = 3;
constexpr size_t kSmemLimit = 227 * 1024;

template <int NL, int MODE, bool BF16>
__global__ void __launch_bounds__(kBwdThreads, 1)
    backproject_kernel(GeomParams P, DevPtrs D, const typename TabT<BF16>::type* __restrict__ tab_g,
                       const typename ET<BF16>::type* __restrict__ e_g, const int4* __restrict__ items,
                       int nitems, int* __restrict__ counter, float* __restrict__ partial, int nst, int3 lat)
{
    using Tab = typename TabT<BF16>::type;
    using E = typename ET<BF16>::type;
    extern __shared__ __align__(128) unsigned char smem[];
    const int S = table_stride(P.Tw4);
    const int R = P.Q + 1;
    const size_t tab_bytes = ((size_t)P.Gt * R * S * sizeof(Tab) + 127) & ~(size_t)127;
    const size_t ebytes = ((size_t)P.Mp * sizeof(E) + 127) & ~(size_t)127;
    Tab* tab = reinterpret_cast<Tab*>(smem);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int h = warp / kBwdRows, hw = warp % kBwdRows, ht = tid % kBwdHalfThreads;
    const int halves = blockDim.x / kBwdHalfThreads;
    E* ering = reinterpret_cast<E*>(smem + tab_bytes + (size_t)h * nst * ebytes);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + tab_bytes + (size_t)halves * nst * ebytes);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(bars + halves * nst) + h;
    volatile int* next_item = reinterpret_cast<volatile int*>(bars + halves * nst) + 2 + h;
    const uint32_t bar0 = smem_u32(bars + h * nst);

    load_table_smem(tab, tab_g, tab_bytes, tid, blockDim.x);
    if (tid == 0) {
        for (int b = 0; b < halves * nst; ++b) mbar_init(smem_u32(bars + b), 1);
        for (int b = 0; b < halves; ++b) reinterpret_cast<volatile int*>(bars + halves * nst)[b] = 0;
        fence_mbar_init();
    }
    __syncthreads();

    uint32_t par = 0;                    // expected phase parity per stage (bit s)
    for (;;) {
        if (ht == 0) *next_item = atomicAdd(counter, 1);
        worker_barrier(h);
        const int it = *next_item;
        worker_barrier(h);               // every thread has read the slot before it is reused
        if (it >= nitems) break;
        if (!backproject_item<NL, MODE, BF16>(P, D, tab, e_g, __ldg(items + it), partial, ering, bar0, nst, ebytes,
                                              abort_flag, par, h, hw, lane, ht, lat))
            break;
    }
}

// b = sum over transmitter groups of the partial images (fixed order,
// compensated); pixels of tiles that cannot reach the record are zero.
__global__ void backproject_reduce_kernel(GeomParams P, const RowInfo* __restrict__ rows,
                                          const float* __restrict__ partial, int ngroups, float* __restrict__ b)
{
    const int N = P.W * P.H;
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= N) return;
    const int row = v / P.W;
    const int row0 = (row / kBwdRows) * kBwdRows;
    if (__ldg(&rows[row0].tvert) >= (float)(P.M - 1)) {
        b[v] = 0.0f;
        return;
    }
    float s = 0.0f, c = 0.0f;
    for (int g = 0; g < ngroups; ++g) {
        const float val = partial[(size_t)g * N + v];
        const float t = s + val;
        c += (fabsf(s) >= fabsf(val)) ? (s - t) + val : (val - t) + s;
        s = t;
    }
    b[v] = s + c;
}

// b on the pixels (r, c) = (i s + r0, j s + c0) of one lattice, lat = (s, r0, c0), Wc x Hc of them, from
// the partial images of its items: one warp per pixel, lane l compensating groups l, l + 32, ..., then a
// fixed shuffle tree (deterministic); pixels of lattice tiles that cannot reach the record (no items) are
// zero.  Other pixels of b are not written.
__global__ void backproject_reduce_lattice_kernel(GeomParams P, const RowInfo* __restrict__ rows,
                                                  const float* __restrict__ partial, int ngroups, int3 lat, int Wc,
                                                  int Nc, float* __restrict__ b)
{
    const int N = P.W * P.H;
    const int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (t >= Nc) return;                         // whole warps
    const int ri = t / Wc, ci = t - ri * Wc;
    const int row = ri * lat.x + lat.y, col = ci * lat.x + lat.z;
    const int v = row * P.W + col;
    const int row0 = (ri / kBwdRows) * kBwdRows * lat.x + lat.y;
    if (__ldg(&rows[row0].tvert) >= (float)(P.M - 1)) {
        if (lane == 0) b[v] = 0.0f;
        return;
    }
    float s = 0.0f, c = 0.0f;
    for (int g = lane; g < ngroups; g += 32) {
        const float val = partial[(size_t)g * N + v];
        const float t2 = s + val;
        c += (fabsf(s) >= fabsf(val)) ? (s - t2) + val : (val - t2) + s;
        s = t2;
    }
    float tot = s + c;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
    if (lane == 0) b[v] = tot;
}

// Estimated A^T r cost per (16 x 32 pixel tile, transmitter position), in
// warp tap iterations: a warp runs the whole tap loop (Tw4 taps) for an
// A-scan as soon as one of its pixels has an active pair, and every warp pays
// a fixed overhead per A-scan (leg loads, pair set-up, ring wait, barrier).
constexpr float kBwdAscanOverhead = 16.0f;

template <int NL, int MODE>
__global__ void __launch_bounds__(kBwdHalfThreads)
    bwd_tile_cost_kernel(GeomParams P, DevPtrs D, int ntc, float* __restrict__ cost)
{
    __shared__ int s_active[kBwdRows];
    const int tile = blockIdx.x;
    const int tr = tile / ntc, tc = tile - tr * ntc;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row = tr * kBwdRows + warp, col = tc * 32 + lane;
    const bool pix_ok = col < P.W && row < P.H;
    const RowInfo ri = load_row(D.rows, min(row, P.H - 1));
    const bool row_ok = pix_ok && ri.tvert < (float)(P.M - 1);
    const int colc = min(col, P.W - 1);
    for (int i = 0; i < P.n_tx; ++i) {
        Leg tx = {0.f, 0.f, 0.f, 0.f};
        if (row_ok) tx = get_leg<NL, MODE>(P, D, ri, row, colc, __ldg(D.txpos + i));
        int na = 0;
        for (int j = 0; j < P.n_rx; ++j) {
            const int k = i * P.n_rx + j;
            bool act = false;
            if (row_ok) {
                const Leg rx = get_leg<NL, MODE>(P, D, ri, row, colc, __ldg(D.rxpos + k));
                const Pair pr = make_pair(P, tx, rx, ri.tau);
                act = pr.w != 0.0f && pr.n0 >= 0 && pr.n0 + 1 < P.M;
            }
            na += __any_sync(0xffffffffu, act) ? 1 : 0;
        }
        if (lane == 0) s_active[warp] = na;
        __syncthreads();
        if (threadIdx.x == 0) {
            int tot = 0;
            for (int w = 0; w < kBwdRows; ++w) tot += s_active[w];
            cost[(size_t)tile * P.n_tx + i] = (float)tot * P.Tw4 + kBwdAscanOverhead * kBwdRows * P.n_rx;
        }
        __syncthreads();
    }
}

// Fills h_cost (ntr x ntc x n_tx, host) with the estimates above; synchronous.
cudaError_t backproject_tile_costs(const mbir_geometry* g, int ntr, int ntc, float* h_cost, cudaStream_t st)
{
    const GeomParams& P = g->P;
    const size_t n = (size_t)ntr * ntc * P.n_tx;
    float* d = nullptr;
    cudaError_t ce = cudaMalloc((void**)&d, sizeof(float) * std::max<size_t>(n, 1));
    if (ce != cudaSuccess) return ce;
    DevPtrs D = dev_ptrs(g);
    const int blocks = ntr * ntc;
    if (P.mode == MBIR_MODE_TAB)
        bwd_tile_cost_kernel<1, kModeTAB><<<blocks, kBwdHalfThreads, 0, st>>>(P, D, ntc, d);
    else if (P.L <= 2)
        bwd_tile_cost_kernel<2, kModeOTF><<<blocks, kBwdHalfThreads, 0, st>>>(P, D, ntc, d);
    else if (P.L <= 4)
        bwd_tile_cost_kernel<4, kModeOTF><<<blocks, kBwdHalfThreads, 0, st>>>(P, D, ntc, d);
    else
        bwd_tile_cost_kernel<8, kModeOTF><<<blocks, kBwdHalfThreads, 0, st>>>(P, D, ntc, d);
    ce = cudaGetLastError();
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(h_cost, d, sizeof(float) * n, cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    cudaFree(d);
    return ce;
}

// Shared memory of a (workers, stages) configuration; 0 if it exceeds the limit.
static size_t bwd_smem_for(const GeomParams& P, int halves, int nst)
{
    size_t esz = P.precision == MBIR_PREC_BF16 ? 2 : 4;
    size_t tsz = P.precision == MBIR_PREC_BF16 ? 4 : 8;
    size_t tab = ((size_t)P.Gt * (P.Q + 1) * table_stride(P.Tw4) * tsz + 127) & ~(size_t)127;
    size_t eb = ((size_t)P.Mp * esz + 127) & ~(size_t)127;
    size_t total = tab + (size_t)halves * nst * eb + 8 * halves * nst + 32;   // + abort flags, item slots
    return total <= kSmemLimit ? total : 0;
}

// Picks two tile workers with a 3-deep ring if it fits, else 2-deep, else one
// worker; false if even that exceeds shared memory.
bool backproject_config(const GeomParams& P, int* halves, int* stages)
{
    const int opts[3][2] = {{2, 3}, {2, 2}, {1, 2}};
    for (auto& o : opts)
        if (bwd_smem_for(P, o[0], o[1])) {
            *halves = o[0];
            *stages = o[1];
            return true;
        }
    return false;
}

size_t backproject_smem(const mbir_geometry* g) { return bwd_smem_for(g->P, g->bwd_halves, g->bwd_stages); }

int backproject_tile_rows() { return kBwdRows; }

template <int NL, int MODE, bool BF16>
static cudaError_t launch_bwd_t(const mbir_geometry* g, const DevPtrs& D, const void* e, float* b, cudaStream_t st)
{
    const GeomParams& P = g->P;
    size_t sm = backproject_smem(g);
    auto kern = backproject_kernel<NL, MODE, BF16>;
    cudaError_t ce = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (ce != cudaSuccess) return ce;
    using Tab = typename TabT<BF16>::type;
    const Tab* tab = BF16 ? (const Tab*)(const void*)g->d_tab_bf16 : (const Tab*)(const void*)g->d_tab;
    if (g->n_items > 0) {
        ce = cudaMemsetAsync(g->d_bwd_counter, 0, sizeof(int), st);
        if (ce != cudaSuccess) return ce;
        int grid = std::min(g->n_sm, (g->n_items + g->bwd_halves - 1) / g->bwd_halves);
        kern<<<grid, g->bwd_halves * kBwdHalfThreads, sm, st>>>(P, D, tab, (const typename ET<BF16>::type*)e,
                                                                g->d_items, g->n_items, g->d_bwd_counter,
                                                                g->w_bpart, g->bwd_stages, make_int3(1, 0, 0));
        ce = cudaGetLastError();
        if (ce != cudaSuccess) return ce;
    }
    const int N = P.W * P.H;
    backproject_reduce_kernel<<<(N + 255) / 256, 256, 0, st>>>(P, g->d_rows, g->w_bpart, g->n_groups, b);
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
    if (g->d_tb4_bop) return launch_backproject_tcs(g, e_pad, e_bf, b, st);
    if (g->P.mode == MBIR_MODE_TAB)
        return bf ? launch_bwd_nl<kModeTAB, true>(g, e_bf, b, st) : launch_bwd_nl<kModeTAB, false>(g, e_pad, b, st);
    return bf ? launch_bwd_nl<kModeOTF, true>(g, e_bf, b, st) : launch_bwd_nl<kModeOTF, false>(g, e_pad, b, st);
}

// Same launch as launch_backproject, with the per-group partial images in a
// caller-provided buffer (n_groups x N floats) instead of the handle's.
template <int NL, int MODE, bool BF16>
static cudaError_t launch_bwd_partials_t(const mbir_geometry* g, const void* e, float* b, float* partial,
                                         cudaStream_t st)
{
    const GeomParams& P = g->P;
    size_t sm = backproject_smem(g);
    auto kern = backproject_kernel<NL, MODE, BF16>;
    cudaError_t ce = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (ce != cudaSuccess) return ce;
    using Tab = typename TabT<BF16>::type;
    const Tab* tab = BF16 ? (const Tab*)(const void*)g->d_tab_bf16 : (const Tab*)(const void*)g->d_tab;
    if (g->n_items > 0) {
        ce = cudaMemsetAsync(g->d_bwd_counter, 0, sizeof(int), st);
        if (ce != cudaSuccess) return ce;
        int grid = std::min(g->n_sm, (g->n_items + g->bwd_halves - 1) / g->bwd_halves);
        kern<<<grid, g->bwd_halves * kBwdHalfThreads, sm, st>>>(P, dev_ptrs(g), tab,
                                                                (const typename ET<BF16>::type*)e, g->d_items,
                                                                g->n_items, g->d_bwd_counter, partial,
                                                                g->bwd_stages, make_int3(1, 0, 0));
        ce = cudaGetLastError();
        if (ce != cudaSuccess) return ce;
    }
    const int N = P.W * P.H;
    backproject_reduce_kernel<<<(N + 255) / 256, 256, 0, st>>>(P, g->d_rows, partial, g->n_groups, b);
    return cudaGetLastError();
}

// A^T r on the pixels of one lattice only (CUDA-core kernel): items = (lattice tile row, lattice tile
// column, A-scan range, group) of that lattice, partial = ngroups x N floats.
template <int NL, int MODE, bool BF16>
static cudaError_t launch_bwd_lattice_t(const mbir_geometry* g, const int4* items, int nitems, int ngroups, int3 lat,
                                        float* partial, const void* e, float* b, cudaStream_t st)
{
    const GeomParams& P = g->P;
    size_t sm = backproject_smem(g);
    auto kern = backproject_kernel<NL, MODE, BF16>;
    cudaError_t ce = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (ce != cudaSuccess) return ce;
    using Tab = typename TabT<BF16>::type;
    const Tab* tab = BF16 ? (const Tab*)(const void*)g->d_tab_bf16 : (const Tab*)(const void*)g->d_tab;
    if (nitems > 0) {
        ce = cudaMemsetAsync(g->d_bwd_counter, 0, sizeof(int), st);
        if (ce != cudaSuccess) return ce;
        int grid = std::min(g->n_sm, (nitems + g->bwd_halves - 1) / g->bwd_halves);
        kern<<<grid, g->bwd_halves * kBwdHalfThreads, sm, st>>>(P, dev_ptrs(g), tab,
                                                                (const typename ET<BF16>::type*)e, items, nitems,
                                                                g->d_bwd_counter, partial, g->bwd_stages, lat);
        ce = cudaGetLastError();
        if (ce != cudaSuccess) return ce;
    }
    const int Hc = (P.H - lat.y + lat.x - 1) / lat.x, Wc = (P.W - lat.z + lat.x - 1) / lat.x;
    const int Nc = Hc * Wc;
    if (Nc > 0)
        backproject_reduce_lattice_kernel<<<(Nc + 7) / 8, 256, 0, st>>>(P, g->d_rows, partial, ngroups, lat, Wc, Nc,
                                                                       b);
    return cudaGetLastError();
}

cudaError_t launch_backproject_lattice(const mbir_geometry* g, const int4* items, int nitems, int ngroups, int3 lat,
                                       float* partial, const float* e_pad, const __nv_bfloat16* e_bf, float* b,
                                       cudaStream_t st)
{
    const bool bf = g->P.precision == MBIR_PREC_BF16;
    const void* e = bf ? (const void*)e_bf : (const void*)e_pad;
    if (g->P.mode == MBIR_MODE_TAB)
        return bf ? launch_bwd_lattice_t<1, kModeTAB, true>(g, items, nitems, ngroups, lat, partial, e, b, st)
                  : launch_bwd_lattice_t<1, kModeTAB, false>(g, items, nitems, ngroups, lat, partial, e, b, st);
    if (g->P.L <= 2)
        return bf ? launch_bwd_lattice_t<2, kModeOTF, true>(g, items, nitems, ngroups, lat, partial, e, b, st)
                  : launch_bwd_lattice_t<2, kModeOTF, false>(g, items, nitems, ngroups, lat, partial, e, b, st);
    if (g->P.L <= 4)
        return bf ? launch_bwd_lattice_t<4, kModeOTF, true>(g, items, nitems, ngroups, lat, partial, e, b, st)
                  : launch_bwd_lattice_t<4, kModeOTF, false>(g, items, nitems, ngroups, lat, partial, e, b, st);
    return bf ? launch_bwd_lattice_t<8, kModeOTF, true>(g, items, nitems, ngroups, lat, partial, e, b, st)
              : launch_bwd_lattice_t<8, kModeOTF, false>(g, items, nitems, ngroups, lat, partial, e, b, st);
}

// Loads the FP32 CUDA-core adjoint kernels that launch_backproject_partials runs for g (a query of their
// attributes loads a lazily loaded module), so that a later launch does not load them.
cudaError_t load_backproject_partials(const mbir_geometry* g)
{
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, backproject_reduce_kernel);
    if (e != cudaSuccess) return e;
    if (g->P.mode == MBIR_MODE_TAB) return cudaFuncGetAttributes(&a, backproject_kernel<1, kModeTAB, false>);
    if (g->P.L <= 2) return cudaFuncGetAttributes(&a, backproject_kernel<2, kModeOTF, false>);
    if (g->P.L <= 4) return cudaFuncGetAttributes(&a, backproject_kernel<4, kModeOTF, false>);
    return cudaFuncGetAttributes(&a, backproject_kernel<8, kModeOTF, false>);
}

cudaError_t launch_backproject_partials(const mbir_geometry* g, const float* e_pad, const __nv_bfloat16* e_bf,
                                        float* b, float* partial, cudaStream_t st)
{
    const bool bf = g->P.precision == MBIR_PREC_BF16;
    if (g->P.mode == MBIR_MODE_TAB)
        return bf ? launch_bwd_partials_t<1, kModeTAB, true>(g, e_bf, b, partial, st)
                  : launch_bwd_partials_t<1, kModeTAB, false>(g, e_pad, b, partial, st);
    if (g->P.L <= 2)
        return bf ? launch_bwd_partials_t<2, kModeOTF, true>(g, e_bf, b, partial, st)
                  : launch_bwd_partials_t<2, kModeOTF, false>(g, e_pad, b, partial, st);
    if (g->P.L <= 4)
        return bf ? launch_bwd_partials_t<4, kModeOTF, true>(g, e_bf, b, partial, st)
                  : launch_bwd_partials_t<4, kModeOTF, false>(g, e_pad, b, partial, st);
    return bf ? launch_bwd_partials_t<8, kModeOTF, true>(g, e_bf, b, partial, st)
              : launch_bwd_partials_t<8, kModeOTF, false>(g, e_pad, b, partial, st);
}

}  // namespace mbir
