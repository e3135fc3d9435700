// A x of the BF16 storage form on the tensor cores.
//
// With the bilinear pulse table, a pair (first tap n0, table rows of its
// phase and attenuation bins, weights c) adds c T[row][m] x_v to sample
// n0 + 1 + m of its A-scan (eq. 13).  Grouping the pairs of an A-scan by n0,
//     S[n0][row] = sum over pairs with that n0 of their weight on `row` times x_v,
//     y[n] = sum_row sum_m T[row][m] S[n - 1 - m][row],
// so for a tile of 128 values of n0 the work is one matrix product
//     U (128 x taps) = S (128 x rows) T (rows x taps)
// followed by the sums of U along its anti-diagonals, y[n0 + 1 + m] += U[n0][m].
// S is accumulated in FP32 in shared memory (each cell owned by one thread,
// pairs added in record order: deterministic), rounded once to BF16 for the
// tcgen05 MMA (FP32 accumulation in tensor memory), in two column halves so
// that the FP32 accumulator stays small.  The tau = t0 tap of flagged pairs
// (outside the open window of eq. 10) is subtracted from y directly.
#include <algorithm>
#include <cmath>
#include <vector>

#include "tc_apply.cuh"

namespace mbir {

TfLayout tf_layout(const GeomParams& P)
{
    TfLayout L{};
    L.ncols = P.G * (P.Q + 1);
    L.c0 = std::min(((L.ncols / 2) + 15) & ~15, L.ncols);
    L.k0 = L.c0;                                        // K of the first half (multiple of 16)
    L.k1 = ((L.ncols - L.c0) + 15) & ~15;               // K of the second half, padded
    L.ka = std::max(L.k0, L.k1);                        // columns of the BF16 operand buffer
    L.kb = L.k0 + L.k1;                                 // columns of the table operand image
    L.ntap = (P.Tw + 15) & ~15;                         // MMA N (taps), multiple of 16
    L.astride = L.k0 + 1;                               // FP32 row stride, first half
    L.astride1 = std::max(L.k1 + 1, L.ntap + 1);        // second half (later the product tile)
    L.ustride = L.ntap + 1;
    L.off_b = 1024;
    // first-half accumulator; the BF16 operand buffer is written over it once its sums are in registers
    L.off_acc = (L.off_b + (size_t)L.ntap * L.kb * 2 + 1023) & ~(size_t)1023;
    // the two halves' BF16 operands follow each other over the first half's sums
    const size_t acc0 = std::max((size_t)kTfTile * L.astride * 4, (size_t)2 * kTfTile * L.ka * 2);
    L.off_a = L.off_acc;
    L.off_acc1 = (L.off_acc + acc0 + 127) & ~(size_t)127;
    L.off_y = (L.off_acc1 + (size_t)kTfTile * L.astride1 * 4 + 127) & ~(size_t)127;
    L.ylen = ((P.M + kTfTile - 1) / kTfTile) * kTfTile + L.ntap + 2;   // every anti-diagonal target
    L.smem = L.off_y + (size_t)L.ylen * 4;
    const int per_thread = (kTfTile * (L.k0 / 8) + kTfThreads - 1) / kTfThreads;
    L.ok = L.ntap <= 256 && L.k0 > 0 && L.k0 % 16 == 0 && L.smem <= 227 * 1024 && L.ncols <= 4096 &&
           per_thread <= kTfStage;
    return L;
}

Tf3Layout tf3_layout(const GeomParams& P)
{
    Tf3Layout L{};
    const int R = P.Q + 1;
    L.phsplit = R / 2;
    L.ncol[0] = (L.phsplit + 1) * P.G;
    L.ncol[1] = (R - L.phsplit) * P.G;
    L.pstride = std::max(L.phsplit + 1, R - L.phsplit);
    L.kb = (L.pstride * P.G + 15) & ~15;
    L.kc = std::min(48, L.kb);
    L.ntap = (P.Tw + 15) & ~15;
    L.astride = (L.kb + 4 + 3) & ~3;                   // float4 rows, not a multiple of 32 banks
    L.ustride = L.ntap + 1;
    L.bhalf = (size_t)2 * L.ntap * L.kb * 2;
    L.off_b = 1024;
    L.off_s = (L.off_b + L.bhalf + 1023) & ~(size_t)1023;
    L.off_a = (L.off_s + (size_t)kTfTile * std::max(L.astride, L.ustride) * 4 + 1023) & ~(size_t)1023;
    L.ylen = ((P.M + kTfTile - 1) / kTfTile) * kTfTile + L.ntap + 2;
    for (L.nbuf = 2; L.nbuf >= 1; --L.nbuf) {
        L.off_y = (L.off_a + (size_t)L.nbuf * 2 * kTfTile * L.kc * 2 + 127) & ~(size_t)127;
        L.smem = L.off_y + (size_t)L.ylen * 4;
        if (L.smem <= 227 * 1024) break;
    }
    if (L.nbuf < 1) L.nbuf = 1;
    L.ok = R >= 2 && L.ntap <= 128 && L.smem <= 227 * 1024 && (P.Q + 1) * P.G <= 4096 && L.kc % 16 == 0;
    return L;
}

__global__ void tc_gather_x_kernel(long long nrec, const int2* __restrict__ rkey, const float* __restrict__ x,
                                   float* __restrict__ xr)
{
    tc_gather_x(nrec, rkey, x, xr);
}

__global__ void __launch_bounds__(kTfThreads, 1) fwd_tc_kernel(TcFwdView V, int* __restrict__ status)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    tc_header_init(smem, kTfCols);
    const uint32_t tmem = *reinterpret_cast<volatile uint32_t*>(smem + 8);
    uint32_t phase = 0;
    tc_forward_pool(V, smem, tmem, phase, status);
    tc_header_release(smem, tmem, kTfCols);
}

__global__ void __launch_bounds__(kTfThreads, 1) fwd_tc32_kernel(TcFwd32View V, int* __restrict__ status)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    tc_header_init(smem, kTf3Cols);
    const uint32_t tmem = *reinterpret_cast<volatile uint32_t*>(smem + 8);
    uint32_t phase = 0, bphase = 0;
    tc_forward32_pool(V, smem, tmem, phase, bphase, status);
    tc_header_release(smem, tmem, kTf3Cols);
}

// first record of every sample n0 of every A-scan (records sorted by n0)
__global__ void tf_n0_off_kernel(GeomParams P, const long long* __restrict__ rec_off, const int2* __restrict__ rkey,
                                 int* __restrict__ n0_off)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (long long)P.K * (P.M + 1)) return;
    const int k = (int)(i / (P.M + 1)), n = (int)(i - (long long)k * (P.M + 1));
    const long long base = rec_off[k];
    int lo = 0, hi = (int)(rec_off[k + 1] - base);
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if ((rkey[base + mid].y >> kRecShift) < n) lo = mid + 1;
        else hi = mid;
    }
    n0_off[i] = lo;
}

// start of every phase class (table phase mod 4) inside every (A-scan, n0)
// bucket; buckets are ordered by class.  *too_long is set for a bucket of
// more than 65535 records (the offsets are 16-bit).
__global__ void tf_grp_off_kernel(GeomParams P, const long long* __restrict__ rec_off, const int2* __restrict__ rkey,
                                  const int* __restrict__ n0_off, ushort4* __restrict__ grp_off,
                                  int* __restrict__ too_long)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (long long)P.K * P.M) return;
    const int k = (int)(i / P.M), n = (int)(i - (long long)k * P.M);
    const long long base = rec_off[k];
    const int a = n0_off[(size_t)k * (P.M + 1) + n], z = n0_off[(size_t)k * (P.M + 1) + n + 1];
    const int R = P.Q + 1;
    if (z - a > 65535) atomicExch(too_long, 1);
    int st[4] = {0, 0, 0, 0};
    int c = 0;
    for (int r = a; r < z; ++r) {
        const int cls = ((((rkey[base + r].y >> 1) & 0xfff) % R) & 3);
        while (c < cls) st[++c] = r - a;
    }
    while (c < 3) st[++c] = z - a;
    grp_off[i] = make_ushort4((unsigned short)st[1], (unsigned short)st[2], (unsigned short)st[3], 0);
}

// FP32 form: start of every (half, phase class) group inside every (A-scan, n0) bucket (buckets are
// ordered by half, then class; half 1 = phases >= phsplit), groups 1..7 as 16-bit offsets.
__global__ void tf3_grp_off_kernel(GeomParams P, int phsplit, const long long* __restrict__ rec_off,
                                   const int2* __restrict__ rkey, const int* __restrict__ n0_off,
                                   uint4* __restrict__ grp_off, int* __restrict__ too_long)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (long long)P.K * P.M) return;
    const int k = (int)(i / P.M), n = (int)(i - (long long)k * P.M);
    const long long base = rec_off[k];
    const int a = n0_off[(size_t)k * (P.M + 1) + n], z = n0_off[(size_t)k * (P.M + 1) + n + 1];
    const int R = P.Q + 1;
    if (z - a > 65535) atomicExch(too_long, 1);
    int st[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    int c = 0;
    for (int r = a; r < z; ++r) {
        const int ph = (((rkey[base + r].y >> 1) & 0xfff) % R);
        const int grp = (ph >= phsplit ? 4 : 0) + (ph & 3);
        while (c < grp) st[++c] = r - a;
    }
    while (c < 7) st[++c] = z - a;
    grp_off[i] = make_uint4((uint32_t)st[1] | (uint32_t)st[2] << 16, (uint32_t)st[3] | (uint32_t)st[4] << 16,
                            (uint32_t)st[5] | (uint32_t)st[6] << 16, (uint32_t)st[7]);
}

// Tables of the tensor-core A x for a geometry with records (BF16 form: one BF16 table operand; FP32
// form: both row halves' two-part FP16 operands); cudaErrorNotSupported keeps the CUDA-core A x.
cudaError_t build_tc_forward(mbir_geometry* g, cudaStream_t st)
{
    const GeomParams& P = g->P;
    const bool bf = P.precision == MBIR_PREC_BF16;
    // the record-ordered x of each apply lives in the adjoint's contribution buffer
    if (!g->d_rec_key || g->n_records <= 0 || !g->w_tc_contrib) return cudaErrorNotSupported;
    const TfLayout L = tf_layout(P);
    Tf3Layout L3 = tf3_layout(P);
    if ((bf ? !L.ok : !L3.ok) || (long long)P.K * (P.M + 1) >= (1LL << 31)) return cudaErrorNotSupported;
    const int nq = P.Q * P.Tw + 1, R = P.Q + 1;
    std::vector<__nv_bfloat16> bimg;
    if (bf) {
        // table operand: row m (tap), column c = plane * (Q + 1) + phase (plane-major, so that the planes a
        // tile's records reach are one column range); the second half starts at column k0
        bimg.assign((size_t)L.ntap * L.kb, __float2bfloat16_rn(0.0f));
        for (int c = 0; c < L.ncols; ++c) {
            const int gpl = c / R, ph = c % R;
            const int kcol = c < L.c0 ? c : L.k0 + (c - L.c0);
            for (int m = 0; m < P.Tw; ++m)
                bimg[kmajor_offset(m, kcol, L.kb) / 2] =
                    __float2bfloat16_rn((float)g->tab_host[(size_t)gpl * nq + m * P.Q + ph]);
        }
    } else {
        // per row half h (phases [0, phsplit] / [phsplit, Q]): the FP32 table as the CUDA-core kernels
        // read it, times 2^texp (largest magnitude into [2^14, 2^15)), split into two FP16 parts
        // t = t1 + t2; row m (tap), column plane * pstride + (phase - first): plane-major, so that the
        // planes a tile's records reach are one column range
        float tmax = 0.0f;
        for (size_t i = 0; i < (size_t)P.G * nq; ++i) tmax = std::max(tmax, std::fabs((float)g->tab_host[i]));
        int ex = 0;
        std::frexp(tmax, &ex);
        L3.texp = tmax > 0.0f ? std::min(15 - ex, 126) : 0;
        bimg.assign(L3.bhalf, __float2bfloat16_rn(0.0f));    // bhalf bytes = both halves' elements (16-bit)
        __half* himg = reinterpret_cast<__half*>(bimg.data());
        const size_t part = (size_t)L3.ntap * L3.kb;
        for (int h = 0; h < 2; ++h) {
            const int phb = h ? L3.phsplit : 0, phe = h ? R - 1 : L3.phsplit;
            const size_t base = (size_t)h * 2 * part;
            for (int ph = phb; ph <= phe; ++ph)
                for (int gpl = 0; gpl < P.G; ++gpl)
                    for (int m = 0; m < P.Tw; ++m) {
                        const float t = std::ldexp((float)g->tab_host[(size_t)gpl * nq + m * P.Q + ph], L3.texp);
                        const __half p1 = __float2half_rn(t);
                        const __half p2 = __float2half_rn(t - __half2float(p1));
                        const size_t o = kmajor_offset(m, gpl * L3.pstride + (ph - phb), L3.kb) / 2;
                        himg[base + o] = p1;
                        himg[base + part + o] = p2;
                    }
        }
    }
    // A-scans by decreasing record count
    std::vector<long long> roff((size_t)P.K + 1);
    cudaError_t e = cudaMemcpy(roff.data(), g->d_rec_off, sizeof(long long) * (P.K + 1), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return e;
    std::vector<int> order(P.K);
    for (int k = 0; k < P.K; ++k) order[k] = k;
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return roff[a + 1] - roff[a] > roff[b + 1] - roff[b]; });
    uint4* d_b = nullptr;
    int *d_n0 = nullptr, *d_ord = nullptr, *d_ctr = nullptr;
    void* d_grp = nullptr;
    const size_t grp_bytes = (bf ? sizeof(ushort4) : sizeof(uint4)) * (size_t)P.K * P.M;
    e = cudaMalloc((void**)&d_b, bimg.size() * 2);
    if (e == cudaSuccess) e = cudaMalloc((void**)&d_n0, sizeof(int) * (size_t)P.K * (P.M + 1));
    if (e == cudaSuccess) e = cudaMalloc((void**)&d_ord, sizeof(int) * (size_t)P.K);
    if (e == cudaSuccess) e = cudaMalloc((void**)&d_ctr, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&d_grp, grp_bytes);
    if (e == cudaSuccess) e = cudaMemcpy(d_b, bimg.data(), bimg.size() * 2, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_ord, order.data(), sizeof(int) * (size_t)P.K, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        const long long n = (long long)P.K * (P.M + 1);
        tf_n0_off_kernel<<<(int)((n + 255) / 256), 256, 0, st>>>(P, g->d_rec_off, g->d_rec_key, d_n0);
        e = cudaGetLastError();
    }
    int too_long = 0;
    if (e == cudaSuccess) e = cudaMemsetAsync(d_ctr, 0, sizeof(int), st);
    if (e == cudaSuccess) {
        const long long n = (long long)P.K * P.M;
        if (bf)
            tf_grp_off_kernel<<<(int)((n + 255) / 256), 256, 0, st>>>(P, g->d_rec_off, g->d_rec_key, d_n0,
                                                                      (ushort4*)d_grp, d_ctr);
        else
            tf3_grp_off_kernel<<<(int)((n + 255) / 256), 256, 0, st>>>(P, L3.phsplit, g->d_rec_off, g->d_rec_key,
                                                                       d_n0, (uint4*)d_grp, d_ctr);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&too_long, d_ctr, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess && too_long) e = cudaErrorNotSupported;   // buckets beyond 16-bit offsets
    if (e != cudaSuccess) {
        cudaFree(d_b);
        cudaFree(d_n0);
        cudaFree(d_ord);
        cudaFree(d_ctr);
        cudaFree(d_grp);
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? cudaErrorNotSupported : e;
    }
    if (bf) {
        g->tf = L;
        g->d_tf_bop = d_b;
        g->d_tf_grpoff = (ushort4*)d_grp;
    } else {
        g->tf3 = L3;
        g->d_tf3_bop = d_b;
        g->d_tf3_grpoff = (uint4*)d_grp;
    }
    g->d_tf_n0off = d_n0;
    g->d_tf_order = d_ord;
    g->d_tf_counter = d_ctr;
    g->bytes += bimg.size() * 2 + sizeof(int) * ((size_t)P.K * (P.M + 1) + P.K + 1) + grp_bytes;
    return cudaSuccess;
}

cudaError_t launch_forward_tc(const mbir_geometry* g, const float* x, float* yf, __nv_bfloat16* yb, int stride,
                              cudaStream_t st)
{
    const GeomParams& P = g->P;
    const TfLayout& L = g->tf;
    cudaError_t ce = cudaFuncSetAttribute(fwd_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(g->d_tf_counter, 0, sizeof(int), st);
    if (ce != cudaSuccess) return ce;
    const int grid = std::max(1, std::min(g->n_sm, P.K));
    // x per record, in record order (the adjoint's contribution buffer is free between applies)
    tc_gather_x_kernel<<<g->n_sm * 8, 256, 0, st>>>(g->n_records, g->d_rec_key, x, g->w_tc_contrib);
    ce = cudaGetLastError();
    if (ce != cudaSuccess) return ce;
    TcFwdView V{P, L, g->d_tf_bop, g->d_tab_bf16, g->d_rec_off, g->d_tf_n0off, g->d_tf_grpoff, g->d_rec_key,
                 g->d_rec_w, g->d_tf_order, g->w_tc_contrib, yf, yb, stride, g->d_tf_counter};
    fwd_tc_kernel<<<grid, kTfThreads, L.smem, st>>>(V, g->d_status);
    return cudaGetLastError();
}

cudaError_t launch_forward_tc32(const mbir_geometry* g, const float* x, float* yf, int stride, cudaStream_t st)
{
    const GeomParams& P = g->P;
    const Tf3Layout& L = g->tf3;
    cudaError_t ce = cudaFuncSetAttribute(fwd_tc32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(g->d_tf_counter, 0, sizeof(int), st);
    if (ce != cudaSuccess) return ce;
    const int grid = std::max(1, std::min(g->n_sm, P.K));
    tc_gather_x_kernel<<<g->n_sm * 8, 256, 0, st>>>(g->n_records, g->d_rec_key, x, g->w_tc_contrib);
    ce = cudaGetLastError();
    if (ce != cudaSuccess) return ce;
    TcFwd32View V{P, L, g->d_tf3_bop, g->d_tab, g->d_rec_off, g->d_tf_n0off, g->d_tf3_grpoff, g->d_rec_key,
                  g->d_rec_w, g->d_tf_order, g->w_tc_contrib, yf, stride, g->d_tf_counter};
    fwd_tc32_kernel<<<grid, kTfThreads, L.smem, st>>>(V, g->d_status);
    return cudaGetLastError();
}

}  // namespace mbir
