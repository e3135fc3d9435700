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
#include <vector>

#include "apply_common.cuh"
#include "tc_common.cuh"

namespace mbir {

constexpr int kTfTile = 128;          // values of n0 per MMA tile (M)
constexpr int kTfThreads = 512;       // scatter: 4 threads per n0 (phase classes mod 4)
constexpr int kTfUnroll = 8;          // records in flight per scatter thread
constexpr int kTfStage = 6;           // 8-column groups per thread held in registers while converting

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
    const size_t acc0 = std::max((size_t)kTfTile * L.astride * 4, (size_t)kTfTile * L.ka * 2);
    L.off_a = L.off_acc;
    L.off_acc1 = (L.off_acc + acc0 + 127) & ~(size_t)127;
    L.off_y = (L.off_acc1 + (size_t)kTfTile * L.astride1 * 4 + 127) & ~(size_t)127;
    L.ylen = ((P.M + kTfTile - 1) / kTfTile) * kTfTile + L.ntap + 2;   // every anti-diagonal target
    L.smem = L.off_y + (size_t)L.ylen * 4;
    const int per_thread = (kTfTile * (L.k0 / 8) + kTfThreads - 1) / kTfThreads;
    L.ok = L.ntap <= 256 && L.k0 > 0 && L.smem <= 227 * 1024 && L.ncols <= 4096 && per_thread <= kTfStage;
    return L;
}

__global__ void __launch_bounds__(kTfThreads, 1)
    fwd_tc_kernel(GeomParams P, TfLayout T, const uint4* __restrict__ bop, const __nv_bfloat162* __restrict__ tab,
                  const long long* __restrict__ rec_off, const int* __restrict__ n0_off,
                  const int2* __restrict__ rkey, const float4* __restrict__ rw, const int* __restrict__ order,
                  const float* __restrict__ x, float* __restrict__ y_f32, __nv_bfloat16* __restrict__ y_bf16,
                  int out_stride, int* __restrict__ counter, int* __restrict__ status)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + 8);
    volatile int* next = reinterpret_cast<volatile int*>(smem + 16);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(smem + 20);
    unsigned char* sB = smem + T.off_b;
    unsigned char* sA = smem + T.off_a;
    float* sAcc = reinterpret_cast<float*>(smem + T.off_acc);
    float* sAcc1 = reinterpret_cast<float*>(smem + T.off_acc1);
    float* sY = reinterpret_cast<float*>(smem + T.off_y);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int R = P.Q + 1, S = table_stride(P.Tw4);

    // table operand: rows = taps, columns = table rows (phase * G + plane), K-major
    const int nb16 = (int)((size_t)T.ntap * T.kb * 2 / 16);
    for (int i = tid; i < nb16; i += blockDim.x) reinterpret_cast<uint4*>(sB)[i] = __ldg(bop + i);
    if (tid == 0) {
        mbar_init(smem_u32(bar), 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 0) tmem_alloc(smem_u32(tslot), 128);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    const int ntile = (P.M + kTfTile - 1) / kTfTile;
    const uint32_t lbo = 128, sboA = (uint32_t)(T.ka / 8) * 128, sboB = (uint32_t)(T.kb / 8) * 128;
    const uint32_t idesc = umma_idesc_bf16(kTfTile, T.ntap);
    const int si = tid >> 2, pj = tid & 3;            // scatter role: n0 row and phase class
    uint32_t phase = 0;
    for (;;) {
        if (tid == 0) *next = atomicAdd(counter, 1);
        __syncthreads();
        const int idx = *next;
        if (idx >= P.K) break;
        const int k = __ldg(order + idx);
        const long long base = __ldg(rec_off + k);
        const int* no = n0_off + (size_t)k * (P.M + 1);
        for (int i = tid; i < T.ylen; i += blockDim.x) sY[i] = 0.0f;
        for (int t = 0; t < ntile; ++t) {
            const int ts = t * kTfTile;
            const int n0 = ts + si;
            const int ra = n0 < P.M ? __ldg(no + n0) : 0, rz = n0 < P.M ? __ldg(no + n0 + 1) : 0;
            for (int i = tid; i < kTfTile * T.astride; i += blockDim.x) sAcc[i] = 0.0f;
            for (int i = tid; i < kTfTile * T.astride1; i += blockDim.x) sAcc1[i] = 0.0f;
            __syncthreads();
            // scatter: thread (n0 row si, phase class pj) adds the corners that fall in its cells
            float* arow0 = sAcc + si * T.astride;
            float* arow1 = sAcc1 + si * T.astride1 - T.c0;
            for (int rb = ra; rb < rz; rb += kTfUnroll) {
                int2 key[kTfUnroll];
                float4 w4[kTfUnroll];
                float xv[kTfUnroll];
#pragma unroll
                for (int u = 0; u < kTfUnroll; ++u)
                    if (rb + u < rz) {
                        key[u] = __ldg(rkey + base + rb + u);
                        w4[u] = __ldg(rw + base + rb + u);
                    }
#pragma unroll
                for (int u = 0; u < kTfUnroll; ++u)
                    if (rb + u < rz) xv[u] = __ldg(x + key[u].x);
#pragma unroll
                for (int u = 0; u < kTfUnroll; ++u) {
                    if (rb + u >= rz) break;
                    const int trow = (key[u].y >> 1) & 0xfff;
                    const int gi = trow / R, ph = trow - gi * R;
                    const int g1 = min(gi + 1, P.G - 1);
                    if ((ph & 3) == pj) {
                        const int c = ph * P.G;
                        (c + gi < T.c0 ? arow0 : arow1)[c + gi] += w4[u].x * xv[u];
                        (c + g1 < T.c0 ? arow0 : arow1)[c + g1] += w4[u].y * xv[u];
                    }
                    if (((ph + 1) & 3) == pj) {
                        const int c = (ph + 1) * P.G;
                        (c + gi < T.c0 ? arow0 : arow1)[c + gi] += w4[u].z * xv[u];
                        (c + g1 < T.c0 ? arow0 : arow1)[c + g1] += w4[u].w * xv[u];
                    }
                    if (pj == 0 && (key[u].y & 1)) {
                        // tau = t0 exactly: the last tap of the upper phase row lies outside
                        const float2 tl = __bfloat1622float2(__ldg(tab + ((size_t)gi * R + ph + 1) * S + P.Tw - 1));
                        sY[n0 + P.Tw] -= xv[u] * (w4[u].z * tl.x + w4[u].w * tl.y);
                    }
                }
            }
            __syncthreads();
            for (int h = 0; h < 2; ++h) {
                const int cw = h ? P.G * R - T.c0 : T.c0, kh = h ? T.k1 : T.k0;
                if (cw <= 0) break;
                const float* src = h ? sAcc1 : sAcc;
                const int astr = h ? T.astride1 : T.astride;
                const int kc = kh / 8;
                // FP32 sums -> registers -> BF16 operand (K-major, 8 columns per 16-byte store);
                // the first half's operand is written over its own sums
                uint4 pk[kTfStage];
#pragma unroll
                for (int q = 0; q < kTfStage; ++q) {
                    const int c = tid + q * kTfThreads;
                    if (c < kTfTile * kc) {
                        const int i = c / kc, j = c - i * kc;
                        const float* sp = src + i * astr + 8 * j;
                        uint32_t w[4];
#pragma unroll
                        for (int e2 = 0; e2 < 4; ++e2) {
                            const int cc = 8 * j + 2 * e2;
                            const float a = cc < cw ? sp[2 * e2] : 0.0f, b = cc + 1 < cw ? sp[2 * e2 + 1] : 0.0f;
                            const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
                            w[e2] = *reinterpret_cast<const uint32_t*>(&v);
                        }
                        pk[q] = make_uint4(w[0], w[1], w[2], w[3]);
                    }
                }
                if (h == 1) {
                    // the first half's MMA reads the operand buffer: wait before rewriting it
                    if (!mbar_wait_bounded(smem_u32(bar), phase, status)) *abort_flag = 1;
                    phase ^= 1u;
                }
                __syncthreads();
                if (*abort_flag) break;
#pragma unroll
                for (int q = 0; q < kTfStage; ++q) {
                    const int c = tid + q * kTfThreads;
                    if (c < kTfTile * kc) {
                        const int i = c / kc, j = c - i * kc;
                        *reinterpret_cast<uint4*>(sA + kmajor_offset(i, 8 * j, T.ka)) = pk[q];
                    }
                }
                fence_async_smem();
                __syncthreads();
                if (tid == 0) {
                    tc_fence_after();
                    const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB) + (uint32_t)((h ? T.c0 : 0) / 8) * 128;
                    for (int s = 0; s < kh / 16; ++s)
                        umma_bf16(tmem, umma_desc(a0 + 256 * s, lbo, sboA), umma_desc(b0 + 256 * s, lbo, sboB), idesc,
                                  h > 0 || s > 0);
                    umma_commit(smem_u32(bar));
                }
            }
            if (*abort_flag) break;
            if (!mbar_wait_bounded(smem_u32(bar), phase, status)) *abort_flag = 1;
            phase ^= 1u;
            __syncthreads();
            tc_fence_after();
            if (*abort_flag) break;
            // U (tensor memory) -> shared, rows = n0 - ts, columns = taps
            {
                const int q = warp & 3, part = warp >> 2;        // 16 warps: lane quarter x column quarter
                const int row = q * 32 + lane;
                const int cwid = T.ntap / 4;
                for (int c = part * cwid; c < part * cwid + cwid; c += 4) {
                    float v[4];
                    tmem_ld4(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c, v);
#pragma unroll
                    for (int j = 0; j < 4; ++j) sAcc1[row * T.ustride + c + j] = v[j];
                }
            }
            tc_fence_before();
            __syncthreads();
            // anti-diagonals: y[ts + 1 + j] += sum_i U[i][j - i]
            for (int j = tid; j < kTfTile + T.ntap - 1; j += blockDim.x) {
                float acc = 0.0f;
                const int i0 = max(0, j - T.ntap + 1), i1 = min(kTfTile - 1, j);
                for (int i = i0; i <= i1; ++i) acc += sAcc1[i * T.ustride + j - i];
                sY[ts + 1 + j] += acc;
            }
            __syncthreads();
        }
        if (*abort_flag) break;
        float* yo = y_f32 ? y_f32 + (size_t)k * out_stride : nullptr;
        __nv_bfloat16* yb = y_f32 ? nullptr : y_bf16 + (size_t)k * out_stride;
        for (int n = tid; n < out_stride; n += blockDim.x) {
            const float v = n < P.M ? sY[n] : 0.0f;
            if (yo) yo[n] = v;
            else yb[n] = __float2bfloat16_rn(v);
        }
        __syncthreads();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, 128);
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

// Tables of the tensor-core A x for a BF16 geometry with records;
// cudaErrorNotSupported keeps the CUDA-core A x.
cudaError_t build_tc_forward(mbir_geometry* g, cudaStream_t st)
{
    const GeomParams& P = g->P;
    if (P.precision != MBIR_PREC_BF16 || !g->d_rec_key || g->n_records <= 0) return cudaErrorNotSupported;
    const TfLayout L = tf_layout(P);
    if (!L.ok || (long long)P.K * (P.M + 1) >= (1LL << 31)) return cudaErrorNotSupported;
    const int nq = P.Q * P.Tw + 1;
    // table operand: row m (tap), column c = phase * G + plane; the second half starts at column k0
    std::vector<__nv_bfloat16> bimg((size_t)L.ntap * L.kb, __float2bfloat16_rn(0.0f));
    for (int c = 0; c < L.ncols; ++c) {
        const int gpl = c % P.G, ph = c / P.G;
        const int kcol = c < L.c0 ? c : L.k0 + (c - L.c0);
        for (int m = 0; m < P.Tw; ++m)
            bimg[kmajor_offset(m, kcol, L.kb) / 2] = __float2bfloat16_rn((float)g->tab_host[(size_t)gpl * nq + m * P.Q + ph]);
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
    e = cudaMalloc((void**)&d_b, bimg.size() * 2);
    if (e == cudaSuccess) e = cudaMalloc((void**)&d_n0, sizeof(int) * (size_t)P.K * (P.M + 1));
    if (e == cudaSuccess) e = cudaMalloc((void**)&d_ord, sizeof(int) * (size_t)P.K);
    if (e == cudaSuccess) e = cudaMalloc((void**)&d_ctr, sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpy(d_b, bimg.data(), bimg.size() * 2, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_ord, order.data(), sizeof(int) * (size_t)P.K, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        const long long n = (long long)P.K * (P.M + 1);
        tf_n0_off_kernel<<<(int)((n + 255) / 256), 256, 0, st>>>(P, g->d_rec_off, g->d_rec_key, d_n0);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        cudaFree(d_b);
        cudaFree(d_n0);
        cudaFree(d_ord);
        cudaFree(d_ctr);
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? cudaErrorNotSupported : e;
    }
    g->tf = L;
    g->d_tf_bop = d_b;
    g->d_tf_n0off = d_n0;
    g->d_tf_order = d_ord;
    g->d_tf_counter = d_ctr;
    g->bytes += bimg.size() * 2 + sizeof(int) * ((size_t)P.K * (P.M + 1) + P.K + 1);
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
    fwd_tc_kernel<<<grid, kTfThreads, L.smem, st>>>(P, L, g->d_tf_bop, g->d_tab_bf16, g->d_rec_off, g->d_tf_n0off,
                                                    g->d_rec_key, g->d_rec_w, g->d_tf_order, x, yf, yb, stride,
                                                    g->d_tf_counter, g->d_status);
    return cudaGetLastError();
}

}  // namespace mbir
