// A x on the tensor cores (FP32 and BF16 storage forms): set-up tables and the
// single-request kernel.  The work itself is tcs_forward_pool (tc_stream.cuh).
#include <algorithm>
#include <cmath>
#include <vector>

#include "tc_stream.cuh"

namespace mbir {

Tf4Layout tf4_layout(const GeomParams& P, int kwmax)
{
    Tf4Layout L{};
    const bool bf = P.precision == MBIR_PREC_BF16;
    L.parts = bf ? 1 : 2;
    L.R = P.Q + 1;
    L.kb = (P.G * L.R + 15) & ~15;
    L.ntap = (P.Tw + 15) & ~15;
    L.kwmax = std::min(kwmax, L.kb);
    L.astride = ((L.kwmax + 31) & ~31) + 4;            // 4 mod 32: a warp's row reads hit distinct banks
    L.bbytes = (size_t)L.parts * L.ntap * L.kb * 2;
    const int ntile = (P.M + kTsTile - 1) / kTsTile;
    L.off_part = 1024;                                 // the epilogue warps' anti-diagonal sums, 64 floats each
    const int nw = ts_warps(bf);
    L.off_rs = L.off_part + (size_t)nw * kTsPart * 4;   // per A-scan: part boundaries, column ranges
    L.off_b = (L.off_rs + (size_t)ntile * (nw + 2) * 4 + 1023) & ~(size_t)1023;
    L.off_s = (L.off_b + L.bbytes + 1023) & ~(size_t)1023;
    L.ylen = kTsYRing;
    L.off_y = L.off_s + (size_t)kTsTile * L.astride * 4;
    L.smem = L.off_y + (size_t)L.ylen * 4;
    L.ok = L.R >= 2 && L.ntap <= 128 && L.ntap / 4 <= 32 && L.kwmax >= 16 && L.kwmax % 16 == 0 &&
           L.parts * L.kwmax / 2 <= (int)kTsDCol && L.smem <= 227 * 1024 && L.bbytes < (1u << 20) &&
           P.G * L.R <= kTcMaxRows && P.M <= kTcMaxSamples && (long long)P.W * P.H <= kTcMaxPixels &&
           (long long)P.K * (P.M + 1) < (1LL << 31);
    return L;
}

// The call-independent part of the view is read from device memory (written at set-up) and the per-call
// fields come as parameters routed through registers: with every field register-resident the pool ran the
// 512x1024 A x in 13.7 ms against 16.5 ms with the whole view read from the parameter space.
template <bool BF16, int FV>
__global__ void __launch_bounds__(TsShape<BF16>::threads, 1)
    fwd_tcs_kernel(const TsView* __restrict__ base, const float* x, void* y, int y_bf16, int out_stride,
                   int* __restrict__ status)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    tc_header_init(smem, kTsCols);
    const uint32_t tmem = *reinterpret_cast<volatile uint32_t*>(smem + 8);
    uint32_t mphase = 0, bphase = 0;
    TsView V = *base;
    asm volatile("" : "+l"(x), "+l"(y), "+r"(y_bf16), "+r"(out_stride));
    V.x = x;
    V.y = y;
    V.y_bf16 = y_bf16;
    V.out_stride = out_stride;
    tcs_forward_pool<BF16, FV>(V, smem, tmem, mphase, bphase, status);
    tc_header_release(smem, tmem, kTsCols);
}

// first record of every sample n0 of every A-scan (records sorted by n0)
__global__ void ts_n0_off_kernel(GeomParams P, const long long* __restrict__ rec_off, const int2* __restrict__ rkey,
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

// Per (A-scan, tile of 128 n0): the column range of the planes its records reach (warp per tile; the widest
// range goes to *wmax) and the boundaries of the warps' parts: the tile's records cut at n0 boundaries into
// nw parts of about equal count (part w starts at the first n0 whose first record lies at or after the
// w/nw point of the tile's range).
__global__ void ts_tiles_kernel(GeomParams P, int R, int kb, int nw, const long long* __restrict__ rec_off,
                                const int2* __restrict__ rkey, const int* __restrict__ n0_off,
                                uint32_t* __restrict__ crange, int* __restrict__ split, int* __restrict__ wmax)
{
    const int ntile = (P.M + kTsTile - 1) / kTsTile;
    const long long wid = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (wid >= (long long)P.K * ntile) return;
    const int k = (int)(wid / ntile), t = (int)(wid - (long long)k * ntile);
    const long long base = rec_off[k];
    const int* no = n0_off + (size_t)k * (P.M + 1);
    const int n_lo = t * kTsTile, n_hi = min((t + 1) * kTsTile, P.M);
    const int r0 = no[n_lo], r1 = no[n_hi];
    int glo = P.G, ghi = -1;
    for (int r = r0 + lane; r < r1; r += 32) {
        const int trow = (rkey[base + r].y >> 1) & 0xfff;
        const int gi = trow / R;
        glo = min(glo, gi);
        ghi = max(ghi, min(gi + 1, P.G - 1));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        glo = min(glo, __shfl_xor_sync(0xffffffffu, glo, o));
        ghi = max(ghi, __shfl_xor_sync(0xffffffffu, ghi, o));
    }
    if (lane == 0) {
        uint32_t v = 0;
        if (ghi >= glo) {
            const int c_lo = (glo * R) & ~15;
            const int c_hi = min(kb, ((ghi + 1) * R + 15) & ~15);
            v = (uint32_t)c_lo | (uint32_t)c_hi << 16;
            atomicMax(wmax, c_hi - c_lo);
        }
        crange[wid] = v;
    }
    if (lane <= nw) {
        int s = r1;
        if (lane == 0) s = r0;
        else if (lane < nw) {
            const long long target = r0 + ((long long)(r1 - r0) * lane) / nw;
            int lo = n_lo, hi = n_hi;                    // first n0 in [n_lo, n_hi] with no[n0] >= target
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (no[mid] < target) lo = mid + 1;
                else hi = mid;
            }
            s = no[lo];
        }
        split[wid * (nw + 1) + lane] = s;
    }
}

// The records of every warp part interleaved and packed (tc_apply.cuh): batch b of a part (stored positions
// 32 b .. 32 b + 31) takes the part's sorted records b, b + q, b + 2 q, ... (q = its length / 32; the first
// length % 32 lanes hold one more), so records of one (n0, table row), adjacent in sorted order, seldom share
// a batch, and where they do they sit in adjacent lanes as the segmented sums require.  Each record's pair
// quantities are evaluated again from the legs, as when the records were sorted (tab_pair), so the packed
// fractions come from the delay and attenuation coordinates themselves.  Block per (A-scan, tile).
template <bool BF16>
__global__ void ts_pack_kernel(GeomParams P, DevPtrs D, const long long* __restrict__ rec_off,
                               const int* __restrict__ split, const int2* __restrict__ skey,
                               uint2* __restrict__ key, typename TcW<BF16>::type* __restrict__ w)
{
    const int ntile = (P.M + kTsTile - 1) / kTsTile;
    const int k = (int)(blockIdx.x / ntile), t = (int)(blockIdx.x % ntile);
    constexpr int nw = TsShape<BF16>::warps;
    const int* sp = split + ((size_t)k * ntile + t) * (nw + 1);
    const long long base = rec_off[k];
    const int R = P.Q + 1;
    for (int p = 0; p < nw; ++p) {
        const int a = sp[p], len = sp[p + 1] - a;
        const int q = len >> 5, r = len & 31;
        for (int s = threadIdx.x; s < len; s += blockDim.x) {
            const int l = s & 31, o = l * q + min(l, r) + (s >> 5);
            const int v = skey[base + a + o].x & kRecPixel;
            Pair pr;
            typename TcW<BF16>::type pw;
            if (tab_pair(P, D, k, v, pr)) {
                key[base + a + s] = tc_pack_key(v, pr.gi * R + pr.r, pr);
                tc_pack_w(pr, pw);
            } else {
                // (not reached: the record was made from the same active pair) a zero-weight record
                key[base + a + s] = make_uint2((uint32_t)v, (uint32_t)(t * kTsTile) << kTcN0Shift);
                pw = typename TcW<BF16>::type{};
            }
            w[base + a + s] = pw;
        }
    }
}

// Marks every batch of 32 records (per warp part, as the kernel reads them) whose lanes' four corner cells
// (n0, row), (n0, row + dR), (n0, row + 1), (n0, row + dR + 1) are all distinct between lanes: bit 31 of
// key.x of the batch's first record.  Such a batch has no equal keys, so the kernel adds its corners without
// the segmented sums and in one step.  Warp per batch, blocks per (A-scan, tile).
__global__ void ts_batch_flag_kernel(GeomParams P, int R, int nparts, const long long* __restrict__ rec_off,
                                     const int* __restrict__ split, uint2* __restrict__ key)
{
    const int ntile = (P.M + kTsTile - 1) / kTsTile;
    const int k = (int)(blockIdx.x / ntile), t = (int)(blockIdx.x % ntile);
    const int* sp = split + ((size_t)k * ntile + t) * (nparts + 1);
    const long long base = rec_off[k];
    const int dR = P.G > 1 ? R : 0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const uint32_t full = 0xffffffffu;
    for (int p = 0; p < nparts; ++p) {
        const int a = sp[p], z = sp[p + 1];
        for (int b = a + 32 * warp; b < z; b += 32 * nw) {
            const int r = b + lane;
            int c[4];
            if (r < z) {
                const uint2 kk = key[base + r];
                const int n0 = tc_rec_n0(kk), trow = tc_rec_row(kk);
                c[0] = (n0 << 13) | trow;
                c[1] = (n0 << 13) | (trow + dR);
                c[2] = c[0] + 1;
                c[3] = c[1] + 1;
            } else {
                c[0] = c[1] = c[2] = c[3] = -1 - lane;       // matches nothing
            }
            bool clash = false;
            for (int d = 1; d < 32; ++d) {
                const int src = (lane + d) & 31;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int o = __shfl_sync(full, c[j], src);
                    clash |= (o == c[0]) | (o == c[1]) | (o == c[2]) | (o == c[3]);
                }
            }
            if (!__any_sync(full, clash) && lane == 0) key[base + b].x |= kTcMark;
        }
    }
}

// Tables of the tensor-core A x for a geometry with records: the A-scan order, the per-tile column ranges and
// warp parts (from the first record of every n0), the table operand (FP32 form: two FP16 parts of the table scaled by
// 2^texp; BF16 form: the BF16 table); cudaErrorNotSupported keeps the CUDA-core A x.
cudaError_t build_tc_forward_stream(mbir_geometry* g, cudaStream_t st)
{
    const GeomParams& P = g->P;
    if (!g->d_rec_key || g->n_records <= 0) return cudaErrorNotSupported;
    Tf4Layout L{};
    for (int kw : {512, 448, 384, 320, 256, 224, 192, 160, 128, 96, 64}) {
        L = tf4_layout(P, kw);
        if (L.ok) break;
    }
    if (!L.ok) return cudaErrorNotSupported;
    const int ntile = (P.M + kTsTile - 1) / kTsTile;
    // A-scans by decreasing record count
    std::vector<long long> roff((size_t)P.K + 1);
    cudaError_t e = cudaMemcpy(roff.data(), g->d_rec_off, sizeof(long long) * (P.K + 1), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return e;
    std::vector<int> order(P.K);
    for (int k = 0; k < P.K; ++k) order[k] = k;
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return roff[a + 1] - roff[a] > roff[b + 1] - roff[b]; });
    int *d_n0 = nullptr, *d_ord = nullptr, *d_ctr = nullptr, *d_sp = nullptr, *d_w = nullptr;
    uint32_t* d_cr = nullptr;
    uint4* d_b = nullptr;
    e = cudaMalloc((void**)&d_n0, sizeof(int) * (size_t)P.K * (P.M + 1));
    if (e == cudaSuccess) e = cudaMalloc((void**)&d_ord, sizeof(int) * (size_t)P.K);
    if (e == cudaSuccess) e = cudaMalloc((void**)&d_ctr, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc((void**)&d_cr, sizeof(uint32_t) * (size_t)P.K * ntile);
    const int nw = ts_warps(P.precision == MBIR_PREC_BF16);
    if (e == cudaSuccess) e = cudaMalloc((void**)&d_sp, sizeof(int) * (size_t)P.K * ntile * (nw + 1));
    if (e == cudaSuccess) e = cudaMalloc((void**)&d_w, sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpy(d_ord, order.data(), sizeof(int) * (size_t)P.K, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_w, 0, sizeof(int), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_ctr, 0, sizeof(int), st);
    if (e == cudaSuccess) {
        const long long n = (long long)P.K * (P.M + 1);
        ts_n0_off_kernel<<<(int)((n + 255) / 256), 256, 0, st>>>(P, g->d_rec_off, g->d_rec_key, d_n0);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        const long long threads = (long long)P.K * ntile * 32;
        ts_tiles_kernel<<<(int)((threads + 255) / 256), 256, 0, st>>>(P, L.R, L.kb, nw, g->d_rec_off, g->d_rec_key, d_n0,
                                                                      d_cr, d_sp, d_w);
        e = cudaGetLastError();
    }
    int wmax = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&wmax, d_w, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(d_w);
    if (e == cudaSuccess && wmax > L.kwmax) e = cudaErrorNotSupported;   // a tile reaches too many planes
    if (e == cudaSuccess) {
        // the sum tile as wide as the widest tile's column range (a multiple of 16), no wider: the shared
        // memory left over goes to the L1, which keeps the gathered x
        const Tf4Layout Lt = tf4_layout(P, std::max(wmax, 16));
        if (Lt.ok) L = Lt;
    }
    // table operand: row m (tap), column plane * R + phase (K-major)
    if (e == cudaSuccess) {
        const int nq = P.Q * P.Tw + 1;
        const size_t part = (size_t)L.ntap * L.kb;
        std::vector<uint16_t> img((size_t)L.parts * part, 0);
        if (P.precision == MBIR_PREC_BF16) {
            L.texp = 0;
            for (int gpl = 0; gpl < P.G; ++gpl)
                for (int ph = 0; ph < L.R; ++ph)
                    for (int m = 0; m < P.Tw; ++m) {
                        const __nv_bfloat16 v = __float2bfloat16_rn((float)g->tab_host[(size_t)gpl * nq + m * P.Q + ph]);
                        img[kmajor_offset(m, gpl * L.R + ph, L.kb) / 2] = *reinterpret_cast<const uint16_t*>(&v);
                    }
        } else {
            // the FP32 kernel table times 2^texp (largest magnitude into [2^14, 2^15)), split t = t1 + t2
            float tmax = 0.0f;
            for (size_t i = 0; i < (size_t)P.G * nq; ++i) tmax = std::max(tmax, std::fabs((float)g->tab_host[i]));
            int ex = 0;
            std::frexp(tmax, &ex);
            L.texp = tmax > 0.0f ? std::min(15 - ex, 126) : 0;
            for (int gpl = 0; gpl < P.G; ++gpl)
                for (int ph = 0; ph < L.R; ++ph)
                    for (int m = 0; m < P.Tw; ++m) {
                        const float t = std::ldexp((float)g->tab_host[(size_t)gpl * nq + m * P.Q + ph], L.texp);
                        const __half p1 = __float2half_rn(t);
                        const __half p2 = __float2half_rn(t - __half2float(p1));
                        const size_t o = kmajor_offset(m, gpl * L.R + ph, L.kb) / 2;
                        img[o] = *reinterpret_cast<const uint16_t*>(&p1);
                        img[part + o] = *reinterpret_cast<const uint16_t*>(&p2);
                    }
        }
        e = cudaMalloc((void**)&d_b, L.bbytes);
        if (e == cudaSuccess) e = cudaMemcpy(d_b, img.data(), L.bbytes, cudaMemcpyHostToDevice);
    }
    // the packed records (16 B per pair in the FP32 form, 12 B in the BF16 form), interleaved within every warp
    // part and carrying the batch marks; the sorted records stay intact until these exist, so a failure here
    // leaves the CUDA-core A x usable
    const bool bf = P.precision == MBIR_PREC_BF16;
    const size_t wsz = bf ? sizeof(uint32_t) : sizeof(uint2);
    const size_t nrec = (size_t)std::max<long long>(g->n_records, 1);
    uint2* d_key = nullptr;
    void* d_pw = nullptr;
    if (e == cudaSuccess) e = cudaMalloc((void**)&d_key, sizeof(uint2) * nrec);
    if (e == cudaSuccess) e = cudaMalloc(&d_pw, wsz * nrec);
    if (e == cudaSuccess) {
        const DevPtrs D = dev_ptrs(g);
        if (bf)
            ts_pack_kernel<true><<<P.K * ntile, 256, 0, st>>>(P, D, g->d_rec_off, d_sp, g->d_rec_key, d_key,
                                                              reinterpret_cast<uint32_t*>(d_pw));
        else
            ts_pack_kernel<false><<<P.K * ntile, 256, 0, st>>>(P, D, g->d_rec_off, d_sp, g->d_rec_key, d_key,
                                                               reinterpret_cast<uint2*>(d_pw));
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        ts_batch_flag_kernel<<<P.K * ntile, 256, 0, st>>>(P, L.R, nw, g->d_rec_off, d_sp, d_key);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    // the kernel's view without the per-call fields
    TsView* d_view = nullptr;
    if (e == cudaSuccess) {
        const void* tab = bf ? (const void*)g->d_tab_bf16 : (const void*)g->d_tab;
        const TsView V{P, L, d_b, tab, g->d_rec_off, d_cr, d_sp, d_key, d_pw, d_ord, nullptr, nullptr, 0, 0, d_ctr};
        e = cudaMalloc((void**)&d_view, sizeof(TsView));
        if (e == cudaSuccess) e = cudaMemcpy(d_view, &V, sizeof(TsView), cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
        void* ptrs[] = {d_n0, d_ord, d_ctr, d_cr, d_sp, d_b, d_view, d_key, d_pw};
        for (void* p : ptrs) cudaFree(p);
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? cudaErrorNotSupported : e;
    }
    // the sorted records are not read again (the CUDA-core A x no longer runs for this geometry)
    cudaFree(g->d_rec_key);
    cudaFree(g->d_rec_w);
    g->d_rec_key = nullptr;
    g->d_rec_w = nullptr;
    g->bytes -= (sizeof(int2) + sizeof(float4)) * nrec;
    g->bytes += (sizeof(uint2) + wsz) * nrec;
    g->d_tc_key = d_key;
    g->d_tc_w = d_pw;
    cudaFree(d_n0);
    g->d_tf_view = d_view;
    g->tf4 = L;
    g->d_tf_order = d_ord;
    g->d_tf_counter = d_ctr;
    g->d_tf4_bop = d_b;
    g->d_tf4_crange = d_cr;
    g->d_tf4_split = d_sp;
    g->tf4_wmax = wmax;
    g->bytes += L.bbytes + sizeof(int) * ((size_t)P.K + 1) + sizeof(int) * (size_t)P.K * ntile * (nw + 2);
    return cudaSuccess;
}

cudaError_t launch_forward_tcs(const mbir_geometry* g, const float* x, float* yf, __nv_bfloat16* yb, int stride,
                               cudaStream_t st)
{
    const GeomParams& P = g->P;
    const Tf4Layout& L = g->tf4;
    const bool bf = P.precision == MBIR_PREC_BF16;
    auto kern = bf ? (g->tc_fvar ? fwd_tcs_kernel<true, 1> : fwd_tcs_kernel<true, 0>)
                   : (g->tc_fvar ? fwd_tcs_kernel<false, 1> : fwd_tcs_kernel<false, 0>);
    cudaError_t ce = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(g->d_tf_counter, 0, sizeof(int), st);
    if (ce != cudaSuccess) return ce;
    const int grid = std::max(1, std::min(g->n_sm, P.K));
    kern<<<grid, 32 * ts_warps(bf), L.smem, st>>>(g->d_tf_view, x, yf ? (void*)yf : (void*)yb, yf ? 0 : 1, stride,
                                           g->d_status);
    return cudaGetLastError();
}

}  // namespace mbir

namespace mbir {

// Times each variant of the tensor-core A x and A^T once on this geometry (x = 1, a constant residual; the
// first run of each warms up) and keeps the fastest of each: the autotuner of the tensor-core pools.
// Leaves g->tc_tune_ms with {A x variant 0, 1, A^T variant 0, 1} in ms.  Synchronous.
cudaError_t tune_tc_applies(mbir_geometry* g, cudaStream_t st)
{
    const GeomParams& P = g->P;
    const bool bf = P.precision == MBIR_PREC_BF16;
    const size_t N = (size_t)P.W * P.H, KMp = (size_t)P.K * P.Mp;
    float *x = nullptr, *y = nullptr, *b = nullptr, *e = nullptr;
    __nv_bfloat16* ebf = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t ce = cudaMalloc((void**)&x, sizeof(float) * N);
    if (ce == cudaSuccess) ce = cudaMalloc((void**)&b, sizeof(float) * N);
    if (ce == cudaSuccess) ce = cudaMalloc((void**)&y, (bf ? 2 : 4) * (size_t)P.K * P.M);
    if (ce == cudaSuccess && g->d_tb4_bop) {
        if (bf) ce = cudaMalloc((void**)&ebf, sizeof(__nv_bfloat16) * KMp);
        else ce = cudaMalloc((void**)&e, sizeof(float) * KMp);
    }
    if (ce == cudaSuccess) ce = cudaEventCreate(&e0);
    if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
    if (ce == cudaSuccess) {
        std::vector<float> ones(std::max(N, KMp), 1.0f);
        ce = cudaMemcpy(x, ones.data(), sizeof(float) * N, cudaMemcpyHostToDevice);
        if (ce == cudaSuccess && e) ce = cudaMemcpy(e, ones.data(), sizeof(float) * KMp, cudaMemcpyHostToDevice);
        if (ce == cudaSuccess && ebf) {
            std::vector<__nv_bfloat16> ob(KMp, __float2bfloat16_rn(1.0f));
            ce = cudaMemcpy(ebf, ob.data(), sizeof(__nv_bfloat16) * KMp, cudaMemcpyHostToDevice);
        }
    }
    auto timed = [&](auto&& launch, double& ms) -> cudaError_t {
        float t = 0.0f;
        cudaError_t r = cudaSuccess;
        for (int rep = 0; rep < 2 && r == cudaSuccess; ++rep) {
            r = cudaEventRecord(e0, st);
            if (r == cudaSuccess) r = launch();
            if (r == cudaSuccess) r = cudaEventRecord(e1, st);
            if (r == cudaSuccess) r = cudaEventSynchronize(e1);
            if (r == cudaSuccess) r = cudaEventElapsedTime(&t, e0, e1);
        }
        ms = t;
        return r;
    };
    const int keep_f = g->tc_fvar, keep_b = g->tc_bvar;
    for (int v = 0; v < kTcVariants && ce == cudaSuccess && g->d_tf4_bop; ++v) {
        g->tc_fvar = v;
        ce = timed([&] { return launch_forward_tcs(g, x, bf ? nullptr : y, bf ? (__nv_bfloat16*)y : nullptr, P.M, st); },
                   g->tc_tune_ms[v]);
    }
    for (int v = 0; v < kTcVariants && ce == cudaSuccess && g->d_tb4_bop; ++v) {
        g->tc_bvar = v;
        ce = timed([&] { return launch_backproject_tcs(g, e, ebf, b, st); }, g->tc_tune_ms[kTcVariants + v]);
    }
    g->tc_fvar = keep_f;
    g->tc_bvar = keep_b;
    if (ce == cudaSuccess && g->d_tf4_bop) g->tc_fvar = g->tc_tune_ms[1] < g->tc_tune_ms[0] ? 1 : 0;
    if (ce == cudaSuccess && g->d_tb4_bop) g->tc_bvar = g->tc_tune_ms[3] < g->tc_tune_ms[2] ? 1 : 0;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(x);
    cudaFree(y);
    cudaFree(b);
    cudaFree(e);
    cudaFree(ebf);
    return ce;
}

}  // namespace mbir
