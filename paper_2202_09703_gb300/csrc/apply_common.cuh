// Device building blocks of the apply kernels, shared by the single-request
// kernels and the batched engine's grouped kernels.
#pragma once

#include "device_common.cuh"

namespace mbir {

constexpr int kRecShift = 13;                     // record key: n0 << 13 | table row << 1 | flag0

// Copies a pulse table (tab_bytes, a multiple of 16) into shared memory.
__device__ __forceinline__ void load_table_smem(void* dst, const void* src, size_t tab_bytes, int tid, int nthreads)
{
    const int4* s = reinterpret_cast<const int4*>(src);
    int4* d = reinterpret_cast<int4*>(dst);
    const int n16 = (int)(tab_bytes / 16);
    for (int t = tid; t < n16; t += nthreads) d[t] = __ldg(s + t);
}

// One pair of A^T r: the taps of the pair against a residual row in shared
// memory (ev points at sample n0 + 1), weighted by the bilinear corners of
// the table.  Returns the pair's contribution w * sum_m H(m) e[n0 + 1 + m].
template <bool BF16>
__device__ __forceinline__ float pair_taps(const typename TabT<BF16>::type* __restrict__ A, int S, int Tw, int Tw4,
                                           const typename ET<BF16>::type* __restrict__ ev, const Pair& pr)
{
    float2 sa = make_float2(0.f, 0.f), sb = make_float2(0.f, 0.f);
    const typename TabT<BF16>::type* B = A + S;
    for (int m = 0; m < Tw4; m += 4) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const float e = ET<BF16>::ld(ev + m + u);
            const float2 ee = make_float2(e, e);
            sa = __ffma2_rn(TabT<BF16>::ld(A + m + u), ee, sa);
            sb = __ffma2_rn(TabT<BF16>::ld(B + m + u), ee, sb);
        }
    }
    const float p1 = pr.psi, p0 = 1.0f - pr.psi;
    float hv = pr.w0 * (p0 * sa.x + p1 * sa.y) + pr.w1 * (p0 * sb.x + p1 * sb.y);
    if (pr.flag0) {
        // tau = t0 exactly: outside the open window of eq. 10
        const float2 bl = TabT<BF16>::ld(B + Tw - 1);
        hv -= pr.w1 * (p0 * bl.x + p1 * bl.y) * ET<BF16>::ld(ev + Tw - 1);
    }
    return pr.w * hv;
}

__device__ __forceinline__ void neumaier_add(float& sum, float& comp, float v)
{
    const float t = sum + v;
    comp += (fabsf(sum) >= fabsf(v)) ? (sum - t) + v : (v - t) + sum;
    sum = t;
}

// One 32-sample span of A x from the sorted record list: records [r_lo, r_hi)
// of A-scan base `base`.  sr / sw are this warp's 32-entry staging slots.
// Returns the lane's output sample value (compensated across batches).
template <bool BF16>
__device__ __forceinline__ float span_gather(const typename TabT<BF16>::type* __restrict__ tab, int S, int Tw,
                                             const int2* __restrict__ rkey, const float4* __restrict__ rw,
                                             long long base, int r_lo, int r_hi, const float* __restrict__ x,
                                             int n, int lane, int4* sr, float4* sw)
{
    using Tab = typename TabT<BF16>::type;
    float sum = 0.0f, comp = 0.0f;
    int2 kv = make_int2(0, 0);
    float4 wv = make_float4(0.f, 0.f, 0.f, 0.f);
    float xv = 0.0f;
    if (r_lo + lane < r_hi) {
        kv = __ldg(rkey + base + r_lo + lane);
        wv = __ldg(rw + base + r_lo + lane);
        xv = __ldg(x + kv.x);
    }
    for (int r0 = r_lo; r0 < r_hi; r0 += 32) {
        const int cnt = min(32, r_hi - r0);
        if (lane < cnt) {
            const int key = kv.y;
            const int lo = (key >> kRecShift) + 1;
            const int len = Tw - (key & 1);                 // tau = t0 exactly lies outside
            sr[lane] = make_int4(lo, len, ((key >> 1) & 0xfff) * S - lo, 0);
            sw[lane] = make_float4(wv.x * xv, wv.y * xv, wv.z * xv, wv.w * xv);
        }
        __syncwarp();
        if (r0 + 32 + lane < r_hi) {
            kv = __ldg(rkey + base + r0 + 32 + lane);
            wv = __ldg(rw + base + r0 + 32 + lane);
            xv = __ldg(x + kv.x);
        }
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll 4
        for (int j = 0; j < cnt; ++j) {
            const int4 d = sr[j];
            if ((unsigned)(n - d.x) < (unsigned)d.y) {
                const float4 w4 = sw[j];
                const Tab* A = tab + (d.z + n);
                acc = __ffma2_rn(TabT<BF16>::ld(A), make_float2(w4.x, w4.y), acc);
                acc = __ffma2_rn(TabT<BF16>::ld(A + S), make_float2(w4.z, w4.w), acc);
            }
        }
        __syncwarp();
        neumaier_add(sum, comp, acc.x + acc.y);
    }
    return sum + comp;
}

}  // namespace mbir
