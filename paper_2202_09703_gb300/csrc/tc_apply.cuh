// Shared pieces of the tensor-core apply kernels (tc_stream.cuh): the
// shared-memory header set-up (mbarriers, tensor-memory allocation) and the
// two-part FP16 split of the FP32 form.
#pragma once

#include "apply_common.cuh"
#include <cuda_fp16.h>

#include "tc_common.cuh"

namespace mbir {

// Records of the tensor-core forms, packed once per geometry from the sorted records (ts_pack_kernel):
//   key.x = pixel (bits 0-19) | table row (bits 20-30) | batch mark of the A x (bit 31)
//   key.y = n0 (bits 19-31) | tau = t0 flag (bit 18) | fa x 2^18 (bits 0-17)
// with fa the bilinear weight of the table row's phase node (eq. 13 with the bilinear table), and the pair's
// weight w (tau(l_v) phi_tx phi_rx) with its attenuation-plane fraction psi:
//   FP32 form: uint2 {w as FP32, psi x 2^20}: 16 B per pair (the sorted records hold 24 B);
//   BF16 form: uint32 {w16 | psi x 2^15 << 16}: 12 B per pair, with w16 the weight (0 < w <= 1) as a 16-bit
//   float of a 6-bit exponent and a 10-bit mantissa: FP32's bits 13-28 after rounding, exponents 2^-63 .. 2^0
//   (FP16's 5-bit exponent would flush the weights of far, steep pairs, below 2^-24, to zero).
// The four bilinear corners are w fa (1 - psi), w fa psi, w (1 - fa)(1 - psi) and w (1 - fa) psi at the table
// columns row, row + dR, row + 1 and row + dR + 1, with dR = Q + 1 (the next attenuation plane; 0 for a
// single plane).  The fixed-point fractions are exact binary values; their rounding (2^-19 for fa, 2^-21 for
// psi in the FP32 form) is no coarser than the FP32 rounding of the delay and attenuation coordinates they
// come from; the BF16 form (psi to 2^-16, w to 2^-12 relative) keeps errors below its table's 8-bit rounding.
constexpr uint32_t kTcPixelMask = 0xfffffu;
constexpr int kTcRowShift = 20;
constexpr uint32_t kTcRowMask = 0x7ffu;
constexpr int kTcN0Shift = 19;
constexpr uint32_t kTcFlag0 = 1u << 18;
constexpr uint32_t kTcMark = 0x80000000u;
constexpr uint32_t kTcNone = 0xffffffffu;    // key.y of no record (n0 = 8191 is never a record's first tap)
constexpr long long kTcMaxPixels = 1LL << 20;
constexpr int kTcMaxRows = 2048;             // table rows G (Q + 1)
constexpr int kTcMaxSamples = 8191;          // M

template <bool BF16> struct TcW { using type = uint2; };
template <> struct TcW<true> { using type = uint32_t; };

// q 2^-s for an integer 0 <= q <= 2^(23 - s): 1 + q 2^-s formed in the mantissa, less one (both exact)
__device__ __forceinline__ float tc_fixed(uint32_t q, int s)
{
    return __uint_as_float(0x3f800000u + (q << (23 - s))) - 1.0f;
}
__device__ __forceinline__ float tc_rec_fa(uint2 k) { return tc_fixed(k.y & 0x3ffffu, 18); }
__device__ __forceinline__ int tc_rec_n0(uint2 k) { return (int)(k.y >> kTcN0Shift); }
__device__ __forceinline__ int tc_rec_row(uint2 k) { return (int)((k.x >> kTcRowShift) & kTcRowMask); }
__device__ __forceinline__ float tc_rec_w(uint2 w) { return __uint_as_float(w.x); }
__device__ __forceinline__ float tc_rec_psi(uint2 w) { return tc_fixed(w.y, 20); }
__device__ __forceinline__ float tc_rec_w(uint32_t w) { return __uint_as_float(((w & 0xffffu) << 13) + 0x20000000u); }
__device__ __forceinline__ float tc_rec_psi(uint32_t w) { return tc_fixed(w >> 16, 15); }

// The packed record of an active pair (ts_pack_kernel); the batch mark is added later.
__device__ __forceinline__ uint2 tc_pack_key(int v, int trow, const Pair& pr)
{
    const uint32_t qa = min((uint32_t)__float2uint_rn(pr.w0 * 262144.0f), 0x3ffffu);
    return make_uint2((uint32_t)v | ((uint32_t)trow << kTcRowShift),
                      ((uint32_t)pr.n0 << kTcN0Shift) | (pr.flag0 ? kTcFlag0 : 0u) | qa);
}
__device__ __forceinline__ void tc_pack_w(const Pair& pr, uint2& w)
{
    w = make_uint2(__float_as_uint(pr.w), __float2uint_rn(pr.psi * 1048576.0f));
}
__device__ __forceinline__ void tc_pack_w(const Pair& pr, uint32_t& w)
{
    // round to 10 mantissa bits (a carry moves into the exponent), then rebase the exponent at 2^-63
    const uint32_t u = __float_as_uint(pr.w) + 0x1000u;
    const uint32_t w16 = pr.w >= 0x1p-63f ? min((u >> 13) - (64u << 10), 0xffffu) : 0u;
    w = w16 | (__float2uint_rn(pr.psi * 32768.0f) << 16);
}

// Shared-memory header of the tensor-core kernels: offset 0 the MMA mbarrier, 8 the tensor-memory address,
// 16 the item slot, 20 the abort flag, 32 the table-copy mbarrier.
__device__ __forceinline__ void tc_header_init(unsigned char* smem, uint32_t ncols)
{
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
    if (threadIdx.x == 0) {
        mbar_init(smem_u32(bar), 1);
        mbar_init(smem_u32(smem + 32), 1);
        *reinterpret_cast<volatile int*>(smem + 20) = 0;
        fence_mbar_init();
    }
    if ((threadIdx.x >> 5) == 0) tmem_alloc(smem_u32(smem + 8), ncols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
}

__device__ __forceinline__ void tc_header_release(unsigned char* smem, uint32_t tmem, uint32_t ncols)
{
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if ((threadIdx.x >> 5) == 0) tmem_dealloc(tmem, ncols);
}

// Two values into packed FP16 high and low parts: hi = x rounded to 11 significant bits by Veltkamp's
// splitting, (x (2^13 + 1)) - ((x (2^13 + 1)) - x) (exact in FP16 for |x| in [2^-14, 2^15]), and
// lo = x - hi (exact in FP32) rounded to FP16; x = hi + lo to 2^-23 relative.  No packed conversion
// is spent on the high part's remainder.
__device__ __forceinline__ void split2h_pair(float x0, float x1, uint32_t& hi, uint32_t& lo)
{
    const float t0 = __fmul_rn(x0, 8193.0f), t1 = __fmul_rn(x1, 8193.0f);
    const float h0 = __fsub_rn(t0, __fsub_rn(t0, x0)), h1 = __fsub_rn(t1, __fsub_rn(t1, x1));
    const __half2 H = __floats2half2_rn(h0, h1);
    const __half2 L = __floats2half2_rn(__fsub_rn(x0, h0), __fsub_rn(x1, h1));
    hi = *reinterpret_cast<const uint32_t*>(&H);
    lo = *reinterpret_cast<const uint32_t*>(&L);
}

}  // namespace mbir
