// Shared pieces of the tensor-core apply kernels (tc_stream.cuh): the
// shared-memory header set-up (mbarriers, tensor-memory allocation) and the
// two-part FP16 split of the FP32 form.
#pragma once

#include "apply_common.cuh"
#include <cuda_fp16.h>

#include "tc_common.cuh"

namespace mbir {

constexpr int kTcThreads = 512;      // 16 warps: four per tensor-memory lane quarter

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
