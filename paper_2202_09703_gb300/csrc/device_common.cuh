// Device helpers shared by the apply kernels: leg access for the two modes,
// pulse-table addressing, mbarrier / bulk-copy PTX wrappers and bounded waits.
#pragma once

#include "mbir_internal.h"

namespace mbir {

constexpr int kModeOTF = MBIR_MODE_OTF;
constexpr int kModeTAB = MBIR_MODE_TAB;
constexpr long long kWaitCycles = 4000000000LL;   // ~2 s at 2 GHz

// Pulse-table row stride (float2 entries): the next odd number >= Tw4, so that
// rows of different phases start on different 8-byte bank pairs.
__host__ __device__ inline int table_stride(int Tw4) { return Tw4 + 1; }

struct DevPtrs {
    const RowInfo* rows;
    const float2* colx;
    const float2* pos;
    const int* txpos;
    const int* rxpos;
    const float4* legs;
    const int* hidx;
    int* status;
};

DevPtrs dev_ptrs(const mbir_geometry* g);

template <int NL, int MODE>
__device__ __forceinline__ Leg get_leg(const GeomParams& P, const DevPtrs& D, const RowInfo& ri,
                                       int row, int col, int posidx)
{
    if constexpr (MODE == kModeTAB) {
        int hi = __ldg(D.hidx + (size_t)posidx * P.W + col);
        float4 v = __ldg(D.legs + (size_t)row * P.nh + hi);
        return Leg{v.x, v.y, v.z, v.w};
    } else {
        df h = abs_diff(__ldg(D.colx + col), __ldg(D.pos + posidx));
        return solve_leg<NL>(P, ri, h);
    }
}

__device__ __forceinline__ RowInfo load_row(const RowInfo* rows, int r)
{
    RowInfo ri;
    const int4* p = reinterpret_cast<const int4*>(rows + r);
    int4 a = __ldg(p), b = __ldg(p + 1);
    ri.nl = a.x;
    ri.pmax = __int_as_float(a.y);
    ri.eta_last = make_float2(__int_as_float(a.z), __int_as_float(a.w));
    ri.tau = __int_as_float(b.x);
    ri.tvert = __int_as_float(b.y);
    ri.mrow = __int_as_float(b.z);
    ri.pad = b.w;
    return ri;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, int count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// 1-D bulk copy global -> shared, completing `bytes` on the mbarrier.
// Both addresses 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

// Prefetch [p, p + bytes) of global memory into L2 (bulk, fire and forget): the start is rounded down and
// the end down to 16-byte bounds (the range never leaves the caller's array, whose allocation starts on a
// 256-byte bound), cut into 32 KB pieces, piece i issued by lane i of the calling warp (pieces past 32 are
// dropped).
__device__ __forceinline__ void prefetch_l2_range(const void* p, size_t bytes, int lane)
{
    if (bytes == 0) return;
    const uintptr_t a = reinterpret_cast<uintptr_t>(p) & ~(uintptr_t)15;
    const uintptr_t z = (reinterpret_cast<uintptr_t>(p) + bytes) & ~(uintptr_t)15;
    const uintptr_t q = a + (uintptr_t)lane * 32768;
    if (q < z) {
        const uint32_t n = (uint32_t)((z - q) < 32768 ? (z - q) : 32768);
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(q), "r"(n) : "memory");
    }
}

// Read-only loads with an L1 eviction hint: streamed data read once (L1::no_allocate keeps it from pushing
// reused lines out of the L1), and gathered data that is read again (L1::evict_last).
__device__ __forceinline__ uint2 ldg_stream(const uint2* p)
{
    uint2 v;
    asm("ld.global.nc.L1::no_allocate.v2.u32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "l"(p));
    return v;
}
__device__ __forceinline__ uint32_t ldg_stream(const uint32_t* p)
{
    uint32_t v;
    asm("ld.global.nc.L1::no_allocate.u32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ float ldg_keep(const float* p)
{
    float v;
    asm("ld.global.nc.L1::evict_last.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
}

// *p += v in global memory as a reduction that returns nothing: the address is taken into the global window
// explicitly, so a pointer read from memory (a generic pointer to the compiler) still gets the
// fire-and-forget form rather than an atomic that waits for the old value.
__device__ __forceinline__ void red_add_global_u64(unsigned long long* p, unsigned long long v)
{
    asm volatile("red.relaxed.gpu.global.add.u64 [%0], %1;" ::"l"(__cvta_generic_to_global(p)), "l"(v) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for an mbarrier phase with a cycle limit; returns false (and records
// the failure in *status) if the limit is reached.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, int* status)
{
    if (mbar_try_wait(bar, parity)) return true;
    long long start = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - start > kWaitCycles) {
            atomicExch(status, 1);
            return false;
        }
    }
    return true;
}

template <bool BF16>
struct TabT;
template <>
struct TabT<false> {
    using type = float2;
    __device__ static float2 ld(const float2* p) { return *p; }
};
template <>
struct TabT<true> {
    using type = __nv_bfloat162;
    __device__ static float2 ld(const __nv_bfloat162* p) { return __bfloat1622float2(*p); }
};

template <bool BF16>
struct ET;
template <>
struct ET<false> {
    using type = float;
    __device__ static float ld(const float* p) { return *p; }
};
template <>
struct ET<true> {
    using type = __nv_bfloat16;
    __device__ static float ld(const __nv_bfloat16* p) { return __bfloat162float(*p); }
};

}  // namespace mbir
