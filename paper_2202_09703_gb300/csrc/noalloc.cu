// mbir_backproject_noalloc: A^T r without any device allocation.
//
// Some callers cannot allocate device memory at the point where they apply
// the adjoint: real-time loops that forbid allocator calls after start-up
// (an allocation can block for an unbounded time), and hosts whose device
// memory is one pool sized and handed out in advance by another component.
// mbir_backproject may allocate its workspace on first use; this entry point
// instead takes its scratch from one fixed array that is part of the library
// image.
//
// The scratch holds the residual rows padded with a zero tail (K x Mp floats)
// followed by the per-transmitter-group partial images (groups x N floats).
// Both are completely rewritten by every call before they are read, so
// nothing has to be cleared between calls.  The array is shared by all calls
// in the process: two calls whose work overlaps on the GPU (different
// streams, or different host threads) race on it and must be serialised by
// the caller.  The call also uses the geometry's own adjoint work counter,
// so it must not overlap any other adjoint on the same geometry either.
//
// Set-up happens when a geometry that the entry point takes is created
// (noalloc_prepare, called by mbir_create_geometry with the geometry's device
// current): the array's device address is looked up once per device, which
// also loads the module that holds the array when modules load lazily, and
// the kernels of the call are loaded too.  The call itself then loads and
// allocates nothing.
#include <mutex>

#include "device_common.cuh"

namespace {

// 16 MiB of scratch, held by every GPU that loads the library until exit.
constexpr size_t kNoAllocFloats = (size_t)16 * 1024 * 1024 / sizeof(float);
static __device__ __align__(256) float g_noalloc_scratch[kNoAllocFloats];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
float* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on `dev` (the current device).  The
// host-side symbol is only a stand-in, so the address is looked up once per
// device and cached.
cudaError_t scratch_for(int dev, float** out)
{
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = static_cast<float*>(p);
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

// Whether the entry point takes g: FP32 storage and a scratch of at most kNoAllocFloats.
bool noalloc_fits(const mbir_geometry* g, size_t* rows_out, size_t* parts_out)
{
    const size_t rows = (size_t)g->P.K * g->P.Mp;
    const size_t parts = (size_t)g->n_groups * g->P.W * g->P.H;
    *rows_out = rows;
    *parts_out = parts;
    return g->P.precision == MBIR_PREC_FP32 && ((rows + 63) & ~(size_t)63) + parts <= kNoAllocFloats;
}

}  // namespace

namespace mbir {
cudaError_t noalloc_prepare(const mbir_geometry* g)
{
    size_t rows, parts;
    if (g->device < 0 || g->device >= kMaxDevices || !noalloc_fits(g, &rows, &parts)) return cudaSuccess;
    float* scratch = nullptr;
    cudaError_t e = scratch_for(g->device, &scratch);
    if (e == cudaSuccess) e = load_pad_rows();
    if (e == cudaSuccess) e = load_backproject_partials(g);
    return e;
}
}  // namespace mbir

extern "C" int mbir_backproject_noalloc(const mbir_geometry* g, const float* r_dev, float* x_dev, void* stream)
{
    if (!g || !r_dev || !x_dev) return MBIR_ERR_INVALID_ARG;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != g->device || dev < 0 || dev >= kMaxDevices)
        return MBIR_ERR_INVALID_ARG;
    size_t rows, parts;
    if (!noalloc_fits(g, &rows, &parts)) return MBIR_ERR_UNSUPPORTED;   // BF16, or beyond the fixed 16 MiB
    float* scratch = nullptr;                   // resolved when g was created: a cached lookup here
    if (scratch_for(dev, &scratch) != cudaSuccess) return MBIR_ERR_CUDA;
    float* e_pad = scratch;
    float* partial = scratch + ((rows + 63) & ~(size_t)63);
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = mbir::launch_pad_rows(g, r_dev, 0, e_pad, st);
    if (e == cudaSuccess) e = mbir::launch_backproject_partials(g, e_pad, nullptr, x_dev, partial, st);
    return e == cudaSuccess ? MBIR_OK : MBIR_ERR_CUDA;
}
