// Allocation-free variant of the A^T X pass (rsvdgb_pass_atx_noalloc).
//
// Who needs it: code that must not allocate device memory at call time --
// for example a caller running inside a memory pool or arena that owns all of
// the device's memory, a caller that must not synchronise the device (a
// cudaMalloc / cudaFree can), or a real-time caller with a fixed memory
// budget.  Such a caller passes its inputs and outputs and gets the product
// without the library touching the allocator.
//
// How: the split-K partial sums of this pass live in one file-scope device
// array of RSVDGB_NOALLOC_SCRATCH_BYTES.  Every GPU that loads the library
// holds this array until the process exits.  Host code only has a host-side
// stand-in for the array's name, so the first call on each device looks up
// the array's device address with cudaGetSymbolAddress (with that device
// current) and caches it, keyed by the CUDA context; that first call should
// therefore come before any stream capture.  All calls on a device share the
// array and it keeps the last call's contents: calls whose work overlaps on
// the GPU (different streams, or host threads racing on one stream) corrupt
// each other's partial sums.  Each split writes every element of its partial before the
// reduction reads it, so nothing has to be cleared between calls.
#include <cuda.h>

#include <algorithm>
#include <mutex>

#include "internal.cuh"

namespace rsvdgb {
namespace {

constexpr size_t kScratchFloats = RSVDGB_NOALLOC_SCRATCH_BYTES / sizeof(float);
static __device__ __align__(256) float noalloc_scratch[kScratchFloats];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;

// The address is cached per CUDA context, not per device ordinal: a
// cudaDeviceReset destroys the device's primary context and the array with it,
// and the next call, made in the new context (which has another unique id),
// looks the address up again.
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

CtxGetIdFn ctx_get_id()
{
    static CtxGetIdFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &ptr, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (CtxGetIdFn)ptr;
    }
    return fn;
}

struct ScratchEntry {
    unsigned long long ctx_id = 0;
    float* ptr = nullptr;
};
ScratchEntry g_scratch[kMaxDevices];

// Device address of the scratch array in the current device's context (set-up
// on the first call in each context).  Returns nullptr on failure.
float* scratch_for_current_device(int dev)
{
    if (dev < 0 || dev >= kMaxDevices) return nullptr;
    std::lock_guard<std::mutex> lock(g_mutex);
    // make the device's primary context current (cudaSetDevice initialises
    // it) before asking for its id
    if (cudaSetDevice(dev) != cudaSuccess) return nullptr;
    unsigned long long id = 0;
    CtxGetIdFn get_id = ctx_get_id();
    if (!get_id || get_id(nullptr, &id) != CUDA_SUCCESS) return nullptr;
    ScratchEntry& e = g_scratch[dev];
    if (!e.ptr || e.ctx_id != id) {
        void* ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, noalloc_scratch) != cudaSuccess) return nullptr;
        e.ptr = static_cast<float*>(ptr);
        e.ctx_id = id;
    }
    return e.ptr;
}

}  // namespace
}  // namespace rsvdgb

using namespace rsvdgb;

extern "C" int rsvdgb_pass_atx_noalloc(void* cuda_stream, const void* A, int64_t m, int64_t n, int64_t lda, int dtype,
                                       const float* X, int64_t ldx, int l, float* Z, int64_t ldz)
{
    if (!A || !X || !Z || m < 1 || n < 1 || l < 1 || lda < n || ldx < l || ldz < l) return RSVDGB_ERR_INVALID_ARG;
    if (dtype != RSVDGB_F32 && dtype != RSVDGB_BF16) return RSVDGB_ERR_INVALID_ARG;
    // one partial of Z (n x l, leading dimension ldz) must fit in the scratch
    const int64_t per_split = n * ldz;
    if (per_split > (int64_t)kScratchFloats) return RSVDGB_ERR_INVALID_ARG;
    // an error left pending by earlier work is not this call's to report or
    // to clear: refuse to queue anything on top of it
    if (cudaPeekAtLastError() != cudaSuccess) return RSVDGB_ERR_CUDA;
    int sm = 0, dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return RSVDGB_ERR_CUDA;
    if (cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sm < 1)
        return RSVDGB_ERR_CUDA;
    float* scratch = scratch_for_current_device(dev);
    if (!scratch) return RSVDGB_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)cuda_stream;

    // Z = A^T X: op(A)(i,k) = A[k*lda + i] (i < n, k < m), X row-major m x l.
    const int64_t tiles = ceil_div(n, 64) * ceil_div(l, 64);
    int64_t splits = ceil_div(4 * (int64_t)sm, tiles);
    splits = std::min<int64_t>(splits, std::max<int64_t>(1, m / 256));
    splits = std::min<int64_t>(splits, (int64_t)kScratchFloats / per_split);
    splits = std::max<int64_t>(1, std::min<int64_t>(splits, 256));

    GemmArgs a{};
    a.A = A;
    a.lda = lda;
    a.a_bf16 = dtype == RSVDGB_BF16;
    a.B = X;
    a.ldb = ldx;
    a.M = n;
    a.N = l;
    a.K = m;
    a.C = scratch;
    a.ldc = ldz;
    a.splits = (int)splits;
    a.split_stride = per_split;
    launch_simt_gemm(s, true, false, false, a);
    launch_reduce_splits(s, scratch, (int)splits, per_split, n, l, ldz, Z, ldz);
    if (cudaGetLastError() != cudaSuccess) return RSVDGB_ERR_CUDA;
    return RSVDGB_OK;
}
