// pp_expect_noalloc: the <0..0|O~|0..0> reduction for callers that cannot
// allocate device memory.
//
// Some callers of this library cannot call cudaMalloc (or any allocator) at the
// point where they need the expectation value: code running while a CUDA stream
// is being captured into a graph (allocation there would break the capture),
// code that owns every byte of device memory through its own pool and forbids
// foreign allocations, and hosts that must not touch the CUDA allocator for
// latency reasons.  pp_expect needs a handle, whose reduction scratch comes from
// the handle's allocator.  This variant takes the terms from the caller's own
// device buffers and keeps its scratch -- the per-chunk partial sums of the
// exact fixed-point reduction -- in a file-scope device array of fixed size,
// created when the library is loaded and held by every GPU that loads it until
// the process exits.
//
// Shared state: every call uses the same array, which keeps whatever the last
// call left in it.  Each call overwrites the partials it reads before reading
// them, so nothing needs to start at zero; calls that overlap on the GPU (two
// streams, or two host threads) race on the array and must be serialised by
// the caller.
#include <cstdio>
#include <mutex>

#include "pp.h"
#include "pp_device.cuh"

namespace {

constexpr size_t kNoAllocChunk = 16384;                       // terms per partial sum
constexpr size_t kNoAllocPartials = PP_NOALLOC_MAX_TERMS / kNoAllocChunk;

static_assert(PP_NOALLOC_MAX_TERMS % kNoAllocChunk == 0, "limit must be whole chunks");

// The scratch: one 128-bit fixed-point partial per chunk (128 KiB).
static __device__ __align__(256) __int128 g_noalloc_partials[kNoAllocPartials];

// Each block reduces one chunk of terms (row-major [n][W] masks) into its partial.
template <int W>
__global__ void k_expect_noalloc_partials(const uint64_t* x, const double* c, size_t n, __int128* part) {
    __shared__ __int128 s[256];
    const size_t begin = (size_t)blockIdx.x * kNoAllocChunk;
    const size_t end = begin + kNoAllocChunk < n ? begin + kNoAllocChunk : n;
    __int128 acc = 0;
    bool bad = false;
    for (size_t i = begin + threadIdx.x; i < end; i += blockDim.x) {
        bool diag = true;
#pragma unroll
        for (int w = 0; w < W; ++w) diag = diag && x[i * W + w] == 0ull;
        if (diag) {
            if (pp::fix80_valid(c[i])) acc += pp::to_fixed80(c[i]);
            else bad = true;
        }
    }
    s[threadIdx.x] = acc;
    bad = __syncthreads_or(bad);
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) s[threadIdx.x] += s[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = bad ? FIX80_INVALID : s[0];
}

// One block folds the partials and writes the value as a double.
__global__ void k_expect_noalloc_final(const __int128* part, int nparts, double* out) {
    __shared__ __int128 s[256];
    __int128 acc = 0;
    bool bad = false;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) {
        if (part[i] == FIX80_INVALID) bad = true;
        else acc += part[i];
    }
    s[threadIdx.x] = acc;
    bad = __syncthreads_or(bad);
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) s[threadIdx.x] += s[threadIdx.x + h];
        __syncthreads();
    }
    // rounded exactly as pp_expect rounds its total (same routine)
    if (threadIdx.x == 0) *out = pp::fixed80_to_double(bad ? FIX80_INVALID : s[0]);
}

// Device address of the scratch array, looked up once per device.
constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
__int128* g_scratch_addr[kMaxDevices] = {};

cudaError_t scratch_for_current_device(__int128** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
        void* ptr = nullptr;
        // In host code the array's name is only a host-side stand-in; the
        // device address comes from the runtime, with this device current.
        e = cudaGetSymbolAddress(&ptr, g_noalloc_partials);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = static_cast<__int128*>(ptr);
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" pp_status pp_expect_noalloc(int n_qubits, size_t n_terms, const uint64_t* x_dev,
                                       const double* c_dev, double* value_dev, void* cuda_stream) {
    if (n_qubits < 1 || n_qubits > 128 || !value_dev) return PP_ERR_ARG;
    if (n_terms && (!x_dev || !c_dev)) return PP_ERR_ARG;
    if (n_terms > PP_NOALLOC_MAX_TERMS) return PP_ERR_CAPACITY;
    __int128* part = nullptr;
    if (scratch_for_current_device(&part) != cudaSuccess) {
        cudaGetLastError();
        return PP_ERR_CUDA;
    }
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const int W = (n_qubits + 63) / 64;
    const int nparts = (int)((n_terms + kNoAllocChunk - 1) / kNoAllocChunk);
    if (nparts > 0) {
        if (W == 1) k_expect_noalloc_partials<1><<<nparts, 256, 0, st>>>(x_dev, c_dev, n_terms, part);
        else k_expect_noalloc_partials<2><<<nparts, 256, 0, st>>>(x_dev, c_dev, n_terms, part);
    }
    k_expect_noalloc_final<<<1, 256, 0, st>>>(part, nparts, value_dev);
    return cudaGetLastError() == cudaSuccess ? PP_OK : PP_ERR_CUDA;
}
