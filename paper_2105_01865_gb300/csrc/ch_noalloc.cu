// ch_mass_noalloc: the FP64 mass reduction without any device allocation.
//
// ch_mass needs a handle, and ch_create allocates the handle's tables with
// cudaMalloc.  Some callers cannot call cudaMalloc: an application that owns
// the whole device memory budget through its own pool and forbids libraries
// to allocate behind its back, or a plug-in that is handed only input and
// output pointers by its host.  This entry point gives them h^3 * sum(C) with
// the block partial sums kept in a fixed, file-scope device array instead of
// allocated scratch.  Every call outside a stream capture looks up that
// array's device address (cudaGetSymbolAddress, with the device current), so a
// device reset or a new primary context is picked up; a call on a capturing
// stream reuses the address of the last call on that device, so make one call
// on the device before any stream capture.  All calls share the one array, so
// calls whose kernels overlap on the GPU (different streams, or different
// host threads on one device) race and may return wrong sums.
#include <cuda_runtime.h>

#include <mutex>

#include "ch_internal.h"

namespace {

constexpr int kThreads = 256;
constexpr int kPerThread = 16;
constexpr int64_t kCellsPerBlock = (int64_t)kThreads * kPerThread;  // 4096 cells per partial sum
constexpr int kMaxPartials = 65536;                                   // 512 KB of partials
constexpr int kMaxDevices = 64;

// The scratch: one FP64 partial sum per block of 4096 cells.  Every GPU that
// loads this library holds it (512 KB) until the process exits.
static __device__ __align__(256) double g_partials[kMaxPartials];

double* g_partials_addr[kMaxDevices];  // device address of g_partials, per device
std::mutex g_setup_mutex;

__device__ __forceinline__ double block_sum(double v) {
    __shared__ double ws[kThreads / 32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) ws[w] = v;
    __syncthreads();
    v = (threadIdx.x < kThreads / 32) ? ws[threadIdx.x] : 0.0;
    if (w == 0)
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block b sums cells [b * 4096, (b + 1) * 4096) into partials[b]; every slot
// the finish kernel reads is written by this launch, so nothing is cleared.
template <typename T>
__global__ void __launch_bounds__(kThreads) mass_partials(const T* __restrict__ C, int64_t n, double* partials) {
    const int64_t base = (int64_t)blockIdx.x * kCellsPerBlock;
    double acc = 0.0;
#pragma unroll
    for (int m = 0; m < kPerThread; ++m) {
        const int64_t e = base + (int64_t)m * kThreads + threadIdx.x;
        if (e < n) acc += (double)C[e];
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

__global__ void __launch_bounds__(kThreads) mass_finish(const double* partials, int nb, double scale, double* out) {
    double acc = 0.0;
    for (int b = threadIdx.x; b < nb; b += kThreads) acc += partials[b];
    acc = block_sum(acc);
    if (threadIdx.x == 0) *out = acc * scale;
}

// Device address of g_partials on the current device.  Looked up afresh on
// every call that is not being captured (the address changes if the device's
// context is torn down and created again); a capturing call takes the last
// address looked up on this device and fails if there is none.
cudaError_t partials_for_current_device(cudaStream_t s, double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(s, &cap);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (cap == cudaStreamCaptureStatusNone) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_partials);
        if (e != cudaSuccess) return e;
        g_partials_addr[dev] = (double*)p;
    }
    if (!g_partials_addr[dev]) return cudaErrorStreamCaptureUnsupported;
    *out = g_partials_addr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" int ch_mass_noalloc(const void* C, int64_t nx, int64_t ny, int64_t nz, double h, int precision,
                               double* out, void* stream) {
    if (!C || !out || nx < 1 || ny < 1 || nz < 1 || !(h > 0)) return CH_EINVAL;
    if (precision != CH_F32 && precision != CH_F64) return CH_EINVAL;
    if (nx > ((int64_t)1 << 40) / ny / nz) return CH_EINVAL;
    const int64_t n = nx * ny * nz;
    const int64_t blocks = (n + kCellsPerBlock - 1) / kCellsPerBlock;
    if (blocks > kMaxPartials) {
        fprintf(stderr,
                "ch_mass_noalloc: %lld cells exceed the fixed scratch limit of %lld cells "
                "(%d partial sums of %lld cells)\n",
                (long long)n, (long long)kMaxPartials * kCellsPerBlock, kMaxPartials, (long long)kCellsPerBlock);
        return CH_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    double* partials = nullptr;
    if (partials_for_current_device(s, &partials) != cudaSuccess) return CH_ECUDA;
    if (precision == CH_F64)
        mass_partials<double><<<(unsigned)blocks, kThreads, 0, s>>>((const double*)C, n, partials);
    else
        mass_partials<float><<<(unsigned)blocks, kThreads, 0, s>>>((const float*)C, n, partials);
    if (cudaGetLastError() != cudaSuccess) return CH_ECUDA;
    mass_finish<<<1, kThreads, 0, s>>>(partials, (int)blocks, h * h * h, out);
    if (cudaGetLastError() != cudaSuccess) return CH_ECUDA;
    return CH_OK;
}
