// flood_storage_static: the FP64 water volume of one depth field, computed
// without allocating any memory.
//
// Some callers cannot call cudaMalloc at all: code that runs inside a stream
// capture (an allocation there fails or becomes part of the graph), code that
// runs under a fixed device-memory budget managed by someone else (an
// embedding application's pool), or real-time loops that must never block on
// the allocator.  They pass their own input and output buffers; the block
// partial sums this reduction needs live in a file-scope device array of a
// fixed size, so nothing is allocated per call.
//
// The arithmetic is the same as the library's own storage reduction (rows of
// 16 per block, 256 threads, a shared-memory tree, then the block partials
// added in block order), so for the same depth field the two agree bit for
// bit.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/flood.h"

namespace {

constexpr int kRowsPerBlock = 16;
constexpr int kThreads = 256;
constexpr int kMaxBlocks = FLOOD_STATIC_MAX_ROWS / kRowsPerBlock;
constexpr int kMaxDevices = 64;

// Block partials of the current call.  One array per device that loads the
// library, shared by every call on that device: each call overwrites the
// partials it uses before reading them, and two calls that overlap on the GPU
// (different streams, no ordering between them) race on it.
static __device__ __align__(256) double g_partials[kMaxBlocks];

double* g_scratch[kMaxDevices] = {};
std::once_flag g_once[kMaxDevices];
cudaError_t g_setup_err[kMaxDevices] = {};
thread_local std::string g_msg;

__global__ void partial_kernel(const float* __restrict__ h, int ny, int nx, int ld,
                               double* __restrict__ part)
{
    const int r0 = blockIdx.x * kRowsPerBlock, r1 = min(r0 + kRowsPerBlock, ny);
    double acc = 0.0;
    for (int r = r0; r < r1; ++r)
        for (int c = threadIdx.x; c < nx; c += blockDim.x) acc += (double)h[(size_t)r * ld + c];
    __shared__ double red[kThreads];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void final_kernel(const double* __restrict__ part, int nb, double area,
                             double* __restrict__ out)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double acc = 0.0;
    for (int b = 0; b < nb; ++b) acc += part[b];
    *out = acc * area;
}

int fail(int code, const std::string& m)
{
    g_msg = m;
    return code;
}

}  // namespace

extern "C" const char* flood_storage_static_error(void) { return g_msg.c_str(); }

extern "C" int flood_storage_static(const float* h, int ny, int nx, int ld, double dx, double* out,
                                    void* stream)
{
    if (!h || !out) return fail(FLOOD_ERR_ARG, "h and out must be device pointers");
    if (ny < 1 || nx < 1 || ld < nx) return fail(FLOOD_ERR_ARG, "need ny >= 1, nx >= 1, ld >= nx");
    if (ny > FLOOD_STATIC_MAX_ROWS)
        return fail(FLOOD_ERR_ARG, "ny exceeds FLOOD_STATIC_MAX_ROWS (" +
                                       std::to_string(FLOOD_STATIC_MAX_ROWS) + " rows)");
    if (!(dx > 0.0)) return fail(FLOOD_ERR_ARG, "dx must be positive");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(FLOOD_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail(FLOOD_ERR_ARG, "device ordinal out of range");
    // First call on this device (with it current): find where the partials
    // array lives.  The name g_partials in host code is only a stand-in for
    // the device array, not its address.
    std::call_once(g_once[dev], [dev]() {
        void* p = nullptr;
        g_setup_err[dev] = cudaGetSymbolAddress(&p, g_partials);
        if (g_setup_err[dev] == cudaSuccess) g_scratch[dev] = static_cast<double*>(p);
    });
    if (g_setup_err[dev] != cudaSuccess || !g_scratch[dev])
        return fail(FLOOD_ERR_CUDA, std::string("cudaGetSymbolAddress: ") +
                                        cudaGetErrorString(g_setup_err[dev]));
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int nb = (ny + kRowsPerBlock - 1) / kRowsPerBlock;
    partial_kernel<<<nb, kThreads, 0, s>>>(h, ny, nx, ld, g_scratch[dev]);
    final_kernel<<<1, 32, 0, s>>>(g_scratch[dev], nb, dx * dx, out);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(FLOOD_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
    return FLOOD_OK;
}
