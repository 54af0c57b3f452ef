// Image sharpness without any device allocation.
//
// Same quantity as sas_sharpness (S = sum|I|^4 / (sum|I|^2)^2, N, D and the
// gradient g = 2 I (|I|^2/D^2 - N/D^3)), for callers that are not allowed to
// allocate GPU memory once they are running: a vehicle-borne processor that
// reserves all of its memory at start-up so a long mission can never stop on a
// failed or fragmenting allocation next to other GPU programs, or a host
// framework whose own memory manager forbids cudaMalloc/cudaFree because those
// calls synchronise the device.  The per-block partial sums live in a
// fixed-size array compiled into the library instead of in allocated memory.
#include "sas_common.cuh"

#include <mutex>

namespace sas {
namespace {

constexpr int CHUNK = 16384;                       // elements reduced by one block
constexpr int MAX_BLOCKS = 4096;                   // partial-sum slots in the array
constexpr int TPB = 256;
constexpr long long MAX_N = (long long)CHUNK * MAX_BLOCKS;   // 67,108,864 elements

// (N, D) partial sums, one pair per block.  Every GPU that loads the library
// holds these 64 KiB until the process exits.
static __device__ __align__(256) double g_sharp_scratch[2 * MAX_BLOCKS];

// Device addresses of g_sharp_scratch, looked up once per device.
std::mutex g_mu;
double* g_scratch_dev[64] = {nullptr};

int scratch_for_current_device(double** out) {
    int dev = 0;
    SAS_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) {
        set_error("sas_sharpness_static: device index %d out of range", dev);
        return SAS_ERR_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_dev[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_sharp_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_sharp_scratch)");
        g_scratch_dev[dev] = static_cast<double*>(p);
    }
    *out = g_scratch_dev[dev];
    return SAS_OK;
}

__device__ __forceinline__ void block_sum2(double& a, double& b) {
    __shared__ double ra[TPB / 32], rb[TPB / 32];
    for (int o = 16; o; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if ((threadIdx.x & 31) == 0) {
        ra[threadIdx.x >> 5] = a;
        rb[threadIdx.x >> 5] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        a = 0.0;
        b = 0.0;
        for (int k = 0; k < TPB / 32; ++k) {
            a += ra[k];
            b += rb[k];
        }
    }
}

// block b reduces elements [b*CHUNK, min(n, (b+1)*CHUNK)) into slot b
__global__ void __launch_bounds__(TPB) chunk_partials(const float2* __restrict__ img, long long n,
                                                      double* __restrict__ part) {
    const long long lo = (long long)blockIdx.x * CHUNK;
    const long long hi = min(n, lo + CHUNK);
    double N = 0.0, D = 0.0;
    for (long long i = lo + threadIdx.x; i < hi; i += TPB) {
        const float2 v = img[i];
        const double a = (double)v.x * v.x + (double)v.y * v.y;
        N += a * a;
        D += a;
    }
    block_sum2(N, D);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = N;
        part[2 * blockIdx.x + 1] = D;
    }
}

// reads only the nblocks slots written by this call's chunk_partials
__global__ void __launch_bounds__(TPB) chunk_final(const double* __restrict__ part, int nblocks,
                                                   double* __restrict__ out3) {
    double N = 0.0, D = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += TPB) {
        N += part[2 * b];
        D += part[2 * b + 1];
    }
    block_sum2(N, D);
    if (threadIdx.x == 0) {
        out3[0] = D > 0.0 ? N / (D * D) : 0.0;
        out3[1] = N;
        out3[2] = D;
    }
}

__global__ void grad_from_sums(const float2* __restrict__ img, long long n, const double* __restrict__ out3,
                               float2* __restrict__ g) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double N = out3[1], D = out3[2];
    const float2 v = img[i];
    const double a = (double)v.x * v.x + (double)v.y * v.y;
    const double k = D > 0.0 ? 2.0 * (a / (D * D) - N / (D * D * D)) : 0.0;
    g[i] = make_float2((float)(k * v.x), (float)(k * v.y));
}

}  // namespace
}  // namespace sas

using namespace sas;

extern "C" int sas_sharpness_static(const void* d_image, int64_t n, double* d_out3, void* d_grad, void* stream) {
    if (!d_image || !d_out3 || n < 1) {
        set_error("sas_sharpness_static: bad argument");
        return SAS_ERR_ARG;
    }
    if (n > MAX_N) {
        set_error("sas_sharpness_static: %lld elements exceed the built-in limit of %lld "
                  "(use sas_sharpness, which allocates its scratch)",
                  (long long)n, MAX_N);
        return SAS_ERR_ARG;
    }
    double* part = nullptr;
    int rc = scratch_for_current_device(&part);
    if (rc != SAS_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const int nblocks = (int)((n + CHUNK - 1) / CHUNK);
    chunk_partials<<<nblocks, TPB, 0, st>>>((const float2*)d_image, n, part);
    SAS_CUDA(cudaGetLastError());
    chunk_final<<<1, TPB, 0, st>>>(part, nblocks, d_out3);
    SAS_CUDA(cudaGetLastError());
    if (d_grad) {
        grad_from_sums<<<(unsigned)((n + 255) / 256), 256, 0, st>>>((const float2*)d_image, n, d_out3,
                                                                   (float2*)d_grad);
        SAS_CUDA(cudaGetLastError());
    }
    return SAS_OK;
}
