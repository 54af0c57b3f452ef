// Image sharpness S = sum|I|^4 / (sum|I|^2)^2 and its Wirtinger gradient
// g = dS/dI* = 2 I (|I|^2 / D^2 - N / D^3), N = sum|I|^4, D = sum|I|^2.
// The focus measure driving the autofocus loop (per-ping offsets are adjusted
// to maximise S).  Sums are FP64 in a fixed order: a fixed number of blocks,
// each reducing a fixed strided subset, then one block over the partials.
#include "sas_common.cuh"

namespace sas {
namespace {

constexpr int SBLOCKS = 1024;
constexpr int STHREADS = 256;

__device__ __forceinline__ void block_sum2(double& a, double& b) {
    __shared__ double ra[STHREADS / 32], rb[STHREADS / 32];
    for (int o = 16; o; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        ra[w] = a;
        rb[w] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        a = 0.0;
        b = 0.0;
        for (int k = 0; k < STHREADS / 32; ++k) {
            a += ra[k];
            b += rb[k];
        }
    }
}

__global__ void __launch_bounds__(STHREADS) sharp_partials(const float2* __restrict__ img, long long n,
                                                           double* __restrict__ part) {
    double N = 0.0, D = 0.0;
    for (long long i = blockIdx.x * (long long)STHREADS + threadIdx.x; i < n; i += (long long)SBLOCKS * STHREADS) {
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

__global__ void __launch_bounds__(STHREADS) sharp_final(const double* __restrict__ part, double* __restrict__ out3) {
    double N = 0.0, D = 0.0;
    for (int b = threadIdx.x; b < SBLOCKS; b += STHREADS) {
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

__global__ void sharp_grad(const float2* __restrict__ img, long long n, const double* __restrict__ out3,
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

int sharpness(const float2* img, long long n, double* out3, float2* grad, double* part, cudaStream_t st) {
    sharp_partials<<<SBLOCKS, STHREADS, 0, st>>>(img, n, part);
    SAS_CUDA(cudaGetLastError());
    sharp_final<<<1, STHREADS, 0, st>>>(part, out3);
    SAS_CUDA(cudaGetLastError());
    if (grad) {
        sharp_grad<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(img, n, out3, grad);
        SAS_CUDA(cudaGetLastError());
    }
    return SAS_OK;
}

size_t sharpness_scratch_bytes() { return sizeof(double) * 2 * SBLOCKS; }

}  // namespace sas

using namespace sas;

extern "C" int sas_sharpness(const void* d_image, int64_t n, double* d_out3, void* d_grad, void* stream) {
    if (!d_image || !d_out3 || n < 1) {
        set_error("sas_sharpness: bad argument");
        return SAS_ERR_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    double* part = nullptr;
    SAS_CUDA(cudaMallocAsync(&part, sharpness_scratch_bytes(), st));
    int rc = sharpness((const float2*)d_image, n, d_out3, (float2*)d_grad, part, st);
    cudaFreeAsync(part, st);
    return rc;
}
