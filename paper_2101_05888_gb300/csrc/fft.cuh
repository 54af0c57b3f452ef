// Complex FFT of one row held in shared memory, for the conditioning
// kernels (whitening, matched filtering).  Stockham autosort form, radix 4
// with a final radix-2 stage when log2 N is odd, done in place: every thread
// reads the inputs of its butterflies into registers, the block
// synchronises, then it writes the outputs.  Forward: X[f] = sum_n x[n]
// exp(-2 pi i f n / N); inverse: the same with +i and no 1/N (callers scale).
// Twiddles from a table tw[j] = exp(-2 pi i j / N), j < N/2, that the block
// fills once (fft_twiddles, sincospif: FP32, a few ulp).  N = 2^m,
// 4 <= N <= 16384, blockDim.x a multiple of 32, at most 1024.
#pragma once

#include <cuda_runtime.h>

namespace sas {
namespace fftdev {

constexpr int MAX_N = 16384;
constexpr int R4_PER_THREAD = 4;     // radix-4 butterflies per thread per stage: blockDim.x >= N / 16

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

// tw[j] = exp(-2 pi i j / N), j < N / 2 (shared memory, filled by the block)
__device__ void fft_twiddles(float2* tw, int N) {
    for (int j = threadIdx.x; j < N / 2; j += blockDim.x) {
        float s, c;
        sincospif(-2.f * (float)j / (float)N, &s, &c);
        tw[j] = make_float2(c, s);
    }
    __syncthreads();
}

// sign = -1 forward, +1 inverse.  R4: radix-4 butterflies a thread holds per
// stage (2 R4 radix-2 ones); requires blockDim.x >= N / (4 R4), so that every
// butterfly of a stage is held in registers by the loops below.  R4 = 1 for
// blockDim.x = N / 4 keeps the register footprint (and so the occupancy) of
// small transforms low.
template <int R4 = R4_PER_THREAD>
__device__ void fft_smem(float2* buf, const float2* tw, int N, float sign) {
    constexpr int R2 = 2 * R4;
    const int nt = blockDim.x, tid = threadIdx.x;
    const int N4 = N >> 2;
    int L = 1;
    while (4 * L <= N) {
        float2 y[4 * R4];
#pragma unroll
        for (int c = 0; c < R4; ++c) {
            const int j = tid + c * nt;
            if (j < N4) {
                const int k = j & (L - 1);
                const float2 t1 = tw[k * (N / (4 * L))];                 // exp(-2 pi i k / (4L))
                const float2 w1 = make_float2(t1.x, -sign * t1.y);        // exp(sign 2 pi i k / (4L))
                const float2 w2 = cmul(w1, w1), w3 = cmul(w2, w1);
                const float2 a0 = buf[j], b1 = cmul(w1, buf[j + N4]), b2 = cmul(w2, buf[j + 2 * N4]),
                             b3 = cmul(w3, buf[j + 3 * N4]);
                const float2 s02 = make_float2(a0.x + b2.x, a0.y + b2.y), d02 = make_float2(a0.x - b2.x, a0.y - b2.y);
                const float2 s13 = make_float2(b1.x + b3.x, b1.y + b3.y), d13 = make_float2(b1.x - b3.x, b1.y - b3.y);
                const float2 jd = make_float2(-sign * d13.y, sign * d13.x);   // (sign i) d13
                y[4 * c + 0] = make_float2(s02.x + s13.x, s02.y + s13.y);
                y[4 * c + 1] = make_float2(d02.x + jd.x, d02.y + jd.y);
                y[4 * c + 2] = make_float2(s02.x - s13.x, s02.y - s13.y);
                y[4 * c + 3] = make_float2(d02.x - jd.x, d02.y - jd.y);
            }
        }
        __syncthreads();
#pragma unroll
        for (int c = 0; c < R4; ++c) {
            const int j = tid + c * nt;
            if (j < N4) {
                const int k = j & (L - 1), i = j - k;
#pragma unroll
                for (int q = 0; q < 4; ++q) buf[4 * i + k + q * L] = y[4 * c + q];
            }
        }
        __syncthreads();
        L *= 4;
    }
    if (L < N) {   // one radix-2 stage
        const int N2 = N >> 1;
        float2 y[2 * R2];
#pragma unroll
        for (int c = 0; c < R2; ++c) {
            const int j = tid + c * nt;
            if (j < N2) {
                const int k = j & (L - 1);
                const float2 t1 = tw[k * (N / (2 * L))];                 // exp(-2 pi i k / (2L))
                const float2 a = buf[j], b = cmul(make_float2(t1.x, -sign * t1.y), buf[j + N2]);
                y[2 * c + 0] = make_float2(a.x + b.x, a.y + b.y);
                y[2 * c + 1] = make_float2(a.x - b.x, a.y - b.y);
            }
        }
        __syncthreads();
#pragma unroll
        for (int c = 0; c < R2; ++c) {
            const int j = tid + c * nt;
            if (j < N2) {
                const int k = j & (L - 1), i = j - k;
                buf[2 * i + k] = y[2 * c + 0];
                buf[2 * i + k + L] = y[2 * c + 1];
            }
        }
        __syncthreads();
    }
}

// Threads for an N-point transform: one radix-4 butterfly each up to 1024.
inline int fft_threads(int N) {
    int t = N / 4;
    if (t > 1024) t = 1024;
    if (t < 32) t = 32;
    return t;
}

}  // namespace fftdev
}  // namespace sas
