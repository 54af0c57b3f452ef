// Register-resident complex FFT of rows of N = 2^m points, 256 <= N <= 16384,
// for the conditioning kernels (matched filtering, whitening).
//
// A row is spread over T = N / (16 B) threads; thread t holds the 16 B points
// x[m] = row[t + T m] ("natural slots").  The transform is the Stockham
// autosort form with radix-16 stages (a final radix 2, 4 or 8 stage when
// log2 N is not a multiple of 4).  Stage (R, L), butterfly j < N / R, k = j mod
// L: inputs row[j + q N / R] times w^q, w = exp(s 2 pi i k / (R L)), an R-point
// DFT, outputs to position R (j - k) + k + q L.  The inputs of every stage are
// natural slots of the thread that computes the butterfly, so each stage runs
// in registers; its outputs go through shared memory (one pad point every 16,
// which keeps the scattered writes free of bank conflicts) to the next
// stage's natural slots, and the last stage's outputs are, in place, the
// natural slots of the transform.  A transform therefore takes its input from
// and leaves its output in registers, with one shared-memory exchange between
// consecutive stages (3 for N = 16384; the radix-4 form in fft.cuh makes 7
// passes).  Forward (s = -1): X[f] = sum_n x[n] exp(-2 pi i f n / N); inverse
// (s = +1): +i and no 1/N.  Twiddles from the half table exp(-2 pi i j / N),
// j < N / 2 (exp(-2 pi i j / N) = -tw(j - N/2) above it), stored at
// tpad(j) = j + j/16 + j/256: a stage reads w^h at h k N / (R L) for the lanes'
// consecutive k, power-of-two strides that the skew spreads over the banks
// (about 1.5 wavefronts a request instead of 4 to 10 unskewed): w, w^2, w^3,
// w^4, w^8, w^12 looked up, the other powers one product of two of them.
#pragma once

#include <cuda_runtime.h>

namespace sas {
namespace fftreg {

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }

// (s i) a for s = -1 (forward) or +1 (inverse)
template <bool FWD>
__device__ __forceinline__ float2 mul_si(float2 a) {
    return FWD ? make_float2(a.y, -a.x) : make_float2(-a.y, a.x);
}

// shared-memory index of row position i: one pad point every 16
__device__ __forceinline__ int pad(int i) { return i + (i >> 4); }
__host__ __device__ constexpr int padded(int n) { return n + n / 16; }

// twiddle table: entry j at tpad(j); tpad_size(n2) entries hold j < n2
__device__ __forceinline__ int tpad(int j) { return j + (j >> 4) + (j >> 8); }
__host__ __device__ constexpr int tpad_size(int n2) { return n2 + n2 / 16 + n2 / 256 + 1; }

// tw(j) = exp(-2 pi i j / N), j < N / 2, filled by the block
__device__ void twiddles(float2* tw, int N) {
    for (int j = threadIdx.x; j < N / 2; j += blockDim.x) {
        float s, c;
        sincospif(-2.f * (float)j / (float)N, &s, &c);
        tw[tpad(j)] = make_float2(c, s);
    }
    __syncthreads();
}

template <bool FWD>
__device__ __forceinline__ void dft2(float2& a0, float2& a1) {
    const float2 t = a0;
    a0 = cadd(t, a1);
    a1 = csub(t, a1);
}

// in place: a_f = sum_n a_n (s i)^(f n)
template <bool FWD>
__device__ __forceinline__ void dft4(float2& a0, float2& a1, float2& a2, float2& a3) {
    const float2 s02 = cadd(a0, a2), d02 = csub(a0, a2), s13 = cadd(a1, a3), d13 = mul_si<FWD>(csub(a1, a3));
    a0 = cadd(s02, s13);
    a1 = cadd(d02, d13);
    a2 = csub(s02, s13);
    a3 = csub(d02, d13);
}

// exp(s 2 pi i e / 16) for the e = n2 f1 that occur below
template <bool FWD>
__device__ __forceinline__ float2 w16(int e) {
    constexpr float C1 = 0.92387953251128674f, S1 = 0.38268343236508978f, R2 = 0.70710678118654752f;
    const float sg = FWD ? -1.f : 1.f;
    switch (e) {
        case 1: return make_float2(C1, sg * S1);
        case 2: return make_float2(R2, sg * R2);
        case 3: return make_float2(S1, sg * C1);
        case 4: return make_float2(0.f, sg);
        case 6: return make_float2(-R2, sg * R2);
        default: return make_float2(-C1, -sg * S1);   // e = 9
    }
}

// 16-point DFT, n = 4 n1 + n2, f = f1 + 4 f2: four 4-point DFTs over n1,
// the twiddles exp(s 2 pi i n2 f1 / 16), four 4-point DFTs over n2; output f
// in a[perm16(f)]
__host__ __device__ constexpr int perm16(int f) { return 4 * (f & 3) + (f >> 2); }
template <bool FWD>
__device__ __forceinline__ void dft16(float2 (&a)[16]) {
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) dft4<FWD>(a[n2], a[n2 + 4], a[n2 + 8], a[n2 + 12]);
#pragma unroll
    for (int n2 = 1; n2 < 4; ++n2)
#pragma unroll
        for (int f1 = 1; f1 < 4; ++f1) {
            const int e = n2 * f1;
            if (e == 4) a[n2 + 4 * f1] = mul_si<FWD>(a[n2 + 4 * f1]);
            else a[n2 + 4 * f1] = cmul(a[n2 + 4 * f1], w16<FWD>(e));
        }
#pragma unroll
    for (int f1 = 0; f1 < 4; ++f1) dft4<FWD>(a[4 * f1], a[4 * f1 + 1], a[4 * f1 + 2], a[4 * f1 + 3]);
}

// 8-point DFT, n = 2 n1 + n2, f = f1 + 4 f2; output f in a[perm8(f)]
__host__ __device__ constexpr int perm8(int f) { return 2 * (f & 3) + (f >> 2); }
template <bool FWD>
__device__ __forceinline__ void dft8(float2 (&a)[8]) {
    constexpr float R2 = 0.70710678118654752f;
    const float sg = FWD ? -1.f : 1.f;
#pragma unroll
    for (int n2 = 0; n2 < 2; ++n2) dft4<FWD>(a[n2], a[n2 + 2], a[n2 + 4], a[n2 + 6]);
    a[3] = cmul(a[3], make_float2(R2, sg * R2));      // exp(s 2 pi i / 8)
    a[5] = mul_si<FWD>(a[5]);                         // exp(s 2 pi i 2 / 8)
    a[7] = cmul(a[7], make_float2(-R2, sg * R2));     // exp(s 2 pi i 3 / 8)
#pragma unroll
    for (int f1 = 0; f1 < 4; ++f1) dft2<FWD>(a[2 * f1], a[2 * f1 + 1]);
}

template <int R>
__host__ __device__ constexpr int perm(int f) {
    return R == 16 ? perm16(f) : (R == 8 ? perm8(f) : f);
}

template <int R, bool FWD>
__device__ __forceinline__ void dft(float2 (&a)[R]) {
    if constexpr (R == 16) dft16<FWD>(a);
    else if constexpr (R == 8) dft8<FWD>(a);
    else if constexpr (R == 4) dft4<FWD>(a[0], a[1], a[2], a[3]);
    else dft2<FWD>(a[0], a[1]);
}

// exp(s 2 pi i t / N) from the half table
template <int N, bool FWD>
__device__ __forceinline__ float2 twiddle(const float2* tw, int t) {
    float2 v = t < N / 2 ? tw[tpad(t)] : tw[tpad(t - N / 2)];
    if (t >= N / 2) v = make_float2(-v.x, -v.y);
    return FWD ? v : make_float2(v.x, -v.y);
}

// one stage (R, L) over the thread's natural slots x
template <int N, int B, int R, int L, bool FWD>
__device__ __forceinline__ void stage(float2 (&x)[16 * B], float2* row, const float2* tw, int tid) {
    constexpr int T = N / (16 * B), NB = 16 * B / R;
    constexpr bool LAST = R * L == N;
#pragma unroll
    for (int c = 0; c < NB; ++c) {
        const int j = tid + c * T, k = j & (L - 1);
        float2 a[R];
#pragma unroll
        for (int q = 0; q < R; ++q) a[q] = x[c + q * NB];
        if constexpr (L > 1) {
            // w, w^2, w^3 and w^4, w^8, w^12 from the table, w^(4 a + b) = w^(4 a) w^b:
            // every power within one product of the table
            constexpr int ST = N / (R * L);
            const float2 w1 = twiddle<N, FWD>(tw, k * ST);
            a[1] = cmul(a[1], w1);
            if constexpr (R > 2) {
                const float2 w2 = twiddle<N, FWD>(tw, 2 * k * ST), w3 = twiddle<N, FWD>(tw, 3 * k * ST);
                a[2] = cmul(a[2], w2);
                a[3] = cmul(a[3], w3);
                if constexpr (R > 4) {
#pragma unroll
                    for (int h = 4; h < R; h += 4) {
                        const float2 wh = twiddle<N, FWD>(tw, h * k * ST);
                        a[h] = cmul(a[h], wh);
                        a[h + 1] = cmul(a[h + 1], cmul(wh, w1));
                        a[h + 2] = cmul(a[h + 2], cmul(wh, w2));
                        a[h + 3] = cmul(a[h + 3], cmul(wh, w3));
                    }
                }
            }
        }
        dft<R, FWD>(a);
        if constexpr (LAST) {
#pragma unroll
            for (int q = 0; q < R; ++q) x[c + q * NB] = a[perm<R>(q)];
        } else {
#pragma unroll
            for (int q = 0; q < R; ++q) row[pad(R * (j - k) + k + q * L)] = a[perm<R>(q)];
        }
    }
    if constexpr (!LAST) {
        __syncthreads();
#pragma unroll
        for (int m = 0; m < 16 * B; ++m) x[m] = row[pad(tid + T * m)];
        __syncthreads();
    }
}

template <int N, int B, int L, bool FWD>
__device__ __forceinline__ void stages(float2 (&x)[16 * B], float2* row, const float2* tw, int tid) {
    if constexpr (16 * L <= N) {
        stage<N, B, 16, L, FWD>(x, row, tw, tid);
        if constexpr (16 * L < N) stages<N, B, 16 * L, FWD>(x, row, tw, tid);
    } else {
        stage<N, B, N / L, L, FWD>(x, row, tw, tid);
    }
}

// The transform of the row whose natural slots thread tid (< N / (16 B)) of
// its group holds in x; row: the group's padded shared buffer (padded(N)
// points); tw: the table that twiddles() fills (tpad_size(N / 2) points).  Every thread of the block calls it (the
// exchanges synchronise the block).
template <int N, int B, bool FWD>
__device__ __forceinline__ void fft(float2 (&x)[16 * B], float2* row, const float2* tw, int tid) {
    static_assert(N >= 256 && N <= 16384 && (N & (N - 1)) == 0, "N: a power of two in [256, 16384]");
    stages<N, B, 1, FWD>(x, row, tw, tid);
}

// points per thread: 16 up to 4096 points, 32 above (T = N / 32 threads)
template <int N>
__host__ __device__ constexpr int points_b() { return N > 4096 ? 2 : 1; }

}  // namespace fftreg
}  // namespace sas
