// Data conditioning around the backprojection (Sec. II-E) and range
// compression:
//  * sas_matched_filter: correlation of raw echo rows with the transmitted
//    replica, y[k] = sum_l e[k + l] conj(p[l]) / sum_l |p[l]|^2, by
//    overlap-save with FP32 register-resident FFTs (fftreg.cuh; a group of
//    threads per block of outputs of a row);
//  * sas_whiten (Eq. 9): P(f) = mean over rows of |FFT(e)|^2 (FP32 sums over
//    runs of rows added in FP64 per chunk of rows, the chunks reduced in a
//    fixed order), G(f) = 1 / (gamma mean P + P(f)), scaled so that max G = 1,
//    applied as a power gain (rows times sqrt G);
//  * sas_tvg (Eq. 10): P(t) = median over rows of the FP32 power |e(t)|^2,
//    exact selection of both middle values by a three-level radix select on
//    the FP32 bit patterns per 8-column strip (one CTA per strip),
//    G(t) = 1 / (alpha mean P + P(t)), applied as a power gain;
//  * sas_drc (Eqs. 11-12): I_n = |I| / max |I| (FP32), the median of I_n by
//    the same three-level select over the whole image, q from Eq. 12, the
//    rational map of Eq. 11.
// The radix-4 shared-memory FFT of fft.cuh serves the replica spectrum and
// whitening rows shorter than 256 points.
// Medians of an even count are the FP64 mean of the two middle values.
#include "fft.cuh"
#include "fftreg.cuh"
#include "sas_common.cuh"

#include <algorithm>
#include <cmath>

namespace sas {
namespace {

using fftdev::fft_smem;
using fftdev::fft_threads;

__device__ __forceinline__ float power_f32(float2 v) { return __fadd_rn(__fmul_rn(v.x, v.x), __fmul_rn(v.y, v.y)); }

// ----------------------------------------------------------------------------
// matched filter

// Pc[f] = conj(FFT(p zero-padded to NF))[f] / (NF sum |p|^2)
__global__ void __launch_bounds__(1024) mf_replica_kernel(const float2* __restrict__ rep, int L, int NF, float2* __restrict__ Pc) {
    extern __shared__ float2 buf[];
    float2* tw = buf + NF;
    fftdev::fft_twiddles(tw, NF);
    __shared__ double esum[32];
    double e = 0.0;
    for (int j = threadIdx.x; j < NF; j += blockDim.x) {
        const float2 v = j < L ? rep[j] : make_float2(0.f, 0.f);
        buf[j] = v;
        e += (double)v.x * v.x + (double)v.y * v.y;
    }
    for (int o = 16; o; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
    if ((threadIdx.x & 31) == 0) esum[threadIdx.x >> 5] = e;
    __syncthreads();
    fft_smem(buf, tw, NF, -1.f);
    double E = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) E += esum[w];
    const float s = (float)(1.0 / ((double)NF * E));
    for (int j = threadIdx.x; j < NF; j += blockDim.x) Pc[j] = make_float2(buf[j].x * s, -buf[j].y * s);
}

// Register-FFT kernels: a CTA of G groups of T = N / (16 B) threads, one row
// (or row block) per group, G = 256 / T up to N = 4096, else 1.
template <int N>
struct RegPlan {
    static constexpr int B = fftreg::points_b<N>(), P = 16 * B, T = N / P;
    static constexpr int G = T >= 256 ? 1 : 256 / T, THREADS = T * G;
    static constexpr int MINB = THREADS <= 256 ? 2 : 1;     // at most 128 registers a thread
    // the matched filter's 16-point rows fit 80 registers without spills: three CTAs an SM
    static constexpr int MINB_MF = B == 1 ? 3 : MINB;
    static constexpr size_t SMEM = sizeof(float2) * ((size_t)G * fftreg::padded(N) + fftreg::tpad_size(N / 2));
};

// One group per (row, block of M outputs): circular correlation of NF inputs
// (the segment raw[k0 .. k0 + NF), zero past the row end) with the replica,
// through the spectra: IFFT(FFT(x) Pc); the first M outputs are the linear
// correlation.
template <int NF>
__global__ void __launch_bounds__(RegPlan<NF>::THREADS, RegPlan<NF>::MINB_MF) mf_reg_kernel(const float2* __restrict__ raw, int n, int M,
                                                                      int nblk, long long items,
                                                                      const float2* __restrict__ Pc,
                                                                      float2* __restrict__ out) {
    using RP = RegPlan<NF>;
    extern __shared__ float2 sm[];
    float2* tw = sm + RP::G * fftreg::padded(NF);
    fftreg::twiddles(tw, NF);
    const int g = threadIdx.x / RP::T, tid = threadIdx.x % RP::T;
    const long long item = (long long)blockIdx.x * RP::G + g;
    const bool live = item < items;
    const long long row = live ? item / nblk : 0;
    const long long k0 = live ? (long long)(item % nblk) * M : 0;
    const float2* src = raw + row * (long long)n;
    float2 x[RP::P];
#pragma unroll
    for (int m = 0; m < RP::P; ++m) {
        const long long k = k0 + tid + RP::T * m;
        x[m] = live && k < n ? src[k] : make_float2(0.f, 0.f);
    }
    float2* rowbuf = sm + g * fftreg::padded(NF);
    fftreg::fft<NF, RP::B, true>(x, rowbuf, tw, tid);
#pragma unroll
    for (int m = 0; m < RP::P; ++m) x[m] = fftreg::cmul(x[m], Pc[tid + RP::T * m]);
    fftreg::fft<NF, RP::B, false>(x, rowbuf, tw, tid);
    float2* dst = out + row * (long long)n;
#pragma unroll
    for (int m = 0; m < RP::P; ++m) {
        const int j = tid + RP::T * m;
        const long long k = k0 + j;
        if (live && j < M && k < n) dst[k] = x[m];
    }
}

template <int NF>
cudaError_t mf_reg_launch(const float2* raw, long long rows, int n, int M, int nblk, const float2* Pc, float2* out,
                          cudaStream_t st) {
    using RP = RegPlan<NF>;
    cudaError_t e = cudaFuncSetAttribute(mf_reg_kernel<NF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)RP::SMEM);
    if (e != cudaSuccess) return e;
    const long long items = rows * nblk;
    mf_reg_kernel<NF><<<(unsigned)((items + RP::G - 1) / RP::G), RP::THREADS, RP::SMEM, st>>>(raw, n, M, nblk, items,
                                                                                             Pc, out);
    return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// whitening

// pass 1: spectra of rows blockIdx.x, blockIdx.x + gridDim.x, ... into out
__global__ void __launch_bounds__(1024) whiten_spectra_kernel(const float2* __restrict__ in, float2* __restrict__ out,
                                                              long long rows, int n) {
    extern __shared__ float2 buf[];
    float2* tw = buf + n;
    fftdev::fft_twiddles(tw, n);
    for (long long r = blockIdx.x; r < rows; r += gridDim.x) {
        for (int j = threadIdx.x; j < n; j += blockDim.x) buf[j] = in[r * n + j];
        __syncthreads();
        fft_smem(buf, tw, n, -1.f);
        for (int j = threadIdx.x; j < n; j += blockDim.x) out[r * n + j] = buf[j];
        __syncthreads();
    }
}

// Sum of |S(f)|^2 over the rows of chunk blockIdx.y: part[chunk][f].  Two
// bins a thread (16-byte loads, eight rows in flight); |S|^2 in FP32, summed
// in FP32 over runs of 32 rows, the runs added in FP64 (FP64 arithmetic is a
// small fraction of the FP32 rate on this part).  n even; VEC: S 16-byte
// aligned (else the two bins are read as two 8-byte loads).
constexpr int WP_RUN = 32;
template <bool VEC>
__device__ __forceinline__ float4 load_bins2(const float2* S, long long i) {
    if constexpr (VEC) return reinterpret_cast<const float4*>(S)[i];
    const float2 a = S[2 * i], b = S[2 * i + 1];
    return make_float4(a.x, a.y, b.x, b.y);
}

template <bool VEC>
__global__ void __launch_bounds__(256) whiten_power_kernel(const float2* __restrict__ S, long long rows, int n,
                                                           int nchunks, double* __restrict__ part) {
    const int f2 = blockIdx.x * blockDim.x + threadIdx.x;     // bins 2 f2, 2 f2 + 1
    if (2 * f2 >= n) return;
    const long long r0 = rows * blockIdx.y / nchunks, r1 = rows * (blockIdx.y + 1) / nchunks;
    const long long n2 = n / 2;
    double acc0 = 0.0, acc1 = 0.0;
    for (long long ra = r0; ra < r1; ra += WP_RUN) {
        const long long rb = ra + WP_RUN < r1 ? ra + WP_RUN : r1;
        float s0 = 0.f, s1 = 0.f;
        long long r = ra;
        for (; r + 8 <= rb; r += 8) {
            float4 v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = load_bins2<VEC>(S, (r + u) * n2 + f2);
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                s0 = fmaf(v[u].x, v[u].x, fmaf(v[u].y, v[u].y, s0));
                s1 = fmaf(v[u].z, v[u].z, fmaf(v[u].w, v[u].w, s1));
            }
        }
        for (; r < rb; ++r) {
            const float4 v = load_bins2<VEC>(S, r * n2 + f2);
            s0 = fmaf(v.x, v.x, fmaf(v.y, v.y, s0));
            s1 = fmaf(v.z, v.z, fmaf(v.w, v.w, s1));
        }
        acc0 += (double)s0;
        acc1 += (double)s1;
    }
    part[(size_t)blockIdx.y * n + 2 * f2] = acc0;
    part[(size_t)blockIdx.y * n + 2 * f2 + 1] = acc1;
}

// P(f) = sum over the chunks in order / rows
__global__ void whiten_reduce_kernel(const double* __restrict__ part, int nparts, int n, long long rows,
                                     double* __restrict__ P) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= n) return;
    double s = 0.0;
    for (int b = 0; b < nparts; ++b) s += part[(size_t)b * n + f];
    P[f] = s / (double)rows;
}

// one CTA: stats = {gamma mean_f P + min_f P} (the numerator of G / max G)
__global__ void __launch_bounds__(1024) whiten_stats_kernel(const double* __restrict__ P, int n, double gamma,
                                                            double* __restrict__ stats) {
    __shared__ double red[32], mn[32];
    double s = 0.0, pmin = 1.0 / 0.0;
    for (int f = threadIdx.x; f < n; f += blockDim.x) {
        s += P[f];
        pmin = fmin(pmin, P[f]);
    }
    for (int o = 16; o; o >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, o);
        pmin = fmin(pmin, __shfl_xor_sync(0xffffffffu, pmin, o));
    }
    if ((threadIdx.x & 31) == 0) {
        red[threadIdx.x >> 5] = s;
        mn[threadIdx.x >> 5] = pmin;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0, m = 1.0 / 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            t += red[w];
            m = fmin(m, mn[w]);
        }
        stats[0] = gamma * (t / (double)n);
        stats[1] = stats[0] + m;
    }
}

// gain(f) = sqrt(G(f) / max G) = sqrt((gamma Pbar + Pmin) / (gamma Pbar + P(f)))
__global__ void whiten_gain_kernel(const double* __restrict__ P, int n, const double* __restrict__ stats,
                                   float* __restrict__ gain) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= n) return;
    gain[f] = (float)sqrt(stats[1] / (stats[0] + P[f]));
}

// pass 2: out[r] = IFFT(out[r] * gain) (the spectra from pass 1)
__global__ void __launch_bounds__(1024) whiten_apply_kernel(float2* __restrict__ out, long long rows, int n, const float* __restrict__ gain) {
    extern __shared__ float2 buf[];
    float2* tw = buf + n;
    fftdev::fft_twiddles(tw, n);
    const float inv = 1.f / (float)n;
    for (long long r = blockIdx.x; r < rows; r += gridDim.x) {
        for (int j = threadIdx.x; j < n; j += blockDim.x) {
            const float2 v = out[r * n + j];
            const float g = gain[j];
            buf[j] = make_float2(v.x * g, v.y * g);
        }
        __syncthreads();
        fft_smem(buf, tw, n, 1.f);
        for (int j = threadIdx.x; j < n; j += blockDim.x) out[r * n + j] = make_float2(buf[j].x * inv, buf[j].y * inv);
        __syncthreads();
    }
}

// Register-FFT forms of the two whitening passes for n >= 256: groups of
// threads hold a row in registers (see RegPlan); the CTAs stride over groups
// of G rows.  Pass 1 writes the spectra; pass 2 reads them, applies the gain
// and writes IFFT / n.
template <int N>
__global__ void __launch_bounds__(RegPlan<N>::THREADS, RegPlan<N>::MINB) whiten_spectra_reg_kernel(const float2* __restrict__ in,
                                                                                 float2* __restrict__ out,
                                                                                 long long rows) {
    using RP = RegPlan<N>;
    extern __shared__ float2 sm[];
    float2* tw = sm + RP::G * fftreg::padded(N);
    fftreg::twiddles(tw, N);
    const int g = threadIdx.x / RP::T, tid = threadIdx.x % RP::T;
    float2* rowbuf = sm + g * fftreg::padded(N);
    for (long long r0 = (long long)blockIdx.x * RP::G; r0 < rows; r0 += (long long)gridDim.x * RP::G) {
        const long long r = r0 + g;
        const bool live = r < rows;
        const float2* src = in + (live ? r : 0) * N;
        float2 x[RP::P];
#pragma unroll
        for (int m = 0; m < RP::P; ++m) x[m] = src[tid + RP::T * m];
        fftreg::fft<N, RP::B, true>(x, rowbuf, tw, tid);
        if (live) {
#pragma unroll
            for (int m = 0; m < RP::P; ++m) out[r * N + tid + RP::T * m] = x[m];
        }
    }
}

template <int N>
__global__ void __launch_bounds__(RegPlan<N>::THREADS, RegPlan<N>::MINB) whiten_apply_reg_kernel(float2* __restrict__ out,
                                                                               long long rows,
                                                                               const float* __restrict__ gain) {
    using RP = RegPlan<N>;
    extern __shared__ float2 sm[];
    float2* tw = sm + RP::G * fftreg::padded(N);
    fftreg::twiddles(tw, N);
    const int g = threadIdx.x / RP::T, tid = threadIdx.x % RP::T;
    float2* rowbuf = sm + g * fftreg::padded(N);
    const float inv = 1.f / (float)N;
    for (long long r0 = (long long)blockIdx.x * RP::G; r0 < rows; r0 += (long long)gridDim.x * RP::G) {
        const long long r = r0 + g;
        const bool live = r < rows;
        float2* row = out + (live ? r : 0) * N;
        float2 x[RP::P];
#pragma unroll
        for (int m = 0; m < RP::P; ++m) {
            const float2 v = row[tid + RP::T * m];
            const float gg = gain[tid + RP::T * m];
            x[m] = make_float2(v.x * gg, v.y * gg);
        }
        fftreg::fft<N, RP::B, false>(x, rowbuf, tw, tid);
        if (live) {
#pragma unroll
            for (int m = 0; m < RP::P; ++m) row[tid + RP::T * m] = make_float2(x[m].x * inv, x[m].y * inv);
        }
    }
}

template <int N>
cudaError_t whiten_reg_launch(bool apply, const float2* in, float2* out, long long rows, const float* gain,
                              cudaStream_t st) {
    using RP = RegPlan<N>;
    const long long groups = (rows + RP::G - 1) / RP::G;
    if (!apply) {
        cudaError_t e = cudaFuncSetAttribute(whiten_spectra_reg_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)RP::SMEM);
        if (e != cudaSuccess) return e;
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, whiten_spectra_reg_kernel<N>, RP::THREADS, RP::SMEM);
        if (e != cudaSuccess) return e;
        const long long grid = std::min<long long>(groups, (long long)std::max(per_sm, 1) * sm_count());
        whiten_spectra_reg_kernel<N><<<(unsigned)grid, RP::THREADS, RP::SMEM, st>>>(in, out, rows);
    } else {
        cudaError_t e = cudaFuncSetAttribute(whiten_apply_reg_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)RP::SMEM);
        if (e != cudaSuccess) return e;
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, whiten_apply_reg_kernel<N>, RP::THREADS, RP::SMEM);
        if (e != cudaSuccess) return e;
        const long long grid = std::min<long long>(groups, (long long)std::max(per_sm, 1) * sm_count());
        whiten_apply_reg_kernel<N><<<(unsigned)grid, RP::THREADS, RP::SMEM, st>>>(out, rows, gain);
    }
    return cudaGetLastError();
}

// the register path for n in [256, 16384] (false: n outside it)
bool whiten_reg_dispatch(int n, bool apply, const float2* in, float2* out, long long rows, const float* gain,
                         cudaStream_t st, cudaError_t* err) {
    switch (n) {
        case 256: *err = whiten_reg_launch<256>(apply, in, out, rows, gain, st); return true;
        case 512: *err = whiten_reg_launch<512>(apply, in, out, rows, gain, st); return true;
        case 1024: *err = whiten_reg_launch<1024>(apply, in, out, rows, gain, st); return true;
        case 2048: *err = whiten_reg_launch<2048>(apply, in, out, rows, gain, st); return true;
        case 4096: *err = whiten_reg_launch<4096>(apply, in, out, rows, gain, st); return true;
        case 8192: *err = whiten_reg_launch<8192>(apply, in, out, rows, gain, st); return true;
        case 16384: *err = whiten_reg_launch<16384>(apply, in, out, rows, gain, st); return true;
        default: return false;
    }
}

// ----------------------------------------------------------------------------
// TVG: both middle order statistics of the FP32 power of every column of
// e [rows][n], by a three-level radix select on the bit patterns (as for DRC
// below): level 1 on the top 12 bits (1/8-octave bins), levels 2 and 3 on the
// next 10 bits of the values matching each rank's chosen prefix: three reads
// of the echo.  One CTA per strip of TVG_COLS columns, its histograms (2048
// bins a column at level 1, 2 x 1024 at levels 2 and 3) in shared memory;
// thread t reads column t mod TVG_COLS of rows t / TVG_COLS + k TVG_RPI, eight
// rows in flight.
constexpr int TVG_COLS = 8;
constexpr int TVG_THREADS = 256;
constexpr int TVG_RPI = TVG_THREADS / TVG_COLS;   // rows an iteration reads
constexpr size_t TVG_SMEM = sizeof(unsigned) * TVG_COLS * 2048;

__device__ __forceinline__ unsigned tvg_bits(float2 v) {
    return min(__float_as_uint(power_f32(v)), 0x7fffffffu);   // a NaN with the sign bit: the largest NaN
}

// One level over the strip: every value of column c whose bits >> PSH equal
// that rank's prefix >> PSH adds to bin (bits >> BSH) & (NB - 1) of h[r][c].
// (rows: the rows the select sees, physical rows 0, rstep, 2 rstep, ...)
template <int LEVEL>
__device__ __forceinline__ void tvg_level(const float2* __restrict__ e, long long rows, long long rstep, int n, int col,
                                          bool colok, unsigned* h, const unsigned* prefix) {
    constexpr int NB = LEVEL == 1 ? 2048 : 1024, BSH = LEVEL == 1 ? 20 : (LEVEL == 2 ? 10 : 0);
    constexpr int PSH = LEVEL == 2 ? 20 : 10;
    const int c = threadIdx.x % TVG_COLS;
    unsigned p0 = 0u, p1 = 0u;
    if (LEVEL > 1) {
        p0 = prefix[2 * c] >> PSH;
        p1 = prefix[2 * c + 1] >> PSH;
    }
    unsigned* h0 = h + (LEVEL == 1 ? c * NB : (2 * c) * NB);
    unsigned* h1 = h0 + NB;
    auto add = [&](unsigned bits) {
        const unsigned k = (bits >> BSH) & (NB - 1);
        if (LEVEL == 1) {
            atomicAdd(&h0[k], 1u);
        } else {
            if ((bits >> PSH) == p0) atomicAdd(&h0[k], 1u);
            if ((bits >> PSH) == p1) atomicAdd(&h1[k], 1u);
        }
    };
    if (!colok) return;
    const long long r0 = threadIdx.x / TVG_COLS;
    long long r = r0;
    for (; r + 7 * TVG_RPI < rows; r += 8 * TVG_RPI) {
        float2 v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = e[(r + u * TVG_RPI) * rstep * n + col];
#pragma unroll
        for (int u = 0; u < 8; ++u) add(tvg_bits(v[u]));
    }
    for (; r < rows; r += TVG_RPI) add(tvg_bits(e[r * rstep * n + col]));
}

// The bins of every (column, rank) holding the rank's residual: one warp per
// (column, rank) pair, the lanes summing 32-bin slices and scanning.
template <int LEVEL>
__device__ __forceinline__ void tvg_pick(const unsigned* h, unsigned* prefix, unsigned* rank) {
    constexpr int NB = LEVEL == 1 ? 2048 : 1024, PER = NB / 32, SH = LEVEL == 1 ? 20 : (LEVEL == 2 ? 10 : 0);
    const int lane = threadIdx.x & 31;
    for (int pr = threadIdx.x >> 5; pr < 2 * TVG_COLS; pr += TVG_THREADS / 32) {
        const int c = pr >> 1;
        const unsigned* hh = h + (LEVEL == 1 ? c * NB : pr * NB);   // level 1: one histogram a column
        const unsigned rk = rank[pr];
        unsigned tot = 0u;
        for (int k = 0; k < PER; ++k) tot += hh[lane * PER + k];
        unsigned x = tot;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        unsigned below = x - tot;
        const bool mine = rk >= below && rk - below < tot;
        unsigned bin = 0u, before = 0u;
        if (mine) {
            for (int k = 0; k < PER; ++k) {
                const unsigned hk = hh[lane * PER + k];
                if (rk - below < hk) {
                    bin = lane * PER + k;
                    before = below;
                    break;
                }
                below += hk;
            }
        }
        const unsigned who = __ballot_sync(0xffffffffu, mine);
        const int src = who ? __ffs(who) - 1 : 0;
        bin = __shfl_sync(0xffffffffu, bin, src);
        before = __shfl_sync(0xffffffffu, before, src);
        if (lane == 0) {
            rank[pr] = rk - before;
            prefix[pr] |= bin << SH;
        }
    }
}

// Two order statistics (ranks r_lo <= r_hi) of every column of the strip, over
// rows 0, rstep, 2 rstep, ... (rows of them).  Writes the midpoint of the
// two (the median when the ranks are the middle ones) to med, or, with
// bracket set, their bit patterns.
__global__ void __launch_bounds__(TVG_THREADS, 2) tvg_select_kernel(const float2* __restrict__ e, long long rows,
                                                                   long long rstep, int n, unsigned r_lo,
                                                                   unsigned r_hi, double* __restrict__ med,
                                                                   uint2* __restrict__ bracket) {
    extern __shared__ unsigned tvg_h[];                       // TVG_COLS x 2048 counters
    __shared__ unsigned prefix[2 * TVG_COLS], rank[2 * TVG_COLS];   // index 2 c + r
    const int col = blockIdx.x * TVG_COLS + (int)(threadIdx.x % TVG_COLS);
    const bool colok = col < n;
    if (threadIdx.x < 2 * TVG_COLS) {
        prefix[threadIdx.x] = 0u;
        rank[threadIdx.x] = (threadIdx.x & 1) ? r_hi : r_lo;
    }
    for (int t = threadIdx.x; t < TVG_COLS * 2048; t += TVG_THREADS) tvg_h[t] = 0u;
    __syncthreads();
    tvg_level<1>(e, rows, rstep, n, col, colok, tvg_h, prefix);
    __syncthreads();
    tvg_pick<1>(tvg_h, prefix, rank);
    __syncthreads();
    for (int t = threadIdx.x; t < TVG_COLS * 2048; t += TVG_THREADS) tvg_h[t] = 0u;
    __syncthreads();
    tvg_level<2>(e, rows, rstep, n, col, colok, tvg_h, prefix);
    __syncthreads();
    tvg_pick<2>(tvg_h, prefix, rank);
    __syncthreads();
    for (int t = threadIdx.x; t < TVG_COLS * 2048; t += TVG_THREADS) tvg_h[t] = 0u;
    __syncthreads();
    tvg_level<3>(e, rows, rstep, n, col, colok, tvg_h, prefix);
    __syncthreads();
    tvg_pick<3>(tvg_h, prefix, rank);
    __syncthreads();
    if (threadIdx.x < TVG_COLS && blockIdx.x * TVG_COLS + (int)threadIdx.x < n) {
        const int c = threadIdx.x, gc = blockIdx.x * TVG_COLS + c;
        if (bracket) {
            bracket[gc] = make_uint2(prefix[2 * c], prefix[2 * c + 1]);
        } else {
            const float lo = __uint_as_float(prefix[2 * c]), hi = __uint_as_float(prefix[2 * c + 1]);
            med[gc] = 0.5 * ((double)lo + (double)hi);
        }
    }
}

// Bracketed select (large row counts).  An exact select on every rstep-th row
// gives each column a bracket [lo, hi] (bit patterns) that holds the column's
// middle order statistics with overwhelming probability; one pass over all
// rows counts the values below lo and collects those inside the bracket
// (at most TVG_CAP a column); a block per column then selects both middle
// ranks among the collected values.  A column whose bracket misses a middle
// rank, or whose collection overflowed, is flagged and selected again over
// all its rows by a block of its own (the three radix levels), so the result
// is exact in every case.
constexpr int TVG_CAP = 8192;
constexpr long long TVG_BRACKET_MIN_ROWS = 16384;   // fewer rows: the three-level select directly
constexpr long long TVG_SAMPLE = 2048;              // rows of the sample (about)

__global__ void __launch_bounds__(TVG_THREADS) tvg_collect_kernel(const float2* __restrict__ e, long long rows, int n,
                                                                  const uint2* __restrict__ bracket,
                                                                  unsigned* __restrict__ cand,
                                                                  unsigned* __restrict__ below,
                                                                  unsigned* __restrict__ nin) {
    __shared__ unsigned s_cnt[TVG_COLS], s_below[TVG_COLS];
    const int c = threadIdx.x % TVG_COLS, col = blockIdx.x * TVG_COLS + c;
    if (threadIdx.x < TVG_COLS) s_cnt[threadIdx.x] = s_below[threadIdx.x] = 0u;
    __syncthreads();
    if (col < n) {
        const uint2 br = bracket[col];
        unsigned* cc = cand + (size_t)col * TVG_CAP;
        unsigned nb = 0u;
        auto put = [&](unsigned bits) {
            if (bits < br.x) {
                ++nb;
            } else if (bits <= br.y) {
                const unsigned pos = atomicAdd(&s_cnt[c], 1u);
                if (pos < (unsigned)TVG_CAP) cc[pos] = bits;
            }
        };
        long long r = threadIdx.x / TVG_COLS;
        for (; r + 7 * TVG_RPI < rows; r += 8 * TVG_RPI) {
            float2 v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = e[(r + u * TVG_RPI) * n + col];
#pragma unroll
            for (int u = 0; u < 8; ++u) put(tvg_bits(v[u]));
        }
        for (; r < rows; r += TVG_RPI) put(tvg_bits(e[r * n + col]));
        atomicAdd(&s_below[c], nb);
    }
    __syncthreads();
    if (threadIdx.x < TVG_COLS && blockIdx.x * TVG_COLS + (int)threadIdx.x < n) {
        below[blockIdx.x * TVG_COLS + threadIdx.x] = s_below[threadIdx.x];
        nin[blockIdx.x * TVG_COLS + threadIdx.x] = s_cnt[threadIdx.x];
    }
}

// One radix level's pick for a block selecting two ranks of one column: warp
// r (r = 0, 1) finds the bin of h holding rank r's residual (level 0: one
// histogram of NB bins for both; later levels: 1024 bins per rank at h + 1024 r),
// appends it to pre[r] at bit SH and keeps the rank within the bin.
__device__ void tvg_block_pick(const unsigned* h, int L, int NB, int SH, unsigned* pre, unsigned* rk) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (wid >= 2) return;
    const unsigned* hh = h + (L == 0 ? 0 : wid * 1024);
    const int PER = NB / 32;
    const unsigned want = rk[wid];
    unsigned tot = 0u;
    for (int k = 0; k < PER; ++k) tot += hh[lane * PER + k];
    unsigned x = tot;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    unsigned bl = x - tot, bin = 0u, before = 0u;
    const bool mine = want >= bl && want - bl < tot;
    if (mine) {
        for (int k = 0; k < PER; ++k) {
            const unsigned hk = hh[lane * PER + k];
            if (want - bl < hk) {
                bin = lane * PER + k;
                before = bl;
                break;
            }
            bl += hk;
        }
    }
    const unsigned who = __ballot_sync(0xffffffffu, mine);
    const int src = who ? __ffs(who) - 1 : 0;
    bin = __shfl_sync(0xffffffffu, bin, src);
    before = __shfl_sync(0xffffffffu, before, src);
    if (lane == 0) {
        rk[wid] = want - before;
        pre[wid] |= bin << SH;
    }
}

// One column per block: checks the bracket and selects both middle ranks
// among its collected values (three radix levels on the bit patterns, as
// above), else flags the column.
__global__ void __launch_bounds__(256) tvg_bracket_select_kernel(const unsigned* __restrict__ cand,
                                                                 const unsigned* __restrict__ below,
                                                                 const unsigned* __restrict__ nin, long long rows,
                                                                 double* __restrict__ med, int* __restrict__ flags) {
    __shared__ unsigned v[TVG_CAP];
    __shared__ unsigned h[2048];     // level 0: one histogram of 2048 bins; levels 1, 2: one of 1024 per rank
    __shared__ unsigned pre[2], rk[2];
    const int col = blockIdx.x;
    const unsigned nb = below[col], ni = nin[col];
    const unsigned R0 = (unsigned)((rows - 1) / 2), R1 = (unsigned)(rows / 2);
    const bool ok = ni <= (unsigned)TVG_CAP && nb <= R0 && R1 < nb + ni;
    if (threadIdx.x == 0) flags[col] = ok ? 0 : 1;
    if (!ok) return;
    for (unsigned t = threadIdx.x; t < ni; t += blockDim.x) v[t] = cand[(size_t)col * TVG_CAP + t];
    if (threadIdx.x < 2) {
        pre[threadIdx.x] = 0u;
        rk[threadIdx.x] = (threadIdx.x ? R1 : R0) - nb;
    }
#pragma unroll 1
    for (int L = 0; L < 3; ++L) {
        const int NB = L == 0 ? 2048 : 1024, SH = L == 0 ? 20 : (L == 1 ? 10 : 0), PSH = L == 1 ? 20 : 10;
        for (int t = threadIdx.x; t < 2048; t += blockDim.x) h[t] = 0u;
        __syncthreads();
        const unsigned p0 = pre[0] >> PSH, p1 = pre[1] >> PSH;
        for (unsigned t = threadIdx.x; t < ni; t += blockDim.x) {
            const unsigned b = v[t], k = (b >> SH) & (unsigned)(NB - 1);
            if (L == 0 || (b >> PSH) == p0) atomicAdd(&h[k], 1u);
            if (L > 0 && (b >> PSH) == p1) atomicAdd(&h[1024 + k], 1u);
        }
        __syncthreads();
        tvg_block_pick(h, L, NB, SH, pre, rk);
        __syncthreads();
    }
    if (threadIdx.x == 0) med[col] = 0.5 * ((double)__uint_as_float(pre[0]) + (double)__uint_as_float(pre[1]));
}

// The exact select of a flagged column over all its rows, one block per
// column (columns not flagged return at once): the three radix levels, each
// thread reading every 256th row, eight rows in flight.
__global__ void __launch_bounds__(256) tvg_column_select_kernel(const float2* __restrict__ e, long long rows, int n,
                                                                const int* __restrict__ flags,
                                                                double* __restrict__ med) {
    const int col = blockIdx.x;
    if (!flags[col]) return;
    __shared__ unsigned h[2048];
    __shared__ unsigned pre[2], rk[2];
    if (threadIdx.x < 2) {
        pre[threadIdx.x] = 0u;
        rk[threadIdx.x] = (unsigned)(threadIdx.x ? rows / 2 : (rows - 1) / 2);
    }
#pragma unroll 1
    for (int L = 0; L < 3; ++L) {
        const int NB = L == 0 ? 2048 : 1024, SH = L == 0 ? 20 : (L == 1 ? 10 : 0), PSH = L == 1 ? 20 : 10;
        for (int t = threadIdx.x; t < 2048; t += blockDim.x) h[t] = 0u;
        __syncthreads();
        const unsigned p0 = pre[0] >> PSH, p1 = pre[1] >> PSH;
        auto add = [&](unsigned b) {
            const unsigned k = (b >> SH) & (unsigned)(NB - 1);
            if (L == 0 || (b >> PSH) == p0) atomicAdd(&h[k], 1u);
            if (L > 0 && (b >> PSH) == p1) atomicAdd(&h[1024 + k], 1u);
        };
        long long r = threadIdx.x;
        for (; r + 7 * 256 < rows; r += 8 * 256) {
            float2 v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = e[(r + u * 256) * n + col];
#pragma unroll
            for (int u = 0; u < 8; ++u) add(tvg_bits(v[u]));
        }
        for (; r < rows; r += 256) add(tvg_bits(e[r * n + col]));
        __syncthreads();
        tvg_block_pick(h, L, NB, SH, pre, rk);
        __syncthreads();
    }
    if (threadIdx.x == 0) med[col] = 0.5 * ((double)__uint_as_float(pre[0]) + (double)__uint_as_float(pre[1]));
}

// Every block forms the mean of the medians (the same sum in the same order:
// the result does not depend on the block) and the gains of its 256 columns:
// the FP64 square roots and divisions spread over the SMs.
__global__ void __launch_bounds__(256) tvg_gain_kernel(const double* __restrict__ med, int n, double alpha,
                                                       float* __restrict__ gain) {
    __shared__ double red[256];
    double s = 0.0;
    for (int t = threadIdx.x; t < n; t += blockDim.x) s += med[t];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    const double pbar = red[0] / (double)n;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) {
        const double den = alpha * pbar + med[t];
        gain[t] = den > 0.0 ? (float)sqrt(1.0 / den) : 1.f;    // silent median, alpha = 0: no correction
    }
}

// out[r][c] = in[r][c] gain[c]: thread = column (its gain in a register),
// rows blockIdx.y, blockIdx.y + gridDim.y, ..., four in flight
__global__ void scale_columns_kernel(const float2* __restrict__ in, float2* __restrict__ out, long long rows, int n,
                                     const float* __restrict__ gain) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    const float g = gain[c];
    const long long step = gridDim.y;
    long long r = blockIdx.y;
    for (; r + 3 * step < rows; r += 4 * step) {
        float2 v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = in[(r + u * step) * n + c];
#pragma unroll
        for (int u = 0; u < 4; ++u) out[(r + u * step) * n + c] = make_float2(v[u].x * g, v[u].y * g);
    }
    for (; r < rows; r += step) {
        const float2 v = in[r * n + c];
        out[r * n + c] = make_float2(v.x * g, v.y * g);
    }
}

// ----------------------------------------------------------------------------
// DRC: magnitude, maximum and the two middle order statistics of |I| by a
// three-level radix select on the FP32 bit patterns (non-negative floats order
// like their bits): level 1 the top 12 bits (sign, exponent and 3 mantissa
// bits: 1/8-octave bins, so the magnitudes of a speckled image spread over many
// bins), level 2 the next 10 bits of the pixels in the two chosen level-1
// bins, level 3 the last 10 bits of those matching the chosen 22-bit
// prefixes.  Both ranks (npix - 1) / 2 and npix / 2 are selected together.

constexpr int DRC_NB1 = 2048;   // bits >> 20 of a non-negative float
constexpr int DRC_NB = 1024;    // levels 2 and 3
constexpr int DRC_T = 256;      // threads of the magnitude, level and map kernels

struct DrcState {
    unsigned maxbits;        // max |I| (FP32 bits)
    unsigned done[3];        // blocks finished, per level
    unsigned rank[2];        // rank still to find within the chosen prefix
    unsigned prefix[2];      // bits chosen so far, per middle rank
    unsigned hist1[DRC_NB1];
    unsigned hist2[2][DRC_NB];
    unsigned hist3[2][DRC_NB];
};

__global__ void __launch_bounds__(1024) drc_init_kernel(DrcState* st, long long npix) {
    unsigned* w = reinterpret_cast<unsigned*>(st);
    for (int i = threadIdx.x; i < (int)(sizeof(DrcState) / sizeof(unsigned)); i += blockDim.x) w[i] = 0u;
    if (threadIdx.x == 0) {
        st->rank[0] = (unsigned)((npix - 1) / 2);
        st->rank[1] = (unsigned)(npix / 2);
    }
}

// For each middle rank r, the bin of `hist` (this level's histogram for r)
// that holds its residual rank: the bin is appended to the prefix (shifted by
// `shift`) and the rank within the bin is kept.  Run by the last block of a
// level kernel (DRC_T threads) once every block's counts are in; the counts
// other blocks added are read from L2.
template <int NB>
__device__ void drc_pick(DrcState* st, const unsigned* hist0, const unsigned* hist1, int shift) {
    constexpr int PER = NB / DRC_T, NW = DRC_T / 32;
    __shared__ unsigned wsum[NW];
    __shared__ unsigned pick_bin[2], pick_below[2];
    if (threadIdx.x < 2) pick_bin[threadIdx.x] = pick_below[threadIdx.x] = 0u;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int r = 0; r < 2; ++r) {
        const unsigned* hist = r ? hist1 : hist0;
        const unsigned rk = __ldcg(&st->rank[r]);
        unsigned c[PER], tot = 0u;
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            c[k] = __ldcg(&hist[threadIdx.x * PER + k]);
            tot += c[k];
        }
        unsigned x = tot;                                   // inclusive scan over the warp
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[wid] = x;
        __syncthreads();
        unsigned below = x - tot;                           // pixels in the bins before this thread's
        for (int w = 0; w < wid; ++w) below += wsum[w];
        if (rk >= below && rk - below < tot) {              // exactly one thread
#pragma unroll
            for (int k = 0; k < PER; ++k) {
                if (rk - below < c[k]) {
                    pick_bin[r] = threadIdx.x * PER + k;
                    pick_below[r] = below;
                    break;
                }
                below += c[k];
            }
        }
        __syncthreads();
    }
    if (threadIdx.x < 2) {
        const int r = threadIdx.x;
        st->rank[r] = __ldcg(&st->rank[r]) - pick_below[r];
        st->prefix[r] = __ldcg(&st->prefix[r]) | (pick_bin[r] << shift);
    }
}

// Adds a block's shared histogram (n bins) to the global one; returns true in
// the last block of the grid to finish, after which every block's counts are
// visible to it.
__device__ bool drc_flush(const unsigned* h, unsigned* g, int n, unsigned* done) {
    __shared__ bool last;
    __syncthreads();
    for (int t = threadIdx.x; t < n; t += blockDim.x)
        if (h[t]) atomicAdd(&g[t], h[t]);
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (last) __threadfence();
    return last;
}

// Level 1: |I| (correctly rounded), its maximum and the histogram of the top
// 12 bits; the last block picks the level-1 bins.  A NaN with the sign bit set
// (only a NaN can have it) is stored as the largest positive NaN, so that
// every bit pattern the levels see is below 2^31.
__device__ __forceinline__ float drc_magnitude(float2 v) {
    return __uint_as_float(min(__float_as_uint(__fsqrt_rn(power_f32(v))), 0x7fffffffu));
}

__global__ void __launch_bounds__(DRC_T) drc_mag_kernel(const float2* __restrict__ img, long long npix,
                                                        float* __restrict__ mag, DrcState* st) {
    __shared__ unsigned h[DRC_NB1];
    for (int t = threadIdx.x; t < DRC_NB1; t += blockDim.x) h[t] = 0u;
    __syncthreads();
    unsigned mx = 0u;
    const long long stride = (long long)gridDim.x * blockDim.x;
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    for (; i + 3 * stride < npix; i += 4 * stride) {     // four independent loads in flight
        float2 v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = img[i + u * stride];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const float m = drc_magnitude(v[u]);
            mag[i + u * stride] = m;
            const unsigned bits = __float_as_uint(m);
            mx = max(mx, bits);
            atomicAdd(&h[bits >> 20], 1u);
        }
    }
    for (; i < npix; i += stride) {
        const float m = drc_magnitude(img[i]);
        mag[i] = m;
        const unsigned bits = __float_as_uint(m);
        mx = max(mx, bits);
        atomicAdd(&h[bits >> 20], 1u);
    }
    for (int o = 16; o; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) atomicMax(&st->maxbits, mx);
    if (drc_flush(h, st->hist1, DRC_NB1, &st->done[0])) drc_pick<DRC_NB1>(st, st->hist1, st->hist1, 20);
}

// Levels 2 and 3: the pixels whose top bits match a rank's chosen prefix
// (level 2: bits >> 20, level 3: bits >> 10) are histogrammed on the next 10
// bits, one histogram per middle rank; the last block picks the bins, and at
// level 3, where the two order statistics are complete, derives q (Eq. 12)
// from their mean: stats = {q, median of I_n, max |I|}.
template <int LEVEL>
__global__ void __launch_bounds__(DRC_T) drc_level_kernel(const float* __restrict__ mag, long long npix,
                                                          DrcState* st, double b, double* __restrict__ stats) {
    constexpr int SH = LEVEL == 2 ? 20 : 10;
    __shared__ unsigned h[2][DRC_NB];
    for (int t = threadIdx.x; t < 2 * DRC_NB; t += blockDim.x) (&h[0][0])[t] = 0u;
    __syncthreads();
    const unsigned p0 = st->prefix[0] >> SH, p1 = st->prefix[1] >> SH;
    auto add = [&](unsigned bits) {
        const unsigned k = (bits >> (SH - 10)) & (DRC_NB - 1);
        if ((bits >> SH) == p0) atomicAdd(&h[0][k], 1u);
        if ((bits >> SH) == p1) atomicAdd(&h[1][k], 1u);
    };
    // mag is the 256-byte aligned scratch: quads of pixels, two in flight
    const float4* m4 = reinterpret_cast<const float4*>(mag);
    const long long n4 = npix >> 2, stride = (long long)gridDim.x * blockDim.x;
    long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    for (; j + stride < n4; j += 2 * stride) {
        const float4 v = m4[j], w = m4[j + stride];
        add(__float_as_uint(v.x)); add(__float_as_uint(v.y)); add(__float_as_uint(v.z)); add(__float_as_uint(v.w));
        add(__float_as_uint(w.x)); add(__float_as_uint(w.y)); add(__float_as_uint(w.z)); add(__float_as_uint(w.w));
    }
    if (j < n4) {
        const float4 v = m4[j];
        add(__float_as_uint(v.x)); add(__float_as_uint(v.y)); add(__float_as_uint(v.z)); add(__float_as_uint(v.w));
    }
    for (long long i = 4 * n4 + blockIdx.x * (long long)blockDim.x + threadIdx.x; i < npix; i += stride)
        add(__float_as_uint(mag[i]));
    unsigned* g = LEVEL == 2 ? &st->hist2[0][0] : &st->hist3[0][0];
    if (!drc_flush(&h[0][0], g, 2 * DRC_NB, &st->done[LEVEL - 1])) return;
    drc_pick<DRC_NB>(st, g, g + DRC_NB, SH - 10);
    if (LEVEL == 3) {
        __syncthreads();
        if (threadIdx.x == 0) {
            const float M = __uint_as_float(__ldcg(&st->maxbits));
            const float lo = __uint_as_float(__ldcg(&st->prefix[0])), hi = __uint_as_float(__ldcg(&st->prefix[1]));
            const double med = 0.5 * ((double)__fdiv_rn(lo, M) + (double)__fdiv_rn(hi, M));
            // Eq. 12 has no value at a median of 1 (all pixels at the maximum:
            // identity map) or 0 (q -> infinity: every non-zero pixel maps to 1)
            stats[0] = med >= 1.0 ? 1.0 : (med <= 0.0 ? (1.0 / 0.0) : (b - b * med) / (med - b * med));
            stats[1] = med;
            stats[2] = (double)M;
        }
    }
}

// Eq. 11 map: I_n = |I| / max |I|, out = q I_n / ((q - 1) I_n + 1).  vec: the
// output is 16-byte aligned (quads of pixels, two in flight).
__global__ void __launch_bounds__(DRC_T) drc_map_kernel(const float* __restrict__ mag, long long npix,
                                                        const DrcState* st, const double* __restrict__ stats,
                                                        float* __restrict__ out, int vec) {
    const float M = __uint_as_float(st->maxbits);
    const float q = (float)stats[0];
    const bool qinf = isinf(stats[0]);
    auto map = [&](float m) {
        const float In = __fdiv_rn(m, M);
        return qinf ? (In > 0.f ? 1.f : 0.f) : __fdiv_rn(q * In, fmaf(q - 1.f, In, 1.f));
    };
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    long long i = t0;
    if (vec) {
        const float4* m4 = reinterpret_cast<const float4*>(mag);
        float4* o4 = reinterpret_cast<float4*>(out);
        const long long n4 = npix >> 2;
        long long j = t0;
        for (; j + stride < n4; j += 2 * stride) {
            const float4 v = m4[j], w = m4[j + stride];
            o4[j] = make_float4(map(v.x), map(v.y), map(v.z), map(v.w));
            o4[j + stride] = make_float4(map(w.x), map(w.y), map(w.z), map(w.w));
        }
        if (j < n4) {
            const float4 v = m4[j];
            o4[j] = make_float4(map(v.x), map(v.y), map(v.z), map(v.w));
        }
        i = 4 * n4 + t0;
    }
    for (; i < npix; i += stride) out[i] = map(mag[i]);
}

bool pow2_in(long long n, long long lo, long long hi) { return n >= lo && n <= hi && (n & (n - 1)) == 0; }

}  // namespace
}  // namespace sas

using namespace sas;

extern "C" int sas_matched_filter(const void* d_raw, int64_t rows, int32_t n, const void* d_replica, int32_t L,
                                  void* d_out, void* stream) {
    if (!d_raw || !d_replica || !d_out || rows < 0 || n < 1 || L < 1 || L > 4096) {
        set_error("sas_matched_filter: bad argument (1 <= L <= 4096)");
        return SAS_ERR_ARG;
    }
    if (rows == 0) return SAS_OK;
    cudaStream_t st = (cudaStream_t)stream;
    int NF = 256;
    while (NF < 4 * L && NF < fftdev::MAX_N) NF *= 2;        // at least 3/4 of each block is output
    const int M = NF - L + 1;
    const int nblk = (int)((n + M - 1) / M);
    float2* Pc = nullptr;
    SAS_CUDA(cudaMallocAsync((void**)&Pc, sizeof(float2) * NF, st));
    const int nt = fft_threads(NF);
    const size_t sm = sizeof(float2) * (NF + NF / 2);       // row + twiddles
    int rc = SAS_OK;
    cudaError_t e = cudaFuncSetAttribute(mf_replica_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e == cudaSuccess) {
        mf_replica_kernel<<<1, nt, sm, st>>>((const float2*)d_replica, L, NF, Pc);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        const float2* raw = (const float2*)d_raw;
        float2* o = (float2*)d_out;
        switch (NF) {
            case 256: e = mf_reg_launch<256>(raw, rows, n, M, nblk, Pc, o, st); break;
            case 512: e = mf_reg_launch<512>(raw, rows, n, M, nblk, Pc, o, st); break;
            case 1024: e = mf_reg_launch<1024>(raw, rows, n, M, nblk, Pc, o, st); break;
            case 2048: e = mf_reg_launch<2048>(raw, rows, n, M, nblk, Pc, o, st); break;
            case 4096: e = mf_reg_launch<4096>(raw, rows, n, M, nblk, Pc, o, st); break;
            case 8192: e = mf_reg_launch<8192>(raw, rows, n, M, nblk, Pc, o, st); break;
            default: e = mf_reg_launch<16384>(raw, rows, n, M, nblk, Pc, o, st); break;
        }
    }
    if (e != cudaSuccess) rc = cuda_fail(e, "matched filter");
    cudaFreeAsync(Pc, st);
    return rc;
}

extern "C" int sas_whiten(const void* d_in, void* d_out, int64_t rows, int32_t n, double gamma, float* d_gain,
                          void* stream) {
    if (!d_in || !d_out || rows < 1 || !pow2_in(n, 4, fftdev::MAX_N) || !(gamma >= 0.0)) {
        set_error("sas_whiten: bad argument (n a power of two in [4, 16384], gamma >= 0)");
        return SAS_ERR_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int nparts = (int)std::min<long long>(rows, 64LL);
    double* part = nullptr;
    double* P = nullptr;
    float* gain = d_gain;
    SAS_CUDA(cudaMallocAsync((void**)&part, sizeof(double) * ((size_t)nparts * n + n + 2), st));
    P = part + (size_t)nparts * n;
    double* wstats = P + n;
    float* own_gain = nullptr;
    int rc = SAS_OK;
    if (!gain) {
        cudaError_t e = cudaMallocAsync((void**)&own_gain, sizeof(float) * n, st);
        if (e != cudaSuccess) {
            cudaFreeAsync(part, st);
            return cuda_fail(e, "whitening gain");
        }
        gain = own_gain;
    }
    const int nt = fft_threads(n);
    const size_t sm = sizeof(float2) * (n + n / 2);          // row + twiddles
    cudaError_t e = cudaFuncSetAttribute(whiten_spectra_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(whiten_apply_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e == cudaSuccess &&
        !whiten_reg_dispatch(n, false, (const float2*)d_in, (float2*)d_out, rows, gain, st, &e)) {
        whiten_spectra_kernel<<<(unsigned)std::min<long long>(rows, 8LL * sm_count()), nt, sm, st>>>(
            (const float2*)d_in, (float2*)d_out, rows, n);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        const dim3 pgrid((n / 2 + 255) / 256, nparts);
        if (((uintptr_t)d_out & 15) == 0)
            whiten_power_kernel<true><<<pgrid, 256, 0, st>>>((const float2*)d_out, rows, n, nparts, part);
        else
            whiten_power_kernel<false><<<pgrid, 256, 0, st>>>((const float2*)d_out, rows, n, nparts, part);
        whiten_reduce_kernel<<<(n + 255) / 256, 256, 0, st>>>(part, nparts, n, rows, P);
        whiten_stats_kernel<<<1, 1024, 0, st>>>(P, n, gamma, wstats);
        whiten_gain_kernel<<<(n + 255) / 256, 256, 0, st>>>(P, n, wstats, gain);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && !whiten_reg_dispatch(n, true, nullptr, (float2*)d_out, rows, gain, st, &e)) {
        whiten_apply_kernel<<<(unsigned)std::min<long long>(rows, 8LL * sm_count()), nt, sm, st>>>(
            (float2*)d_out, rows, n, gain);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) rc = cuda_fail(e, "whitening");
    cudaFreeAsync(part, st);
    if (own_gain) cudaFreeAsync(own_gain, st);
    return rc;
}

extern "C" int sas_tvg(const void* d_in, void* d_out, int64_t rows, int32_t n, double alpha, float* d_gain,
                       double* d_median, void* stream) {
    if (!d_in || !d_out || rows < 1 || rows > 0x7fffffffLL || n < 1 || !(alpha >= 0.0)) {
        set_error("sas_tvg: bad argument");
        return SAS_ERR_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    double* med = d_median;
    double* own = nullptr;
    float* gain = d_gain;
    if (!med || !gain) {
        SAS_CUDA(cudaMallocAsync((void**)&own, sizeof(double) * n + sizeof(float) * n, st));
        if (!med) med = own;
        if (!gain) gain = reinterpret_cast<float*>(own + n);
    }
    cudaError_t e0 = cudaFuncSetAttribute(tvg_select_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TVG_SMEM);
    if (e0 != cudaSuccess) {
        if (own) cudaFreeAsync(own, st);
        return cuda_fail(e0, "tvg");
    }
    const unsigned strips = (unsigned)((n + TVG_COLS - 1) / TVG_COLS);
    const float2* ein = (const float2*)d_in;
    if (rows < TVG_BRACKET_MIN_ROWS) {
        tvg_select_kernel<<<strips, TVG_THREADS, TVG_SMEM, st>>>(ein, rows, 1, n, (unsigned)((rows - 1) / 2),
                                                                 (unsigned)(rows / 2), med, nullptr);
    } else {
        // the sample: every rstep-th row (m of them), its ranks m/2 -+ about four standard deviations
        const long long rstep = rows / TVG_SAMPLE, m = (rows + rstep - 1) / rstep;
        const long long d = (long long)std::ceil(2.0 * std::sqrt((double)m)) + 1;
        const unsigned k_lo = (unsigned)std::max(0LL, (m - 1) / 2 - d), k_hi = (unsigned)std::min(m - 1, m / 2 + d);
        // scratch: brackets, candidates, counts, flags
        const size_t o_c = (sizeof(uint2) * n + 255) / 256 * 256;
        const size_t o_b = o_c + sizeof(unsigned) * (size_t)n * TVG_CAP;
        const size_t o_n = o_b + sizeof(unsigned) * n, o_f = o_n + sizeof(unsigned) * n;
        char* scr = nullptr;
        cudaError_t ea = cudaMallocAsync((void**)&scr, o_f + sizeof(int) * n, st);
        if (ea != cudaSuccess) {
            if (own) cudaFreeAsync(own, st);
            return cuda_fail(ea, "tvg scratch");
        }
        uint2* br = reinterpret_cast<uint2*>(scr);
        unsigned* cand = reinterpret_cast<unsigned*>(scr + o_c);
        unsigned* nb = reinterpret_cast<unsigned*>(scr + o_b);
        unsigned* ni = reinterpret_cast<unsigned*>(scr + o_n);
        int* fl = reinterpret_cast<int*>(scr + o_f);
        tvg_select_kernel<<<strips, TVG_THREADS, TVG_SMEM, st>>>(ein, m, rstep, n, k_lo, k_hi, nullptr, br);
        tvg_collect_kernel<<<strips, TVG_THREADS, 0, st>>>(ein, rows, n, br, cand, nb, ni);
        tvg_bracket_select_kernel<<<(unsigned)n, 256, 0, st>>>(cand, nb, ni, rows, med, fl);
        tvg_column_select_kernel<<<(unsigned)n, 256, 0, st>>>(ein, rows, n, fl, med);
        cudaFreeAsync(scr, st);
    }
    tvg_gain_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(med, n, alpha, gain);
    const unsigned gx = (unsigned)((n + 255) / 256);
    const unsigned gy = (unsigned)std::max<long long>(1, std::min<long long>(rows, (16LL * sm_count() + gx - 1) / gx));
    scale_columns_kernel<<<dim3(gx, gy), 256, 0, st>>>((const float2*)d_in, (float2*)d_out, rows, n, gain);
    cudaError_t e = cudaGetLastError();
    if (own) cudaFreeAsync(own, st);
    if (e != cudaSuccess) return cuda_fail(e, "tvg");
    return SAS_OK;
}

extern "C" int sas_drc(const void* d_image, int64_t npix, double b, float* d_out, double* d_stats, void* stream) {
    if (!d_image || !d_out || npix < 1 || npix > 0xffffffffLL || !(b > 0.0 && b < 1.0)) {
        set_error("sas_drc: bad argument (0 < b < 1)");
        return SAS_ERR_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    // scratch: |I| [npix] floats, the selection state and three doubles, each
    // part starting on a 256-byte boundary
    auto up256 = [](size_t x) { return (x + 255) / 256 * 256; };
    const size_t off_ds = up256(sizeof(float) * (size_t)npix);
    const size_t off_st = up256(off_ds + sizeof(DrcState));
    char* scratch = nullptr;
    SAS_CUDA(cudaMallocAsync((void**)&scratch, off_st + 3 * sizeof(double), st));
    float* mag = reinterpret_cast<float*>(scratch);
    DrcState* ds = reinterpret_cast<DrcState*>(scratch + off_ds);
    double* stats = d_stats ? d_stats : reinterpret_cast<double*>(scratch + off_st);
    const unsigned grid = (unsigned)std::min<long long>((npix + DRC_T - 1) / DRC_T, 8LL * sm_count());
    const int vec = ((uintptr_t)d_out & 15) == 0;
    drc_init_kernel<<<1, 1024, 0, st>>>(ds, npix);
    drc_mag_kernel<<<grid, DRC_T, 0, st>>>((const float2*)d_image, npix, mag, ds);
    drc_level_kernel<2><<<grid, DRC_T, 0, st>>>(mag, npix, ds, b, stats);
    drc_level_kernel<3><<<grid, DRC_T, 0, st>>>(mag, npix, ds, b, stats);
    drc_map_kernel<<<grid, DRC_T, 0, st>>>(mag, npix, ds, stats, d_out, vec);
    const cudaError_t e = cudaGetLastError();
    cudaFreeAsync(scratch, st);
    if (e != cudaSuccess) return cuda_fail(e, "drc");
    return SAS_OK;
}
