// Data conditioning around the backprojection (Sec. II-E) and range
// compression:
//  * sas_matched_filter: correlation of raw echo rows with the transmitted
//    replica, y[k] = sum_l e[k + l] conj(p[l]) / sum_l |p[l]|^2, by
//    overlap-save with FP32 FFTs in shared memory (one CTA per block of
//    outputs of a row);
//  * sas_whiten (Eq. 9): P(f) = mean over rows of |FFT(e)|^2 (FP64 per-CTA
//    partial sums, reduced in a fixed order), G(f) = 1 / (gamma mean P + P(f)),
//    scaled so that max G = 1, applied as a power gain (rows times sqrt G);
//  * sas_tvg (Eq. 10): P(t) = median over rows of the FP32 power |e(t)|^2,
//    exact selection by a 4-pass radix select on the FP32 bit patterns per
//    32-column strip (one CTA per strip), G(t) = 1 / (alpha mean P + P(t)),
//    applied as a power gain;
//  * sas_drc (Eqs. 11-12): I_n = |I| / max |I| (FP32), the median of I_n by
//    the same radix select over the whole image, q from Eq. 12, the rational
//    map of Eq. 11.
// Medians of an even count are the FP64 mean of the two middle values.
#include "fft.cuh"
#include "sas_common.cuh"

#include <algorithm>

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

// One CTA per (row, block of M outputs): circular correlation of NF inputs.
// R4 = 1 for NF <= 4096 (NF / 4 threads, one butterfly each per stage).
template <int R4>
__global__ void __launch_bounds__(1024) mf_block_kernel(const float2* __restrict__ raw, int n, int NF, int M, int nblk,
                                const float2* __restrict__ Pc, float2* __restrict__ out) {
    extern __shared__ float2 buf[];
    float2* tw = buf + NF;
    fftdev::fft_twiddles(tw, NF);
    const long long row = blockIdx.x / nblk;
    const int b = blockIdx.x % nblk;
    const long long k0 = (long long)b * M;
    const float2* src = raw + row * (long long)n;
    for (int j = threadIdx.x; j < NF; j += blockDim.x) {
        const long long k = k0 + j;
        buf[j] = k < n ? src[k] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    fft_smem<R4>(buf, tw, NF, -1.f);
    for (int j = threadIdx.x; j < NF; j += blockDim.x) buf[j] = fftdev::cmul(buf[j], Pc[j]);
    __syncthreads();
    fft_smem<R4>(buf, tw, NF, 1.f);
    float2* dst = out + row * (long long)n;
    for (int j = threadIdx.x; j < M; j += blockDim.x) {
        const long long k = k0 + j;
        if (k < n) dst[k] = buf[j];
    }
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

// FP64 sum of |S(f)|^2 over the rows of chunk blockIdx.y: part[chunk][f]
__global__ void whiten_power_kernel(const float2* __restrict__ S, long long rows, int n, int nchunks,
                                    double* __restrict__ part) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= n) return;
    const long long r0 = rows * blockIdx.y / nchunks, r1 = rows * (blockIdx.y + 1) / nchunks;
    double acc = 0.0;
    for (long long r = r0; r < r1; ++r) {
        const float2 v = S[r * n + f];
        acc += (double)v.x * v.x + (double)v.y * v.y;
    }
    part[(size_t)blockIdx.y * n + f] = acc;
}

// P(f) = sum over CTAs in order / rows; then (one CTA) the gain sqrt(G / max G)
__global__ void whiten_reduce_kernel(const double* __restrict__ part, int nparts, int n, long long rows,
                                     double* __restrict__ P) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= n) return;
    double s = 0.0;
    for (int b = 0; b < nparts; ++b) s += part[(size_t)b * n + f];
    P[f] = s / (double)rows;
}

__global__ void whiten_gain_kernel(const double* __restrict__ P, int n, double gamma, float* __restrict__ gain) {
    __shared__ double red[1024];
    __shared__ double pmin_s[1024];
    double s = 0.0, pmin = 1.0 / 0.0;
    for (int f = threadIdx.x; f < n; f += blockDim.x) {
        s += P[f];
        pmin = fmin(pmin, P[f]);
    }
    red[threadIdx.x] = s;
    pmin_s[threadIdx.x] = pmin;
    __syncthreads();
    for (int o = blockDim.x / 2; o; o >>= 1) {
        if ((int)threadIdx.x < o) {
            red[threadIdx.x] += red[threadIdx.x + o];
            pmin_s[threadIdx.x] = fmin(pmin_s[threadIdx.x], pmin_s[threadIdx.x + o]);
        }
        __syncthreads();
    }
    const double pbar = red[0] / (double)n;
    const double gmax = 1.0 / (gamma * pbar + pmin_s[0]);
    for (int f = threadIdx.x; f < n; f += blockDim.x) gain[f] = (float)sqrt((1.0 / (gamma * pbar + P[f])) / gmax);
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

// ----------------------------------------------------------------------------
// exact selection of order statistics of non-negative FP32 values (their bit
// patterns order like the values): ranks klo <= khi, returns both values

// TVG: one CTA per strip of 32 columns of e [rows][n]; value = FP32 power.
constexpr int SEL_COLS = 32;
constexpr int SEL_THREADS = 256;

__global__ void __launch_bounds__(SEL_THREADS) tvg_median_kernel(const float2* __restrict__ e, long long rows, int n,
                                                                 double* __restrict__ med) {
    __shared__ unsigned hist[256][SEL_COLS];
    __shared__ unsigned prefix[SEL_COLS], rank_s[SEL_COLS];
    __shared__ unsigned cnt_le[SEL_COLS], min_gt[SEL_COLS];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = SEL_THREADS / 32;
    const int col = blockIdx.x * SEL_COLS + lane;
    const bool colok = col < n;
    const unsigned klo = (unsigned)((rows - 1) / 2), khi = (unsigned)(rows / 2);
    if (threadIdx.x < SEL_COLS) {
        prefix[threadIdx.x] = 0u;
        rank_s[threadIdx.x] = klo;
    }
    for (int pass = 0; pass < 4; ++pass) {
        const int shift = 24 - 8 * pass;
        for (int t = threadIdx.x; t < 256 * SEL_COLS; t += SEL_THREADS) (&hist[0][0])[t] = 0u;
        __syncthreads();
        const unsigned pre = prefix[lane];
        const unsigned himask = pass == 0 ? 0u : (0xffffffffu << (32 - 8 * pass));
        if (colok) {
            for (long long r = warp; r < rows; r += nw) {
                const unsigned bits = __float_as_uint(power_f32(e[r * n + col]));
                if ((bits & himask) == pre) atomicAdd(&hist[(bits >> shift) & 255u][lane], 1u);
            }
        }
        __syncthreads();
        if (threadIdx.x < SEL_COLS) {
            const int c = threadIdx.x;
            unsigned rk = rank_s[c], acc = 0u;
            int bsel = 255;
            for (int bb = 0; bb < 256; ++bb) {
                const unsigned h = hist[bb][c];
                if (acc + h > rk) {
                    bsel = bb;
                    break;
                }
                acc += h;
            }
            rank_s[c] = rk - acc;
            prefix[c] |= (unsigned)bsel << shift;
        }
        __syncthreads();
    }
    // the second middle value: equal to the first if enough values tie with
    // it, otherwise the smallest value above it
    if (threadIdx.x < SEL_COLS) {
        cnt_le[threadIdx.x] = 0u;
        min_gt[threadIdx.x] = 0xffffffffu;
    }
    __syncthreads();
    const unsigned vlo = prefix[lane];
    if (colok) {
        unsigned le = 0u, mg = 0xffffffffu;
        for (long long r = warp; r < rows; r += nw) {
            const unsigned bits = __float_as_uint(power_f32(e[r * n + col]));
            if (bits <= vlo) ++le;
            else mg = min(mg, bits);
        }
        atomicAdd(&cnt_le[lane], le);
        atomicMin(&min_gt[lane], mg);
    }
    __syncthreads();
    if (threadIdx.x < SEL_COLS && blockIdx.x * SEL_COLS + (int)threadIdx.x < n) {
        const int c = threadIdx.x;
        const unsigned lo = prefix[c];
        const unsigned hi = (cnt_le[c] > khi) ? lo : min_gt[c];
        med[blockIdx.x * SEL_COLS + c] = 0.5 * ((double)__uint_as_float(lo) + (double)__uint_as_float(hi));
    }
}

__global__ void tvg_gain_kernel(const double* __restrict__ med, int n, double alpha, float* __restrict__ gain) {
    __shared__ double red[1024];
    double s = 0.0;
    for (int t = threadIdx.x; t < n; t += blockDim.x) s += med[t];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    const double pbar = red[0] / (double)n;
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
        const double den = alpha * pbar + med[t];
        gain[t] = den > 0.0 ? (float)sqrt(1.0 / den) : 1.f;    // silent median, alpha = 0: no correction
    }
}

__global__ void scale_columns_kernel(const float2* __restrict__ in, float2* __restrict__ out, long long total, int n,
                                     const float* __restrict__ gain) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const float g = gain[i % n];
        const float2 v = in[i];
        out[i] = make_float2(v.x * g, v.y * g);
    }
}

// ----------------------------------------------------------------------------
// DRC: magnitude, maximum, global radix select, map

struct DrcState {
    unsigned maxbits;       // max |I| (FP32 bits)
    unsigned prefix, rank;  // selection of rank klo
    unsigned cnt_le, min_gt;
    unsigned hist[256];
};

__global__ void drc_mag_kernel(const float2* __restrict__ img, long long npix, float* __restrict__ mag,
                               DrcState* st) {
    unsigned mx = 0u;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < npix;
         i += (long long)gridDim.x * blockDim.x) {
        const float m = __fsqrt_rn(power_f32(img[i]));
        mag[i] = m;
        mx = max(mx, __float_as_uint(m));
    }
    for (int o = 16; o; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) atomicMax(&st->maxbits, mx);
}

__global__ void drc_hist_kernel(const float* __restrict__ mag, long long npix, int pass, DrcState* st) {
    __shared__ unsigned h[256];
    for (int t = threadIdx.x; t < 256; t += blockDim.x) h[t] = 0u;
    __syncthreads();
    const int shift = 24 - 8 * pass;
    const unsigned himask = pass == 0 ? 0u : (0xffffffffu << (32 - 8 * pass));
    const unsigned pre = st->prefix;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < npix;
         i += (long long)gridDim.x * blockDim.x) {
        const unsigned bits = __float_as_uint(mag[i]);
        if ((bits & himask) == pre) atomicAdd(&h[(bits >> shift) & 255u], 1u);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < 256; t += blockDim.x)
        if (h[t]) atomicAdd(&st->hist[t], h[t]);
}

__global__ void drc_pick_kernel(int pass, DrcState* st) {
    const int shift = 24 - 8 * pass;
    unsigned rk = st->rank, acc = 0u;
    int bsel = 255;
    for (int bb = 0; bb < 256; ++bb) {
        const unsigned h = st->hist[bb];
        if (acc + h > rk) {
            bsel = bb;
            break;
        }
        acc += h;
    }
    st->rank = rk - acc;
    st->prefix |= (unsigned)bsel << shift;
    for (int bb = 0; bb < 256; ++bb) st->hist[bb] = 0u;
}

__global__ void drc_second_kernel(const float* __restrict__ mag, long long npix, DrcState* st) {
    const unsigned vlo = st->prefix;
    unsigned le = 0u, mg = 0xffffffffu;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < npix;
         i += (long long)gridDim.x * blockDim.x) {
        const unsigned bits = __float_as_uint(mag[i]);
        if (bits <= vlo) ++le;
        else mg = min(mg, bits);
    }
    for (int o = 16; o; o >>= 1) {
        le += __shfl_xor_sync(0xffffffffu, le, o);
        mg = min(mg, __shfl_xor_sync(0xffffffffu, mg, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&st->cnt_le, le);
        atomicMin(&st->min_gt, mg);
    }
}

// q from Eq. 12 on the median of I_n = |I| / max |I|; stats = {q, median, max}
__global__ void drc_q_kernel(long long npix, double b, DrcState* st, double* __restrict__ stats) {
    const unsigned long long khi = (unsigned long long)(npix / 2);
    const float M = __uint_as_float(st->maxbits);
    const float lo = __uint_as_float(st->prefix);
    const float hi = (st->cnt_le > khi) ? lo : __uint_as_float(st->min_gt);
    const double med = 0.5 * ((double)__fdiv_rn(lo, M) + (double)__fdiv_rn(hi, M));
    // Eq. 12 has no value at a median of 1 (all pixels at the maximum: identity
    // map) or 0 (q -> infinity: every non-zero pixel maps to 1)
    stats[0] = med >= 1.0 ? 1.0 : (med <= 0.0 ? (1.0 / 0.0) : (b - b * med) / (med - b * med));
    stats[1] = med;
    stats[2] = (double)M;
}

__global__ void drc_map_kernel(const float* __restrict__ mag, long long npix, const DrcState* st,
                               const double* __restrict__ stats, float* __restrict__ out) {
    const float M = __uint_as_float(st->maxbits);
    const float q = (float)stats[0];
    const bool qinf = isinf(stats[0]);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < npix;
         i += (long long)gridDim.x * blockDim.x) {
        const float In = __fdiv_rn(mag[i], M);
        out[i] = qinf ? (In > 0.f ? 1.f : 0.f) : __fdiv_rn(q * In, fmaf(q - 1.f, In, 1.f));
    }
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
    // one radix-4 butterfly per thread when NF / 4 threads fit in a block
    auto blk = NF <= 4096 ? mf_block_kernel<1> : mf_block_kernel<fftdev::R4_PER_THREAD>;
    cudaError_t e = cudaFuncSetAttribute(mf_replica_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(blk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e == cudaSuccess) {
        mf_replica_kernel<<<1, nt, sm, st>>>((const float2*)d_replica, L, NF, Pc);
        blk<<<(unsigned)(rows * nblk), nt, sm, st>>>((const float2*)d_raw, n, NF, M, nblk, Pc, (float2*)d_out);
        e = cudaGetLastError();
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
    SAS_CUDA(cudaMallocAsync((void**)&part, sizeof(double) * ((size_t)nparts * n + n), st));
    P = part + (size_t)nparts * n;
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
    if (e == cudaSuccess) {
        whiten_spectra_kernel<<<(unsigned)std::min<long long>(rows, 8LL * sm_count()), nt, sm, st>>>(
            (const float2*)d_in, (float2*)d_out, rows, n);
        whiten_power_kernel<<<dim3((n + 255) / 256, nparts), 256, 0, st>>>((const float2*)d_out, rows, n, nparts,
                                                                           part);
        whiten_reduce_kernel<<<(n + 255) / 256, 256, 0, st>>>(part, nparts, n, rows, P);
        whiten_gain_kernel<<<1, 1024, 0, st>>>(P, n, gamma, gain);
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
    tvg_median_kernel<<<(n + SEL_COLS - 1) / SEL_COLS, SEL_THREADS, 0, st>>>((const float2*)d_in, rows, n, med);
    tvg_gain_kernel<<<1, 1024, 0, st>>>(med, n, alpha, gain);
    const long long total = rows * (long long)n;
    scale_columns_kernel<<<(unsigned)std::min<long long>((total + 255) / 256, 16LL * sm_count()), 256, 0, st>>>(
        (const float2*)d_in, (float2*)d_out, total, n, gain);
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
    cudaError_t e = cudaMemsetAsync(ds, 0, sizeof(DrcState), st);
    if (e == cudaSuccess) {
        const unsigned klo = (unsigned)((npix - 1) / 2);
        e = cudaMemcpyAsync(&ds->rank, &klo, sizeof(unsigned), cudaMemcpyHostToDevice, st);
        const unsigned ones = 0xffffffffu;
        if (e == cudaSuccess) e = cudaMemcpyAsync(&ds->min_gt, &ones, sizeof(unsigned), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);   // the two host values are stack variables
    }
    if (e == cudaSuccess) {
        const unsigned grid = (unsigned)std::min<long long>((npix + 255) / 256, 8LL * sm_count());
        drc_mag_kernel<<<grid, 256, 0, st>>>((const float2*)d_image, npix, mag, ds);
        for (int pass = 0; pass < 4; ++pass) {
            drc_hist_kernel<<<grid, 256, 0, st>>>(mag, npix, pass, ds);
            drc_pick_kernel<<<1, 1, 0, st>>>(pass, ds);
        }
        drc_second_kernel<<<grid, 256, 0, st>>>(mag, npix, ds);
        drc_q_kernel<<<1, 1, 0, st>>>(npix, b, ds, stats);
        drc_map_kernel<<<grid, 256, 0, st>>>(mag, npix, ds, stats, d_out);
        e = cudaGetLastError();
    }
    cudaFreeAsync(scratch, st);
    if (e != cudaSuccess) return cuda_fail(e, "drc");
    return SAS_OK;
}
