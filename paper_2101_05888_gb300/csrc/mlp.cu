// Learned fractional-delay interpolator: an MLP 1 -> 64 -> 64 -> 8 (GELU,
// FP16-stored weights, FP32 arithmetic) mapping the fractional sample
// position f to the 8 taps at offsets -3 .. 4 from floor(u), trained to
// reproduce a 32-tap Kaiser-windowed-sinc interpolation of echo windows, then
// tabulated for the backprojection kernels (which use it through the same
// interpolator slot as the Kaiser-sinc; the paper itself names no
// interpolator).
//
// Network (x = 2 f - 1):  a1 = gelu(W1 x + b1), a2 = gelu(W2 a1 + b2), t = W3 a2 + b3,
// gelu(z) = z/2 (1 + erf(z / sqrt 2)).  Loss on windows s_b (8 complex) with
// targets y_b:  L = (1/B) sum_b |sum_m t_m(f_b) s_b,m - y_b|^2.
// With a prior (the normalised 8-tap Kaiser-sinc at beta_p) the interpolator's
// taps are prior + t: the targets are the 32-tap interpolation minus the
// prior's 8-tap interpolation of the window, and the table adds the prior.
// Parameter vector (FP32 masters): W1 [64][1], b1 [64], W2 [64][64] ([out][in]),
// b2 [64], W3 [8][64], b3 [8].
#include "sas_common.cuh"

namespace sas {
namespace {

constexpr int H = 64;
constexpr int NT = 8;
constexpr int NPAR = SAS_MLP_NPARAMS;
constexpr int O_W1 = 0, O_B1 = 64, O_W2 = 128, O_B2 = 128 + 4096, O_W3 = O_B2 + 64, O_B3 = O_W3 + 512;
static_assert(O_B3 + 8 == NPAR, "parameter layout");

constexpr int SPB = 64;      // samples per block in the loss/gradient kernel
constexpr int TPB = 256;

__device__ __forceinline__ float fp16_round(float v) { return __half2float(__float2half_rn(v)); }

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z) {
    return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * expf(-0.5f * z * z) * 0.39894228040143268f;
}

// ---------------------------------------------------------------------------
// Training windows and 32-tap Kaiser-sinc targets (FP64 weights).

__device__ double i0_series_d(double x) {
    const double q = 0.25 * x * x;
    double term = 1.0, sum = 1.0;
    for (int m = 1; m < 200; ++m) {
        term *= q / ((double)m * (double)m);
        sum += term;
        if (term < 1e-17 * sum) break;
    }
    return sum;
}

// Normalised Kaiser-windowed sinc of NTAPS taps at offsets k = 1 - NTAPS/2 .. NTAPS/2
// from floor(u), for the fraction f (FP64).
template <int NTAPS>
__device__ void kaiser_taps(double f, double beta, double* w) {
    const double h = 0.5 * NTAPS, i0b = i0_series_d(beta);
    double sum = 0.0;
    for (int m = 0; m < NTAPS; ++m) {
        const double d = f - (double)(m - NTAPS / 2 + 1);
        double v = 0.0;
        if (fabs(d) < h) {
            const double sinc = (d == 0.0) ? 1.0 : sin(M_PI * d) / (M_PI * d);
            v = sinc * i0_series_d(beta * sqrt(1.0 - (d / h) * (d / h))) / i0b;
        }
        w[m] = v;
        sum += v;
    }
    for (int m = 0; m < NTAPS; ++m) w[m] /= sum;
}

__global__ void make_windows_kernel(const float2* __restrict__ echo, int rows, int Ns, const float* __restrict__ frac,
                                    const int32_t* __restrict__ row, const int32_t* __restrict__ pos, long long n,
                                    double beta, double prior_beta, float2* __restrict__ win,
                                    float2* __restrict__ tgt) {
    const long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (b >= n) return;
    const int r = min(max(row[b], 0), rows - 1);
    const long long p0 = pos[b];
    const float2* e = echo + (size_t)r * Ns;
    for (int m = 0; m < NT; ++m) {
        const long long j = p0 + m - 3;
        win[b * NT + m] = (j >= 0 && j < Ns) ? e[j] : make_float2(0.f, 0.f);
    }
    // 32 taps k = -15 .. 16, normalised Kaiser-windowed sinc at distance f - k
    const double f = (double)frac[b];
    double w[32];
    kaiser_taps<32>(f, beta, w);
    double yr = 0.0, yi = 0.0;
    for (int m = 0; m < 32; ++m) {
        const long long j = p0 + m - 15;
        if (j < 0 || j >= Ns) continue;
        yr += w[m] * (double)e[j].x;
        yi += w[m] * (double)e[j].y;
    }
    if (prior_beta >= 0.0) {
        // residual target: less the prior's 8-tap interpolation of the window
        double wp[NT];
        kaiser_taps<NT>(f, prior_beta, wp);
        for (int m = 0; m < NT; ++m) {
            const long long j = p0 + m - 3;
            if (j < 0 || j >= Ns) continue;
            yr -= wp[m] * (double)e[j].x;
            yi -= wp[m] * (double)e[j].y;
        }
    }
    tgt[b] = make_float2((float)yr, (float)yi);
}

// ---------------------------------------------------------------------------
// Loss and gradient: each block handles SPB samples and writes its partial
// gradient; a second kernel adds the partials in block order.

__global__ void __launch_bounds__(TPB) mlp_block_kernel(const float* __restrict__ theta, const float* __restrict__ frac,
                                                        const float2* __restrict__ win, const float2* __restrict__ tgt,
                                                        long long n, float* __restrict__ part_grad,
                                                        float* __restrict__ part_loss) {
    extern __shared__ float sh[];
    float* W = sh;                           // NPAR rounded weights
    float* A1 = W + NPAR;                    // [SPB][H] a1
    float* G1 = A1 + SPB * H;                // [SPB][H] gelu'(z1), later dz1
    float* A2 = G1 + SPB * H;                // [SPB][H] a2
    float* G2 = A2 + SPB * H;                // [SPB][H] gelu'(z2), later dz2
    float* X = G2 + SPB * H;                 // [SPB] x
    float* DT = X + SPB;                     // [SPB][NT] dL/dt
    float* red = DT + SPB * NT;              // [TPB/32]
    const int tid = threadIdx.x;
    const long long s0 = (long long)blockIdx.x * SPB;
    const int ns = (int)min((long long)SPB, n - s0);
    const float invB = 1.0f / (float)n;

    for (int k = tid; k < NPAR; k += TPB) W[k] = fp16_round(theta[k]);
    for (int s = tid; s < SPB; s += TPB) X[s] = s < ns ? 2.0f * frac[s0 + s] - 1.0f : 0.0f;
    __syncthreads();
    // layer 1
    for (int k = tid; k < SPB * H; k += TPB) {
        const int s = k / H, j = k % H;
        const float z = fmaf(W[O_W1 + j], X[s], W[O_B1 + j]);
        A1[k] = gelu(z);
        G1[k] = gelu_grad(z);
    }
    __syncthreads();
    // layer 2
    for (int k = tid; k < SPB * H; k += TPB) {
        const int s = k / H, i = k % H;
        float z = W[O_B2 + i];
        const float* w2 = W + O_W2 + i * H;
        const float* a = A1 + s * H;
        for (int j = 0; j < H; ++j) z = fmaf(w2[j], a[j], z);
        A2[k] = gelu(z);
        G2[k] = gelu_grad(z);
    }
    __syncthreads();
    // output taps, residual and dL/dt (one thread per sample)
    float lsum = 0.f;
    for (int s = tid; s < SPB; s += TPB) {
        if (s >= ns) {
            for (int m = 0; m < NT; ++m) DT[s * NT + m] = 0.f;
            continue;
        }
        float rx = -tgt[s0 + s].x, ry = -tgt[s0 + s].y;
        for (int m = 0; m < NT; ++m) {
            float v = W[O_B3 + m];
            const float* w3 = W + O_W3 + m * H;
            const float* a = A2 + s * H;
            for (int i = 0; i < H; ++i) v = fmaf(w3[i], a[i], v);
            const float2 wv = win[(s0 + s) * NT + m];
            rx = fmaf(v, wv.x, rx);
            ry = fmaf(v, wv.y, ry);
        }
        lsum += rx * rx + ry * ry;
        for (int m = 0; m < NT; ++m) {
            const float2 wv = win[(s0 + s) * NT + m];
            DT[s * NT + m] = 2.0f * invB * (rx * wv.x + ry * wv.y);   // 2/B Re(conj(r) s_m)
        }
    }
    // block loss
    for (int o = 16; o; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    if ((tid & 31) == 0) red[tid >> 5] = lsum;
    __syncthreads();
    if (tid == 0) {
        float t = 0.f;
        for (int k = 0; k < TPB / 32; ++k) t += red[k];
        part_loss[blockIdx.x] = t * invB;
    }
    float* pg = part_grad + (size_t)blockIdx.x * NPAR;
    // dW3, db3
    for (int k = tid; k < NT * H + NT; k += TPB) {
        if (k < NT * H) {
            const int m = k / H, i = k % H;
            float g = 0.f;
            for (int s = 0; s < ns; ++s) g = fmaf(DT[s * NT + m], A2[s * H + i], g);
            pg[O_W3 + k] = g;
        } else {
            const int m = k - NT * H;
            float g = 0.f;
            for (int s = 0; s < ns; ++s) g += DT[s * NT + m];
            pg[O_B3 + m] = g;
        }
    }
    // dz2 = (W3^T dt) * gelu'(z2)  (in place of G2)
    for (int k = tid; k < SPB * H; k += TPB) {
        const int s = k / H, i = k % H;
        float d = 0.f;
        for (int m = 0; m < NT; ++m) d = fmaf(W[O_W3 + m * H + i], DT[s * NT + m], d);
        G2[k] = d * G2[k];
    }
    __syncthreads();
    // dW2, db2
    for (int k = tid; k < H * H + H; k += TPB) {
        if (k < H * H) {
            const int i = k / H, j = k % H;
            float g = 0.f;
            for (int s = 0; s < ns; ++s) g = fmaf(G2[s * H + i], A1[s * H + j], g);
            pg[O_W2 + k] = g;
        } else {
            const int i = k - H * H;
            float g = 0.f;
            for (int s = 0; s < ns; ++s) g += G2[s * H + i];
            pg[O_B2 + i] = g;
        }
    }
    // dz1 = (W2^T dz2) * gelu'(z1)  (in place of G1)
    for (int k = tid; k < SPB * H; k += TPB) {
        const int s = k / H, j = k % H;
        float d = 0.f;
        for (int i = 0; i < H; ++i) d = fmaf(W[O_W2 + i * H + j], G2[s * H + i], d);
        G1[k] = d * G1[k];
    }
    __syncthreads();
    // dW1, db1
    for (int k = tid; k < 2 * H; k += TPB) {
        const int j = k % H;
        float g = 0.f;
        if (k < H)
            for (int s = 0; s < ns; ++s) g = fmaf(G1[s * H + j], X[s], g);
        else
            for (int s = 0; s < ns; ++s) g += G1[s * H + j];
        pg[(k < H ? O_W1 : O_B1) + j] = g;
    }
}

__global__ void sum_partials_kernel(const float* __restrict__ part_grad, const float* __restrict__ part_loss,
                                    int nblocks, float* __restrict__ grad, float* __restrict__ loss) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < NPAR) {
        double g = 0.0;
        for (int b = 0; b < nblocks; ++b) g += part_grad[(size_t)b * NPAR + k];
        grad[k] = (float)g;
    }
    if (k == 0) {
        double l = 0.0;
        for (int b = 0; b < nblocks; ++b) l += part_loss[b];
        *loss = (float)l;
    }
}

__global__ void adam_kernel(float* __restrict__ theta, const float* __restrict__ grad, float* __restrict__ m,
                            float* __restrict__ v, int step, float lr, float b1, float b2, float eps) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= NPAR) return;
    const float g = grad[k];
    const float mk = b1 * m[k] + (1.0f - b1) * g;
    const float vk = b2 * v[k] + (1.0f - b2) * g * g;
    m[k] = mk;
    v[k] = vk;
    const float mh = mk / (1.0f - powf(b1, (float)step));
    const float vh = vk / (1.0f - powf(b2, (float)step));
    theta[k] -= lr * mh / (sqrtf(vh) + eps);
}

// One thread per fraction f = j / table_n: the prior's taps (if any) plus the network's.
__global__ void tabulate_kernel(const float* __restrict__ theta, int table_n, double prior_beta,
                                float* __restrict__ out) {
    __shared__ float W[NPAR];
    for (int k = threadIdx.x; k < NPAR; k += blockDim.x) W[k] = fp16_round(theta[k]);
    __syncthreads();
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j > table_n) return;
    const float x = 2.0f * ((float)j / (float)table_n) - 1.0f;
    float a1[H];
    for (int q = 0; q < H; ++q) a1[q] = gelu(fmaf(W[O_W1 + q], x, W[O_B1 + q]));
    float a2[H];
    for (int i = 0; i < H; ++i) {
        float z = W[O_B2 + i];
        for (int q = 0; q < H; ++q) z = fmaf(W[O_W2 + i * H + q], a1[q], z);
        a2[i] = gelu(z);
    }
    double wp[NT];
    if (prior_beta >= 0.0) kaiser_taps<NT>((double)j / (double)table_n, prior_beta, wp);
    for (int m = 0; m < NT; ++m) {
        float v = W[O_B3 + m];
        for (int i = 0; i < H; ++i) v = fmaf(W[O_W3 + m * H + i], a2[i], v);
        out[(size_t)j * NT + m] = prior_beta >= 0.0 ? (float)(wp[m] + (double)v) : v;
    }
}

size_t block_smem() { return sizeof(float) * (NPAR + 4 * SPB * H + SPB + SPB * NT + TPB / 32); }

}  // namespace
}  // namespace sas

using namespace sas;

extern "C" int sas_mlp_make_windows(const void* d_echo, int32_t rows, int32_t n_samples, const float* d_frac,
                                    const int32_t* d_row, const int32_t* d_pos, int64_t n, double target_beta,
                                    double prior_beta, void* d_windows, void* d_targets, void* stream) {
    if (!d_echo || rows < 1 || n_samples < 1 || n < 0 || (n > 0 && (!d_frac || !d_row || !d_pos || !d_windows ||
                                                                     !d_targets))) {
        set_error("sas_mlp_make_windows: bad argument");
        return SAS_ERR_ARG;
    }
    if (n == 0) return SAS_OK;
    make_windows_kernel<<<(unsigned)((n + 127) / 128), 128, 0, (cudaStream_t)stream>>>(
        (const float2*)d_echo, rows, n_samples, d_frac, d_row, d_pos, n, target_beta, prior_beta,
        (float2*)d_windows, (float2*)d_targets);
    SAS_CUDA(cudaGetLastError());
    return SAS_OK;
}

extern "C" int64_t sas_mlp_workspace_bytes(int64_t n) {
    if (n < 1) return 0;
    const int64_t nb = (n + SPB - 1) / SPB;
    return nb * (int64_t)NPAR * 4 + nb * 4 + 256;
}

extern "C" int sas_mlp_loss_grad(const float* d_theta, const float* d_frac, const void* d_windows,
                                 const void* d_targets, int64_t n, float* d_loss, float* d_grad, void* d_work,
                                 void* stream) {
    if (!d_theta || !d_frac || !d_windows || !d_targets || n < 1 || !d_loss || !d_grad || !d_work) {
        set_error("sas_mlp_loss_grad: bad argument");
        return SAS_ERR_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int nb = (int)((n + SPB - 1) / SPB);
    float* part_grad = (float*)d_work;
    float* part_loss = part_grad + (size_t)nb * NPAR;
    const size_t smem = block_smem();
    SAS_CUDA(cudaFuncSetAttribute(mlp_block_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    mlp_block_kernel<<<nb, TPB, smem, st>>>(d_theta, d_frac, (const float2*)d_windows, (const float2*)d_targets, n,
                                            part_grad, part_loss);
    SAS_CUDA(cudaGetLastError());
    sum_partials_kernel<<<(NPAR + 255) / 256, 256, 0, st>>>(part_grad, part_loss, nb, d_grad, d_loss);
    SAS_CUDA(cudaGetLastError());
    return SAS_OK;
}

extern "C" int sas_mlp_adam(float* d_theta, const float* d_grad, float* d_m, float* d_v, int32_t step, float lr,
                            float beta1, float beta2, float eps, void* stream) {
    if (!d_theta || !d_grad || !d_m || !d_v || step < 1) {
        set_error("sas_mlp_adam: bad argument");
        return SAS_ERR_ARG;
    }
    adam_kernel<<<(NPAR + 255) / 256, 256, 0, (cudaStream_t)stream>>>(d_theta, d_grad, d_m, d_v, step, lr, beta1,
                                                                      beta2, eps);
    SAS_CUDA(cudaGetLastError());
    return SAS_OK;
}

extern "C" int sas_interp_tabulate_mlp(const float* d_theta, int32_t table_n, double prior_beta, float* d_table_out,
                                       void* stream) {
    if (!d_theta || !d_table_out || table_n < 1 || !(prior_beta < 50.0)) {
        set_error("sas_interp_tabulate_mlp: bad argument");
        return SAS_ERR_ARG;
    }
    tabulate_kernel<<<(table_n + 1 + 127) / 128, 128, 0, (cudaStream_t)stream>>>(d_theta, table_n, prior_beta,
                                                                               d_table_out);
    SAS_CUDA(cudaGetLastError());
    return SAS_OK;
}
