// libsas host API: handle and device slab, sensor geometry (Eq. 2), echo
// storage, interpolator fitting, status reporting.
#include "sas_common.cuh"

#include <cudaTypedefs.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>

namespace sas {

static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

int cuda_fail(cudaError_t e, const char* what) {
    set_error("%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
    return e == cudaErrorMemoryAllocation ? SAS_ERR_OOM : SAS_ERR_CUDA;
}

int sm_count() {
    static int cached[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return 1;
    if (!cached[dev]) {
        int n = 0;
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        cached[dev] = n > 0 ? n : 1;
    }
    return cached[dev];
}

// ---------------------------------------------------------------------------
// Tensor maps for the bulk-copy engine

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

int encode_echo_map(CUtensorMap* map, const void* base, int elem_bytes, int Ns, int rows, int box_len) {
    auto fn = encode_fn();
    if (!fn) {
        set_error("cuTensorMapEncodeTiled unavailable from the driver");
        return SAS_ERR_CUDA;
    }
    const cuuint64_t dims[2] = {(cuuint64_t)Ns, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)Ns * (cuuint64_t)elem_bytes};
    const cuuint32_t box[2] = {(cuuint32_t)box_len, 1u};
    const cuuint32_t estr[2] = {1u, 1u};
    const CUtensorMapDataType dt = elem_bytes == 8 ? CU_TENSOR_MAP_DATA_TYPE_INT64 : CU_TENSOR_MAP_DATA_TYPE_UINT32;
    CUresult r = fn(map, dt, 2, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("cuTensorMapEncodeTiled failed (%d): Ns=%d rows=%d box=%d elem=%d", (int)r, Ns, rows, box_len,
                  elem_bytes);
        return SAS_ERR_CUDA;
    }
    return SAS_OK;
}

// ---------------------------------------------------------------------------
// Sensor positions (Sec. II-C): x_TX,i = p_i + dp_i + R_i l_TX, x_RX,i,c = p_i + dp_i + R_i l_c,
// with R_i the attitude rotation of Eq. 2 (attitude_rotation).
__global__ void geometry_kernel(int P, int C, const double* __restrict__ pos, const double* __restrict__ att,
                                const double* __restrict__ lever, const double* __restrict__ off,
                                double* __restrict__ tx, double* __restrict__ rx, float* __restrict__ rotc,
                                float2* __restrict__ txs, float2* __restrict__ rxs) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P) return;
    double R[9];
    attitude_rotation(att[3 * i + 0], att[3 * i + 1], att[3 * i + 2], R);
    const double b0 = pos[3 * i] + off[3 * i], b1 = pos[3 * i + 1] + off[3 * i + 1],
                 b2 = pos[3 * i + 2] + off[3 * i + 2];
    // columns 0 and 1 of R: body-frame components (R^T v).x, (R^T v).y of a NED vector v
    rotc[6 * i + 0] = (float)R[0];
    rotc[6 * i + 1] = (float)R[3];
    rotc[6 * i + 2] = (float)R[6];
    rotc[6 * i + 3] = (float)R[1];
    rotc[6 * i + 4] = (float)R[4];
    rotc[6 * i + 5] = (float)R[7];
    for (int c = -1; c < C; ++c) {
        const double* l = lever + 3 * (c + 1);
        double* o = (c < 0) ? tx + 3 * (size_t)i : rx + 3 * ((size_t)i * C + c);
        o[0] = b0 + R[0] * l[0] + R[1] * l[1] + R[2] * l[2];
        o[1] = b1 + R[3] * l[0] + R[4] * l[1] + R[5] * l[2];
        o[2] = b2 + R[6] * l[0] + R[7] * l[1] + R[8] * l[2];
        float2* os = (c < 0) ? txs + 3 * (size_t)i : rxs + 3 * ((size_t)i * C + c);
        for (int k = 0; k < 3; ++k) os[k] = df_split(o[k]);
    }
}

static int run_geometry(sas_geometry_t h, cudaStream_t st) {
    geometry_kernel<<<(h->P + 127) / 128, 128, 0, st>>>(h->P, h->C, h->d_pos, h->d_att, h->d_lever, h->d_off,
                                                        h->d_tx, h->d_rx, h->d_rotc, h->d_txs, h->d_rxs);
    SAS_CUDA(cudaGetLastError());
    return SAS_OK;
}

// ---------------------------------------------------------------------------
// Echo storage: per-row max |component| scale and 16-bit rounding.

template <typename T>
__device__ __forceinline__ T pack2(float a, float b);
template <>
__device__ __forceinline__ __half2 pack2<__half2>(float a, float b) {
    return __floats2half2_rn(a, b);
}
template <>
__device__ __forceinline__ __nv_bfloat162 pack2<__nv_bfloat162>(float a, float b) {
    return __floats2bfloat162_rn(a, b);
}

template <typename T>
__global__ void quantize_rows_kernel(const float2* __restrict__ src, T* __restrict__ dst, float* __restrict__ scale,
                                     int Ns) {
    const size_t row = blockIdx.x;
    const float2* s = src + row * Ns;
    float m = 0.f;
    for (int j = threadIdx.x; j < Ns; j += blockDim.x) {
        const float2 v = s[j];
        m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y)));
    }
    __shared__ float red[32];
    for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        m = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.f;
        for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (threadIdx.x == 0) red[0] = m;
    }
    __syncthreads();
    const float sc = red[0] > 0.f ? red[0] : 1.f;
    const float inv = 1.0f / sc;
    if (threadIdx.x == 0) scale[row] = sc;
    T* d = dst + row * Ns;
    for (int j = threadIdx.x; j < Ns; j += blockDim.x) {
        const float2 v = s[j];
        d[j] = pack2<T>(v.x * inv, v.y * inv);
    }
}

template <typename T>
__device__ __forceinline__ float2 unpack2(T v);
template <>
__device__ __forceinline__ float2 unpack2<__half2>(__half2 v) {
    return __half22float2(v);
}
template <>
__device__ __forceinline__ float2 unpack2<__nv_bfloat162>(__nv_bfloat162 v) {
    return __bfloat1622float2(v);
}

template <typename T>
__global__ void dequantize_rows_kernel(const T* __restrict__ src, const float* __restrict__ scale,
                                       float2* __restrict__ dst, int Ns) {
    const size_t row = blockIdx.x;
    const float sc = scale[row];
    for (int j = threadIdx.x; j < Ns; j += blockDim.x) {
        const float2 v = unpack2<T>(src[row * Ns + j]);
        dst[row * Ns + j] = make_float2(v.x * sc, v.y * sc);
    }
}

// ---------------------------------------------------------------------------
// Interpolator in Farrow form on half-sample sub-intervals.  On each half h
// of the sample interval, Chebyshev interpolation of each tap's weight
// w_m(f) at the NP first-kind Chebyshev nodes of f in [h/2, (h+1)/2],
// converted to monomials of g = 2 f - h - 1/2.  FP64 throughout.

__device__ double i0_series(double x) {
    const double q = 0.25 * x * x;
    double term = 1.0, sum = 1.0;
    for (int m = 1; m < 200; ++m) {
        term *= q / ((double)m * (double)m);
        sum += term;
        if (term < 1e-17 * sum) break;
    }
    return sum;
}

// weights of all TAPS taps at fraction f (kind 0: Kaiser-sinc; 1: table, linear in f)
__device__ void interp_weights(int kind, double beta, int table_n, const float* table, double f, double* w) {
    if (kind == SAS_INTERP_KAISER_SINC) {
        const double h = 0.5 * TAPS, i0b = i0_series(beta);
        double sum = 0.0;
        for (int m = 0; m < TAPS; ++m) {
            const double d = f - (double)(m - TAPS / 2 + 1);
            double v = 0.0;
            if (fabs(d) < h) {
                const double s2 = 1.0 - (d / h) * (d / h);
                const double sinc = (d == 0.0) ? 1.0 : sin(M_PI * d) / (M_PI * d);
                v = sinc * i0_series(beta * sqrt(s2)) / i0b;
            }
            w[m] = v;
            sum += v;
        }
        for (int m = 0; m < TAPS; ++m) w[m] /= sum;
    } else {
        double x = f * table_n;
        int j = (int)floor(x);
        if (j < 0) j = 0;
        if (j > table_n - 1) j = table_n - 1;
        const double r = x - j;
        for (int m = 0; m < TAPS; ++m)
            w[m] = (1.0 - r) * (double)table[(size_t)j * TAPS + m] + r * (double)table[(size_t)(j + 1) * TAPS + m];
    }
}

// Monomial coefficients in g of tap t's weight on half h, from its values at
// the N Chebyshev nodes of the half (FP64, not rounded).
template <int N>
__device__ void fit_half_tap(const double (*node_w)[TAPS], int t, double mono_g[N]) {
    // Chebyshev coefficients a_k = (2/N) sum_j y_j T_k(x_j), a_0 halved
    double a[N];
    for (int k = 0; k < N; ++k) {
        double s = 0.0;
        for (int j = 0; j < N; ++j) s += node_w[j][t] * cos(M_PI * k * (j + 0.5) / N);
        a[k] = 2.0 * s / N;
    }
    a[0] *= 0.5;
    // monomials in x: T_0 = 1, T_1 = x, T_{k+1} = 2x T_k - T_{k-1}
    double tkm1[N] = {0}, tk[N] = {0}, mono[N] = {0};
    tkm1[0] = 1.0;
    tk[1] = 1.0;
    mono[0] += a[0];
    for (int p = 0; p < N; ++p) mono[p] += a[1] * tk[p];
    for (int k = 2; k < N; ++k) {
        double tn[N] = {0};
        for (int p = 0; p < N; ++p) tn[p] = (p > 0 ? 2.0 * tk[p - 1] : 0.0) - tkm1[p];
        for (int p = 0; p < N; ++p) {
            tkm1[p] = tk[p];
            tk[p] = tn[p];
            mono[p] += a[k] * tn[p];
        }
    }
    double s = 1.0;
    for (int p = 0; p < N; ++p) {  // x = 2 g
        mono_g[p] = mono[p] * s;
        s *= 2.0;
    }
}

// max over f in [0, 1] (2049 points, strided by thread) of |Farrow form - definition|
template <int N>
__device__ double form_error(int kind, double beta, int table_n, const float* table, const float (*c)[TAPS][N]) {
    double e = 0.0;
    for (int q = threadIdx.x; q <= 2048; q += blockDim.x) {
        const double f = q / 2048.0;
        double w[TAPS];
        interp_weights(kind, beta, table_n, table, f, w);
        const int h = min((int)(2.0 * f), NH - 1);
        const double g = 2.0 * f - h - 0.5;
        for (int m = 0; m < TAPS; ++m) {
            double v = 0.0;
            for (int p = N - 1; p >= 0; --p) v = v * g + (double)c[h][m][p];
            e = fmax(e, fabs(v - w[m]));
        }
    }
    return e;
}

__global__ void fit_interp_kernel(int kind, double beta, int table_n, const float* table, FarrowCoef* out,
                                  double* err) {
    __shared__ double node_c[NH][NP][TAPS], node_q[NH][NQ][TAPS];
    __shared__ double emax[2][128];
    const int t = threadIdx.x;
    if (t < NH * NP) {
        const int h = t / NP, j = t % NP;
        const double x = cos(M_PI * (j + 0.5) / NP);
        interp_weights(kind, beta, table_n, table, 0.5 * (h + 0.5 + 0.5 * x), node_c[h][j]);
    } else if (t < NH * NP + NH * NQ) {
        const int h = (t - NH * NP) / NQ, j = (t - NH * NP) % NQ;
        const double x = cos(M_PI * (j + 0.5) / NQ);
        interp_weights(kind, beta, table_n, table, 0.5 * (h + 0.5 + 0.5 * x), node_q[h][j]);
    }
    __syncthreads();
    if (t < NH * TAPS) {
        const int h = t / TAPS, m = t % TAPS;
        double mono[NP];
        fit_half_tap<NP>(node_c[h], m, mono);
        for (int p = 0; p < NP; ++p) out->c[h][m][p] = (float)mono[p];
    } else if (t < 2 * NH * TAPS) {
        const int h = (t - NH * TAPS) / TAPS, m = (t - NH * TAPS) % TAPS;
        double mono[NQ];
        fit_half_tap<NQ>(node_q[h], m, mono);
        for (int p = 0; p < NQ; ++p) out->q[h][m][p] = (float)mono[p];
    }
    __syncthreads();
    // deviation of the (float-rounded) polynomials from the definition
    emax[0][t] = form_error<NP>(kind, beta, table_n, table, out->c);
    emax[1][t] = form_error<NQ>(kind, beta, table_n, table, out->q);
    __syncthreads();
    if (t < 2) {
        double m = 0.0;
        for (int k = 0; k < blockDim.x; ++k) m = fmax(m, emax[t][k]);
        if (err) err[t] = m;
    }
}

int fit_interp(const sas_interp* it, FarrowCoef* d_coef, double* d_err, cudaStream_t st) {
    if (!it) {
        set_error("interp is NULL");
        return SAS_ERR_ARG;
    }
    if (it->taps != TAPS) {
        set_error("only %d-tap interpolators are supported (got %d)", TAPS, it->taps);
        return SAS_ERR_UNSUPPORTED;
    }
    if (it->kind == SAS_INTERP_KAISER_SINC) {
        if (!(it->kaiser_beta >= 0.0 && it->kaiser_beta < 50.0)) {
            set_error("kaiser_beta out of range");
            return SAS_ERR_ARG;
        }
    } else if (it->kind == SAS_INTERP_TABLE) {
        if (!it->d_table || it->table_n < 1) {
            set_error("table interpolator needs d_table and table_n >= 1");
            return SAS_ERR_ARG;
        }
    } else {
        set_error("unknown interpolator kind %d", it->kind);
        return SAS_ERR_ARG;
    }
    fit_interp_kernel<<<1, 128, 0, st>>>(it->kind, it->kaiser_beta, it->table_n, it->d_table, d_coef, d_err);
    SAS_CUDA(cudaGetLastError());
    return SAS_OK;
}

template <int N>
__global__ void interp_eval_kernel(const float (*__restrict__ c)[TAPS][N], const float* __restrict__ f, long long n,
                                   float* __restrict__ taps) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    // the half of the interval (fractions outside [0, 1) extend the nearer half's polynomial)
    const int h = min(max((int)floorf(2.0f * f[i]), 0), NH - 1);
    const float g = fmaf(2.0f, f[i], -(float)h - 0.5f);
    for (int m = 0; m < TAPS; ++m) {
        float v = c[h][m][N - 1];
        for (int p = N - 2; p >= 0; --p) v = fmaf(v, g, c[h][m][p]);
        taps[i * TAPS + m] = v;
    }
}

}  // namespace sas

using namespace sas;

// ---------------------------------------------------------------------------
// C ABI

extern "C" int sas_version(void) { return SAS_VERSION; }
extern "C" const char* sas_last_error(void) { return g_err; }

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

extern "C" int sas_geometry_create(const sas_nav* nav, const sas_signal* sig, void* stream, sas_geometry_t* out) {
    if (!nav || !sig || !out || !nav->ping_pos || !nav->ping_att || !nav->tx_lever || !nav->rx_lever) {
        set_error("sas_geometry_create: null argument");
        return SAS_ERR_ARG;
    }
    *out = nullptr;
    if (nav->n_pings < 1 || nav->n_rx < 1 || sig->n_samples < 8 || (sig->n_samples % 4) != 0 ||
        !(sig->fs > 0) || !(sig->c > 0) || !std::isfinite(sig->fc) || !std::isfinite(sig->t0)) {
        set_error("sas_geometry_create: bad sizes or signal (P=%d C=%d Ns=%d fs=%g c=%g)", nav->n_pings, nav->n_rx,
                  sig->n_samples, sig->fs, sig->c);
        return SAS_ERR_ARG;
    }
    if ((long long)nav->n_pings * nav->n_rx > 0x7fffffffLL) {
        set_error("sas_geometry_create: too many (ping, channel) rows");
        return SAS_ERR_UNSUPPORTED;
    }
    cudaStream_t st = (cudaStream_t)stream;
    sas_geometry_t h = new (std::nothrow) sas_geometry_s();
    if (!h) {
        set_error("host allocation failed");
        return SAS_ERR_OOM;
    }
    h->P = nav->n_pings;
    h->C = nav->n_rx;
    h->Ns = sig->n_samples;
    h->sig = *sig;
    h->echo_dtype = -1;
    h->beam_side = 1;
    cudaGetDevice(&h->device);
    const size_t P = h->P, C = h->C;
    size_t o = 0;
    const size_t o_pos = o; o = align256(o + P * 3 * 8);
    const size_t o_att = o; o = align256(o + P * 3 * 8);
    const size_t o_lev = o; o = align256(o + (1 + C) * 3 * 8);
    const size_t o_off = o; o = align256(o + P * 3 * 8);
    const size_t o_tx = o;  o = align256(o + P * 3 * 8);
    const size_t o_rx = o;  o = align256(o + P * C * 3 * 8);
    const size_t o_rc = o;  o = align256(o + P * 6 * 4);
    const size_t o_txs = o; o = align256(o + P * 3 * 8);
    const size_t o_rxs = o; o = align256(o + P * C * 3 * 8);
    const size_t o_vl = o;  o = align256(o + P * 3 * 8);
    const size_t o_st = o;  o = align256(o + 16);
    const size_t o_cu = o;  o = align256(o + 4 * 8);
    const size_t o_cf = o;  o = align256(o + sizeof(FarrowCoef));
    const size_t o_fe = o;  o = align256(o + 2 * 8);
    cudaError_t e = cudaMalloc(&h->slab, o);
    if (e != cudaSuccess) {
        delete h;
        return cuda_fail(e, "cudaMalloc(slab)");
    }
    char* b = (char*)h->slab;
    h->d_pos = (double*)(b + o_pos);
    h->d_att = (double*)(b + o_att);
    h->d_lever = (double*)(b + o_lev);
    h->d_off = (double*)(b + o_off);
    h->d_tx = (double*)(b + o_tx);
    h->d_rx = (double*)(b + o_rx);
    h->d_rotc = (float*)(b + o_rc);
    h->d_txs = (float2*)(b + o_txs);
    h->d_rxs = (float2*)(b + o_rxs);
    h->d_vel = (double*)(b + o_vl);
    h->d_status = (uint32_t*)(b + o_st);
    h->d_cull = (unsigned long long*)(b + o_cu);
    h->d_coef = (FarrowCoef*)(b + o_cf);
    h->d_fit_err = (double*)(b + o_fe);
    int rc = SAS_OK;
    auto ck = [&](cudaError_t err, const char* w) {
        if (rc == SAS_OK && err != cudaSuccess) rc = cuda_fail(err, w);
    };
    ck(cudaMemcpyAsync(h->d_pos, nav->ping_pos, P * 3 * 8, cudaMemcpyHostToDevice, st), "copy ping_pos");
    ck(cudaMemcpyAsync(h->d_att, nav->ping_att, P * 3 * 8, cudaMemcpyHostToDevice, st), "copy ping_att");
    ck(cudaMemcpyAsync(h->d_lever, nav->tx_lever, 3 * 8, cudaMemcpyHostToDevice, st), "copy tx_lever");
    ck(cudaMemcpyAsync(h->d_lever + 3, nav->rx_lever, C * 3 * 8, cudaMemcpyHostToDevice, st), "copy rx_lever");
    ck(cudaMemsetAsync(h->d_off, 0, P * 3 * 8, st), "zero offsets");
    ck(cudaMemsetAsync(h->d_status, 0, 16, st), "zero status");
    ck(cudaMemsetAsync(h->d_cull, 0, 4 * 8, st), "zero culling counts");
    if (rc == SAS_OK) rc = run_geometry(h, st);
    if (rc != SAS_OK) {
        cudaFree(h->slab);
        delete h;
        return rc;
    }
    *out = h;
    return SAS_OK;
}

extern "C" int sas_geometry_set_offsets(sas_geometry_t h, const double* offsets, int on_device, void* stream) {
    if (!h) {
        set_error("null handle");
        return SAS_ERR_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const size_t bytes = (size_t)h->P * 3 * 8;
    if (!offsets)
        SAS_CUDA(cudaMemsetAsync(h->d_off, 0, bytes, st));
    else
        SAS_CUDA(cudaMemcpyAsync(h->d_off, offsets, bytes,
                                 on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
    return run_geometry(h, st);
}

extern "C" int sas_geometry_set_beam(sas_geometry_t h, double beam_width, int side) {
    if (!h || !(beam_width < M_PI) || (side != 1 && side != -1)) {
        set_error("sas_geometry_set_beam: need a handle, beam_width < pi and side = +1 or -1");
        return SAS_ERR_ARG;
    }
    h->beam_tan = beam_width > 0.0 ? tan(0.5 * beam_width) : 0.0;
    h->beam_side = side;
    return SAS_OK;
}

extern "C" int sas_geometry_set_refraction(sas_geometry_t h, double z_interface, double c_sediment) {
    if (!h || !std::isfinite(z_interface) || !std::isfinite(c_sediment)) {
        set_error("sas_geometry_set_refraction: need a handle and finite arguments");
        return SAS_ERR_ARG;
    }
    h->z_int = z_interface;
    h->c_sed = c_sediment > 0.0 ? c_sediment : 0.0;
    return SAS_OK;
}

extern "C" int sas_geometry_set_velocity(sas_geometry_t h, const double* vel, int on_device, void* stream) {
    if (!h) {
        set_error("null handle");
        return SAS_ERR_ARG;
    }
    if (!vel) {
        h->has_vel = 0;
        return SAS_OK;
    }
    SAS_CUDA(cudaMemcpyAsync(h->d_vel, vel, (size_t)h->P * 3 * 8,
                             on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, (cudaStream_t)stream));
    if (!on_device) SAS_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    h->has_vel = 1;
    return SAS_OK;
}

extern "C" int sas_geometry_positions(sas_geometry_t h, double* d_tx, double* d_rx, void* stream) {
    if (!h) {
        set_error("null handle");
        return SAS_ERR_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    if (d_tx) SAS_CUDA(cudaMemcpyAsync(d_tx, h->d_tx, (size_t)h->P * 3 * 8, cudaMemcpyDeviceToDevice, st));
    if (d_rx)
        SAS_CUDA(cudaMemcpyAsync(d_rx, h->d_rx, (size_t)h->P * h->C * 3 * 8, cudaMemcpyDeviceToDevice, st));
    return SAS_OK;
}

extern "C" int sas_geometry_destroy(sas_geometry_t h) {
    if (!h) return SAS_OK;
    cudaDeviceSynchronize();
    if (h->d_echo) cudaFree(h->d_echo);
    if (h->d_scale) cudaFree(h->d_scale);
    if (h->d_scratch) cudaFree(h->d_scratch);
    if (h->slab) cudaFree(h->slab);
    delete h;
    return SAS_OK;
}

extern "C" int sas_echo_upload(sas_geometry_t h, const void* echo, int on_device, int store_dtype, void* stream) {
    if (!h || !echo) {
        set_error("sas_echo_upload: null argument");
        return SAS_ERR_ARG;
    }
    if (store_dtype != SAS_ECHO_C64 && store_dtype != SAS_ECHO_C32_F16 && store_dtype != SAS_ECHO_C32_BF16) {
        set_error("sas_echo_upload: bad store_dtype %d", store_dtype);
        return SAS_ERR_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const size_t rows = (size_t)h->P * h->C, Ns = h->Ns;
    const size_t elem = store_dtype == SAS_ECHO_C64 ? 8 : 4;
    const size_t need = rows * Ns * elem;
    if (h->echo_bytes != need) {
        if (h->d_echo) {
            SAS_CUDA(cudaStreamSynchronize(st));
            cudaFree(h->d_echo);
            h->d_echo = nullptr;
            h->echo_bytes = 0;
        }
        SAS_CUDA(cudaMalloc(&h->d_echo, need));
        h->echo_bytes = need;
    }
    if (store_dtype != SAS_ECHO_C64 && !h->d_scale) SAS_CUDA(cudaMalloc(&h->d_scale, rows * sizeof(float)));
    h->echo_dtype = -1;
    if (store_dtype == SAS_ECHO_C64) {
        SAS_CUDA(cudaMemcpyAsync(h->d_echo, echo, need, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                 st));
    } else {
        // quantise from a device complex64 source; host sources go through a
        // bounded staging buffer, a block of rows at a time
        const float2* src = (const float2*)echo;
        float2* stage = nullptr;
        size_t chunk_rows = rows;
        if (!on_device) {
            chunk_rows = std::max<size_t>(1, (size_t)(256u << 20) / (Ns * 8));
            chunk_rows = std::min(chunk_rows, rows);
            SAS_CUDA(cudaMalloc(&stage, chunk_rows * Ns * 8));
        }
        int rc = SAS_OK;
        for (size_t r0 = 0; r0 < rows && rc == SAS_OK; r0 += chunk_rows) {
            const size_t nr = std::min(chunk_rows, rows - r0);
            const float2* s = src + r0 * Ns;
            if (!on_device) {
                cudaError_t e = cudaMemcpyAsync(stage, s, nr * Ns * 8, cudaMemcpyHostToDevice, st);
                if (e != cudaSuccess) {
                    rc = cuda_fail(e, "stage echo");
                    break;
                }
                s = stage;
            }
            if (store_dtype == SAS_ECHO_C32_F16)
                quantize_rows_kernel<__half2><<<(unsigned)nr, 256, 0, st>>>(s, (__half2*)h->d_echo + r0 * Ns,
                                                                         h->d_scale + r0, (int)Ns);
            else
                quantize_rows_kernel<__nv_bfloat162><<<(unsigned)nr, 256, 0, st>>>(
                    s, (__nv_bfloat162*)h->d_echo + r0 * Ns, h->d_scale + r0, (int)Ns);
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) rc = cuda_fail(e, "quantize_rows_kernel");
            if (!on_device) {
                // the staging buffer is reused by the next block of rows
                e = cudaStreamSynchronize(st);
                if (rc == SAS_OK && e != cudaSuccess) rc = cuda_fail(e, "stage sync");
            }
        }
        if (stage) cudaFree(stage);
        if (rc != SAS_OK) return rc;
    }
    h->echo_dtype = store_dtype;
    return SAS_OK;
}

extern "C" int sas_echo_download(sas_geometry_t h, void* d_out, void* stream) {
    if (!h || !d_out) {
        set_error("sas_echo_download: null argument");
        return SAS_ERR_ARG;
    }
    if (h->echo_dtype < 0) {
        set_error("no echo uploaded");
        return SAS_ERR_STATE;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const size_t rows = (size_t)h->P * h->C;
    if (h->echo_dtype == SAS_ECHO_C64) {
        SAS_CUDA(cudaMemcpyAsync(d_out, h->d_echo, h->echo_bytes, cudaMemcpyDeviceToDevice, st));
    } else if (h->echo_dtype == SAS_ECHO_C32_F16) {
        dequantize_rows_kernel<__half2><<<(unsigned)rows, 256, 0, st>>>((const __half2*)h->d_echo, h->d_scale,
                                                                      (float2*)d_out, h->Ns);
        SAS_CUDA(cudaGetLastError());
    } else {
        dequantize_rows_kernel<__nv_bfloat162><<<(unsigned)rows, 256, 0, st>>>(
            (const __nv_bfloat162*)h->d_echo, h->d_scale, (float2*)d_out, h->Ns);
        SAS_CUDA(cudaGetLastError());
    }
    return SAS_OK;
}

static int check_grid(const sas_grid* g, int dim3) {
    if (!g || g->nx < 1 || g->ny < 1 || g->nz < 1 || (!dim3 && g->nz != 1) || !std::isfinite(g->dx) ||
        !std::isfinite(g->dy) || !std::isfinite(g->x0) || !std::isfinite(g->y0) || !std::isfinite(g->z0) ||
        (dim3 && !std::isfinite(g->dz))) {
        set_error("bad grid");
        return SAS_ERR_ARG;
    }
    return SAS_OK;
}

// Fits the interpolator into the handle; a Kaiser fit is kept while its
// parameters are unchanged (tables are refitted on every call, their contents
// may change between calls).
static int handle_fit(sas_geometry_t h, const sas_interp* it, cudaStream_t st) {
    if (it && it->kind == SAS_INTERP_KAISER_SINC && h->fit_valid && h->fit_taps == it->taps &&
        h->fit_beta == it->kaiser_beta)
        return SAS_OK;
    h->fit_valid = 0;
    int rc = fit_interp(it, h->d_coef, h->d_fit_err, st);
    if (rc == SAS_OK && it->kind == SAS_INTERP_KAISER_SINC) {
        h->fit_valid = 1;
        h->fit_taps = it->taps;
        h->fit_beta = it->kaiser_beta;
    }
    return rc;
}

static int backproject(sas_geometry_t h, const sas_grid* g, const sas_interp* it, void* img, int acc, void* stream,
                       int dim3) {
    if (!h || !img) {
        set_error("backproject: null argument");
        return SAS_ERR_ARG;
    }
    int rc = check_grid(g, dim3);
    if (rc != SAS_OK) return rc;
    if (h->echo_dtype < 0) {
        set_error("backproject: no echo uploaded");
        return SAS_ERR_STATE;
    }
    if (h->c_sed > 0.0 && (h->has_vel || h->beam_tan > 0.0)) {
        set_error("backproject: the refraction model does not combine with receiver motion or a beam");
        return SAS_ERR_UNSUPPORTED;
    }
    cudaStream_t st = (cudaStream_t)stream;
    rc = handle_fit(h, it, st);
    if (rc != SAS_OK) return rc;
    ForwardArgs a{h, *g, (float2*)img, dim3, acc ? 1 : 0, st};
    return launch_forward(a);
}

extern "C" int sas_backproject_2d(sas_geometry_t h, const sas_grid* g, const sas_interp* it, void* img, int acc,
                                  void* stream) {
    return backproject(h, g, it, img, acc, stream, 0);
}

extern "C" int sas_backproject_3d(sas_geometry_t h, const sas_grid* g, const sas_interp* it, void* img, int acc,
                                  void* stream) {
    return backproject(h, g, it, img, acc, stream, 1);
}

extern "C" int sas_backproject_adjoint(sas_geometry_t h, const sas_grid* g, const sas_interp* it,
                                       const void* d_grad_image, void* d_echo_adj, double* d_grad_offsets,
                                       void* stream) {
    if (!h || !d_grad_image || (!d_echo_adj && !d_grad_offsets)) {
        set_error("sas_backproject_adjoint: null argument");
        return SAS_ERR_ARG;
    }
    int rc = check_grid(g, g && g->nz > 1);
    if (rc != SAS_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    if (d_grad_offsets && h->echo_dtype < 0) {
        set_error("sas_backproject_adjoint: the offset gradient needs an uploaded echo");
        return SAS_ERR_STATE;
    }
    rc = handle_fit(h, it, st);
    if (rc != SAS_OK) return rc;
    AdjointArgs a{h, *g, (const float2*)d_grad_image, (float2*)d_echo_adj, d_grad_offsets, st};
    return launch_adjoint(a);
}

extern "C" int sas_interp_eval_form(const sas_interp* it, int degree, const float* d_f, int64_t n, float* d_taps,
                                    double* d_max_err, void* stream) {
    if (!it || (n > 0 && (!d_f || !d_taps)) || n < 0 || (degree != NP - 1 && degree != NQ - 1)) {
        set_error("sas_interp_eval_form: bad argument");
        return SAS_ERR_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const size_t cf_bytes = (sizeof(FarrowCoef) + 255) / 256 * 256;
    FarrowCoef* d_coef = nullptr;
    SAS_CUDA(cudaMallocAsync(&d_coef, cf_bytes + 16, st));
    double* d_err = (double*)((char*)d_coef + cf_bytes);
    int rc = fit_interp(it, d_coef, d_err, st);
    const bool cubic = degree == NP - 1;
    if (rc == SAS_OK && n > 0) {
        const unsigned nb = (unsigned)((n + 255) / 256);
        if (cubic)
            interp_eval_kernel<NP><<<nb, 256, 0, st>>>(d_coef->c, d_f, n, d_taps);
        else
            interp_eval_kernel<NQ><<<nb, 256, 0, st>>>(d_coef->q, d_f, n, d_taps);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) rc = cuda_fail(e, "interp_eval_kernel");
    }
    if (rc == SAS_OK && d_max_err) {
        cudaError_t e = cudaMemcpyAsync(d_max_err, d_err + (cubic ? 0 : 1), 8, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) rc = cuda_fail(e, "copy fit error");
    }
    cudaFreeAsync(d_coef, st);
    return rc;
}

extern "C" int sas_interp_eval(const sas_interp* it, const float* d_f, int64_t n, float* d_taps, double* d_max_err,
                               void* stream) {
    return sas_interp_eval_form(it, NP - 1, d_f, n, d_taps, d_max_err, stream);
}

extern "C" int sas_sync_status(sas_geometry_t h, void* stream) {
    if (!h) {
        set_error("null handle");
        return SAS_ERR_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    uint32_t v = 0;
    SAS_CUDA(cudaStreamSynchronize(st));
    SAS_CUDA(cudaMemcpy(&v, h->d_status, 4, cudaMemcpyDeviceToHost));
    if (v) {
        SAS_CUDA(cudaMemset(h->d_status, 0, 4));
        if (v & DEV_TIMEOUT) {
            set_error("a kernel's bounded wait ran out (status 0x%x); its results are invalid", v);
            return SAS_ERR_TIMEOUT;
        }
        set_error("a kernel's Farrow-row index left the tile's window (status 0x%x); its results are invalid", v);
        return SAS_ERR_CHECK;
    }
    return SAS_OK;
}

extern "C" int sas_build_flags(void) {
#ifdef SAS_CHECKED
    return 1;
#else
    return 0;
#endif
}

extern "C" int sas_cull_stats(sas_geometry_t h, long long* out, int reset, void* stream) {
    if (!h || !out) {
        set_error("null argument");
        return SAS_ERR_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    unsigned long long v[4];
    SAS_CUDA(cudaStreamSynchronize(st));
    SAS_CUDA(cudaMemcpy(v, h->d_cull, sizeof(v), cudaMemcpyDeviceToHost));
    for (int k = 0; k < 3; ++k) out[k] = (long long)v[k];
    if (reset) SAS_CUDA(cudaMemset(h->d_cull, 0, sizeof(v)));
    return SAS_OK;
}

extern "C" int sas_debug_starve_copies(sas_geometry_t h, int skip, int32_t wait_limit_ms) {
    if (!h || wait_limit_ms < 0) {
        set_error("bad argument");
        return SAS_ERR_ARG;
    }
    h->debug_skip_copies = skip ? 1 : 0;
    h->debug_wait_ms = skip ? (wait_limit_ms > 0 ? wait_limit_ms : 200) : 0;
    return SAS_OK;
}
