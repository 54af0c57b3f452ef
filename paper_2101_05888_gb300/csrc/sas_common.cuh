// Internal definitions shared by the libsas translation units.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "../../include/sas.h"

namespace sas {

// ---------------------------------------------------------------------------
// Error reporting (host)

void set_error(const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* what);

#define SAS_CUDA(call)                                   \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

// Device status bits (handle status word).
enum : uint32_t { DEV_TIMEOUT = 1u, DEV_ROW_RANGE = 2u };

// The Farrow row a kernel reads, clamped into [0, last].  The host sizes the
// window so that the clamp never moves an index; in the checked build
// (compiled with -DSAS_CHECKED) an index it had to move sets DEV_ROW_RANGE in
// the handle's status word, which sas_sync_status reports.
__device__ __forceinline__ unsigned row_index(unsigned raw, unsigned last, uint32_t* status) {
#ifdef SAS_CHECKED
    if (raw > last) atomicOr(status, DEV_ROW_RANGE);
#else
    (void)status;
#endif
    return min(raw, last);
}

// ---------------------------------------------------------------------------
// Interpolator in Farrow form on half-sample sub-intervals: the sample
// interval [i0, i0 + 1) splits into the halves h = floor(2 f) (f = u - i0),
// and on half h tap m (offset k_m = m - 3) has the weight
//   w_m(f) = sum_{p<NP} coef[h][m][p] g^p,  g = 2 f - h - 1/2 in [-1/2, 1/2),
// so the interpolated value is a cubic in g whose coefficients are FIR
// outputs of the echo:  s = sum_p g^p E_p^h[i0],  E_p^h[i] = sum_m coef[h][m][p] e[i + k_m].
// g is the fraction of the half-sample coordinate 2u: with n = floor(2u),
// i0 = floor(n / 2) and h = n mod 2.
// ---------------------------------------------------------------------------
// Attitude rotation of Eq. 2 (roll phi, pitch theta, yaw psi), row-major R:
//   [ ct cps,  cps st sph - cph sps,  cph cps st + sph sps ]
//   [ ct sps,  cph cps + st sph sps,  cph st sps - cps sph ]
//   [ -st,     ct sph,                ct cph               ]
__device__ __forceinline__ void attitude_rotation(double roll, double pitch, double yaw, double R[9]) {
    double sph, cph, sth, cth, sps, cps;
    sincos(roll, &sph, &cph);
    sincos(pitch, &sth, &cth);
    sincos(yaw, &sps, &cps);
    R[0] = cth * cps; R[1] = cps * sth * sph - cph * sps; R[2] = cph * cps * sth + sph * sps;
    R[3] = cth * sps; R[4] = cph * cps + sth * sph * sps; R[5] = cph * sth * sps - cps * sph;
    R[6] = -sth;      R[7] = cth * sph;                   R[8] = cth * cph;
}

constexpr int TAPS = 8;
constexpr int NH = 2;            // sub-intervals (halves) of a sample interval
constexpr int NP = 4;            // polynomial degree 3 on each
constexpr int NQ = 3;            // degree 2 on each (16-bit echoes, forward pass)
struct FarrowCoef {
    float c[NH][TAPS][NP];       // cubic form
    float q[NH][TAPS][NQ];       // quadratic form of the same interpolator
};

// Fits the interpolator to both Farrow forms on the device (FP64 Chebyshev
// interpolation at NP, resp. NQ, nodes of each half, converted to monomials
// in g).  d_coef: device FarrowCoef; d_err: optional device double[2], max
// |fit - definition| over the weights of the cubic and of the quadratic form.
int fit_interp(const sas_interp* interp, FarrowCoef* d_coef, double* d_err, cudaStream_t st);

// ---------------------------------------------------------------------------
// PTX helpers (device)

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

// Announces `bytes` more transaction bytes on the barrier's current phase
// without arriving (one call per bulk copy that will complete on it).
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// One test of the phase with the given parity; while it is incomplete the
// thread may be suspended until it completes or suspend_ns pass.
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity, uint32_t suspend_ns) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity), "r"(suspend_ns)
        : "memory");
    return ok != 0;
}

// Waits for the barrier phase with the given parity to complete; gives up
// after limit_ns of wall time (returns false).  Never spins unboundedly.
// Each test suspends the waiting warp (up to 200 us) rather than spinning, so
// a warp that waits does not take issue slots from the warps that work.
constexpr uint32_t MBAR_SUSPEND_NS = 200000;
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, uint64_t limit_ns) {
    if (mbar_try_wait(bar, parity, MBAR_SUSPEND_NS)) return true;
    const uint64_t t0 = globaltimer_ns();
    for (;;) {
        if (mbar_try_wait(bar, parity, MBAR_SUSPEND_NS)) return true;
        if (globaltimer_ns() - t0 > limit_ns) return false;
    }
}

// 2D tiled bulk tensor copy global -> shared, completion on an mbarrier.
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int32_t x, int32_t y,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cta.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(dst), "l"(map), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void named_bar_sync(uint32_t id, uint32_t count) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// Packed FP32 pair arithmetic (sm_100+), round to nearest on both halves:
// ffma2 = a * b + c, fadd2 = a + b, fsub2 = a - b, fmul2 = a * b.
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) {
    uint64_t ra = *reinterpret_cast<uint64_t*>(&a), rb = *reinterpret_cast<uint64_t*>(&b),
             rc = *reinterpret_cast<uint64_t*>(&c), rd;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(rd) : "l"(ra), "l"(rb), "l"(rc));
    return *reinterpret_cast<float2*>(&rd);
}
__device__ __forceinline__ float2 fadd2(float2 a, float2 b) {
    uint64_t ra = *reinterpret_cast<uint64_t*>(&a), rb = *reinterpret_cast<uint64_t*>(&b), rd;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(rd) : "l"(ra), "l"(rb));
    return *reinterpret_cast<float2*>(&rd);
}
__device__ __forceinline__ float2 fsub2(float2 a, float2 b) {
    uint64_t ra = *reinterpret_cast<uint64_t*>(&a), rb = *reinterpret_cast<uint64_t*>(&b), rd;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(rd) : "l"(ra), "l"(rb));
    return *reinterpret_cast<float2*>(&rd);
}
__device__ __forceinline__ float2 fmul2(float2 a, float2 b) {
    uint64_t ra = *reinterpret_cast<uint64_t*>(&a), rb = *reinterpret_cast<uint64_t*>(&b), rd;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(rd) : "l"(ra), "l"(rb));
    return *reinterpret_cast<float2*>(&rd);
}
// The value of x, opaque to the compiler: it cannot be recomputed at its uses
// from the (FP64) expression that produced it, so it stays in a register.
__device__ __forceinline__ float opaque(float x) {
    float y;
    asm volatile("mov.b32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// ---------------------------------------------------------------------------
// Double-float arithmetic: a value is hi + lo with |lo| <= ulp(hi) / 2, about
// 48 significant bits, on the FP32 pipe (the FP64 pipe of this GPU is slow
// and its long latency chains stalled the per-pair reference terms).  Sums
// use the two-sum of Knuth, products the exact FMA residual (Dekker's
// product with a fused multiply-add); every operation is written with explicit
// roundings so that no contraction or reassociation changes it.
struct dfl {
    float hi, lo;
};
__device__ __forceinline__ dfl df_fast(float a, float b) {   // |a| >= |b| (or a = 0)
    const float s = __fadd_rn(a, b);
    return dfl{s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ dfl df_add(dfl x, dfl y) {
    const float s = __fadd_rn(x.hi, y.hi);
    const float bb = __fsub_rn(s, x.hi);
    const float e = __fadd_rn(__fsub_rn(x.hi, __fsub_rn(s, bb)), __fsub_rn(y.hi, bb));
    return df_fast(s, __fadd_rn(e, __fadd_rn(x.lo, y.lo)));
}
__device__ __forceinline__ dfl df_neg(dfl x) { return dfl{-x.hi, -x.lo}; }
__device__ __forceinline__ dfl df_mul(dfl x, dfl y) {
    const float p = __fmul_rn(x.hi, y.hi);
    const float e = fmaf(x.hi, y.lo, fmaf(x.lo, y.hi, fmaf(x.hi, y.hi, -p)));
    return df_fast(p, e);
}
// square root of a > 0: the FP32 root refined by one Newton step on the residual
__device__ __forceinline__ dfl df_sqrt(dfl a) {
    const float r = __fsqrt_rn(a.hi);
    const float e = __fadd_rn(fmaf(-r, r, a.hi), a.lo);   // a - r^2 (exact FMA residual of the high part)
    return df_fast(r, __fmul_rn(e, __fdiv_rn(0.5f, r)));
}
__device__ __forceinline__ float df_float(dfl x) { return __fadd_rn(x.hi, x.lo); }
// the double-float nearest a double (host and device)
__host__ __device__ inline float2 df_split(double v) {
    const float hi = (float)v;
    return make_float2(hi, (float)(v - (double)hi));
}

// elementwise max / min of pairs (two scalar operations)
__device__ __forceinline__ float2 fmax2(float2 a, float2 b) { return make_float2(fmaxf(a.x, b.x), fmaxf(a.y, b.y)); }
__device__ __forceinline__ float2 fmin2(float2 a, float2 b) { return make_float2(fminf(a.x, b.x), fminf(a.y, b.y)); }

// Integer rounding on the FP32 pipe: for |v| < 2^22, t = v + 1.5*2^23 (round
// to nearest) holds the nearest integer n of v in its low mantissa bits
// (bits(t) = bits(1.5*2^23) + n) and t - 1.5*2^23 = n exactly.
constexpr float FLOOR_MAGIC = 12582912.0f;  // 1.5 * 2^23

}  // namespace sas

// ---------------------------------------------------------------------------
// Handle

struct sas_geometry_s {
    int device;
    int P, C, Ns;
    sas_signal sig;
    // one slab: positions, attitude, levers, offsets, sensor positions, status
    void* slab;
    double* d_pos;     // [P][3]
    double* d_att;     // [P][3]
    double* d_lever;   // [1 + C][3]  (TX first)
    double* d_off;     // [P][3]
    double* d_tx;      // [P][3]
    double* d_rx;      // [P][C][3]
    float2* d_txs;     // [P][3] the same as double-floats (hi, lo)
    float2* d_rxs;     // [P][C][3]
    float* d_rotc;     // [P][6]: columns 0 and 1 of the attitude matrix (beam tests)
    double* d_vel;     // [P][3]: receiver velocity during reception (valid if has_vel)
    int has_vel;       // 0: stop-and-hop
    double beam_tan;   // tan(beam width / 2); <= 0: no beam field of view
    int beam_side;     // +1 starboard, -1 port
    // seabed refraction (forward backprojection): interface depth, sediment sound speed (<= 0: off)
    double z_int;
    double c_sed;
    uint32_t* d_status;
    unsigned long long* d_cull;   // [4] ray-culling counts (candidate, computed, beam edge, -)
    sas::FarrowCoef* d_coef;
    double* d_fit_err;
    int fit_valid;       // d_coef holds the Kaiser fit for (fit_taps, fit_beta)
    int fit_taps;
    double fit_beta;
    // echo storage
    void* d_echo;
    float* d_scale;    // [P][C] (16-bit storage)
    int echo_dtype;    // -1 = none
    size_t echo_bytes;
    // adjoint / VJP scratch (grown on demand)
    void* d_scratch;
    size_t scratch_bytes;
    // failure-detection test hook
    int debug_skip_copies;
    int32_t debug_wait_ms;
};

namespace sas {

struct ForwardArgs {
    sas_geometry_t h;
    sas_grid grid;
    float2* image;
    int dim3;
    int accumulate;
    cudaStream_t stream;
};
int launch_forward(const ForwardArgs& a);

struct AdjointArgs {
    sas_geometry_t h;
    sas_grid grid;
    const float2* grad_image;
    float2* echo_adj;
    double* grad_offsets;
    cudaStream_t stream;
};
int launch_adjoint(const AdjointArgs& a);

// Tensor map encoder obtained from the driver (no link-time libcuda dependency).
int encode_echo_map(CUtensorMap* map, const void* base, int elem_bytes, int Ns, int rows, int box_len);

int sm_count();

}  // namespace sas
