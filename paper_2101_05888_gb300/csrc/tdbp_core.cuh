// Shared machinery of the backprojection kernels that read the echo:
// the forward pass (echo -> image) and the gradient with respect to per-ping
// position offsets (image gradient -> offset gradient).
//
// Both evaluate, for every pixel x of the grid, ping i and channel c
// (Sec. II-A: Eq. 1 inverted per pixel):
//   tau = (|x - x_TX,i| + |x - x_RX,i,c|) / c,  u = (tau - t0) fs,
//   s(u) = sum_k w_k(frac u) e[i][c][floor u + k]          (zero outside the row)
// forward:   I(x) += s(u) exp(+j 2 pi fc tau)
// gradient:  dL/d(dp_i) += 2 Re{ conj(G(x)) (fs s'(u) + j 2 pi fc s(u)) exp(j 2 pi fc tau) } * (-(u_T + u_R)/c)
// with G = dL/dI* and u_T, u_R unit vectors from the sensors to the pixel.
//
// One CTA per image tile; warp 0 is the producer, warps 1..7 the consumers.
//  * producer, one lane per (ping, channel) pair, 32 pairs a stage: FP64
//    reference terms at the tile centre x0 (R = x0 - sensor, |R|, tau_ref,
//    floor(u_ref), fraction, carrier phase mod 1) written to shared memory,
//    and a 2D bulk tensor copy of the echo segment the tile can reach into a
//    ring of NSTAGE stages, completion on an mbarrier (transaction bytes).
//    Samples outside the row are zero-filled by the copy engine.
//  * consumers, 8 pixels a thread:
//    - Farrow expansion for 4 pairs at a time: the interpolator's taps are
//      degree-7 polynomials of g = f - 1/2, so s = sum_p g^p E_p[floor u] with
//      E_p[i] = sum_m coef[m][p] e[i + k_m], computed once per (pair, tile)
//      for every integer position the tile can reach.  Complex64 echoes:
//      E_0..E_3 are kept in FP32 and E_4..E_7 (weighted by |g|^p <= 1/16) in
//      BF16 (FP32 exponent range, so no overflow at any echo amplitude), and
//      the forward pass evaluates that tail in packed BF16.  16-bit echoes
//      (rows normalised to |e| <= 1, so |E_p| <= 5.2): all eight in FP16 and
//      the forward Horner in packed FP16, the row scale applied afterwards in
//      FP32.  One 48-byte row per position either way.
//    - per pixel and pair, with the pair's reference terms broadcast by warp
//      shuffle: differential range dr = (2 R.d + |d|^2) / (|R + d| + |R|), an
//      exact identity evaluated in FP32 on small quantities (d = x - x0); u
//      and the phase from the reference values plus dr-derived offsets;
//      floor/fraction on the FP32 pipe; three 16-byte shared loads; Horner in
//      g; SFU rsqrt, rcp, sin, cos.
//  * every mbarrier wait is bounded in wall time: on expiry the CTA records a
//    timeout in the status word, stops, and the producer waits (bounded) for
//    the copies it has in flight before exiting.
#pragma once

#include "sas_common.cuh"

namespace sas {
namespace core {

constexpr int NCW = 7;                  // consumer warps
constexpr int NCONS = 32 * NCW;         // consumer threads
constexpr int NTHREADS = NCONS + 32;    // + producer warp
constexpr int PAIRS = 32;               // (ping, channel) pairs per stage
constexpr int NSTAGE = 3;               // copy ring depth
constexpr int GROUP = 4;                // pairs per Farrow group
constexpr int GPS = PAIRS / GROUP;      // groups per stage
constexpr int PX = 8;                   // pixels per consumer thread
constexpr int EROW = 48;                // bytes per Farrow row: E0..E3 float2, E4..E7 bfloat162
constexpr int BAR_CONS = 1;             // named barrier of the consumer warps

enum { MODE_FORWARD = 0, MODE_OFFSET_GRAD = 1 };

// producer record fields (structure of arrays in shared memory, one column per pair)
enum { F_TX, F_TY, F_TZ, F_NT2, F_NT, F_RX, F_RY, F_RZ, F_NR2, F_NR, F_UF, F_PH, F_SCALE, F_OFF, NREC };
constexpr int NHOLD = 13;               // fields the per-pixel work needs (F_TX .. F_SCALE)

struct KParams {
    const double* tx;       // [P][3]
    const double* rx;       // [P][C][3]
    const float* scale;     // [P*C] or null
    const FarrowCoef* coef;
    float2* image;          // forward output
    const float2* gimage;   // gradient input dL/dI*
    double* partials;       // gradient output [tiles][P][3]
    uint32_t* status;
    double x0, y0, z0, dx, dy, dz;
    int nx, ny, nz;
    int tiles_x, tiles_y, tiles_z, nsplit, pings_per_split;
    int P, C;
    double t0, fs, fc, inv_c;
    float fs_c, fc_c;       // fs/c, fc/c
    float fs_f, wfc;        // fs, 2 pi fc
    float grad_scale;       // -2/c (factor 2 of dL/dp = 2 Re(...), -1/c of dtau/dp)
    int U, npos, seglen, seg_align, slot_bytes;
    int accumulate, atomic_out, skip_copies;
    unsigned long long wait_ns;
};

template <bool DIM3>
struct Tile;
template <>
struct Tile<false> {  // 2D: 56 (x) x 32 (y); warp w covers x in [8w, 8w+8), rows (lane>>3) + 4s
    static constexpr int TX = 56, TY = 32, TZ = 1;
    __device__ static void pixel(int ct, int s, int& lx, int& ly, int& lz) {
        const int w = ct >> 5, l = ct & 31;
        lx = w * 8 + (l & 7);
        ly = (l >> 3) + 4 * s;
        lz = 0;
    }
};
template <>
struct Tile<true> {   // 3D: 8 (x) x 28 (y) x 8 (z); warp w covers y in [4w, 4w+4), z = s
    static constexpr int TX = 8, TY = 28, TZ = 8;
    __device__ static void pixel(int ct, int s, int& lx, int& ly, int& lz) {
        const int w = ct >> 5, l = ct & 31;
        lx = l & 7;
        ly = w * 4 + (l >> 3);
        lz = s;
    }
};

template <typename ET>
__device__ __forceinline__ float2 load_sample(const unsigned char* slot, int idx, float sc);
template <>
__device__ __forceinline__ float2 load_sample<float2>(const unsigned char* slot, int idx, float) {
    return reinterpret_cast<const float2*>(slot)[idx];
}
template <>
__device__ __forceinline__ float2 load_sample<__half2>(const unsigned char* slot, int idx, float sc) {
    const float2 v = __half22float2(reinterpret_cast<const __half2*>(slot)[idx]);
    return make_float2(v.x * sc, v.y * sc);
}
template <>
__device__ __forceinline__ float2 load_sample<__nv_bfloat162>(const unsigned char* slot, int idx, float sc) {
    const float2 v = __bfloat1622float2(reinterpret_cast<const __nv_bfloat162*>(slot)[idx]);
    return make_float2(v.x * sc, v.y * sc);
}

__device__ __forceinline__ float rsqrt_sfu(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcp_sfu(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// sin and cos of 2 pi x for |x| <= 1/2 on the SFU
__device__ __forceinline__ void sincos_2pi(float x, float& sn, float& cs) {
    const float a = x * 6.28318530717958647f;
    asm("sin.approx.ftz.f32 %0, %1;" : "=f"(sn) : "f"(a));
    asm("cos.approx.ftz.f32 %0, %1;" : "=f"(cs) : "f"(a));
}

__device__ __forceinline__ __half2 h2_of_bits(uint32_t b) {
    return *reinterpret_cast<__half2*>(&b);
}

__device__ __forceinline__ __nv_bfloat162 b2_of_bits(uint32_t b) {
    return *reinterpret_cast<__nv_bfloat162*>(&b);
}

// FP64 reference terms of pair q (ping q / C, channel q % C) at the tile
// centre (X0, Y0, Z0), written to the record column rc (stride PAIRS):
// 2R and |R|^2, |R| for transmitter and receiver (R = x0 - sensor), the
// fraction of u_ref = (tau_ref - t0) fs and the carrier phase fc tau_ref mod 1.
// Returns the raw sample index of Farrow position 0, tap 0: floor(u_ref) - U - 3.
__device__ __forceinline__ int pair_record(const KParams& p, double X0, double Y0, double Z0, long long q, float* rc) {
    const int i = (int)(q / p.C);
    const double* t = p.tx + 3 * (size_t)i;
    const double* r = p.rx + 3 * (size_t)q;
    const double Tx = X0 - t[0], Ty = Y0 - t[1], Tz = Z0 - t[2];
    const double Rx = X0 - r[0], Ry = Y0 - r[1], Rz = Z0 - r[2];
    const double nT2 = Tx * Tx + Ty * Ty + Tz * Tz, nR2 = Rx * Rx + Ry * Ry + Rz * Rz;
    const double nT = sqrt(nT2), nR = sqrt(nR2);
    const double tau = (nT + nR) * p.inv_c;
    double u = (tau - p.t0) * p.fs;
    u = fmin(fmax(u, -268435456.0), 268435456.0);  // keep sample coordinates in int range
    const double iref = floor(u);
    const double ph = p.fc * tau;
    rc[F_TX * PAIRS] = (float)(2.0 * Tx);
    rc[F_TY * PAIRS] = (float)(2.0 * Ty);
    rc[F_TZ * PAIRS] = (float)(2.0 * Tz);
    rc[F_NT2 * PAIRS] = (float)nT2;
    rc[F_NT * PAIRS] = (float)nT;
    rc[F_RX * PAIRS] = (float)(2.0 * Rx);
    rc[F_RY * PAIRS] = (float)(2.0 * Ry);
    rc[F_RZ * PAIRS] = (float)(2.0 * Rz);
    rc[F_NR2 * PAIRS] = (float)nR2;
    rc[F_NR * PAIRS] = (float)nR;
    rc[F_UF * PAIRS] = (float)(u - iref);
    rc[F_PH * PAIRS] = (float)(ph - floor(ph));
    return (int)iref - p.U - 3;
}

// Shared-memory size and launch geometry, host side.
struct Layout {
    int U, npos, seglen, align, slot_bytes;
    size_t smem;
};

inline size_t smem_bytes(int slot_bytes, int npos) {
    return (size_t)NSTAGE * PAIRS * slot_bytes          // echo segments
           + (size_t)2 * GROUP * npos * EROW            // Farrow rows, double buffered
           + (size_t)NSTAGE * NREC * PAIRS * 4          // producer records
           + (size_t)TAPS * NP * 4                      // coefficients
           + (size_t)2 * NHOLD * PAIRS * 4              // consumer copy of the records
           + (size_t)NCW * 4 * 8                        // cross-warp reduction (gradient)
           + (size_t)(2 * NSTAGE + 4) * 8 + 16;         // mbarriers (copy ring, Farrow buffers), abort flag
}

// ----------------------------------------------------------------------------
template <typename ET, bool DIM3, int MODE>
__global__ void __launch_bounds__(NTHREADS, 2) tdbp_kernel(const __grid_constant__ CUtensorMap tmap, const KParams p) {
    using T = Tile<DIM3>;
    // FP16 Farrow rows for 16-bit echoes in the forward pass
    constexpr bool E16 = (MODE == MODE_FORWARD) && (sizeof(ET) == 4);
    extern __shared__ __align__(1024) unsigned char smem[];
    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;

    unsigned char* seg = smem;
    unsigned char* ebuf = seg + (size_t)NSTAGE * PAIRS * p.slot_bytes;
    const int ebuf_pair = p.npos * EROW;
    float* rec = reinterpret_cast<float*>(ebuf + 2 * GROUP * ebuf_pair);
    float* coef_s = rec + NSTAGE * NREC * PAIRS;
    float* hold = coef_s + TAPS * NP;
    double* wred = reinterpret_cast<double*>(hold + 2 * NHOLD * PAIRS);
    uint64_t* bars = reinterpret_cast<uint64_t*>(wred + NCW * 4);      // full[NSTAGE], empty[NSTAGE]
    uint64_t* ebar = bars + 2 * NSTAGE;                                   // Farrow buffers: efull[2], eempty[2]
    volatile int* abort_flag = reinterpret_cast<volatile int*>(ebar + 4);

    const int ntiles = p.tiles_x * p.tiles_y * p.tiles_z;
    const int tile = blockIdx.x % ntiles;
    const int split = blockIdx.x / ntiles;
    const int tx0 = (tile % p.tiles_x) * T::TX;
    const int ty0 = ((tile / p.tiles_x) % p.tiles_y) * T::TY;
    const int tz0 = (tile / (p.tiles_x * p.tiles_y)) * T::TZ;
    // pairs of this CTA: whole pings [ping0, ping1)
    const int ping0 = min(p.P, split * p.pings_per_split);
    const int ping1 = min(p.P, ping0 + p.pings_per_split);
    const long long q0 = (long long)ping0 * p.C;
    const long long q1 = (long long)ping1 * p.C;
    const int nq = (int)(q1 - q0);
    const int nstages = (nq + PAIRS - 1) / PAIRS;
    const int ngroups = (nq + GROUP - 1) / GROUP;
    const double cx = tx0 + 0.5 * (T::TX - 1), cy = ty0 + 0.5 * (T::TY - 1), cz = tz0 + 0.5 * (T::TZ - 1);

    if (tid == 0) {
        for (int s = 0; s < NSTAGE; ++s) {
            mbar_init(smem_u32(&bars[s]), 1);
            mbar_init(smem_u32(&bars[NSTAGE + s]), NCW);
        }
        for (int b = 0; b < 4; ++b) mbar_init(smem_u32(&ebar[b]), NCW);
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (tid < TAPS * NP) coef_s[tid] = (&p.coef->c[0][0])[tid];
    __syncthreads();

    if (warp == 0) {
        // ================= producer =================
        const double X0 = p.x0 + cx * p.dx, Y0 = p.y0 + cy * p.dy, Z0 = p.z0 + (DIM3 ? cz * p.dz : 0.0);
        const uint32_t seg_bytes = (uint32_t)p.seglen * (uint32_t)sizeof(ET);
        int k = 0;
        for (; k < nstages; ++k) {
            const int s = k % NSTAGE;
            if (k >= NSTAGE) {
                const bool ok =
                    mbar_wait_bounded(smem_u32(&bars[NSTAGE + s]), ((k / NSTAGE) - 1) & 1, p.wait_ns);
                if (!ok && lane == 0) {
                    *abort_flag = 1;
                    atomicOr(p.status, DEV_TIMEOUT);
                }
            }
            __syncwarp();
            if (*abort_flag) break;
            const long long q = q0 + (long long)k * PAIRS + lane;
            const bool valid = q < q1;
            int seg_start = 0;
            if (valid) {
                const int base = pair_record(p, X0, Y0, Z0, q, rec + s * NREC * PAIRS + lane);
                seg_start = base - (((base % p.seg_align) + p.seg_align) % p.seg_align);
                float* rc = rec + s * NREC * PAIRS;
                rc[F_OFF * PAIRS + lane] = __int_as_float(base - seg_start);
                rc[F_SCALE * PAIRS + lane] = p.scale ? p.scale[q] : 1.0f;
            }
            __syncwarp();
            if (lane == 0) {
                const int nvalid = (int)min((long long)PAIRS, q1 - (q0 + (long long)k * PAIRS));
                mbar_arrive_expect_tx(smem_u32(&bars[s]), (uint32_t)nvalid * seg_bytes);
            }
            __syncwarp();
            if (valid && !p.skip_copies)
                tma_load_2d(smem_u32(seg + ((size_t)s * PAIRS + lane) * p.slot_bytes), &tmap, seg_start, (int32_t)q,
                            smem_u32(&bars[s]));
        }
        // every issued stage must have landed before the CTA may exit
        for (int kk = max(0, k - NSTAGE); kk < k; ++kk)
            mbar_wait_bounded(smem_u32(&bars[kk % NSTAGE]), (kk / NSTAGE) & 1, p.wait_ns);
        return;
    }

    // ================= consumers =================
    const int ct = tid - 32;
    float dxv, dyv_c, d2c = 0.f;
    float dvar[PX], dT[PX];
    float2 acc[PX];                       // forward: image accumulators; gradient: G(x)
    float rsum[MODE == MODE_OFFSET_GRAD ? PX : 1];
    {
        int lx, ly, lz;
        T::pixel(ct, 0, lx, ly, lz);
        dxv = (float)((tx0 + lx - cx) * p.dx);
        dyv_c = (float)((ty0 + ly - cy) * p.dy);
#pragma unroll
        for (int s = 0; s < PX; ++s) {
            T::pixel(ct, s, lx, ly, lz);
            const float dxs = (float)((tx0 + lx - cx) * p.dx);
            const float dys = (float)((ty0 + ly - cy) * p.dy);
            const float dzs = DIM3 ? (float)((tz0 + lz - cz) * p.dz) : 0.f;
            dvar[s] = DIM3 ? dzs : dys;
            d2c = DIM3 ? dxs * dxs + dys * dys : dxs * dxs;
            dT[s] = 0.f;
            if (MODE == MODE_FORWARD) {
                acc[s] = make_float2(0.f, 0.f);
            } else {
                const int ix = tx0 + lx, iy = ty0 + ly, iz = tz0 + lz;
                acc[s] = (ix < p.nx && iy < p.ny && iz < p.nz) ? p.gimage[((size_t)iz * p.ny + iy) * p.nx + ix]
                                                              : make_float2(0.f, 0.f);
                rsum[MODE == MODE_OFFSET_GRAD ? s : 0] = 0.f;
            }
        }
    }
    float gacc0 = 0.f, gacc1 = 0.f, gacc2 = 0.f;   // gradient: receiver-side sum for the current ping

    float r_cur[NHOLD];
#pragma unroll
    for (int f = 0; f < NHOLD; ++f) r_cur[f] = 0.f;
    const int Ep = ct & 7;
    const int Erun = ct >> 3;                       // 0 .. NRUNSLOT - 1
    constexpr int NRUNSLOT = NCONS / 8;
    constexpr int RMAX = 12;                        // longest run of positions per thread
    // runs of R positions, as few as needed for every run slot to get at most one
    const int runs_per_pair_min = max(1, NRUNSLOT / GROUP);
    const int R = min(RMAX, (p.npos + runs_per_pair_min - 1) / runs_per_pair_min);
    const int runs_per_pair = (p.npos + R - 1) / R;

    // Farrow expansion of group gg into ebuf[gg & 1]
    auto expand = [&](int gg) {
        const int stage = gg / GPS;
        const int s = stage % NSTAGE;
        const float* rc = rec + s * NREC * PAIRS;
        unsigned char* eb = ebuf + (gg & 1) * GROUP * ebuf_pair;
        float cc[TAPS];
#pragma unroll
        for (int m = 0; m < TAPS; ++m) cc[m] = coef_s[m * NP + Ep];
        const int total = GROUP * runs_per_pair;
        for (int run = Erun; run < total; run += NRUNSLOT) {
            const int j = run / runs_per_pair;
            const int pos0 = (run - j * runs_per_pair) * R;
            const int pr = (gg % GPS) * GROUP + j;
            if (stage * PAIRS + pr >= nq) continue;
            const unsigned char* slot = seg + ((size_t)s * PAIRS + pr) * p.slot_bytes;
            const int off = __float_as_int(rc[F_OFF * PAIRS + pr]);
            const float sc = E16 ? 1.0f : rc[F_SCALE * PAIRS + pr];
            const int nout = min(R, p.npos - pos0);
            float2 w[RMAX + TAPS - 1];
#pragma unroll
            for (int t = 0; t < RMAX + TAPS - 1; ++t)
                w[t] = (t < nout + TAPS - 1) ? load_sample<ET>(slot, off + pos0 + t, sc) : make_float2(0.f, 0.f);
            unsigned char* dst = eb + j * ebuf_pair + pos0 * EROW;
#pragma unroll
            for (int kq = 0; kq < RMAX; ++kq) {
                if (kq < nout) {
                    float2 e = make_float2(0.f, 0.f);
#pragma unroll
                    for (int m = 0; m < TAPS; ++m) e = ffma2(make_float2(cc[m], cc[m]), w[kq + m], e);
                    if (E16)
                        *reinterpret_cast<__half2*>(dst + kq * EROW + Ep * 4) = __floats2half2_rn(e.x, e.y);
                    else if (Ep < 4)
                        *reinterpret_cast<float2*>(dst + kq * EROW + Ep * 8) = e;
                    else
                        *reinterpret_cast<__nv_bfloat162*>(dst + kq * EROW + 32 + (Ep - 4) * 4) =
                            __floats2bfloat162_rn(e.x, e.y);
                }
            }
        }
    };

    auto hold_records = [&](int stage) {
        const float* rc = rec + (stage % NSTAGE) * NREC * PAIRS;
        float* hd = hold + (stage & 1) * NHOLD * PAIRS;
        for (int t = ct; t < NHOLD * PAIRS; t += NCONS) hd[t] = rc[t];
    };

    auto maybe_release = [&](int gg) {
        const int stage = gg / GPS;
        if (((gg % GPS) == GPS - 1) || (gg == ngroups - 1)) {
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&bars[NSTAGE + stage % NSTAGE]));
        }
    };

    auto wait_stage = [&](int stage) -> bool {
        const bool ok = mbar_wait_bounded(smem_u32(&bars[stage % NSTAGE]), (stage / NSTAGE) & 1, p.wait_ns);
        if (!ok) {
            *abort_flag = 1;
            atomicOr(p.status, DEV_TIMEOUT);
        }
        return ok;
    };

    // gradient: fold the transmitter term of the finished ping into the
    // per-thread sum, reduce over the CTA in FP64 and write the tile's partial
    float tT0 = 0.f, tT1 = 0.f, tT2 = 0.f, tNT2 = 0.f, tNT = 0.f;   // transmitter terms of the current ping
    auto flush_ping = [&](int ping) {
        if (MODE != MODE_OFFSET_GRAD) return;
        const float Ax = DIM3 ? fmaf(tT0, dxv, tT1 * dyv_c) : tT0 * dxv;
        float hx = 0.5f * tT0 + dxv;
        float hy = DIM3 ? 0.5f * tT1 + dyv_c : 0.f;
        float hz = DIM3 ? 0.f : 0.5f * tT2;
#pragma unroll
        for (int s = 0; s < PX; ++s) {
            const float d2 = fmaf(dvar[s], dvar[s], d2c);
            const float a = DIM3 ? fmaf(tT2, dvar[s], d2) + Ax : fmaf(tT1, dvar[s], d2) + Ax;
            const float sm = tNT2 + a;
            const float k = rsum[MODE == MODE_OFFSET_GRAD ? s : 0] * rsqrt_sfu(sm);   // r / |R_T + d|
            // R_T + d: (R.x + dx, R.y + dy or R.y + dy_s, R.z + dz_s)
            const float vy = DIM3 ? hy : 0.5f * tT1 + dvar[s];
            const float vz = DIM3 ? 0.5f * tT2 + dvar[s] : hz;
            gacc0 = fmaf(k, hx, gacc0);
            gacc1 = fmaf(k, vy, gacc1);
            gacc2 = fmaf(k, vz, gacc2);
            rsum[MODE == MODE_OFFSET_GRAD ? s : 0] = 0.f;
        }
        (void)hy;
        double v0 = gacc0, v1 = gacc1, v2 = gacc2;
        gacc0 = gacc1 = gacc2 = 0.f;
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            v0 += __shfl_xor_sync(0xffffffffu, v0, o);
            v1 += __shfl_xor_sync(0xffffffffu, v1, o);
            v2 += __shfl_xor_sync(0xffffffffu, v2, o);
        }
        const int cw = ct >> 5;
        if (lane == 0) {
            wred[cw * 4 + 0] = v0;
            wred[cw * 4 + 1] = v1;
            wred[cw * 4 + 2] = v2;
        }
        named_bar_sync(BAR_CONS, NCONS);
        if (ct < 3) {
            double sum = 0.0;
            for (int w2 = 0; w2 < NCW; ++w2) sum += wred[w2 * 4 + ct];
            p.partials[((size_t)tile * p.P + ping) * 3 + ct] = sum * (double)p.grad_scale;
        }
        named_bar_sync(BAR_CONS, NCONS);
        (void)tNT;
    };

    // Farrow buffer handoff between consumer warps: efull[b] completes when all
    // warps wrote their share of the rows of buffer b, eempty[b] when all warps
    // finished reading it; warps may drift apart by one group.
    auto warp_arrive = [&](uint64_t* bar) {
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(bar));
    };
    auto wait_bar = [&](uint64_t* bar, uint32_t parity) {
        if (!mbar_wait_bounded(smem_u32(bar), parity, p.wait_ns)) {
            *abort_flag = 1;
            atomicOr(p.status, DEV_TIMEOUT);
        }
    };

    bool aborted = false;
    if (ngroups > 0) {
        const bool ok = wait_stage(0);
        if (ok) {
            hold_records(0);
            expand(0);
            maybe_release(0);
        }
        warp_arrive(&ebar[0]);
        aborted = *abort_flag != 0;
    }

    int prev_ping = -1;
    int cur_ping = ping0, cur_ch = 0;     // (ping, channel) of the next pair, no divisions
    for (int gg = 0; gg < ngroups && !aborted; ++gg) {
        const int nxt = gg + 1;
        if (nxt < ngroups) {
            bool ok = true;
            if (nxt >= 2) wait_bar(&ebar[2 + (nxt & 1)], ((nxt - 2) >> 1) & 1);   // readers of group nxt-2 done
            if (nxt % GPS == 0) {
                ok = wait_stage(nxt / GPS);
                if (ok) hold_records(nxt / GPS);
            }
            if (ok && !*abort_flag) {
                expand(nxt);
                maybe_release(nxt);
            }
            warp_arrive(&ebar[nxt & 1]);
        }
        wait_bar(&ebar[gg & 1], (gg >> 1) & 1);                  // rows of group gg complete
        if (*abort_flag) {
            aborted = true;
            break;
        }
        if (gg % GPS == 0) {
            const float* hd = hold + ((gg / GPS) & 1) * NHOLD * PAIRS;
#pragma unroll
            for (int f = 0; f < NHOLD; ++f) r_cur[f] = hd[f * PAIRS + lane];
        }
        const int stage = gg / GPS;
        const unsigned char* eb = ebuf + (gg & 1) * GROUP * ebuf_pair;
#pragma unroll 1
        for (int j = 0; j < GROUP; ++j) {
            const int pr = (gg % GPS) * GROUP + j;
            if (stage * PAIRS + pr >= nq) break;
            if (cur_ch == 0) {
                const int ping = cur_ping;
                if (prev_ping >= 0) flush_ping(prev_ping);
                prev_ping = ping;
                tT0 = __shfl_sync(0xffffffffu, r_cur[F_TX], pr);
                tT1 = __shfl_sync(0xffffffffu, r_cur[F_TY], pr);
                tT2 = __shfl_sync(0xffffffffu, r_cur[F_TZ], pr);
                tNT2 = __shfl_sync(0xffffffffu, r_cur[F_NT2], pr);
                tNT = __shfl_sync(0xffffffffu, r_cur[F_NT], pr);
                const float Ax = DIM3 ? fmaf(tT0, dxv, tT1 * dyv_c) : tT0 * dxv;
#pragma unroll
                for (int s = 0; s < PX; ++s) {
                    const float d2 = fmaf(dvar[s], dvar[s], d2c);
                    const float a = DIM3 ? fmaf(tT2, dvar[s], d2) + Ax : fmaf(tT1, dvar[s], d2) + Ax;
                    const float sm = tNT2 + a;
                    const float den = fmaf(sm, rsqrt_sfu(sm), tNT);
                    dT[s] = a * rcp_sfu(den);
                }
            }
            const float tRx = __shfl_sync(0xffffffffu, r_cur[F_RX], pr);
            const float tRy = __shfl_sync(0xffffffffu, r_cur[F_RY], pr);
            const float tRz = __shfl_sync(0xffffffffu, r_cur[F_RZ], pr);
            const float nR2 = __shfl_sync(0xffffffffu, r_cur[F_NR2], pr);
            const float nR = __shfl_sync(0xffffffffu, r_cur[F_NR], pr);
            const float uf = __shfl_sync(0xffffffffu, r_cur[F_UF], pr);
            const float phr = __shfl_sync(0xffffffffu, r_cur[F_PH], pr);
            const float scl = E16 ? __shfl_sync(0xffffffffu, r_cur[F_SCALE], pr) : 1.0f;
            const float Ax = DIM3 ? fmaf(tRx, dxv, tRy * dyv_c) : tRx * dxv;
            const unsigned char* erow = eb + j * ebuf_pair;
#pragma unroll
            for (int s = 0; s < PX; ++s) {
                const float d2 = fmaf(dvar[s], dvar[s], d2c);
                const float a = DIM3 ? fmaf(tRz, dvar[s], d2) + Ax : fmaf(tRy, dvar[s], d2) + Ax;
                const float sm = nR2 + a;
                const float rs = rsqrt_sfu(sm);                     // 1 / |R_R + d|
                const float den = fmaf(sm, rs, nR);
                const float D = fmaf(a, rcp_sfu(den), dT[s]);       // two-way differential path [m]
                const float u = fmaf(D, p.fs_c, uf);                 // sample position rel. to floor(u_ref)
                const float ph = fmaf(D, p.fc_c, phr);               // carrier phase [cycles]
                float fl;
                const int di = floor_magic(u, fl);
                const float g = (u - fl) - 0.5f;
                const unsigned pos = min((unsigned)(di + p.U), (unsigned)(p.npos - 1));
                const float4* e = reinterpret_cast<const float4*>(erow + pos * EROW);
                const float pt = __fadd_rn(ph, FLOOR_MAGIC) - FLOOR_MAGIC;   // rint(ph)
                float sn, cs;
                sincos_2pi(ph - pt, sn, cs);
                if (E16) {
                    // packed FP16 Horner over E_7 .. E_0, scale and accumulate in FP32
                    const uint4 lo = *reinterpret_cast<const uint4*>(e), hi = *reinterpret_cast<const uint4*>(e + 1);
                    const __half2 g16 = __float2half2_rn(g);
                    __half2 h = __hfma2(h2_of_bits(hi.w), g16, h2_of_bits(hi.z));
                    h = __hfma2(h, g16, h2_of_bits(hi.y));
                    h = __hfma2(h, g16, h2_of_bits(hi.x));
                    h = __hfma2(h, g16, h2_of_bits(lo.w));
                    h = __hfma2(h, g16, h2_of_bits(lo.z));
                    h = __hfma2(h, g16, h2_of_bits(lo.y));
                    h = __hfma2(h, g16, h2_of_bits(lo.x));
                    const float2 hv = __half22float2(h);
                    const float vx = hv.x * scl, vy = hv.y * scl;
                    acc[s].x = fmaf(vx, cs, fmaf(-vy, sn, acc[s].x));
                    acc[s].y = fmaf(vx, sn, fmaf(vy, cs, acc[s].y));
                    continue;
                }
                const float4 e01 = e[0], e23 = e[1];
                const uint4 eh = *reinterpret_cast<const uint4*>(e + 2);
                const float2 gg2 = make_float2(g, g);
                if (MODE == MODE_FORWARD) {
                    // high-order part in packed BF16: h = ((E7 g + E6) g + E5) g + E4
                    const __nv_bfloat162 g16 = __float2bfloat162_rn(g);
                    __nv_bfloat162 h = __hfma2(b2_of_bits(eh.w), g16, b2_of_bits(eh.z));
                    h = __hfma2(h, g16, b2_of_bits(eh.y));
                    h = __hfma2(h, g16, b2_of_bits(eh.x));
                    float2 v = __bfloat1622float2(h);
                    v = ffma2(v, gg2, make_float2(e23.z, e23.w));
                    v = ffma2(v, gg2, make_float2(e23.x, e23.y));
                    v = ffma2(v, gg2, make_float2(e01.z, e01.w));
                    v = ffma2(v, gg2, make_float2(e01.x, e01.y));
                    acc[s].x = fmaf(v.x, cs, fmaf(-v.y, sn, acc[s].x));
                    acc[s].y = fmaf(v.x, sn, fmaf(v.y, cs, acc[s].y));
                } else {
                    // value and derivative in g (FP32): b = s(g), d = s'(g)
                    float2 b = __bfloat1622float2(b2_of_bits(eh.w));
                    float2 d = make_float2(0.f, 0.f);
                    const float2 c6 = __bfloat1622float2(b2_of_bits(eh.z)), c5 = __bfloat1622float2(b2_of_bits(eh.y)),
                                 c4 = __bfloat1622float2(b2_of_bits(eh.x));
                    d = ffma2(d, gg2, b); b = ffma2(b, gg2, c6);
                    d = ffma2(d, gg2, b); b = ffma2(b, gg2, c5);
                    d = ffma2(d, gg2, b); b = ffma2(b, gg2, c4);
                    d = ffma2(d, gg2, b); b = ffma2(b, gg2, make_float2(e23.z, e23.w));
                    d = ffma2(d, gg2, b); b = ffma2(b, gg2, make_float2(e23.x, e23.y));
                    d = ffma2(d, gg2, b); b = ffma2(b, gg2, make_float2(e01.z, e01.w));
                    d = ffma2(d, gg2, b); b = ffma2(b, gg2, make_float2(e01.x, e01.y));
                    // a = fs s' + j 2 pi fc s ;  r = Re{ conj(G) a exp(j phase) }
                    const float ax = fmaf(p.fs_f, d.x, -p.wfc * b.y);
                    const float ay = fmaf(p.fs_f, d.y, p.wfc * b.x);
                    const float Hx = fmaf(acc[s].x, cs, acc[s].y * sn);       // conj(G) exp(j phase)
                    const float Hy = fmaf(acc[s].x, sn, -acc[s].y * cs);
                    const float r = fmaf(Hx, ax, -Hy * ay);
                    rsum[MODE == MODE_OFFSET_GRAD ? s : 0] += r;
                    // receiver unit vector (R_R + d) / |R_R + d| times r
                    const float kr = r * rs;
                    const float vx = fmaf(0.5f, tRx, dxv);
                    const float vy = DIM3 ? fmaf(0.5f, tRy, dyv_c) : fmaf(0.5f, tRy, dvar[s]);
                    const float vz = DIM3 ? fmaf(0.5f, tRz, dvar[s]) : 0.5f * tRz;
                    gacc0 = fmaf(kr, vx, gacc0);
                    gacc1 = fmaf(kr, vy, gacc1);
                    gacc2 = fmaf(kr, vz, gacc2);
                }
            }
            if (++cur_ch == p.C) {
                cur_ch = 0;
                ++cur_ping;
            }
        }
        warp_arrive(&ebar[2 + (gg & 1)]);
    }
    if (aborted) return;
    if (MODE == MODE_OFFSET_GRAD) {
        if (prev_ping >= 0) flush_ping(prev_ping);
        return;
    }

#pragma unroll
    for (int s = 0; s < PX; ++s) {
        int lx, ly, lz;
        T::pixel(ct, s, lx, ly, lz);
        const int ix = tx0 + lx, iy = ty0 + ly, iz = tz0 + lz;
        if (ix >= p.nx || iy >= p.ny || iz >= p.nz) continue;
        float2* dst = p.image + ((size_t)iz * p.ny + iy) * p.nx + ix;
        if (p.atomic_out) {
            atomicAdd(dst, acc[s]);
        } else if (p.accumulate) {
            const float2 o = *dst;
            *dst = make_float2(o.x + acc[s].x, o.y + acc[s].y);
        } else {
            *dst = acc[s];
        }
    }
}

// ----------------------------------------------------------------------------
// Host side: shared launch set-up.

struct Setup {
    KParams prm;
    CUtensorMap map;
    size_t smem;
    int blocks;
    int elem;
};

inline void tile_dims(int dim3, int& TXs, int& TYs, int& TZs) {
    if (dim3) {
        TXs = Tile<true>::TX; TYs = Tile<true>::TY; TZs = Tile<true>::TZ;
    } else {
        TXs = Tile<false>::TX; TYs = Tile<false>::TY; TZs = Tile<false>::TZ;
    }
}

// Fills the launch description for grid g; min_ctas: aim for at least this
// many CTAs by splitting the pings of each tile (0 = never split).
int prepare(sas_geometry_t h, const sas_grid& g, int dim3, long long min_ctas, Setup& S, bool need_echo = true);

template <int MODE>
int launch_mode(const Setup& S, int echo_dtype, int dim3, cudaStream_t st);

}  // namespace core
}  // namespace sas
