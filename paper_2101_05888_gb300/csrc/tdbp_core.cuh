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
//    ring of NSEG stages, completion on an mbarrier (transaction bytes).
//    Samples outside the row are zero-filled by the copy engine.  The
//    producer also expands each stage's pairs, 4 at a time (a group), into a
//    ring of NBUF Farrow buffers handed to the consumers by mbarriers:
//    - Farrow expansion: on each half of a sample interval the interpolator's
//      taps are cubics in g (the fraction of the half-sample coordinate 2u,
//      minus 1/2), so s = sum_p g^p E_p^h[floor u] with
//      E_p^h[i] = sum_m coef[h][m][p] e[i + k_m], computed once per (pair,
//      tile) for both halves of every sample position the tile can reach:
//      one row per half-sample position.  Complex64 echoes: E_0..E_3 in FP32,
//      a 32-byte row read by two 16-byte loads.  16-bit echoes (rows
//      normalised to |e| <= 1, so |E_p| stays near 1): E_0..E_3 in FP16, a
//      16-byte row, and the forward Horner in packed FP16, the row scale
//      applied afterwards in FP32.
//  * consumers, 8 pixels a thread, group after group:
//    - per pixel and pair, with the pair's reference terms read by uniform
//      16-byte loads: differential range dr = (2 R.d + |d|^2) / (|R + d| + |R|), an
//      exact identity evaluated in FP32 on small quantities (d = x - x0); 2u
//      and the phase from the reference values plus dr-derived offsets;
//      floor/fraction on the FP32 pipe; the row (two 16-byte shared loads,
//      or one for FP16 rows); cubic Horner in g; SFU rsqrt, rcp, sin, cos (the
//      carrier phase in radians, taken directly while it stays within 512 rad).
//    - the pixels of a warp form an 8 x 4 block (4 x 2 per quarter-warp), so
//      the rows one 16-byte load instruction reads span fewer than 8
//      consecutive half-sample positions (quarter-warp phases) and fall in
//      distinct bank groups.
//  * every mbarrier wait is bounded in wall time: on expiry the CTA records a
//    timeout in the status word, stops, and the producer waits (bounded) for
//    the copies it has in flight before exiting.
#pragma once

#include "sas_common.cuh"

#include <type_traits>

namespace sas {
namespace core {

constexpr int NCW = 7;                  // consumer warps
constexpr int NCONS = 32 * NCW;         // consumer threads
constexpr int NTHREADS = NCONS + 32;    // + producer warp
constexpr int PAIRS = 32;               // (ping, channel) pairs per stage
constexpr int NSEG = 2;                 // echo-segment ring depth (stages)
constexpr int NRS = 3;                  // record ring depth (stages)
constexpr int NBUF = 3;                 // Farrow buffers (groups)
constexpr int GROUP = 4;                // pairs per Farrow group
constexpr int GPS = PAIRS / GROUP;      // groups per stage
constexpr int PX = 8;                   // pixels per consumer thread
constexpr int ROW32 = 32;               // bytes of an FP32 Farrow row: E0..E3 as FP32 pairs
constexpr int ROW24 = 24;               // bytes of a quadratic FP32 Farrow row (16-bit echoes, forward pass)
constexpr int RUN = 15;                 // sample positions per expansion run
constexpr int BAR_CONS = 1;             // named barrier of the consumer warps

enum { MODE_FORWARD = 0, MODE_OFFSET_GRAD = 1 };
// group descriptor flags: the group ends its stage / is the last one
enum { GD_STAGE_END = 1, GD_LAST = 2 };

// record fields of one (ping, channel) pair, in the order of the float4 a
// consumer loads: {2R_R, |R_R|^2}, {|R_R|, 2 frac u_ref - 1/2, phase [rad], scale},
// {2R_T, |R_T|^2}, {|R_T|, ping, flags, segment offset}, {c0, c1.x},
// {c1.y, c1.z, -, -} (c0, c1: columns 0 and 1 of the attitude matrix), and
// with receiver motion {v/c, R_R.v/c}, {2R_R at the ping time, -} (R_R is
// then taken from the receiver's position at the reception of the tile
// centre's echo; the beam tests use the ping-time position)
enum {
    F_RX, F_RY, F_RZ, F_NR2, F_NR, F_UF, F_PH, F_SCALE, F_TX, F_TY, F_TZ, F_NT2, F_NT, F_PING, F_FLAGS, F_OFF,
    F_C0X, F_C0Y, F_C0Z, F_C1X, F_C1Y, F_C1Z, F_PAD0, F_PAD1, F_VX, F_VY, F_VZ, F_RV, F_BRX, F_BRY, F_BRZ, F_PAD2,
    NREC
};
// pair flags: the whole tile lies inside the transmitter / receiver beam;
// the transmitter / receiver leg refracts into the sediment for some pixel
enum { FL_TX_FULL = 1, FL_RX_FULL = 2, FL_T_REFR = 4, FL_R_REFR = 8 };
// With the seabed refraction model the record has two more blocks of RF_N
// fields after the first sixteen (the receiver leg's, then the
// transmitter leg's), in place of the beam and motion fields:
// {a, rho_r^2, rho_r, xi_r}, {sigma_r, |W_r|, |V_r|, f_r}, {df/drho, df/db, K_r, K_s}
// (see refr_leg_ref)
enum { RF_A, RF_RHO2, RF_RHO, RF_XI, RF_SIG, RF_W, RF_V, RF_F, RF_DFR, RF_DFB, RF_KR, RF_KS, RF_N };
enum { F_RREF = 16, F_TREF = F_RREF + RF_N, NREC_REFR = F_TREF + RF_N };
static_assert(NREC_REFR % 4 == 0 && F_RREF % 4 == 0 && F_TREF % 4 == 0, "refraction blocks are float4-aligned");

struct KParams {
    const double* tx;       // [P][3]
    const double* rx;       // [P][C][3]
    const float2* txs;      // [P][3] as double-floats
    const float2* rxs;      // [P][C][3] as double-floats
    float2 k_fs_c, k_t0fs, k_fc_c;   // fs / c, t0 fs, fc / c as double-floats
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
    float hs_c, wfc_c;      // 2 fs/c (half samples per metre of path), 2 pi fc/c (radians per metre)
    float2 hs_c2, wfc_c2;   // the same, duplicated for packed pixel pairs
    int phase_direct;       // carrier phases stay within +-PHASE_DIRECT_MAX rad: no reduction
    float fs2_f, wfc;       // 2 fs (ds/du = 2 ds/dg), 2 pi fc
    float grad_scale;       // -2/c (factor 2 of dL/dp = 2 Re(...), -1/c of dtau/dp)
    // beam field of view (Sec. II-C): sensor sees x iff b = R^T (x - sensor) has
    // side b_y > 0 and |b_x| <= beam_tan side b_y; rotc [P][6] = columns 0, 1 of R
    const float* rotc;
    int beam;
    float beam_tan, beam_side;
    unsigned long long* cull;   // [3] candidate, computed, beam-edge (ping, channel, tile) blocks
    // receiver motion during reception: velocity [P][3] (m/s) or null (stop-and-hop)
    const double* vel;
    // seabed refraction (forward pass): interface depth, n = c / c_s, and the
    // constants of the crossing solve with r = max(n, 1/n): r^2, r^2 - 1,
    // (r^2 - 1)^(-1/2); refr_tol: the crossing-point tolerance [m]
    int refract, refr_fast_sed;    // refr_fast_sed: n < 1, the sediment is the faster medium
    double z_int, refr_n;
    float refr_nf, refr_r2, refr_M, refr_isM, refr_tol;
    float hx, hy, hz;       // half extents of a tile's pixel-centre box [m]
    int U, npos, npos_pad, seglen, seg_align, slot_bytes;
    int accumulate, atomic_out, skip_copies;
    unsigned long long wait_ns;
};

template <bool DIM3>
struct Tile;
// Lane l of a warp holds column (l & 3) + 4 (l >> 4) and row (l >> 2) & 3 of an
// 8 x 4 block: a half-warp is a 4 x 4 block, a quarter-warp a 4 x 2 block.
__device__ __forceinline__ int lane_col(int l) { return (l & 3) + ((l >> 2) & 4); }
__device__ __forceinline__ int lane_row(int l) { return (l >> 2) & 3; }
template <>
struct Tile<false> {  // 2D: 56 (x) x 32 (y); warp w covers x in [8w, 8w+8), rows lane_row + 4s
    static constexpr int TX = 56, TY = 32, TZ = 1;
    __device__ static void pixel(int ct, int s, int& lx, int& ly, int& lz) {
        const int w = ct >> 5, l = ct & 31;
        lx = w * 8 + lane_col(l);
        ly = lane_row(l) + 4 * s;
        lz = 0;
    }
};
template <>
struct Tile<true> {   // 3D: 8 (x) x 28 (y) x 8 (z); warp w covers y in [4w, 4w+4), z = s
    static constexpr int TX = 8, TY = 28, TZ = 8;
    __device__ static void pixel(int ct, int s, int& lx, int& ly, int& lz) {
        const int w = ct >> 5, l = ct & 31;
        lx = lane_col(l);
        ly = w * 4 + lane_row(l);
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

// sin and cos on the SFU; callers reduce the argument to [-pi, pi] first
// (the range on which the SFU approximations are accurate)
__device__ __forceinline__ void sincos_sfu(float a, float& sn, float& cs) {
    asm("sin.approx.ftz.f32 %0, %1;" : "=f"(sn) : "f"(a));
    asm("cos.approx.ftz.f32 %0, %1;" : "=f"(cs) : "f"(a));
}
__device__ __forceinline__ void sincos_2pi(float x, float& sn, float& cs) {
    sincos_sfu(x * 6.28318530717958647f, sn, cs);
}
constexpr float TWO_PI_F = 6.28318530717958647f;

// Carrier phases: x = phase_ref + 2 pi fc/c D in radians.  sin.approx and
// cos.approx keep an absolute error of about |x| 1.5e-7 (measured: 6.6e-5 at
// |x| = 450, 1.1e-7 rms on [-pi, pi]) -- the error of rounding x itself at that
// magnitude -- so while every phase of a launch stays within PHASE_DIRECT_MAX
// they take x directly.  Beyond it the phase is first reduced to [-pi, pi] by
// x - 2 pi n, n = rint(x / 2 pi), with 2 pi split in two constants (C1 exact
// in 8 bits, so n C1 is exact for |n| < 2^15).
constexpr double PHASE_DIRECT_MAX = 512.0;
constexpr float PHASE_C1 = 6.28125f;
constexpr float PHASE_C2 = 1.9353071795864769e-3f;   // 2 pi - C1
__device__ __forceinline__ float2 reduce_phase2(float2 x) {
    const float2 M = make_float2(FLOOR_MAGIC, FLOOR_MAGIC);
    const float2 n = fsub2(ffma2(x, make_float2(0.15915494309189535f, 0.15915494309189535f), M), M);
    x = ffma2(n, make_float2(-PHASE_C1, -PHASE_C1), x);
    return ffma2(n, make_float2(-PHASE_C2, -PHASE_C2), x);
}
__device__ __forceinline__ float reduce_phase(float x) {
    const float n = __fadd_rn(fmaf(x, 0.15915494309189535f, FLOOR_MAGIC), -FLOOR_MAGIC);
    return fmaf(n, -PHASE_C2, fmaf(n, -PHASE_C1, x));
}



// Farrow rows, one per half-sample position r = 2 n + h (sample position n
// of the tile's window, half h), in a group buffer [GROUP][npos_pad * NH]:
//  * ROW32 (complex64 echoes, and every echo in the gradient pass): E0..E3
//    as FP32 pairs in two planes of 16-byte rows, (E0, E1) and (E2, E3), read
//    by two 16-byte loads.  A 16-byte load is served a quarter-warp (a 4 x 2
//    pixel block) per wavefront, and the rows one quarter-warp reads span fewer
//    than 8 half samples, so they fall in distinct bank groups of a plane.
//  * ROW24 (16-bit echoes, forward pass): the quadratic form, E0..E2 as FP32
//    pairs, (E0, E1) in a plane of 16-byte rows and E2 in a plane of 8-byte
//    rows, read by a 16-byte and an 8-byte load.  The 16-bit echo's error
//    budget admits the quadratic's interpolation error (7.5e-4 rms on echoes
//    band-limited to a quarter of the sample rate, against 3.7e-5 for the
//    cubic), and it saves a quarter of the expansion and a packed FMA a
//    pixel.
//  (Measured alternatives: one degree-5 polynomial per sample interval in
//  48-byte FP32 rows reads 1.5x the bytes per update and bound the kernel at
//  the shared-memory data pipe; 24-byte rows with E2, E3 in BF16 read by three
//  8-byte loads were 2.5 % slower, and the BF16 rounding made the forward
//  pass depart from the exact transpose of the adjoint by 2e-5; one 32-byte
//  row per position with its halves swapped every fourth row spent five
//  integer operations a pixel on the addresses.)


// FP64 vectors from the pair's sensors to the tile centre (X0, Y0, Z0):
// R_T = x0 - x_TX (ping i = q / C), R_R = x0 - x_RX (pair q).
struct PairGeo {
    double Tx, Ty, Tz, Rx, Ry, Rz;
};
__device__ __forceinline__ PairGeo pair_geo(const KParams& p, double X0, double Y0, double Z0, long long q, int i) {
    const double* t = p.tx + 3 * (size_t)i;
    const double* r = p.rx + 3 * (size_t)q;
    return PairGeo{X0 - t[0], Y0 - t[1], Z0 - t[2], X0 - r[0], Y0 - r[1], Z0 - r[2]};
}

// FP64 reference terms of a pair written to the record rc (field f at
// rc[f * stride]): 2R and |R|^2, |R| for transmitter and receiver, twice the
// fraction of u_ref = (tau_ref - t0) fs minus 1/2 (so that rounding
// 2(u - floor u_ref) - 1/2 to the nearest integer gives the half-sample index
// floor(2(u - floor u_ref))) and the carrier phase 2 pi fc tau_ref reduced to
// [-pi, pi) (radians).
// Returns the raw sample index of Farrow position 0, tap 0: floor(u_ref) - U - 3.
// LT0, LR0 >= 0: leg lengths at x0 in water metres (seabed refraction) that
// replace |R_T|, |R_R| in tau_ref; the differential fields stay the straight ones.
__device__ __forceinline__ int pair_record(const KParams& p, PairGeo G, float* rc, int stride, const double* v,
                                           double LT0 = -1.0, double LR0 = -1.0) {
    const double nT2 = G.Tx * G.Tx + G.Ty * G.Ty + G.Tz * G.Tz;
    const double nT = sqrt(nT2);
    if (v) {
        // receiver moving during reception (Sec. II-D): the tile centre's
        // echo arrives at tau with c tau = |R_T| + |R_R - v tau|; fixed-point
        // iteration (contraction |v|/c), then R_R from the receiver's position
        // at that time
        const double vx = v[0], vy = v[1], vz = v[2];
        rc[F_BRX * stride] = (float)(2.0 * G.Rx);
        rc[F_BRY * stride] = (float)(2.0 * G.Ry);
        rc[F_BRZ * stride] = (float)(2.0 * G.Rz);
        double tau = (nT + sqrt(G.Rx * G.Rx + G.Ry * G.Ry + G.Rz * G.Rz)) * p.inv_c;
        for (int it = 0; it < 12; ++it) {
            const double wx = G.Rx - vx * tau, wy = G.Ry - vy * tau, wz = G.Rz - vz * tau;
            const double t2 = (nT + sqrt(wx * wx + wy * wy + wz * wz)) * p.inv_c;
            const double step = fabs(t2 - tau);
            tau = t2;
            if (step <= 1e-16 * tau) break;
        }
        G.Rx -= vx * tau;
        G.Ry -= vy * tau;
        G.Rz -= vz * tau;
        rc[F_VX * stride] = (float)(vx * p.inv_c);
        rc[F_VY * stride] = (float)(vy * p.inv_c);
        rc[F_VZ * stride] = (float)(vz * p.inv_c);
        rc[F_RV * stride] = (float)((G.Rx * vx + G.Ry * vy + G.Rz * vz) * p.inv_c);
    }
    const double nR2 = G.Rx * G.Rx + G.Ry * G.Ry + G.Rz * G.Rz;
    const double nR = sqrt(nR2);
    const double tau = ((LT0 >= 0.0 ? LT0 : nT) + (LR0 >= 0.0 ? LR0 : nR)) * p.inv_c;
    double u = (tau - p.t0) * p.fs;
    u = fmin(fmax(u, -268435456.0), 268435456.0);  // keep sample coordinates in int range
    const double iref = floor(u);
    const double ph = p.fc * tau;
    rc[F_TX * stride] = (float)(2.0 * G.Tx);
    rc[F_TY * stride] = (float)(2.0 * G.Ty);
    rc[F_TZ * stride] = (float)(2.0 * G.Tz);
    rc[F_NT2 * stride] = (float)nT2;
    rc[F_NT * stride] = (float)nT;
    rc[F_RX * stride] = (float)(2.0 * G.Rx);
    rc[F_RY * stride] = (float)(2.0 * G.Ry);
    rc[F_RZ * stride] = (float)(2.0 * G.Rz);
    rc[F_NR2 * stride] = (float)nR2;
    rc[F_NR * stride] = (float)nR;
    rc[F_UF * stride] = (float)(2.0 * (u - iref) - 0.5);
    const double phf = ph - floor(ph);   // [0, 1) cycles -> [-pi, pi) rad
    rc[F_PH * stride] = (float)(2.0 * M_PI * (phf < 0.5 ? phf : phf - 1.0));
    return (int)iref - p.U - 3;
}

// The same pair vectors and reference terms in double-float arithmetic (the
// stop-and-hop model with straight legs): R = x0 - sensor to about 48 bits,
// |R|^2 and |R| (|R| to a few units of 2^-45 relative), the two-way path, u_ref
// and the carrier phase.  The outputs are the FP32 fields pair_record writes;
// the phase and the fraction of u_ref keep about 1e-10 of a cycle / sample.
struct PairGeoDF {
    dfl T[3], R[3];
};
__device__ __forceinline__ PairGeoDF pair_geo_df(const KParams& p, const dfl* X0, int q, int i) {
    const float2* t = p.txs + 3 * (size_t)i;
    const float2* r = p.rxs + 3 * (size_t)q;
    PairGeoDF G;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float2 tk = t[k], rk = r[k];
        G.T[k] = df_add(X0[k], dfl{-tk.x, -tk.y});
        G.R[k] = df_add(X0[k], dfl{-rk.x, -rk.y});
    }
    return G;
}
__device__ __forceinline__ int pair_record_df(const KParams& p, const PairGeoDF& G, float* rc, int stride) {
    const dfl nT2 = df_add(df_add(df_mul(G.T[0], G.T[0]), df_mul(G.T[1], G.T[1])), df_mul(G.T[2], G.T[2]));
    const dfl nR2 = df_add(df_add(df_mul(G.R[0], G.R[0]), df_mul(G.R[1], G.R[1])), df_mul(G.R[2], G.R[2]));
    const dfl nT = df_sqrt(nT2), nR = df_sqrt(nR2);
    const dfl path = df_add(nT, nR);                                   // c tau_ref [m]
    const dfl kfs{p.k_fs_c.x, p.k_fs_c.y}, kt0{p.k_t0fs.x, p.k_t0fs.y}, kfc{p.k_fc_c.x, p.k_fc_c.y};
    dfl u = df_add(df_mul(path, kfs), df_neg(kt0));                   // (tau - t0) fs
    u.hi = fminf(fmaxf(u.hi, -268435456.0f), 268435456.0f);            // keep sample coordinates in int range
    // floor(u) and its fraction from both parts
    const float f0 = floorf(u.hi);
    const float t = __fadd_rn(__fsub_rn(u.hi, f0), u.lo);
    const float f1 = floorf(t);
    const int iref = (int)f0 + (int)f1;
    const float frac = __fsub_rn(t, f1);
    // carrier phase fc tau_ref mod 1 -> [-pi, pi) rad
    const dfl ph = df_mul(path, kfc);
    const float pt = __fadd_rn(__fsub_rn(ph.hi, floorf(ph.hi)), ph.lo);
    float pf = __fsub_rn(pt, floorf(pt));
    pf = pf < 0.5f ? pf : __fsub_rn(pf, 1.0f);
    rc[F_TX * stride] = 2.0f * df_float(G.T[0]);
    rc[F_TY * stride] = 2.0f * df_float(G.T[1]);
    rc[F_TZ * stride] = 2.0f * df_float(G.T[2]);
    rc[F_NT2 * stride] = df_float(nT2);
    rc[F_NT * stride] = df_float(nT);
    rc[F_RX * stride] = 2.0f * df_float(G.R[0]);
    rc[F_RY * stride] = 2.0f * df_float(G.R[1]);
    rc[F_RZ * stride] = 2.0f * df_float(G.R[2]);
    rc[F_NR2 * stride] = df_float(nR2);
    rc[F_NR * stride] = df_float(nR);
    rc[F_UF * stride] = fmaf(2.0f, frac, -0.5f);
    rc[F_PH * stride] = pf * TWO_PI_F;
    return iref - p.U - 3;
}

// Beam class of one sensor for the whole tile (FP32, conservative):
// 0 = no pixel of the tile can be seen, 2 = every pixel is seen, 1 = test per
// pixel.  The tile's pixel-centre box, seen through the linear map
// (b_x, side b_y) = (c0 . w, side c1 . w), is a convex polygon spanned by the
// corners: it misses the beam wedge |b_x| <= k b_y if all corners lie beyond
// one edge or behind the sensor, and lies inside if all corners do.  Margins
// of 1e-5 relative keep both decisions on the safe side of FP32 rounding.
template <bool DIM3>
__device__ __forceinline__ int beam_class(const KParams& p, float vx, float vy, float vz, const float* c) {
    bool all_right = true, all_left = true, all_behind = true, all_in = true;
    const float k = p.beam_tan;
#pragma unroll
    for (int n = 0; n < (DIM3 ? 8 : 4); ++n) {
        const float wx = vx + ((n & 1) ? p.hx : -p.hx);
        const float wy = vy + ((n & 2) ? p.hy : -p.hy);
        const float wz = vz + (DIM3 ? ((n & 4) ? p.hz : -p.hz) : 0.f);
        const float bx = fmaf(c[0], wx, fmaf(c[1], wy, c[2] * wz));
        const float by = p.beam_side * fmaf(c[3], wx, fmaf(c[4], wy, c[5] * wz));
        const float mu = 1e-5f * (fabsf(bx) + fabsf(by)) + 1e-6f;
        all_right = all_right && (bx - k * by > mu);
        all_left = all_left && (-bx - k * by > mu);
        all_behind = all_behind && (by < -mu);
        all_in = all_in && (fabsf(bx) - k * by < -mu) && (by > mu);
    }
    if (all_right || all_left || all_behind) return 0;
    return all_in ? 2 : 1;
}

// Per-pixel beam test (FP32), w = sensor-to-pixel vector.
__device__ __forceinline__ bool beam_sees(const KParams& p, float wx, float wy, float wz, const float* c) {
    const float bx = fmaf(c[0], wx, fmaf(c[1], wy, c[2] * wz));
    const float by = p.beam_side * fmaf(c[3], wx, fmaf(c[4], wy, c[5] * wz));
    return by > 0.f && fabsf(bx) <= p.beam_tan * by;
}

// ---------------------------------------------------------------------------
// Seabed refraction (Sec. III-B).  Interface z = z_int, water above (speed c),
// sediment below (speed c_s), n = c / c_s.  A leg from a sensor at height
// a = z_int - s_z > 0 above the interface to a pixel at depth b = x_z - z_int > 0
// below it, at horizontal distance rho, crosses the interface at horizontal
// distance xi from the sensor (Fermat: the travel time is stationary, which
// is Snell's law) and has the length, in water metres,
//   L = |W| + n |V|,  |W| = sqrt(xi^2 + a^2),  |V| = sqrt(sigma^2 + b^2),  sigma = rho - xi.
// The crossing is solved in the slope v of the leg in the faster medium: with
// r = max(n, 1/n), A the depth of the faster leg and B that of the slower one
// (A = b, B = a for a faster sediment, n < 1), the faster leg runs A v and the
// slower one B v q, q = (r^2 + (r^2 - 1) v^2)^(-1/2), so v solves
//   F(v) = A v + B v q - rho = 0,   F'(v) = A + B r^2 q^3.
// F increases and is concave on v >= 0; the slower leg runs less than
// B / sqrt(r^2 - 1), so A v >= rho - B / sqrt(r^2 - 1) (and A v <= rho).
// Newton's method from the left of the root increases monotonically to it.
//
// Each pair carries, per leg, the crossing at a reference point x_r below the
// interface (the tile centre, or the deepest pixel layer when the centre is
// above it); a pixel's leg is then evaluated as a difference from x_r with
// the identity |U + e| - |U| = (2U.e + |e|^2) / (|U + e| + |U|) for each of
// the two segments, where the crossing point only has to be close to the
// stationary one (the length is stationary there: a crossing error e costs
// L'' e^2 / 2).
// ---------------------------------------------------------------------------

// Crossing slope in the faster medium by Newton's method from the left bound
// (FP32, producer).  Returns v; q and Sd = B r^2 q^3 at v.
__device__ __forceinline__ float refr_solve(const KParams& p, float A, float B, float rho, float& q, float& Sd) {
    const float flo = fmaxf(fmaf(-B, p.refr_isM, rho), 0.f);
    const float vlo = flo / A;
    float v = vlo, prev = 3.0e38f;
    for (int it = 0; it < 64; ++it) {
        q = rsqrtf(fmaf(p.refr_M, v * v, p.refr_r2));
        const float F = fmaf(A, v, fmaf(B * v, q, -rho));
        Sd = B * p.refr_r2 * (q * q * q);
        const float dv = F / (Sd + A);
        v = fmaxf(v - dv, vlo);
        // stop at convergence, or when rounding stops the steps from shrinking
        const float step = fabsf(dv) * fmaxf(A, Sd);
        if (step <= 2e-7f * (rho + B) || step >= prev) break;
        prev = step;
    }
    q = rsqrtf(fmaf(p.refr_M, v * v, p.refr_r2));
    Sd = B * p.refr_r2 * (q * q * q);
    return v;
}

// Reference terms of one leg (producer): hx, hy = horizontal part of x_r - s,
// a = sensor height above the interface, br = depth of x_r below it (FP64).
// Writes rc[RF_A .. RF_DFB] (stride) and returns L(x_r) in water metres.  The
// crossing xi_r is solved in FP32 and L(x_r), sigma_r, |W_r|, |V_r| are then
// evaluated in FP64 at exactly that crossing, so that the per-pixel
// differences start from a consistent reference.  f_r is the faster leg's
// run and df/drho, df/db its derivatives (implicit function of F = 0): the
// per-pixel initial guess.
__device__ __forceinline__ double refr_leg_ref(const KParams& p, double hx, double hy, double a, double br,
                                               float* rc, int stride) {
    const double rho2 = hx * hx + hy * hy;
    const double rho = sqrt(rho2);
    const bool fsed = p.refr_fast_sed;
    const float A = (float)(fsed ? br : a), B = (float)(fsed ? a : br);
    const float rhof = (float)rho;
    float q, Sd;
    const float v = refr_solve(p, A, B, rhof, q, Sd);
    const float fast = A * v, slow = (B * v) * q;
    // the crossing from the better-determined of the two runs
    float xi_f = fsed ? (A < Sd ? rhof - fast : slow) : (A < Sd ? fast : rhof - slow);
    xi_f = fminf(fmaxf(xi_f, 0.f), rhof);
    const double xi = (double)xi_f, sig = rho - xi;
    const double W = sqrt(xi * xi + a * a), V = sqrt(sig * sig + br * br);
    const float Fd = Sd + A;
    rc[RF_A * stride] = (float)a;
    rc[RF_RHO2 * stride] = (float)rho2;
    rc[RF_RHO * stride] = rhof;
    rc[RF_XI * stride] = xi_f;
    rc[RF_SIG * stride] = (float)sig;
    rc[RF_W * stride] = (float)W;
    rc[RF_V * stride] = (float)V;
    rc[RF_F * stride] = fsed ? (float)sig : xi_f;
    rc[RF_DFR * stride] = A / Fd;
    rc[RF_DFB * stride] = fsed ? v * (1.f - A / Fd) : -(A * v) * q / Fd;
    return W + p.refr_n * V;
}

// The refraction blocks of a pair's record (producer, FP64): per leg with
// the sensor above the interface and some pixel layer of the tile below it,
// the crossing at x_r = (x0, y0, Zr) and the offsets K_r, K_s of the
// refracted and the straight slots from the leg at x0 (refracted if x0 is
// below the interface); zeros otherwise.  Fields at rc[(F_RREF + f) stride]
// (receiver) and rc[(F_TREF + f) stride] (transmitter).  Returns the
// FL_*_REFR flags and the legs' lengths at x0 in water metres (LT0, LR0).
__device__ __forceinline__ int refr_pair_blocks(const KParams& p, const PairGeo& G, double tz, double rz,
                                                unsigned bmask, double Zr, double Zc, float* rc, int stride,
                                                double& LT0, double& LR0) {
    int rfl = 0;
#pragma unroll
    for (int leg = 0; leg < 2; ++leg) {
        const double hx = leg ? G.Tx : G.Rx, hy = leg ? G.Ty : G.Ry, hz = leg ? G.Tz : G.Rz;
        const double sz = leg ? tz : rz;
        const double straight = sqrt(hx * hx + hy * hy + hz * hz);
        float* blk = rc + (leg ? F_TREF : F_RREF) * stride;
        double L0 = straight;
        if (bmask && sz < p.z_int) {
            const double Lr = refr_leg_ref(p, hx, hy, p.z_int - sz, Zr - p.z_int, blk, stride);
            if (Zc > p.z_int) L0 = Lr;
            blk[RF_KR * stride] = (float)(Lr - L0);
            blk[RF_KS * stride] = (float)(straight - L0);
            rfl |= leg ? FL_T_REFR : FL_R_REFR;
        } else {
#pragma unroll
            for (int f = 0; f < RF_N; ++f) blk[f * stride] = 0.f;
        }
        (leg ? LT0 : LR0) = L0;
    }
    return rfl;
}

// Refracted leg of one pixel minus the leg at x_r, plus K_r (consumers, FP32).
// r0, r1, r2: the leg's record blocks; rho = rho_r + drho: the pixel's
// horizontal distance; b = b_r + db: its depth below the interface.  Also
// returns the unit vector from the sensor to the crossing point, as
// (uxi, ua) = (xi, a) / |W| (horizontal run and height over the segment's
// length): the derivative of the leg's length with respect to the sensor's
// position is minus that vector (the length is stationary in the crossing).
__device__ __forceinline__ float refr_leg_diff(const KParams& p, const float4 r0, const float4 r1, const float4 r2,
                                               float rho, float drho, float b, float db, float br, float& uxi,
                                               float& ua) {
    const float a = r0.x;
    const bool fsed = p.refr_fast_sed;
    const float A = fsed ? b : a, B = fsed ? a : b;
    const float flo = fmaxf(fmaf(-B, p.refr_isM, rho), 0.f);
    float f = fmaf(r2.x, drho, fmaf(r2.y, db, r1.w));   // predicted run of the faster leg
    f = fminf(fmaxf(f, flo), rho);
    const float iA = rcp_sfu(A);
    const float vlo = flo * iA;
    float v = f * iA, Sd = 0.f;
    for (int it = 0; it < 16; ++it) {
        const float q = rsqrt_sfu(fmaf(p.refr_M, v * v, p.refr_r2));
        const float F = fmaf(A, v, fmaf(B * v, q, -rho));
        Sd = B * p.refr_r2 * (q * q * q);
        const float dv = F * rcp_sfu(Sd + A);
        v = fmaxf(v - dv, vlo);
        // the crossing moved by less than the tolerance
        if (fabsf(dv) * fminf(A, Sd) < p.refr_tol) break;
    }
    const float q = rsqrt_sfu(fmaf(p.refr_M, v * v, p.refr_r2));
    const float fast = A * v, slow = (B * v) * q;
    const bool use_fast = A < Sd;
    float dxi, dsig;
    if (fsed) {   // faster leg in the sediment: its run is sigma
        dsig = use_fast ? fast - r1.x : drho - (slow - r0.w);
        dxi = drho - dsig;
    } else {      // faster leg in the water: its run is xi
        dxi = use_fast ? fast - r0.w : drho - (slow - r1.x);
        dsig = drho - dxi;
    }
    const float xi = r0.w + dxi, sg = r1.x + dsig;
    const float W2 = fmaf(xi, xi, a * a), V2 = fmaf(sg, sg, b * b);
    const float iW = rsqrt_sfu(W2);
    uxi = xi * iW;
    ua = a * iW;
    const float Dw = fmaf(W2, iW, r1.y), Ds = fmaf(V2, rsqrt_sfu(V2), r1.z);   // |W| + |W_r|, |V| + |V_r|
    const float Nw = dxi * fmaf(2.f, r0.w, dxi);                                         // |W|^2 - |W_r|^2
    const float Ns = p.refr_nf * fmaf(dsig, fmaf(2.f, r1.x, dsig), db * (br + b));        // n (|V|^2 - |V_r|^2)
    return fmaf(fmaf(Nw, Ds, Ns * Dw), rcp_sfu(Dw * Ds), r2.z);
}

// The same for two pixels at once (slots 2k, 2k+1), packed FP32x2: two
// Newton steps for both, further steps only while some lane of the warp has
// not converged (callers are warp-uniform here); the last step's q is kept
// for the slower leg's run (the crossing moves by less than the tolerance in
// that step, and the length is stationary in it).
__device__ __forceinline__ float2 refr_leg_diff2(const KParams& p, const float4 r0, const float4 r1,
                                                 const float4 r2, float2 rho, float2 drho, float2 b, float2 db,
                                                 float br, float2& uxi, float2& ua) {
    const float a = r0.x;
    const bool fsed = p.refr_fast_sed;
    const float2 a2 = make_float2(a, a);
    const float2 A = fsed ? b : a2, B = fsed ? a2 : b;
    const float2 zero = make_float2(0.f, 0.f);
    const float2 isM = make_float2(p.refr_isM, p.refr_isM), M2 = make_float2(p.refr_M, p.refr_M);
    const float2 r22 = make_float2(p.refr_r2, p.refr_r2);
    const float2 flo = fmax2(ffma2(make_float2(-B.x, -B.y), isM, rho), zero);
    float2 f = ffma2(make_float2(r2.x, r2.x), drho, ffma2(make_float2(r2.y, r2.y), db, make_float2(r1.w, r1.w)));
    f = fmin2(fmax2(f, flo), rho);
    const float2 iA = make_float2(rcp_sfu(A.x), rcp_sfu(A.y));
    const float2 vlo = fmul2(flo, iA);
    float2 v = fmul2(f, iA), q = zero, Sd = zero, dv = zero;
    const float2 Br2 = fmul2(B, r22);
    auto step = [&]() {
        const float2 t = ffma2(M2, fmul2(v, v), r22);
        q = make_float2(rsqrt_sfu(t.x), rsqrt_sfu(t.y));
        const float2 F = ffma2(A, v, ffma2(fmul2(B, v), q, make_float2(-rho.x, -rho.y)));
        Sd = fmul2(Br2, fmul2(q, fmul2(q, q)));
        const float2 den = fadd2(Sd, A);
        dv = fmul2(F, make_float2(rcp_sfu(den.x), rcp_sfu(den.y)));
        v = fmax2(fsub2(v, dv), vlo);
    };
    auto converged = [&]() {
        return fabsf(dv.x) * fminf(A.x, Sd.x) < p.refr_tol && fabsf(dv.y) * fminf(A.y, Sd.y) < p.refr_tol;
    };
    step();
    step();
    for (int it = 2; it < 16 && __any_sync(__activemask(), !converged()); ++it) step();
    const float2 fast = fmul2(A, v), slow = fmul2(fmul2(B, v), q);
    float2 dxi, dsig;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const bool use_fast = (j ? A.y < Sd.y : A.x < Sd.x);
        const float fj = j ? fast.y : fast.x, sj = j ? slow.y : slow.x, dr = j ? drho.y : drho.x;
        float& dx = j ? dxi.y : dxi.x;
        float& ds = j ? dsig.y : dsig.x;
        if (fsed) {
            ds = use_fast ? fj - r1.x : dr - (sj - r0.w);
            dx = dr - ds;
        } else {
            dx = use_fast ? fj - r0.w : dr - (sj - r1.x);
            ds = dr - dx;
        }
    }
    const float2 xi = fadd2(make_float2(r0.w, r0.w), dxi), sg = fadd2(make_float2(r1.x, r1.x), dsig);
    const float2 W2 = ffma2(xi, xi, make_float2(a * a, a * a)), V2 = ffma2(sg, sg, fmul2(b, b));
    const float2 iW = make_float2(rsqrt_sfu(W2.x), rsqrt_sfu(W2.y));
    uxi = fmul2(xi, iW);
    ua = fmul2(make_float2(a, a), iW);
    const float2 Dw = ffma2(W2, iW, make_float2(r1.y, r1.y));
    const float2 Ds = ffma2(V2, make_float2(rsqrt_sfu(V2.x), rsqrt_sfu(V2.y)), make_float2(r1.z, r1.z));
    const float2 two = make_float2(2.f, 2.f);
    const float2 Nw = fmul2(dxi, ffma2(two, make_float2(r0.w, r0.w), dxi));
    const float2 Ns = fmul2(make_float2(p.refr_nf, p.refr_nf),
                            ffma2(dsig, ffma2(two, make_float2(r1.x, r1.x), dsig), fmul2(db, fadd2(make_float2(br, br), b))));
    const float2 num = ffma2(Nw, Ds, fmul2(Ns, Dw)), den = fmul2(Dw, Ds);
    return ffma2(num, make_float2(rcp_sfu(den.x), rcp_sfu(den.y)), make_float2(r2.z, r2.z));
}

// Horizontal distance of a pixel from a sensor, rho = rho_r + drho, from
// qh = 2 h_r.d_h + |d_h|^2 (h_r: horizontal part of x_r - s; d_h the
// pixel's horizontal offset from x_r).
// (A pixel straight below the sensor has rho = 0, which rounding may take
// slightly negative: clamped.)
__device__ __forceinline__ void refr_rho(const float4 r0, float qh, float& rho, float& drho) {
    const float rho2 = r0.y + qh;
    rho = rho2 > 0.f ? rho2 * rsqrt_sfu(rho2) : 0.f;
    const float den = rho + r0.z;
    drho = den > 0.f ? qh * rcp_sfu(den) : 0.f;
}

// Depth of pixel layer iz, formed as the oracle forms pixel coordinates
// (z0 + iz dz, no fused multiply-add), so that both take the same decision at
// the interface.
__device__ __forceinline__ double layer_z(const KParams& p, int iz) {
    return __dadd_rn(p.z0, __dmul_rn((double)iz, p.dz));
}

// Seabed refraction, per tile (FP64): the slots (pixel layers in 3D; all of
// them in 2D) strictly below the interface, as a bit mask, and the depth Zr
// of the reference point x_r = (x0, y0, Zr): the centre Zc if it is below,
// else the deepest layer.
template <bool DIM3>
__device__ __forceinline__ unsigned refr_tile_layers(const KParams& p, int tz0, double Zc, double& Zr) {
    unsigned bm = 0u;
    double zdeep = -1.0e300;
#pragma unroll 1
    for (int s = 0; s < PX; ++s) {
        const double zs = DIM3 ? layer_z(p, tz0 + s) : p.z0;
        if (zs > p.z_int) {
            bm |= 1u << s;
            zdeep = fmax(zdeep, zs);
        }
    }
    Zr = Zc > p.z_int ? Zc : zdeep;
    return bm;
}

// Pixel offsets d from the tile centre: the fixed part of |d|^2 and of 2R.d
// (x, and y in 3D; the varying coordinate is added per slot as
// a = fma(2R_var, d_var, fma(d_var, d_var, fixed_d2)) + fixed_dot).  Written
// with explicit roundings so that every kernel evaluates the same FP32 path.
template <bool DIM3>
__device__ __forceinline__ float fixed_d2(float dx, float dy) {
    return DIM3 ? fmaf(dx, dx, __fmul_rn(dy, dy)) : __fmul_rn(dx, dx);
}
template <bool DIM3>
__device__ __forceinline__ float fixed_dot(float tx, float ty, float dx, float dy) {
    return DIM3 ? fmaf(tx, dx, __fmul_rn(ty, dy)) : __fmul_rn(tx, dx);
}

// Shared-memory size and launch geometry, host side.
struct Layout {
    int U, npos, seglen, align, slot_bytes;
    size_t smem;
};

// Shared-memory layout (in this order): echo segments, Farrow rows, records,
// coefficients, reduction scratch, group descriptors, mbarriers, abort flag.
// Every part before the descriptors has a size that is a multiple of 16
// bytes (slot_bytes: of 128; the Farrow rows of a sample position: 64 or 48
// bytes; records of a multiple of 4 floats),
// so the 16-byte descriptor loads and stores are aligned.
static_assert((NRS * PAIRS * NREC * 4) % 16 == 0 && (NRS * PAIRS * NREC_REFR * 4) % 16 == 0 &&
                  (NH * TAPS * NP * 4) % 16 == 0 && (NCW * 4 * 8) % 16 == 0 && (NH * ROW32) % 16 == 0 &&
                  (NH * ROW24) % 16 == 0,
              "shared-memory parts must keep 16-byte alignment");
// row_bytes: ROW32 or ROW24
// positions per pair of the Farrow ring in the fixed-layout kernels (a
// multiple of RUN; tiles of 1.5 cm pixels at 40 kHz need 57)
constexpr int NPOS_FIXED = 60;
static_assert(NPOS_FIXED % RUN == 0, "whole expansion runs");

inline size_t smem_bytes(int slot_bytes, int npos_pad, int nrec, int row_bytes) {
    return (size_t)NSEG * PAIRS * slot_bytes                   // echo segments
           + (size_t)NBUF * GROUP * npos_pad * NH * row_bytes  // Farrow rows
           + (size_t)NRS * PAIRS * nrec * 4                    // records
           + (size_t)NH * TAPS * NP * 4                        // coefficients
           + (size_t)NCW * 4 * 8                        // cross-warp reduction (gradient)
           + (size_t)NBUF * 16                          // group descriptors
           + (size_t)(NSEG + NRS + 2 * NBUF) * 8 + 16;  // mbarriers, abort flag
}

// ----------------------------------------------------------------------------
// BEAM: the beam field of view is on (culling in the producer, per-pixel tests
// in tiles on a beam edge); without it every candidate pair is computed.
// MOTION: the receivers move during reception (per-ping velocity).
// REFRACT: seabed refraction (forward pass, without BEAM and MOTION).
// FIXED: the Farrow ring has NPOS_FIXED positions per pair (p.npos_pad ==
// NPOS_FIXED), so the second FP32 plane sits at a constant offset from the
// first and a consumer addresses both with one computed address.
template <typename ET, bool DIM3, int MODE, bool BEAM, bool MOTION, bool REFRACT = false, bool FIXED = false>
__global__ void __launch_bounds__(NTHREADS, 2) tdbp_kernel(const __grid_constant__ CUtensorMap tmap, const KParams p) {
    using T = Tile<DIM3>;
    static_assert(!REFRACT || (!BEAM && !MOTION), "refraction: without the beam or receiver motion");
    constexpr int KREC = REFRACT ? NREC_REFR : NREC;   // record fields
    // FP16 Farrow rows for 16-bit echoes in the forward pass; otherwise rows
    // of FP32 E0, E1 and BF16 E2, E3
    constexpr bool E16 = (MODE == MODE_FORWARD) && (sizeof(ET) == 4);
    constexpr int ROWB = E16 ? ROW24 : ROW32;
    constexpr int NPK = E16 ? NQ : NP;                 // coefficients of a row (cubic or quadratic)
    extern __shared__ __align__(1024) unsigned char smem[];
    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;

    unsigned char* seg = smem;                                           // [NSEG][PAIRS] echo segments
    unsigned char* ebuf = seg + (size_t)NSEG * PAIRS * p.slot_bytes;     // [NBUF][GROUP] Farrow rows
    const int npos_pad = FIXED ? NPOS_FIXED : p.npos_pad;
    const int ebuf_pair = npos_pad * NH * ROWB;       // positions padded to whole expansion runs
    float* rec = reinterpret_cast<float*>(ebuf + (size_t)NBUF * GROUP * ebuf_pair);   // [NRS][PAIRS][KREC]
    float* coef_s = rec + NRS * PAIRS * KREC;                            // [NH][TAPS][NP]
    // every part so far has a size that is a multiple of 16 bytes (see smem_bytes)
    double* wred = reinterpret_cast<double*>(coef_s + NH * TAPS * NP);    // [NCW][4]
    // [NBUF] group descriptors (written before, read after the efull barrier)
    int4* gdesc = reinterpret_cast<int4*>(wred + NCW * 4);
    uint64_t* full = reinterpret_cast<uint64_t*>(gdesc + NBUF);          // [NSEG] copies landed + records
    uint64_t* rempty = full + NSEG;                                      // [NRS] consumers done with records
    uint64_t* efull = rempty + NRS;                                      // [NBUF] Farrow rows written
    uint64_t* eempty = efull + NBUF;                                     // [NBUF] Farrow rows read
    volatile int* abort_flag = reinterpret_cast<volatile int*>(eempty + NBUF);

    const int ntiles = p.tiles_x * p.tiles_y * p.tiles_z;
    const int tile = blockIdx.x % ntiles;
    const int split = blockIdx.x / ntiles;
    const int tx0 = (tile % p.tiles_x) * T::TX;
    const int ty0 = ((tile / p.tiles_x) % p.tiles_y) * T::TY;
    const int tz0 = (tile / (p.tiles_x * p.tiles_y)) * T::TZ;
    // candidate pairs of this CTA: whole pings [ping0, ping1)
    const int ping0 = min(p.P, split * p.pings_per_split);
    const int ping1 = min(p.P, ping0 + p.pings_per_split);
    const long long q0 = (long long)ping0 * p.C;
    const long long q1 = (long long)ping1 * p.C;
    const double cx = tx0 + 0.5 * (T::TX - 1), cy = ty0 + 0.5 * (T::TY - 1), cz = tz0 + 0.5 * (T::TZ - 1);
    const double Zc = p.z0 + (DIM3 ? cz * p.dz : 0.0);   // tile centre depth
    // seabed refraction: the slots (pixel layers in 3D; all of them in 2D)
    // strictly below the interface, and the depth Zr of the reference point
    // x_r = (x0, y0, Zr): the centre if it is below, else the deepest layer
    // (one thread derives them in FP64 and hands them to the block through
    // shared memory: recomputing FP64 terms at their uses would load the
    // slow FP64 pipe)
    __shared__ unsigned s_bmask;
    __shared__ double s_zr;
    if (REFRACT && tid == 0) {
        double zr;
        s_bmask = refr_tile_layers<DIM3>(p, tz0, Zc, zr);
        s_zr = zr;
    }

    if (tid == 0) {
        for (int s = 0; s < NSEG; ++s) mbar_init(smem_u32(&full[s]), 1);
        for (int s = 0; s < NRS; ++s) mbar_init(smem_u32(&rempty[s]), NCW);
        for (int b = 0; b < NBUF; ++b) {
            mbar_init(smem_u32(&efull[b]), 1);
            mbar_init(smem_u32(&eempty[b]), NCW);
        }
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (tid < NH * TAPS * NPK) coef_s[tid] = E16 ? (&p.coef->q[0][0][0])[tid] : (&p.coef->c[0][0][0])[tid];
    __syncthreads();
    const unsigned bmask = REFRACT ? s_bmask : 0u;
    const double Zr = REFRACT ? s_zr : Zc;

    if (warp == 0) {
        // ================= producer =================
        // Stages of up to PAIRS (ping, channel) pairs: the producer scans the
        // candidates 32 at a time, drops those whose beams cannot see the tile,
        // writes each surviving pair's record and issues the copy of its echo
        // segment (announced on the stage's full barrier).  It fills stage k + 1
        // before it expands stage k, group by group, into the Farrow buffers the
        // consumers read; a descriptor per buffer tells them which pairs it holds.
        const double X0 = p.x0 + cx * p.dx, Y0 = p.y0 + cy * p.dy, Z0 = Zc;
        // double-float reference terms for the stop-and-hop straight-path model
        constexpr bool DFREC = !MOTION && !REFRACT;
        dfl X0d[3];
        {
            const float2 a = df_split(X0), b = df_split(Y0), c = df_split(Z0);
            X0d[0] = dfl{a.x, a.y};
            X0d[1] = dfl{b.x, b.y};
            X0d[2] = dfl{c.x, c.y};
        }
        const uint32_t seg_bytes = (uint32_t)p.seglen * (uint32_t)sizeof(ET);
        unsigned n_cand = 0, n_act = 0, n_edge = 0;   // this lane's culling counts
        bool failed = false;
        auto fail = [&]() {
            if (lane == 0) {
                *abort_flag = 1;
                atomicOr(p.status, DEV_TIMEOUT);
            }
            __syncwarp();
            failed = true;
        };
        // candidate scan state (persists across stages)
        long long qb = q0;
        unsigned amask = 0u;
        int nact = 0, done = 0;
        PairGeo Gv{};
        PairGeoDF Gd{};
        int flv = FL_TX_FULL | FL_RX_FULL, iv = 0;
        long long qv = 0;
        float rc6[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        auto load_batch = [&]() {
            qv = qb + lane;
            const bool valid = qv < q1;
            iv = valid ? (int)((unsigned)qv / (unsigned)p.C) : 0;   // pairs < 2^31
            flv = FL_TX_FULL | FL_RX_FULL;
            bool active = valid;
            if (valid) {
                float gt[3], gr[3];   // FP32 pair vectors for the beam tests
                if constexpr (DFREC) {
                    Gd = pair_geo_df(p, X0d, (int)qv, iv);
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        gt[k] = df_float(Gd.T[k]);
                        gr[k] = df_float(Gd.R[k]);
                    }
                } else {
                    Gv = pair_geo(p, X0, Y0, Z0, qv, iv);
                    gt[0] = (float)Gv.Tx; gt[1] = (float)Gv.Ty; gt[2] = (float)Gv.Tz;
                    gr[0] = (float)Gv.Rx; gr[1] = (float)Gv.Ry; gr[2] = (float)Gv.Rz;
                }
                if (BEAM) {
#pragma unroll
                    for (int t = 0; t < 6; ++t) rc6[t] = p.rotc[6 * (size_t)iv + t];
                    const int ct_ = beam_class<DIM3>(p, gt[0], gt[1], gt[2], rc6);
                    const int cr_ = beam_class<DIM3>(p, gr[0], gr[1], gr[2], rc6);
                    active = ct_ != 0 && cr_ != 0;
                    flv = (ct_ == 2 ? FL_TX_FULL : 0) | (cr_ == 2 ? FL_RX_FULL : 0);
                }
            }
            n_cand += valid ? 1u : 0u;
            n_act += active ? 1u : 0u;
            n_edge += (active && flv != (FL_TX_FULL | FL_RX_FULL)) ? 1u : 0u;
            amask = __ballot_sync(0xffffffffu, active);
            nact = __popc(amask);
            done = 0;
            qb += PAIRS;
        };
        // fills stage k; returns its pair count, sets last when no candidate remains
        auto fill = [&](int k, bool& last) -> int {
            const int rs = k % NRS, ss = k % NSEG;
            if (k >= NRS && !mbar_wait_bounded(smem_u32(&rempty[rs]), ((k / NRS) - 1) & 1, p.wait_ns)) fail();
            // the segment slot was last read by this warp's expansion of stage k - NSEG:
            // order those generic-proxy reads before the copies that overwrite it
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            int cnt = 0;
            const uint32_t bar = smem_u32(&full[ss]);
            while (!failed && cnt < PAIRS) {
                if (done >= nact) {
                    if (qb >= q1) break;
                    load_batch();
                    continue;
                }
                const int take = min(PAIRS - cnt, nact - done);
                const bool act = (amask >> lane) & 1u;
                const int rank = __popc(amask & ((1u << lane) - 1u));
                if (act && rank >= done && rank < done + take) {
                    const int slot = cnt + rank - done;
                    float* rc = rec + (rs * PAIRS + slot) * KREC;
                    double LT0 = -1.0, LR0 = -1.0;
                    int rfl = 0;
                    if constexpr (REFRACT)
                        rfl = refr_pair_blocks(p, Gv, p.tx[3 * (size_t)iv + 2], p.rx[3 * (size_t)qv + 2], bmask, Zr,
                                               Zc, rc, 1, LT0, LR0);
                    int base;
                    if constexpr (DFREC)
                        base = pair_record_df(p, Gd, rc, 1);
                    else
                        base = pair_record(p, Gv, rc, 1, MOTION ? p.vel + 3 * (size_t)iv : nullptr, LT0, LR0);
                    const int seg_start = base - (((base % p.seg_align) + p.seg_align) % p.seg_align);
                    rc[F_OFF] = __int_as_float(base - seg_start);
                    rc[F_SCALE] = p.scale ? p.scale[qv] : 1.0f;
                    rc[F_PING] = __int_as_float(iv);
                    rc[F_FLAGS] = __int_as_float(REFRACT ? rfl : flv);
                    if constexpr (!REFRACT) {
#pragma unroll
                        for (int t = 0; t < 6; ++t) rc[F_C0X + t] = rc6[t];
                    }
                    mbar_expect_tx(bar, seg_bytes);
                    if (!p.skip_copies)
                        tma_load_2d(smem_u32(seg + ((size_t)ss * PAIRS + slot) * p.slot_bytes), &tmap, seg_start,
                                    (int32_t)qv, bar);
                }
                cnt += take;
                done += take;
            }
            last = qb >= q1 && done >= nact;
            __syncwarp();
            if (lane == 0) mbar_arrive(bar);
            return cnt;
        };

        // expansion: a lane computes the powers of one half of a run of RUN
        // sample positions and writes them as whole rows of a plane.  Cubic rows:
        // lane = (plane, run slot, half), 2 x 8 x 2, each lane computing the two
        // powers of its plane, (E0, E1) or (E2, E3).  Quadratic rows (16-bit
        // echoes): lane = (run slot, half), 16 x 2, each lane computing E0, E1, E2,
        // so that a 16-bit sample is converted by two lanes.  A quarter-warp
        // writes the four runs of one pair (when the span takes four runs): rows
        // 30 apart, which fall in distinct bank groups.
        constexpr int NPL = E16 ? NQ : 2;         // powers per lane
        constexpr int RSLOTS = E16 ? 16 : 8;
        const int Eh = lane & 1, Erun = (lane >> 1) & (RSLOTS - 1), Eq = E16 ? 0 : lane >> 4;
        const int runs_per_pair = (p.npos + RUN - 1) / RUN;
        float2 cc2[NPL][TAPS];
#pragma unroll
        for (int q = 0; q < NPL; ++q)
#pragma unroll
            for (int m = 0; m < TAPS; ++m) {
                const float c = coef_s[(Eh * TAPS + m) * NPK + 2 * Eq + q];
                cc2[q][m] = make_float2(c, c);
            }
        // the first plane holds (E0, E1) in 16-byte rows, the second (E2, E3) in
        // 16-byte rows (cubic) or E2 in 8-byte rows (quadratic)
        const int plane1 = npos_pad * NH * 16;          // bytes of a pair's first plane
        const int e_off = Eq * plane1;
        int G = 0;   // groups emitted
        auto emit = [&](int rs, int pr0, int ng, int flags, int ss) {
            const int b = G % NBUF;
            if (G >= NBUF && !mbar_wait_bounded(smem_u32(&eempty[b]), ((G / NBUF) - 1) & 1, p.wait_ns)) fail();
            if (!failed && ng > 0) {
                const float* rc = rec + rs * PAIRS * KREC;
                unsigned char* eb = ebuf + (size_t)b * GROUP * ebuf_pair;
                const int total = ng * runs_per_pair;
                for (int run = Erun; run < total; run += RSLOTS) {
                    const int j = run / runs_per_pair;
                    const int pos0 = (run - j * runs_per_pair) * RUN;
                    const int pr = pr0 + j;
                    const unsigned char* slot = seg + ((size_t)ss * PAIRS + pr) * p.slot_bytes;
                    const int off = __float_as_int(rc[pr * KREC + F_OFF]) + pos0;
                    const float sc = rc[pr * KREC + F_SCALE];
                    float2 w[RUN + TAPS - 1];
#pragma unroll
                    for (int t = 0; t < RUN + TAPS - 1; ++t) w[t] = load_sample<ET>(slot, off + t, sc);
                    // row of half h at sample position n: NH n + h
                    unsigned char* dst = eb + j * ebuf_pair + (NH * pos0 + Eh) * 16 + e_off;
                    float2 e[NPL];
                    if constexpr (E16) {
                        unsigned char* dst2 = eb + j * ebuf_pair + plane1 + (NH * pos0 + Eh) * 8;
#pragma unroll
                        for (int kq = 0; kq < RUN; ++kq) {
#pragma unroll
                            for (int q = 0; q < NPL; ++q) e[q] = make_float2(0.f, 0.f);
#pragma unroll
                            for (int m = 0; m < TAPS; ++m)
#pragma unroll
                                for (int q = 0; q < NPL; ++q) e[q] = ffma2(cc2[q][m], w[kq + m], e[q]);
                            *reinterpret_cast<float4*>(dst + kq * (NH * 16)) = make_float4(e[0].x, e[0].y, e[1].x, e[1].y);
                            *reinterpret_cast<float2*>(dst2 + kq * (NH * 8)) = e[NPL - 1];
                        }
                    } else {
#pragma unroll
                        for (int kq = 0; kq < RUN; ++kq) {
#pragma unroll
                            for (int q = 0; q < NPL; ++q) e[q] = make_float2(0.f, 0.f);
#pragma unroll
                            for (int m = 0; m < TAPS; ++m)
#pragma unroll
                                for (int q = 0; q < NPL; ++q) e[q] = ffma2(cc2[q][m], w[kq + m], e[q]);
                            *reinterpret_cast<float4*>(dst + kq * (NH * 16)) = make_float4(e[0].x, e[0].y, e[1].x, e[1].y);
                        }
                    }
                }
            }
            __syncwarp();
            if (lane == 0) {
                gdesc[b] = make_int4(rs, pr0, ng, flags);
                mbar_arrive(smem_u32(&efull[b]));
            }
            ++G;
        };

        bool last_cur = false, last_next = false;
        int kf = 1, kw = 0;   // stages filled; stages whose copies were waited for
        int n_cur = fill(0, last_cur), n_next = 0;
        int k = 0;
        while (!failed) {
            if (!last_cur) {
                n_next = fill(k + 1, last_next);
                ++kf;
            }
            // stage k's copies (and its records) have landed
            if (!failed && !mbar_wait_bounded(smem_u32(&full[k % NSEG]), (k / NSEG) & 1, p.wait_ns)) fail();
            if (failed) break;
            kw = k + 1;
            const int ngrp = (n_cur + GROUP - 1) / GROUP;
            if (ngrp == 0) emit(k % NRS, 0, 0, GD_STAGE_END | (last_cur ? GD_LAST : 0), k % NSEG);
            for (int gi = 0; gi < ngrp && !failed; ++gi) {
                const bool end = gi == ngrp - 1;
                emit(k % NRS, gi * GROUP, min(GROUP, n_cur - gi * GROUP),
                     (end ? GD_STAGE_END : 0) | (end && last_cur ? GD_LAST : 0), k % NSEG);
            }
            if (last_cur) break;
            ++k;
            n_cur = n_next;
            last_cur = last_next;
        }
        // copies issued for a stage that was never expanded must land before
        // exit; if one does not land in time, the CTA leaves with a bulk copy
        // possibly still writing its shared memory: recorded as a timeout
        for (int kk = kw; kk < kf; ++kk) {
            if (!mbar_wait_bounded(smem_u32(&full[kk % NSEG]), (kk / NSEG) & 1, p.wait_ns) && lane == 0)
                atomicOr(p.status, DEV_TIMEOUT);
        }
        if (p.cull) {
            n_cand = __reduce_add_sync(0xffffffffu, n_cand);
            n_act = __reduce_add_sync(0xffffffffu, n_act);
            n_edge = __reduce_add_sync(0xffffffffu, n_edge);
            if (lane == 0) {
                atomicAdd(&p.cull[0], (unsigned long long)n_cand);
                atomicAdd(&p.cull[1], (unsigned long long)n_act);
                atomicAdd(&p.cull[2], (unsigned long long)n_edge);
            }
        }
        return;
    }

    // ================= consumers =================
    const int ct = tid - 32;
    // pixel offsets from the tile centre: x (and y in 3D) fixed per thread; the
    // slot s moves along y (2D, 4 rows a slot) or z (3D): d_var(s) = dv0 + s dvstep
    float dxv, dyv_c, dv0, dvstep;
    // per slot s: the varying offset d_var(s), |d|^2 and the transmitter
    // differential range of the current ping, held as pairs of slots (2k, 2k+1)
    // for the packed geometry.  The offsets are formed exactly as the adjoint
    // kernel forms them, so both evaluate identical paths.
    float2 dvp[PX / 2], d2p[PX / 2], dTp[PX / 2];
#define PXS(arr, s) (((s) & 1) ? arr[(s) >> 1].y : arr[(s) >> 1].x)
    float2 acc[PX];                       // forward: image accumulators; gradient: G(x)
    float rsum[MODE == MODE_OFFSET_GRAD ? PX : 1];
    {
        int lx, ly, lz;
        T::pixel(ct, 0, lx, ly, lz);
        // formed in FP64, kept opaque so that they are not re-derived in FP64 at their uses
        dxv = opaque((float)((tx0 + lx - cx) * p.dx));
        dyv_c = opaque((float)((ty0 + ly - cy) * p.dy));
        dv0 = DIM3 ? opaque((float)((tz0 + lz - cz) * p.dz)) : dyv_c;
        dvstep = DIM3 ? opaque((float)p.dz) : opaque((float)(4.0 * p.dy));
        const float d2c = fixed_d2<DIM3>(dxv, dyv_c);
#pragma unroll
        for (int s = 0; s < PX; ++s) {
            T::pixel(ct, s, lx, ly, lz);
            const float dvs = fmaf((float)s, dvstep, dv0);
            PXS(dvp, s) = dvs;
            PXS(d2p, s) = fmaf(dvs, dvs, d2c);
            PXS(dTp, s) = 0.f;
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
    uint32_t tmask = 0xffu;                         // pixels the current ping's transmitter sees
    // seabed refraction: x_r's depth below the interface and offset from the
    // tile centre; |d_h|^2 of this thread's column (3D)
    __shared__ float s_rf[2];
    if (REFRACT && ct == 0) {
        s_rf[0] = (float)(Zr - p.z_int);
        s_rf[1] = (float)(Zr - Zc);
    }
    if (REFRACT) named_bar_sync(BAR_CONS, NCONS);
    const float r_br = REFRACT ? s_rf[0] : 0.f, r_zoff = REFRACT ? s_rf[1] : 0.f;
    const float r_d2h = REFRACT ? fixed_d2<true>(dxv, dyv_c) : 0.f;
    // depth below the interface of slot s, and its offset from x_r's depth
    auto slot_depth = [&](int s, float& b, float& db) {
        db = DIM3 ? PXS(dvp, s) - r_zoff : 0.f;
        b = fmaxf(r_br + db, 1e-7f);
    };

    auto warp_arrive = [&](uint64_t* bar) {
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(bar));
    };

    // gradient: fold the transmitter term of the finished ping into the
    // per-thread sum, reduce over the CTA in FP64 and write the tile's partial
    float tT0 = 0.f, tT1 = 0.f, tT2 = 0.f, tNT2 = 0.f, tNT = 0.f;   // transmitter terms of the current ping
    // gradient with seabed refraction: the current ping's transmitter-leg blocks
    float4 ftr0 = make_float4(0.f, 0.f, 0.f, 0.f), ftr1 = ftr0, ftr2 = ftr0;
    bool ftrefr = false;
    auto flush_ping = [&](int ping) {
        if (MODE != MODE_OFFSET_GRAD) return;
        const float tTv = DIM3 ? tT2 : tT1;
        const float X = fixed_dot<DIM3>(tT0, tT1, dxv, dyv_c);
        float hx = 0.5f * tT0 + dxv;
        float hy = DIM3 ? 0.5f * tT1 + dyv_c : 0.f;
        float hz = DIM3 ? 0.f : 0.5f * tT2;
        // (3D: the column's horizontal distance from the transmitter, refracted legs)
        float rhoT = 0.f, drhoT = 0.f;
        if (REFRACT && ftrefr && DIM3) refr_rho(ftr0, X + r_d2h, rhoT, drhoT);
#pragma unroll
        for (int s = 0; s < PX; ++s) {
            const float dvs = PXS(dvp, s);
            const float a = __fadd_rn(fmaf(tTv, dvs, PXS(d2p, s)), X);
            const float sm = tNT2 + a;
            const float rsm = rsum[MODE == MODE_OFFSET_GRAD ? s : 0];
            const float vy = DIM3 ? hy : 0.5f * tT1 + dvs;
            const float vz = DIM3 ? 0.5f * tT2 + dvs : hz;
            if (REFRACT && ftrefr && ((bmask >> s) & 1u)) {
                // refracted leg: r times the unit vector from the transmitter to
                // its crossing point, (xi h, a) / |W| with h the horizontal unit
                // vector towards the pixel
                if (!DIM3) refr_rho(ftr0, a, rhoT, drhoT);
                float b, db, uxi, ua;
                slot_depth(s, b, db);
                (void)refr_leg_diff(p, ftr0, ftr1, ftr2, rhoT, drhoT, b, db, r_br, uxi, ua);
                const float ih = rhoT > 0.f ? uxi * rcp_sfu(rhoT) : 0.f;
                gacc0 = fmaf(rsm * ih, hx, gacc0);
                gacc1 = fmaf(rsm * ih, vy, gacc1);
                gacc2 = fmaf(rsm, ua, gacc2);
            } else {
                const float kk = rsm * rsqrt_sfu(sm);   // r / |R_T + d|
                gacc0 = fmaf(kk, hx, gacc0);
                gacc1 = fmaf(kk, vy, gacc1);
                gacc2 = fmaf(kk, vz, gacc2);
            }
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

    // per-pixel work of one pair; MASKED: apply the beam test per pixel.  The
    // geometry runs on pixel pairs (2k, 2k+1) in packed FP32x2: differential
    // path, sample position and carrier phase, the fraction and phase
    // reductions; the SFU, the Farrow rows and the accumulation per pixel.
    //
    // Receiver motion: the reference vector R_R is from the receiver's position
    // at the reception of the tile centre's echo (tau_ref); a pixel's echo
    // arrives dtau later, when the receiver has moved on by v dtau (about a
    // millimetre), which to first order shortens the receive path by
    // u_R.v dtau: c dtau (1 + u_R.v / c) = dr_T + dr_R, so the differential
    // path is D / (1 + eps), eps = u_R.v / c ~ 1e-3, taken as
    // D (1 - eps + eps^2) (neglected: eps^3 D ~ 1e-9 m and the curvature term
    // |v dtau|^2 / (2 |R|) ~ 2e-8 m).
    // DIRECT: the carrier phase goes to the SFU without a range reduction
    // (p.phase_direct); a compile-time branch, so that the reduction's
    // instructions are not issued predicated off on every pixel
    auto pixels = [&](auto masked, auto direct, const float4 q0, const float4 q1, const float* rot, uint32_t rmask_needed,
                      const unsigned char* erow, const float4 q6, const float4 q7, const float4* hr, int rfl) {
        constexpr bool MASKED = decltype(masked)::value;
        constexpr bool DIRECT = decltype(direct)::value;
        const float tRx = q0.x, tRy = q0.y, tRz = q0.z, nR2 = q0.w;
        const float nR = q1.x, ufc = q1.y, phr = q1.z;   // phr: reference carrier phase [rad]
        const float tRv = DIM3 ? tRz : tRy;
        const float X = fixed_dot<DIM3>(tRx, tRy, dxv, dyv_c);
        const float2 Xv = make_float2(X, X), tRvv = make_float2(tRv, tRv);
        const float2 nR2v = make_float2(nR2, nR2), nRv = make_float2(nR, nR);
        const float2 ufv = make_float2(ufc, ufc), phv = make_float2(phr, phr);
        const float2 magic2 = make_float2(FLOOR_MAGIC, FLOOR_MAGIC);
        const unsigned char* erow_b = erow + npos_pad * NH * 16;   // the pair's second plane
        // motion: (R_R + d).v / c = Km + d_var v_var / c
        float2 Kmv = make_float2(0.f, 0.f), vvv = make_float2(0.f, 0.f);
        if constexpr (MOTION) {
            const float Km = DIM3 ? fmaf(q6.x, dxv, fmaf(q6.y, dyv_c, q6.w)) : fmaf(q6.x, dxv, q6.w);
            Kmv = make_float2(Km, Km);
            vvv = DIM3 ? make_float2(q6.z, q6.z) : make_float2(q6.y, q6.y);
        }
        // ping-time receiver vector for the beam test
        const float bRx = MOTION ? q7.x : tRx, bRy = MOTION ? q7.y : tRy, bRz = MOTION ? q7.z : tRz;
        // seabed refraction of the receiver leg: its record blocks and (3D) the
        // column's horizontal distance from the receiver
        const bool rrefr = REFRACT && (rfl & FL_R_REFR);
        float4 rr0 = make_float4(0.f, 0.f, 0.f, 0.f), rr1 = rr0, rr2 = rr0;
        float rhoR = 0.f, drhoR = 0.f;
        if (REFRACT && rrefr) {
            rr0 = hr[F_RREF / 4];
            rr1 = hr[F_RREF / 4 + 1];
            rr2 = hr[F_RREF / 4 + 2];
            if (DIM3) refr_rho(rr0, X + r_d2h, rhoR, drhoR);
        }
#pragma unroll
        for (int k = 0; k < PX / 2; ++k) {
            const float2 a = fadd2(ffma2(tRvv, dvp[k], d2p[k]), Xv);       // 2 R.d + |d|^2
            const float2 sm = fadd2(a, nR2v);                             // |R_R + d|^2
            const float2 rs = make_float2(rsqrt_sfu(sm.x), rsqrt_sfu(sm.y));
            const float2 den = ffma2(sm, rs, nRv);                        // |R_R + d| + |R_R|
            const float2 rc = make_float2(rcp_sfu(den.x), rcp_sfu(den.y));
            float2 D = ffma2(a, rc, dTp[k]);                              // two-way differential path [m]
            float2 kap = make_float2(1.f, 1.f);
            if constexpr (MOTION) {
                const float2 one2 = make_float2(1.f, 1.f);
                const float2 eps = fmul2(ffma2(dvp[k], vvv, Kmv), rs);       // u_R . v / c
                kap = ffma2(eps, fsub2(eps, one2), one2);                    // 1 / (1 + eps)
                D = fmul2(D, kap);
            }
            // refracted receiver legs of the two pixels (offset gradient): which
            // ones, their horizontal distances and crossing directions
            unsigned gbk = 0u;
            float2 grho = make_float2(1.f, 1.f), guxi = make_float2(0.f, 0.f), gua = guxi;
            if constexpr (REFRACT) {
                if (rrefr) {
                    const unsigned bk = (bmask >> (2 * k)) & 3u;   // which of the two slots are below
                    if (bk) {
                        float2 rho2 = make_float2(rhoR, rhoR), drho2 = make_float2(drhoR, drhoR);
                        if (!DIM3) {
                            refr_rho(rr0, a.x, rho2.x, drho2.x);
                            refr_rho(rr0, a.y, rho2.y, drho2.y);
                        }
                        float2 b2, db2;
                        slot_depth(2 * k, b2.x, db2.x);
                        slot_depth(2 * k + 1, b2.y, db2.y);
                        const float2 Dr = fadd2(refr_leg_diff2(p, rr0, rr1, rr2, rho2, drho2, b2, db2, r_br, guxi, gua),
                                                dTp[k]);
                        D.x = (bk & 1u) ? Dr.x : D.x + rr2.w;
                        D.y = (bk & 2u) ? Dr.y : D.y + rr2.w;
                        grho = rho2;
                        gbk = bk;
                    } else {
                        D = fadd2(D, make_float2(rr2.w, rr2.w));
                    }
                }
            }
            const float2 v = ffma2(D, p.hs_c2, ufv);                      // 2 (u - floor u_ref) - 1/2
            float2 x2 = ffma2(D, p.wfc_c2, phv);                          // carrier phase [rad]
            // the nearest integer of v = 2(u - floor u_ref) - 1/2 is the half-sample
            // index floor(2(u - floor u_ref)): it sits in the mantissa of
            // t = v + 1.5*2^23 (round to nearest), and g = v - that = frac(2u) - 1/2
            const float2 t = fadd2(v, magic2);
            const float2 g2 = fsub2(v, fsub2(t, magic2));
            if constexpr (!DIRECT) x2 = reduce_phase2(x2);
#pragma unroll
            for (int j = 0; j < 2; ++j) {
            const int s = 2 * k + j;
            const float g = j ? g2.y : g2.x;
            const float tj = j ? t.y : t.x;
            bool seen = true;
            if (MASKED) {
                const float dvs = PXS(dvp, s);
                const float wx = fmaf(0.5f, bRx, dxv);
                const float wy = DIM3 ? fmaf(0.5f, bRy, dyv_c) : fmaf(0.5f, bRy, dvs);
                const float wz = DIM3 ? fmaf(0.5f, bRz, dvs) : 0.5f * bRz;
                seen = ((tmask >> s) & 1u) && (!rmask_needed || beam_sees(p, wx, wy, wz, rot));
            }
            // half-sample row: floor(2(u - floor u_ref)) + 2U, clamped into the buffer
            const unsigned pos = row_index((unsigned)(__float_as_int(tj) - (__float_as_int(FLOOR_MAGIC) - NH * p.U)),
                                           (unsigned)(NH * p.npos - 1), p.status);
            float sn, cs;
            sincos_sfu(j ? x2.y : x2.x, sn, cs);
            if (MASKED && !seen) {
                sn = 0.f;
                cs = 0.f;
            }
            const float2 gg2 = make_float2(g, g);
            // (E0, E1) from the first plane
            const float4 e01 = *reinterpret_cast<const float4*>(erow + pos * 16);
            if (E16) {
                // quadratic: E2 from the second plane; packed FP32 Horner over E_2 .. E_0
                const float2 e2 = *reinterpret_cast<const float2*>(erow_b + pos * 8);
                float2 v = ffma2(e2, gg2, make_float2(e01.z, e01.w));
                v = ffma2(v, gg2, make_float2(e01.x, e01.y));
                acc[s].x = fmaf(v.x, cs, fmaf(-v.y, sn, acc[s].x));
                acc[s].y = fmaf(v.x, sn, fmaf(v.y, cs, acc[s].y));
                continue;
            }
            // cubic: (E2, E3) from the second plane
            const float4 e23 = *reinterpret_cast<const float4*>(erow_b + pos * 16);
            const float2 e0 = make_float2(e01.x, e01.y), e1 = make_float2(e01.z, e01.w);
            const float2 e2 = make_float2(e23.x, e23.y), e3 = make_float2(e23.z, e23.w);
            if (MODE == MODE_FORWARD) {
                // packed FP32 Horner over E_3 .. E_0
                float2 v = ffma2(e3, gg2, e2);
                v = ffma2(v, gg2, e1);
                v = ffma2(v, gg2, e0);
                acc[s].x = fmaf(v.x, cs, fmaf(-v.y, sn, acc[s].x));
                acc[s].y = fmaf(v.x, sn, fmaf(v.y, cs, acc[s].y));
            } else {
                // value and derivative in g: b = s(g), d = ds/dg (ds/du = 2 d)
                float2 b = e3;
                float2 d = e3;
                b = ffma2(b, gg2, e2);
                d = ffma2(d, gg2, b); b = ffma2(b, gg2, e1);
                d = ffma2(d, gg2, b); b = ffma2(b, gg2, e0);
                // a = fs s' + j 2 pi fc s = 2 fs d + j 2 pi fc b ;  r = Re{ conj(G) a exp(j phase) }
                // (0 outside the beam)
                const float ax = fmaf(p.fs2_f, d.x, -p.wfc * b.y);
                const float ay = fmaf(p.fs2_f, d.y, p.wfc * b.x);
                const float Hx = fmaf(acc[s].x, cs, acc[s].y * sn);       // conj(G) exp(j phase)
                const float Hy = fmaf(acc[s].x, sn, -acc[s].y * cs);
                // dtau/d(dp) carries 1 / (1 + eps) with receiver motion
                const float r = fmaf(Hx, ax, -Hy * ay) * (j ? kap.y : kap.x);
                rsum[MODE == MODE_OFFSET_GRAD ? s : 0] += r;
                // receiver unit vector (R_R + d) / |R_R + d| times r
                const float dvs = PXS(dvp, s);
                const float vx = fmaf(0.5f, tRx, dxv);
                const float vy = DIM3 ? fmaf(0.5f, tRy, dyv_c) : fmaf(0.5f, tRy, dvs);
                const float vz = DIM3 ? fmaf(0.5f, tRz, dvs) : 0.5f * tRz;
                if (REFRACT && ((gbk >> j) & 1u)) {
                    // refracted receiver leg: the unit vector towards its crossing point
                    const float rh = j ? grho.y : grho.x;
                    const float ih = rh > 0.f ? (j ? guxi.y : guxi.x) * rcp_sfu(rh) : 0.f;
                    gacc0 = fmaf(r * ih, vx, gacc0);
                    gacc1 = fmaf(r * ih, vy, gacc1);
                    gacc2 = fmaf(r, j ? gua.y : gua.x, gacc2);
                } else {
                    const float kr = r * (j ? rs.y : rs.x);
                    gacc0 = fmaf(kr, vx, gacc0);
                    gacc1 = fmaf(kr, vy, gacc1);
                    gacc2 = fmaf(kr, vz, gacc2);
                }
            }
            }
        }
    };

    // ---- the groups in the order the producer emits them
    bool aborted = false;
    int prev_ping = -1;
    int seq_ping = ping0, seq_ch = 0;               // candidate order (no culling)
    for (int G = 0;; ++G) {
        const int b = G % NBUF;
        if (!mbar_wait_bounded(smem_u32(&efull[b]), (G / NBUF) & 1, p.wait_ns)) {
            *abort_flag = 1;
            atomicOr(p.status, DEV_TIMEOUT);
        }
        if (*abort_flag) {
            aborted = true;
            break;
        }
        const int4 d = gdesc[b];
        const int rs = d.x, pr0 = d.y, ng = d.z, gflags = d.w;
        const float4* hq = reinterpret_cast<const float4*>(rec + rs * PAIRS * KREC);
        const unsigned char* eb = ebuf + (size_t)b * GROUP * ebuf_pair;
#pragma unroll 1
        for (int j = 0; j < ng; ++j) {
            const int pr = pr0 + j;
            const float4* hr = hq + pr * (KREC / 4);
            // without culling the pairs arrive in candidate order, so the ping
            // is tracked here; with culling it comes from the record
            int ping, flags = FL_TX_FULL | FL_RX_FULL, rfl = 0;
            float4 q3;
            if (REFRACT) {
                q3 = hr[3];
                rfl = __float_as_int(q3.z);
            }
            if (BEAM) {
                q3 = hr[3];
                ping = __float_as_int(q3.y);
                flags = __float_as_int(q3.z);
            } else {
                ping = seq_ping;
                if (++seq_ch == p.C) {
                    seq_ch = 0;
                    ++seq_ping;
                }
            }
            float rot[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            if (BEAM) {
                const float4 q4 = hr[4], q5 = hr[5];
                rot[0] = q4.x; rot[1] = q4.y; rot[2] = q4.z; rot[3] = q4.w; rot[4] = q5.x; rot[5] = q5.y;
            }
            if (ping != prev_ping) {
                if (prev_ping >= 0) flush_ping(prev_ping);
                prev_ping = ping;
                const float4 q2 = hr[2];
                tT0 = q2.x;
                tT1 = q2.y;
                tT2 = q2.z;
                tNT2 = q2.w;
                tNT = (BEAM || REFRACT) ? q3.x : hr[3].x;
                const float tTv = DIM3 ? tT2 : tT1;
                const float X = fixed_dot<DIM3>(tT0, tT1, dxv, dyv_c);
                tmask = 0xffu;
                // seabed refraction of the transmitter leg
                const bool trefr = REFRACT && (rfl & FL_T_REFR);
                float4 tr0 = make_float4(0.f, 0.f, 0.f, 0.f), tr1 = tr0, tr2 = tr0;
                float rhoT = 0.f, drhoT = 0.f;
                if (REFRACT && trefr) {
                    tr0 = hr[F_TREF / 4];
                    tr1 = hr[F_TREF / 4 + 1];
                    tr2 = hr[F_TREF / 4 + 2];
                    if (DIM3) refr_rho(tr0, X + r_d2h, rhoT, drhoT);
                }
                if constexpr (REFRACT && MODE == MODE_OFFSET_GRAD) {
                    ftrefr = trefr;
                    ftr0 = tr0;
                    ftr1 = tr1;
                    ftr2 = tr2;
                }
#pragma unroll
                for (int s = 0; s < PX; ++s) {
                    const float a = __fadd_rn(fmaf(tTv, PXS(dvp, s), PXS(d2p, s)), X);
                    const float sm = tNT2 + a;
                    const float den = fmaf(sm, rsqrt_sfu(sm), tNT);
                    PXS(dTp, s) = a * rcp_sfu(den);
                    if (REFRACT && trefr) {
                        if ((bmask >> s) & 1u) {
                            if (!DIM3) refr_rho(tr0, a, rhoT, drhoT);
                            float b, db;
                            slot_depth(s, b, db);
                            float uxi, ua;
                            PXS(dTp, s) = refr_leg_diff(p, tr0, tr1, tr2, rhoT, drhoT, b, db, r_br, uxi, ua);
                        } else {
                            PXS(dTp, s) += tr2.w;
                        }
                    }
                    if (BEAM && !(flags & FL_TX_FULL)) {
                        const float dvs = PXS(dvp, s);
                        const float wx = fmaf(0.5f, tT0, dxv);
                        const float wy = DIM3 ? fmaf(0.5f, tT1, dyv_c) : fmaf(0.5f, tT1, dvs);
                        const float wz = DIM3 ? fmaf(0.5f, tT2, dvs) : 0.5f * tT2;
                        if (!beam_sees(p, wx, wy, wz, rot)) tmask &= ~(1u << s);
                    }
                }
            }
            const float4 q0 = hr[0], q1 = hr[1];
            const float4 q6 = MOTION ? hr[6] : make_float4(0.f, 0.f, 0.f, 0.f);
            const float4 q7 = (MOTION && BEAM) ? hr[7] : make_float4(0.f, 0.f, 0.f, 0.f);
            const unsigned char* erow = eb + j * ebuf_pair;
            using F_ = std::integral_constant<bool, false>;
            using T_ = std::integral_constant<bool, true>;
            using B_ = std::integral_constant<bool, BEAM>;
            if (!BEAM || (flags & (FL_TX_FULL | FL_RX_FULL)) == (FL_TX_FULL | FL_RX_FULL)) {
                if (p.phase_direct)
                    pixels(F_{}, T_{}, q0, q1, rot, 0u, erow, q6, q7, hr, rfl);
                else
                    pixels(F_{}, F_{}, q0, q1, rot, 0u, erow, q6, q7, hr, rfl);
            } else {
                const uint32_t rmn = (flags & FL_RX_FULL) ? 0u : 1u;
                if (p.phase_direct)
                    pixels(B_{}, T_{}, q0, q1, rot, rmn, erow, q6, q7, hr, rfl);
                else
                    pixels(B_{}, F_{}, q0, q1, rot, rmn, erow, q6, q7, hr, rfl);
            }
        }
        warp_arrive(&eempty[b]);
        if (gflags & GD_STAGE_END) warp_arrive(&rempty[rs]);
        if (gflags & GD_LAST) break;
    }
    if (aborted) return;
    if constexpr (MODE == MODE_OFFSET_GRAD) {
        if (prev_ping >= 0) flush_ping(prev_ping);
        return;
    } else {
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
// many CTAs by splitting the pings of each tile (0 = never split); mode: the
// tdbp_kernel mode the launch runs (sets the Farrow row format).
int prepare(sas_geometry_t h, const sas_grid& g, int dim3, long long min_ctas, Setup& S, bool need_echo = true,
            int mode = MODE_FORWARD);

template <int MODE>
int launch_mode(const Setup& S, int echo_dtype, int dim3, cudaStream_t st);

}  // namespace core
}  // namespace sas
