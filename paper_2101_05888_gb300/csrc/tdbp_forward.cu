// Time-domain backprojection, forward (echo -> image), 2D and 3D.
//
// Computes, for every pixel x of the grid (Sec. II-A: Eq. 1 inverted per
// pixel, every pixel independent):
//   I(x) = sum_i sum_c sum_k w_k(f) e[i][c][floor(u) + k] exp(+j 2 pi fc tau),
//   tau = (|x - x_TX,i| + |x - x_RX,i,c|) / c,  u = (tau - t0) fs,  f = u - floor(u),
// with samples outside [0, Ns) reading as zero.
//
// Structure (one CTA per image tile; optionally the (ping, channel) pairs of a
// tile are split over several CTAs that add into the image):
//  * warp 0 (producer), one lane per (ping, channel) pair, 32 pairs a stage:
//    FP64 reference terms at the tile centre x0 -- vectors R = x0 - sensor,
//    |R|, tau_ref, sample index floor(u_ref), fraction, carrier phase in
//    cycles mod 1 -- written to shared memory, and a 2D bulk tensor copy of the
//    echo segment the tile can touch into a ring of NSTAGE stages (mbarrier
//    complete_tx).  Out-of-range samples are zero-filled by the copy engine.
//  * warps 1..8 (consumers), 8 pixels a thread:
//    - Farrow expansion, 4 pairs at a time: the interpolator's taps are
//      polynomials of degree 7 in g = f - 1/2, so the interpolated value is
//      s = sum_p g^p E_p[i0] with E_p[i] = sum_m coef[m][p] e[i + k_m]; the CTA
//      computes E_p at every integer position the tile can need, once per pair.
//    - per pixel and pair (reference terms broadcast by warp shuffle):
//      differential range  dr = (2 R.d + |d|^2) / (|R + d| + |R|)  (exact
//      identity, FP32, d = x - x0 small), so only |d|-sized quantities are
//      rounded in FP32; u and the phase follow from tau_ref + dr/c; floor and
//      fraction on the FP32 pipe; 4 vector shared loads + 7 packed-FP32 Horner
//      steps; sin/cos of the phase and 1/sqrt, 1/x on the SFU; 4 FMA into
//      register accumulators.
//  * every mbarrier wait is bounded in wall time; on expiry the CTA records
//    SAS timeout status, stops, and the producer drains its copies in flight.
#include "sas_common.cuh"

#include <algorithm>
#include <cmath>

namespace sas {
namespace {

constexpr int NCW = 8;                  // consumer warps
constexpr int NCONS = 32 * NCW;         // consumer threads
constexpr int NTHREADS = NCONS + 32;    // + producer warp
constexpr int PAIRS = 32;               // (ping, channel) pairs per stage
constexpr int NSTAGE = 3;               // copy ring depth
constexpr int GROUP = 4;                // pairs per Farrow group
constexpr int GPS = PAIRS / GROUP;      // groups per stage
constexpr int PX = 8;                   // pixels per consumer thread
constexpr int EROW = 10;                // float2 per E row (8 coefficients + 16 B pad)
constexpr int BAR_CONS = 1;             // named barrier of the consumer warps

// record fields (structure of arrays in shared memory, one column per pair)
enum { F_TX, F_TY, F_TZ, F_NT2, F_NT, F_RX, F_RY, F_RZ, F_NR2, F_NR, F_UF, F_PH, F_OFF, F_SCALE, NREC };
constexpr int NHOLD = 12;               // fields the per-pixel updates need (F_TX .. F_PH)

struct FwdParams {
    const double* tx;   // [P][3]
    const double* rx;   // [P][C][3]
    const float* scale; // [P*C] or null
    const FarrowCoef* coef;
    float2* image;
    uint32_t* status;
    double x0, y0, z0, dx, dy, dz;
    float fdx, fdy, fdz;
    int nx, ny, nz;
    int tiles_x, tiles_y, tiles_z, nsplit;
    int P, C;
    long long npairs;
    double t0, fs, fc, inv_c;
    float fs_c, fc_c;
    int U, npos, seglen, seg_align, slot_bytes;
    int accumulate, atomic_out, skip_copies;
    unsigned long long wait_ns;
};

template <bool DIM3>
struct Tile;
template <>
struct Tile<false> {  // 2D: 32 (x) x 64 (y)
    static constexpr int TX = 32, TY = 64, TZ = 1;
    __device__ static void pixel(int ct, int s, int& lx, int& ly, int& lz) {
        const int w = ct >> 5, l = ct & 31;
        lx = (w & 3) * 8 + (l & 7);
        ly = (w >> 2) * 32 + (l >> 3) + 4 * s;
        lz = 0;
    }
};
template <>
struct Tile<true> {   // 3D: 16 (x) x 16 (y) x 8 (z)
    static constexpr int TX = 16, TY = 16, TZ = 8;
    __device__ static void pixel(int ct, int s, int& lx, int& ly, int& lz) {
        const int w = ct >> 5, l = ct & 31;
        lx = (w & 1) * 8 + (l & 7);
        ly = (w >> 1) * 4 + (l >> 3);
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
    float2 v = __half22float2(reinterpret_cast<const __half2*>(slot)[idx]);
    return make_float2(v.x * sc, v.y * sc);
}
template <>
__device__ __forceinline__ float2 load_sample<__nv_bfloat162>(const unsigned char* slot, int idx, float sc) {
    float2 v = __bfloat1622float2(reinterpret_cast<const __nv_bfloat162*>(slot)[idx]);
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

// Differential range |R + d| - |R| = (2 R.d + |d|^2) / (|R + d| + |R|), with
// tR = 2R, nR2 = |R|^2, nR = |R| and a = 2 R.d + |d|^2 precomputed by caller.
__device__ __forceinline__ float diff_range(float a, float nR2, float nR) {
    const float s = nR2 + a;
    const float den = fmaf(s, rsqrt_sfu(s), nR);
    return a * rcp_sfu(den);
}

template <typename ET, bool DIM3>
__global__ void __launch_bounds__(NTHREADS, 2)
tdbp_forward_kernel(const __grid_constant__ CUtensorMap tmap, const FwdParams p) {
    using T = Tile<DIM3>;
    extern __shared__ __align__(1024) unsigned char smem[];
    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;

    // ---- shared memory carve-up
    unsigned char* seg = smem;                                              // NSTAGE * PAIRS * slot_bytes
    float2* ebuf = reinterpret_cast<float2*>(seg + (size_t)NSTAGE * PAIRS * p.slot_bytes);
    const int ebuf_pair = p.npos * EROW;                                    // float2 per pair
    float* rec = reinterpret_cast<float*>(ebuf + 2 * GROUP * ebuf_pair);   // NSTAGE * NREC * PAIRS
    float* coef_s = rec + NSTAGE * NREC * PAIRS;                            // TAPS * NP
    float* hold = coef_s + TAPS * NP;                                       // 2 * NHOLD * PAIRS
    uint64_t* bars = reinterpret_cast<uint64_t*>(hold + 2 * NHOLD * PAIRS); // full[NSTAGE], empty[NSTAGE]
    volatile int* abort_flag = reinterpret_cast<volatile int*>(bars + 2 * NSTAGE);

    // ---- tile and pair range of this CTA
    const int ntiles = p.tiles_x * p.tiles_y * p.tiles_z;
    const int tile = blockIdx.x % ntiles;
    const int split = blockIdx.x / ntiles;
    const int tx0 = (tile % p.tiles_x) * T::TX;
    const int ty0 = ((tile / p.tiles_x) % p.tiles_y) * T::TY;
    const int tz0 = (tile / (p.tiles_x * p.tiles_y)) * T::TZ;
    const long long per = (p.npairs + p.nsplit - 1) / p.nsplit;
    const long long q0 = (long long)split * per;
    const long long q1 = min(p.npairs, q0 + per);
    const int nq = (int)max(0LL, q1 - q0);
    const int nstages = (nq + PAIRS - 1) / PAIRS;
    const int ngroups = (nq + GROUP - 1) / GROUP;
    // tile centre (index space, may be half-integer)
    const double cx = tx0 + 0.5 * (T::TX - 1), cy = ty0 + 0.5 * (T::TY - 1), cz = tz0 + 0.5 * (T::TZ - 1);

    if (tid == 0) {
        for (int s = 0; s < NSTAGE; ++s) {
            mbar_init(smem_u32(&bars[s]), 1);
            mbar_init(smem_u32(&bars[NSTAGE + s]), NCW);
        }
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
                const bool ok = mbar_wait_bounded(smem_u32(&bars[NSTAGE + s]), ((k / NSTAGE) - 1) & 1, p.wait_ns);
                if (!ok) {
                    if (lane == 0) { *abort_flag = 1; atomicOr(p.status, DEV_TIMEOUT); }
                }
            }
            __syncwarp();
            if (*abort_flag) break;
            const long long q = q0 + (long long)k * PAIRS + lane;
            const bool valid = q < q1;
            int seg_start = 0;
            if (valid) {
                const int i = (int)(q / p.C);
                const double* t = p.tx + 3 * (size_t)i;
                const double* r = p.rx + 3 * (size_t)q;
                const double Tx = X0 - t[0], Ty = Y0 - t[1], Tz = Z0 - t[2];
                const double Rx = X0 - r[0], Ry = Y0 - r[1], Rz = Z0 - r[2];
                const double nT2 = Tx * Tx + Ty * Ty + Tz * Tz, nR2 = Rx * Rx + Ry * Ry + Rz * Rz;
                const double nT = sqrt(nT2), nR = sqrt(nR2);
                const double tau = (nT + nR) * p.inv_c;
                double u = (tau - p.t0) * p.fs;
                u = fmin(fmax(u, -268435456.0), 268435456.0);  // keep copy coordinates in int range
                const double iref = floor(u);
                const double ph = p.fc * tau;
                const int ir = (int)iref;
                const int base = ir - p.U - 3;                         // raw index of E position 0, tap 0
                seg_start = base - (((base % p.seg_align) + p.seg_align) % p.seg_align);
                float* rc = rec + s * NREC * PAIRS;
                rc[F_TX * PAIRS + lane] = (float)(2.0 * Tx);
                rc[F_TY * PAIRS + lane] = (float)(2.0 * Ty);
                rc[F_TZ * PAIRS + lane] = (float)(2.0 * Tz);
                rc[F_NT2 * PAIRS + lane] = (float)nT2;
                rc[F_NT * PAIRS + lane] = (float)nT;
                rc[F_RX * PAIRS + lane] = (float)(2.0 * Rx);
                rc[F_RY * PAIRS + lane] = (float)(2.0 * Ry);
                rc[F_RZ * PAIRS + lane] = (float)(2.0 * Rz);
                rc[F_NR2 * PAIRS + lane] = (float)nR2;
                rc[F_NR * PAIRS + lane] = (float)nR;
                rc[F_UF * PAIRS + lane] = (float)(u - iref);
                rc[F_PH * PAIRS + lane] = (float)(ph - floor(ph));
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
                tma_load_2d(smem_u32(seg + ((size_t)s * PAIRS + lane) * p.slot_bytes), &tmap, seg_start,
                            (int32_t)q, smem_u32(&bars[s]));
        }
        // drain: every issued stage must have landed before the CTA may exit
        const int first = max(0, k - NSTAGE);
        for (int kk = first; kk < k; ++kk)
            mbar_wait_bounded(smem_u32(&bars[kk % NSTAGE]), (kk / NSTAGE) & 1, p.wait_ns);
        return;
    }

    // ================= consumers =================
    const int ct = tid - 32;            // 0 .. NCONS-1
    const int cwarp = ct >> 5;
    // per-pixel geometry relative to the tile centre
    float dxv = 0.f, dyv_c = 0.f;       // per-thread constants (x always; y in 3D)
    float dvar[PX], dT[PX];
    float d2c = 0.f;                    // |d|^2 minus the varying component squared
    float2 acc[PX];
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
            acc[s] = make_float2(0.f, 0.f);
        }
    }

    // one pair's reference terms per lane (pair = lane of the current stage)
    float r_cur[NHOLD];
#pragma unroll
    for (int f = 0; f < NHOLD; ++f) r_cur[f] = 0.f;
    const int Ep = ct & 7;        // Farrow power this thread computes
    const int Erun = ct >> 3;     // run slot (0..31)
    const int runs_per_pair = (p.npos + 7) >> 3;
    const float U = (float)p.U;
    (void)U;

    // Farrow expansion of group gg into ebuf[gg & 1]
    auto expand = [&](int gg) {
        const int stage = gg / GPS;
        const int s = stage % NSTAGE;
        const float* rc = rec + s * NREC * PAIRS;
        float2* eb = ebuf + (gg & 1) * GROUP * ebuf_pair;
        float cc[TAPS];
#pragma unroll
        for (int m = 0; m < TAPS; ++m) cc[m] = coef_s[m * NP + Ep];
        const int total = GROUP * runs_per_pair;
        for (int run = Erun; run < total; run += 32) {
            const int j = run / runs_per_pair;
            const int pos0 = (run - j * runs_per_pair) * 8;
            const int pr = (gg % GPS) * GROUP + j;              // pair within stage
            if ((long long)stage * PAIRS + pr >= nq) continue;
            const unsigned char* slot = seg + ((size_t)s * PAIRS + pr) * p.slot_bytes;
            const int off = __float_as_int(rc[F_OFF * PAIRS + pr]);
            const float sc = rc[F_SCALE * PAIRS + pr];
            float2 w[15];
#pragma unroll
            for (int t = 0; t < 15; ++t) w[t] = load_sample<ET>(slot, off + pos0 + t, sc);
            float2* dst = eb + j * ebuf_pair + pos0 * EROW + Ep;
#pragma unroll
            for (int kq = 0; kq < 8; ++kq) {
                float2 e = make_float2(0.f, 0.f);
#pragma unroll
                for (int m = 0; m < TAPS; ++m) e = ffma2(make_float2(cc[m], cc[m]), w[kq + m], e);
                if (pos0 + kq < p.npos) dst[kq * EROW] = e;
            }
        }
    };

    // copy a stage's per-update fields out of the producer's ring (which is
    // recycled as soon as the stage's last group is expanded)
    auto hold_records = [&](int stage) {
        const float* rc = rec + (stage % NSTAGE) * NREC * PAIRS;
        float* hd = hold + (stage & 1) * NHOLD * PAIRS;
        for (int t = ct; t < NHOLD * PAIRS; t += NCONS) hd[t] = rc[t];
    };
    // a stage may be handed back to the producer once its last group is expanded
    auto maybe_release = [&](int gg) {
        const int stage = gg / GPS;
        const bool last_of_stage = ((gg % GPS) == GPS - 1) || (gg == ngroups - 1);
        if (last_of_stage) {
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

    bool aborted = false;
    if (ngroups > 0) {
        bool ok = wait_stage(0);
        if (ok) {
            hold_records(0);
            expand(0);
            maybe_release(0);
        }
        named_bar_sync(BAR_CONS, NCONS);
        aborted = *abort_flag != 0;
    }

    int prev_ping = -1;
    for (int gg = 0; gg < ngroups && !aborted; ++gg) {
        const int nxt = gg + 1;
        if (nxt < ngroups) {
            bool ok = true;
            if (nxt % GPS == 0) {
                ok = wait_stage(nxt / GPS);
                if (ok) hold_records(nxt / GPS);
            }
            if (ok) {
                expand(nxt);
                maybe_release(nxt);
            }
        }
        if (gg % GPS == 0) {
            const float* hd = hold + ((gg / GPS) & 1) * NHOLD * PAIRS;
#pragma unroll
            for (int f = 0; f < NHOLD; ++f) r_cur[f] = hd[f * PAIRS + lane];
        }
        // ---- per-pixel updates for the pairs of group gg
        const int stage = gg / GPS;
        const float2* eb = ebuf + (gg & 1) * GROUP * ebuf_pair;
#pragma unroll 1
        for (int j = 0; j < GROUP; ++j) {
            const int pr = (gg % GPS) * GROUP + j;
            const long long qrel = (long long)stage * PAIRS + pr;
            if (qrel >= nq) break;
            const int ping = (int)((q0 + qrel) / p.C);
            if (ping != prev_ping) {
                prev_ping = ping;
                const float tTx = __shfl_sync(0xffffffffu, r_cur[0], pr);
                const float tTy = __shfl_sync(0xffffffffu, r_cur[1], pr);
                const float tTz = __shfl_sync(0xffffffffu, r_cur[2], pr);
                const float nT2 = __shfl_sync(0xffffffffu, r_cur[3], pr);
                const float nT = __shfl_sync(0xffffffffu, r_cur[4], pr);
                const float Ax = DIM3 ? fmaf(tTx, dxv, tTy * dyv_c) : tTx * dxv;
#pragma unroll
                for (int s = 0; s < PX; ++s) {
                    const float d2 = fmaf(dvar[s], dvar[s], d2c);
                    const float a = DIM3 ? fmaf(tTz, dvar[s], d2) + Ax : fmaf(tTy, dvar[s], d2) + Ax;
                    dT[s] = diff_range(a, nT2, nT);
                }
                (void)tTz;
            }
            const float tRx = __shfl_sync(0xffffffffu, r_cur[5], pr);
            const float tRy = __shfl_sync(0xffffffffu, r_cur[6], pr);
            const float tRz = __shfl_sync(0xffffffffu, r_cur[7], pr);
            const float nR2 = __shfl_sync(0xffffffffu, r_cur[8], pr);
            const float nR = __shfl_sync(0xffffffffu, r_cur[9], pr);
            const float uf = __shfl_sync(0xffffffffu, r_cur[10], pr);
            const float phr = __shfl_sync(0xffffffffu, r_cur[11], pr);
            const float Ax = DIM3 ? fmaf(tRx, dxv, tRy * dyv_c) : tRx * dxv;
            const float4* e4 = reinterpret_cast<const float4*>(eb + j * ebuf_pair);
#pragma unroll
            for (int s = 0; s < PX; ++s) {
                const float d2 = fmaf(dvar[s], dvar[s], d2c);
                const float a = DIM3 ? fmaf(tRz, dvar[s], d2) + Ax : fmaf(tRy, dvar[s], d2) + Ax;
                const float s_ = nR2 + a;
                const float den = fmaf(s_, rsqrt_sfu(s_), nR);
                const float D = fmaf(a, rcp_sfu(den), dT[s]);     // two-way differential path [m]
                const float u = fmaf(D, p.fs_c, uf);               // sample position rel. to floor(u_ref)
                const float ph = fmaf(D, p.fc_c, phr);             // carrier phase [cycles]
                float fl;
                const int di = floor_magic(u, fl);
                const float g = (u - fl) - 0.5f;
                const unsigned pos = min((unsigned)(di + p.U), (unsigned)(p.npos - 1));
                const float4* e = e4 + pos * (EROW / 2);
                const float4 e01 = e[0], e23 = e[1], e45 = e[2], e67 = e[3];
                const float2 gg2 = make_float2(g, g);
                float2 v = make_float2(e67.z, e67.w);
                v = ffma2(v, gg2, make_float2(e67.x, e67.y));
                v = ffma2(v, gg2, make_float2(e45.z, e45.w));
                v = ffma2(v, gg2, make_float2(e45.x, e45.y));
                v = ffma2(v, gg2, make_float2(e23.z, e23.w));
                v = ffma2(v, gg2, make_float2(e23.x, e23.y));
                v = ffma2(v, gg2, make_float2(e01.z, e01.w));
                v = ffma2(v, gg2, make_float2(e01.x, e01.y));
                const float pt = __fadd_rn(ph, FLOOR_MAGIC) - FLOOR_MAGIC;   // rint(ph)
                const float x = (ph - pt) * 6.28318530717958647f;
                float sn, cs;
                __sincosf(x, &sn, &cs);
                acc[s].x = fmaf(v.x, cs, fmaf(-v.y, sn, acc[s].x));
                acc[s].y = fmaf(v.x, sn, fmaf(v.y, cs, acc[s].y));
            }
        }
        named_bar_sync(BAR_CONS, NCONS);
        aborted = *abort_flag != 0;
    }
    (void)cwarp;
    if (aborted) return;

    // ---- write the tile
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
            float2 o = *dst;
            *dst = make_float2(o.x + acc[s].x, o.y + acc[s].y);
        } else {
            *dst = acc[s];
        }
    }
}

template <typename ET, bool DIM3>
int launch_t(const ForwardArgs& a, const FwdParams& prm, const CUtensorMap& map, size_t smem, int blocks) {
    auto kern = tdbp_forward_kernel<ET, DIM3>;
    SAS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<blocks, NTHREADS, smem, a.stream>>>(map, prm);
    SAS_CUDA(cudaGetLastError());
    return SAS_OK;
}

}  // namespace

int launch_forward(const ForwardArgs& a) {
    sas_geometry_t h = a.h;
    const sas_grid& g = a.grid;
    const int TXs = a.dim3 ? Tile<true>::TX : Tile<false>::TX;
    const int TYs = a.dim3 ? Tile<true>::TY : Tile<false>::TY;
    const int TZs = a.dim3 ? Tile<true>::TZ : Tile<false>::TZ;
    const double dz = a.dim3 ? g.dz : 0.0;
    // largest |x - x0| over a tile -> bound on the differential delay in samples
    const double hx = 0.5 * (TXs - 1) * std::fabs(g.dx), hy = 0.5 * (TYs - 1) * std::fabs(g.dy),
                 hz = 0.5 * (TZs - 1) * std::fabs(dz);
    const double dmax = std::sqrt(hx * hx + hy * hy + hz * hz);
    const double umax = 2.0 * dmax * h->sig.fs / h->sig.c;
    const int U = (int)std::ceil(umax) + 2;
    const int elem = (h->echo_dtype == SAS_ECHO_C64) ? 8 : 4;
    const int align = 16 / elem;
    const int npos = 2 * U + 1;
    int seglen = 2 * U + 7 + align;
    seglen = (seglen + align - 1) / align * align;
    if (seglen > 256) {
        set_error("pixel spacing too coarse: a tile's delay span needs %d samples (max 256)", seglen);
        return SAS_ERR_UNSUPPORTED;
    }
    const int slot_bytes = ((seglen + 8) * elem + 127) / 128 * 128;
    const size_t smem = (size_t)NSTAGE * PAIRS * slot_bytes + (size_t)2 * GROUP * npos * EROW * 8 +
                        (size_t)NSTAGE * NREC * PAIRS * 4 + TAPS * NP * 4 + 2 * NHOLD * PAIRS * 4 + 2 * NSTAGE * 8 + 16;
    if (smem > 227 * 1024) {
        set_error("shared memory need %zu exceeds the per-block limit", smem);
        return SAS_ERR_UNSUPPORTED;
    }

    FwdParams prm{};
    prm.tx = h->d_tx;
    prm.rx = h->d_rx;
    prm.scale = (h->echo_dtype == SAS_ECHO_C64) ? nullptr : h->d_scale;
    prm.coef = h->d_coef;
    prm.status = h->d_status;
    prm.x0 = g.x0; prm.y0 = g.y0; prm.z0 = g.z0;
    prm.dx = g.dx; prm.dy = g.dy; prm.dz = dz;
    prm.fdx = (float)g.dx; prm.fdy = (float)g.dy; prm.fdz = (float)dz;
    prm.nx = g.nx; prm.ny = g.ny; prm.nz = a.dim3 ? g.nz : 1;
    prm.tiles_x = (g.nx + TXs - 1) / TXs;
    prm.tiles_y = (g.ny + TYs - 1) / TYs;
    prm.tiles_z = (prm.nz + TZs - 1) / TZs;
    prm.P = h->P; prm.C = h->C;
    prm.npairs = (long long)h->P * h->C;
    prm.t0 = h->sig.t0; prm.fs = h->sig.fs; prm.fc = h->sig.fc; prm.inv_c = 1.0 / h->sig.c;
    prm.fs_c = (float)(h->sig.fs / h->sig.c);
    prm.fc_c = (float)(h->sig.fc / h->sig.c);
    prm.U = U; prm.npos = npos; prm.seglen = seglen; prm.seg_align = align; prm.slot_bytes = slot_bytes;
    prm.skip_copies = h->debug_skip_copies;
    prm.wait_ns = (unsigned long long)(h->debug_wait_ms > 0 ? h->debug_wait_ms : 4000) * 1000000ull;

    const long long ntiles = (long long)prm.tiles_x * prm.tiles_y * prm.tiles_z;
    const int sms = sm_count();
    // small images: split the pairs of each tile over several CTAs to fill the GPU
    int nsplit = 1;
    if (ntiles < 2LL * sms) {
        nsplit = (int)((2LL * sms + ntiles - 1) / ntiles);
        const long long maxsplit = std::max(1LL, prm.npairs / (2 * PAIRS));
        nsplit = (int)std::min<long long>(nsplit, maxsplit);
    }
    prm.nsplit = nsplit;
    prm.atomic_out = nsplit > 1;
    prm.accumulate = a.accumulate;
    prm.image = a.image;
    if (ntiles * nsplit > 0x7fffffffLL) {
        set_error("grid too large");
        return SAS_ERR_UNSUPPORTED;
    }
    if (prm.atomic_out && !a.accumulate)
        SAS_CUDA(cudaMemsetAsync(a.image, 0, sizeof(float2) * (size_t)g.nx * g.ny * prm.nz, a.stream));

    CUtensorMap map;
    int rc = encode_echo_map(&map, h->d_echo, elem, h->Ns, h->P * h->C, seglen);
    if (rc != SAS_OK) return rc;
    const int blocks = (int)(ntiles * nsplit);
    switch (h->echo_dtype) {
        case SAS_ECHO_C64:
            return a.dim3 ? launch_t<float2, true>(a, prm, map, smem, blocks)
                          : launch_t<float2, false>(a, prm, map, smem, blocks);
        case SAS_ECHO_C32_F16:
            return a.dim3 ? launch_t<__half2, true>(a, prm, map, smem, blocks)
                          : launch_t<__half2, false>(a, prm, map, smem, blocks);
        case SAS_ECHO_C32_BF16:
            return a.dim3 ? launch_t<__nv_bfloat162, true>(a, prm, map, smem, blocks)
                          : launch_t<__nv_bfloat162, false>(a, prm, map, smem, blocks);
        default:
            set_error("no echo uploaded");
            return SAS_ERR_STATE;
    }
}

}  // namespace sas
