// Displaced-phase-centre (DPC) micronavigation (Sec. II-D, Eqs. 3-8):
//  * time-delay estimation between the overlapping receivers of consecutive
//    pings (one thread per measurement window, all lags in its registers);
//  * Eq. 4 residuals and their derivatives in FP64, Eqs. 6-7 regularisers;
//  * Levenberg-Marquardt on Eq. 8 with Gauss-Newton normal equations.  In the
//    velocity variables of the paper the normal matrix is dense (a ping's
//    position integrates all earlier velocities); in the equivalent variables
//    q_j = p_{j+1} (j < P-1, positions of pings 1 .. P-1) and q_{P-1} = v_{P-1}
//    every residual touches at most four consecutive nodes, so the matrix is
//    banded (half-bandwidth 7 over the 2P sway/heave unknowns) and a banded
//    Cholesky solves it.  The minimiser is the same (a linear change of
//    variables); Marquardt's diagonal damping is applied in these variables.
#include "sas_common.cuh"

#include <algorithm>
#include <cmath>
#include <utility>

namespace sas {
namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int BANDW = 7;          // half-bandwidth of the normal matrix
constexpr int BROW = BANDW + 1;   // stored diagonals per row

// ---------------------------------------------------------------------------
// Time-delay estimation

// One thread per measurement m = ((i (C - shift) + c) K + k), 32 consecutive
// m to a warp: e1 = ping i, receiver c + shift; e2 = ping i + 1, receiver c;
// R(tau) = sum_n e2[n] conj(e1[n - tau]) over the window, tau = -L .. L, all
// 2L + 1 lags accumulated in the thread's registers as conj(R): with
// e2 = (bx, by) and e1 = (ax, ay), conj(R) += (bx, bx) (ax, ay) + (by, by)
// (ay, -ax), two packed FP32x2 FMAs, the e2 pairs formed once per sample for
// all lags.  The window is walked in chunks of DPC_CH samples, staged by
// asynchronous copies into two buffers: while a chunk is correlated, the
// warp's copies of the next one (for each of its 32 windows, e2[nb .. nb +
// CH) and e1[nb - L .. nb + CH + L), zero outside the rows and, for e2, past
// the window) are in flight.  Rows have odd strides, so the 32 threads, each
// reading its own window, hit distinct banks.  Energies: sum |e2|^2 over the
// window, and for e1 the total over [n0 - L, n0 + W + L) with its first 2L
// terms kept; the energy under the peak lag is that total less the head
// before and the tail after the shifted window.
constexpr int DPC_TW = 2;         // warps per block
constexpr int DPC_CH = 16;        // samples per window and chunk
constexpr int DPC_MAXL = 15;

template <typename ET, int L>
struct DpcShape {
    static constexpr int NL = 2 * L + 1;
    static constexpr int S2 = DPC_CH + 1;            // odd row strides (elements)
    static constexpr int S1 = DPC_CH + 2 * L + 1;
    static constexpr int NH = L > 0 ? 2 * L : 1;     // head energies kept per window (registers)
    static constexpr int U = L <= 8 ? 8 : 4;         // samples per register block
    static constexpr size_t PAR = 32 * 32;           // window table: 32 B a window
    static constexpr size_t BUF = (sizeof(ET) * 32 * (S1 + S2) + 15) / 16 * 16;   // one chunk of the 32 windows
    static constexpr size_t WARP_BYTES = PAR + 2 * BUF;
    static constexpr size_t SMEM = DPC_TW * WARP_BYTES;
};

struct DpcWin {
    long long e1, e2;   // element offsets of the rows of e1 and e2
    int n0, live;
    float sc1, sc2;
};

template <typename ET>
__device__ __forceinline__ float2 dpc_value(ET v, float sc);
template <>
__device__ __forceinline__ float2 dpc_value<float2>(float2 v, float) {
    return v;
}
template <>
__device__ __forceinline__ float2 dpc_value<__half2>(__half2 v, float sc) {
    const float2 f = __half22float2(v);
    return make_float2(f.x * sc, f.y * sc);
}
template <>
__device__ __forceinline__ float2 dpc_value<__nv_bfloat162>(__nv_bfloat162 v, float sc) {
    const float2 f = __bfloat1622float2(v);
    return make_float2(f.x * sc, f.y * sc);
}

// asynchronous copy of one element into shared memory; zero-filled (nothing
// read) when !valid
template <typename ET>
__device__ __forceinline__ void dpc_copy(ET* dst, const ET* src, bool valid) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    const int n = valid ? (int)sizeof(ET) : 0;
    if constexpr (sizeof(ET) == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d), "l"(src), "r"(n) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(src), "r"(n) : "memory");
}

template <typename ET, int L>
__global__ void __launch_bounds__(32 * DPC_TW)
    dpc_delay_kernel(const ET* __restrict__ echo, const float* __restrict__ scale, int C, int Ns, int shift,
                     const int* __restrict__ centres, int K, int W, long long M, float inv_fs, float inv_wfc,
                     double* __restrict__ coarse, double* __restrict__ fine, double* __restrict__ rho) {
    using S = DpcShape<ET, L>;
    constexpr int NL = S::NL, U = S::U;
    constexpr size_t BUFE = S::BUF / sizeof(ET);
    extern __shared__ __align__(16) unsigned char dpc_smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char* base = dpc_smem + warp * S::WARP_BYTES;
    DpcWin* win = reinterpret_cast<DpcWin*>(base);                            // [32]
    ET* buf0 = reinterpret_cast<ET*>(base + S::PAR);                          // [2] x ([32][S1] e1, [32][S2] e2)
    const long long m0 = ((long long)blockIdx.x * DPC_TW + warp) * 32;
    if (m0 >= M) return;   // whole warps
    const long long m = m0 + lane;
    const bool live = m < M;
    float sc1 = 1.f, sc2 = 1.f;
    {
        DpcWin wn = {0, 0, 0, 0, 1.f, 1.f};
        if (live) {
            const int nc = C - shift;
            const int k = (int)(m % K);
            const long long pr = m / K;
            const int c = (int)(pr % nc);
            const long long i = pr / nc;
            const long long r1 = i * C + c + shift, r2 = (i + 1) * C + c;
            wn.e1 = r1 * Ns;
            wn.e2 = r2 * Ns;
            wn.n0 = centres[k] - W / 2;
            wn.live = 1;
            if (scale) {
                wn.sc1 = scale[r1];
                wn.sc2 = scale[r2];
            }
        }
        sc1 = wn.sc1;
        sc2 = wn.sc2;
        win[lane] = wn;
    }
    __syncwarp();
    // copies of the chunk at `off` of the 32 windows into buffer b
    auto stage = [&](int off, int b) {
        ET* s1 = buf0 + b * BUFE;
        ET* s2 = s1 + 32 * S::S1;
        const int lw = min(DPC_CH, W - off);
        for (int w = 0; w < 32; ++w) {
            const DpcWin wn = win[w];
            const int nb = wn.n0 + off;
            if (lane < DPC_CH) {
                const int n = nb + lane;
                const bool ok = wn.live && lane < lw && n >= 0 && n < Ns;
                dpc_copy(s2 + w * S::S2 + lane, echo + wn.e2 + (ok ? n : 0), ok);
            }
#pragma unroll
            for (int h = 0; h < (DPC_CH + 2 * L + 31) / 32; ++h) {
                const int j = lane + 32 * h, n1 = nb - L + j;
                if (j < DPC_CH + 2 * L) {
                    const bool ok = wn.live && n1 >= 0 && n1 < Ns;
                    dpc_copy(s1 + w * S::S1 + j, echo + wn.e1 + (ok ? n1 : 0), ok);
                }
            }
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    float2 acc[NL];   // conj(R(tau)), tau = t - L
#pragma unroll
    for (int t = 0; t < NL; ++t) acc[t] = make_float2(0.f, 0.f);
    float2 p2v = make_float2(0.f, 0.f);   // sum |e2|^2 (two partial sums)
    float etot = 0.f;                     // sum |e1|^2 over [n0 - L, n0 + W + L)
    float eh[S::NH];                      // its first 2L terms
#pragma unroll
    for (int q = 0; q < S::NH; ++q) eh[q] = 0.f;
    const int nch = (W + DPC_CH - 1) / DPC_CH;
    int len = 0;
    const ET* a1 = buf0;
    stage(0, 0);
    for (int ci = 0; ci < nch; ++ci) {
        const int off = ci * DPC_CH;
        len = min(DPC_CH, W - off);
        if (ci + 1 < nch) {
            stage(off + DPC_CH, (ci + 1) & 1);
            asm volatile("cp.async.wait_group 1;" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;" ::: "memory");
        }
        __syncwarp();
        a1 = buf0 + (ci & 1) * BUFE + lane * S::S1;
        const ET* b2s = buf0 + (ci & 1) * BUFE + 32 * S::S1 + lane * S::S2;
        // e1 energy: the staged samples [nb + L, nb + L + len); in the first
        // chunk also [n0 - L, n0 + L), kept for the head sums
        if (ci == 0) {
#pragma unroll
            for (int q = 0; q < 2 * L; ++q) {
                const float2 v = dpc_value(a1[q], sc1);
                const float e = fmaf(v.x, v.x, v.y * v.y);
                eh[q] = e;
                etot += e;
            }
        }
        for (int q = 0; q < len; ++q) {
            const float2 v = dpc_value(a1[2 * L + q], sc1);
            etot = fmaf(v.x, v.x, fmaf(v.y, v.y, etot));
        }
        // conj(R(tau)) over the chunk (e2 is zero past the window)
#pragma unroll 1
        for (int j0 = 0; j0 < DPC_CH; j0 += U) {
            float2 bx[U], by[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const float2 b = dpc_value(b2s[j0 + u], sc2);
                p2v = ffma2(b, b, p2v);
                bx[u] = make_float2(b.x, b.x);
                by[u] = make_float2(b.y, b.y);
            }
            // e1 staged at j0 + q serves sample j0 + u at lag t = u + 2L - q
#pragma unroll
            for (int q = 0; q < U + 2 * L; ++q) {
                const float2 a = dpc_value(a1[j0 + q], sc1);
                const float2 am = make_float2(a.y, -a.x);
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int t = u + 2 * L - q;
                    if (t >= 0 && t < NL) {
                        acc[t] = ffma2(bx[u], a, acc[t]);
                        acc[t] = ffma2(by[u], am, acc[t]);
                    }
                }
            }
        }
        __syncwarp();   // the buffer is refilled two chunks later
    }
    if (!live) return;
    // largest |R|, the lowest lag on ties
    float best2 = -1.f;
    int bl = 0;
#pragma unroll
    for (int t = 0; t < NL; ++t) {
        const float q = fmaf(acc[t].x, acc[t].x, acc[t].y * acc[t].y);
        if (q > best2) {
            best2 = q;
            bl = t;
        }
    }
    float2 R0 = acc[0], Rm = acc[0], Rp = acc[0];
#pragma unroll
    for (int t = 0; t < NL; ++t) {
        if (t == bl) R0 = acc[t];
        if (t == bl - 1) Rm = acc[t];
        if (t == bl + 1) Rp = acc[t];
    }
    R0.y = -R0.y;   // R: the conjugates of the accumulated sums
    Rm.y = -Rm.y;
    Rp.y = -Rp.y;
    const float best = sqrtf(best2);
    float d = 0.f, Rr = R0.x, Ri = R0.y;
    if (bl > 0 && bl < 2 * L) {
        const float mm = sqrtf(fmaf(Rm.x, Rm.x, Rm.y * Rm.y)), mp = sqrtf(fmaf(Rp.x, Rp.x, Rp.y * Rp.y));
        const float den = mm - 2.f * best + mp;
        d = den != 0.f ? 0.5f * (mm - mp) / den : 0.f;
        Rr = R0.x + 0.5f * d * (Rp.x - Rm.x) + 0.5f * d * d * (Rp.x - 2.f * R0.x + Rm.x);
        Ri = R0.y + 0.5f * d * (Rp.y - Rm.y) + 0.5f * d * d * (Rp.y - 2.f * R0.y + Rm.y);
    }
    // FP32 epilogue (FP64 arithmetic is slow on this part; the outputs carry
    // FP32 accuracy anyway), widened on the store
    if (coarse) coarse[m] = (double)(((float)(bl - L) + d) * inv_fs);
    if (fine) fine[m] = (double)(-atan2f(Ri, Rr) * inv_wfc);
    if (rho) {
        // e1 energy under the peak lag tau = bl - L: the window [n0 - tau, n0 - tau + W)
        // is the extended range less its first 2L - bl and its last bl terms
        float head = 0.f, tail = 0.f;
#pragma unroll
        for (int q = 0; q < 2 * L; ++q)
            if (q < 2 * L - bl) head += eh[q];
        for (int q = 0; q < bl; ++q) {
            const float2 v = dpc_value(a1[len + 2 * L - 1 - q], sc1);
            tail = fmaf(v.x, v.x, fmaf(v.y, v.y, tail));
        }
        const float q1 = etot - head - tail, den2 = (p2v.x + p2v.y) * q1;
        rho[m] = den2 > 0.f ? (double)(best * rsqrtf(den2)) : 0.0;
    }
}

template <typename ET, int L>
cudaError_t dpc_delay_launch(const ET* echo, const float* scale, int C, int Ns, int shift, const int* centres, int K,
                             int W, long long M, float inv_fs, float inv_wfc, double* coarse, double* fine,
                             double* rho, cudaStream_t st) {
    using S = DpcShape<ET, L>;
    cudaError_t e =
        cudaFuncSetAttribute(dpc_delay_kernel<ET, L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::SMEM);
    if (e != cudaSuccess) return e;
    const long long warps = (M + 31) / 32;
    dpc_delay_kernel<ET, L><<<(unsigned)((warps + DPC_TW - 1) / DPC_TW), 32 * DPC_TW, S::SMEM, st>>>(
        echo, scale, C, Ns, shift, centres, K, W, M, inv_fs, inv_wfc, coarse, fine, rho);
    return cudaGetLastError();
}

template <typename ET>
cudaError_t dpc_delay_dispatch(int L, const ET* echo, const float* scale, int C, int Ns, int shift,
                               const int* centres, int K, int W, long long M, float inv_fs, float inv_wfc,
                               double* coarse, double* fine, double* rho, cudaStream_t st) {
#define SAS_DPC_L(LL)                                                                                             \
    case LL:                                                                                                      \
        return dpc_delay_launch<ET, LL>(echo, scale, C, Ns, shift, centres, K, W, M, inv_fs, inv_wfc, coarse,   \
                                        fine, rho, st);
    switch (L) {
        SAS_DPC_L(0) SAS_DPC_L(1) SAS_DPC_L(2) SAS_DPC_L(3) SAS_DPC_L(4) SAS_DPC_L(5) SAS_DPC_L(6) SAS_DPC_L(7)
        SAS_DPC_L(8) SAS_DPC_L(9) SAS_DPC_L(10) SAS_DPC_L(11) SAS_DPC_L(12) SAS_DPC_L(13) SAS_DPC_L(14) SAS_DPC_L(15)
        default: return cudaErrorInvalidValue;
    }
#undef SAS_DPC_L
}

// ---------------------------------------------------------------------------
// Motion model

struct Prob {
    int P, C, shift, K, nc, side;
    long long M;
    double c, lambda1, lambda2, huber;
    const double *p0, *vx, *att, *dt, *ltx, *lrx, *t, *delay, *weight, *zdvl, *ps;
    const double* lev;   // [P][C + 1][3] rotated lever arms R_i l (TX first)
    const double* xpos;  // [P] along-track positions
};

struct V3 {
    double x, y, z;
};
__device__ __forceinline__ V3 v3(const double* a) { return V3{a[0], a[1], a[2]}; }
__device__ __forceinline__ V3 operator+(V3 a, V3 b) { return V3{a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ V3 operator-(V3 a, V3 b) { return V3{a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ V3 operator*(double s, V3 a) { return V3{s * a.x, s * a.y, s * a.z}; }
__device__ __forceinline__ double norm(V3 a) { return sqrt(a.x * a.x + a.y * a.y + a.z * a.z); }

// Position and velocity of ping i from the nodes q (sway, heave) and the known
// along-track terms.
__device__ __forceinline__ void ping_pv(const Prob& pb, const double* q, int i, V3& p, V3& v) {
    auto pos = [&](int j) -> V3 {
        return j == 0 ? v3(pb.p0) : V3{pb.xpos[j], q[2 * (j - 1)], q[2 * (j - 1) + 1]};
    };
    p = pos(i);
    if (i < pb.P - 1) {
        const V3 pn = pos(i + 1);
        const double r = 1.0 / pb.dt[i];
        v = V3{pb.vx[i], (pn.y - p.y) * r, (pn.z - p.z) * r};
    } else {
        v = V3{pb.vx[i], q[2 * i], q[2 * i + 1]};
    }
}

// Rotated lever arms R_i l_TX, R_i l_c and along-track positions (one thread per ping).
__global__ void dpc_lever_kernel(Prob pb, double* lev) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= pb.P) return;
    double R[9];
    attitude_rotation(pb.att[3 * i], pb.att[3 * i + 1], pb.att[3 * i + 2], R);
    for (int c = -1; c < pb.C; ++c) {
        const double* l = c < 0 ? pb.ltx : pb.lrx + 3 * c;
        double* o = lev + 3 * ((size_t)i * (pb.C + 1) + (c + 1));
        o[0] = R[0] * l[0] + R[1] * l[1] + R[2] * l[2];
        o[1] = R[3] * l[0] + R[4] * l[1] + R[5] * l[2];
        o[2] = R[6] * l[0] + R[7] * l[1] + R[8] * l[2];
    }
}

// Nodes q from velocities (positions integrated from p_0), and the along-track positions.
__global__ void dpc_nodes_kernel(Prob pb, const double* vy, const double* vz, double* q, double* xpos) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    double x = pb.p0[0], y = pb.p0[1], z = pb.p0[2];
    xpos[0] = x;
    for (int i = 0; i + 1 < pb.P; ++i) {
        x += pb.vx[i] * pb.dt[i];
        y += vy[i] * pb.dt[i];
        z += vz[i] * pb.dt[i];
        xpos[i + 1] = x;
        q[2 * i] = y;
        q[2 * i + 1] = z;
    }
    q[2 * (pb.P - 1)] = vy[pb.P - 1];
    q[2 * (pb.P - 1) + 1] = vz[pb.P - 1];
}

__global__ void dpc_velocities_kernel(Prob pb, const double* q, double* vy, double* vz) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= pb.P) return;
    V3 p, v;
    ping_pv(pb, q, i, p, v);
    vy[i] = v.y;
    vz[i] = v.z;
}

// Footprint of measurement m from the nodes q (the prior).
__global__ void dpc_footprint_kernel(Prob pb, const double* q, double* ps) {
    const long long m = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= pb.M) return;
    const int k = (int)(m % pb.K);
    const long long pr = m / pb.K;
    const int c = (int)(pr % pb.nc);
    const int i = (int)(pr / pb.nc);
    V3 p, v;
    ping_pv(pb, q, i, p, v);
    const double* lv = pb.lev + 3 * (size_t)i * (pb.C + 1);
    const V3 pc = p + 0.5 * (v3(lv) + v3(lv + 3 * (c + pb.shift + 1)));
    double sy, cy;
    sincos(pb.att[3 * i + 2], &sy, &cy);
    const double rng = 0.5 * pb.c * pb.t[k];
    const double ground = sqrt(fmax(rng * rng - pc.z * pc.z, 0.0));
    ps[3 * m + 0] = pc.x + ground * (-sy) * pb.side;
    ps[3 * m + 1] = pc.y + ground * cy * pb.side;
    ps[3 * m + 2] = 0.0;
}

// r = c g (Eq. 4, metres) of measurement m with the measured delay (or 0), and
// its derivatives with respect to the sway / heave of p_i, v_i, p_{i+1}, v_{i+1}.
struct Res {
    double r;
    double dp1[2], dv1[2], dp2[2], dv2[2];
};
template <bool JAC>
__device__ __forceinline__ Res dpc_residual(const Prob& pb, const double* q, long long m, bool with_delay) {
    const int k = (int)(m % pb.K);
    const long long pr = m / pb.K;
    const int c = (int)(pr % pb.nc);
    const int i = (int)(pr / pb.nc);
    const double t = pb.t[k];
    V3 p1, v1, p2, v2;
    ping_pv(pb, q, i, p1, v1);
    ping_pv(pb, q, i + 1, p2, v2);
    const double* l1 = pb.lev + 3 * (size_t)i * (pb.C + 1);
    const double* l2 = pb.lev + 3 * (size_t)(i + 1) * (pb.C + 1);
    const V3 s = v3(pb.ps + 3 * m);
    const V3 a1 = p1 + v3(l1) - s, b1 = p1 + t * v1 + v3(l1 + 3 * (c + pb.shift + 1)) - s;
    const V3 a2 = p2 + v3(l2) - s, b2 = p2 + t * v2 + v3(l2 + 3 * (c + 1)) - s;
    const double na1 = norm(a1), nb1 = norm(b1), na2 = norm(a2), nb2 = norm(b2);
    Res o;
    o.r = (na1 + nb1) - (na2 + nb2) + (with_delay ? pb.c * pb.delay[m] : 0.0);
    if (JAC) {
        const double ia1 = 1.0 / na1, ib1 = 1.0 / nb1, ia2 = 1.0 / na2, ib2 = 1.0 / nb2;
        o.dp1[0] = a1.y * ia1 + b1.y * ib1;
        o.dp1[1] = a1.z * ia1 + b1.z * ib1;
        o.dv1[0] = t * b1.y * ib1;
        o.dv1[1] = t * b1.z * ib1;
        o.dp2[0] = -(a2.y * ia2 + b2.y * ib2);
        o.dp2[1] = -(a2.z * ia2 + b2.z * ib2);
        o.dv2[0] = -t * b2.y * ib2;
        o.dv2[1] = -t * b2.z * ib2;
    }
    return o;
}

__global__ void dpc_model_kernel(Prob pb, const double* q, double* out) {
    const long long m = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= pb.M) return;
    out[m] = -dpc_residual<false>(pb, q, m, false).r / pb.c;
}

// Eq. 5 / Eq. 3 term and the iteratively reweighted weight of a residual.
__device__ __forceinline__ void robust(const Prob& pb, double r, double om, double& cost, double& w) {
    if (pb.huber > 0.0) {
        const double a = fabs(r);
        if (a <= pb.huber) {
            cost = om * r * r;
            w = om;
        } else {
            cost = om * (2.0 * pb.huber * a - pb.huber * pb.huber);
            w = om * pb.huber / a;
        }
    } else {
        cost = om * r * r;
        w = om;
    }
}

// Band index of the normal matrix entry (a, b), a <= b <= a + BANDW.
__device__ __forceinline__ size_t bidx(int a, int b) { return (size_t)a * BROW + (b - a); }

// DPC part of the loss (acc[0]) and, with JAC, of the normal matrix and the
// gradient: one block per ping pair, its (C - shift) K measurements over the
// threads, a block reduction, one atomic per entry.
template <bool JAC>
__global__ void __launch_bounds__(256) dpc_assemble_kernel(Prob pb, const double* q, double* band, double* grad,
                                                           double* acc) {
    const int i = blockIdx.x;   // ping pair
    const long long per = (long long)pb.nc * pb.K;
    // local unknowns: nodes i-1 (absent for i = 0), i, i+1, sway and heave each
    constexpr int NL = 6, NT = NL * (NL + 1) / 2;
    double cst = 0.0, g[NL] = {0, 0, 0, 0, 0, 0}, H[NT];
#pragma unroll
    for (int e = 0; e < NT; ++e) H[e] = 0.0;
    const double r1 = 1.0 / pb.dt[i];
    const bool last = i + 1 == pb.P - 1;
    const double r2 = last ? 1.0 : 1.0 / pb.dt[i + 1];
    for (long long e = threadIdx.x; e < per; e += blockDim.x) {
        const long long m = (long long)i * per + e;
        const Res o = dpc_residual<JAC>(pb, q, m, true);
        double cm, w;
        robust(pb, o.r, pb.weight ? pb.weight[m] : 1.0, cm, w);
        cst += cm;
        if (JAC) {
            double J[NL];
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                J[a] = i > 0 ? o.dp1[a] - o.dv1[a] * r1 : 0.0;                            // node i-1 (p_i, v_i)
                J[2 + a] = o.dp2[a] + o.dv1[a] * r1 - (last ? 0.0 : o.dv2[a] * r2);     // node i (p_{i+1}, v_i, v_{i+1})
                J[4 + a] = o.dv2[a] * r2;                                               // node i+1 (v_{i+1})
            }
            int t = 0;
#pragma unroll
            for (int a = 0; a < NL; ++a) {
                g[a] = fma(w * J[a], o.r, g[a]);
#pragma unroll
                for (int b = a; b < NL; ++b) {
                    H[t] = fma(w * J[a], J[b], H[t]);
                    ++t;
                }
            }
        }
    }
    // block reduction: warps by shuffles, then across warps in shared memory
    __shared__ double red[8][1 + NL + NT];
    auto wsum = [&](double v) {
#pragma unroll
        for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
        return v;
    };
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    cst = wsum(cst);
    if (JAC) {
#pragma unroll
        for (int a = 0; a < NL; ++a) g[a] = wsum(g[a]);
#pragma unroll
        for (int e = 0; e < NT; ++e) H[e] = wsum(H[e]);
    }
    if (lane == 0) {
        red[warp][0] = cst;
        if (JAC) {
            for (int a = 0; a < NL; ++a) red[warp][1 + a] = g[a];
            for (int e = 0; e < NT; ++e) red[warp][1 + NL + e] = H[e];
        }
    }
    __syncthreads();
    const int nw = blockDim.x >> 5;
    const int nval = JAC ? 1 + NL + NT : 1;
    if ((int)threadIdx.x < nval) {
        double s = 0.0;
        for (int w2 = 0; w2 < nw; ++w2) s += red[w2][threadIdx.x];
        const int v = threadIdx.x;
        if (v == 0) {
            atomicAdd(&acc[0], s);
        } else if (v <= NL) {
            const int a = v - 1;
            const int node = i - 1 + a / 2;
            if (node >= 0) atomicAdd(&grad[2 * node + (a & 1)], s);
        } else {
            // entry e of the upper triangle -> (a, b)
            int e = v - 1 - NL, a = 0;
            while (e >= NL - a) {
                e -= NL - a;
                ++a;
            }
            const int b = a + e;
            const int na = i - 1 + a / 2, nb = i - 1 + b / 2;
            if (na >= 0 && nb >= 0) {
                const int ga = 2 * na + (a & 1), gb = 2 * nb + (b & 1);
                atomicAdd(&band[bidx(min(ga, gb), max(ga, gb))], s);
            }
        }
    }
}

// Regularisers (Eqs. 6, 7): one thread per ping; loss into acc[0].
template <bool JAC>
__global__ void dpc_regular_kernel(Prob pb, const double* q, double* band, double* grad, double* acc) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double cst = 0.0;
    if (i < pb.P) {
        // DVL: p_z,i - z_dvl[i]
        const double pz = i == 0 ? pb.p0[2] : q[2 * (i - 1) + 1];
        const double d = pz - pb.zdvl[i];
        cst += pb.lambda2 * d * d;
        if (JAC && i > 0) {
            const int u = 2 * (i - 1) + 1;
            atomicAdd(&band[bidx(u, u)], pb.lambda2);
            atomicAdd(&grad[u], pb.lambda2 * d);
        }
        // smoothness: v[i+1] - 2 v[i] + v[i-1], sway (comp 0) and heave (comp 1)
        if (i >= 1 && i + 1 < pb.P) {
            for (int comp = 0; comp < 2; ++comp) {
                // v_n = (P_{n+1} - P_n) / dt_n (n < P-1), v_{P-1} = q_{P-1}; P_0 = p0, P_j = q_{j-1}
                int node[4];
                double coef[4], s = 0.0;
                int nn = 0;
                auto add = [&](int nd, double cf) {
                    if (nd < 0) return;
                    for (int z = 0; z < nn; ++z)
                        if (node[z] == nd) {
                            coef[z] += cf;
                            return;
                        }
                    node[nn] = nd;
                    coef[nn] = cf;
                    ++nn;
                };
                auto vel = [&](int n, double wgt) {
                    if (n < pb.P - 1) {
                        const double r = 1.0 / pb.dt[n];
                        const double a = q[2 * n + comp];                                          // P_{n+1} = q_n
                        const double b = n == 0 ? (comp ? pb.p0[2] : pb.p0[1]) : q[2 * (n - 1) + comp];   // P_n
                        s += wgt * (a - b) * r;
                        add(n, wgt * r);
                        add(n - 1, -wgt * r);
                    } else {
                        s += wgt * q[2 * n + comp];
                        add(n, wgt);
                    }
                };
                vel(i + 1, 1.0);
                vel(i, -2.0);
                vel(i - 1, 1.0);
                cst += pb.lambda1 * s * s;
                if (JAC) {
                    for (int a = 0; a < nn; ++a) {
                        const int ga = 2 * node[a] + comp;
                        atomicAdd(&grad[ga], pb.lambda1 * coef[a] * s);
                        for (int b = 0; b < nn; ++b) {
                            const int gb = 2 * node[b] + comp;
                            if (gb >= ga) atomicAdd(&band[bidx(ga, gb)], pb.lambda1 * coef[a] * coef[b]);
                        }
                    }
                }
            }
        }
    }
    // block sum of the loss
    __shared__ double red[32];
    for (int o = 16; o; o >>= 1) cst += __shfl_xor_sync(FULL, cst, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = cst;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        atomicAdd(&acc[0], s);
    }
}

// Damped banded Cholesky solve of (N + mu diag N) delta = -g and the trial
// nodes q + delta, by one warp, right-looking: the pending entries of the next
// BANDW + 1 rows sit in a ring in shared memory; row j's factor U(j, j + d) is
// one multiplication by 1 / sqrt(pending diagonal) per lane, and its rank-1
// update of the trailing 7 x 7 triangle is one FMA on each of 28 lanes, so the
// critical path per row is one reciprocal square root and a few FP64
// operations (no sequential dot products).  The forward substitution
// U^T y = -g rides along (its right-hand side updated the same way); the back
// substitution runs on one lane.  The rows of the band and of g (forward),
// and of U and y (backward, in reverse), stream through shared memory in
// chunks of 2^rlog rows (at most SOL_R) by asynchronous copies, the next chunk
// in flight while the current one is used, so no global-memory latency sits
// on the chain.  acc[1] = 1 when the factorisation fails; acc[2] = max |delta|.
constexpr int SOL_R = 512;
int g_sol_rlog = 9;   // chunk rows 2^9 = SOL_R; smaller through sas_debug_dpc_solve_chunk
static_assert(BANDW == 7, "the back substitution keeps seven deltas in registers");
constexpr size_t SOL_SMEM = sizeof(double) * 2 * SOL_R * (BROW + 1);

__device__ __forceinline__ void sol_copy8(double* dst, const double* src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
}

// rows [c R, min(n, c R + R)) of a [n][w] array into buf [R][w]
__device__ __forceinline__ void sol_stage(double* buf, const double* src, int n, int w, int c, int R, int lane) {
    const int r0 = c * R, r1 = min(n, r0 + R);
    for (int i = lane; i < (r1 - r0) * w; i += 32) sol_copy8(buf + i, src + (size_t)r0 * w + i);
}

__global__ void __launch_bounds__(32) dpc_solve_kernel(int n, const double* band, const double* grad, double mu,
                                                       double* work, const double* q, double* q_try, double* acc,
                                                       int rlog) {
    extern __shared__ __align__(16) double sol_sm[];
    double* bbuf = sol_sm;                          // [2][SOL_R][BROW]: band rows, then U rows
    double* gbuf = sol_sm + 2 * SOL_R * BROW;       // [2][SOL_R]: g, then y
    __shared__ double Pm[BROW][BROW];   // Pm[r % BROW][d] = pending A(r, r + d), rows j .. j + BANDW
    __shared__ double tv[BROW];         // pending right-hand side of those rows
    const int lane = threadIdx.x;
    double* U = work;                   // [n][BROW], the diagonal stored inverted
    double* y = work + (size_t)n * BROW;
    const int R = 1 << rlog;            // chunk rows, 8 .. SOL_R; buffers keep the SOL_R stride
    const int nch = (n + R - 1) / R;
    auto commit = [] { asm volatile("cp.async.commit_group;" ::: "memory"); };
    auto wait1 = [] { asm volatile("cp.async.wait_group 1;" ::: "memory"); };
    auto wait0 = [] { asm volatile("cp.async.wait_group 0;" ::: "memory"); };
    auto stage_fwd = [&](int c) {
        sol_stage(bbuf + (c & 1) * SOL_R * BROW, band, n, BROW, c, R, lane);
        sol_stage(gbuf + (c & 1) * SOL_R, grad, n, 1, c, R, lane);
        commit();
    };
    // lane -> entry (j + ta, j + tb) of the trailing triangle, 1 <= ta <= tb <= BANDW
    int ta = 1, e = lane;
    while (ta <= BANDW && e >= BANDW - ta + 1) {
        e -= BANDW - ta + 1;
        ++ta;
    }
    const int tb = ta + e;
    const bool upd = lane < BANDW * (BANDW + 1) / 2;
    // row r of the damped matrix and of -g (lanes 0 .. BANDW; zero past the end),
    // from its staged chunk
    auto fetch = [&](int r, double& a, double& t) {
        a = 0.0;
        t = 0.0;
        if (lane <= BANDW && r < n && r + lane < n) {
            const int c = r >> rlog, i = r & (R - 1);
            a = bbuf[((c & 1) * SOL_R + i) * BROW + lane];
            if (lane == 0) {
                a += mu * (a + 1e-12);   // Marquardt's scaling, Levenberg's floor
                t = -gbuf[(c & 1) * SOL_R + i];
            }
        }
    };
    if (lane == 0) acc[1] = 0.0;
    stage_fwd(0);
    if (nch > 1) {
        stage_fwd(1);
        wait1();
    } else {
        wait0();
    }
    __syncwarp();
    for (int r = 0; r < BROW; ++r) {
        double a, t;
        fetch(r, a, t);
        if (lane <= BANDW) Pm[r][lane] = a;
        if (lane == 0) tv[r] = t;
    }
    __syncwarp();
    for (int j = 0; j < n; ++j) {
        const int rn = j + BROW;
        if (rn < n && (rn & (R - 1)) == 0) {
            // the fetches move to chunk rn / R: chunk rn / R - 1 is done with,
            // its buffer takes chunk rn / R + 1
            const int c = rn >> rlog;
            __syncwarp();
            if (c + 1 < nch) {
                stage_fwd(c + 1);
                wait1();
            } else {
                wait0();
            }
            __syncwarp();
        }
        double an, tn;
        fetch(rn, an, tn);
        const int sj = j % BROW;
        const double djj = Pm[sj][0];
        if (!(djj > 0.0)) {
            if (lane == 0) acc[1] = 1.0;
            wait0();
            return;
        }
        const double inv = rsqrt(djj);
        double u = 0.0;
        if (lane <= BANDW && j + lane < n) {
            u = lane == 0 ? djj * inv : Pm[sj][lane] * inv;
            U[(size_t)j * BROW + lane] = lane == 0 ? inv : u;
        }
        const double yj = tv[sj] * inv;
        if (lane == 0) y[j] = yj;
        const double ua = __shfl_sync(FULL, u, ta & 31), ub = __shfl_sync(FULL, u, tb & 31);
        __syncwarp();
        if (upd && j + tb < n) Pm[(j + ta) % BROW][tb - ta] -= ua * ub;
        if (lane >= 1 && lane <= BANDW && j + lane < n) tv[(j + lane) % BROW] -= u * yj;
        // row j's slot takes row j + BROW (untouched by rows <= j: it lies beyond their band)
        if (lane <= BANDW) Pm[sj][lane] = an;
        if (lane == 0) tv[sj] = tn;
        __syncwarp();
    }
    wait0();
    // U delta = y, rows n - 1 .. 0, U and y streamed back in reverse chunks
    __threadfence_block();
    __syncwarp();
    auto stage_bwd = [&](int c) {
        sol_stage(bbuf + (c & 1) * SOL_R * BROW, U, n, BROW, c, R, lane);
        sol_stage(gbuf + (c & 1) * SOL_R, y, n, 1, c, R, lane);
        commit();
    };
    stage_bwd(nch - 1);
    if (nch > 1) {
        stage_bwd(nch - 2);
        wait1();
    } else {
        wait0();
    }
    __syncwarp();
    // delta of rows j + 1 .. j + 7 in registers; the terms of rows j + 2 ..
    // j + 7 are summed before delta_{j+1} is known, so one FMA and one
    // multiplication per row are on the dependent chain
    double d1 = 0.0, d2 = 0.0, d3 = 0.0, d4 = 0.0, d5 = 0.0, d6 = 0.0, d7 = 0.0;
    double dmax = 0.0;
    for (int j = n - 1; j >= 0; --j) {
        const int c = j >> rlog, i = j & (R - 1);
        if (i == R - 1 && c < nch - 1) {
            // entering chunk c from above: chunk c + 1 is done with, its buffer
            // takes chunk c - 1
            __syncwarp();
            if (c >= 1) {
                stage_bwd(c - 1);
                wait1();
            } else {
                wait0();
            }
            __syncwarp();
        }
        if (lane == 0) {
            // entries past row n - 1 were never written: only j + d < n is read
            const double* Ur = bbuf + ((c & 1) * SOL_R + i) * BROW;
            double s = gbuf[(c & 1) * SOL_R + i];
            if (j + 7 < n) s -= Ur[7] * d7;
            if (j + 6 < n) s -= Ur[6] * d6;
            if (j + 5 < n) s -= Ur[5] * d5;
            if (j + 4 < n) s -= Ur[4] * d4;
            if (j + 3 < n) s -= Ur[3] * d3;
            if (j + 2 < n) s -= Ur[2] * d2;
            if (j + 1 < n) s -= Ur[1] * d1;
            const double dj = s * Ur[0];
            d7 = d6;
            d6 = d5;
            d5 = d4;
            d4 = d3;
            d3 = d2;
            d2 = d1;
            d1 = dj;
            y[j] = dj;
            dmax = fmax(dmax, fabs(dj));
            q_try[j] = q[j] + dj;
        }
    }
    wait0();
    if (lane == 0) acc[2] = dmax;
}

inline int blocks_for(long long n, int t) { return (int)((n + t - 1) / t); }

int check_problem(const sas_dpc_problem* pr) {
    if (!pr || pr->P < 2 || pr->C < 1 || pr->shift < 0 || pr->shift >= pr->C || pr->K < 1 || !(pr->c > 0) ||
        (pr->side != 1 && pr->side != -1) || !pr->d_p0 || !pr->d_vx || !pr->d_att || !pr->d_dt ||
        !pr->d_tx_lever || !pr->d_rx_lever || !pr->d_t || !(pr->lambda1 >= 0) || !(pr->lambda2 >= 0)) {
        set_error("sas_dpc: bad problem description");
        return SAS_ERR_ARG;
    }
    return SAS_OK;
}

Prob make_prob(const sas_dpc_problem* pr) {
    Prob pb{};
    pb.P = pr->P;
    pb.C = pr->C;
    pb.shift = pr->shift;
    pb.K = pr->K;
    pb.nc = pr->C - pr->shift;
    pb.side = pr->side;
    pb.M = (long long)(pr->P - 1) * pb.nc * pr->K;
    pb.c = pr->c;
    pb.lambda1 = pr->lambda1;
    pb.lambda2 = pr->lambda2;
    pb.huber = pr->huber;
    pb.p0 = pr->d_p0;
    pb.vx = pr->d_vx;
    pb.att = pr->d_att;
    pb.dt = pr->d_dt;
    pb.ltx = pr->d_tx_lever;
    pb.lrx = pr->d_rx_lever;
    pb.t = pr->d_t;
    pb.delay = pr->d_delay;
    pb.weight = pr->d_weight;
    pb.zdvl = pr->d_z_dvl;
    pb.ps = pr->d_ps;
    return pb;
}

// Device scratch of one call: rotated levers, along-track positions, nodes.
struct Scratch {
    double* base = nullptr;
    double *lev, *xpos, *q;
    int alloc(const Prob& pb, size_t extra, cudaStream_t st) {
        const size_t n = (size_t)pb.P * (pb.C + 1) * 3 + (size_t)pb.P + 2 * (size_t)pb.P + extra;
        if (cudaMallocAsync(&base, n * sizeof(double), st) != cudaSuccess) {
            set_error("sas_dpc: device allocation failed");
            return SAS_ERR_OOM;
        }
        lev = base;
        xpos = lev + (size_t)pb.P * (pb.C + 1) * 3;
        q = xpos + pb.P;
        return SAS_OK;
    }
};

// Rotated levers, along-track positions and nodes from the velocities.
int setup(Prob& pb, Scratch& S, const double* vy, const double* vz, cudaStream_t st) {
    dpc_lever_kernel<<<blocks_for(pb.P, 128), 128, 0, st>>>(pb, S.lev);
    dpc_nodes_kernel<<<1, 1, 0, st>>>(pb, vy, vz, S.q, S.xpos);
    SAS_CUDA(cudaGetLastError());
    pb.lev = S.lev;
    pb.xpos = S.xpos;
    return SAS_OK;
}

}  // namespace
}  // namespace sas

using namespace sas;

extern "C" int sas_dpc_delays(sas_geometry_t h, int32_t shift, const int32_t* d_centres, int32_t K, int32_t W,
                              int32_t max_lag, double* d_coarse, double* d_fine, double* d_rho, void* stream) {
    if (!h || !d_centres || K < 1 || W < 1 || W > 4096 || max_lag < 0 || max_lag > DPC_MAXL || shift < 0 ||
        shift >= h->C || h->P < 2) {
        set_error("sas_dpc_delays: bad argument");
        return SAS_ERR_ARG;
    }
    if (h->echo_dtype < 0) {
        set_error("sas_dpc_delays: no echo uploaded");
        return SAS_ERR_STATE;
    }
    const long long M = (long long)(h->P - 1) * (h->C - shift) * K;
    cudaStream_t st = (cudaStream_t)stream;
    const float inv_fs = (float)(1.0 / h->sig.fs), inv_wfc = (float)(1.0 / (2.0 * M_PI * h->sig.fc));
    cudaError_t e;
    switch (h->echo_dtype) {
        case SAS_ECHO_C64:
            e = dpc_delay_dispatch<float2>(max_lag, (const float2*)h->d_echo, nullptr, h->C, h->Ns, shift, d_centres, K,
                                           W, M, inv_fs, inv_wfc, d_coarse, d_fine, d_rho, st);
            break;
        case SAS_ECHO_C32_F16:
            e = dpc_delay_dispatch<__half2>(max_lag, (const __half2*)h->d_echo, h->d_scale, h->C, h->Ns, shift,
                                            d_centres, K, W, M, inv_fs, inv_wfc, d_coarse, d_fine, d_rho, st);
            break;
        default:
            e = dpc_delay_dispatch<__nv_bfloat162>(max_lag, (const __nv_bfloat162*)h->d_echo, h->d_scale, h->C, h->Ns,
                                                   shift, d_centres, K, W, M, inv_fs, inv_wfc, d_coarse, d_fine, d_rho,
                                                   st);
            break;
    }
    SAS_CUDA(e);
    SAS_CUDA(cudaGetLastError());
    return SAS_OK;
}

extern "C" int sas_dpc_footprints(const sas_dpc_problem* pr, const double* d_vy, const double* d_vz, double* d_ps,
                                  void* stream) {
    int rc = check_problem(pr);
    if (rc != SAS_OK) return rc;
    if (!d_vy || !d_vz || !d_ps) {
        set_error("sas_dpc_footprints: null argument");
        return SAS_ERR_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    Prob pb = make_prob(pr);
    Scratch S;
    rc = S.alloc(pb, 0, st);
    if (rc != SAS_OK) return rc;
    rc = setup(pb, S, d_vy, d_vz, st);
    if (rc == SAS_OK) {
        dpc_footprint_kernel<<<blocks_for(pb.M, 256), 256, 0, st>>>(pb, S.q, d_ps);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) rc = cuda_fail(e, "dpc_footprint_kernel");
    }
    cudaFreeAsync(S.base, st);
    return rc;
}

extern "C" int sas_dpc_model_delays(const sas_dpc_problem* pr, const double* d_vy, const double* d_vz, double* d_out,
                                    void* stream) {
    int rc = check_problem(pr);
    if (rc != SAS_OK) return rc;
    if (!d_vy || !d_vz || !d_out || !pr->d_ps) {
        set_error("sas_dpc_model_delays: null argument");
        return SAS_ERR_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    Prob pb = make_prob(pr);
    Scratch S;
    rc = S.alloc(pb, 0, st);
    if (rc != SAS_OK) return rc;
    rc = setup(pb, S, d_vy, d_vz, st);
    if (rc == SAS_OK) {
        dpc_model_kernel<<<blocks_for(pb.M, 256), 256, 0, st>>>(pb, S.q, d_out);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) rc = cuda_fail(e, "dpc_model_kernel");
    }
    cudaFreeAsync(S.base, st);
    return rc;
}

extern "C" int sas_dpc_solve(const sas_dpc_problem* pr, double* d_vy, double* d_vz, int32_t max_iter, double* h_loss,
                             int32_t* h_iters, void* stream) {
    int rc = check_problem(pr);
    if (rc != SAS_OK) return rc;
    if (!d_vy || !d_vz || !pr->d_delay || !pr->d_ps || !pr->d_z_dvl || max_iter < 0) {
        set_error("sas_dpc_solve: bad argument");
        return SAS_ERR_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    Prob pb = make_prob(pr);
    const int n = 2 * pb.P;
    // scratch after the nodes: q_try [n], band [n][BROW], grad [n], work [n][BROW + 1], acc [4]
    const size_t extra = (size_t)n + (size_t)n * BROW + n + (size_t)n * (BROW + 1) + 4;
    Scratch S;
    rc = S.alloc(pb, extra, st);
    if (rc != SAS_OK) return rc;
    double* q_try = S.q + n;
    double* band = q_try + n;
    double* grad = band + (size_t)n * BROW;
    double* work = grad + n;
    double* acc = work + (size_t)n * (BROW + 1);
    double hacc[4];
    int iters = 0;
    double cost = 0.0;
    auto fail = [&](cudaError_t e, const char* what) {
        rc = cuda_fail(e, what);
        return rc;
    };
    auto loss_at = [&](const double* qq, double& out) -> int {
        cudaError_t e = cudaMemsetAsync(acc, 0, sizeof(double), st);
        if (e != cudaSuccess) return fail(e, "memset");
        dpc_assemble_kernel<false><<<pb.P - 1, 256, 0, st>>>(pb, qq, band, grad, acc);
        dpc_regular_kernel<false><<<blocks_for(pb.P, 128), 128, 0, st>>>(pb, qq, band, grad, acc);
        e = cudaGetLastError();
        if (e != cudaSuccess) return fail(e, "dpc loss");
        e = cudaMemcpyAsync(hacc, acc, sizeof(double), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return fail(e, "dpc loss readback");
        out = hacc[0];
        return SAS_OK;
    };
    rc = setup(pb, S, d_vy, d_vz, st);
    if (rc == SAS_OK) {
        const cudaError_t ea =
            cudaFuncSetAttribute(dpc_solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SOL_SMEM);
        if (ea != cudaSuccess) fail(ea, "dpc solve attribute");
    }
    if (rc == SAS_OK) rc = loss_at(S.q, cost);
    double mu = 1e-3;
    for (int it = 0; rc == SAS_OK && it < max_iter; ++it) {
        // normal equations at the current nodes
        cudaError_t e = cudaMemsetAsync(band, 0, sizeof(double) * ((size_t)n * BROW + n), st);
        if (e != cudaSuccess) {
            fail(e, "memset");
            break;
        }
        e = cudaMemsetAsync(acc, 0, sizeof(double), st);
        dpc_assemble_kernel<true><<<pb.P - 1, 256, 0, st>>>(pb, S.q, band, grad, acc);
        dpc_regular_kernel<true><<<blocks_for(pb.P, 128), 128, 0, st>>>(pb, S.q, band, grad, acc);
        e = cudaGetLastError();
        if (e != cudaSuccess) {
            fail(e, "dpc assemble");
            break;
        }
        bool accepted = false, stalled = false;
        double trial = cost;
        for (int tries = 0; tries < 40 && rc == SAS_OK; ++tries) {
            dpc_solve_kernel<<<1, 32, SOL_SMEM, st>>>(n, band, grad, mu, work, S.q, q_try, acc, g_sol_rlog);
            e = cudaGetLastError();
            if (e == cudaSuccess) e = cudaMemcpyAsync(hacc, acc, 4 * sizeof(double), cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) {
                fail(e, "dpc solve");
                break;
            }
            if (hacc[1] != 0.0) {   // not positive definite at this damping
                mu *= 10.0;
                continue;
            }
            const double step = hacc[2];
            if (loss_at(q_try, trial) != SAS_OK) break;
            if (trial <= cost) {
                std::swap(S.q, q_try);
                accepted = true;
                stalled = (cost - trial) <= 1e-14 * cost || step == 0.0;
                mu = std::max(mu / 3.0, 1e-15);
                break;
            }
            mu *= 4.0;
        }
        if (rc != SAS_OK || !accepted) break;
        ++iters;
        cost = trial;
        if (stalled) break;
    }
    if (rc == SAS_OK) {
        dpc_velocities_kernel<<<blocks_for(pb.P, 128), 128, 0, st>>>(pb, S.q, d_vy, d_vz);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = cuda_fail(e, "dpc velocities");
    }
    // S.q may point at the second node buffer after swaps: free the allocation base
    cudaFreeAsync(S.base, st);
    if (rc == SAS_OK) {
        if (h_loss) *h_loss = cost;
        if (h_iters) *h_iters = iters;
    }
    return rc;
}

extern "C" int sas_debug_dpc_solve_chunk(int32_t rows) {
    if (rows == 0) rows = SOL_R;
    int lg = 3;
    while ((1 << lg) < rows && lg < 9) ++lg;
    if (rows < 8 || rows > SOL_R || (1 << lg) != rows) {
        set_error("sas_debug_dpc_solve_chunk: rows must be 0 or a power of two in [8, 512]");
        return SAS_ERR_ARG;
    }
    g_sol_rlog = lg;
    return SAS_OK;
}
