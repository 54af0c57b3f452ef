// Adjoints of the backprojection on a pixel grid:
//  * the linear adjoint B^H (image -> echo), the exact transpose of the
//    forward sum:  e_adj[i][c][floor u + k] += w_k(frac u) exp(-j 2 pi fc tau) I(x);
//  * dispatch of the offset gradient (tdbp_vjp.cu).
//
// Linear adjoint, one CTA per tile (warp 0 computes the FP64 reference terms
// of 32 pairs at a time, warps 1..7 own 8 pixels each).  With the Farrow form
// w_k(f) = sum_p coef[h][k][p] g^p on the half h of the sample interval the
// per-pixel work is a scatter of g^p v (v = I(x) exp(-j 2 pi fc tau)) into
// accumulators A_p[n] in shared memory, n = floor(2u) the half-sample
// index; a transposed FIR e[floor u + k] += sum_h sum_p coef[h][k][p]
// A_p[2 floor u + h] then adds each pair's segment to the echo with global
// atomics.
#include "tdbp_core.cuh"

namespace sas {

int launch_offset_grad(sas_geometry_t h, const sas_grid& g, const float2* grad_image, double* grad_offsets,
                       cudaStream_t st);

namespace core {

// Four consecutive fields f0 .. f0 + 3 of pair pr of a field-major record.
__device__ __forceinline__ float4 rec_block(const float* rec, int f0, int pr) {
    return make_float4(rec[f0 * PAIRS + pr], rec[(f0 + 1) * PAIRS + pr], rec[(f0 + 2) * PAIRS + pr],
                       rec[(f0 + 3) * PAIRS + pr]);
}

// REFRACT: the seabed refraction model (the forward kernel's per-leg
// crossing records and per-pixel solves, evaluated the same way).
template <bool DIM3, bool REFRACT>
__global__ void __launch_bounds__(NTHREADS, 2) adjoint_kernel(const KParams p, const float2* __restrict__ img,
                                                              float2* __restrict__ eadj, int Ns) {
    using T = Tile<DIM3>;
    constexpr int KREC = REFRACT ? NREC_REFR : NREC;
    extern __shared__ __align__(1024) unsigned char smem[];
    const int nrow = NH * p.npos;                                   // half-sample rows per pair
    float2* A = reinterpret_cast<float2*>(smem);                    // [GROUP][nrow][NP]
    float* rec = reinterpret_cast<float*>(A + GROUP * nrow * NP);   // [KREC][PAIRS], field-major
    float* coef_s = rec + KREC * PAIRS;                             // [NH][TAPS][NP]
    int* base_s = reinterpret_cast<int*>(coef_s + NH * TAPS * NP);  // [PAIRS]
    int* rfl_s = base_s + PAIRS;                                    // [PAIRS] refraction flags

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ntiles = p.tiles_x * p.tiles_y * p.tiles_z;
    const int tile = blockIdx.x % ntiles;
    const int split = blockIdx.x / ntiles;
    const int tx0 = (tile % p.tiles_x) * T::TX;
    const int ty0 = ((tile / p.tiles_x) % p.tiles_y) * T::TY;
    const int tz0 = (tile / (p.tiles_x * p.tiles_y)) * T::TZ;
    const int ping0 = min(p.P, split * p.pings_per_split);
    const int ping1 = min(p.P, ping0 + p.pings_per_split);
    const long long q0 = (long long)ping0 * p.C, q1 = (long long)ping1 * p.C;
    const int nq = (int)(q1 - q0);
    const double cx = tx0 + 0.5 * (T::TX - 1), cy = ty0 + 0.5 * (T::TY - 1), cz = tz0 + 0.5 * (T::TZ - 1);
    const double X0 = p.x0 + cx * p.dx, Y0 = p.y0 + cy * p.dy, Z0 = p.z0 + (DIM3 ? cz * p.dz : 0.0);
    // seabed refraction: the layers below the interface and the reference depth
    double Zr = Z0;
    const unsigned bmask = REFRACT ? refr_tile_layers<DIM3>(p, tz0, Z0, Zr) : 0u;
    const float r_br = REFRACT ? (float)(Zr - p.z_int) : 0.f, r_zoff = REFRACT ? (float)(Zr - Z0) : 0.f;
    const int alen = GROUP * nrow * NP;
    const int span = p.npos + TAPS - 1;            // output samples per pair segment

    for (int t = tid; t < alen; t += NTHREADS) A[t] = make_float2(0.f, 0.f);
    if (tid < NH * TAPS * NP) coef_s[tid] = (&p.coef->c[0][0][0])[tid];

    const bool consumer = warp > 0;
    const int ct = tid - 32;
    float dxv = 0.f, dyv_c = 0.f, d2c = 0.f, r_d2h = 0.f;
    float dvar[PX], dT[PX];
    float2 G[PX];
    if (consumer) {
        int lx, ly, lz;
        T::pixel(ct, 0, lx, ly, lz);
        dxv = (float)((tx0 + lx - cx) * p.dx);
        dyv_c = (float)((ty0 + ly - cy) * p.dy);
        // the varying coordinate as the forward kernel forms it (first slot plus
        // s steps, in FP32), so that both take identical beam decisions
        const float dv0 = DIM3 ? (float)((tz0 + lz - cz) * p.dz) : dyv_c;
        const float dvstep = DIM3 ? (float)p.dz : (float)(4.0 * p.dy);
        d2c = fixed_d2<DIM3>(dxv, dyv_c);
        r_d2h = REFRACT ? fixed_d2<true>(dxv, dyv_c) : 0.f;
#pragma unroll
        for (int s = 0; s < PX; ++s) {
            T::pixel(ct, s, lx, ly, lz);
            dvar[s] = fmaf((float)s, dvstep, dv0);
            dT[s] = 0.f;
            const int ix = tx0 + lx, iy = ty0 + ly, iz = tz0 + lz;
            G[s] = (ix < p.nx && iy < p.ny && iz < p.nz) ? img[((size_t)iz * p.ny + iy) * p.nx + ix]
                                                        : make_float2(0.f, 0.f);
        }
    }
    int prev_ping = -1;
    const int nstages = (nq + PAIRS - 1) / PAIRS;
    for (int k = 0; k < nstages; ++k) {
        const long long qs = q0 + (long long)k * PAIRS;
        __syncthreads();   // previous stage's records no longer in use
        if (warp == 0 && qs + lane < q1) {
            const int i = (int)((unsigned)(qs + lane) / (unsigned)p.C);
            // the forward pass's reference terms: double-float for stop-and-hop, FP64 with
            // motion or refraction
            if (REFRACT) {
                const PairGeo G = pair_geo(p, X0, Y0, Z0, qs + lane, i);
                double LT0, LR0;
                rfl_s[lane] = refr_pair_blocks(p, G, p.tx[3 * (size_t)i + 2], p.rx[3 * (size_t)(qs + lane) + 2], bmask,
                                               Zr, Z0, rec + lane, PAIRS, LT0, LR0);
                base_s[lane] = pair_record(p, G, rec + lane, PAIRS, nullptr, LT0, LR0);
            } else if (p.vel) {
                base_s[lane] = pair_record(p, pair_geo(p, X0, Y0, Z0, qs + lane, i), rec + lane, PAIRS,
                                           p.vel + 3 * (size_t)i);
            } else {
                const float2 a = df_split(X0), b = df_split(Y0), c = df_split(Z0);
                const dfl X0d[3] = {dfl{a.x, a.y}, dfl{b.x, b.y}, dfl{c.x, c.y}};
                base_s[lane] = pair_record_df(p, pair_geo_df(p, X0d, (int)(qs + lane), i), rec + lane, PAIRS);
            }
        }
        __syncthreads();
        float r[F_NT + 1];
#pragma unroll
        for (int f = 0; f <= F_NT; ++f) r[f] = rec[f * PAIRS + lane];
        const int npairs = (int)min((long long)PAIRS, q1 - qs);
        for (int g0 = 0; g0 < npairs; g0 += GROUP) {
            if (consumer) {
                for (int j = 0; j < GROUP && g0 + j < npairs; ++j) {
                    const int pr = g0 + j;
                    const int ping = (int)((qs + pr) / p.C);
                    if (ping != prev_ping) {
                        prev_ping = ping;
                        const float tT0 = __shfl_sync(0xffffffffu, r[F_TX], pr);
                        const float tT1 = __shfl_sync(0xffffffffu, r[F_TY], pr);
                        const float tT2 = __shfl_sync(0xffffffffu, r[F_TZ], pr);
                        const float nT2 = __shfl_sync(0xffffffffu, r[F_NT2], pr);
                        const float nT = __shfl_sync(0xffffffffu, r[F_NT], pr);
                        const float Ax = fixed_dot<DIM3>(tT0, tT1, dxv, dyv_c);
                        // seabed refraction of the transmitter leg
                        const bool trefr = REFRACT && (rfl_s[pr] & FL_T_REFR);
                        float4 tr0 = make_float4(0.f, 0.f, 0.f, 0.f), tr1 = tr0, tr2 = tr0;
                        float rhoT = 0.f, drhoT = 0.f;
                        if (REFRACT && trefr) {
                            tr0 = rec_block(rec, F_TREF, pr);
                            tr1 = rec_block(rec, F_TREF + 4, pr);
                            tr2 = rec_block(rec, F_TREF + 8, pr);
                            if (DIM3) refr_rho(tr0, Ax + r_d2h, rhoT, drhoT);
                        }
#pragma unroll
                        for (int s = 0; s < PX; ++s) {
                            const float d2 = fmaf(dvar[s], dvar[s], d2c);
                            const float a = __fadd_rn(fmaf(DIM3 ? tT2 : tT1, dvar[s], d2), Ax);
                            const float sm = nT2 + a;
                            dT[s] = a * rcp_sfu(fmaf(sm, rsqrt_sfu(sm), nT));
                            if (REFRACT && trefr) {
                                if ((bmask >> s) & 1u) {
                                    if (!DIM3) refr_rho(tr0, a, rhoT, drhoT);
                                    const float db = DIM3 ? dvar[s] - r_zoff : 0.f, b = fmaxf(r_br + db, 1e-7f);
                                    float uxi, ua;
                                    dT[s] = refr_leg_diff(p, tr0, tr1, tr2, rhoT, drhoT, b, db, r_br, uxi, ua);
                                } else {
                                    dT[s] += tr2.w;
                                }
                            }
                        }
                    }
                    const float tRx = __shfl_sync(0xffffffffu, r[F_RX], pr);
                    const float tRy = __shfl_sync(0xffffffffu, r[F_RY], pr);
                    const float tRz = __shfl_sync(0xffffffffu, r[F_RZ], pr);
                    const float nR2 = __shfl_sync(0xffffffffu, r[F_NR2], pr);
                    const float nR = __shfl_sync(0xffffffffu, r[F_NR], pr);
                    const float ufc = __shfl_sync(0xffffffffu, r[F_UF], pr);
                    const float phr = __shfl_sync(0xffffffffu, r[F_PH], pr);
                    const float Ax = fixed_dot<DIM3>(tRx, tRy, dxv, dyv_c);
                    // receiver motion: (R_R + d).v / c = Km + d_var v_var / c, as the forward
                    // kernel forms it; the beam test keeps the ping-time receiver vector
                    float Km = 0.f, vv = 0.f, bRx = tRx, bRy = tRy, bRz = tRz;
                    if (p.vel) {
                        const float* rp = rec + pr;
                        Km = DIM3 ? fmaf(rp[F_VX * PAIRS], dxv, fmaf(rp[F_VY * PAIRS], dyv_c, rp[F_RV * PAIRS]))
                                  : fmaf(rp[F_VX * PAIRS], dxv, rp[F_RV * PAIRS]);
                        vv = DIM3 ? rp[F_VZ * PAIRS] : rp[F_VY * PAIRS];
                        bRx = rp[F_BRX * PAIRS];
                        bRy = rp[F_BRY * PAIRS];
                        bRz = rp[F_BRZ * PAIRS];
                    }
                    float2* Aj = A + j * nrow * NP;
                    // seabed refraction of the receiver leg
                    const bool rrefr = REFRACT && (rfl_s[pr] & FL_R_REFR);
                    float4 rr0 = make_float4(0.f, 0.f, 0.f, 0.f), rr1 = rr0, rr2 = rr0;
                    float rhoR = 0.f, drhoR = 0.f;
                    if (REFRACT && rrefr) {
                        rr0 = rec_block(rec, F_RREF, pr);
                        rr1 = rec_block(rec, F_RREF + 4, pr);
                        rr2 = rec_block(rec, F_RREF + 8, pr);
                        if (DIM3) refr_rho(rr0, Ax + r_d2h, rhoR, drhoR);
                    }
                    float rot[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                    float tT0 = 0.f, tT1 = 0.f, tT2 = 0.f;
                    if (p.beam) {
#pragma unroll
                        for (int t = 0; t < 6; ++t) rot[t] = p.rotc[6 * (size_t)ping + t];
                        tT0 = __shfl_sync(0xffffffffu, r[F_TX], pr);
                        tT1 = __shfl_sync(0xffffffffu, r[F_TY], pr);
                        tT2 = __shfl_sync(0xffffffffu, r[F_TZ], pr);
                    }
#pragma unroll
                    for (int s = 0; s < PX; ++s) {
                        if (p.beam) {
                            // both beams must see the pixel (sensor-to-pixel vectors R + d)
                            const float dy = DIM3 ? dyv_c : dvar[s], dz = DIM3 ? dvar[s] : 0.f;
                            if (!beam_sees(p, fmaf(0.5f, tT0, dxv), fmaf(0.5f, tT1, dy), fmaf(0.5f, tT2, dz), rot) ||
                                !beam_sees(p, fmaf(0.5f, bRx, dxv), fmaf(0.5f, bRy, dy), fmaf(0.5f, bRz, dz), rot))
                                continue;
                        }
                        const float d2 = fmaf(dvar[s], dvar[s], d2c);
                        const float a = __fadd_rn(fmaf(DIM3 ? tRz : tRy, dvar[s], d2), Ax);
                        const float sm = nR2 + a;
                        const float rs = rsqrt_sfu(sm);
                        float D = fmaf(a, rcp_sfu(fmaf(sm, rs, nR)), dT[s]);
                        if (REFRACT && rrefr) {
                            if ((bmask >> s) & 1u) {
                                float rho = rhoR, drho = drhoR;
                                if (!DIM3) refr_rho(rr0, a, rho, drho);
                                const float db = DIM3 ? dvar[s] - r_zoff : 0.f, b = fmaxf(r_br + db, 1e-7f);
                                float uxi, ua;
                                D = refr_leg_diff(p, rr0, rr1, rr2, rho, drho, b, db, r_br, uxi, ua) + dT[s];
                            } else {
                                D += rr2.w;
                            }
                        }
                        if (p.vel) {
                            const float eps = fmaf(dvar[s], vv, Km) * rs;         // u_R . v / c
                            D = D * fmaf(eps, eps - 1.f, 1.f);                   // / (1 + eps)
                        }
                        const float v = fmaf(D, p.hs_c, ufc);              // 2 (u - floor u_ref) - 1/2
                        float ph = fmaf(D, p.wfc_c, phr);                  // carrier phase [rad]
                        // nearest integer of v = the half-sample index; g = frac(2u) - 1/2
                        const float t = __fadd_rn(v, FLOOR_MAGIC);
                        const float g = v - (t - FLOOR_MAGIC);
                        const unsigned pos = row_index(
                            (unsigned)(__float_as_int(t) - (__float_as_int(FLOOR_MAGIC) - NH * p.U)), (unsigned)(nrow - 1),
                            p.status);
                        if (!p.phase_direct) ph = reduce_phase(ph);
                        float sn, cs;
                        sincos_sfu(ph, sn, cs);
                        // v = G exp(-j phase)
                        float vx = fmaf(G[s].x, cs, G[s].y * sn);
                        float vy = fmaf(G[s].y, cs, -G[s].x * sn);
                        float* dst = reinterpret_cast<float*>(Aj + pos * NP);
#pragma unroll
                        for (int q = 0; q < NP; ++q) {
                            atomicAdd(dst + 2 * q, vx);
                            atomicAdd(dst + 2 * q + 1, vy);
                            vx *= g;
                            vy *= g;
                        }
                    }
                }
            }
            __syncthreads();
            // transposed FIR and flush: out[t] = sum_m sum_h sum_p coef[h][m][p] A_p[2 (t - m) + h]
            const int items = GROUP * span;
            for (int it = tid; it < items; it += NTHREADS) {
                const int j = it / span, t = it - j * span;
                const int pr = g0 + j;
                if (pr >= npairs) continue;
                const float2* Aj = A + j * nrow * NP;
                float ox = 0.f, oy = 0.f;
#pragma unroll
                for (int m = 0; m < TAPS; ++m) {
                    const int pos = t - m;
                    if (pos < 0 || pos >= p.npos) continue;
#pragma unroll
                    for (int h = 0; h < NH; ++h) {
#pragma unroll
                        for (int q = 0; q < NP; ++q) {
                            const float c = coef_s[(h * TAPS + m) * NP + q];
                            const float2 v = Aj[(NH * pos + h) * NP + q];
                            ox = fmaf(c, v.x, ox);
                            oy = fmaf(c, v.y, oy);
                        }
                    }
                }
                const long long idx = (long long)base_s[pr] + t;
                if (idx >= 0 && idx < Ns && (ox != 0.f || oy != 0.f))
                    atomicAdd(eadj + (size_t)(qs + pr) * Ns + idx, make_float2(ox, oy));
            }
            __syncthreads();
            for (int t = tid; t < alen; t += NTHREADS) A[t] = make_float2(0.f, 0.f);
        }
    }
}

}  // namespace core

static int launch_linear_adjoint(sas_geometry_t h, const sas_grid& g, const float2* img, float2* eadj,
                                 cudaStream_t st) {
    const int dim3 = g.nz > 1;
    core::Setup S;
    int rc = core::prepare(h, g, dim3, 2LL * sm_count(), S, false);
    if (rc != SAS_OK) return rc;
    if (S.prm.refract && (S.prm.beam || S.prm.vel)) {
        set_error("the refraction model does not combine with receiver motion or a beam");
        return SAS_ERR_UNSUPPORTED;
    }
    SAS_CUDA(cudaMemsetAsync(eadj, 0, sizeof(float2) * (size_t)h->P * h->C * h->Ns, st));
    const int krec = S.prm.refract ? (int)core::NREC_REFR : (int)core::NREC;
    const size_t smem = sizeof(float2) * core::GROUP * NH * S.prm.npos * NP + sizeof(float) * krec * core::PAIRS +
                        sizeof(float) * NH * TAPS * NP + 2 * sizeof(int) * core::PAIRS;
    auto k = dim3 ? (S.prm.refract ? core::adjoint_kernel<true, true> : core::adjoint_kernel<true, false>)
                  : (S.prm.refract ? core::adjoint_kernel<false, true> : core::adjoint_kernel<false, false>);
    SAS_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k<<<S.blocks, core::NTHREADS, smem, st>>>(S.prm, img, eadj, h->Ns);
    SAS_CUDA(cudaGetLastError());
    return SAS_OK;
}

int launch_adjoint(const AdjointArgs& a) {
    if (a.grad_offsets) {
        int rc = launch_offset_grad(a.h, a.grid, a.grad_image, a.grad_offsets, a.stream);
        if (rc != SAS_OK) return rc;
    }
    if (a.echo_adj) return launch_linear_adjoint(a.h, a.grid, a.grad_image, a.echo_adj, a.stream);
    return SAS_OK;
}

}  // namespace sas
