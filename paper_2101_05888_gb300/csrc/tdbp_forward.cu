// Forward backprojection (echo -> image), 2D and 3D: instantiation of the
// shared kernel template and the launch set-up common to all modes.
#include "tdbp_core.cuh"

#include <algorithm>
#include <cmath>

namespace sas {
namespace core {

int prepare(sas_geometry_t h, const sas_grid& g, int dim3, long long min_ctas, Setup& S, bool need_echo, int mode) {
    int TXs, TYs, TZs;
    tile_dims(dim3, TXs, TYs, TZs);
    const double dz = dim3 ? g.dz : 0.0;
    const int nz = dim3 ? g.nz : 1;
    // largest |x - x0| over a tile bounds the differential delay (|dr| <= |d| per leg)
    const double hx = 0.5 * (TXs - 1) * std::fabs(g.dx), hy = 0.5 * (TYs - 1) * std::fabs(g.dy),
                 hz = 0.5 * (TZs - 1) * std::fabs(dz);
    const double dmax = std::sqrt(hx * hx + hy * hy + hz * hz);
    // with seabed refraction a leg's length in water metres is Lipschitz with
    // constant max(1, n), n = c / c_s (a straight segment costs at most that much)
    const bool refract = h->c_sed > 0.0;
    const double n_refr = refract ? h->sig.c / h->c_sed : 1.0;
    const int U = (int)std::ceil(2.0 * std::max(1.0, n_refr) * dmax * h->sig.fs / h->sig.c) + 2;
    const int elem = (h->echo_dtype == SAS_ECHO_C32_F16 || h->echo_dtype == SAS_ECHO_C32_BF16) ? 4 : 8;
    const int align = 16 / elem;
    const int npos = 2 * U + 1;
    int seglen = 2 * U + 7 + align;
    seglen = (seglen + align - 1) / align * align;
    if (seglen > 256) {
        set_error("pixel spacing too coarse: a tile's delay span needs %d samples (max 256)", seglen);
        return SAS_ERR_UNSUPPORTED;
    }
    int npos_pad = (npos + RUN - 1) / RUN * RUN;
    // spans that fit take the fixed ring layout (see tdbp_kernel's FIXED)
    if (!refract && npos_pad <= NPOS_FIXED) npos_pad = NPOS_FIXED;
    // expansion runs of the padded positions read up to sample
    // (offset < align) + npos_pad + 6 of the slot: pad the slot past the copied segment
    const int slot_samples = std::max(seglen, npos_pad + align + 6);
    const int slot_bytes = (slot_samples * elem + 127) / 128 * 128;
    // quadratic rows for 16-bit echoes in the forward pass, else cubic rows
    const int row_bytes = (mode == MODE_FORWARD && elem == 4) ? ROW24 : ROW32;
    const size_t smem = smem_bytes(slot_bytes, npos_pad, refract ? (int)NREC_REFR : (int)NREC, row_bytes);
    if (smem > 227 * 1024) {
        set_error("shared memory need %zu exceeds the per-block limit", smem);
        return SAS_ERR_UNSUPPORTED;
    }
    KParams& prm = S.prm;
    prm = KParams{};
    prm.tx = h->d_tx;
    prm.rx = h->d_rx;
    prm.txs = h->d_txs;
    prm.rxs = h->d_rxs;
    prm.k_fs_c = df_split(h->sig.fs / h->sig.c);
    prm.k_t0fs = df_split(h->sig.t0 * h->sig.fs);
    prm.k_fc_c = df_split(h->sig.fc / h->sig.c);
    prm.scale = (elem == 8) ? nullptr : h->d_scale;
    prm.coef = h->d_coef;
    prm.status = h->d_status;
    prm.x0 = g.x0; prm.y0 = g.y0; prm.z0 = g.z0;
    prm.dx = g.dx; prm.dy = g.dy; prm.dz = dz;
    prm.nx = g.nx; prm.ny = g.ny; prm.nz = nz;
    prm.tiles_x = (g.nx + TXs - 1) / TXs;
    prm.tiles_y = (g.ny + TYs - 1) / TYs;
    prm.tiles_z = (nz + TZs - 1) / TZs;
    prm.P = h->P; prm.C = h->C;
    prm.t0 = h->sig.t0; prm.fs = h->sig.fs; prm.fc = h->sig.fc; prm.inv_c = 1.0 / h->sig.c;
    prm.hs_c = (float)(2.0 * h->sig.fs / h->sig.c);
    prm.wfc_c = (float)(2.0 * M_PI * h->sig.fc / h->sig.c);
    prm.hs_c2 = make_float2(prm.hs_c, prm.hs_c);
    prm.wfc_c2 = make_float2(prm.wfc_c, prm.wfc_c);
    // largest carrier phase a pixel can take from its reference: the reference in
    // [-pi, pi) plus 2 pi fc times the differential delay, which the window bound
    // U - 2 samples limits to (U - 2) / fs
    prm.phase_direct = M_PI + 2.0 * M_PI * h->sig.fc * (U - 2) / h->sig.fs <= PHASE_DIRECT_MAX;
    prm.fs2_f = (float)(2.0 * h->sig.fs);
    prm.wfc = (float)(2.0 * M_PI * h->sig.fc);
    prm.grad_scale = (float)(-2.0 / h->sig.c);
    prm.U = U; prm.npos = npos; prm.npos_pad = npos_pad; prm.seglen = seglen; prm.seg_align = align; prm.slot_bytes = slot_bytes;
    prm.rotc = h->d_rotc;
    prm.beam = h->beam_tan > 0.0;
    prm.beam_tan = (float)h->beam_tan;
    prm.beam_side = (float)h->beam_side;
    prm.cull = h->d_cull;
    prm.vel = h->has_vel ? h->d_vel : nullptr;
    prm.refract = refract;
    if (refract) {
        const double r = std::max(n_refr, 1.0 / n_refr), M = r * r - 1.0;
        prm.refr_fast_sed = n_refr < 1.0;
        prm.z_int = h->z_int;
        prm.refr_n = n_refr;
        prm.refr_nf = (float)n_refr;
        prm.refr_r2 = (float)(r * r);
        prm.refr_M = (float)M;
        prm.refr_isM = M > 0.0 ? (float)(1.0 / std::sqrt(M)) : INFINITY;
        // crossing-point tolerance: 1/2000 of a carrier wavelength
        prm.refr_tol = (float)(5e-4 * h->sig.c / h->sig.fc);
    }
    prm.hx = (float)hx;
    prm.hy = (float)hy;
    prm.hz = (float)hz;
    prm.skip_copies = h->debug_skip_copies;
    prm.wait_ns = (unsigned long long)(h->debug_wait_ms > 0 ? h->debug_wait_ms : 4000) * 1000000ull;
    const long long ntiles = (long long)prm.tiles_x * prm.tiles_y * prm.tiles_z;
    // small grids: split the pings of each tile over several CTAs (whole pings,
    // so that every (tile, ping) belongs to exactly one CTA)
    int nsplit = 1;
    if (min_ctas > 0 && ntiles < min_ctas) {
        nsplit = (int)std::min<long long>((min_ctas + ntiles - 1) / ntiles, h->P);
        const long long min_pairs = 2 * PAIRS;   // keep at least two stages per CTA
        nsplit = (int)std::max<long long>(1, std::min<long long>(nsplit, (long long)h->P * h->C / min_pairs));
    }
    prm.pings_per_split = (h->P + nsplit - 1) / nsplit;
    nsplit = (h->P + prm.pings_per_split - 1) / prm.pings_per_split;
    prm.nsplit = nsplit;
    if (ntiles * nsplit > 0x7fffffffLL) {
        set_error("grid too large");
        return SAS_ERR_UNSUPPORTED;
    }
    S.smem = smem;
    S.blocks = (int)(ntiles * nsplit);
    S.elem = elem;
    if (!need_echo) return SAS_OK;
    return encode_echo_map(&S.map, h->d_echo, elem, h->Ns, h->P * h->C, seglen);
}

template <typename ET, bool DIM3, int MODE>
static int launch_one(const Setup& S, cudaStream_t st) {
    const bool mv = S.prm.vel != nullptr;
    auto kern = S.prm.beam ? (mv ? tdbp_kernel<ET, DIM3, MODE, true, true> : tdbp_kernel<ET, DIM3, MODE, true, false>)
                           : (mv ? tdbp_kernel<ET, DIM3, MODE, false, true> : tdbp_kernel<ET, DIM3, MODE, false, false>);
    if constexpr (MODE == MODE_FORWARD) {
        if (S.prm.refract) {
            if (S.prm.beam || mv) {
                set_error("the refraction model does not combine with receiver motion or a beam");
                return SAS_ERR_UNSUPPORTED;
            }
            kern = tdbp_kernel<ET, DIM3, MODE, false, false, true>;
        }
    } else if (S.prm.refract) {
        set_error("the offset gradient is not available with the refraction model");
        return SAS_ERR_UNSUPPORTED;
    }
    if (!S.prm.refract && !S.prm.beam && !mv && S.prm.npos_pad == NPOS_FIXED)
        kern = tdbp_kernel<ET, DIM3, MODE, false, false, false, true>;
    SAS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S.smem));
    kern<<<S.blocks, NTHREADS, S.smem, st>>>(S.map, S.prm);
    SAS_CUDA(cudaGetLastError());
    return SAS_OK;
}

template <int MODE>
int launch_mode(const Setup& S, int echo_dtype, int dim3, cudaStream_t st) {
    switch (echo_dtype) {
        case SAS_ECHO_C64:
            return dim3 ? launch_one<float2, true, MODE>(S, st) : launch_one<float2, false, MODE>(S, st);
        case SAS_ECHO_C32_F16:
            return dim3 ? launch_one<__half2, true, MODE>(S, st) : launch_one<__half2, false, MODE>(S, st);
        case SAS_ECHO_C32_BF16:
            return dim3 ? launch_one<__nv_bfloat162, true, MODE>(S, st)
                        : launch_one<__nv_bfloat162, false, MODE>(S, st);
        default:
            set_error("no echo uploaded");
            return SAS_ERR_STATE;
    }
}

template int launch_mode<MODE_FORWARD>(const Setup&, int, int, cudaStream_t);

}  // namespace core

int launch_forward(const ForwardArgs& a) {
    core::Setup S;
    int rc = core::prepare(a.h, a.grid, a.dim3, 2LL * sm_count(), S);
    if (rc != SAS_OK) return rc;
    S.prm.image = a.image;
    S.prm.accumulate = a.accumulate;
    S.prm.atomic_out = S.prm.nsplit > 1;
    if (S.prm.atomic_out && !a.accumulate)
        SAS_CUDA(cudaMemsetAsync(a.image, 0, sizeof(float2) * (size_t)a.grid.nx * a.grid.ny * S.prm.nz, a.stream));
    return core::launch_mode<core::MODE_FORWARD>(S, a.h->echo_dtype, a.dim3, a.stream);
}

}  // namespace sas
