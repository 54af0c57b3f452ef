// Gradient of a real loss with respect to per-ping position offsets, given
// the image gradient G = dL/dI* (the autofocus VJP), and its deterministic
// reduction over image tiles.
#include "tdbp_core.cuh"

namespace sas {
namespace core {

template <typename ET, bool DIM3, int MODE>
static int launch_one_grad(const Setup& S, cudaStream_t st) {
    const bool mv = S.prm.vel != nullptr;
    auto kern = S.prm.beam ? (mv ? tdbp_kernel<ET, DIM3, MODE, true, true> : tdbp_kernel<ET, DIM3, MODE, true, false>)
                           : (mv ? tdbp_kernel<ET, DIM3, MODE, false, true> : tdbp_kernel<ET, DIM3, MODE, false, false>);
    if (S.prm.refract) {
        if (S.prm.beam || mv) {
            set_error("the refraction model does not combine with receiver motion or a beam");
            return SAS_ERR_UNSUPPORTED;
        }
        kern = tdbp_kernel<ET, DIM3, MODE, false, false, true>;
    } else if (!S.prm.beam && !mv && S.prm.npos_pad == NPOS_FIXED) {
        kern = tdbp_kernel<ET, DIM3, MODE, false, false, false, true>;
    }
    SAS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S.smem));
    kern<<<S.blocks, NTHREADS, S.smem, st>>>(S.map, S.prm);
    SAS_CUDA(cudaGetLastError());
    return SAS_OK;
}

template <>
int launch_mode<MODE_OFFSET_GRAD>(const Setup& S, int echo_dtype, int dim3, cudaStream_t st) {
    switch (echo_dtype) {
        case SAS_ECHO_C64:
            return dim3 ? launch_one_grad<float2, true, MODE_OFFSET_GRAD>(S, st)
                        : launch_one_grad<float2, false, MODE_OFFSET_GRAD>(S, st);
        case SAS_ECHO_C32_F16:
            return dim3 ? launch_one_grad<__half2, true, MODE_OFFSET_GRAD>(S, st)
                        : launch_one_grad<__half2, false, MODE_OFFSET_GRAD>(S, st);
        case SAS_ECHO_C32_BF16:
            return dim3 ? launch_one_grad<__nv_bfloat162, true, MODE_OFFSET_GRAD>(S, st)
                        : launch_one_grad<__nv_bfloat162, false, MODE_OFFSET_GRAD>(S, st);
        default:
            set_error("no echo uploaded");
            return SAS_ERR_STATE;
    }
}

// out[t] = sum over tiles (in tile order, FP64) of partials[tile][t], t = 3 ping + axis
__global__ void reduce_tiles_kernel(const double* __restrict__ partials, int ntiles, int n, double* __restrict__ out) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    double s = 0.0;
    for (int k = 0; k < ntiles; ++k) s += partials[(size_t)k * n + t];
    out[t] = s;
}

}  // namespace core

int launch_offset_grad(sas_geometry_t h, const sas_grid& g, const float2* grad_image, double* grad_offsets,
                       cudaStream_t st) {
    const int dim3 = g.nz > 1;
    core::Setup S;
    int rc = core::prepare(h, g, dim3, 2LL * sm_count(), S, true, core::MODE_OFFSET_GRAD);
    if (rc != SAS_OK) return rc;
    const long long ntiles = (long long)S.prm.tiles_x * S.prm.tiles_y * S.prm.tiles_z;
    const size_t need = (size_t)ntiles * h->P * 3 * sizeof(double);
    if (h->scratch_bytes < need) {
        if (h->d_scratch) {
            SAS_CUDA(cudaStreamSynchronize(st));
            cudaFree(h->d_scratch);
            h->d_scratch = nullptr;
            h->scratch_bytes = 0;
        }
        SAS_CUDA(cudaMalloc(&h->d_scratch, need));
        h->scratch_bytes = need;
    }
    // (tile, ping) partials with no pair inside the beams are never written
    SAS_CUDA(cudaMemsetAsync(h->d_scratch, 0, need, st));
    S.prm.gimage = grad_image;
    S.prm.partials = (double*)h->d_scratch;
    rc = core::launch_mode<core::MODE_OFFSET_GRAD>(S, h->echo_dtype, dim3, st);
    if (rc != SAS_OK) return rc;
    const int n = h->P * 3;
    core::reduce_tiles_kernel<<<(n + 255) / 256, 256, 0, st>>>((const double*)h->d_scratch, (int)ntiles, n,
                                                                 grad_offsets);
    SAS_CUDA(cudaGetLastError());
    return SAS_OK;
}

}  // namespace sas
