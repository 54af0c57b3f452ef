// Learned interpolator kernels (placeholder until the MLP kernels land).
#include "sas_common.cuh"

using namespace sas;

extern "C" int sas_mlp_make_windows(const void*, int32_t, int32_t, const float*, const int32_t*, const int32_t*,
                                    int64_t, double, void*, void*, void*) {
    set_error("not built yet");
    return SAS_ERR_UNSUPPORTED;
}
extern "C" int64_t sas_mlp_workspace_bytes(int64_t) { return 0; }
extern "C" int sas_mlp_loss_grad(const float*, const float*, const void*, const void*, int64_t, float*, float*, void*,
                                 void*) {
    set_error("not built yet");
    return SAS_ERR_UNSUPPORTED;
}
extern "C" int sas_mlp_adam(float*, const float*, float*, float*, int32_t, float, float, float, float, void*) {
    set_error("not built yet");
    return SAS_ERR_UNSUPPORTED;
}
extern "C" int sas_interp_tabulate_mlp(const float*, int32_t, float*, void*) {
    set_error("not built yet");
    return SAS_ERR_UNSUPPORTED;
}
