// Adjoints of the backprojection (placeholder until the adjoint kernels land).
#include "sas_common.cuh"

namespace sas {
int launch_adjoint(const AdjointArgs&) {
    set_error("sas_backproject_adjoint: not built yet");
    return SAS_ERR_UNSUPPORTED;
}
}  // namespace sas
