// Forward kernels for tetrahedra, P1 symmetric-gradient elasticity.
#include "fem_fwd.cuh"

namespace fem {
cudaError_t launch_fwd_d3_ela(const FwdLaunch& L) {
  if (L.form != ELASTIC_P1) return cudaErrorInvalidValue;
  return launch_fwd_form<3, ELASTIC_P1>(L);
}
}  // namespace fem
