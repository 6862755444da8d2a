// fem_fwd_w1.cu -- forward instantiations of the Laplacian with a P1
// coefficient given by its vertex values (Eqs. 20-23): P1 and P2 bases on
// triangles and tetrahedra.
#include "fem_fwd.cuh"

namespace fem {

cudaError_t launch_fwd_w1(const FwdLaunch& L) {
  if (L.dim == 2) {
    if (L.form == LAPLACE_P1_W1) return launch_fwd_form<2, LAPLACE_P1_W1>(L);
    if (L.form == LAPLACE_P2_W1) return launch_fwd_form<2, LAPLACE_P2_W1>(L);
  } else {
    if (L.form == LAPLACE_P1_W1) return launch_fwd_form<3, LAPLACE_P1_W1>(L);
    if (L.form == LAPLACE_P2_W1) return launch_fwd_form<3, LAPLACE_P2_W1>(L);
  }
  return cudaErrorInvalidValue;
}

}  // namespace fem
