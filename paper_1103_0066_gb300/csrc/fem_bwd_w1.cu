// fem_bwd_w1.cu -- the adjoint element kernel for the P1-coefficient Laplacian
// (Eqs. 20-23): coordinate gradient and the gradient of the coefficient's
// vertex values, with the compensated Jacobian or det J saved by the forward.
#include "fem_bwd.cuh"

namespace fem {

template <int D, int FORM>
static cudaError_t launch_w1_form(const BwdLaunch& L) {
  if (L.det_in)
    return L.atomic ? launch_bwd_t<D, FORM, JAC_SAVED, true>(L) : launch_bwd_t<D, FORM, JAC_SAVED, false>(L);
  if (L.jac != JAC_COMP) return cudaErrorInvalidValue;
  return L.atomic ? launch_bwd_t<D, FORM, JAC_COMP, true>(L) : launch_bwd_t<D, FORM, JAC_COMP, false>(L);
}

cudaError_t launch_bwd_elem_w1(const BwdLaunch& L) {
  if (L.dim == 2) return L.form == LAPLACE_P1_W1 ? launch_w1_form<2, LAPLACE_P1_W1>(L) : launch_w1_form<2, LAPLACE_P2_W1>(L);
  return L.form == LAPLACE_P1_W1 ? launch_w1_form<3, LAPLACE_P1_W1>(L) : launch_w1_form<3, LAPLACE_P2_W1>(L);
}

}  // namespace fem
