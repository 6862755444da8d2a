// fem_bwd.cu -- launchers of the adjoint element kernel (device code and the
// launch template in fem_bwd.cuh; the P1-coefficient forms in fem_bwd_w1.cu).
#include "fem_bwd.cuh"

namespace fem {

template <int D, int FORM>
static cudaError_t launch_bwd_form(const BwdLaunch& L) {
  if (L.det_in)  // det J saved by the forward
    return L.atomic ? launch_bwd_t<D, FORM, JAC_SAVED, true>(L) : launch_bwd_t<D, FORM, JAC_SAVED, false>(L);
  switch (L.jac) {
    case JAC_COMP:
      return L.atomic ? launch_bwd_t<D, FORM, JAC_COMP, true>(L) : launch_bwd_t<D, FORM, JAC_COMP, false>(L);
    case JAC_F64:
      return L.atomic ? launch_bwd_t<D, FORM, JAC_F64, true>(L) : launch_bwd_t<D, FORM, JAC_F64, false>(L);
    case JAC_F32:
      return L.atomic ? launch_bwd_t<D, FORM, JAC_F32, true>(L) : launch_bwd_t<D, FORM, JAC_F32, false>(L);
    default:
      return cudaErrorInvalidValue;
  }
}

cudaError_t launch_bwd_elem(const BwdLaunch& L) {
  if (L.form == LAPLACE_P1_W1 || L.form == LAPLACE_P2_W1) return launch_bwd_elem_w1(L);
  if (L.dim == 2) {
    switch (L.form) {
      case LAPLACE_P1: return launch_bwd_form<2, LAPLACE_P1>(L);
      case LAPLACE_P2: return launch_bwd_form<2, LAPLACE_P2>(L);
      case ELASTIC_P1: return launch_bwd_form<2, ELASTIC_P1>(L);
    }
  } else {
    switch (L.form) {
      case LAPLACE_P1: return launch_bwd_form<3, LAPLACE_P1>(L);
      case LAPLACE_P2: return launch_bwd_form<3, LAPLACE_P2>(L);
      case ELASTIC_P1: return launch_bwd_form<3, ELASTIC_P1>(L);
    }
  }
  return cudaErrorInvalidValue;
}

}  // namespace fem
