// fem_bwd.cu -- launchers of the adjoint element kernel (device code in fem_bwd.cuh).
#include "fem_bwd.cuh"

namespace fem {

template <int D, int FORM, int JAC, bool ATOMIC>
static cudaError_t launch_bwd_t(const BwdLaunch& L) {
  using PL = BwdPlan<D, FORM>;
  BwdParams p;
  p.conn = L.conn;
  p.coords = L.coords;
  p.coef = L.coef;
  p.dA = L.dA;
  p.tile_rec = ATOMIC ? nullptr : L.tile_rec;
  p.rank = L.rank;
  p.rec_span = L.rec_span;
  p.rec_dest = L.rec_dest;
  p.records = L.records;
  p.dcoef = L.dcoef;
  p.dcoords = L.dcoords;
  p.n_elem = L.n_elem;
  p.n_vert = L.n_vert;
  p.dev_err = L.dev_err;
  p.vec_conn = (D == 3) && (reinterpret_cast<uintptr_t>(L.conn) % 16 == 0);
  p.vec_dA = reinterpret_cast<uintptr_t>(L.dA) % 16 == 0;
  p.det = L.det_in;
  auto kern = fem_bwd_elem_kernel<D, FORM, JAC, ATOMIC>;
  constexpr int max_warps = BwdShape<D, FORM, JAC>::threads / 32;  // the kernel's launch bounds
  const int want = L.warps > 0 ? L.warps : max_warps;
  const int warps = clamp_warps(want < max_warps ? want : max_warps, PL::per_warp);
  const size_t smem = size_t(warps) * PL::per_warp;
  cudaError_t st = ensure_smem(reinterpret_cast<const void*>(kern), smem);
  if (st != cudaSuccess) return st;
  const unsigned grid = pipeline_grid(reinterpret_cast<const void*>(kern), warps, smem, L.n_elem, L.ctas_per_sm);
  kern<<<grid, warps * 32, smem, L.stream>>>(p);
  return cudaGetLastError();
}

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
