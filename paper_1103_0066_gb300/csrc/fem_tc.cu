// fem_tc.cu -- the tensor-core contraction (fem_tc.cuh) for the affine forms it
// serves: P2 Laplacian and P1 elasticity on triangles and tetrahedra.
#include "fem_tc.cuh"

namespace fem {

// Reference tensors of the forms the tensor-core kernel serves, in constant memory.
__constant__ RefTensor<3, ELASTIC_P1> kTcK3e = make_ref_tensor<3, ELASTIC_P1>();
__constant__ RefTensor<3, LAPLACE_P2> kTcK3p = make_ref_tensor<3, LAPLACE_P2>();
__constant__ RefTensor<2, ELASTIC_P1> kTcK2e = make_ref_tensor<2, ELASTIC_P1>();
__constant__ RefTensor<2, LAPLACE_P2> kTcK2p = make_ref_tensor<2, LAPLACE_P2>();

struct TcKRefAffine {
  template <int D, int FORM>
  __device__ __forceinline__ static int k(int g, int i, int j) {
    if constexpr (D == 3 && FORM == ELASTIC_P1) return kTcK3e.v[g][i][j];
    if constexpr (D == 3 && FORM == LAPLACE_P2) return kTcK3p.v[g][i][j];
    if constexpr (D == 2 && FORM == ELASTIC_P1) return kTcK2e.v[g][i][j];
    if constexpr (D == 2 && FORM == LAPLACE_P2) return kTcK2p.v[g][i][j];
    return 0;
  }
};

cudaError_t launch_fwd_tc(const FwdLaunch& L) {
  if (L.coord_f64 || L.out_f64) return cudaErrorInvalidValue;
  if (L.dim == 3 && L.form == ELASTIC_P1) return launch_tc_t<3, ELASTIC_P1, TcGeoAffine, TcKRefAffine>(L, nullptr);
  if (L.dim == 3 && L.form == LAPLACE_P2) return launch_tc_t<3, LAPLACE_P2, TcGeoAffine, TcKRefAffine>(L, nullptr);
  if (L.dim == 2 && L.form == ELASTIC_P1) return launch_tc_t<2, ELASTIC_P1, TcGeoAffine, TcKRefAffine>(L, nullptr);
  if (L.dim == 2 && L.form == LAPLACE_P2) return launch_tc_t<2, LAPLACE_P2, TcGeoAffine, TcKRefAffine>(L, nullptr);
  return cudaErrorInvalidValue;
}

}  // namespace fem
