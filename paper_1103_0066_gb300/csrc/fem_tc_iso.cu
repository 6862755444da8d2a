// fem_tc_iso.cu -- the tensor-core contraction (fem_tc.cuh) for the P2
// Laplacian on non-affine elements (Eqs. 16-19).  G^{(k mu),(l nu)} of the
// curved element (78 folded slots on tets, 21 on triangles) is split into
// three BF16 terms; K^{ij}_{(k mu),(l nu)} * DEN is exact in BF16 (at most
// 768 = 3 * 2^8 in magnitude).  The contraction is 59% dense on tets (2538
// of 78 x 55 products), the shape the tensor cores serve.
#include "fem_iso.cuh"
#include "fem_tc.cuh"

namespace fem {

static_assert(tc_b_exact<3, LAPLACE_P2_ISO>() && tc_b_exact<2, LAPLACE_P2_ISO>(), "K' * DEN must be exact in BF16");
__device__ const TcBImage<3, LAPLACE_P2_ISO> kTcB3iso = make_tc_b_image<3, LAPLACE_P2_ISO>();
__device__ const TcBImage<2, LAPLACE_P2_ISO> kTcB2iso = make_tc_b_image<2, LAPLACE_P2_ISO>();

struct TcKRefIso {
  template <int D, int FORM>
  __device__ __forceinline__ static const TcBImage<D, FORM>* b_image() {
    if constexpr (D == 3) {
      return &kTcB3iso;
    } else {
      return &kTcB2iso;
    }
  }
};

// G of a curved element: w |J(centroid)| J^{-1}_{mu a,k} J^{-1}_{nu a,l} / DEN over
// the folded slot pairs (Eq. 18), each entry as the FP32 kernel forms it.
struct TcGeoIso {
  template <int D, int FORM>
  __device__ __forceinline__ static int tile_g(const FwdParams<float, float>&, const float* mid, int64_t e,
                                               const float (&X)[D + 1][D], float w,
                                               float (&G)[FormTraits<D, FORM>::NG]) {
    constexpr int NE = D * (D + 1) / 2, NP = FormTraits<D, FORM>::NP;
    float ji[D + 1][D][D], scale;
    if (!iso_geometry<D, FORM>(X, mid + e * (NE * D), w, ji, scale)) return DEVERR_DEGENERATE;  // G stays 0
#pragma unroll
    for (int pp = 0; pp < NP; ++pp)
#pragma unroll
      for (int qq = pp; qq < NP; ++qq) {
        float s = 0.f;
#pragma unroll
        for (int al = 0; al < D; ++al) s = fmaf(ji[pp / D][pp % D][al], ji[qq / D][qq % D][al], s);
        G[pair_index(pp, qq, NP)] = scale * s;
      }
    return 0;
  }
};

cudaError_t launch_fwd_iso_tc(const FwdLaunch& L, const float* mid) {
  if (L.form != LAPLACE_P2_ISO) return cudaErrorInvalidValue;
  if (L.dim == 3) return launch_tc_t<3, LAPLACE_P2_ISO, TcGeoIso, TcKRefIso>(L, mid);
  return launch_tc_t<2, LAPLACE_P2_ISO, TcGeoIso, TcKRefIso>(L, mid);
}

}  // namespace fem
