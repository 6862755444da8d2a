// fem_tc.cu -- the tensor-core contraction (fem_tc.cuh) for the affine forms it
// serves: the P2 Laplacian (with a per-element or a P1 coefficient) and P1
// elasticity on triangles and tetrahedra.
#include <cudaTypedefs.h>

#include <mutex>

#include "fem_tc.cuh"

namespace fem {

namespace {
PFN_cuTensorMapEncodeTiled_v12000 tc_map_encoder() {
  static std::once_flag once;
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
  });
  return fn;
}
}  // namespace

bool encode_tc_rows_map(CUtensorMap* map, const void* base, int64_t rows, int cols) {
  if (!base || rows <= 0 || rows > (int64_t(1) << 32) || reinterpret_cast<uintptr_t>(base) % 16 != 0 ||
      (cols * 4) % 16 != 0)
    return false;
  PFN_cuTensorMapEncodeTiled_v12000 fn = tc_map_encoder();
  if (!fn) return false;
  const cuuint64_t dims[2] = {cuuint64_t(cols), cuuint64_t(rows)};
  const cuuint64_t strides[1] = {cuuint64_t(cols) * 4};  // bytes between rows
  const cuuint32_t box[2] = {32, 32};                    // 128-byte row segments of one warp's 32 elements
  const cuuint32_t estr[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// B operands of the forms the tensor-core kernel serves, built at compile time.
static_assert(tc_b_exact<3, ELASTIC_P1>() && tc_b_exact<3, LAPLACE_P2>() && tc_b_exact<2, ELASTIC_P1>() &&
                  tc_b_exact<2, LAPLACE_P2>() && tc_b_exact<3, LAPLACE_P2_W1>() && tc_b_exact<2, LAPLACE_P2_W1>(),
              "K' * DEN must be exact in BF16");
__device__ const TcBImage<3, ELASTIC_P1> kTcB3e = make_tc_b_image<3, ELASTIC_P1>();
__device__ const TcBImage<3, LAPLACE_P2> kTcB3p = make_tc_b_image<3, LAPLACE_P2>();
__device__ const TcBImage<2, ELASTIC_P1> kTcB2e = make_tc_b_image<2, ELASTIC_P1>();
__device__ const TcBImage<2, LAPLACE_P2> kTcB2p = make_tc_b_image<2, LAPLACE_P2>();
__device__ const TcBImage<3, LAPLACE_P2_W1> kTcB3w = make_tc_b_image<3, LAPLACE_P2_W1>();
__device__ const TcBImage<2, LAPLACE_P2_W1> kTcB2w = make_tc_b_image<2, LAPLACE_P2_W1>();

struct TcKRefAffine {
  template <int D, int FORM>
  __device__ __forceinline__ static const TcBImage<D, FORM>* b_image() {
    if constexpr (D == 3 && FORM == ELASTIC_P1) {
      return &kTcB3e;
    } else if constexpr (D == 3 && FORM == LAPLACE_P2) {
      return &kTcB3p;
    } else if constexpr (D == 2 && FORM == ELASTIC_P1) {
      return &kTcB2e;
    } else if constexpr (D == 2 && FORM == LAPLACE_P2) {
      return &kTcB2p;
    } else if constexpr (D == 3 && FORM == LAPLACE_P2_W1) {
      return &kTcB3w;
    } else {
      static_assert(D == 2 && FORM == LAPLACE_P2_W1, "form without a tensor-core B operand");
      return &kTcB2w;
    }
  }
};

// G of the Laplacian with a P1 coefficient (Eq. 22): slot k * d(d+1)/2 + g holds
// w_k G_g, with w_k the coefficient at the element's vertex k (vw: [n_vert]
// vertex values, or NULL for w = 1) and G_g = (adj adj^T)_g / (|det J| DEN) in
// compensated FP32, as the FP32 kernel forms them.
struct TcGeoW1 {
  template <int D, int FORM>
  __device__ __forceinline__ static int tile_g(const FwdParams<float, float>& p, const float* vw, int64_t e,
                                               const float (&X)[D + 1][D], float,
                                               float (&G)[FormTraits<D, FORM>::NG]) {
    using FT = FormTraits<D, FORM>;
    Jac<D, float> jac;
    const bool nondeg = jacobian<D, JAC_COMP>(X, jac);
    const float scale = nondeg ? __fdividef(1.f, dev_abs(jac.det) * float(FT::DEN)) : 0.f;
    float Gt[FT::NGB];
    geometric_tensor<D, FT::BASE>(jac.adj, scale, Gt);
    int v[D + 1];  // in range: the caller gathered the coordinates of these vertices
    load_conn<D>(p.conn, e, p.n_elem, 0, v);
#pragma unroll
    for (int k = 0; k <= D; ++k) {
      const float wk = vw ? __ldg(vw + v[k]) : 1.f;
#pragma unroll
      for (int g = 0; g < FT::NGB; ++g) G[k * FT::NGB + g] = wk * Gt[g];
    }
    return nondeg ? 0 : DEVERR_DEGENERATE;
  }
};

cudaError_t launch_fwd_tc(const FwdLaunch& L) {
  if (L.coord_f64 || L.out_f64) return cudaErrorInvalidValue;
  if (L.dim == 3 && L.form == ELASTIC_P1) return launch_tc_t<3, ELASTIC_P1, TcGeoAffine, TcKRefAffine>(L, nullptr);
  if (L.dim == 3 && L.form == LAPLACE_P2) return launch_tc_t<3, LAPLACE_P2, TcGeoAffine, TcKRefAffine>(L, nullptr);
  if (L.dim == 2 && L.form == ELASTIC_P1) return launch_tc_t<2, ELASTIC_P1, TcGeoAffine, TcKRefAffine>(L, nullptr);
  if (L.dim == 2 && L.form == LAPLACE_P2) return launch_tc_t<2, LAPLACE_P2, TcGeoAffine, TcKRefAffine>(L, nullptr);
  if (L.form == LAPLACE_P2_W1) {  // the vertex values go to the geometry, not to the per-element load
    FwdLaunch Lw = L;
    Lw.coef = nullptr;
    return L.dim == 3 ? launch_tc_t<3, LAPLACE_P2_W1, TcGeoW1, TcKRefAffine>(Lw, L.coef)
                      : launch_tc_t<2, LAPLACE_P2_W1, TcGeoW1, TcKRefAffine>(Lw, L.coef);
  }
  return cudaErrorInvalidValue;
}

}  // namespace fem
