// fem_fwd_iso.cu -- forward integration of the Laplacian on non-affine
// (quadratic-geometry) elements, Eqs. 16-19.
//
// Each element is given by its d+1 vertices (conn, coords) and the d(d+1)/2
// edge-midpoint nodes of its quadratic geometry map (mid, element by
// element).  Per lane (one element):
//   1. the nodes relative to vertex 0 (so the map's derivatives see small
//      differences, not absolute coordinates);
//   2. J at every vertex k from the derivatives of the quadratic geometry
//      basis there (small integers, compile time), its adjugate and det, and
//      J^{-1}_k = adj / det -- the values the projection of Eq. 17 interpolates;
//   3. |J| = |det J| at the centroid (Eq. 17 keeps |J| outside the integral);
//   4. G^{(k mu),(l nu)} = w |J| / DEN  sum_a J^{-1}_{mu a,k} J^{-1}_{nu a,l}
//      over the folded slot pairs (Eq. 18), each entry (without the common
//      factor w |J| / DEN) added into the accumulators of A as soon as it is
//      formed (A_ij += K^{ij}_g G_g with K as immediates, g in increasing
//      order: the sums of the G-first contraction, without holding all of G
//      in registers), the factor applied once per entry of A, then the same
//      tile store as the affine kernel (Eq. 19).
// The Jacobian steps run in plain FP32: this path serves curved, non-sliver
// elements; an element with a singular J at a vertex or at the centroid is
// flagged degenerate and gets A = 0.
#include "fem_fwd.cuh"
#include "fem_iso.cuh"

namespace fem {

namespace {

// acc[T] += K'[G][T] * gv over the unique entries T of A (zero terms generate no code).
template <int D, int FORM, int G, int T>
__device__ __forceinline__ void kscatter(float* acc, float gv) {
  using FT = FormTraits<D, FORM>;
  constexpr int k = Ref<D, FORM>::K.v[G][tri_row(T, FT::N)][tri_col(T, FT::N)];
  if constexpr (k == 1) {
    acc[T] += gv;
  } else if constexpr (k == -1) {
    acc[T] -= gv;
  } else if constexpr (k != 0) {
    acc[T] = fmaf(gv, float(k), acc[T]);
  }
}

template <int D, int FORM, int G, int... Ts>
__device__ __forceinline__ void scatter_g(float* acc, float gv, std::integer_sequence<int, Ts...>) {
  (kscatter<D, FORM, G, Ts>(acc, gv), ...);
}

// G_g / scale for the slot pair g = (p, q), p <= q, p = (k mu):
// sum_a Jinv_{mu a,k} Jinv_{nu a,l}.
template <int D, int FORM, int G>
__device__ __forceinline__ void iso_term(const float (&ji)[D + 1][D][D], float* acc) {
  using FT = FormTraits<D, FORM>;
  constexpr int pp = tri_row(G, FT::NP), qq = tri_col(G, FT::NP);
  float s = 0.f;
#pragma unroll
  for (int al = 0; al < D; ++al) s = fmaf(ji[pp / D][pp % D][al], ji[qq / D][qq % D][al], s);
  scatter_g<D, FORM, G>(acc, s, std::make_integer_sequence<int, FT::NT>{});
}

// acc = scale * sum_g K_g G_g / scale: the common factor scale = w |J| / DEN
// once per entry of A rather than once per G entry.
template <int D, int FORM, int... Gs>
__device__ __forceinline__ void iso_accumulate(const float (&ji)[D + 1][D][D], float scale, float* acc,
                                               std::integer_sequence<int, Gs...>) {
  (iso_term<D, FORM, Gs>(ji, acc), ...);
#pragma unroll
  for (int t = 0; t < FormTraits<D, FORM>::NT; ++t) acc[t] *= scale;
}

template <int D, int FORM, class Sink, int... Ts>
__device__ __forceinline__ void put_all(Sink& sink, const float* acc, std::integer_sequence<int, Ts...>) {
  using FT = FormTraits<D, FORM>;
  (sink.template put<tri_row(Ts, FT::N), tri_col(Ts, FT::N)>(acc[Ts]), ...);
}

// CTA shape: warps never wait for one another, so the CTA size only sets how
// finely the register file is shared out.  On tets the P1 form runs one-warp
// CTAs with at least 20 resident per SM, which holds it to 96 registers
// without spills (21 warps per SM against 16 at 128 registers); the P2 form
// with at least 16, which holds its 55 accumulators and four inverse
// Jacobians to 128 registers without spills (16 warps per SM, against 8 at
// the 245 registers it takes unbounded).
template <int D, int FORM>
struct IsoShape {
  static constexpr bool tight = (D == 3);
  static constexpr int threads = tight ? 32 : 128;
  static constexpr int min_ctas = tight ? (FORM == LAPLACE_P1_ISO ? 20 : 16) : 1;
};

template <int D, int FORM>
__global__ void __launch_bounds__(IsoShape<D, FORM>::threads, IsoShape<D, FORM>::min_ctas)
    fem_fwd_iso_kernel(FwdParams<float, float> p, const float* __restrict__ mid) {
  using FT = FormTraits<D, FORM>;
  using PL = FwdPlan<D, FORM, float, float>;
  constexpr int NE = D * (D + 1) / 2;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  float* st = reinterpret_cast<float*>(smem_raw + size_t(warp) * PL::per_warp);
  const int64_t ntiles = (p.n_elem + 31) / 32;
  int err = 0;
  for (int64_t t = int64_t(blockIdx.x) * nwarps + warp; t < ntiles; t += int64_t(gridDim.x) * nwarps) {
    const int64_t e = t * 32 + lane;
    int v[D + 1];
    float X[D + 1][D];
    load_conn<D>(p.conn, e, p.n_elem, p.vec_conn, v);
    const int flags = gather_regs<D>(p.coords, p.n_vert, e, p.n_elem, v, X);
    float ji[D + 1][D][D];
    float scale = 0.f;
    bool ok = false;
    if (flags & GF_OK) {
      const float w = (p.coef && e < p.n_elem) ? __ldg(p.coef + e) : 1.f;
      ok = iso_geometry<D, FORM>(X, mid + e * (NE * D), w, ji, scale);
      if (!ok) err |= DEVERR_DEGENERATE;
    } else if (flags & GF_ELEM) {
      err |= DEVERR_CONN;
    }
    fwd_fill_store<D, FORM, float, float, false>(
        p, t, lane,
        [&](auto& sink) {
          float acc[FT::NT];
#pragma unroll
          for (int i = 0; i < FT::NT; ++i) acc[i] = 0.f;
          if (ok) iso_accumulate<D, FORM>(ji, scale, acc, std::make_integer_sequence<int, FT::NG>{});
          put_all<D, FORM>(sink, acc, std::make_integer_sequence<int, FT::NT>{});
        },
        st, nullptr);
  }
  err = __reduce_or_sync(0xffffffffu, err);
  if (err && lane == 0 && p.dev_err) atomicOr(p.dev_err, err);
}

template <int D, int FORM>
cudaError_t launch_iso_t(const FwdLaunch& L, const float* mid) {
  using PL = FwdPlan<D, FORM, float, float>;
  FwdParams<float, float> p;
  p.conn = L.conn;
  p.coords = static_cast<const float*>(L.coords);
  p.coef = L.coef;
  p.A = static_cast<float*>(L.A);
  p.n_elem = L.n_elem;
  p.n_vert = L.n_vert;
  p.dev_err = L.dev_err;
  p.vec_conn = (D == 3) && (reinterpret_cast<uintptr_t>(L.conn) % 16 == 0);
  p.vec_store = (reinterpret_cast<uintptr_t>(L.A) % 16 == 0);
  auto kern = fem_fwd_iso_kernel<D, FORM>;
  const int warps = IsoShape<D, FORM>::threads / 32;
  const size_t smem = size_t(warps) * PL::per_warp;
  cudaError_t st = ensure_smem(reinterpret_cast<const void*>(kern), smem);
  if (st != cudaSuccess) return st;
  const unsigned grid = pipeline_grid(reinterpret_cast<const void*>(kern), warps, smem, L.n_elem, L.ctas_per_sm);
  kern<<<grid, warps * 32, smem, L.stream>>>(p, mid);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_fwd_iso(const FwdLaunch& L, const float* mid) {
  if (L.dim == 2) {
    if (L.form == LAPLACE_P1_ISO) return launch_iso_t<2, LAPLACE_P1_ISO>(L, mid);
    if (L.form == LAPLACE_P2_ISO) return launch_iso_t<2, LAPLACE_P2_ISO>(L, mid);
  } else {
    if (L.form == LAPLACE_P1_ISO) return launch_iso_t<3, LAPLACE_P1_ISO>(L, mid);
    if (L.form == LAPLACE_P2_ISO) return launch_iso_t<3, LAPLACE_P2_ISO>(L, mid);
  }
  return cudaErrorInvalidValue;
}

}  // namespace fem
