// fem_iso.cuh -- the Jacobians of a quadratic-geometry (non-affine) simplex,
// Eqs. 16-17: the map from the reference element through the P2 geometry
// basis psi_a of the d+1 vertices and d(d+1)/2 edge-midpoint nodes, its
// Jacobian at each vertex (whose inverses Eq. 17 interpolates) and at the
// centroid (where |J| is taken).
#pragma once
#include <utility>

#include "fem_core.cuh"

namespace fem {

// d psi_a / d xi_mu of the quadratic geometry basis (vertices, then edges in
// the P2 order) at reference vertex k (k <= D); all integers.
template <int D>
constexpr int geo_dpsi(int a, int mu, int k) {
  if (a <= D) return (a == k ? 3 : -1) * dlam(a, mu);
  int t = a - (D + 1);
  for (int p = 0; p <= D; ++p)
    for (int q = p + 1; q <= D; ++q) {
      if (t == 0) return 4 * ((p == k ? dlam(q, mu) : 0) + (q == k ? dlam(p, mu) : 0));
      --t;
    }
  return 0;
}

constexpr int n_geo(int D) { return (D + 1) * (D + 2) / 2; }

// e[mu][al] = sum_a geo_dpsi(a, mu, K) * node_a[al] with node 0 at the origin.
template <int D, int K>
__device__ __forceinline__ void geo_jacobian(const float (&nd)[n_geo(D)][D], float (&e)[D][D]) {
#pragma unroll
  for (int mu = 0; mu < D; ++mu)
#pragma unroll
    for (int al = 0; al < D; ++al) {
      float s = 0.f;
#pragma unroll
      for (int a = 1; a < n_geo(D); ++a) {
        const int c = geo_dpsi<D>(a, mu, K);
        if (c != 0) s = fmaf(float(c), nd[a][al], s);
      }
      e[mu][al] = s;
    }
}

template <int D>
__device__ __forceinline__ float det_adj(const float (&e)[D][D], float (&adj)[D][D]) {
  adjugate(e, adj);
  float det = 0.f;
#pragma unroll
  for (int al = 0; al < D; ++al) det = fmaf(e[0][al], adj[0][al], det);
  return det;
}

// J^{-1} at vertex K into ji[K]; J at vertex K added into esum.
template <int D, int K>
__device__ __forceinline__ bool vertex_jinv(const float (&nd)[n_geo(D)][D], float (&ji)[D + 1][D][D],
                                            float (&esum)[D][D]) {
  float e[D][D], adj[D][D];
  geo_jacobian<D, K>(nd, e);
#pragma unroll
  for (int mu = 0; mu < D; ++mu)
#pragma unroll
    for (int al = 0; al < D; ++al) esum[mu][al] = K == 0 ? e[mu][al] : esum[mu][al] + e[mu][al];
  const float det = det_adj<D>(e, adj);
  const float r = __frcp_rn(det);
#pragma unroll
  for (int mu = 0; mu < D; ++mu)
#pragma unroll
    for (int al = 0; al < D; ++al) ji[K][mu][al] = adj[mu][al] * r;  // (J^{-1})_{mu al} at vertex K
  return det != 0.f;
}

template <int D, int... Ks>
__device__ __forceinline__ bool all_vertex_jinv(const float (&nd)[n_geo(D)][D], float (&ji)[D + 1][D][D],
                                                float (&esum)[D][D], std::integer_sequence<int, Ks...>) {
  return (vertex_jinv<D, Ks>(nd, ji, esum) & ...);
}

// One element's inverse Jacobians at its vertices (ji[k][mu][al] = (J^{-1})_{mu al}
// at vertex k) and scale = w |det J(centroid)| / DEN, from its vertex
// coordinates X and its edge nodes m (d(d+1)/2 points, P2 edge order).  False
// (ji, scale undefined) when J is singular at a vertex or at the centroid.
template <int D, int FORM>
__device__ __forceinline__ bool iso_geometry(const float (&X)[D + 1][D], const float* m, float w,
                                             float (&ji)[D + 1][D][D], float& scale) {
  constexpr int NE = D * (D + 1) / 2;
  float nd[n_geo(D)][D];  // geometry nodes relative to vertex 0
#pragma unroll
  for (int a = 0; a <= D; ++a)
#pragma unroll
    for (int al = 0; al < D; ++al) nd[a][al] = X[a][al] - X[0][al];
#pragma unroll
  for (int q = 0; q < NE; ++q)
#pragma unroll
    for (int al = 0; al < D; ++al) nd[D + 1 + q][al] = __ldcs(m + q * D + al) - X[0][al];
  // J is affine in xi (psi quadratic), so the sum of the vertex Jacobians is
  // (D + 1) J at the centroid
  float ec[D][D], adjc[D][D];
  bool ok = all_vertex_jinv<D>(nd, ji, ec, std::make_integer_sequence<int, D + 1>{});
  float detc = det_adj<D>(ec, adjc);
  detc *= D == 2 ? (1.f / 9.f) : (1.f / 64.f);  // det scales by (D + 1)^D
  ok &= detc != 0.f;
  scale = w * fabsf(detc) * (1.f / float(FormTraits<D, FORM>::DEN));
  return ok;
}

}  // namespace fem
