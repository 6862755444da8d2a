// fem_iso_adj.cuh -- per-element pieces of the adjoint of the non-affine
// (quadratic-geometry) forward, Eqs. 16-19, shared by the FP32 adjoint kernel
// (fem_bwd_iso.cu) and the one whose contraction adjoint runs on the tensor
// cores (fem_bwd_iso_tc.cu): the slot-pair terms, the pullback of the vertex
// Jacobians to the geometry nodes, and the 16-byte staging of a tile's edge
// nodes.
#pragma once

#include "fem_bwd.cuh"
#include "fem_iso.cuh"

namespace fem {

// Folded slot pair G with the contraction's adjoint s (s = sum_T K'[G][T] sym(dA)_T):
// dsc += s H_G and the two inverse-Jacobian rows of the pair.
template <int D, int FORM, int G>
__device__ __forceinline__ void iso_adj_apply(float s, const float (&ji)[D + 1][D][D], float sc,
                                              float (&dji)[D + 1][D][D], float& dsc) {
  using FT = FormTraits<D, FORM>;
  constexpr int pp = tri_row(G, FT::NP), qq = tri_col(G, FT::NP);
  constexpr int kp = pp / D, mp = pp % D, kq = qq / D, mq = qq % D;
  float h = 0.f;
#pragma unroll
  for (int a = 0; a < D; ++a) h = fmaf(ji[kp][mp][a], ji[kq][mq][a], h);
  dsc = fmaf(s, h, dsc);
  const float t = s * sc;
  if constexpr (pp == qq) {
#pragma unroll
    for (int a = 0; a < D; ++a) dji[kp][mp][a] = fmaf(2.f * t, ji[kp][mp][a], dji[kp][mp][a]);
  } else {
#pragma unroll
    for (int a = 0; a < D; ++a) {
      dji[kp][mp][a] = fmaf(t, ji[kq][mq][a], dji[kp][mp][a]);
      dji[kq][mq][a] = fmaf(t, ji[kp][mp][a], dji[kq][mq][a]);
    }
  }
}

template <int D, int FORM, int G, class Sym>
__device__ __forceinline__ void iso_adj_term(const Sym& sym, const float (&ji)[D + 1][D][D], float sc,
                                             float (&dji)[D + 1][D][D], float& dsc) {
  using FT = FormTraits<D, FORM>;
  iso_adj_apply<D, FORM, G>(kcol<D, FORM, G>(sym, std::make_integer_sequence<int, FT::NT>{}), ji, sc, dji, dsc);
}

template <int D, int FORM, class Sym, int... Gs>
__device__ __forceinline__ void iso_adj_all(const Sym& sym, const float (&ji)[D + 1][D][D], float sc,
                                            float (&dji)[D + 1][D][D], float& dsc, std::integer_sequence<int, Gs...>) {
  (iso_adj_term<D, FORM, Gs>(sym, ji, sc, dji, dsc), ...);
}

// d nd_a[al] += sum_mu dpsi_a/dxi_mu(vertex K) de[mu][al] over the nodes a >= 1.
template <int D, int K>
__device__ __forceinline__ void geo_pullback(const float (&de)[D][D], float (&dnd)[n_geo(D)][D]) {
#pragma unroll
  for (int a = 1; a < n_geo(D); ++a)
#pragma unroll
    for (int mu = 0; mu < D; ++mu) {
      const int c = geo_dpsi<D>(a, mu, K);
      if (c != 0)
#pragma unroll
        for (int al = 0; al < D; ++al) dnd[a][al] = fmaf(float(c), de[mu][al], dnd[a][al]);
    }
}

// ji[k] = e_k^{-T}: d e_k = -ji[k] dji[k]^T ji[k] + dec, pulled back to the nodes.
template <int D, int K>
__device__ __forceinline__ void vertex_pullback(const float (&ji)[D + 1][D][D], const float (&dji)[D + 1][D][D],
                                                const float (&dec)[D][D], float (&dnd)[n_geo(D)][D]) {
  float m[D][D];  // dji[K]^T ji[K]: m[be][al] = sum_nu dji[K][nu][be] ji[K][nu][al]
#pragma unroll
  for (int be = 0; be < D; ++be)
#pragma unroll
    for (int al = 0; al < D; ++al) {
      float s = 0.f;
#pragma unroll
      for (int nu = 0; nu < D; ++nu) s = fmaf(dji[K][nu][be], ji[K][nu][al], s);
      m[be][al] = s;
    }
  float de[D][D];
#pragma unroll
  for (int mu = 0; mu < D; ++mu)
#pragma unroll
    for (int al = 0; al < D; ++al) {
      float s = dec[mu][al];
#pragma unroll
      for (int be = 0; be < D; ++be) s = fmaf(-ji[K][mu][be], m[be][al], s);
      de[mu][al] = s;
    }
  geo_pullback<D, K>(de, dnd);
}

template <int D, int... Ks>
__device__ __forceinline__ void all_vertex_pullback(const float (&ji)[D + 1][D][D], const float (&dji)[D + 1][D][D],
                                                    const float (&dec)[D][D], float (&dnd)[n_geo(D)][D],
                                                    std::integer_sequence<int, Ks...>) {
  (vertex_pullback<D, Ks>(ji, dji, dec, dnd), ...);
}

// A tile's contiguous run of nf floats between global and shared memory, as
// 16-byte pieces when both ends allow it (the edge nodes of 32 elements are
// 2304 bytes on tets, 768 on triangles), else word by word.
__device__ __forceinline__ void tile_load_async(float* st, const float* g, int nf, int lane) {
  if ((reinterpret_cast<uintptr_t>(g) & 15) == 0 && (nf & 3) == 0) {
    for (int q = lane; q < nf / 4; q += 32) cp_async<16>(st + 4 * q, g + 4 * q);
  } else {
    for (int q = lane; q < nf; q += 32) cp_async<4>(st + q, g + q);
  }
}

__device__ __forceinline__ void tile_store(float* g, const float* st, int nf, int lane) {
  if ((reinterpret_cast<uintptr_t>(g) & 15) == 0 && (nf & 3) == 0) {
    for (int q = lane; q < nf / 4; q += 32)
      __stcs(reinterpret_cast<float4*>(g) + q, *reinterpret_cast<const float4*>(st + 4 * q));
  } else {
    for (int q = lane; q < nf; q += 32) __stcs(g + q, st[q]);
  }
}

}  // namespace fem
