// fem_core.cuh -- per-element device math: Jacobian, geometric tensor G and
// the sparse G:K contraction (Knepley & Terrel, Sec. 3, Eqs. 1, 5-8, 14-15).
//
// Affine map of the reference simplex {0, e_1, .., e_d}:
//   x(xi) = x_0 + sum_mu xi_mu (x_{mu+1} - x_0),  so  J_{a mu} = x_{mu+1,a} - x_{0,a}.
// The edge vectors e_mu = x_{mu+1} - x_0 are the columns of J.  We keep
// adj(J) (rows adj[mu][a], J^{-1} = adj / det J) and det J; with them
//   Laplacian   G^{mu nu}        = w |J| sum_a Jinv_{mu a} Jinv_{nu a} = (w/|det|) sum_a adj_{mu a} adj_{nu a}  (Eq. 8)
//   elasticity  G^{(mu a),(nu b)} = w |J| Jinv_{mu a} Jinv_{nu b}      = (w/|det|) adj_{mu a} adj_{nu b}
// w is the optional per-element coefficient (piecewise-constant case of Eq. 20).
//
// Precision of the Jacobian steps (selected at compile time):
//   JAC_F64  : J, adj, det and G in FP64 (exact edge vectors for FP32 input).
//   JAC_COMP : compensated FP32.  Edge vectors split exactly into hi + lo by
//              TwoSum (Knuth); the cross product e_1 x e_2 is formed as a
//              double-float with FMA-based TwoProduct; det = e_0 . (e_1 x e_2) is
//              accumulated with the compensated dot product of Ogita, Rump and
//              Oishi ("Accurate sum and dot product", SIAM J. Sci. Comput. 2005);
//              the lo parts enter through the first-order term sum_mu lo_mu . adj_mu.
//              For sliver elements det J cancels catastrophically in plain FP32;
//              this keeps its relative error near (few eps^2) / (height ratio).
//   JAC_F32  : plain FP32 (for error studies).
//   JAC_SAVED: the adjoint with det J saved by the forward: FP32 edge vectors
//              and adjugate (the hi parts of the compensated mode), det J as
//              given.
#pragma once
#include <cstdint>
#include <type_traits>
#include <utility>

#include "fem_forms.cuh"

namespace fem {

enum JacMode : int { JAC_F64 = 1, JAC_COMP = 2, JAC_F32 = 3, JAC_SAVED = 4 };
enum DevErr : int { DEVERR_CONN = 1, DEVERR_DEGENERATE = 2, DEVERR_TIMEOUT = 4 };

// ---------------------------------------------------------------- error-free transforms
// The _rn intrinsics are never contracted into FMAs or reordered by the compiler.
__device__ __forceinline__ float two_sum(float a, float b, float& err) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  err = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return s;
}
__device__ __forceinline__ float two_prod(float a, float b, float& err) {
  float p = __fmul_rn(a, b);
  err = __fmaf_rn(a, b, -p);
  return p;
}
// a*d - b*c as an unevaluated sum hi + lo
__device__ __forceinline__ float diff_prod_df(float a, float d, float b, float c, float& lo) {
  float e1, e2, t;
  float p1 = two_prod(a, d, e1);
  float p2 = two_prod(b, c, e2);
  float s = two_sum(p1, -p2, t);
  lo = __fadd_rn(t, __fsub_rn(e1, e2));
  return s;
}

// ---------------------------------------------------------------- Jacobian

template <int D, class GT>
struct Jac {
  GT e[D][D];    // edge vectors e[mu][a] (hi parts for the compensated mode)
  GT adj[D][D];  // adj(J)[mu][a]
  GT det;        // det J (accurately rounded in JAC_COMP)
  double det_hp; // det J to the precision the mode reaches (double-float value in JAC_COMP)
};

// x * y - z * w with the rounding spelled out (one product rounded, then a
// fused multiply-add), so that every kernel forms the same bits.
__device__ __forceinline__ float cross_term(float x, float y, float z, float w) {
  return __fmaf_rn(x, y, -__fmul_rn(z, w));
}
__device__ __forceinline__ double cross_term(double x, double y, double z, double w) {
  return __fma_rn(x, y, -__dmul_rn(z, w));
}

// adjugate rows from edge vectors (d det / d e_mu = adj[mu])
template <class GT>
__device__ __forceinline__ void adjugate(const GT (&e)[3][3], GT (&adj)[3][3]) {
#pragma unroll
  for (int mu = 0; mu < 3; ++mu) {
    const GT* a = e[(mu + 1) % 3];
    const GT* b = e[(mu + 2) % 3];
    adj[mu][0] = cross_term(a[1], b[2], a[2], b[1]);
    adj[mu][1] = cross_term(a[2], b[0], a[0], b[2]);
    adj[mu][2] = cross_term(a[0], b[1], a[1], b[0]);
  }
}
template <class GT>
__device__ __forceinline__ void adjugate(const GT (&e)[2][2], GT (&adj)[2][2]) {
  adj[0][0] = e[1][1];
  adj[0][1] = -e[1][0];
  adj[1][0] = -e[0][1];
  adj[1][1] = e[0][0];
}

// Returns false when det J == 0 (degenerate element).
template <int D, int JAC, class CT, class GT>
__device__ __forceinline__ bool jacobian(const CT (&X)[D + 1][D], Jac<D, GT>& j) {
  if constexpr (JAC == JAC_F64 || JAC == JAC_F32) {
    using W = typename std::conditional<JAC == JAC_F64, double, float>::type;
    W e[D][D], adj[D][D];
#pragma unroll
    for (int mu = 0; mu < D; ++mu)
#pragma unroll
      for (int a = 0; a < D; ++a) e[mu][a] = W(X[mu + 1][a]) - W(X[0][a]);
    adjugate(e, adj);
    W det = 0;
#pragma unroll
    for (int a = 0; a < D; ++a) det += e[0][a] * adj[0][a];
#pragma unroll
    for (int mu = 0; mu < D; ++mu)
#pragma unroll
      for (int a = 0; a < D; ++a) {
        j.e[mu][a] = GT(e[mu][a]);
        j.adj[mu][a] = GT(adj[mu][a]);
      }
    j.det = GT(det);
    j.det_hp = double(det);
    return det != W(0);
  } else {
    static_assert(JAC == JAC_COMP, "jacobian mode");
    float eh[D][D], el[D][D], adj[D][D];
#pragma unroll
    for (int mu = 0; mu < D; ++mu)
#pragma unroll
      for (int a = 0; a < D; ++a) eh[mu][a] = two_sum(float(X[mu + 1][a]), -float(X[0][a]), el[mu][a]);
    adjugate(eh, adj);
    // det(H) = e_0 . adj_0 with adj_0 formed as a double-float, then a compensated dot
    float ch[D], cl[D];
    if constexpr (D == 3) {
      ch[0] = diff_prod_df(eh[1][1], eh[2][2], eh[1][2], eh[2][1], cl[0]);
      ch[1] = diff_prod_df(eh[1][2], eh[2][0], eh[1][0], eh[2][2], cl[1]);
      ch[2] = diff_prod_df(eh[1][0], eh[2][1], eh[1][1], eh[2][0], cl[2]);
    } else {
      ch[0] = eh[1][1];
      cl[0] = 0.f;
      ch[1] = -eh[1][0];
      cl[1] = 0.f;
    }
    float err;
    float p = two_prod(eh[0][0], ch[0], err);
#pragma unroll
    for (int a = 1; a < D; ++a) {
      float r, q;
      float h = two_prod(eh[0][a], ch[a], r);
      p = two_sum(p, h, q);
      err = __fadd_rn(err, __fadd_rn(q, r));
    }
    float corr = 0.f;  // lo parts of the components of adj_0 and of every edge vector
#pragma unroll
    for (int a = 0; a < D; ++a) corr = __fmaf_rn(eh[0][a], cl[a], corr);
#pragma unroll
    for (int mu = 0; mu < D; ++mu)
#pragma unroll
      for (int a = 0; a < D; ++a) corr = __fmaf_rn(el[mu][a], adj[mu][a], corr);
    float det = __fadd_rn(p, __fadd_rn(err, corr));
#pragma unroll
    for (int mu = 0; mu < D; ++mu)
#pragma unroll
      for (int a = 0; a < D; ++a) {
        j.e[mu][a] = GT(eh[mu][a]);
        j.adj[mu][a] = GT(adj[mu][a]);
      }
    j.det = GT(det);
    j.det_hp = double(p) + (double(err) + double(corr));
    return det != 0.f;
  }
}

// Edge vectors and adjugate in FP32 with det J given (saved by the forward);
// false when det J == 0.
template <int D>
__device__ __forceinline__ bool jacobian_saved(const float (&X)[D + 1][D], float det, Jac<D, float>& j) {
#pragma unroll
  for (int mu = 0; mu < D; ++mu)
#pragma unroll
    for (int a = 0; a < D; ++a) j.e[mu][a] = __fsub_rn(X[mu + 1][a], X[0][a]);
  adjugate(j.e, j.adj);
  j.det = det;
  j.det_hp = double(det);
  return det != 0.f;
}

// ---------------------------------------------------------------- geometric tensor

// Folded G scaled by scale = w / (|det| * DEN): the contraction then uses the
// integer K' * DEN as immediates.
template <int D, int FORM, class GT>
__device__ __forceinline__ void geometric_tensor(const GT (&adj)[D][D], GT scale,
                                                 GT (&G)[FormTraits<D, FORM>::NG]) {
  using FT = FormTraits<D, FORM>;
  if constexpr (FORM != ELASTIC_P1) {
#pragma unroll
    for (int mu = 0; mu < D; ++mu)
#pragma unroll
      for (int nu = mu; nu < D; ++nu) {
        GT s = 0;
#pragma unroll
        for (int a = 0; a < D; ++a) s += adj[mu][a] * adj[nu][a];
        G[pair_index(mu, nu, D)] = s * scale;
      }
  } else {
    GT sa[FT::NP];
#pragma unroll
    for (int p = 0; p < FT::NP; ++p) sa[p] = adj[p / D][p % D] * scale;
#pragma unroll
    for (int p = 0; p < FT::NP; ++p)
#pragma unroll
      for (int q = p; q < FT::NP; ++q) G[pair_index(p, q, FT::NP)] = sa[p] * adj[q / D][q % D];
  }
}

// ---------------------------------------------------------------- sparse contraction
// A_ij = sum_g G[g] K'[g][i][j], with K' * DEN an integer immediate; zero terms
// generate no code.  Only i <= j is evaluated (A is symmetric).

template <int D, int FORM, int I, int J, int G, class T>
__device__ __forceinline__ void kterm(T& acc, const T* Gv) {
  constexpr int k = Ref<D, FORM>::K.v[G][I][J];
  if constexpr (k == 1) {
    acc += Gv[G];
  } else if constexpr (k == -1) {
    acc -= Gv[G];
  } else if constexpr (k != 0) {
    acc = fma(Gv[G], T(k), acc);
  }
}

template <int D, int FORM, int I, int J, class T, int... Gs>
__device__ __forceinline__ T kentry(const T* Gv, std::integer_sequence<int, Gs...>) {
  T acc = 0;
  (kterm<D, FORM, I, J, Gs>(acc, Gv), ...);
  return acc;
}

// sink.put(i, j, value) is called once per unique entry (i <= j) with compile-time i, j
template <int D, int FORM, class T, class Sink, int... Ts>
__device__ __forceinline__ void contract_seq(const T* Gv, Sink& sink,
                                             std::integer_sequence<int, Ts...>) {
  using FT = FormTraits<D, FORM>;
  (sink.template put<tri_row(Ts, FT::N), tri_col(Ts, FT::N)>(
       kentry<D, FORM, tri_row(Ts, FT::N), tri_col(Ts, FT::N)>(
           Gv, std::make_integer_sequence<int, FT::NG>{})),
   ...);
}

template <int D, int FORM, class T, class Sink>
__device__ __forceinline__ void contract(const T* Gv, Sink& sink) {
  contract_seq<D, FORM>(Gv, sink, std::make_integer_sequence<int, FormTraits<D, FORM>::NT>{});
}

// Adjoint of the contraction: Gbar[g] = sum_{i<=j} s_ij K'[g][i][j] where
// s_ii = dA_ii and s_ij = dA_ij + dA_ji (i < j).  sym(t) yields s for the
// linear upper-triangle index t.
template <int D, int FORM, int G, int T, class Sym>
__device__ __forceinline__ void kcolterm(float& acc, const Sym& sym) {
  using FT = FormTraits<D, FORM>;
  constexpr int k = Ref<D, FORM>::K.v[G][tri_row(T, FT::N)][tri_col(T, FT::N)];
  if constexpr (k == 1) {
    acc += sym.template get<T>();
  } else if constexpr (k == -1) {
    acc -= sym.template get<T>();
  } else if constexpr (k != 0) {
    acc = fmaf(sym.template get<T>(), float(k), acc);
  }
}

template <int D, int FORM, int G, class Sym, int... Ts>
__device__ __forceinline__ float kcol(const Sym& sym, std::integer_sequence<int, Ts...>) {
  float acc = 0.f;
  (kcolterm<D, FORM, G, Ts>(acc, sym), ...);
  return acc;
}

template <int D, int FORM, class Sym, int... Gs>
__device__ __forceinline__ void contract_adjoint_seq(const Sym& sym, float* Gbar,
                                                     std::integer_sequence<int, Gs...>) {
  using FT = FormTraits<D, FORM>;
  ((Gbar[Gs] = kcol<D, FORM, Gs>(sym, std::make_integer_sequence<int, FT::NT>{})), ...);
}

template <int D, int FORM, class Sym>
__device__ __forceinline__ void contract_adjoint(const Sym& sym,
                                                 float (&Gbar)[FormTraits<D, FORM>::NG]) {
  contract_adjoint_seq<D, FORM>(sym, Gbar, std::make_integer_sequence<int, FormTraits<D, FORM>::NG>{});
}

// ---------------------------------------------------------------- small helpers

template <class T>
__device__ __forceinline__ T dev_abs(T x) {
  return x < T(0) ? -x : x;
}

}  // namespace fem
