// fem_forms.cuh -- reference (analytic) tensors K of the weak forms, built at
// compile time in exact integer arithmetic.
//
// Knepley & Terrel, Sec. 3: the element tensor is the contraction
// A^{ij} = G^{mu nu} K^{ij}_{mu nu} (Eq. 1, Eq. 6), where K depends only on
// the form and the reference element (Eq. 7) and can be computed a priori
// (end of Sec. 3.1).  Here K is generated by constexpr C++ from the basis
// written in barycentric coordinates, so the CUDA kernels see every entry as
// an immediate and skip the zero entries at compile time (sparse contraction
// with no index arrays).
//
// Forms (ids match the C ABI):
//   LAPLACE_P1 / LAPLACE_P2 : K^{ij}_{mu nu} = int_ref d_mu phi_i d_nu phi_j     (Eq. 7)
//   ELASTIC_P1 : eps(v):eps(u), i.e. Eq. 10 scaled by the 1/4 of Eq. 14.  With the
//     symmetric gradient the geometric tensor needs both spatial indices,
//     G^{(mu a),(nu b)} = |J| Jinv_{mu a} Jinv_{nu b}, and
//     K^{(c,i),(c',j)}_{(mu a),(nu b)} = Kref^{ij}_{mu nu} (d_{cc'} d_{ab} + d_{a c'} d_{b c}) / 2
//     (reading of Eqs. 9-15: Eq. 15's d x d G as printed would give the vector
//     Laplacian, which does not vanish on rigid rotations).
//
// Folding: G is symmetric under (p <-> q) for p, q its two index slots, so only
// the pairs p <= q are kept (d(d+1)/2 Laplacian entries, d^2(d^2+1)/2 elasticity
// entries); K is folded to K'_{pq} = K_{pq} + K_{qp} (p < q).  The folded K' is
// symmetric in (i, j), so A is symmetric and only i <= j is computed.
//
//   LAPLACE_P1_W1 / LAPLACE_P2_W1 : the Laplacian with a P1 coefficient
//     w = sum_k w_k lambda_k given by its vertex values (Eqs. 20-23): the
//     reference tensor gains the coefficient's index,
//     K^{ij k}_{mu nu} = int_ref lambda_k d_mu phi_i d_nu phi_j   (Eq. 21),
//     and the geometric tensor becomes w_k G^{mu nu} (Eq. 22), so the
//     contraction runs over (d+1) x d(d+1)/2 slots, slot k * NGB + g.
//
//   LAPLACE_P1_ISO / LAPLACE_P2_ISO : the Laplacian on non-affine elements
//     (Eqs. 16-19): J^{-1} is projected onto P1 by its vertex values, so G
//     gains the vertex indices, G^{(k mu),(l nu)} = |J| J^{-1}_{mu a,k} J^{-1}_{nu a,l},
//     and K^{ij}_{(k mu),(l nu)} = int_ref lambda_k lambda_l d_mu phi_i d_nu phi_j;
//     the slot (k mu) ranges over (d+1) d values and G is folded over the
//     symmetric pairs of slots like elasticity's.
//
// Integer scaling: every entry is stored as K' * DEN with DEN = (d+2)! (twice
// that for elasticity; (d+3)! for the P1-coefficient forms and (d+4)! for the
// non-affine forms, whose integrands have one or two more linear factors),
// using  int_ref lambda^a = a! / (|a| + d)!.
#pragma once
#include <cstdint>

namespace fem {

enum FormId : int {
  LAPLACE_P1 = 0,
  LAPLACE_P2 = 1,
  ELASTIC_P1 = 2,
  LAPLACE_P1_W1 = 3,
  LAPLACE_P2_W1 = 4,
  LAPLACE_P1_ISO = 5,
  LAPLACE_P2_ISO = 6,
  DIV_P1P1 = 7,  // coupling block int q div v, q in P1, v in [P1]^d
  DIV_P2P1 = 8   // the same with v in [P2]^d (the Taylor-Hood pair)
};

template <int D, int FORM>
struct FormTraits {
  static_assert(D == 2 || D == 3, "dimension");
  static constexpr bool W1 = FORM == LAPLACE_P1_W1 || FORM == LAPLACE_P2_W1;     // P1 coefficient
  static constexpr bool ISO = FORM == LAPLACE_P1_ISO || FORM == LAPLACE_P2_ISO;  // non-affine elements
  static constexpr int BASE = (FORM == LAPLACE_P1_W1 || FORM == LAPLACE_P1_ISO)   ? LAPLACE_P1
                              : (FORM == LAPLACE_P2_W1 || FORM == LAPLACE_P2_ISO) ? LAPLACE_P2
                                                                                  : FORM;
  static constexpr int NV = D + 1;                                // vertices
  static constexpr int DEG = BASE == LAPLACE_P2 ? 2 : 1;
  static constexpr int NB = DEG == 1 ? D + 1 : (D + 1) * (D + 2) / 2;  // scalar basis
  static constexpr int NC = FORM == ELASTIC_P1 ? D : 1;           // components
  static constexpr int N = NB * NC;                               // rows of A_e
  static constexpr int NN = N * N;
  static constexpr int NP = FORM == ELASTIC_P1 ? D * D : ISO ? (D + 1) * D : D;  // range of one G slot
  static constexpr int NGB = NP * (NP + 1) / 2;                   // folded G entries of the base form
  static constexpr int NW = W1 ? NV : 1;                          // coefficient values per element
  static constexpr int NG = NW * NGB;                             // contraction slots
  static constexpr int NT = N * (N + 1) / 2;                      // unique A entries
  static constexpr int DEN = ISO ? (D == 2 ? 720 : 5040)
                             : W1 ? (D == 2 ? 120 : 720) : (D == 2 ? 24 : 120) * (FORM == ELASTIC_P1 ? 2 : 1);
};

// index of the pair (p, q), p <= q, in row-major upper-triangle order
constexpr int pair_index(int p, int q, int np) { return p * np - p * (p - 1) / 2 + (q - p); }
constexpr int tri_row(int t, int n) {
  int i = 0;
  while (t >= n - i) { t -= n - i; ++i; }
  return i;
}
constexpr int tri_col(int t, int n) {
  int i = 0;
  while (t >= n - i) { t -= n - i; ++i; }
  return i + t;
}

// d lambda_k / d xi_mu on the reference simplex (lambda_0 = 1 - sum xi, lambda_k = xi_k)
constexpr int dlam(int k, int mu) { return k == 0 ? -1 : (k - 1 == mu ? 1 : 0); }

// d_mu phi_i as a linear polynomial c0 + sum_m c[m] lambda_m (integer coefficients)
struct Lin {
  int c0;
  int c[4];
};

template <int D, int DEG>
constexpr Lin basis_deriv(int i, int mu) {
  Lin r{0, {0, 0, 0, 0}};
  if (DEG == 1) {
    r.c0 = dlam(i, mu);
    return r;
  }
  if (i <= D) {  // vertex function lambda_i (2 lambda_i - 1): derivative (4 lambda_i - 1) dlam_i
    r.c[i] = 4 * dlam(i, mu);
    r.c0 = -dlam(i, mu);
    return r;
  }
  int t = i - (D + 1);  // edge functions 4 lambda_a lambda_b, a < b lexicographic
  for (int a = 0; a <= D; ++a)
    for (int b = a + 1; b <= D; ++b) {
      if (t == 0) {
        r.c[b] += 4 * dlam(a, mu);
        r.c[a] += 4 * dlam(b, mu);
        return r;
      }
      --t;
    }
  return r;
}

// (d+2)! * int_ref (p)(q) dxi for two linear polynomials in the barycentrics
template <int D>
constexpr int integrate_lin_lin(const Lin& p, const Lin& q) {
  int s = p.c0 * q.c0 * (D + 1) * (D + 2);
  int sp = 0, sq = 0;
  for (int m = 0; m <= D; ++m) { sp += p.c[m]; sq += q.c[m]; }
  s += (p.c0 * sq + q.c0 * sp) * (D + 2);
  for (int m = 0; m <= D; ++m)
    for (int n = 0; n <= D; ++n) s += p.c[m] * q.c[n] * (m == n ? 2 : 1);
  return s;
}

// (d+3)! * int_ref lambda_k (p)(q) dxi.  Each linear polynomial is made
// homogeneous (c0 = c0 sum_m lambda_m), and (d+3)! int_ref lambda_a lambda_b
// lambda_c = a!b!c!-style multiplicity: 6 when a = b = c, 2 when exactly two
// indices agree, 1 otherwise.
template <int D>
constexpr int integrate_lam_lin_lin(int k, const Lin& p, const Lin& q) {
  int s = 0;
  for (int a = 0; a <= D; ++a)
    for (int b = 0; b <= D; ++b) {
      const int pa = p.c[a] + p.c0, qb = q.c[b] + q.c0;
      if (pa == 0 || qb == 0) continue;
      const int m = (a == k && b == k) ? 6 : (a == k || b == k || a == b) ? 2 : 1;
      s += pa * qb * m;
    }
  return s;
}

// (d+4)! * int_ref lambda_k lambda_l (p)(q) dxi: four homogeneous linear
// factors; (d+4)! int_ref of a degree-4 monomial is the product of the
// factorials of its exponents.
template <int D>
constexpr int integrate_lam2_lin_lin(int k, int l, const Lin& p, const Lin& q) {
  int s = 0;
  for (int a = 0; a <= D; ++a)
    for (int b = 0; b <= D; ++b) {
      const int pa = p.c[a] + p.c0, qb = q.c[b] + q.c0;
      if (pa == 0 || qb == 0) continue;
      int cnt[4] = {0, 0, 0, 0};
      ++cnt[k];
      ++cnt[l];
      ++cnt[a];
      ++cnt[b];
      int m = 1;
      for (int t = 0; t <= D; ++t)
        for (int f = 2; f <= cnt[t]; ++f) m *= f;
      s += pa * qb * m;
    }
  return s;
}

template <int D, int FORM>
struct RefTensor {
  using T = FormTraits<D, FORM>;
  int v[T::NG][T::N][T::N];  // K' * DEN, folded
};

template <int D, int FORM>
constexpr RefTensor<D, FORM> make_ref_tensor() {
  using T = FormTraits<D, FORM>;
  RefTensor<D, FORM> r{};
  // scalar Laplacian tensor Kref[mu][nu][i][j] * (d+2)!
  int kref[D][D][T::NB][T::NB] = {};
  for (int mu = 0; mu < D; ++mu)
    for (int nu = 0; nu < D; ++nu)
      for (int i = 0; i < T::NB; ++i)
        for (int j = 0; j < T::NB; ++j)
          kref[mu][nu][i][j] = integrate_lin_lin<D>(basis_deriv<D, T::DEG>(i, mu),
                                                    basis_deriv<D, T::DEG>(j, nu));
  if constexpr (T::ISO) {
    // slot p = k * D + mu; folded over p <= q
    for (int pp = 0; pp < T::NP; ++pp)
      for (int qq = pp; qq < T::NP; ++qq) {
        const int g = pair_index(pp, qq, T::NP);
        const int k = pp / D, mu = pp % D, l = qq / D, nu = qq % D;
        for (int i = 0; i < T::NB; ++i)
          for (int j = 0; j < T::NB; ++j) {
            int v = integrate_lam2_lin_lin<D>(k, l, basis_deriv<D, T::DEG>(i, mu), basis_deriv<D, T::DEG>(j, nu));
            if (pp != qq)
              v += integrate_lam2_lin_lin<D>(l, k, basis_deriv<D, T::DEG>(i, nu), basis_deriv<D, T::DEG>(j, mu));
            r.v[g][i][j] = v;
          }
      }
  } else if constexpr (T::W1) {
    for (int k = 0; k <= D; ++k)
      for (int mu = 0; mu < D; ++mu)
        for (int nu = mu; nu < D; ++nu) {
          int g = k * T::NGB + pair_index(mu, nu, D);
          for (int i = 0; i < T::NB; ++i)
            for (int j = 0; j < T::NB; ++j) {
              const Lin di = basis_deriv<D, T::DEG>(i, mu), dj = basis_deriv<D, T::DEG>(j, nu);
              int v = integrate_lam_lin_lin<D>(k, di, dj);
              if (mu != nu)
                v += integrate_lam_lin_lin<D>(k, basis_deriv<D, T::DEG>(i, nu), basis_deriv<D, T::DEG>(j, mu));
              r.v[g][i][j] = v;
            }
        }
  } else if constexpr (FORM != ELASTIC_P1) {
    for (int mu = 0; mu < D; ++mu)
      for (int nu = mu; nu < D; ++nu) {
        int g = pair_index(mu, nu, D);
        for (int i = 0; i < T::NB; ++i)
          for (int j = 0; j < T::NB; ++j)
            r.v[g][i][j] = kref[mu][nu][i][j] + (mu != nu ? kref[nu][mu][i][j] : 0);
      }
  } else {
    // unfolded K_{(mu a),(nu b)}^{(c,i),(c',j)} * 2 (d+2)! = Kref * (d_cc' d_ab + d_ac' d_bc)
    for (int p = 0; p < T::NP; ++p)
      for (int q = p; q < T::NP; ++q) {
        int g = pair_index(p, q, T::NP);
        for (int I = 0; I < T::N; ++I)
          for (int J = 0; J < T::N; ++J) {
            int c = I / T::NB, i = I % T::NB, cp = J / T::NB, j = J % T::NB;
            auto term = [&](int pp, int qq) {
              int mu = pp / D, a = pp % D, nu = qq / D, b = qq % D;
              int w = (c == cp && a == b ? 1 : 0) + (a == cp && b == c ? 1 : 0);
              return kref[mu][nu][i][j] * w;
            };
            r.v[g][I][J] = term(p, q) + (p != q ? term(q, p) : 0);
          }
      }
  }
  return r;
}

template <int D, int FORM>
struct Ref {
  static constexpr RefTensor<D, FORM> K = make_ref_tensor<D, FORM>();
};

// ---------------------------------------------------------------- coupling blocks
// The off-diagonal block of a multiphysics pair (a scalar field q in P1 and a
// vector field v in [P_VDEG]^d), B = int w q div v:
//   B_{i,(c,j)} = int_T w phi_i d psi_j / d x_c = sum_mu G^{mu c} K^{ij}_mu
//   G^{mu c}    = w |J| J^{-1}_{mu c} = w sgn(det J) adj(J)_{mu c}
//   K^{ij}_mu   = int_ref lambda_i d_mu psi_j
// (Eq. 1 with one basis-function value and one derivative in K, as Sec. 3.1
// allows for any multilinear form).  Rows i = 0..d, columns c * NBV + j
// (component-major).  G needs no division by det J: only its sign.  K is
// stored scaled by DEN = (d+2)! as exact integers.
template <int D, int VDEG>
struct DivTraits {
  static_assert(D == 2 || D == 3, "dimension");
  static constexpr int NQ = D + 1;                                    // rows (P1 scalar basis)
  static constexpr int NBV = VDEG == 1 ? D + 1 : (D + 1) * (D + 2) / 2;  // basis of one component
  static constexpr int NCOL = D * NBV;
  static constexpr int NN = NQ * NCOL;
  static constexpr int NG = D * D;                                    // G slots g = mu * D + c
  static constexpr int DEN = D == 2 ? 24 : 120;
};

template <int D, int VDEG>
struct DivRefTensor {
  int v[D][D + 1][DivTraits<D, VDEG>::NBV];  // K^{ij}_mu * DEN
};

template <int D, int VDEG>
constexpr DivRefTensor<D, VDEG> make_div_ref() {
  DivRefTensor<D, VDEG> r{};
  for (int mu = 0; mu < D; ++mu)
    for (int i = 0; i <= D; ++i) {
      Lin li{0, {0, 0, 0, 0}};
      li.c[i] = 1;
      for (int j = 0; j < DivTraits<D, VDEG>::NBV; ++j)
        r.v[mu][i][j] = integrate_lin_lin<D>(li, basis_deriv<D, VDEG>(j, mu));
    }
  return r;
}

template <int D, int VDEG>
struct DivRef {
  static constexpr DivRefTensor<D, VDEG> K = make_div_ref<D, VDEG>();
};

}  // namespace fem
