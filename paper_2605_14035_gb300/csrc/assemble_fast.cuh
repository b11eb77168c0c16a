// Element kernels with the quadrature fixed at compile time.
//
// For the usual rules (curves: 3 Gauss points; triangles: 3 points for P1,
// 7 points for P2; tetrahedra: 4 points for P1, 14 points for P2) the whole
// quadrature loop is unrolled and every reference quantity is a compile-time
// offset into a table that travels as a kernel parameter (constant bank), so
// the FP32 multiply-adds read it as an immediate operand: no table loads.
// The tables fold the weight into the basis products (Eqs.
// reference_quadrature_mass, reference_quadrature_stiffness):
//   TM[q][u]     = w_q phi_a(xi_q) phi_b(xi_q)                     (u = (a <= b))
//   TA[q][kk][u] = w_q (d_m phi_a d_n phi_b + d_n phi_a d_m phi_b)  (kk = (m < n))
//                  w_q  d_m phi_a d_m phi_b                         (kk = (m = n))
//   DPSI[q][k][m] = d_m (4 l_i l_j)(xi_q)   (edge bubbles, hierarchical Jacobian)
// so that, with Hh = adj(G) / s (Sec. 3.2, the cofactor form of s G^{-1}),
//   M_u  += s TM,   MC_u += s c_q TM,   A_u += sum_kk Hh_kk TA[kk].
#pragma once

#include "lfem.h"
#include "lfem_internal.cuh"

namespace lfem {

// Quadrature sizes of the compile-time rules.
template <int D, int P>
struct FastQ {
  static constexpr int Q = D == 1 ? 3 : (D == 2 ? (P == 1 ? 3 : 7) : (P == 1 ? 4 : 14));
};

// Per point: DPSI, TM, then for curves TA; triangles and tetrahedra keep the
// reference gradients DPHI[q][b][m] and the weight w_q instead and accumulate
// the stiffness point by point (triangles in a form whose rounding grows with
// sqrt(cond G) rather than cond G; for tetrahedra a product table would also
// outgrow the constant cache).
template <int D, int P>
struct FastLayout {
  static constexpr int Q = FastQ<D, P>::Q;
  static constexpr int REF = Ref<D, P>::REF;
  static constexpr int U = Ref<D, P>::U;
  static constexpr int NE = Ref<D, P>::NE;
  static constexpr int NK = D * (D + 1) / 2;
  static constexpr int PER_Q = NE * D + U + (D >= 2 ? REF * D + 1 : NK * U);
  static constexpr int SIZE = Q * PER_Q;
  static constexpr int dpsi(int q, int k, int m) { return q * PER_Q + k * D + m; }
  static constexpr int tm(int q, int u) { return q * PER_Q + NE * D + u; }
  static constexpr int ta(int q, int kk, int u) { return q * PER_Q + NE * D + U + kk * U + u; }
  static constexpr int dphi(int q, int b, int m) { return q * PER_Q + NE * D + U + b * D + m; }
  static constexpr int w(int q) { return q * PER_Q + NE * D + U + REF * D; }
};

// One table per (D, P) of curves and triangles, at fixed offsets.
struct FastBank {
  static constexpr int OFF11 = 0;
  static constexpr int OFF12 = OFF11 + FastLayout<1, 1>::SIZE;
  static constexpr int OFF21 = OFF12 + FastLayout<1, 2>::SIZE;
  static constexpr int OFF22 = OFF21 + FastLayout<2, 1>::SIZE;
  static constexpr int SIZE = OFF22 + FastLayout<2, 2>::SIZE;
  template <int D, int P>
  static constexpr int off() {
    return D == 1 ? (P == 1 ? OFF11 : OFF12) : (P == 1 ? OFF21 : OFF22);
  }
  float v[SIZE];
};

// Tetrahedra (P1, P2).
struct FastBankTet {
  static constexpr int OFF31 = 0;
  static constexpr int OFF32 = OFF31 + FastLayout<3, 1>::SIZE;
  static constexpr int SIZE = OFF32 + FastLayout<3, 2>::SIZE;
  template <int D, int P>
  static constexpr int off() {
    return P == 1 ? OFF31 : OFF32;
  }
  float v[SIZE];
};

// Host: the table of (dim, order) for rule quad into dst (FastLayout order);
// false if the rule's size is not the compile-time one.
bool fast_tables_host(int dim, int order, const lfem_quad* quad, float* dst);

// a b - c d with one explicit rounding order (the same in every kernel that
// inlines it: implicit multiply-add contraction may differ between contexts)
__device__ __forceinline__ float dif_prod(float a, float b, float c, float d) { return fmaf(a, b, -__fmul_rn(c, d)); }

// Outcome of the per-point tests of one element: good = every |det DF| is
// finite and not numerically zero; cond = the metric passed the conditioning
// threshold (only the stiffness depends on it: mass-type matrices need s only).
struct Checks {
  bool good = true;
  bool cond = true;
};

// Curves: s_q = |t| and Hh_q = 1 / s_q at every point of the compile-time rule
// (the weight sits in the tables); ck.good = false on a zero or non-finite
// length (the element is then redone in double by the caller).
template <int NA, int P, typename Bank>
__device__ __forceinline__ void curve_fast(const ElemData<1, NA, P, float>& ed, const Bank& bank,
                                           float (&sq)[FastLayout<1, P>::Q], float (&hq)[FastLayout<1, P>::Q][1],
                                           Checks& ck) {
  using L = FastLayout<1, P>;
  constexpr int NE = L::NE, Q = L::Q;
  constexpr int OFF = Bank::template off<1, P>();
  const float* tv = bank.v;
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    float t[NA];
#pragma unroll
    for (int i = 0; i < NA; ++i) {
      float acc = ed.e[0][i];
#pragma unroll
      for (int k = 0; k < NE; ++k) acc = fmaf(ed.dl[k][i], tv[OFF + L::dpsi(q, k, 0)], acc);
      t[i] = acc;
    }
    float tt = 0.f;
#pragma unroll
    for (int i = 0; i < NA; ++i) tt = fmaf(t[i], t[i], tt);
    const float inv = rsqrtf(tt);
    sq[q] = tt * inv;
    hq[q][0] = inv;
    ck.good &= (tt > 0.f) & (tt <= 3.0e38f);
  }
}

// Triangles (surface or plane): s_q at every point and, when asked, the
// stiffness accumulated point by point.  With J = Q R (R upper triangular:
// r11 = |t1|, r12 = t1.t2 / r11, r22 = s / r11), grad^T G^{-1} grad =
// |R^{-T} grad|^2, so A_ab += y_a . y_b with
//   y_b = sqrt(w s) R^{-T} grad phi_b = (c1 g_b1, c2 g_b2 - c3 g_b1),
//   c1 = sqrt(w s) / r11, c2 = sqrt(w s) r11 / s, c3 = sqrt(w s) g12 / (r11 s):
// every term of the sum is a product of two well-scaled factors, so rounding
// grows with cond(R) = sqrt(cond G) (the adj(G) form grows with cond G).
template <int NA, int P, typename Bank>
__device__ __forceinline__ void tri_fast(const ElemData<2, NA, P, float>& ed, const Bank& bank, float qthr,
                                         bool do_a, float (&sq)[FastLayout<2, P>::Q], float (&Ao)[Ref<2, P>::U],
                                         Checks& ck) {
  using L = FastLayout<2, P>;
  constexpr int REF = L::REF, NE = L::NE, Q = L::Q, U = L::U;
  constexpr int OFF = Bank::template off<2, P>();
  const float* tv = bank.v;
#pragma unroll
  for (int u = 0; u < U; ++u) Ao[u] = 0.f;
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    float J[NA][2];
#pragma unroll
    for (int i = 0; i < NA; ++i)
#pragma unroll
      for (int m = 0; m < 2; ++m) {
        float acc = ed.e[m][i];
#pragma unroll
        for (int k = 0; k < NE; ++k) acc = fmaf(ed.dl[k][i], tv[OFF + L::dpsi(q, k, m)], acc);
        J[i][m] = acc;
      }
    float g11 = 0.f, g12 = 0.f, g22 = 0.f;
#pragma unroll
    for (int i = 0; i < NA; ++i) {
      g11 = fmaf(J[i][0], J[i][0], g11);
      g12 = fmaf(J[i][0], J[i][1], g12);
      g22 = fmaf(J[i][1], J[i][1], g22);
    }
    float s, s2;
    if constexpr (NA == 2) {
      const float det = dif_prod(J[0][0], J[1][1], J[0][1], J[1][0]);
      s = fabsf(det);
      s2 = __fmul_rn(det, det);
    } else {
      const float n0 = dif_prod(J[1][0], J[2][1], J[2][0], J[1][1]);
      const float n1 = dif_prod(J[2][0], J[0][1], J[0][0], J[2][1]);
      const float n2 = dif_prod(J[0][0], J[1][1], J[1][0], J[0][1]);
      s2 = fmaf(n2, n2, fmaf(n1, n1, __fmul_rn(n0, n0)));
      s = s2 * rsqrtf(s2);
    }
    sq[q] = s;
    // metric quality det G / (tr G / 2)^2 against the threshold, without a division
    const float tr = 0.5f * (g11 + g22);
    ck.good &= (s2 > 1e-12f * (tr * tr)) & (s2 <= 3.0e38f);
    ck.cond &= s2 >= qthr * (tr * tr);
    if (do_a) {
      const float ir11 = rsqrtf(g11);
      const float ws = tv[OFF + L::w(q)] * s;
      const float sws = ws * rsqrtf(ws);
      const float k = __fdividef(sws * ir11, s);
      const float c1 = sws * ir11, c2 = k * g11, c3 = k * g12;
      float y[REF][2];
#pragma unroll
      for (int b = 0; b < REF; ++b) {
        const float gb1 = tv[OFF + L::dphi(q, b, 0)], gb2 = tv[OFF + L::dphi(q, b, 1)];
        y[b][0] = c1 * gb1;
        y[b][1] = fmaf(c2, gb2, -__fmul_rn(c3, gb1));
      }
#pragma unroll
      for (int a = 0; a < REF; ++a)
#pragma unroll
        for (int b = a; b < REF; ++b) {
          const int u = upper_index(REF, a, b);
          Ao[u] = fmaf(y[a][1], y[b][1], fmaf(y[a][0], y[b][0], Ao[u]));
        }
    }
  }
}

// Mass-type matrix from per-point factors f_q (s_q, or s_q c_q):
// V_u = sum_q f_q TM[q][u], written to dst[u].
template <int D, int P, typename Bank>
__device__ __forceinline__ void contract_mass(const Bank& bank, const float (&f)[FastLayout<D, P>::Q], float* dst) {
  using L = FastLayout<D, P>;
  constexpr int OFF = Bank::template off<D, P>();
  const float* tv = bank.v;
#pragma unroll
  for (int u = 0; u < L::U; ++u) {
    float acc = 0.f;
#pragma unroll
    for (int q = 0; q < L::Q; ++q) acc = fmaf(f[q], tv[OFF + L::tm(q, u)], acc);
    dst[u] = acc;
  }
}

// Stiffness: A_u = sum_q sum_kk Hh_q,kk TA[q][kk][u], written to dst[u].
template <int D, int P, typename Bank>
__device__ __forceinline__ void contract_stiff(const Bank& bank,
                                               const float (&hq)[FastLayout<D, P>::Q][FastLayout<D, P>::NK],
                                               float* dst) {
  using L = FastLayout<D, P>;
  constexpr int OFF = Bank::template off<D, P>();
  const float* tv = bank.v;
#pragma unroll
  for (int u = 0; u < L::U; ++u) {
    float acc = 0.f;
#pragma unroll
    for (int q = 0; q < L::Q; ++q)
#pragma unroll
      for (int kk = 0; kk < L::NK; ++kk) acc = fmaf(hq[q][kk], tv[OFF + L::ta(q, kk, u)], acc);
    dst[u] = acc;
  }
}

// Tetrahedra, stiffness point by point: Hw = w_q adj(G) / s from the
// cofactors of J, y_b = Hw grad phi_b, A_ab += grad phi_a . y_b; also the
// conditioning test of every point.
template <int NA, int P, typename Bank>
__device__ __forceinline__ void stiff_tet_fast(const ElemData<3, NA, P, float>& ed, const Bank& bank, float qthr,
                                               float* dst, Checks& ck) {
  using L = FastLayout<3, P>;
  constexpr int REF = L::REF, U = L::U, NE = L::NE, Q = L::Q;
  constexpr int OFF = Bank::template off<3, P>();
  const float* tv = bank.v;
  float Ao[U];
#pragma unroll
  for (int u = 0; u < U; ++u) Ao[u] = 0.f;
  // the point loop stays rolled: unrolled, 14 points of 10 x 10 gradient
  // products outgrow the instruction cache (the table reads are then uniform
  // constant-cache loads)
#pragma unroll 1
  for (int q = 0; q < Q; ++q) {
    float J[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        float acc = ed.e[m][i];
#pragma unroll
        for (int k = 0; k < NE; ++k) acc = fmaf(ed.dl[k][i], tv[OFF + L::dpsi(q, k, m)], acc);
        J[i][m] = acc;
      }
    float c[3][3];
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      const int m1 = (m + 1) % 3, m2 = (m + 2) % 3;
      c[m][0] = dif_prod(J[1][m1], J[2][m2], J[2][m1], J[1][m2]);
      c[m][1] = dif_prod(J[2][m1], J[0][m2], J[0][m1], J[2][m2]);
      c[m][2] = dif_prod(J[0][m1], J[1][m2], J[1][m1], J[0][m2]);
    }
    const float det = fmaf(J[2][0], c[0][2], fmaf(J[1][0], c[0][1], __fmul_rn(J[0][0], c[0][0])));
    const float winv = __fdividef(tv[OFF + L::w(q)], fabsf(det));
    float H[3][3];
#pragma unroll
    for (int m = 0; m < 3; ++m)
#pragma unroll
      for (int n = m; n < 3; ++n)
        H[m][n] = H[n][m] =
            __fmul_rn(fmaf(c[m][2], c[n][2], fmaf(c[m][1], c[n][1], __fmul_rn(c[m][0], c[n][0]))), winv);
    float tr = 0.f;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int m = 0; m < 3; ++m) tr = fmaf(J[i][m], J[i][m], tr);
    tr *= (1.0f / 3.0f);
    const float s2 = __fmul_rn(det, det);
    ck.good &= (s2 > 1e-12f * (tr * tr * tr)) & (s2 <= 3.0e38f);
    ck.cond &= s2 >= qthr * (tr * tr * tr);
#pragma unroll
    for (int b = 0; b < REF; ++b) {
      float y[3];
#pragma unroll
      for (int m = 0; m < 3; ++m)
        y[m] = fmaf(H[m][2], tv[OFF + L::dphi(q, b, 2)],
                    fmaf(H[m][1], tv[OFF + L::dphi(q, b, 1)], __fmul_rn(H[m][0], tv[OFF + L::dphi(q, b, 0)])));
#pragma unroll
      for (int a = 0; a <= b; ++a) {
        const int u = upper_index(REF, a, b);
        float acc = Ao[u];
#pragma unroll
        for (int m = 0; m < 3; ++m) acc = fmaf(tv[OFF + L::dphi(q, a, m)], y[m], acc);
        Ao[u] = acc;
      }
    }
  }
#pragma unroll
  for (int u = 0; u < U; ++u) dst[u] = Ao[u];
}

// Tetrahedra, |det J| at every point (mass-type matrices) and the test.
template <int NA, int P, typename Bank>
__device__ __forceinline__ void jac_tet_fast(const ElemData<3, NA, P, float>& ed, const Bank& bank, float qthr,
                                             float (&sq)[FastLayout<3, P>::Q], Checks& ck) {
  using L = FastLayout<3, P>;
  constexpr int NE = L::NE, Q = L::Q;
  constexpr int OFF = Bank::template off<3, P>();
  const float* tv = bank.v;
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    float J[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        float acc = ed.e[m][i];
#pragma unroll
        for (int k = 0; k < NE; ++k) acc = fmaf(ed.dl[k][i], tv[OFF + L::dpsi(q, k, m)], acc);
        J[i][m] = acc;
      }
    const float c0 = dif_prod(J[1][1], J[2][2], J[2][1], J[1][2]);
    const float c1 = dif_prod(J[2][1], J[0][2], J[0][1], J[2][2]);
    const float c2 = dif_prod(J[0][1], J[1][2], J[1][1], J[0][2]);
    const float det = fmaf(J[2][0], c2, fmaf(J[1][0], c1, __fmul_rn(J[0][0], c0)));
    sq[q] = fabsf(det);
    float tr = 0.f;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int m = 0; m < 3; ++m) tr = fmaf(J[i][m], J[i][m], tr);
    tr *= (1.0f / 3.0f);
    const float s2 = __fmul_rn(det, det);
    ck.good &= (s2 > 1e-12f * (tr * tr * tr)) & (s2 <= 3.0e38f);
    ck.cond &= s2 >= qthr * (tr * tr * tr);
  }
}

// Local matrices of one element with the compile-time rule, stored (upper
// layout, requested matrices in the order M, A, MC): the geometry of every
// point first (a few values per point), then each output entry as one
// contraction with the tables.
template <int D, int NA, int P, typename Bank>
__device__ __forceinline__ void element_fast_store(const ElemData<D, NA, P, float>& ed, const Bank& bank,
                                                   const float* cs, const double* cd, float qthr, unsigned which,
                                                   float* dst, int mstride, Checks& ck) {
  using L = FastLayout<D, P>;
  constexpr int Q = L::Q;
  float cq[Q];
  if (which & LFEM_CMASS) {
#pragma unroll
    for (int q = 0; q < Q; ++q) cq[q] = cs ? __ldg(cs + q) : (float)__ldg(cd + q);
  }
  float sq[Q];
  int slot = 0;
  if constexpr (D == 3) {
    if (which & (LFEM_MASS | LFEM_CMASS)) jac_tet_fast<NA, P>(ed, bank, qthr, sq, ck);
    if (which & LFEM_MASS) contract_mass<D, P>(bank, sq, dst + mstride * slot++);
    if (which & LFEM_STIFF) stiff_tet_fast<NA, P>(ed, bank, qthr, dst + mstride * slot++, ck);
  } else if constexpr (D == 2) {
    float Ao[Ref<D, P>::U];
    const bool do_a = which & LFEM_STIFF;
    tri_fast<NA, P>(ed, bank, qthr, do_a, sq, Ao, ck);
    if (which & LFEM_MASS) contract_mass<D, P>(bank, sq, dst + mstride * slot++);
    if (do_a) {
      float* d = dst + mstride * slot++;
#pragma unroll
      for (int u = 0; u < Ref<D, P>::U; ++u) d[u] = Ao[u];
    }
  } else {
    float hq[Q][L::NK];
    curve_fast<NA, P>(ed, bank, sq, hq, ck);
    if (which & LFEM_MASS) contract_mass<D, P>(bank, sq, dst + mstride * slot++);
    if (which & LFEM_STIFF) contract_stiff<D, P>(bank, hq, dst + mstride * slot++);
  }
  if (which & LFEM_CMASS) {
    float sc[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) sc[q] = sq[q] * cq[q];
    contract_mass<D, P>(bank, sc, dst + mstride * slot);
  }
}

}  // namespace lfem
