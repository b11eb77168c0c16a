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

// Curves and triangles take the packed form: two quadrature points per
// instruction (f32x2 multiply-adds on point pairs (2k, 2k+1)) for the geometry
// and the stiffness, and two upper-triangle entries per instruction for the
// mass-type contractions.  Every table operand is a float pair at an even
// offset of the parameter bank, read as an immediate 64-bit operand.  With an
// odd number of points the last pair is the last point twice with half its
// weight in each half (the sum is unchanged; the mass-type contractions keep
// the original points).
//   DPSI2[k][e][m] = (d_m psi_e(xi_2k), d_m psi_e(xi_2k+1))
//   DPHI2[k][b][m] = (d_m phi_b(xi_2k), d_m phi_b(xi_2k+1))      (triangles)
//   W2[k]          = (w'_2k, w'_2k+1)                             (triangles)
//   TA2[k][u]      = (w'_2k d phi_a d phi_b, ...)                 (curves)
//   TMU[q][j]      = (w_q phi_a phi_b at u = 2j, at u = 2j + 1)   (u = U: 0)
template <int D, int P>
struct FastLayout2 {
  static_assert(D <= 2, "packed tables: curves and triangles");
  static constexpr int Q = FastQ<D, P>::Q;
  static constexpr int QP = (Q + 1) / 2;
  static constexpr int REF = Ref<D, P>::REF;
  static constexpr int U = Ref<D, P>::U;
  static constexpr int UH = (U + 1) / 2;
  static constexpr int NE = Ref<D, P>::NE;
  static constexpr int PER_PAIR = 2 * NE * D + (D == 2 ? 2 * REF * D + 2 : 2 * U);
  static constexpr int MASS0 = QP * PER_PAIR;
  static constexpr int SIZE = MASS0 + 2 * Q * UH;
  // offsets in floats (all even)
  static constexpr int dpsi2(int k, int e, int m) { return k * PER_PAIR + 2 * (e * D + m); }
  static constexpr int dphi2(int k, int b, int m) { return k * PER_PAIR + 2 * NE * D + 2 * (b * D + m); }
  static constexpr int w2(int k) { return k * PER_PAIR + 2 * NE * D + 2 * REF * D; }
  static constexpr int ta2(int k, int u) { return k * PER_PAIR + 2 * NE * D + 2 * u; }
  static constexpr int tmu(int q, int j) { return MASS0 + 2 * (q * UH + j); }
};

// One packed table per (D, P) of curves and triangles, at fixed even offsets.
struct alignas(16) FastBank {
  static constexpr int OFF11 = 0;
  static constexpr int OFF12 = OFF11 + FastLayout2<1, 1>::SIZE;
  static constexpr int OFF21 = OFF12 + FastLayout2<1, 2>::SIZE;
  static constexpr int OFF22 = OFF21 + FastLayout2<2, 1>::SIZE;
  static constexpr int SIZE = OFF22 + FastLayout2<2, 2>::SIZE;
  template <int D, int P>
  static constexpr int off() {
    return D == 1 ? (P == 1 ? OFF11 : OFF12) : (P == 1 ? OFF21 : OFF22);
  }
  float v[SIZE];
};
static_assert(FastBank::OFF12 % 2 == 0 && FastBank::OFF21 % 2 == 0 && FastBank::OFF22 % 2 == 0, "even offsets");

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

// Host: the table of (dim, order) for rule quad into dst (FastLayout2 order
// for curves and triangles, FastLayout for tetrahedra); false if the rule's
// size is not the compile-time one.
bool fast_tables_host(int dim, int order, const lfem_quad* quad, float* dst);
// Floats of that table.
int fast_table_size(int dim, int order);

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

// ---- packed (f32x2) helpers --------------------------------------------------
__device__ __forceinline__ float2 f2(float x) { return make_float2(x, x); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
// a b - c d per half, rounded as dif_prod
__device__ __forceinline__ float2 dif_prod2(float2 a, float2 b, float2 c, float2 d) {
  const float2 cd = __fmul2_rn(c, d);
  return __ffma2_rn(a, b, make_float2(-cd.x, -cd.y));
}
template <int OFF>
__device__ __forceinline__ float2 tab2(const float* v, int off) {
  return reinterpret_cast<const float2*>(v + OFF)[off >> 1];
}

// Curves, two points per instruction: s_q = |t| at every point of the rule and
// the stiffness A_u = sum_q (1 / s_q) TA[q][u] (the weight in the table);
// ck.good = false on a zero or non-finite length (the element is then redone
// in double by the caller).
template <int NA, int P, typename Bank>
__device__ __forceinline__ void curve_fast2(const ElemData<1, NA, P, float>& ed, const Bank& bank, bool do_a,
                                            float (&sq)[FastLayout2<1, P>::Q], float (&Ao)[lsm_stride(Ref<1, P>::U)],
                                            Checks& ck) {
  using L = FastLayout2<1, P>;
  constexpr int NE = L::NE, Q = L::Q, U = L::U;
  constexpr int OFF = Bank::template off<1, P>();
  const float* tv = bank.v;
  float2 A2[U];
#pragma unroll
  for (int u = 0; u < U; ++u) A2[u] = f2(0.f);
#pragma unroll
  for (int k = 0; k < L::QP; ++k) {
    float2 tt = f2(0.f);
#pragma unroll
    for (int i = 0; i < NA; ++i) {
      float2 t = f2(ed.e[0][i]);
#pragma unroll
      for (int e = 0; e < NE; ++e) t = fma2(f2(ed.dl[e][i]), tab2<OFF>(tv, L::dpsi2(k, e, 0)), t);
      tt = fma2(t, t, tt);
    }
    const float2 inv = make_float2(rsqrtf(tt.x), rsqrtf(tt.y));
    const float2 sv = mul2(tt, inv);
    sq[2 * k] = sv.x;
    if (2 * k + 1 < Q) sq[2 * k + 1] = sv.y;
    ck.good &= (tt.x > 0.f) & (tt.x <= 3.0e38f) & (tt.y > 0.f) & (tt.y <= 3.0e38f);
    if (do_a) {
#pragma unroll
      for (int u = 0; u < U; ++u) A2[u] = fma2(inv, tab2<OFF>(tv, L::ta2(k, u)), A2[u]);
    }
  }
#pragma unroll
  for (int u = 0; u < U; ++u) Ao[u] = A2[u].x + A2[u].y;
  if constexpr (U & 1) Ao[U] = 0.f;
}

// Triangles (surface or plane), two points per instruction: s_q at every
// point and, when asked, the stiffness accumulated point pair by point pair.
// With J = Q R (R upper triangular: r11 = |t1|, r12 = t1.t2 / r11,
// r22 = s / r11), grad^T G^{-1} grad = |R^{-T} grad|^2, so A_ab += y_a . y_b with
//   y_b = sqrt(w s) R^{-T} grad phi_b = (c1 g_b1, c2 g_b2 - c3 g_b1),
//   c1 = sqrt(w s) / r11, c2 = sqrt(w s) r11 / s, c3 = sqrt(w s) g12 / (r11 s):
// every term of the sum is a product of two well-scaled factors, so rounding
// grows with cond(R) = sqrt(cond G) (the adj(G) form grows with cond G).
template <int NA, int P, typename Bank>
__device__ __forceinline__ void tri_fast2(const ElemData<2, NA, P, float>& ed, const Bank& bank, float qthr,
                                          bool do_a, float (&sq)[FastLayout2<2, P>::Q],
                                          float (&Ao)[lsm_stride(Ref<2, P>::U)], Checks& ck) {
  using L = FastLayout2<2, P>;
  constexpr int REF = L::REF, NE = L::NE, Q = L::Q, U = L::U;
  constexpr int OFF = Bank::template off<2, P>();
  const float* tv = bank.v;
  float2 A2[U];
#pragma unroll
  for (int u = 0; u < U; ++u) A2[u] = f2(0.f);
  bool good = true, cond = true;
#pragma unroll
  for (int k = 0; k < L::QP; ++k) {
    float2 J[NA][2];
#pragma unroll
    for (int i = 0; i < NA; ++i)
#pragma unroll
      for (int m = 0; m < 2; ++m) {
        float2 acc = f2(ed.e[m][i]);
#pragma unroll
        for (int e = 0; e < NE; ++e) acc = fma2(f2(ed.dl[e][i]), tab2<OFF>(tv, L::dpsi2(k, e, m)), acc);
        J[i][m] = acc;
      }
    float2 g11 = mul2(J[0][0], J[0][0]), g12 = mul2(J[0][0], J[0][1]), g22 = mul2(J[0][1], J[0][1]);
#pragma unroll
    for (int i = 1; i < NA; ++i) {
      g11 = fma2(J[i][0], J[i][0], g11);
      g12 = fma2(J[i][0], J[i][1], g12);
      g22 = fma2(J[i][1], J[i][1], g22);
    }
    float2 s, s2;
    if constexpr (NA == 2) {
      const float2 det = dif_prod2(J[0][0], J[1][1], J[0][1], J[1][0]);
      s = make_float2(fabsf(det.x), fabsf(det.y));
      s2 = mul2(det, det);
    } else {
      const float2 n0 = dif_prod2(J[1][0], J[2][1], J[2][0], J[1][1]);
      const float2 n1 = dif_prod2(J[2][0], J[0][1], J[0][0], J[2][1]);
      const float2 n2 = dif_prod2(J[0][0], J[1][1], J[1][0], J[0][1]);
      s2 = fma2(n2, n2, fma2(n1, n1, mul2(n0, n0)));
      s = mul2(s2, make_float2(rsqrtf(s2.x), rsqrtf(s2.y)));
    }
    sq[2 * k] = s.x;
    if (2 * k + 1 < Q) sq[2 * k + 1] = s.y;
    // metric quality det G / (tr G / 2)^2 against the threshold, without a division
    const float2 tr = mul2(f2(0.5f), add2(g11, g22));
    const float2 tr2 = mul2(tr, tr);
    const float2 lo = mul2(f2(1e-12f), tr2), th = mul2(f2(qthr), tr2);
    good &= (s2.x > lo.x) & (s2.x <= 3.0e38f) & (s2.y > lo.y) & (s2.y <= 3.0e38f);
    cond &= (s2.x >= th.x) & (s2.y >= th.y);
    if (do_a) {
      const float2 ws = mul2(tab2<OFF>(tv, L::w2(k)), s);
      const float2 sws = mul2(ws, make_float2(rsqrtf(ws.x), rsqrtf(ws.y)));
      const float2 c1 = mul2(sws, make_float2(rsqrtf(g11.x), rsqrtf(g11.y)));
      const float2 kk = mul2(c1, make_float2(__fdividef(1.0f, s.x), __fdividef(1.0f, s.y)));
      const float2 c2 = mul2(kk, g11), c3 = mul2(kk, g12);
      const float2 nc3 = make_float2(-c3.x, -c3.y);
      float2 y0[REF], y1[REF];
#pragma unroll
      for (int b = 0; b < REF; ++b) {
        const float2 gb1 = tab2<OFF>(tv, L::dphi2(k, b, 0)), gb2 = tab2<OFF>(tv, L::dphi2(k, b, 1));
        y0[b] = mul2(c1, gb1);
        y1[b] = fma2(c2, gb2, mul2(nc3, gb1));
      }
#pragma unroll
      for (int a = 0; a < REF; ++a)
#pragma unroll
        for (int b = a; b < REF; ++b) {
          const int u = upper_index(REF, a, b);
          A2[u] = fma2(y1[a], y1[b], fma2(y0[a], y0[b], A2[u]));
        }
    }
  }
  ck.good &= good;
  ck.cond &= cond;
#pragma unroll
  for (int u = 0; u < U; ++u) Ao[u] = A2[u].x + A2[u].y;
  if constexpr (U & 1) Ao[U] = 0.f;
}

// Mass-type matrix of a curve or triangle from per-point factors f_q (s_q, or
// s_q c_q), two entries per instruction: V_u = sum_q f_q TM[q][u], written as
// float pairs (entries 2j, 2j + 1) to dst[6 j] (the tile's interleaved
// local-matrix layout, dst already offset to the matrix slot; the pad entry
// of an odd U is 0).
template <int D, int P, typename Bank>
__device__ __forceinline__ void contract_mass2(const Bank& bank, const float (&f)[FastLayout2<D, P>::Q], float* dst) {
  using L = FastLayout2<D, P>;
  constexpr int OFF = Bank::template off<D, P>();
  const float* tv = bank.v;
#pragma unroll
  for (int j = 0; j < L::UH; ++j) {
    float2 acc = mul2(f2(f[0]), tab2<OFF>(tv, L::tmu(0, j)));
#pragma unroll
    for (int q = 1; q < L::Q; ++q) acc = fma2(f2(f[q]), tab2<OFF>(tv, L::tmu(q, j)), acc);
    *reinterpret_cast<float2*>(dst + 6 * j) = acc;
  }
}

// Local matrices of one curve or triangle with the compile-time rule, stored
// into the element's block of the interleaved layout (dst = element base,
// 8-byte aligned; matrix slots in the order M, A, MC of the requested ones).
template <int D, int NA, int P, typename Bank>
__device__ __forceinline__ void element_fast_store2(const ElemData<D, NA, P, float>& ed, const Bank& bank,
                                                    const float* cs, const double* cd, float qthr, unsigned which,
                                                    float* dst, Checks& ck) {
  using L = FastLayout2<D, P>;
  constexpr int Q = L::Q, UP = lsm_stride(L::U);
  float cq[Q];
  if (which & LFEM_CMASS) {
#pragma unroll
    for (int q = 0; q < Q; ++q) cq[q] = cs ? __ldg(cs + q) : (float)__ldg(cd + q);
  }
  float sq[Q];
  float Ao[UP];
  const bool do_a = which & LFEM_STIFF;
  if constexpr (D == 2) tri_fast2<NA, P>(ed, bank, qthr, do_a, sq, Ao, ck);
  else curve_fast2<NA, P>(ed, bank, do_a, sq, Ao, ck);
  int slot = 0;
  if (which & LFEM_MASS) contract_mass2<D, P>(bank, sq, dst + 2 * slot++);
  if (do_a) {
    float* d = dst + 2 * slot++;
#pragma unroll
    for (int j = 0; j < UP / 2; ++j) *reinterpret_cast<float2*>(d + 6 * j) = make_float2(Ao[2 * j], Ao[2 * j + 1]);
  }
  if (which & LFEM_CMASS) {
    float sc[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) sc[q] = sq[q] * cq[q];
    contract_mass2<D, P>(bank, sc, dst + 2 * slot);
  }
}

// Mass-type matrix of a tetrahedron from per-point factors f_q (s_q, or
// s_q c_q): V_u = sum_q f_q TM[q][u], written to dst[u].
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

// Local matrices of one tetrahedron with the compile-time rule, stored (upper
// layout, requested matrices in the order M, A, MC): the geometry of every
// point first (a few values per point), then each output entry as one
// contraction with the tables.
template <int D, int NA, int P, typename Bank>
__device__ __forceinline__ void element_fast_store(const ElemData<D, NA, P, float>& ed, const Bank& bank,
                                                   const float* cs, const double* cd, float qthr, unsigned which,
                                                   float* dst, int mstride, Checks& ck) {
  static_assert(D == 3, "curves and triangles: element_fast_store2");
  using L = FastLayout<D, P>;
  constexpr int Q = L::Q;
  float cq[Q];
  if (which & LFEM_CMASS) {
#pragma unroll
    for (int q = 0; q < Q; ++q) cq[q] = cs ? __ldg(cs + q) : (float)__ldg(cd + q);
  }
  float sq[Q];
  int slot = 0;
  if (which & (LFEM_MASS | LFEM_CMASS)) jac_tet_fast<NA, P>(ed, bank, qthr, sq, ck);
  if (which & LFEM_MASS) contract_mass<D, P>(bank, sq, dst + mstride * slot++);
  if (which & LFEM_STIFF) stiff_tet_fast<NA, P>(ed, bank, qthr, dst + mstride * slot++, ck);
  if (which & LFEM_CMASS) {
    float sc[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) sc[q] = sq[q] * cq[q];
    contract_mass<D, P>(bank, sc, dst + mstride * slot);
  }
}

}  // namespace lfem
