// Element-level building blocks of the assembly (geometry per quadrature
// point and local upper-triangle matrices, Sec. 3.2.1-3.2.2; Eqs.
// reference_quadrature_mass / _stiffness), the compensated accumulator, and
// the element-stage kernels (physical points, geometry, local matrices).
#pragma once

#include <cstdio>

#include "lfem_internal.cuh"

namespace lfem {

struct AsmArgs {
  const int32_t* conn;
  const double* coords;
  const void* coef;
  int coef_f32;
  const int64_t* row_ptr;
  const int32_t* inc_ptr;
  const uint8_t* inc_pos;
  const uint16_t* inc_local;
  const int32_t* tile_row0;
  const int32_t* tile_elem_ptr;
  const int32_t* tile_elem;
  void* out[3];        // outputs in accumulator order
  int nm;              // number of requested matrices
  int mat[3];          // matrix kind (0 = M, 1 = A, 2 = MC) of accumulator slot m
  unsigned which;
  TabRef tab;
  int chunk;           // elements per chunk
  int slots_cap;       // tile slot capacity
  float qmin;          // metric quality below which a mixed element is redone in double
  int32_t* status;
  unsigned long long* fallback;
  int64_t tile_begin;  // first tile of this launch
};

template <typename R>
struct AccOf;
template <>
struct AccOf<float> {
  using T = float2;
};
template <>
struct AccOf<double> {
  using T = double;
};

__device__ __forceinline__ void acc_zero(float2& a) { a = make_float2(0.f, 0.f); }
__device__ __forceinline__ void acc_zero(double& a) { a = 0.0; }
// Kahan-compensated float sum: (sum, compensation).
__device__ __forceinline__ void acc_add(float2& a, float v) {
  float y = v - a.y;
  float t = a.x + y;
  a.y = (t - a.x) - y;
  a.x = t;
}
__device__ __forceinline__ void acc_add(double& a, double v) { a += v; }
__device__ __forceinline__ void acc_init(float2& a, float v) { a = make_float2(v, 0.f); }
__device__ __forceinline__ void acc_init(double& a, double v) { a = v; }
__device__ __forceinline__ float acc_final(const float2& a) { return a.x - a.y; }
__device__ __forceinline__ double acc_final(const double& a) { return a; }

template <typename T>
__device__ __forceinline__ T load_coef(const void* p, int f32, int64_t i) {
  return f32 ? (T)__ldg((const float*)p + i) : (T)__ldg((const double*)p + i);
}

// Local matrices of one element in precision R; returns the minimum metric
// quality and whether a quadrature point had s = 0 or a non-finite s.
template <int D, int NA, int P, typename R, bool DM, bool DA, bool DC>
__device__ __forceinline__ void element_pass(const ElemData<D, NA, P, R>& ed, const TabView<R>& tb, const void* coef,
                                             int coef_f32, int64_t e, R (&Mo)[Ref<D, P>::U],
                                             R (&Ao)[Ref<D, P>::U], R (&Co)[Ref<D, P>::U], R& qual, bool& bad) {
  constexpr int U = Ref<D, P>::U;
#pragma unroll
  for (int u = 0; u < U; ++u) {
    if (DM) Mo[u] = 0;
    if (DA) Ao[u] = 0;
    if (DC) Co[u] = 0;
  }
#pragma unroll 1
  for (int q = 0; q < tb.q; ++q) {
    const R wq = tb.w[q];
    QpGeom<D, NA, P, R> g;
    qp_geometry<D, NA, P, R>(ed, tb, q, wq, g);
    qual = fmin(qual, g.quality);
    // numerically zero |det DF|: metric quality det G / (tr G / D)^D at rounding level
    bad |= !(g.s > (R)0) || !isfinite(g.s) || !(g.quality > (sizeof(R) == 8 ? (R)1e-28 : (R)1e-12));
    R cq = 0;
    if (DC) cq = load_coef<R>(coef, coef_f32, e * tb.q + q);
    qp_accumulate<D, NA, P, R, DM, DA, DC>(g, tb, q, wq, cq, Mo, Ao, Co);
  }
}

// Float pair (hi, lo) with hi + lo = x to ~2^-47 relative, from integer
// operations on the bits of x (no FP64 instruction: on GB300 the FP64 pipe
// runs at 1/64 of the FP32 rate).  hi = x truncated to 24 significant bits
// (so differences of nearby hi values are exact), lo = the next 23 bits.
// |x| >= 2^128 sets ok = false (the element is redone in double); |x| < 2^-103
// keeps only hi, |x| < 2^-126 maps to 0.
__device__ __forceinline__ void split_f64(double x, float& hi, float& lo, bool& ok) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const uint32_t hw = (uint32_t)(u >> 32), lw = (uint32_t)u;
  const uint32_t E = (hw >> 20) & 0x7FFu;
  const uint32_t sign = hw & 0x80000000u;
  const uint32_t hadj = (hw & 0x7FFFFFFFu) - (896u << 20);
  const uint32_t hbits = sign | __funnelshift_l(lw, hadj, 3);
  const uint32_t ef = (E - 919u) << 23;
  const float lo_mag = __uint_as_float(ef | ((lw >> 6) & 0x7FFFFFu)) - __uint_as_float(ef);
  hi = E >= 897u ? __uint_as_float(hbits) : 0.0f;
  lo = E >= 920u ? __uint_as_float(__float_as_uint(lo_mag) ^ sign) : 0.0f;
  ok = ok && (E <= 1150u);
}

// Element data in float from the split coordinates: corner edge vectors and
// edge-node deviations, each a difference of nearby values done on the hi
// parts (exact) plus the lo parts.
template <int D, int NA, int P>
__device__ __forceinline__ bool load_element_data_split(const double* __restrict__ coords,
                                                        const int32_t (&nodes)[Ref<D, P>::REF],
                                                        ElemData<D, NA, P, float>& ed) {
  constexpr int REF = Ref<D, P>::REF;
  float xh[REF][NA], xl[REF][NA];
  bool ok = true;
#pragma unroll
  for (int b = 0; b < REF; ++b) {
    const double* p = coords + (int64_t)nodes[b] * NA;
#pragma unroll
    for (int i = 0; i < NA; ++i) split_f64(__ldg(p + i), xh[b][i], xl[b][i], ok);
  }
#pragma unroll
  for (int m = 0; m < D; ++m)
#pragma unroll
    for (int i = 0; i < NA; ++i) ed.e[m][i] = (xh[m + 1][i] - xh[0][i]) + (xl[m + 1][i] - xl[0][i]);
#pragma unroll
  for (int k = 0; k < Ref<D, P>::NE; ++k) {
    const int I = edge_i<D>(k), J = edge_j<D>(k), Ed = D + 1 + k;
#pragma unroll
    for (int i = 0; i < NA; ++i) {
      const float dh = (xh[Ed][i] - xh[I][i]) - 0.5f * (xh[J][i] - xh[I][i]);
      const float dlo = (xl[Ed][i] - xl[I][i]) - 0.5f * (xl[J][i] - xl[I][i]);
      ed.dl[k][i] = dh + dlo;
    }
  }
  if constexpr (P >= 3) {
#pragma unroll
    for (int a = 1; a < REF; ++a)
#pragma unroll
      for (int d = 0; d < NA; ++d) ed.rel[a][d] = (xh[a][d] - xh[0][d]) + (xl[a][d] - xl[0][d]);
  }
  return ok;
}

// Compute the requested local matrices of element e in precision R and store
// them to dst: FULL = ref x ref per matrix (dst[m * ref^2 + a * ref + b]),
// otherwise the upper triangle (dst[m * dst_stride_m + u]); m in accumulator order.
template <int D, int NA, int P, typename R, typename RS, bool FULL>
__device__ __forceinline__ void element_store_ed(const ElemData<D, NA, P, R>& ed, const TabView<R>& tb,
                                                 const void* coef, int coef_f32, int64_t e, unsigned which,
                                                 RS* dst, int dst_stride_m, R& qual, bool& bad) {
  constexpr int U = Ref<D, P>::U;
  constexpr int REF = Ref<D, P>::REF;
  R Mo[U], Ao[U], Co[U];
  const bool wm = which & LFEM_MASS, wa = which & LFEM_STIFF, wc = which & LFEM_CMASS;
  const int im = 0, ia = wm ? 1 : 0, ic = (wm ? 1 : 0) + (wa ? 1 : 0);
  auto put = [&](const R(&v)[U], int slot) {
    if constexpr (FULL) {
      RS* d = dst + slot * (REF * REF);
#pragma unroll
      for (int x = 0; x < REF; ++x)
#pragma unroll
        for (int y = x; y < REF; ++y) {
          const RS val = (RS)v[upper_index(REF, x, y)];
          d[x * REF + y] = val;
          if (y != x) d[y * REF + x] = val;
        }
    } else {
#pragma unroll
      for (int u = 0; u < U; ++u) dst[slot * dst_stride_m + u] = (RS)v[u];
    }
  };
  if constexpr (D == 3) {
    // two passes keep the register footprint at two matrices
    if (wm || wc) {
      if (wm && wc) element_pass<D, NA, P, R, true, false, true>(ed, tb, coef, coef_f32, e, Mo, Ao, Co, qual, bad);
      else if (wm) element_pass<D, NA, P, R, true, false, false>(ed, tb, coef, coef_f32, e, Mo, Ao, Co, qual, bad);
      else element_pass<D, NA, P, R, false, false, true>(ed, tb, coef, coef_f32, e, Mo, Ao, Co, qual, bad);
      if (wm) put(Mo, im);
      if (wc) put(Co, ic);
    }
    if (wa) {
      element_pass<D, NA, P, R, false, true, false>(ed, tb, coef, coef_f32, e, Mo, Ao, Co, qual, bad);
      put(Ao, ia);
    }
  } else {
    if (wm && wa && wc) element_pass<D, NA, P, R, true, true, true>(ed, tb, coef, coef_f32, e, Mo, Ao, Co, qual, bad);
    else if (wm && wa) element_pass<D, NA, P, R, true, true, false>(ed, tb, coef, coef_f32, e, Mo, Ao, Co, qual, bad);
    else if (wm && wc) element_pass<D, NA, P, R, true, false, true>(ed, tb, coef, coef_f32, e, Mo, Ao, Co, qual, bad);
    else if (wa && wc) element_pass<D, NA, P, R, false, true, true>(ed, tb, coef, coef_f32, e, Mo, Ao, Co, qual, bad);
    else if (wm) element_pass<D, NA, P, R, true, false, false>(ed, tb, coef, coef_f32, e, Mo, Ao, Co, qual, bad);
    else if (wa) element_pass<D, NA, P, R, false, true, false>(ed, tb, coef, coef_f32, e, Mo, Ao, Co, qual, bad);
    else if (wc) element_pass<D, NA, P, R, false, false, true>(ed, tb, coef, coef_f32, e, Mo, Ao, Co, qual, bad);
    if (wm) put(Mo, im);
    if (wa) put(Ao, ia);
    if (wc) put(Co, ic);
  }
}

// Double-precision recomputation of one element (upper layout), kept out of
// line so the float hot path does not carry its registers.
template <int D, int NA, int P, typename RS, bool FULL>
__device__ __noinline__ void element_fp64(const double* __restrict__ coords, const int32_t* __restrict__ nodes,
                                          TabRef tab, const void* coef, int coef_f32, int64_t e, unsigned which,
                                          RS* dst, int dst_stride_m, bool* bad_out) {
  constexpr int REF = Ref<D, P>::REF;
  int32_t nd[REF];
#pragma unroll
  for (int b = 0; b < REF; ++b) nd[b] = nodes[b];
  double X[REF][NA];
  gather_coords<D, NA, P>(coords, nd, X);
  ElemData<D, NA, P, double> ed;
  load_element_data<D, NA, P, double>(X, ed);
  const TabView<double> tb = tab_view<D, P, double>(tab);
  double qual = 1.0;
  bool bad = false;
  element_store_ed<D, NA, P, double, RS, FULL>(ed, tb, coef, coef_f32, e, which, dst, dst_stride_m, qual, bad);
  *bad_out = bad;
}

// Double recomputation of one element, one matrix per pass so the registers
// needed stay below those of the float hot path (upper layout, stored as RS).
// IL = false: matrix k at dst[k stride_m + u stride_u]; IL = true: the
// interleaved tile layout, matrix slot slot0 + k at dst[lsm_word(u, slot0 + k)].
template <int D, int NA, int P, typename RS, bool IL = false>
__device__ __forceinline__ void element_fp64_lean(const double* __restrict__ coords,
                                                  const int32_t (&nd)[Ref<D, P>::REF], TabRef tab, const void* coef,
                                                  int coef_f32, int64_t e, unsigned which, RS* dst, int stride_m,
                                                  bool& bad, int slot0 = 0, int stride_u = 1) {
  constexpr int REF = Ref<D, P>::REF;
  constexpr int U = Ref<D, P>::U;
  double X[REF][NA];
  gather_coords<D, NA, P>(coords, nd, X);
  ElemData<D, NA, P, double> ed;
  load_element_data<D, NA, P, double>(X, ed);
  const TabView<double> tb = tab_view<D, P, double>(tab);
  double qual = 1.0;
  double V[U], dummy1[U], dummy2[U];
  int slot = slot0;
  auto put = [&](int u, double v) {
    if constexpr (IL) dst[lsm_word(u, slot)] = (RS)v;
    else dst[slot * stride_m + u * stride_u] = (RS)v;
  };
  if (which & LFEM_MASS) {
    element_pass<D, NA, P, double, true, false, false>(ed, tb, coef, coef_f32, e, V, dummy1, dummy2, qual, bad);
#pragma unroll
    for (int u = 0; u < U; ++u) put(u, V[u]);
    ++slot;
  }
  if (which & LFEM_STIFF) {
    element_pass<D, NA, P, double, false, true, false>(ed, tb, coef, coef_f32, e, dummy1, V, dummy2, qual, bad);
#pragma unroll
    for (int u = 0; u < U; ++u) put(u, V[u]);
    ++slot;
  }
  if (which & LFEM_CMASS) {
    element_pass<D, NA, P, double, false, false, true>(ed, tb, coef, coef_f32, e, dummy1, dummy2, V, qual, bad);
#pragma unroll
    for (int u = 0; u < U; ++u) put(u, V[u]);
  }
}

// Compute (upper layout) from double coordinates, precision R.
template <int D, int NA, int P, typename R, typename RS>
__device__ __forceinline__ void element_store(const double (&X)[Ref<D, P>::REF][NA], const TabView<R>& tb,
                                              const void* coef, int coef_f32, int64_t e, unsigned which,
                                              RS* dst, int dst_stride_m, R& qual, bool& bad) {
  ElemData<D, NA, P, R> ed;
  load_element_data<D, NA, P, R>(X, ed);
  element_store_ed<D, NA, P, R, RS, false>(ed, tb, coef, coef_f32, e, which, dst, dst_stride_m, qual, bad);
}

// Launch shape: the float kernel needs ~160 registers, so 192 threads x 2
// CTAs per SM; the double kernel runs 256 threads x 1 CTA.
// ----------------------------------------------------------------------------
// Element-stage kernels (FP64): physical points, geometry, local matrices.
// ----------------------------------------------------------------------------
template <int D, int NA, int P>
__global__ void k_eval_points(const int32_t* __restrict__ conn, int64_t nE, const double* __restrict__ coords,
                              TabRef tab, double* __restrict__ out) {
  constexpr int REF = Ref<D, P>::REF;
  const TabView<double> tb = tab_view<D, P, double>(tab);
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nE; e += (int64_t)gridDim.x * blockDim.x) {
    int32_t nodes[REF];
#pragma unroll
    for (int b = 0; b < REF; ++b) nodes[b] = conn[e * REF + b];
    double X[REF][NA];
    gather_coords<D, NA, P>(coords, nodes, X);
    for (int q = 0; q < tb.q; ++q) {
#pragma unroll
      for (int i = 0; i < NA; ++i) {
        double acc = 0.0;
#pragma unroll
        for (int b = 0; b < REF; ++b) acc = fma(tb.phi[q * REF + b], X[b][i], acc);
        out[(e * tb.q + q) * NA + i] = acc;
      }
    }
  }
}

template <int D, int NA, int P>
__global__ void k_geometry(const int32_t* __restrict__ conn, int64_t nE, const double* __restrict__ coords,
                           TabRef tab, double* __restrict__ Jout, double* __restrict__ sout,
                           double* __restrict__ Gout) {
  constexpr int REF = Ref<D, P>::REF;
  const TabView<double> tb = tab_view<D, P, double>(tab);
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nE; e += (int64_t)gridDim.x * blockDim.x) {
    int32_t nodes[REF];
#pragma unroll
    for (int b = 0; b < REF; ++b) nodes[b] = conn[e * REF + b];
    double X[REF][NA];
    gather_coords<D, NA, P>(coords, nodes, X);
    ElemData<D, NA, P, double> ed;
    load_element_data<D, NA, P, double>(X, ed);
    for (int q = 0; q < tb.q; ++q) {
      QpGeom<D, NA, P, double> g;
      qp_geometry<D, NA, P, double>(ed, tb, q, 1.0, g);  // with w = 1: H = s G^{-1}
      const int64_t bq = e * tb.q + q;
      if (Jout)
#pragma unroll
        for (int i = 0; i < NA; ++i)
#pragma unroll
          for (int m = 0; m < D; ++m) Jout[(bq * NA + i) * D + m] = g.J[i][m];
      if (sout) sout[bq] = g.s;
      if (Gout)
#pragma unroll
        for (int m = 0; m < D; ++m)
#pragma unroll
          for (int k = 0; k < D; ++k) Gout[(bq * D + m) * D + k] = g.H[m][k] / g.s;
    }
  }
}

template <int D, int NA, int P>
__global__ void k_local(const int32_t* __restrict__ conn, int64_t nE, const double* __restrict__ coords,
                        TabRef tab, const double* __restrict__ coef, unsigned which, double* __restrict__ M,
                        double* __restrict__ A, double* __restrict__ C) {
  constexpr int REF = Ref<D, P>::REF;
  constexpr int U = Ref<D, P>::U;
  const TabView<double> tb = tab_view<D, P, double>(tab);
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nE; e += (int64_t)gridDim.x * blockDim.x) {
    int32_t nodes[REF];
#pragma unroll
    for (int b = 0; b < REF; ++b) nodes[b] = conn[e * REF + b];
    double X[REF][NA];
    gather_coords<D, NA, P>(coords, nodes, X);
    double tmp[3 * U];
    double qual = 1.0;
    bool bad = false;
    element_store<D, NA, P, double, double>(X, tb, coef, 0, e, which, tmp, U, qual, bad);
    int m = 0;
    if (which & LFEM_MASS) {
      for (int u = 0; u < U; ++u) M[e * U + u] = tmp[m * U + u];
      ++m;
    }
    if (which & LFEM_STIFF) {
      for (int u = 0; u < U; ++u) A[e * U + u] = tmp[m * U + u];
      ++m;
    }
    if (which & LFEM_CMASS) {
      for (int u = 0; u < U; ++u) C[e * U + u] = tmp[m * U + u];
      ++m;
    }
  }
}

// ----------------------------------------------------------------------------
// Host launchers
// ----------------------------------------------------------------------------
struct StageArgs {
  const int32_t* conn;
  int64_t nE;
  const double* coords;
  TabRef tab;
  const double* coef;
  unsigned which;
  double* o0;
  double* o1;
  double* o2;
};

static inline unsigned stage_grid(int64_t n) {
  int64_t g = (n + 127) / 128;
  if (g > 152 * 32) g = 152 * 32;
  return (unsigned)(g < 1 ? 1 : g);
}

template <int D, int NA, int P>
lfem_status launch_stage(int kind, const StageArgs& s, cudaStream_t st) {
  if (s.nE == 0) return LFEM_OK;
  if (kind == 0) k_eval_points<D, NA, P><<<stage_grid(s.nE), 128, 0, st>>>(s.conn, s.nE, s.coords, s.tab, s.o0);
  else if (kind == 1)
    k_geometry<D, NA, P><<<stage_grid(s.nE), 128, 0, st>>>(s.conn, s.nE, s.coords, s.tab, s.o0, s.o1, s.o2);
  else
    k_local<D, NA, P><<<stage_grid(s.nE), 128, 0, st>>>(s.conn, s.nE, s.coords, s.tab, s.coef, s.which, s.o0, s.o1,
                                                         s.o2);
  LFEM_CUDA(cudaGetLastError());
  return LFEM_OK;
}

}  // namespace lfem
