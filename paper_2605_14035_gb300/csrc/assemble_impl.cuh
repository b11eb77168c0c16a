// Assembly kernels, templated on the element type (D, NA, P).
//
// Fused tile kernel (one CTA per row tile):
//   phase 1  element per thread: gather coordinates, geometry per quadrature
//            point, local upper-triangle matrices in registers -> shared memory
//            (Sec. 3.2.1-3.2.2; Eqs. reference_quadrature_mass / _stiffness)
//   phase 2  (row, matrix) per thread: add the tile elements' local rows into
//            the tile's CSR slots in shared memory, incidences in ascending
//            element order -> a fixed summation order, no atomics
//            (Eqs. M matrix, A matrix: sum over elements)
//   phase 3  write the tile's contiguous slot range [row_ptr[r0], row_ptr[r1])
//            with coalesced stores
// Each tile owns whole CSR rows, so no other CTA writes its slots; elements
// touching several tiles are recomputed by each (halo recompute).
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
  for (int q = 0; q < tb.q; ++q) {
    const R wq = tb.w[q];
    QpGeom<D, NA, P, R> g;
    qp_geometry<D, NA, P, R>(ed, tb, q, wq, g);
    qual = fmin(qual, g.quality);
    bad |= !(g.s > (R)0) || !isfinite(g.s);
    R cq = 0;
    if (DC) cq = load_coef<R>(coef, coef_f32, e * tb.q + q);
    qp_accumulate<D, NA, P, R, DM, DA, DC>(g, tb, q, wq, cq, Mo, Ao, Co);
  }
}

// Compute the requested local matrices of element e in precision R and store
// them to dst[m * U + u] (m in accumulator order).
template <int D, int NA, int P, typename R, typename RS>
__device__ __forceinline__ void element_store(const double (&X)[Ref<D, P>::REF][NA], const TabView<R>& tb,
                                              const void* coef, int coef_f32, int64_t e, unsigned which,
                                              RS* dst, int dst_stride_m, R& qual, bool& bad) {
  constexpr int U = Ref<D, P>::U;
  ElemData<D, NA, P, R> ed;
  load_element_data<D, NA, P, R>(X, ed);
  R Mo[U], Ao[U], Co[U];
  const bool wm = which & LFEM_MASS, wa = which & LFEM_STIFF, wc = which & LFEM_CMASS;
  const int im = 0, ia = wm ? 1 : 0, ic = (wm ? 1 : 0) + (wa ? 1 : 0);
  auto put = [&](const R(&v)[U], int slot) {
#pragma unroll
    for (int u = 0; u < U; ++u) dst[slot * dst_stride_m + u] = (RS)v[u];
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

template <int D, int NA, int P, typename R, typename PosT>
__global__ void __launch_bounds__(256) k_assemble_tiles(const AsmArgs a) {
  constexpr int REF = Ref<D, P>::REF;
  constexpr int U = Ref<D, P>::U;
  using Acc = typename AccOf<R>::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nm = a.nm;
  const int S = a.slots_cap;
  Acc* acc = reinterpret_cast<Acc*>(smem_raw);
  R* lsm = reinterpret_cast<R*>(smem_raw + sizeof(Acc) * (size_t)nm * S);
  const int lstride = nm * U;

  const int64_t t = a.tile_begin + blockIdx.x;
  const int32_t r0 = a.tile_row0[t], r1 = a.tile_row0[t + 1];
  const int64_t s0 = a.row_ptr[r0];
  const int ns = (int)(a.row_ptr[r1] - s0);
  const int32_t el0 = a.tile_elem_ptr[t];
  const int nel = a.tile_elem_ptr[t + 1] - el0;
  const int nrows = r1 - r0;

  for (int i = threadIdx.x; i < nm * ns; i += blockDim.x) acc_zero(acc[(i / ns) * S + (i % ns)]);

  const TabView<R> tb = tab_view<D, P, R>(a.tab);
  for (int c0 = 0; c0 < nel; c0 += a.chunk) {
    const int cn = min(a.chunk, nel - c0);
    // ---- phase 1: local matrices, element per thread
    for (int j = threadIdx.x; j < cn; j += blockDim.x) {
      const int64_t e = a.tile_elem[el0 + c0 + j];
      const int32_t* cn_e = a.conn + e * REF;
      int32_t nodes[REF];
#pragma unroll
      for (int b = 0; b < REF; ++b) nodes[b] = __ldg(cn_e + b);
      double X[REF][NA];
      gather_coords<D, NA, P>(a.coords, nodes, X);
      R qual = (R)1;
      bool bad = false;
      R* dst = lsm + (size_t)j * lstride;
      element_store<D, NA, P, R, R>(X, tb, a.coef, a.coef_f32, e, a.which, dst, U, qual, bad);
      const bool owner = nodes[0] >= r0 && nodes[0] < r1;
      if constexpr (sizeof(R) == 4) {
        if (D > 1 && (qual < (R)a.qmin || bad)) {
          // ill-conditioned metric: redo the element in double
          const TabView<double> tb64 = tab_view<D, P, double>(a.tab);
          double q64 = 1.0;
          bool bad64 = false;
          element_store<D, NA, P, double, R>(X, tb64, a.coef, a.coef_f32, e, a.which, dst, U, q64, bad64);
          if (owner) atomicAdd(a.fallback, 1ull);
          bad = bad64;
        }
      }
      if (bad && owner) atomicOr(a.status, ST_DEGENERATE);
    }
    __syncthreads();
    // ---- phase 2: per (row, matrix), incidences in ascending element order
    for (int w = threadIdx.x; w < nrows * nm; w += blockDim.x) {
      const int rl = w / nm, m = w - rl * nm;
      const int32_t r = r0 + rl;
      const int base = (int)(a.row_ptr[r] - s0);
      Acc* accm = acc + (size_t)m * S + base;
      const R* lm = lsm + m * U;
      const int32_t kb = a.inc_ptr[r], ke = a.inc_ptr[r + 1];
      for (int32_t k = kb; k < ke; ++k) {
        const uint16_t lk = a.inc_local[k];
        const int loc = (lk >> 4) - c0;
        if (loc < 0) continue;
        if (loc >= cn) break;
        const int ai = lk & 15;
        const PosT* pos = reinterpret_cast<const PosT*>(a.inc_pos) + (int64_t)k * REF;
        const R* lrow = lm + (size_t)loc * lstride;
#pragma unroll
        for (int b = 0; b < REF; ++b) {
          const int u = ai <= b ? upper_index(REF, ai, b) : upper_index(REF, b, ai);
          acc_add(accm[pos[b]], lrow[u]);
        }
      }
    }
    __syncthreads();
  }
  // ---- phase 3: coalesced stores of the tile's slot range
  for (int i = threadIdx.x; i < nm * ns; i += blockDim.x) {
    const int m = i / ns, s = i - m * ns;
    R* o = reinterpret_cast<R*>(a.out[m]);
    o[s0 + s] = (R)acc_final(acc[(size_t)m * S + s]);
  }
}

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

template <int D, int NA, int P, typename R>
size_t tile_smem_bytes(int nm, int slots, int chunk) {
  using Acc = typename AccOf<R>::T;
  return sizeof(Acc) * (size_t)nm * slots + sizeof(R) * (size_t)chunk * nm * Ref<D, P>::U;
}

template <int D, int NA, int P, typename R>
lfem_status launch_tiles(const AsmArgs& a0, int64_t n_tiles, int threads, int pos_bytes, cudaStream_t st) {
  if (n_tiles == 0) return LFEM_OK;
  const size_t smem = tile_smem_bytes<D, NA, P, R>(a0.nm, a0.slots_cap, a0.chunk);
  if (smem > 227 * 1024) return fail(LFEM_E_ARG, "tile configuration needs more than 227 KB of shared memory");
  auto kern = pos_bytes == 1 ? k_assemble_tiles<D, NA, P, R, uint8_t> : k_assemble_tiles<D, NA, P, R, uint16_t>;
  LFEM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  AsmArgs a = a0;
  const int64_t max_grid = 1ll << 30;
  for (int64_t t0 = 0; t0 < n_tiles; t0 += max_grid) {
    a.tile_begin = t0;
    const int64_t nb = n_tiles - t0 < max_grid ? n_tiles - t0 : max_grid;
    kern<<<(unsigned)nb, threads, smem, st>>>(a);
    LFEM_CUDA(cudaGetLastError());
  }
  return LFEM_OK;
}

}  // namespace lfem
