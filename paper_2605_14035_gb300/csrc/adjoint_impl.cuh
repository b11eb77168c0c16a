// Adjoint of the assembly: dL/d(CSR values) -> dL/d(node coordinates), FP64
// (and a mixed variant: FP32 geometry, double recomputation of the elements
// that fail the conditioning test, double per-node sums).
//
// For L = sum_s gM[s] M[s] + gA[s] A[s] + gMC[s] MC[s] and one element, with
// Gb the element's gathered gradients and s = |det DF|, G = J^T J:
//   m_q   = sum_ab (GbM_ab + c_q GbC_ab) phi_a phi_b
//   K_q   = sym(sum_ab GbA_ab grad^phi_a grad^phi_b^T)
//   dL/dJ = w_q s [ (m_q + <K_q, G^-1>) J G^-1 - 2 J G^-1 K_q G^-1 ]
//   dL/dx_{E[k]} += dL/dJ grad^phi_k
// (variation of s and of s G^-1 under dJ; the local matrices are those of
// Eqs. reference_quadrature_mass / reference_quadrature_stiffness).  Geometry
// is recomputed per quadrature point, never stored.  The per-node sum runs in
// the same row tiles as the assembly: each tile owns its rows' gradients and
// adds the incidences in ascending element order (deterministic, no atomics).
#pragma once

#include "assemble_impl.cuh"
#include "lfem_internal.cuh"

namespace lfem {

struct AdjArgs {
  const int32_t* conn;
  const double* coords;
  const double* coef;
  const double* gM;
  const double* gA;
  const double* gC;
  double* g_coords;
  double* g_coef;
  const int64_t* row_ptr;
  const int32_t* inc_ptr;
  const uint8_t* inc_pos;
  const uint16_t* inc_local;
  const int32_t* elem_inc;
  const int32_t* tile_row0;
  const int32_t* tile_elem_ptr;
  const int32_t* tile_elem;
  TabRef tab;
  int chunk;
  int64_t tile_begin;
  int mixed;                     // FP32 geometry with a double recomputation of flagged elements
  float qmin;                    // conditioning threshold of the mixed path (metric quality)
  unsigned long long* fallback;  // elements recomputed in double (mixed)
  // orders 3, 4 (warp per element, then a per-node pass)
  const int32_t* inc_key;        // [n_inc] (e << key_shift) | a, ascending per node
  int key_shift;
  int64_t n_elem;
  int32_t n_nodes;
  double* buf;                   // [n_elem][ref][ambient] element node gradients
};

// R = double: the reference computation; R = float: the mixed path, which
// reports (redo) an element whose coordinates leave the float range or whose
// metric fails the conditioning or finiteness test, for a double recomputation.
template <int D, int NA, int P, typename PosT, typename R>
__device__ __forceinline__ void adjoint_element(const AdjArgs& a, int64_t e, const int32_t (&nodes)[Ref<D, P>::REF],
                                                const TabView<R>& tb, bool write_coef,
                                                double (&ge_out)[Ref<D, P>::REF][NA], bool& redo) {
  constexpr int REF = Ref<D, P>::REF;
  constexpr int U = Ref<D, P>::U;
  // symmetric gathered gradients per upper pair: Gb_ab + Gb_ba (a < b), Gb_aa
  double GMd[U], GAd[U], GCd[U];
#pragma unroll
  for (int u = 0; u < U; ++u) GMd[u] = GAd[u] = GCd[u] = 0.0;
#pragma unroll
  for (int ai = 0; ai < REF; ++ai) {
    const int32_t k = __ldg(a.elem_inc + e * REF + ai);
    const int64_t rb = __ldg(a.row_ptr + nodes[ai]);
    int pos[REF];
    load_pos<PosT, REF>(a.inc_pos, k, pos);
#pragma unroll
    for (int b = 0; b < REF; ++b) {
      const int64_t s = rb + pos[b];
      const int u = sym_index(REF, ai, b);
      if (a.gM) GMd[u] += __ldg(a.gM + s);
      if (a.gA) GAd[u] += __ldg(a.gA + s);
      if (a.gC) GCd[u] += __ldg(a.gC + s);
    }
  }
  R GM[U], GA[U], GC[U];
#pragma unroll
  for (int u = 0; u < U; ++u) {
    GM[u] = (R)GMd[u];
    GA[u] = (R)GAd[u];
    GC[u] = (R)GCd[u];
  }
  R ge[REF][NA];
#pragma unroll
  for (int ai = 0; ai < REF; ++ai)
#pragma unroll
    for (int i = 0; i < NA; ++i) ge[ai][i] = (R)0;
  ElemData<D, NA, P, R> ed;
  bool ok = true;
  if constexpr (sizeof(R) == 4) {
    ok = load_element_data_split<D, NA, P>(a.coords, nodes, ed);
  } else {
    double X[REF][NA];
    gather_coords<D, NA, P>(a.coords, nodes, X);
    load_element_data<D, NA, P, double>(X, ed);
  }
  R qual = (R)1;
  bool bad = false;
  for (int q = 0; q < tb.q; ++q) {
    const R wq = tb.w[q];
    QpGeom<D, NA, P, R> g;
    qp_geometry<D, NA, P, R>(ed, tb, q, (R)1, g);  // H = s G^-1
    qual = fmin(qual, g.quality);
    bad |= !(g.s > (R)0) || !isfinite(g.s);
    const R s = g.s;
    R Gi[D][D];
#pragma unroll
    for (int m = 0; m < D; ++m)
#pragma unroll
      for (int k = 0; k < D; ++k) Gi[m][k] = g.H[m][k] / s;
    const R* ph = tb.phi + q * REF;
    const R* dph = tb.dphi + q * REF * D;
    const R cq = (a.coef && a.gC) ? (R)__ldg(a.coef + e * tb.q + q) : (R)0;
    R mq = 0, mc = 0;
    R K[D][D];
#pragma unroll
    for (int m = 0; m < D; ++m)
#pragma unroll
      for (int k = 0; k < D; ++k) K[m][k] = 0;
#pragma unroll
    for (int ai = 0; ai < REF; ++ai)
#pragma unroll
      for (int b = ai; b < REF; ++b) {
        const int u = upper_index(REF, ai, b);
        const R pp = ph[ai] * ph[b];
        mq += (GM[u] + cq * GC[u]) * pp;
        mc += GC[u] * pp;
        // symmetric part of GA_u grad phi_a grad phi_b^T (halved for a < b since GA sums both orders)
        const R f = (ai == b) ? GA[u] : (R)0.5 * GA[u];
#pragma unroll
        for (int m = 0; m < D; ++m)
#pragma unroll
          for (int k = 0; k < D; ++k) K[m][k] += f * (dph[ai * D + m] * dph[b * D + k] + (ai == b ? (R)0 : dph[b * D + m] * dph[ai * D + k]));
      }
    R KG = 0;
#pragma unroll
    for (int m = 0; m < D; ++m)
#pragma unroll
      for (int k = 0; k < D; ++k) KG += K[m][k] * Gi[m][k];
    R T[D][D], B[D][D];
#pragma unroll
    for (int m = 0; m < D; ++m)
#pragma unroll
      for (int k = 0; k < D; ++k) {
        R t = 0;
#pragma unroll
        for (int l = 0; l < D; ++l) t += Gi[m][l] * K[l][k];
        T[m][k] = t;
      }
#pragma unroll
    for (int m = 0; m < D; ++m)
#pragma unroll
      for (int k = 0; k < D; ++k) {
        R t = 0;
#pragma unroll
        for (int l = 0; l < D; ++l) t += T[m][l] * Gi[l][k];
        B[m][k] = t;
      }
    R dLdJ[NA][D];
    const R ws = wq * s;
#pragma unroll
    for (int i = 0; i < NA; ++i)
#pragma unroll
      for (int k = 0; k < D; ++k) {
        R jg = 0, jb = 0;
#pragma unroll
        for (int m = 0; m < D; ++m) {
          jg += g.J[i][m] * Gi[m][k];
          jb += g.J[i][m] * B[m][k];
        }
        dLdJ[i][k] = ws * ((mq + KG) * jg - (R)2 * jb);
      }
#pragma unroll
    for (int ai = 0; ai < REF; ++ai)
#pragma unroll
      for (int i = 0; i < NA; ++i) {
        R t = 0;
#pragma unroll
        for (int k = 0; k < D; ++k) t += dLdJ[i][k] * dph[ai * D + k];
        ge[ai][i] += t;
      }
    if (write_coef) a.g_coef[e * tb.q + q] = (double)(ws * mc);
  }
#pragma unroll
  for (int ai = 0; ai < REF; ++ai)
#pragma unroll
    for (int i = 0; i < NA; ++i) ge_out[ai][i] = (double)ge[ai][i];
  if constexpr (sizeof(R) == 4) redo = !ok || bad || (D > 1 && qual < (R)a.qmin) || !(qual > (R)1e-12);
}

template <int D, int NA, int P, typename PosT, bool MIXED>
__global__ void __launch_bounds__(128) k_adjoint_tiles(const AdjArgs a) {
  constexpr int REF = Ref<D, P>::REF;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* gsm = reinterpret_cast<double*>(smem_raw);  // [chunk][REF][NA]
  __shared__ int s_nredo;
  __shared__ int s_redo[128];  // mixed: chunk elements to recompute in double (chunk <= 128)
  const int64_t t = a.tile_begin + blockIdx.x;
  const int32_t r0 = a.tile_row0[t], r1 = a.tile_row0[t + 1];
  const int32_t el0 = a.tile_elem_ptr[t];
  const int nel = a.tile_elem_ptr[t + 1] - el0;
  const int nrows = r1 - r0;
  const TabView<double> tb = tab_view<D, P, double>(a.tab);
  const TabView<float> tbf = tab_view<D, P, float>(a.tab);
  const int nchunks = nel == 0 ? 1 : (nel + a.chunk - 1) / a.chunk;
  for (int ci = 0; ci < nchunks; ++ci) {
    const int c0 = ci * a.chunk;
    const int cn = max(0, min(a.chunk, nel - c0));
    if (MIXED && threadIdx.x == 0) s_nredo = 0;
    if (MIXED) __syncthreads();
    for (int j = threadIdx.x; j < cn; j += blockDim.x) {
      const int64_t e = a.tile_elem[el0 + c0 + j];
      int32_t nodes[REF];
#pragma unroll
      for (int b = 0; b < REF; ++b) nodes[b] = __ldg(a.conn + e * REF + b);
      const bool owner = nodes[0] >= r0 && nodes[0] < r1;
      double ge[REF][NA];
      bool redo = false;
      if constexpr (MIXED) {
        adjoint_element<D, NA, P, PosT, float>(a, e, nodes, tbf, owner && a.g_coef != nullptr, ge, redo);
        if (redo) s_redo[atomicAdd(&s_nredo, 1)] = j;  // recomputed below by whole warps
      } else {
        adjoint_element<D, NA, P, PosT, double>(a, e, nodes, tb, owner && a.g_coef != nullptr, ge, redo);
      }
#pragma unroll
      for (int ai = 0; ai < REF; ++ai)
#pragma unroll
        for (int i = 0; i < NA; ++i) gsm[((size_t)j * REF + ai) * NA + i] = ge[ai][i];
    }
    __syncthreads();
    if constexpr (MIXED) {
      // double recomputation over the compacted list (the FP64 pipe costs the
      // same for a warp instruction with few active lanes)
      const int nr = s_nredo;
      for (int t = threadIdx.x; t < nr; t += blockDim.x) {
        const int j = s_redo[t];
        const int64_t e = a.tile_elem[el0 + c0 + j];
        int32_t nodes[REF];
#pragma unroll
        for (int b = 0; b < REF; ++b) nodes[b] = __ldg(a.conn + e * REF + b);
        const bool owner = nodes[0] >= r0 && nodes[0] < r1;
        double ge[REF][NA];
        bool unused = false;
        adjoint_element<D, NA, P, PosT, double>(a, e, nodes, tb, owner && a.g_coef != nullptr, ge, unused);
        if (owner) atomicAdd(a.fallback, 1ull);
#pragma unroll
        for (int ai = 0; ai < REF; ++ai)
#pragma unroll
          for (int i = 0; i < NA; ++i) gsm[((size_t)j * REF + ai) * NA + i] = ge[ai][i];
      }
      __syncthreads();
    }
    for (int w = threadIdx.x; w < nrows * NA; w += blockDim.x) {
      const int rl = w / NA, i = w - rl * NA;
      const int32_t r = r0 + rl;
      double sum = 0.0;
      for (int32_t k = a.inc_ptr[r]; k < a.inc_ptr[r + 1]; ++k) {
        const uint16_t lk = a.inc_local[k];
        const int loc = (lk >> 4) - c0;
        if (loc < 0) continue;
        if (loc >= cn) break;
        sum += gsm[((size_t)loc * REF + (lk & 15)) * NA + i];
      }
      double* o = a.g_coords + (int64_t)r * NA + i;
      if (ci == 0) *o = sum;
      else *o += sum;
    }
    __syncthreads();
  }
}

template <int D, int NA, int P>
lfem_status launch_adjoint(const AdjArgs& a0, int64_t n_tiles, int pos_bytes, cudaStream_t st) {
  if (n_tiles == 0) return LFEM_OK;
  constexpr int REF = Ref<D, P>::REF;
  const size_t smem = sizeof(double) * (size_t)a0.chunk * REF * NA;
  auto kern = a0.mixed ? (pos_bytes == 1 ? k_adjoint_tiles<D, NA, P, uint8_t, true> : k_adjoint_tiles<D, NA, P, uint16_t, true>)
                       : (pos_bytes == 1 ? k_adjoint_tiles<D, NA, P, uint8_t, false> : k_adjoint_tiles<D, NA, P, uint16_t, false>);
  LFEM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  AdjArgs a = a0;
  const int64_t max_grid = 1ll << 30;
  for (int64_t t0 = 0; t0 < n_tiles; t0 += max_grid) {
    a.tile_begin = t0;
    const int64_t nb = n_tiles - t0 < max_grid ? n_tiles - t0 : max_grid;
    kern<<<(unsigned)nb, 128, smem, st>>>(a);
    LFEM_CUDA(cudaGetLastError());
  }
  return LFEM_OK;
}

}  // namespace lfem
