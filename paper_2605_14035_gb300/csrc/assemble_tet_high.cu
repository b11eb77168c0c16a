// Orders 3 and 4 on tetrahedra (20 and 35 nodes; 210 and 630 upper entries
// per matrix), element-major like the other tets: local matrices into the
// buffer [nE][nm][U], then every CSR slot sums its list (k_slot_gather).
//
// A local matrix this large does not fit one thread's registers, so one warp
// takes one element:
//   * the basis table phi_b, grad^phi_b at the rule's points (Eq. F_map with
//     the Lagrange basis of the nodes alpha/p) is tabulated once per launch in
//     FP64 by k_tet_high_table and staged into every CTA's shared memory;
//   * the geometry is computed by lanes over quadrature points: J = sum_b
//     (x_b - x_0) grad^phi_b^T, s = |det J|, H = w s G^{-1} = (w / s) adj(G)
//     with adj(G)_mk = c_m . c_k, c_m the cross product of J's other two
//     columns (Eq. basic integral formula, Eqs. jacobian_inv);
//   * each lane owns a register block of RA rows x RB columns of the matrix
//     (order 3: 4 x 2 blocks, 30 lanes; order 4: 5 x 5, 28 lanes; the blocks
//     on or above the diagonal) and sums it over the points (Eqs.
//     reference_quadrature_mass, reference_quadrature_stiffness):
//       M_ab += (w s phi_b) phi_a,  A_ab += grad^phi_a . (H grad^phi_b),
//       C_ab += (c_q w s phi_b) phi_a,
//     with the per-point node factors (w s phi_b, H grad^phi_b) computed once
//     per node into shared memory: per point a lane reads RA + RB rows for
//     RA RB entries.
// LFEM_MIXED: float geometry and sums; an element whose metric fails the
// conditioning test (or is not finite) anywhere is listed and recomputed in
// FP64 by a second launch over the list.
#include "dispatch.cuh"
#include "tet_high.cuh"

namespace lfem {

// Origin (r0, c0) of lane's block: the blocks on or above the diagonal in
// column-major order; r0 = -1 for a lane without one.
template <int P>
__device__ __forceinline__ void tet_high_block(int lane, int& r0, int& c0) {
  using T = TetHigh<P>;
  r0 = -1;
  c0 = 0;
  int k = 0;
  for (int j = 0; j < T::NCB; ++j)
    for (int i = 0; i < T::NRB; ++i)
      if (i * T::RA <= j * T::RB + T::RB - 1) {
        if (k == lane) {
          r0 = i * T::RA;
          c0 = j * T::RB;
        }
        ++k;
      }
}

// The lane's register block of one element summed over the points q0, q0 + qs,
// ...: MODE 0 mass, 1 stiffness, 2 coefficient-weighted mass (in acc), 3 mass
// (accm) and stiffness (acc) in one sweep: the node factors (w s phi_b,
// H grad^phi_b) share one row, so a point costs one factor stage and one set
// of row loads for both matrices.
template <int P, typename R, int MODE>
__device__ __forceinline__ void tet_high_accumulate(const V4<R>* tab, V4<R>* hb, const V4<R>* geo, int Q, int q0,
                                                    int qs, int lane, int r0, int c0,
                                                    R (&acc)[TetHigh<P>::RA][TetHigh<P>::RB],
                                                    R (&accm)[TetHigh<P>::RA][TetHigh<P>::RB]) {
  constexpr int REF = TetHigh<P>::REF, ROW = TetHigh<P>::ROW, RA = TetHigh<P>::RA, RB = TetHigh<P>::RB;
  constexpr int NRB = TetHigh<P>::NRB, NCB = TetHigh<P>::NCB;
  constexpr bool STIFF = MODE == 1 || MODE == 3, MASS = MODE != 1;
  const int rb = r0 / RA, cb = c0 / RB;  // the block's slots (row_slot, col_slot)
#pragma unroll
  for (int i = 0; i < RA; ++i)
#pragma unroll
    for (int j = 0; j < RB; ++j) acc[i][j] = accm[i][j] = (R)0;
  for (int q = q0; q < Q; q += qs) {
    const V4<R> g0 = geo[2 * q], g1 = geo[2 * q + 1];
    const V4<R>* tq = tab + q * ROW;
    for (int b = lane; b < REF; b += 32) {
      const V4<R> d = tq[TetHigh<P>::row_slot(b)];
      V4<R> h;
      h.x = MASS ? (MODE == 2 ? g0.x * g1.w : g0.x) * d.x : (R)0;
      if constexpr (STIFF) {
        h.y = fma(g0.y, d.y, fma(g0.z, d.z, g0.w * d.w));
        h.z = fma(g0.z, d.y, fma(g1.x, d.z, g1.y * d.w));
        h.w = fma(g0.w, d.y, fma(g1.y, d.z, g1.z * d.w));
      } else {
        h.y = h.z = h.w = (R)0;
      }
      hb[TetHigh<P>::col_slot(b)] = h;
    }
    __syncwarp();
    if (r0 >= 0) {
      if constexpr (STIFF) {
        V4<R> hv[RB];
#pragma unroll
        for (int j = 0; j < RB; ++j) hv[j] = hb[j * NCB + cb];
#pragma unroll
        for (int i = 0; i < RA; ++i) {
          const V4<R> da = tq[i * NRB + rb];
#pragma unroll
          for (int j = 0; j < RB; ++j) {
            acc[i][j] = fma(da.y, hv[j].y, fma(da.z, hv[j].z, fma(da.w, hv[j].w, acc[i][j])));
            if constexpr (MODE == 3) accm[i][j] = fma(da.x, hv[j].x, accm[i][j]);
          }
        }
      } else {
        R hx[RB];
#pragma unroll
        for (int j = 0; j < RB; ++j) hx[j] = hb[j * NCB + cb].x;
#pragma unroll
        for (int i = 0; i < RA; ++i) {
          const R pa = tq[i * NRB + rb].x;
#pragma unroll
          for (int j = 0; j < RB; ++j) acc[i][j] = fma(pa, hx[j], acc[i][j]);
        }
      }
    }
    __syncwarp();
  }
}

// The lane's block of the upper triangle to dst (and dst2, MODE 3), entry u
// at u * su.
template <int P, typename R, typename RS, int MODE>
__device__ __forceinline__ void tet_high_store(int r0, int c0, const R (&acc)[TetHigh<P>::RA][TetHigh<P>::RB],
                                               const R (&accm)[TetHigh<P>::RA][TetHigh<P>::RB], RS* dst, RS* dst2,
                                               int su) {
  constexpr int REF = TetHigh<P>::REF, RA = TetHigh<P>::RA, RB = TetHigh<P>::RB;
  if (r0 < 0) return;
#pragma unroll
  for (int i = 0; i < RA; ++i)
#pragma unroll
    for (int j = 0; j < RB; ++j)
      if (r0 + i <= c0 + j) {
        const int u = upper_index(REF, r0 + i, c0 + j) * su;
        if constexpr (MODE == 3) {
          dst[u] = (RS)accm[i][j];
          dst2[u] = (RS)acc[i][j];
        } else {
          dst[u] = (RS)acc[i][j];
        }
      }
}

// One element, every point, one warp: MODE 0 mass, 1 stiffness, 2 coefficient-
// weighted mass (into dst), 3 mass and stiffness in one sweep (dst, dst2).
template <int P, typename R, typename RS, int MODE>
__device__ __forceinline__ void tet_high_pass(const V4<R>* tab, V4<R>* hb, const V4<R>* geo, int Q, int lane, int r0,
                                              int c0, RS* dst, RS* dst2, int su) {
  R acc[TetHigh<P>::RA][TetHigh<P>::RB], accm[TetHigh<P>::RA][TetHigh<P>::RB];
  tet_high_accumulate<P, R, MODE>(tab, hb, geo, Q, 0, 1, lane, r0, c0, acc, accm);
  tet_high_store<P, R, RS, MODE>(r0, c0, acc, accm, dst, dst2, su);
}

// Geometry of point q of element e (rel = x_b - x_0): (w s, H00, H01, H02) and
// (H11, H12, H22, c_q) with H = w s G^{-1} = (w / s) adj(G) from the cofactors
// of J; bad: |det J| zero or not finite; redo (float): the conditioning test failed.
template <int P, typename R>
__device__ __forceinline__ void tet_high_point(const TwoPassArgs& a, const V4<R>* tab, const V4<R>* rel,
                                               const double* w64, int64_t e, int q, V4<R>* geo, bool& bad,
                                               bool& redo) {
  constexpr int REF = TetHigh<P>::REF, ROW = TetHigh<P>::ROW;
  const int Q = a.tab.q;
  const V4<R>* tq = tab + q * ROW;
  R J[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  for (int b = 1; b < REF; ++b) {
    const V4<R> r = rel[b], d = tq[TetHigh<P>::row_slot(b)];
    J[0][0] = fma(r.x, d.y, J[0][0]);
    J[0][1] = fma(r.x, d.z, J[0][1]);
    J[0][2] = fma(r.x, d.w, J[0][2]);
    J[1][0] = fma(r.y, d.y, J[1][0]);
    J[1][1] = fma(r.y, d.z, J[1][1]);
    J[1][2] = fma(r.y, d.w, J[1][2]);
    J[2][0] = fma(r.z, d.y, J[2][0]);
    J[2][1] = fma(r.z, d.z, J[2][1]);
    J[2][2] = fma(r.z, d.w, J[2][2]);
  }
  R c[3][3];
#pragma unroll
  for (int m = 0; m < 3; ++m) {
    const int m1 = (m + 1) % 3, m2 = (m + 2) % 3;
    c[m][0] = J[1][m1] * J[2][m2] - J[2][m1] * J[1][m2];
    c[m][1] = J[2][m1] * J[0][m2] - J[0][m1] * J[2][m2];
    c[m][2] = J[0][m1] * J[1][m2] - J[1][m1] * J[0][m2];
  }
  const R det = J[0][0] * c[0][0] + J[1][0] * c[0][1] + J[2][0] * c[0][2];
  const R s = fabs(det);
  const R wq = (R)w64[q];
  const R f = wq * rcp_(s);
  R H[6];
  int h = 0;
#pragma unroll
  for (int m = 0; m < 3; ++m)
#pragma unroll
    for (int k = m; k < 3; ++k) H[h++] = f * (c[m][0] * c[k][0] + c[m][1] * c[k][1] + c[m][2] * c[k][2]);
  R tr = 0;
#pragma unroll
  for (int ii = 0; ii < 3; ++ii)
#pragma unroll
    for (int m = 0; m < 3; ++m) tr = fma(J[ii][m], J[ii][m], tr);
  tr *= (R)(1.0 / 3.0);
  const R quality = (s * s) * rcp_(tr * tr * tr);
  bad |= !(s > (R)0) || !isfinite(s) || !(quality > (sizeof(R) == 8 ? (R)1e-28 : (R)1e-12));
  if constexpr (sizeof(R) == 4) redo |= quality < (R)a.qmin;
  R cq = (R)0;
  if (a.which & LFEM_CMASS)
    cq = a.coef_f32 ? (R)__ldg(static_cast<const float*>(a.coef) + e * Q + q)
                    : (R)__ldg(static_cast<const double*>(a.coef) + e * Q + q);
  geo[2 * q] = V4<R>{wq * s, H[0], H[1], H[2]};
  geo[2 * q + 1] = V4<R>{H[3], H[4], H[5], cq};
}

// list == nullptr: every element; else the list[0 .. *list_n) (FP64 recomputation).
// flags (float pass only): flags[0] counts, flags[1 ..] lists the elements to redo.
template <int P, typename R, typename RS>
__global__ void __launch_bounds__(kTetHighWarps * 32) k_tet_high(const TwoPassArgs a, const V4<R>* __restrict__ gtab,
                                                                 const uint32_t* __restrict__ list,
                                                                 const uint32_t* __restrict__ list_n,
                                                                 uint32_t* __restrict__ flags) {
  constexpr int REF = TetHigh<P>::REF, U = TetHigh<P>::U, ROW = TetHigh<P>::ROW;
  const int Q = a.tab.q;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V4<R>* tab = reinterpret_cast<V4<R>*>(smem_raw);  // [Q][ROW]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  V4<R>* rel = tab + Q * ROW + warp * (2 * REF + 2 * Q);  // [REF] x_b - x_0
  V4<R>* hb = rel + REF;                                 // [REF] per-point node factors
  V4<R>* geo = hb + REF;                                 // [Q][2] (w s, H00, H01, H02), (H11, H12, H22, c_q)
  // the basis rows of every point in their row_slot order (padding unused)
  for (int t = threadIdx.x; t < Q * REF; t += blockDim.x) {
    const int q = t / REF, b = t - q * REF;
    tab[q * ROW + TetHigh<P>::row_slot(b)] = gtab[q * ROW + b];
  }
  __syncthreads();
  const double* w64 = bank<double>() + a.tab.off64;
  int r0, c0;  // this lane's register block
  tet_high_block<P>(lane, r0, c0);
  const int64_t n_work = list ? (int64_t)*list_n : a.n_elem;
  // consecutive work items go to different CTAs first: a short list (the FP64
  // pass) then spreads over every SM's FP64 pipe instead of a few SMs' warps
  for (int64_t i = (int64_t)warp * gridDim.x + blockIdx.x; i < n_work; i += (int64_t)gridDim.x * kTetHighWarps) {
    const int64_t e = list ? (int64_t)list[1 + i] : i;
    const int32_t* cn = a.conn + e * REF;
    const int64_t n0 = __ldg(cn);
    const double x0 = __ldg(a.coords + 3 * n0), y0 = __ldg(a.coords + 3 * n0 + 1), z0 = __ldg(a.coords + 3 * n0 + 2);
    for (int b = lane; b < REF; b += 32) {
      const int64_t nb = __ldg(cn + b);
      rel[b] = V4<R>{(R)(__ldg(a.coords + 3 * nb) - x0), (R)(__ldg(a.coords + 3 * nb + 1) - y0),
                     (R)(__ldg(a.coords + 3 * nb + 2) - z0), (R)0};
    }
    __syncwarp();
    bool bad = false, redo = false;
    for (int q = lane; q < Q; q += 32) tet_high_point<P, R>(a, tab, rel, w64, e, q, geo, bad, redo);
    if constexpr (sizeof(R) == 4) {
      if (__any_sync(0xffffffffu, bad || redo)) {
        if (lane == 0) {
          flags[1 + atomicAdd(flags, 1u)] = (uint32_t)e;
          atomicAdd(a.fallback, 1ull);
        }
        __syncwarp();
        continue;
      }
    } else {
      if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(a.status, ST_DEGENERATE);
    }
    __syncwarp();
    // mixed (float) results [e][U][nm] for the interleaved slot gather, FP64 [e][nm][U]
    constexpr bool IL = sizeof(RS) == 4;
    const int ms = IL ? 1 : U, su = IL ? a.nm : 1;
    RS* dst = static_cast<RS*>(a.lbuf) + (size_t)e * a.nm * U;
    if ((a.which & LFEM_MASS) && (a.which & LFEM_STIFF)) {
      tet_high_pass<P, R, RS, 3>(tab, hb, geo, Q, lane, r0, c0, dst, dst + ms, su);
      dst += 2 * ms;
    } else if (a.which & LFEM_MASS) {
      tet_high_pass<P, R, RS, 0>(tab, hb, geo, Q, lane, r0, c0, dst, nullptr, su);
      dst += ms;
    } else if (a.which & LFEM_STIFF) {
      tet_high_pass<P, R, RS, 1>(tab, hb, geo, Q, lane, r0, c0, dst, nullptr, su);
      dst += ms;
    }
    if (a.which & LFEM_CMASS) tet_high_pass<P, R, RS, 2>(tab, hb, geo, Q, lane, r0, c0, dst, nullptr, su);
  }
}

// The elements the float pass listed (list[0] of them, from list[1]) again in
// FP64, one CTA per element: the CTA computes the geometry of every point, each
// warp sums its register blocks over the points w, w + kTetHighWarps, ..., and
// warp 0 adds the other warps' partial blocks in warp order (fixed, so
// reruns are bit-identical).  Four warps per element keep the SM's FP64 pipe
// busy where one warp's dependent chains would leave it idle.
template <int P, int MODE>
__device__ __forceinline__ void tet_high_list_pass(const V4<double>* tab, V4<double>* hb, const V4<double>* geo, int Q,
                                                   int warp, int lane, int r0, int c0, double* part, float* dst,
                                                   float* dst2, int su) {
  constexpr int RA = TetHigh<P>::RA, RB = TetHigh<P>::RB, NB = RA * RB;
  double acc[RA][RB], accm[RA][RB];
  tet_high_accumulate<P, double, MODE>(tab, hb, geo, Q, warp, kTetHighWarps, lane, r0, c0, acc, accm);
  if (warp > 0) {
    double* pw = part + (size_t)(warp - 1) * 2 * NB * 32;
#pragma unroll
    for (int k = 0; k < NB; ++k) {
      pw[k * 32 + lane] = acc[k / RB][k % RB];
      pw[(NB + k) * 32 + lane] = accm[k / RB][k % RB];
    }
  }
  __syncthreads();
  if (warp == 0) {
    for (int w = 1; w < kTetHighWarps; ++w) {
      const double* pw = part + (size_t)(w - 1) * 2 * NB * 32;
#pragma unroll
      for (int k = 0; k < NB; ++k) {
        acc[k / RB][k % RB] += pw[k * 32 + lane];
        accm[k / RB][k % RB] += pw[(NB + k) * 32 + lane];
      }
    }
    tet_high_store<P, double, float, MODE>(r0, c0, acc, accm, dst, dst2, su);
  }
  __syncthreads();
}

template <int P>
__global__ void __launch_bounds__(kTetHighWarps * 32) k_tet_high_list(const TwoPassArgs a,
                                                                      const V4<double>* __restrict__ gtab,
                                                                      const uint32_t* __restrict__ list) {
  constexpr int REF = TetHigh<P>::REF, U = TetHigh<P>::U, ROW = TetHigh<P>::ROW;
  const int Q = a.tab.q;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V4<double>* tab = reinterpret_cast<V4<double>*>(smem_raw);  // [Q][ROW]
  V4<double>* rel = tab + (size_t)Q * ROW;                    // [REF] x_b - x_0
  V4<double>* geo = rel + REF;                                // [Q][2]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  V4<double>* hb = geo + 2 * Q + warp * REF;                               // per warp [REF]
  double* part = reinterpret_cast<double*>(geo + 2 * Q + kTetHighWarps * REF);  // [warps - 1][2 RA RB][32]
  __shared__ int s_bad;
  for (int t = threadIdx.x; t < Q * REF; t += blockDim.x) {
    const int q = t / REF, b = t - q * REF;
    tab[q * ROW + TetHigh<P>::row_slot(b)] = gtab[q * ROW + b];
  }
  const double* w64 = bank<double>() + a.tab.off64;
  int r0, c0;
  tet_high_block<P>(lane, r0, c0);
  const int64_t n_work = list[0];
  for (int64_t i = blockIdx.x; i < n_work; i += gridDim.x) {
    const int64_t e = list[1 + i];
    const int32_t* cn = a.conn + e * REF;
    const int64_t n0 = __ldg(cn);
    __syncthreads();  // the table is staged; the previous element has left rel and geo
    if (threadIdx.x == 0) s_bad = 0;
    for (int b = threadIdx.x; b < REF; b += blockDim.x) {
      const int64_t nb = __ldg(cn + b);
      rel[b] = V4<double>{__ldg(a.coords + 3 * nb) - __ldg(a.coords + 3 * n0),
                          __ldg(a.coords + 3 * nb + 1) - __ldg(a.coords + 3 * n0 + 1),
                          __ldg(a.coords + 3 * nb + 2) - __ldg(a.coords + 3 * n0 + 2), 0.0};
    }
    __syncthreads();
    bool bad = false, redo = false;
    for (int q = threadIdx.x; q < Q; q += blockDim.x) tet_high_point<P, double>(a, tab, rel, w64, e, q, geo, bad, redo);
    if (bad) s_bad = 1;
    __syncthreads();
    if (threadIdx.x == 0 && s_bad) atomicOr(a.status, ST_DEGENERATE);
    // [e][U][nm], as the float pass writes it
    const int su = a.nm;
    float* dst = static_cast<float*>(a.lbuf) + (size_t)e * a.nm * U;
    if ((a.which & LFEM_MASS) && (a.which & LFEM_STIFF)) {
      tet_high_list_pass<P, 3>(tab, hb, geo, Q, warp, lane, r0, c0, part, dst, dst + 1, su);
      dst += 2;
    } else if (a.which & LFEM_MASS) {
      tet_high_list_pass<P, 0>(tab, hb, geo, Q, warp, lane, r0, c0, part, dst, nullptr, su);
      dst += 1;
    } else if (a.which & LFEM_STIFF) {
      tet_high_list_pass<P, 1>(tab, hb, geo, Q, warp, lane, r0, c0, part, dst, nullptr, su);
      dst += 1;
    }
    if (a.which & LFEM_CMASS) tet_high_list_pass<P, 2>(tab, hb, geo, Q, warp, lane, r0, c0, part, dst, nullptr, su);
  }
}

template <int P>
static size_t tet_high_list_smem(int Q) {
  constexpr int REF = TetHigh<P>::REF, NB = TetHigh<P>::RA * TetHigh<P>::RB;
  return sizeof(V4<double>) * ((size_t)Q * TetHigh<P>::ROW + REF + 2 * (size_t)Q + (size_t)kTetHighWarps * REF) +
         sizeof(double) * (size_t)(kTetHighWarps - 1) * 2 * NB * 32;
}

template <int P>
static lfem_status launch_tet_high_list(const TwoPassArgs& a, const V4<double>* gtab, const uint32_t* list, int sms,
                                        cudaStream_t st) {
  const size_t smem = tet_high_list_smem<P>(a.tab.q);
  auto kern = k_tet_high_list<P>;
  LFEM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int occ = 0;
  LFEM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kTetHighWarps * 32, smem));
  if (occ < 1) return fail(LFEM_E_TOO_LARGE, "order-3/4 tet tables exceed shared memory");
  // the count is on the device: one CTA per SM and element, grid-strided beyond
  kern<<<(unsigned)sms, kTetHighWarps * 32, smem, st>>>(a, gtab, list);
  LFEM_CUDA(cudaGetLastError());
  return LFEM_OK;
}

template <int P, typename R>
static size_t tet_high_smem(int Q) {
  return sizeof(V4<R>) * ((size_t)Q * TetHigh<P>::ROW + (size_t)kTetHighWarps * (2 * TetHigh<P>::REF + 2 * Q));
}

template <int P, typename R, typename RS>
static lfem_status launch_tet_high_pass(const TwoPassArgs& a, const V4<R>* gtab, const uint32_t* list,
                                        uint32_t* flags, int64_t n, int sms, cudaStream_t st) {
  const size_t smem = tet_high_smem<P, R>(a.tab.q);
  auto kern = k_tet_high<P, R, RS>;
  LFEM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int occ = 0;
  LFEM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kTetHighWarps * 32, smem));
  if (occ < 1) return fail(LFEM_E_TOO_LARGE, "order-3/4 tet tables exceed shared memory");
  int64_t g = (n + kTetHighWarps - 1) / kTetHighWarps;
  if (g > (int64_t)sms * occ) g = (int64_t)sms * occ;
  if (g < 1) g = 1;
  kern<<<(unsigned)g, kTetHighWarps * 32, smem, st>>>(a, gtab, list, list, flags);
  LFEM_CUDA(cudaGetLastError());
  return LFEM_OK;
}

template <int P>
static lfem_status run_tet_high_p(bool mixed, const TwoPassArgs& a, void* scratch, int sms, cudaStream_t st) {
  constexpr int REF = TetHigh<P>::REF, U = TetHigh<P>::U, ROW = TetHigh<P>::ROW;
  const int Q = a.tab.q;
  V4<double>* t64 = static_cast<V4<double>*>(scratch);
  V4<float>* t32 = reinterpret_cast<V4<float>*>(t64 + (size_t)Q * ROW);
  uint32_t* flags = reinterpret_cast<uint32_t*>(t32 + (size_t)Q * ROW);
  if (a.n_elem > 0) {
    k_tet_high_table<P><<<(Q * REF + 127) / 128, 128, 0, st>>>(a.tab, t64, t32);
    LFEM_CUDA(cudaGetLastError());
    lfem_status s;
    if (mixed) {
      LFEM_CUDA(cudaMemsetAsync(flags, 0, sizeof(uint32_t), st));
      if ((s = launch_tet_high_pass<P, float, float>(a, t32, nullptr, flags, a.n_elem, sms, st)) != LFEM_OK) return s;
      // the listed elements again in FP64, a CTA per element
      if ((s = launch_tet_high_list<P>(a, t64, flags, sms, st)) != LFEM_OK) return s;
    } else if ((s = launch_tet_high_pass<P, double, double>(a, t64, nullptr, nullptr, a.n_elem, sms, st)) != LFEM_OK) {
      return s;
    }
  }
  if (a.nnz > 0) {
    int64_t g = (a.nnz + 255) / 256;
    if (g > (int64_t)sms * 16) g = (int64_t)sms * 16;
    if (!mixed) k_slot_gather<U, double><<<(unsigned)g, 256, 0, st>>>(a);
    else if (a.nm == 1) k_slot_gather_il<1><<<(unsigned)g, 256, 0, st>>>(a);
    else if (a.nm == 2) k_slot_gather_il<2><<<(unsigned)g, 256, 0, st>>>(a);
    else k_slot_gather_il<3><<<(unsigned)g, 256, 0, st>>>(a);
    LFEM_CUDA(cudaGetLastError());
  }
  return LFEM_OK;
}

// Load vector of order-3/4 tets, one warp per element (FP64): lanes over the
// points compute w_q s_q f_h(x_q), f_h = sum_b f_b phi_b; lanes over the nodes
// then sum loc_a = sum_q (w s f_h)_q phi_a(q) (Sec. 2, b = M f).
template <int P>
__global__ void __launch_bounds__(kTetHighWarps * 32) k_tet_high_load(const VecArgs a, const V4<double>* __restrict__ gtab) {
  constexpr int REF = TetHigh<P>::REF, ROW = TetHigh<P>::ROW;
  const int Q = a.tab.q;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V4<double>* tab = reinterpret_cast<V4<double>*>(smem_raw);  // [Q][ROW]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  V4<double>* rel = tab + Q * ROW + warp * (REF + (REF + Q + 3) / 4);
  double* fv = reinterpret_cast<double*>(rel + REF);  // [REF] nodal values, then [Q] point factors
  double* fq = fv + REF;
  for (int t = threadIdx.x; t < Q * ROW; t += blockDim.x) tab[t] = gtab[t];
  __syncthreads();
  const double* w64 = bank<double>() + a.tab.off64;
  for (int64_t e = (int64_t)blockIdx.x * kTetHighWarps + warp; e < a.n_elem; e += (int64_t)gridDim.x * kTetHighWarps) {
    const int32_t* cn = a.conn + e * REF;
    const int64_t n0 = __ldg(cn);
    const double x0 = __ldg(a.coords + 3 * n0), y0 = __ldg(a.coords + 3 * n0 + 1), z0 = __ldg(a.coords + 3 * n0 + 2);
    for (int b = lane; b < REF; b += 32) {
      const int64_t nb = __ldg(cn + b);
      rel[b] = V4<double>{__ldg(a.coords + 3 * nb) - x0, __ldg(a.coords + 3 * nb + 1) - y0,
                          __ldg(a.coords + 3 * nb + 2) - z0, 0.0};
      fv[b] = __ldg(a.u + nb);
    }
    __syncwarp();
    for (int q = lane; q < Q; q += 32) {
      const V4<double>* tq = tab + q * ROW;
      double J[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
      double fh = 0.0;
      for (int b = 0; b < REF; ++b) {
        const V4<double> r = rel[b], d = tq[b];
        fh = fma(fv[b], d.x, fh);
        J[0][0] = fma(r.x, d.y, J[0][0]);
        J[0][1] = fma(r.x, d.z, J[0][1]);
        J[0][2] = fma(r.x, d.w, J[0][2]);
        J[1][0] = fma(r.y, d.y, J[1][0]);
        J[1][1] = fma(r.y, d.z, J[1][1]);
        J[1][2] = fma(r.y, d.w, J[1][2]);
        J[2][0] = fma(r.z, d.y, J[2][0]);
        J[2][1] = fma(r.z, d.z, J[2][1]);
        J[2][2] = fma(r.z, d.w, J[2][2]);
      }
      const double det = J[0][0] * (J[1][1] * J[2][2] - J[2][1] * J[1][2]) -
                         J[1][0] * (J[0][1] * J[2][2] - J[2][1] * J[0][2]) +
                         J[2][0] * (J[0][1] * J[1][2] - J[1][1] * J[0][2]);
      fq[q] = w64[q] * fabs(det) * fh;
    }
    __syncwarp();
    for (int b = lane; b < REF; b += 32) {
      double acc = 0.0;
      for (int q = 0; q < Q; ++q) acc = fma(fq[q], tab[q * ROW + b].x, acc);
      a.loc[e * REF + b] = acc;
    }
    __syncwarp();
  }
}

template <int P>
static lfem_status run_tet_high_load_p(const VecArgs& a, void* scratch, int sms, cudaStream_t st) {
  constexpr int REF = TetHigh<P>::REF, ROW = TetHigh<P>::ROW;
  const int Q = a.tab.q;
  V4<double>* t64 = static_cast<V4<double>*>(scratch);
  V4<float>* t32 = reinterpret_cast<V4<float>*>(t64 + (size_t)Q * ROW);
  if (a.n_elem > 0) {
    k_tet_high_table<P><<<(Q * REF + 127) / 128, 128, 0, st>>>(a.tab, t64, t32);
    LFEM_CUDA(cudaGetLastError());
    const size_t smem = sizeof(V4<double>) * ((size_t)Q * ROW + (size_t)kTetHighWarps * (REF + (REF + Q + 3) / 4));
    auto kern = k_tet_high_load<P>;
    LFEM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int occ = 0;
    LFEM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kTetHighWarps * 32, smem));
    if (occ < 1) return fail(LFEM_E_TOO_LARGE, "order-3/4 tet tables exceed shared memory");
    int64_t g = (a.n_elem + kTetHighWarps - 1) / kTetHighWarps;
    if (g > (int64_t)sms * occ) g = (int64_t)sms * occ;
    kern<<<(unsigned)g, kTetHighWarps * 32, smem, st>>>(a, t64);
    LFEM_CUDA(cudaGetLastError());
  }
  return run_vec_gather(a, REF, 1, st);
}

lfem_status run_tet_high_load(int P, const VecArgs& a, void* scratch, int sms, cudaStream_t st) {
  if (P == 3) return run_tet_high_load_p<3>(a, scratch, sms, st);
  if (P == 4) return run_tet_high_load_p<4>(a, scratch, sms, st);
  return fail(LFEM_E_UNSUPPORTED, "element type");
}

size_t tet_high_scratch_bytes(int P, int Q, int64_t n_elem) {
  const int ROW = P == 3 ? TetHigh<3>::ROW : TetHigh<4>::ROW;
  return (size_t)Q * ROW * (sizeof(V4<double>) + sizeof(V4<float>)) + sizeof(uint32_t) * ((size_t)n_elem + 1);
}

lfem_status run_tet_high(int P, bool mixed, const TwoPassArgs& a, void* scratch, int sms, cudaStream_t st) {
  if (P == 3) return run_tet_high_p<3>(mixed, a, scratch, sms, st);
  if (P == 4) return run_tet_high_p<4>(mixed, a, scratch, sms, st);
  return fail(LFEM_E_UNSUPPORTED, "element type");
}

lfem_status bank_upload_tet_high(const void* src, size_t bytes, size_t offset) {
  LFEM_CUDA(cudaMemcpyToSymbol(c_bank, src, bytes, offset, cudaMemcpyHostToDevice));
  return LFEM_OK;
}

}  // namespace lfem
