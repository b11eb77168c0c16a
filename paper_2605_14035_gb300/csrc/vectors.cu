// Vector assembly on the same pattern: the load vector of the Poisson problem
// (Sec. 2: b_j = integral of f_h phi_j with f_h the interpolant of nodal
// values, so b = M f) and the non-linear vectors of the mean curvature flow
// system (Sec. 5.1: integrals of |grad_Gamma nu_h|^2 (nu_h)_k phi_j and of
// |grad_Gamma nu_h|^2 H_h phi_j for u = (nu, H) at the nodes).  FP64.
//
// Two passes, deterministic and atomic-free like the matrices: every element
// once (its local vector into a scratch buffer [nE][ref][nc]), then every node
// sums its incidences in ascending element order.
#include "dispatch.cuh"

namespace lfem {


// KIND 0: load vector (nc = 1); KIND 1: mean-curvature-flow vectors (nc = 4, surfaces).
template <int D, int NA, int P, int KIND>
__global__ void __launch_bounds__(128) k_vec_local(const VecArgs a) {
  constexpr int REF = Ref<D, P>::REF;
  constexpr int NC = KIND == 0 ? 1 : 4;
  const TabView<double> tb = tab_view<D, P, double>(a.tab);
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < a.n_elem;
       e += (int64_t)gridDim.x * blockDim.x) {
    int32_t nodes[REF];
#pragma unroll
    for (int b = 0; b < REF; ++b) nodes[b] = __ldg(a.conn + e * REF + b);
    double X[REF][NA];
    gather_coords<D, NA, P>(a.coords, nodes, X);
    ElemData<D, NA, P, double> ed;
    load_element_data<D, NA, P, double>(X, ed);
    double U[REF][NC];
#pragma unroll
    for (int b = 0; b < REF; ++b)
#pragma unroll
      for (int c = 0; c < NC; ++c) U[b][c] = __ldg(a.u + (int64_t)nodes[b] * NC + c);
    double loc[REF][NC];
#pragma unroll
    for (int b = 0; b < REF; ++b)
#pragma unroll
      for (int c = 0; c < NC; ++c) loc[b][c] = 0.0;
    for (int q = 0; q < tb.q; ++q) {
      const double wq = tb.w[q];
      QpGeom<D, NA, P, double> g;
      qp_geometry<D, NA, P, double>(ed, tb, q, wq, g);
      const double* ph = tb.phi + q * REF;
      // values at the point
      double val[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        double v = 0.0;
#pragma unroll
        for (int b = 0; b < REF; ++b) v = fma(U[b][c], ph[b], v);
        val[c] = v;
      }
      double f;  // factor of val_c phi_a in the integrand, times w_q s_q
      if constexpr (KIND == 0) {
        f = wq * g.s;
      } else {
        // |grad_Gamma nu_h|^2 w s = sum_k g_k^T (w s G^{-1}) g_k, g_k = sum_b nu_bk grad^phi_b
        const double* dph = tb.dphi + q * REF * D;
        f = 0.0;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          double gk[D];
#pragma unroll
          for (int m = 0; m < D; ++m) {
            double v = 0.0;
#pragma unroll
            for (int b = 0; b < REF; ++b) v = fma(U[b][k], dph[b * D + m], v);
            gk[m] = v;
          }
#pragma unroll
          for (int m = 0; m < D; ++m)
#pragma unroll
            for (int n = 0; n < D; ++n) f = fma(gk[m], g.H[m][n] * gk[n], f);
        }
      }
#pragma unroll
      for (int b = 0; b < REF; ++b)
#pragma unroll
        for (int c = 0; c < NC; ++c) loc[b][c] = fma(f * val[c], ph[b], loc[b][c]);
    }
    double* dst = a.loc + e * REF * NC;
#pragma unroll
    for (int b = 0; b < REF; ++b)
#pragma unroll
      for (int c = 0; c < NC; ++c) dst[b * NC + c] = loc[b][c];
  }
}

// Node i: out[c][i] = sum over its incidences (e, a), ascending e, of loc[e][a][c].
template <int NC>
__global__ void __launch_bounds__(256) k_vec_gather(const VecArgs a, int ref) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n_nodes;
       i += (int64_t)gridDim.x * blockDim.x) {
    double s[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) s[c] = 0.0;
    const int32_t k0 = __ldg(a.inc_ptr + i), k1 = __ldg(a.inc_ptr + i + 1);
    for (int32_t k = k0; k < k1; ++k) {
      const int32_t key = __ldg(a.inc_key + k);
      const int64_t e = key >> a.key_shift;
      const int lidx = key & ((1 << a.key_shift) - 1);
      const double* l = a.loc + (e * ref + lidx) * NC;
#pragma unroll
      for (int c = 0; c < NC; ++c) s[c] += l[c];
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) a.out[(int64_t)c * a.n_nodes + i] = s[c];
  }
}

static unsigned vec_grid(int64_t n, int threads) {
  const int64_t g = (n + threads - 1) / threads;
  return (unsigned)(g < 152 * 32 ? (g > 0 ? g : 1) : 152 * 32);
}

lfem_status run_vec_gather(const VecArgs& a, int ref, int nc, cudaStream_t st) {
  if (a.n_nodes > 0) {
    if (nc == 1) k_vec_gather<1><<<vec_grid(a.n_nodes, 256), 256, 0, st>>>(a, ref);
    else if (nc == 4) k_vec_gather<4><<<vec_grid(a.n_nodes, 256), 256, 0, st>>>(a, ref);
    else return fail(LFEM_E_ARG, "vector components");
    LFEM_CUDA(cudaGetLastError());
  }
  return LFEM_OK;
}

template <int D, int NA, int P, int KIND>
static lfem_status launch_vec(const VecArgs& a, cudaStream_t st) {
  constexpr int NC = KIND == 0 ? 1 : 4;
  if (a.n_elem > 0) {
    k_vec_local<D, NA, P, KIND><<<vec_grid(a.n_elem, 128), 128, 0, st>>>(a);
    LFEM_CUDA(cudaGetLastError());
  }
  return run_vec_gather(a, Ref<D, P>::REF, NC, st);
}

template <int D, int NA, int P>
static lfem_status launch_kind(int kind, const VecArgs& a, cudaStream_t st) {
  if (kind == 0) return launch_vec<D, NA, P, 0>(a, st);
  if constexpr (D == 2 && NA == 3) return launch_vec<D, NA, P, 1>(a, st);
  return fail(LFEM_E_UNSUPPORTED, "the non-linear vectors need a surface (dim 2 in R^3)");
}

lfem_status run_vectors(int D, int NA, int P, int kind, const VecArgs& a, cudaStream_t st) {
#define LFEM_VEC_CASE(DD, NN, PP) \
  if (D == DD && NA == NN && P == PP) return launch_kind<DD, NN, PP>(kind, a, st);
  LFEM_VEC_CASE(1, 1, 1)
  LFEM_VEC_CASE(1, 1, 2)
  LFEM_VEC_CASE(1, 2, 1)
  LFEM_VEC_CASE(1, 2, 2)
  LFEM_VEC_CASE(1, 3, 1)
  LFEM_VEC_CASE(1, 3, 2)
  LFEM_VEC_CASE(2, 2, 1)
  LFEM_VEC_CASE(2, 2, 2)
  LFEM_VEC_CASE(2, 3, 1)
  LFEM_VEC_CASE(2, 3, 2)
  LFEM_VEC_CASE(3, 3, 1)
  LFEM_VEC_CASE(3, 3, 2)
  LFEM_VEC_CASE(1, 1, 3)
  LFEM_VEC_CASE(1, 1, 4)
  LFEM_VEC_CASE(1, 2, 3)
  LFEM_VEC_CASE(1, 2, 4)
  LFEM_VEC_CASE(1, 3, 3)
  LFEM_VEC_CASE(1, 3, 4)
  LFEM_VEC_CASE(2, 2, 3)
  LFEM_VEC_CASE(2, 2, 4)
  LFEM_VEC_CASE(2, 3, 3)
  LFEM_VEC_CASE(2, 3, 4)
#undef LFEM_VEC_CASE
  return fail(LFEM_E_UNSUPPORTED, "element type");
}

lfem_status bank_upload_vec(const void* src, size_t bytes, size_t offset) {
  LFEM_CUDA(cudaMemcpyToSymbol(c_bank, src, bytes, offset, cudaMemcpyHostToDevice));
  return LFEM_OK;
}

}  // namespace lfem
