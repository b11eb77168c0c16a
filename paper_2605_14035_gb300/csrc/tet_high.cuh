// Shared pieces of the order-3/4 kernels (tets: assembly, load vector; all
// element types: the adjoint): the warp-per-element sizes, a 4-wide row type
// and the device tabulation of the order-p tetrahedron basis.
#pragma once

#include "lfem_internal.cuh"

namespace lfem {

constexpr int kTetHighWarps = 4;

template <int P>
struct TetHigh {
  static constexpr int REF = (P + 1) * (P + 2) * (P + 3) / 6;
  static constexpr int U = REF * (REF + 1) / 2;
  // register blocks of the matrix, one per lane (blocks on or above the diagonal)
  static constexpr int RA = P == 3 ? 4 : 5, RB = P == 3 ? 2 : 5;
  static constexpr int NRB = REF / RA, NCB = REF / RB;
  static_assert(NRB * RA == REF && NCB * RB == REF, "blocks tile the matrix");
  // table row stride in 16-byte units, odd: lanes reading rows of different
  // points (the geometry phase) then fall on distinct banks
  static constexpr int ROW = REF | 1;
  // shared-memory slot of basis row r (r = RA blk + i -> i NRB + blk) and of
  // node factor c (c = RB cb + j -> j NCB + cb): the lanes' block rows r0 + i
  // (and columns c0 + j) are then consecutive 16-byte slots, free of bank
  // conflicts, instead of RA (RB) rows apart
  __host__ __device__ static constexpr int row_slot(int r) { return (r % RA) * NRB + r / RA; }
  __host__ __device__ static constexpr int col_slot(int c) { return (c % RB) * NCB + c / RB; }
};

template <typename R>
struct alignas(4 * sizeof(R) > 16 ? 16 : 4 * sizeof(R)) V4 {
  R x, y, z, w;
};

// Barycentric multi-index of local node a (library node order): corners;
// edges (0,1), (1,2), (2,0), (0,3), (1,3), (2,3), each from its first corner
// towards its second; faces (0,1,2), (0,1,3), (0,2,3), (1,2,3), each face
// (i, j, l) by increasing (alpha_j, alpha_l); interior nodes by increasing
// (alpha_1, alpha_2, alpha_3).
__device__ inline void tet_node_alpha(int p, int a, int (&al)[4]) {
  const int E[6][2] = {{0, 1}, {1, 2}, {2, 0}, {0, 3}, {1, 3}, {2, 3}};
  const int F[4][3] = {{0, 1, 2}, {0, 1, 3}, {0, 2, 3}, {1, 2, 3}};
  al[0] = al[1] = al[2] = al[3] = 0;
  if (a < 4) {
    al[a] = p;
    return;
  }
  int r = a - 4;
  if (r < 6 * (p - 1)) {
    const int k = r / (p - 1), t = r % (p - 1) + 1;
    al[E[k][0]] = p - t;
    al[E[k][1]] = t;
    return;
  }
  r -= 6 * (p - 1);
  const int nf = (p - 1) * (p - 2) / 2;
  if (r < 4 * nf) {
    const int f = r / nf;
    int t = r % nf;
    for (int aj = 1; aj < p; ++aj)
      for (int al2 = 1; aj + al2 < p; ++al2)
        if (t-- == 0) {
          al[F[f][0]] = p - aj - al2;
          al[F[f][1]] = aj;
          al[F[f][2]] = al2;
          return;
        }
  }
  r -= 4 * nf;
  for (int a1 = 1; a1 < p; ++a1)
    for (int a2 = 1; a1 + a2 < p; ++a2)
      for (int a3 = 1; a1 + a2 + a3 < p; ++a3)
        if (r-- == 0) {
          al[0] = p - a1 - a2 - a3;
          al[1] = a1;
          al[2] = a2;
          al[3] = a3;
          return;
        }
}

// phi_alpha = prod_i l_{alpha_i}(lambda_i) with l_k(t) = prod_{j<k} (p t - j) / (j + 1):
// value and derivative of one factor.
__device__ __forceinline__ void lagrange_1d(int p, int k, double t, double& v, double& dv) {
  v = 1.0;
  dv = 0.0;
  for (int j = 0; j < k; ++j) {
    const double inv = 1.0 / (double)(j + 1);
    const double f = ((double)p * t - (double)j) * inv;
    dv = fma(dv, f, v * ((double)p * inv));
    v *= f;
  }
}

// table[q][b] = (phi_b, d phi_b / d xi_1, d xi_2, d xi_3) at point q, in FP64 and
// float; rows ROW apart (the padding entries are never read).
template <int P>
__global__ void k_tet_high_table(TabRef rule_ref, V4<double>* __restrict__ t64, V4<float>* __restrict__ t32) {
  constexpr int REF = TetHigh<P>::REF;
  const int Q = rule_ref.q;
  const double* rule = bank<double>() + rule_ref.off64;  // w[Q], then xi[Q][3]
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < Q * REF; t += gridDim.x * blockDim.x) {
    const int q = t / REF, b = t - q * REF;
    int al[4];
    tet_node_alpha(P, b, al);
    const double x1 = rule[Q + 3 * q], x2 = rule[Q + 3 * q + 1], x3 = rule[Q + 3 * q + 2];
    const double lam[4] = {1.0 - (x1 + x2 + x3), x1, x2, x3};
    double v[4], dv[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) lagrange_1d(P, al[i], lam[i], v[i], dv[i]);
    // d phi / d lambda_i, then the chain rule with lambda_0 = 1 - xi_1 - xi_2 - xi_3
    const double d0 = dv[0] * v[1] * v[2] * v[3], d1 = v[0] * dv[1] * v[2] * v[3];
    const double d2 = v[0] * v[1] * dv[2] * v[3], d3 = v[0] * v[1] * v[2] * dv[3];
    const V4<double> r{v[0] * v[1] * v[2] * v[3], d1 - d0, d2 - d0, d3 - d0};
    t64[q * TetHigh<P>::ROW + b] = r;
    t32[q * TetHigh<P>::ROW + b] = V4<float>{(float)r.x, (float)r.y, (float)r.z, (float)r.w};
  }
}

}  // namespace lfem
