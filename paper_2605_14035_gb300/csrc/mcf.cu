// One step of the classical evolving-surface scheme the paper's flow example
// starts from (Sec. 5.1, Dziuk's method for mean curvature flow):
//   (M(x^{n-1}) + tau A(x^{n-1})) x^n = M(x^{n-1}) x^{n-1},
// one linear system per coordinate, assembled on the pattern (FP64) and solved
// by a hand-written Jacobi-preconditioned conjugate gradient on the CSR
// values.  The n coordinate columns are solved together (one sparse
// product serves all of them).  Every reduction runs in a fixed order (per-block
// tree, then one block over the block sums), so the step is bit-reproducible.
#include "dispatch.cuh"

namespace lfem {

constexpr int kRedBlocks = 256;
constexpr int kRedThreads = 256;

// K = M + tau A on the pattern, and the inverse of K's diagonal.
__global__ void k_mcf_combine(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col_idx,
                              const double* __restrict__ M, const double* __restrict__ A, double tau, int32_t n,
                              double* __restrict__ K, double* __restrict__ dinv) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double d = 0.0;
    for (int64_t s = row_ptr[i]; s < row_ptr[i + 1]; ++s) {
      const double v = M[s] + tau * A[s];
      K[s] = v;
      if (col_idx[s] == i) d = v;
    }
    dinv[i] = d != 0.0 ? 1.0 / d : 1.0;  // empty rows (unreferenced nodes) keep their value
  }
}

// Y[i][c] = sum_j S_ij X[j][c], c < NC (rows in ascending column order).
template <int NC>
__global__ void k_mcf_spmv(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col_idx,
                           const double* __restrict__ S, const double* __restrict__ X, int32_t n,
                           double* __restrict__ Y) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double y[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) y[c] = 0.0;
    for (int64_t s = row_ptr[i]; s < row_ptr[i + 1]; ++s) {
      const double v = S[s];
      const double* x = X + (int64_t)col_idx[s] * NC;
#pragma unroll
      for (int c = 0; c < NC; ++c) y[c] = fma(v, x[c], y[c]);
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) Y[i * NC + c] = y[c];
  }
}

// Per-column dot products <A_c, B_c>, first stage: one partial per block.
template <int NC>
__global__ void __launch_bounds__(kRedThreads) k_mcf_dot_part(const double* __restrict__ A,
                                                              const double* __restrict__ B, int32_t n,
                                                              double* __restrict__ part) {
  __shared__ double sh[kRedThreads][NC];
  double acc[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) acc[c] = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[c] = fma(A[i * NC + c], B[i * NC + c], acc[c]);
#pragma unroll
  for (int c = 0; c < NC; ++c) sh[threadIdx.x][c] = acc[c];
  __syncthreads();
  for (int h = kRedThreads / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h)
#pragma unroll
      for (int c = 0; c < NC; ++c) sh[threadIdx.x][c] += sh[threadIdx.x + h][c];
    __syncthreads();
  }
  if (threadIdx.x == 0)
#pragma unroll
    for (int c = 0; c < NC; ++c) part[blockIdx.x * NC + c] = sh[0][c];
}

// Second stage (one block): out[c] = sum of the block partials in a fixed tree.
template <int NC>
__global__ void __launch_bounds__(kRedBlocks) k_mcf_dot_final(const double* __restrict__ part, double* __restrict__ out) {
  __shared__ double sh[kRedBlocks][NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) sh[threadIdx.x][c] = part[threadIdx.x * NC + c];
  __syncthreads();
  for (int h = kRedBlocks / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h)
#pragma unroll
      for (int c = 0; c < NC; ++c) sh[threadIdx.x][c] += sh[threadIdx.x + h][c];
    __syncthreads();
  }
  if (threadIdx.x == 0)
#pragma unroll
    for (int c = 0; c < NC; ++c) out[c] = sh[0][c];
}


// R = B - K X (K X in Q), Z = Dinv R, P = Z.
template <int NC>
__global__ void k_mcf_init(const double* __restrict__ B, const double* __restrict__ Q,
                           const double* __restrict__ dinv, int32_t n, double* __restrict__ R,
                           double* __restrict__ Z, double* __restrict__ P) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const double r = B[i * NC + c] - Q[i * NC + c];
      R[i * NC + c] = r;
      Z[i * NC + c] = dinv[i] * r;
      P[i * NC + c] = dinv[i] * r;
    }
}

// alpha = rz / pq; X += alpha P; R -= alpha Q; Z = Dinv R.
template <int NC>
__global__ void k_mcf_update_xr(const McfScalars* __restrict__ sc, const double* __restrict__ P,
                                const double* __restrict__ Q, const double* __restrict__ dinv, int32_t n,
                                double* __restrict__ X, double* __restrict__ R, double* __restrict__ Z) {
  double alpha[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) alpha[c] = sc->pq[c] != 0.0 ? sc->rz[c] / sc->pq[c] : 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      X[i * NC + c] = fma(alpha[c], P[i * NC + c], X[i * NC + c]);
      const double r = fma(-alpha[c], Q[i * NC + c], R[i * NC + c]);
      R[i * NC + c] = r;
      Z[i * NC + c] = dinv[i] * r;
    }
}

// beta = rz_new / rz; P = Z + beta P (rz <- rz_new happens in k_mcf_shift).
template <int NC>
__global__ void k_mcf_update_p(const McfScalars* __restrict__ sc, const double* __restrict__ Z, int32_t n,
                               double* __restrict__ P) {
  double beta[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) beta[c] = sc->rz[c] != 0.0 ? sc->rz_new[c] / sc->rz[c] : 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
#pragma unroll
    for (int c = 0; c < NC; ++c) P[i * NC + c] = fma(beta[c], P[i * NC + c], Z[i * NC + c]);
}

__global__ void k_mcf_shift(McfScalars* sc) {
  if (threadIdx.x < 3) sc->rz[threadIdx.x] = sc->rz_new[threadIdx.x];
}

static unsigned mcf_grid(int64_t n) {
  const int64_t g = (n + 255) / 256;
  return (unsigned)(g < 152 * 16 ? (g > 0 ? g : 1) : 152 * 16);
}

template <int NC>
static lfem_status mcf_dot(const double* a, const double* b, int32_t n, double* part, double* out, cudaStream_t st) {
  k_mcf_dot_part<NC><<<kRedBlocks, kRedThreads, 0, st>>>(a, b, n, part);
  k_mcf_dot_final<NC><<<1, kRedBlocks, 0, st>>>(part, out);
  LFEM_CUDA(cudaGetLastError());
  return LFEM_OK;
}

template <int NC>
static lfem_status mcf_solve(const McfSolveArgs& s, cudaStream_t st, int* iterations) {
  const int32_t n = s.n;
  const unsigned g = mcf_grid(n);
  McfScalars* sc = s.scalars;
  k_mcf_combine<<<g, 256, 0, st>>>(s.row_ptr, s.col_idx, s.M, s.A, s.tau, n, s.K, s.dinv);
  k_mcf_spmv<NC><<<g, 256, 0, st>>>(s.row_ptr, s.col_idx, s.M, s.X0, n, s.B);  // B = M x^{n-1}
  LFEM_CUDA(cudaMemcpyAsync(s.X, s.X0, sizeof(double) * (size_t)n * NC, cudaMemcpyDeviceToDevice, st));
  k_mcf_spmv<NC><<<g, 256, 0, st>>>(s.row_ptr, s.col_idx, s.K, s.X, n, s.Q);
  k_mcf_init<NC><<<g, 256, 0, st>>>(s.B, s.Q, s.dinv, n, s.R, s.Z, s.P);
  LFEM_CUDA(cudaGetLastError());
  lfem_status e;
  if ((e = mcf_dot<NC>(s.R, s.Z, n, s.part, sc->rz, st)) != LFEM_OK) return e;
  if ((e = mcf_dot<NC>(s.B, s.B, n, s.part, sc->bb, st)) != LFEM_OK) return e;
  McfScalars h{};
  int it = 0;
  const int check_every = 8;
  while (it < s.max_iter) {
    k_mcf_spmv<NC><<<g, 256, 0, st>>>(s.row_ptr, s.col_idx, s.K, s.P, n, s.Q);
    if ((e = mcf_dot<NC>(s.P, s.Q, n, s.part, sc->pq, st)) != LFEM_OK) return e;
    k_mcf_update_xr<NC><<<g, 256, 0, st>>>(sc, s.P, s.Q, s.dinv, n, s.X, s.R, s.Z);
    if ((e = mcf_dot<NC>(s.R, s.Z, n, s.part, sc->rz_new, st)) != LFEM_OK) return e;
    k_mcf_update_p<NC><<<g, 256, 0, st>>>(sc, s.Z, n, s.P);
    k_mcf_shift<<<1, 32, 0, st>>>(sc);
    LFEM_CUDA(cudaGetLastError());
    ++it;
    if (it % check_every == 0 || it == s.max_iter) {
      if ((e = mcf_dot<NC>(s.R, s.R, n, s.part, sc->rr, st)) != LFEM_OK) return e;
      LFEM_CUDA(cudaMemcpyAsync(&h, sc, sizeof(McfScalars), cudaMemcpyDeviceToHost, st));
      LFEM_CUDA(cudaStreamSynchronize(st));
      bool done = true;
      for (int c = 0; c < NC; ++c) done = done && (h.rr[c] <= s.rtol * s.rtol * h.bb[c]);
      if (done) break;
    }
  }
  *iterations = it;
  LFEM_CUDA(cudaMemcpyAsync(s.X_out, s.X, sizeof(double) * (size_t)n * NC, cudaMemcpyDeviceToDevice, st));
  return LFEM_OK;
}

lfem_status run_mcf_solve(int nc, const McfSolveArgs& s, cudaStream_t st, int* iterations) {
  if (nc == 2) return mcf_solve<2>(s, st, iterations);
  if (nc == 3) return mcf_solve<3>(s, st, iterations);
  return fail(LFEM_E_UNSUPPORTED, "mean curvature flow needs a curve or surface in R^2 or R^3");
}

}  // namespace lfem
