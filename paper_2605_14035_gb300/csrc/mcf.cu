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

constexpr int kMcfThreads = 256;

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

// ---- fixed-order reductions ------------------------------------------------
// Every kernel below runs kMcfBlocks blocks of kMcfThreads threads with the
// same grid-stride row assignment, so a block's partial of a dot product is
// always the same sum; a consumer reduces the kMcfBlocks partials itself, in
// one fixed order, so every block (and every run) gets the same scalar.

// The block's partial sums of acc[c] to part[blockIdx.x][c] (fixed tree).
template <int NC>
__device__ __forceinline__ void block_partial(const double (&acc)[NC], double* __restrict__ part) {
  __shared__ double sh[kMcfThreads][NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) sh[threadIdx.x][c] = acc[c];
  __syncthreads();
  for (int h = kMcfThreads / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h)
#pragma unroll
      for (int c = 0; c < NC; ++c) sh[threadIdx.x][c] += sh[threadIdx.x + h][c];
    __syncthreads();
  }
  if (threadIdx.x == 0)
#pragma unroll
    for (int c = 0; c < NC; ++c) part[blockIdx.x * NC + c] = sh[0][c];
}

// out[c] = the sum of the kMcfBlocks partials (thread t adds t, t + 256, ...,
// then a fixed tree); every thread of the block receives it.
template <int NC>
__device__ __forceinline__ void block_total(const double* __restrict__ part, double (&out)[NC]) {
  __shared__ double sh[kMcfThreads][NC];
  double a[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) a[c] = 0.0;
  for (int b = threadIdx.x; b < kMcfBlocks; b += kMcfThreads)
#pragma unroll
    for (int c = 0; c < NC; ++c) a[c] += part[b * NC + c];
#pragma unroll
  for (int c = 0; c < NC; ++c) sh[threadIdx.x][c] = a[c];
  __syncthreads();
  for (int h = kMcfThreads / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h)
#pragma unroll
      for (int c = 0; c < NC; ++c) sh[threadIdx.x][c] += sh[threadIdx.x + h][c];
    __syncthreads();
  }
#pragma unroll
  for (int c = 0; c < NC; ++c) out[c] = sh[0][c];
  __syncthreads();
}

// Partials of <A_c, B_c>.
template <int NC>
__global__ void __launch_bounds__(kMcfThreads) k_mcf_dot(const double* __restrict__ A, const double* __restrict__ B,
                                                         int32_t n, double* __restrict__ part) {
  double acc[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) acc[c] = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[c] = fma(A[i * NC + c], B[i * NC + c], acc[c]);
  block_partial<NC>(acc, part);
}

// One block: out[c] = the total of the partials.
template <int NC>
__global__ void __launch_bounds__(kMcfThreads) k_mcf_total(const double* __restrict__ part, double* __restrict__ out) {
  double t[NC];
  block_total<NC>(part, t);
  if (threadIdx.x == 0)
#pragma unroll
    for (int c = 0; c < NC; ++c) out[c] = t[c];
}

// R = B - K X (K X in Q), Z = Dinv R, P = Z; partials of <R, Z>.
template <int NC>
__global__ void __launch_bounds__(kMcfThreads) k_mcf_init(const double* __restrict__ B, const double* __restrict__ Q,
                                                          const double* __restrict__ dinv, int32_t n,
                                                          double* __restrict__ R, double* __restrict__ Z,
                                                          double* __restrict__ P, double* __restrict__ part_rz) {
  double acc[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) acc[c] = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const double r = B[i * NC + c] - Q[i * NC + c];
      const double z = dinv[i] * r;
      R[i * NC + c] = r;
      Z[i * NC + c] = z;
      P[i * NC + c] = z;
      acc[c] = fma(r, z, acc[c]);
    }
  block_partial<NC>(acc, part_rz);
}

// CG iteration, part 1: Q = K P and the partials of <P, Q> (a thread per
// row: with about a dozen entries per row, four lanes per row measured slower).
template <int NC>
__global__ void __launch_bounds__(kMcfThreads) k_cg_spmv_pq(const int64_t* __restrict__ row_ptr,
                                                            const int32_t* __restrict__ col_idx,
                                                            const double* __restrict__ K, const double* __restrict__ P,
                                                            int32_t n, double* __restrict__ Q,
                                                            double* __restrict__ part_pq) {
  double acc[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) acc[c] = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double y[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) y[c] = 0.0;
    for (int64_t s = row_ptr[i]; s < row_ptr[i + 1]; ++s) {
      const double v = K[s];
      const double* x = P + (int64_t)col_idx[s] * NC;
#pragma unroll
      for (int c = 0; c < NC; ++c) y[c] = fma(v, x[c], y[c]);
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      Q[i * NC + c] = y[c];
      acc[c] = fma(P[i * NC + c], y[c], acc[c]);
    }
  }
  block_partial<NC>(acc, part_pq);
}

// Part 2: alpha = rz / pq; X += alpha P; R -= alpha Q; Z = Dinv R; partials of <R, Z>.
template <int NC>
__global__ void __launch_bounds__(kMcfThreads) k_cg_xr(const double* __restrict__ part_rz,
                                                       const double* __restrict__ part_pq,
                                                       const double* __restrict__ P, const double* __restrict__ Q,
                                                       const double* __restrict__ dinv, int32_t n,
                                                       double* __restrict__ X, double* __restrict__ R,
                                                       double* __restrict__ Z, double* __restrict__ part_rz_new) {
  double rz[NC], pq[NC], alpha[NC], acc[NC];
  block_total<NC>(part_rz, rz);
  block_total<NC>(part_pq, pq);
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    alpha[c] = pq[c] != 0.0 ? rz[c] / pq[c] : 0.0;
    acc[c] = 0.0;
  }
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      X[i * NC + c] = fma(alpha[c], P[i * NC + c], X[i * NC + c]);
      const double r = fma(-alpha[c], Q[i * NC + c], R[i * NC + c]);
      const double z = dinv[i] * r;
      R[i * NC + c] = r;
      Z[i * NC + c] = z;
      acc[c] = fma(r, z, acc[c]);
    }
  block_partial<NC>(acc, part_rz_new);
}

// Part 3: beta = rz_new / rz; P = Z + beta P.
template <int NC>
__global__ void __launch_bounds__(kMcfThreads) k_cg_p(const double* __restrict__ part_rz,
                                                      const double* __restrict__ part_rz_new,
                                                      const double* __restrict__ Z, int32_t n,
                                                      double* __restrict__ P) {
  double rz[NC], rzn[NC], beta[NC];
  block_total<NC>(part_rz, rz);
  block_total<NC>(part_rz_new, rzn);
#pragma unroll
  for (int c = 0; c < NC; ++c) beta[c] = rz[c] != 0.0 ? rzn[c] / rz[c] : 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
#pragma unroll
    for (int c = 0; c < NC; ++c) P[i * NC + c] = fma(beta[c], P[i * NC + c], Z[i * NC + c]);
}

static unsigned mcf_grid(int64_t n) {
  const int64_t g = (n + 255) / 256;
  return (unsigned)(g < 152 * 16 ? (g > 0 ? g : 1) : 152 * 16);
}

// k CG iterations starting from the partial set `par` of <r, z> (k even: the
// set alternates, so it ends where it began).
template <int NC>
static lfem_status cg_iterations(const McfSolveArgs& s, int k, int par, cudaStream_t st) {
  const int32_t n = s.n;
  double* rz[2] = {s.part + 2 * kMcfBlocks * NC, s.part + 3 * kMcfBlocks * NC};
  double* pq = s.part;
  for (int j = 0; j < k; ++j) {
    const int a = (par + j) & 1, b = a ^ 1;
    k_cg_spmv_pq<NC><<<kMcfBlocks, kMcfThreads, 0, st>>>(s.row_ptr, s.col_idx, s.K, s.P, n, s.Q, pq);
    k_cg_xr<NC><<<kMcfBlocks, kMcfThreads, 0, st>>>(rz[a], pq, s.P, s.Q, s.dinv, n, s.X, s.R, s.Z, rz[b]);
    k_cg_p<NC><<<kMcfBlocks, kMcfThreads, 0, st>>>(rz[a], rz[b], s.Z, n, s.P);
  }
  LFEM_CUDA(cudaGetLastError());
  return LFEM_OK;
}

template <int NC>
static lfem_status mcf_solve(const McfSolveArgs& s, cudaStream_t st, int* iterations) {
  const int32_t n = s.n;
  const unsigned g = mcf_grid(n);
  McfScalars* sc = s.scalars;
  double* part_tmp = s.part + kMcfBlocks * NC;  // rr / bb partials
  double* rz0 = s.part + 2 * kMcfBlocks * NC;
  k_mcf_combine<<<g, 256, 0, st>>>(s.row_ptr, s.col_idx, s.M, s.A, s.tau, n, s.K, s.dinv);
  k_mcf_spmv<NC><<<g, 256, 0, st>>>(s.row_ptr, s.col_idx, s.M, s.X0, n, s.B);  // B = M x^{n-1}
  LFEM_CUDA(cudaMemcpyAsync(s.X, s.X0, sizeof(double) * (size_t)n * NC, cudaMemcpyDeviceToDevice, st));
  k_mcf_spmv<NC><<<g, 256, 0, st>>>(s.row_ptr, s.col_idx, s.K, s.X, n, s.Q);
  k_mcf_init<NC><<<kMcfBlocks, kMcfThreads, 0, st>>>(s.B, s.Q, s.dinv, n, s.R, s.Z, s.P, rz0);
  k_mcf_dot<NC><<<kMcfBlocks, kMcfThreads, 0, st>>>(s.B, s.B, n, part_tmp);
  k_mcf_total<NC><<<1, kMcfThreads, 0, st>>>(part_tmp, sc->bb);
  LFEM_CUDA(cudaGetLastError());
  lfem_status e;
  McfScalars h{};
  int it = 0;
  const int check_every = 8;  // even: the <r, z> partial sets alternate back to rz0
  // the 8-iteration block as a CUDA graph, captured once per scratch layout
  // (needs a stream that can be captured: not the legacy default stream)
  McfGraph& gc = *s.graph;
  const bool use_graph = st != nullptr;
  if (use_graph && (gc.exec == nullptr || gc.buf != s.part || gc.n != n || gc.nc != NC || gc.K != s.K)) {
    if (gc.exec) cudaGraphExecDestroy(gc.exec);
    gc.exec = nullptr;
    LFEM_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    e = cg_iterations<NC>(s, check_every, 0, st);
    cudaGraph_t graph = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(st, &graph);
    if (e != LFEM_OK) {
      if (graph) cudaGraphDestroy(graph);
      return e;
    }
    if (ce != cudaSuccess) return cuda_fail(ce, "cudaStreamEndCapture");
    const cudaError_t ie = cudaGraphInstantiate(&gc.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) {
      gc.exec = nullptr;
      return cuda_fail(ie, "cudaGraphInstantiate");
    }
    gc.buf = s.part;
    gc.n = n;
    gc.nc = NC;
    gc.K = s.K;
  }
  while (it < s.max_iter) {
    const int k = s.max_iter - it < check_every ? s.max_iter - it : check_every;
    if (use_graph && k == check_every) {
      LFEM_CUDA(cudaGraphLaunch(gc.exec, st));
    } else if ((e = cg_iterations<NC>(s, k, 0, st)) != LFEM_OK) {
      return e;
    }
    it += k;
    k_mcf_dot<NC><<<kMcfBlocks, kMcfThreads, 0, st>>>(s.R, s.R, n, part_tmp);
    k_mcf_total<NC><<<1, kMcfThreads, 0, st>>>(part_tmp, sc->rr);
    LFEM_CUDA(cudaGetLastError());
    LFEM_CUDA(cudaMemcpyAsync(&h, sc, sizeof(McfScalars), cudaMemcpyDeviceToHost, st));
    LFEM_CUDA(cudaStreamSynchronize(st));
    bool done = true;
    for (int c = 0; c < NC; ++c) done = done && (h.rr[c] <= s.rtol * s.rtol * h.bb[c]);
    if (done) break;
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
