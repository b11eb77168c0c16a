// Adjoint of the assembly for orders 3 and 4 (curves, triangles, tets), FP64:
// dL/d(CSR values) -> dL/d(node coordinates) and dL/d(coefficient at the
// points), the same derivative as the order-1/2 tile kernel (variation of s
// and of s G^{-1} under dJ):
//   m_q   = sum_ab (GM_ab + c_q GC_ab) phi_a phi_b,   mc_q = sum_ab GC_ab phi_a phi_b
//   K_q   = sym(sum_ab GA_ab grad^phi_a grad^phi_b^T)
//   dL/dJ = w_q s [ (m_q + <K_q, G^-1>) J G^-1 - 2 J G^-1 K_q G^-1 ]
//   dL/dx_{E[a]} += dL/dJ grad^phi_a,      dL/dc_q = w_q s mc_q
// (Eqs. reference_quadrature_mass / _stiffness differentiated; Eq. F_map for
// J with the order-p basis of the nodes alpha / p, Sec. 4).
//
// 20- and 35-node local matrices do not fit one thread, so one warp takes one
// element: the element's gathered gradients GM, GA, GC as full matrices in
// shared memory; lanes over the quadrature points form m_q, K_q and dL/dJ
// (the basis rows of the lane's point against broadcast matrix entries);
// lanes over the nodes then contract dL/dJ with grad^phi_a into the
// element's node gradients, which a per-node pass sums over the node's
// incidences in ascending element order (deterministic, no atomics).
// The FP64 pipe bounds it.  Both precisions of the adjoint run this double
// path at these orders (the mixed request counts every element as redone).
#include "dispatch.cuh"
#include "tet_high.cuh"

namespace lfem {

constexpr int kAdjHighWarps = 2;

template <int D, int P>
struct AdjHigh {
  static constexpr int REF = Ref<D, P>::REF;
  static constexpr int ROW = REF | 1;  // table rows in 32-byte units
};

// Basis rows (phi, d phi / d xi_1 .. d xi_D) at every point into shared memory:
// from the tabulated tets (t64) or the bank's tables (curves, triangles).
template <int D, int P>
__device__ __forceinline__ void adj_high_stage_table(const AdjArgs& a, const V4<double>* __restrict__ t64,
                                                     V4<double>* tab) {
  constexpr int REF = AdjHigh<D, P>::REF, ROW = AdjHigh<D, P>::ROW;
  const int Q = a.tab.q;
  if constexpr (D == 3) {
    static_assert(ROW == TetHigh<P>::ROW, "the tet table rows");
    for (int t = threadIdx.x; t < Q * ROW; t += blockDim.x) tab[t] = t64[t];
  } else {
    const TabView<double> tb = tab_view<D, P, double>(a.tab);
    for (int t = threadIdx.x; t < Q * REF; t += blockDim.x) {
      const int q = t / REF, b = t - q * REF;
      V4<double> r{tb.phi[q * REF + b], tb.dphi[(q * REF + b) * D], 0.0, 0.0};
      if (D > 1) r.z = tb.dphi[(q * REF + b) * D + 1];
      tab[q * ROW + b] = r;
    }
  }
}

template <int D, int NA, int P, typename PosT>
__global__ void __launch_bounds__(kAdjHighWarps * 32) k_adjoint_high(const AdjArgs a, const V4<double>* __restrict__ t64) {
  constexpr int REF = AdjHigh<D, P>::REF, ROW = AdjHigh<D, P>::ROW;
  const int Q = a.tab.q;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V4<double>* tab = reinterpret_cast<V4<double>*>(smem_raw);  // [Q][ROW]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nmat = (a.gM ? 1 : 0) + (a.gA ? 1 : 0) + (a.gC ? 1 : 0);
  double* ws = reinterpret_cast<double*>(tab + (size_t)Q * ROW) +
               (size_t)warp * ((size_t)nmat * REF * REF + 4 * REF + (size_t)Q * NA * D);
  double* Gm = ws;                                    // [REF][REF] per given gradient, in the order M, A, C
  double* Ga = Gm + (a.gM ? REF * REF : 0);
  double* Gc = Ga + (a.gA ? REF * REF : 0);
  double* rel = Gc + (a.gC ? REF * REF : 0);          // [REF][4] x_b - x_0
  double* dl = rel + 4 * REF;                         // [Q][NA][D] dL/dJ
  adj_high_stage_table<D, P>(a, t64, tab);
  __syncthreads();
  const double* w64 = bank<double>() + a.tab.off64;
  for (int64_t e = (int64_t)blockIdx.x * kAdjHighWarps + warp; e < a.n_elem; e += (int64_t)gridDim.x * kAdjHighWarps) {
    const int32_t* cn = a.conn + e * REF;
    const int64_t n0 = __ldg(cn);
    for (int b = lane; b < REF; b += 32) {
      const int64_t nb = __ldg(cn + b);
#pragma unroll
      for (int i = 0; i < 3; ++i) rel[4 * b + i] = i < NA ? __ldg(a.coords + NA * nb + i) - __ldg(a.coords + NA * n0 + i) : 0.0;
      // row b of each given gradient, through the incidence record of (e, b)
      const int32_t k = __ldg(a.elem_inc + e * REF + b);
      const int64_t rb = __ldg(a.row_ptr + nb);
      int pos[REF];
      load_pos<PosT, REF>(a.inc_pos, k, pos);
#pragma unroll 5
      for (int c = 0; c < REF; ++c) {
        const int64_t s = rb + pos[c];
        if (a.gM) Gm[b * REF + c] = __ldg(a.gM + s);
        if (a.gA) Ga[b * REF + c] = __ldg(a.gA + s);
        if (a.gC) Gc[b * REF + c] = __ldg(a.gC + s);
      }
    }
    __syncwarp();
    // lanes over the points
    for (int q = lane; q < Q; q += 32) {
      const V4<double>* tq = tab + q * ROW;
      double J[NA][D];
#pragma unroll
      for (int i = 0; i < NA; ++i)
#pragma unroll
        for (int m = 0; m < D; ++m) J[i][m] = 0.0;
      for (int b = 1; b < REF; ++b) {
        const V4<double> d = tq[b];
        const double dm[3] = {d.y, d.z, d.w};
#pragma unroll
        for (int i = 0; i < NA; ++i)
#pragma unroll
          for (int m = 0; m < D; ++m) J[i][m] = fma(rel[4 * b + i], dm[m], J[i][m]);
      }
      // G = J^T J, s = sqrt(det G), Gi = G^-1
      double G[D][D];
#pragma unroll
      for (int m = 0; m < D; ++m)
#pragma unroll
        for (int n = 0; n < D; ++n) {
          double t = 0.0;
#pragma unroll
          for (int i = 0; i < NA; ++i) t = fma(J[i][m], J[i][n], t);
          G[m][n] = t;
        }
      double Gi[D][D], detG;
      if constexpr (D == 1) {
        detG = G[0][0];
        Gi[0][0] = 1.0 / detG;
      } else if constexpr (D == 2) {
        detG = G[0][0] * G[1][1] - G[0][1] * G[1][0];
        const double r = 1.0 / detG;
        Gi[0][0] = G[1][1] * r;
        Gi[1][1] = G[0][0] * r;
        Gi[0][1] = -G[0][1] * r;
        Gi[1][0] = -G[1][0] * r;
      } else {
        double C[3][3];
#pragma unroll
        for (int m = 0; m < 3; ++m)
#pragma unroll
          for (int n = 0; n < 3; ++n) {
            const int m1 = (m + 1) % 3, m2 = (m + 2) % 3, n1 = (n + 1) % 3, n2 = (n + 2) % 3;
            C[m][n] = G[m1][n1] * G[m2][n2] - G[m1][n2] * G[m2][n1];
          }
        detG = G[0][0] * C[0][0] + G[0][1] * C[0][1] + G[0][2] * C[0][2];
        const double r = 1.0 / detG;
#pragma unroll
        for (int m = 0; m < 3; ++m)
#pragma unroll
          for (int n = 0; n < 3; ++n) Gi[m][n] = C[n][m] * r;
      }
      const double s = sqrt(detG);
      const double cq = (a.coef && a.gC) ? __ldg(a.coef + e * Q + q) : 0.0;
      // quadratic forms with the lane's basis row
      double mq = 0.0, mc = 0.0, Kf[D][D];
#pragma unroll
      for (int m = 0; m < D; ++m)
#pragma unroll
        for (int n = 0; n < D; ++n) Kf[m][n] = 0.0;
      for (int ai = 0; ai < REF; ++ai) {
        double vM = 0.0, vC = 0.0, t[D];
#pragma unroll
        for (int m = 0; m < D; ++m) t[m] = 0.0;
        for (int b = 0; b < REF; ++b) {
          const V4<double> db = tq[b];
          if (a.gM) vM = fma(Gm[ai * REF + b], db.x, vM);
          if (a.gC) vC = fma(Gc[ai * REF + b], db.x, vC);
          if (a.gA) {
            const double g = Ga[ai * REF + b];
            t[0] = fma(g, db.y, t[0]);
            if (D > 1) t[D > 1 ? 1 : 0] = fma(g, db.z, t[D > 1 ? 1 : 0]);
            if (D > 2) t[D > 2 ? 2 : 0] = fma(g, db.w, t[D > 2 ? 2 : 0]);
          }
        }
        const V4<double> da = tq[ai];
        mq = fma(da.x, fma(cq, vC, vM), mq);
        mc = fma(da.x, vC, mc);
        const double gam[3] = {da.y, da.z, da.w};
#pragma unroll
        for (int m = 0; m < D; ++m)
#pragma unroll
          for (int n = 0; n < D; ++n) Kf[m][n] = fma(gam[m], t[n], Kf[m][n]);
      }
      double K[D][D];
#pragma unroll
      for (int m = 0; m < D; ++m)
#pragma unroll
        for (int n = 0; n < D; ++n) K[m][n] = 0.5 * (Kf[m][n] + Kf[n][m]);
      double KG = 0.0;
#pragma unroll
      for (int m = 0; m < D; ++m)
#pragma unroll
        for (int n = 0; n < D; ++n) KG = fma(K[m][n], Gi[m][n], KG);
      double T[D][D], B[D][D];
#pragma unroll
      for (int m = 0; m < D; ++m)
#pragma unroll
        for (int n = 0; n < D; ++n) {
          double t = 0.0;
#pragma unroll
          for (int l = 0; l < D; ++l) t = fma(Gi[m][l], K[l][n], t);
          T[m][n] = t;
        }
#pragma unroll
      for (int m = 0; m < D; ++m)
#pragma unroll
        for (int n = 0; n < D; ++n) {
          double t = 0.0;
#pragma unroll
          for (int l = 0; l < D; ++l) t = fma(T[m][l], Gi[l][n], t);
          B[m][n] = t;
        }
      const double wsq = w64[q] * s;
#pragma unroll
      for (int i = 0; i < NA; ++i)
#pragma unroll
        for (int n = 0; n < D; ++n) {
          double jg = 0.0, jb = 0.0;
#pragma unroll
          for (int m = 0; m < D; ++m) {
            jg = fma(J[i][m], Gi[m][n], jg);
            jb = fma(J[i][m], B[m][n], jb);
          }
          dl[(q * NA + i) * D + n] = wsq * ((mq + KG) * jg - 2.0 * jb);
        }
      if (a.g_coef) a.g_coef[e * Q + q] = wsq * mc;
    }
    __syncwarp();
    // lanes over the nodes: the element's node gradients
    for (int ai = lane; ai < REF; ai += 32) {
      double ge[NA];
#pragma unroll
      for (int i = 0; i < NA; ++i) ge[i] = 0.0;
      for (int q = 0; q < Q; ++q) {
        const V4<double> d = tab[q * ROW + ai];
        const double dm[3] = {d.y, d.z, d.w};
#pragma unroll
        for (int i = 0; i < NA; ++i)
#pragma unroll
          for (int n = 0; n < D; ++n) ge[i] = fma(dl[(q * NA + i) * D + n], dm[n], ge[i]);
      }
#pragma unroll
      for (int i = 0; i < NA; ++i) a.buf[(e * REF + ai) * NA + i] = ge[i];
    }
    if (a.mixed && lane == 0) atomicAdd(a.fallback, 1ull);
    __syncwarp();
  }
}

// Node r: g_coords[r][i] = sum over its incidences (e, a), ascending e, of buf[e][a][i].
template <int NA>
__global__ void __launch_bounds__(256) k_adjoint_high_gather(const AdjArgs a, int ref) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < a.n_nodes; r += (int64_t)gridDim.x * blockDim.x) {
    double s[NA];
#pragma unroll
    for (int i = 0; i < NA; ++i) s[i] = 0.0;
    const int32_t k0 = __ldg(a.inc_ptr + r), k1 = __ldg(a.inc_ptr + r + 1);
    for (int32_t k = k0; k < k1; ++k) {
      const int32_t key = __ldg(a.inc_key + k);
      const int64_t e = key >> a.key_shift;
      const int loc = key & ((1 << a.key_shift) - 1);
      const double* l = a.buf + (e * ref + loc) * NA;
#pragma unroll
      for (int i = 0; i < NA; ++i) s[i] += l[i];
    }
#pragma unroll
    for (int i = 0; i < NA; ++i) a.g_coords[r * NA + i] = s[i];
  }
}

template <int D, int P>
static size_t adj_high_smem(int Q, int NA, int nmat) {
  constexpr int REF = AdjHigh<D, P>::REF, ROW = AdjHigh<D, P>::ROW;
  return sizeof(V4<double>) * (size_t)Q * ROW +
         sizeof(double) * (size_t)kAdjHighWarps * ((size_t)nmat * REF * REF + 4 * REF + (size_t)Q * NA * D);
}

template <int D, int NA, int P>
static lfem_status launch_adjoint_high(const AdjArgs& a, int pos_bytes, void* scratch, int sms, cudaStream_t st) {
  constexpr int REF = AdjHigh<D, P>::REF;
  const int Q = a.tab.q;
  V4<double>* t64 = nullptr;
  if (a.n_elem > 0) {
    if constexpr (D == 3) {
      t64 = static_cast<V4<double>*>(scratch);
      V4<float>* t32 = reinterpret_cast<V4<float>*>(t64 + (size_t)Q * TetHigh<P>::ROW);
      k_tet_high_table<P><<<(Q * REF + 127) / 128, 128, 0, st>>>(a.tab, t64, t32);
      LFEM_CUDA(cudaGetLastError());
    }
    const int nmat = (a.gM ? 1 : 0) + (a.gA ? 1 : 0) + (a.gC ? 1 : 0);
    const size_t smem = adj_high_smem<D, P>(Q, NA, nmat);
    auto kern = pos_bytes == 1 ? k_adjoint_high<D, NA, P, uint8_t> : k_adjoint_high<D, NA, P, uint16_t>;
    LFEM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int occ = 0;
    LFEM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kAdjHighWarps * 32, smem));
    if (occ < 1) return fail(LFEM_E_TOO_LARGE, "order-3/4 adjoint tables exceed shared memory");
    int64_t g = (a.n_elem + kAdjHighWarps - 1) / kAdjHighWarps;
    if (g > (int64_t)sms * occ) g = (int64_t)sms * occ;
    kern<<<(unsigned)g, kAdjHighWarps * 32, smem, st>>>(a, t64);
    LFEM_CUDA(cudaGetLastError());
  }
  if (a.n_nodes > 0) {
    int64_t g = (a.n_nodes + 255) / 256;
    if (g > (int64_t)sms * 8) g = (int64_t)sms * 8;
    k_adjoint_high_gather<NA><<<(unsigned)g, 256, 0, st>>>(a, REF);
    LFEM_CUDA(cudaGetLastError());
  }
  return LFEM_OK;
}

size_t adjoint_high_scratch_bytes(int dim, int P, int Q, int ambient, int64_t n_elem) {
  const int REF = dim == 1 ? P + 1 : (dim == 2 ? (P + 1) * (P + 2) / 2 : (P + 1) * (P + 2) * (P + 3) / 6);
  const size_t buf = ((size_t)n_elem * REF * ambient * sizeof(double) + 255) / 256 * 256;
  const size_t tab = dim == 3 ? (size_t)Q * (REF | 1) * (sizeof(V4<double>) + sizeof(V4<float>)) : 0;
  return buf + tab;
}

lfem_status run_adjoint_high(int dim, int NA, int P, const AdjArgs& a0, int pos_bytes, void* scratch, int sms,
                             cudaStream_t st) {
  const int REF = dim == 1 ? P + 1 : (dim == 2 ? (P + 1) * (P + 2) / 2 : (P + 1) * (P + 2) * (P + 3) / 6);
  AdjArgs a = a0;
  a.buf = static_cast<double*>(scratch);
  void* tabs = static_cast<char*>(scratch) + ((size_t)a.n_elem * REF * NA * sizeof(double) + 255) / 256 * 256;
#define LFEM_ADJ_HIGH(DD, NN, PP) \
  if (dim == DD && NA == NN && P == PP) return launch_adjoint_high<DD, NN, PP>(a, pos_bytes, tabs, sms, st);
  LFEM_ADJ_HIGH(1, 1, 3)
  LFEM_ADJ_HIGH(1, 1, 4)
  LFEM_ADJ_HIGH(1, 2, 3)
  LFEM_ADJ_HIGH(1, 2, 4)
  LFEM_ADJ_HIGH(1, 3, 3)
  LFEM_ADJ_HIGH(1, 3, 4)
  LFEM_ADJ_HIGH(2, 2, 3)
  LFEM_ADJ_HIGH(2, 2, 4)
  LFEM_ADJ_HIGH(2, 3, 3)
  LFEM_ADJ_HIGH(2, 3, 4)
  LFEM_ADJ_HIGH(3, 3, 3)
  LFEM_ADJ_HIGH(3, 3, 4)
#undef LFEM_ADJ_HIGH
  return fail(LFEM_E_UNSUPPORTED, "element type");
}

lfem_status bank_upload_adj_high(const void* src, size_t bytes, size_t offset) {
  LFEM_CUDA(cudaMemcpyToSymbol(c_bank, src, bytes, offset, cudaMemcpyHostToDevice));
  return LFEM_OK;
}

}  // namespace lfem
