// Bulk P2 tetrahedra with the compile-time 14-point rule, mixed precision:
// every element once, local upper triangles to an element-major buffer that
// the slot gather then sums (Eqs. reference_quadrature_mass / _stiffness,
// Sec. 3.3).  One thread per element, shaped for occupancy rather than for
// one thread holding everything:
//   * the element's edge vectors and edge-node deviations live in the warp's
//     shared-memory slab (16-byte rows, reread point by point);
//   * per-point reference tables sit in shared memory and arrive as uniform
//     128-bit loads (the point loop stays rolled: 14 unrolled points of 10 x 10
//     gradient products outgrow the instruction cache);
//   * the stiffness is accumulated two upper-triangle entries per f32x2
//     instruction: columns b in pairs (2j, 2j+1), so
//       y_j[m]    = sum_n Hw[m][n] (d_n phi_2j, d_n phi_2j+1)
//       A[a][j]  += sum_m (d_m phi_a, d_m phi_a) y_j[m]       (2j + 1 >= a)
//     with Hw = w_q adj(G) / |det J| from the cofactors of J -- the same
//     per-entry operations, in the same order, as the scalar form;
//   * |det J| of every point goes to shared memory, and after the loop the
//     mass-type matrices are one packed contraction with the table pairs
//     (TM[q][2j], TM[q][2j+1]) read as immediate operands;
//   * results leave through the warp's slab, so each matrix of the warp's 32
//     elements is written as one contiguous run.
// Buffer layout: [e][u][nm] -- the requested matrices of one entry side by
// side, so the slot gather reads them with one load.
#pragma once

#include "assemble_fast.cuh"
#include "assemble_impl.cuh"
#include "assemble_twopass.cuh"

namespace lfem {

// Tables of the P2 tetrahedron and its 14-point rule, packed for the kernel.
struct alignas(16) Tet2Pack {
  static constexpr int Q = 14, REF = 10, U = 55, NE = 6, NJ = 5, UH = 28;
  // per point (floats; every pair at an even offset, every block 16-byte aligned)
  static constexpr int DPS = 0;    // (d_m psi_k, d_m psi_k)            [6][3][2]
  static constexpr int DPD = 36;   // (d_m phi_a, d_m phi_a)            [10][3][2]
  static constexpr int DPP = 96;   // (d_n phi_2j, d_n phi_2j+1)        [5][3][2]
  static constexpr int WQ = 126;   // w_q, then one float of padding
  static constexpr int PER_Q = 128;
  static constexpr int SMEM = Q * PER_Q;  // the part copied to shared memory
  static constexpr int TM2 = SMEM;        // (TM[q][2j], TM[q][2j+1])  [14][28][2]
  static constexpr int SIZE = TM2 + Q * UH * 2;
  float v[SIZE];
};
static_assert(Tet2Pack::SIZE * 4 <= 16384, "kernel-parameter table");

// Host: Tet2Pack from the FastLayout<3, 2> table of the same rule.
void tet2_pack_host(const float* fl, Tet2Pack& out);

constexpr int kTet2Threads = 128;
constexpr int kTet2MinBlocks = 4;  // 16 warps per SM: at most 128 registers
constexpr int kTet2Slab = 32 * Tet2Pack::U;        // floats per warp: the result stage
constexpr int kTet2Ed = 36;                        // floats per element: 9 rows of 4
static_assert(32 * kTet2Ed <= kTet2Slab, "element data fit in the result stage");
static_assert(sizeof(float) * (Tet2Pack::SMEM + (kTet2Threads / 32) * (kTet2Slab + 32 * Tet2Pack::Q)) <= 48 * 1024,
              "default dynamic shared memory");

// Accumulator index of the pair (a, j), j >= a / 2.
__host__ __device__ constexpr int tet2_pair(int a, int j) {
  // pairs of column j: a = 0 .. 2j + 1; columns before j hold 2 + 4 + ... + 2j
  return j * (j + 1) + a;
}

// The stiffness of one element (upper layout into slab row o, stride 1),
// with s_q = |det J| of every point to sq (stride 32) and the tests.
__device__ __forceinline__ void tet2_stiff(const float* __restrict__ tab, const float* __restrict__ edr, float qthr,
                                           bool do_a, float* __restrict__ sq, float2 (&A2)[30], Checks& ck) {
  using T = Tet2Pack;
#pragma unroll
  for (int i = 0; i < 30; ++i) A2[i] = f2(0.f);
#pragma unroll 1
  for (int q = 0; q < T::Q; ++q) {
    const float* tq = tab + q * T::PER_Q;
    // J[i][m] = e[m][i] + sum_k dl[k][i] d_m psi_k; rows (x, y) packed
    float2 Jxy[3];
    float Jz[3];
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      const float4 em = reinterpret_cast<const float4*>(edr)[m];
      Jxy[m] = make_float2(em.x, em.y);
      Jz[m] = em.z;
    }
#pragma unroll
    for (int k = 0; k < T::NE; ++k) {
      const float4 d = reinterpret_cast<const float4*>(edr)[3 + k];
      const float2 dxy = make_float2(d.x, d.y);
      // pair (k, m) is pair 3k + m of the block
      float2 t[3];
#pragma unroll
      for (int m = 0; m < 3; ++m) t[m] = reinterpret_cast<const float2*>(tq + T::DPS)[3 * k + m];
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        Jxy[m] = fma2(dxy, t[m], Jxy[m]);
        Jz[m] = fmaf(d.z, t[m].x, Jz[m]);
      }
    }
    float J[3][3];
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      J[0][m] = Jxy[m].x;
      J[1][m] = Jxy[m].y;
      J[2][m] = Jz[m];
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
    sq[32 * q] = fabsf(det);
    float tr = 0.f;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int m = 0; m < 3; ++m) tr = fmaf(J[i][m], J[i][m], tr);
    tr *= (1.0f / 3.0f);
    const float s2 = __fmul_rn(det, det);
    ck.good &= (s2 > 1e-12f * (tr * tr * tr)) & (s2 <= 3.0e38f);
    ck.cond &= s2 >= qthr * (tr * tr * tr);
    if (!do_a) continue;
    const float winv = __fdividef(tq[T::WQ], fabsf(det));
    float2 H[3][3];
#pragma unroll
    for (int m = 0; m < 3; ++m)
#pragma unroll
      for (int n = m; n < 3; ++n)
        H[m][n] = H[n][m] =
            f2(__fmul_rn(fmaf(c[m][2], c[n][2], fmaf(c[m][1], c[n][1], __fmul_rn(c[m][0], c[n][0]))), winv));
    float2 y[T::NJ][3];
#pragma unroll
    for (int j = 0; j < T::NJ; ++j) {
      float2 p[3];
#pragma unroll
      for (int n = 0; n < 3; ++n) p[n] = reinterpret_cast<const float2*>(tq + T::DPP)[3 * j + n];
#pragma unroll
      for (int m = 0; m < 3; ++m) y[j][m] = fma2(H[m][2], p[2], fma2(H[m][1], p[1], mul2(H[m][0], p[0])));
    }
#pragma unroll
    for (int a = 0; a < T::REF; ++a) {
      float2 g[3];
#pragma unroll
      for (int m = 0; m < 3; ++m) g[m] = reinterpret_cast<const float2*>(tq + T::DPD)[3 * a + m];
#pragma unroll
      for (int j = a / 2; j < T::NJ; ++j) {
        float2 acc = A2[tet2_pair(a, j)];
#pragma unroll
        for (int m = 0; m < 3; ++m) acc = fma2(g[m], y[j][m], acc);
        A2[tet2_pair(a, j)] = acc;
      }
    }
  }
}

// V_u = sum_q f_q TM[q][u] for the 55 entries, into slab row o (stride 1).
__device__ __forceinline__ void tet2_mass(const Tet2Pack& pk, const float (&f)[Tet2Pack::Q], float* __restrict__ o) {
  using T = Tet2Pack;
  float2 fq[T::Q];
#pragma unroll
  for (int q = 0; q < T::Q; ++q) fq[q] = f2(f[q]);
#pragma unroll
  for (int j = 0; j < T::UH; ++j) {
    float2 acc = mul2(fq[0], reinterpret_cast<const float2*>(pk.v + T::TM2)[j]);
#pragma unroll
    for (int q = 1; q < T::Q; ++q) acc = fma2(fq[q], reinterpret_cast<const float2*>(pk.v + T::TM2)[q * T::UH + j], acc);
    o[2 * j] = acc.x;
    if (2 * j + 1 < T::U) o[2 * j + 1] = acc.y;
  }
}

// The warp's stage (32 rows of 55) to buf[e][u][nm] at matrix position slot.
__device__ __forceinline__ void tet2_flush(const float* __restrict__ stage, float* __restrict__ buf, int64_t e0,
                                           int nvalid, int nm, int slot, int lane) {
  constexpr int U = Tet2Pack::U;
  float* dst = buf + (size_t)e0 * U * nm + slot;
  for (int i = lane; i < nvalid * U; i += 32) dst[(size_t)i * nm] = stage[i];
}

__global__ void __launch_bounds__(kTet2Threads, kTet2MinBlocks) k_tet2_local(const TwoPassArgs a, const __grid_constant__ Tet2Pack pk) {
  using T = Tet2Pack;
  constexpr int REF = T::REF, U = T::U, Q = T::Q;
  extern __shared__ __align__(16) float t2_smem[];
  float* tab = t2_smem;                                   // [Q][PER_Q]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* slab = tab + T::SMEM + warp * (kTet2Slab + 32 * Q);  // stage / element data
  float* sqw = slab + kTet2Slab;                                // [Q][32]
  for (int i = threadIdx.x; i < T::SMEM / 4; i += blockDim.x)
    reinterpret_cast<float4*>(tab)[i] = reinterpret_cast<const float4*>(pk.v)[i];
  __syncthreads();
  float* lb = static_cast<float*>(a.lbuf);
  const int nm = a.nm;
  const bool do_m = a.which & LFEM_MASS, do_a = a.which & LFEM_STIFF, do_c = a.which & LFEM_CMASS;
  const int slot_a = do_m ? 1 : 0, slot_c = (do_m ? 1 : 0) + (do_a ? 1 : 0);
  const int64_t nw = (int64_t)gridDim.x * (kTet2Threads / 32);
  for (int64_t wb = (int64_t)blockIdx.x * (kTet2Threads / 32) + warp; wb * 32 < a.n_elem; wb += nw) {
    const int64_t e0 = wb * 32;
    const int nvalid = a.n_elem - e0 < 32 ? (int)(a.n_elem - e0) : 32;
    const int64_t e = e0 + lane;
    const bool live = lane < nvalid;
    Checks ck;
    bool ok = true;
    float* edr = slab + lane * kTet2Ed;
    if (live) {
      int32_t nodes[REF];
#pragma unroll
      for (int b = 0; b < REF; ++b) nodes[b] = __ldg(a.conn + e * REF + b);
      ElemData<3, 3, 2, float> ed;
      ok = load_element_data_split<3, 3, 2>(a.coords, nodes, ed);
#pragma unroll
      for (int m = 0; m < 3; ++m)
        reinterpret_cast<float4*>(edr)[m] = make_float4(ed.e[m][0], ed.e[m][1], ed.e[m][2], 0.f);
#pragma unroll
      for (int k = 0; k < T::NE; ++k)
        reinterpret_cast<float4*>(edr)[3 + k] = make_float4(ed.dl[k][0], ed.dl[k][1], ed.dl[k][2], 0.f);
    } else {
#pragma unroll
      for (int r = 0; r < 9; ++r) reinterpret_cast<float4*>(edr)[r] = make_float4(0.f, 0.f, 0.f, 0.f);
      // a regular reference tetrahedron keeps the idle lane's arithmetic finite
      edr[0] = 1.f;
      edr[5] = 1.f;
      edr[10] = 1.f;
    }
    float2 A2[30];
    tet2_stiff(tab, edr, a.qmin, do_a, sqw + lane, A2, ck);
    __syncwarp();  // element data read: the slab becomes the result stage
    float* row = slab + lane * U;
    if (do_a) {
#pragma unroll
      for (int aa = 0; aa < REF; ++aa)
#pragma unroll
        for (int j = aa / 2; j < T::NJ; ++j) {
          const float2 v = A2[tet2_pair(aa, j)];
          if (2 * j >= aa) row[upper_index(REF, aa, 2 * j)] = v.x;
          if (2 * j + 1 < REF) row[upper_index(REF, aa, 2 * j + 1)] = v.y;
        }
      __syncwarp();
      tet2_flush(slab, lb, e0, nvalid, nm, slot_a, lane);
      __syncwarp();
    }
    if (do_m || do_c) {
      float s[Q];
#pragma unroll
      for (int q = 0; q < Q; ++q) s[q] = sqw[32 * q + lane];
      if (do_m) {
        tet2_mass(pk, s, row);
        __syncwarp();
        tet2_flush(slab, lb, e0, nvalid, nm, 0, lane);
        __syncwarp();
      }
      if (do_c) {
        if (live) {
          const float* cs = a.coef_f32 ? static_cast<const float*>(a.coef) + e * Q : nullptr;
          const double* cdp = a.coef_f32 ? nullptr : static_cast<const double*>(a.coef) + e * Q;
#pragma unroll
          for (int q = 0; q < Q; ++q) s[q] *= cs ? __ldg(cs + q) : (float)__ldg(cdp + q);
        }
        tet2_mass(pk, s, row);
        __syncwarp();
        tet2_flush(slab, lb, e0, nvalid, nm, slot_c, lane);
        __syncwarp();
      }
    }
    // elements that failed the finiteness or conditioning test are listed and
    // redone whole in double by k_tet2_redo (the float |det J| of a flat tet
    // loses about log2 cond(J) bits, so the mass-type matrices need it too)
    if (live && (!ok || !ck.good || !ck.cond)) a.redo[atomicAdd(a.fallback, 1ull)] = (int32_t)e;
  }
}

// Every listed element in double, over the float results of k_tet2_local.
__global__ void __launch_bounds__(128) k_tet2_redo(const TwoPassArgs a) {
  constexpr int REF = Tet2Pack::REF, U = Tet2Pack::U;
  const unsigned long long n = *a.fallback;
  float* lb = static_cast<float*>(a.lbuf);
  // consecutive list entries go to different CTAs first, so the list spreads
  // over every SM's FP64 pipe
  for (unsigned long long i = (unsigned long long)threadIdx.x * gridDim.x + blockIdx.x; i < n;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const int64_t e = a.redo[i];
    int32_t nodes[REF];
#pragma unroll
    for (int b = 0; b < REF; ++b) nodes[b] = __ldg(a.conn + e * REF + b);
    bool bad = false;
    element_fp64_lean<3, 3, 2, float>(a.coords, nodes, a.tab, a.coef, a.coef_f32, e, a.which,
                                       lb + (size_t)e * U * a.nm, 1, bad, 0, a.nm);
    if (bad) atomicOr(a.status, ST_DEGENERATE);
  }
}

inline size_t tet2_smem_bytes() {
  return sizeof(float) * (Tet2Pack::SMEM + (kTet2Threads / 32) * (kTet2Slab + 32 * Tet2Pack::Q));
}

inline lfem_status launch_tet2(const TwoPassArgs& a, const Tet2Pack& pk, int sm_count, cudaStream_t st) {
  if (a.n_elem > 0) {
    const size_t smem = tet2_smem_bytes();  // below the 48 KB default
    const int64_t warps = (a.n_elem + 31) / 32;
    int64_t g = (warps + kTet2Threads / 32 - 1) / (kTet2Threads / 32);
    if (g > (int64_t)sm_count * 4) g = (int64_t)sm_count * 4;
    k_tet2_local<<<(unsigned)g, kTet2Threads, smem, st>>>(a, pk);
    LFEM_CUDA(cudaGetLastError());
    k_tet2_redo<<<(unsigned)sm_count, 128, 0, st>>>(a);
    LFEM_CUDA(cudaGetLastError());
  }
  if (a.nnz > 0) {
    int64_t g = (a.nnz + 255) / 256;
    if (g > (int64_t)sm_count * 16) g = (int64_t)sm_count * 16;
    if (a.nm == 1) k_slot_gather_il<1><<<(unsigned)g, 256, 0, st>>>(a);
    else if (a.nm == 2) k_slot_gather_il<2><<<(unsigned)g, 256, 0, st>>>(a);
    else k_slot_gather_il<3><<<(unsigned)g, 256, 0, st>>>(a);
    LFEM_CUDA(cudaGetLastError());
  }
  return LFEM_OK;
}

}  // namespace lfem
