// Element-major assembly for bulk tetrahedra.
//
// Row tiles in 3-D recompute most elements several times (a compact block of
// rows is touched by many more tetrahedra than it owns), so tets use two
// passes instead:
//   k_elem_local   every element once: geometry and local upper-triangle
//                  matrices (Eqs. reference_quadrature_mass / _stiffness),
//                  one matrix per pass, into a global buffer [nE][nm][U]
//   k_slot_gather  every CSR slot once: its contributions, precomputed in
//                  ascending (element, a, b) order, summed with a compensated
//                  pair in registers and stored (Eqs. M matrix, A matrix)
// Deterministic and atomic-free like the tiled path.
#pragma once

#include "assemble_fast.cuh"
#include "assemble_impl.cuh"

namespace lfem {

struct TwoPassArgs {
  const int32_t* conn;
  const double* coords;
  const void* coef;
  int coef_f32;
  int64_t n_elem;
  int64_t nnz;
  const int32_t* slot_off;
  const int32_t* slot_ent;
  void* lbuf;  // [nE][nm][U] in precision R
  void* out[3];
  int nm;
  unsigned which;
  TabRef tab;
  float qmin;
  int32_t* status;
  unsigned long long* fallback;
  int32_t* redo;  // [n_elem]: elements to redo in double (P2 tets, compile-time rule)
};

// All requested matrices of one element, one matrix per quadrature pass (keeps
// the register footprint at one upper triangle), upper layout.
template <int D, int NA, int P, typename R, typename RS>
__device__ __forceinline__ void element_lean(const ElemData<D, NA, P, R>& ed, const TabView<R>& tb, const void* coef,
                                             int coef_f32, int64_t e, unsigned which, RS* dst, R& qual, bool& bad) {
  constexpr int U = Ref<D, P>::U;
  R V[U], d1[U], d2[U];
  int slot = 0;
  if (which & LFEM_MASS) {
    element_pass<D, NA, P, R, true, false, false>(ed, tb, coef, coef_f32, e, V, d1, d2, qual, bad);
#pragma unroll
    for (int u = 0; u < U; ++u) dst[slot * U + u] = (RS)V[u];
    ++slot;
  }
  if (which & LFEM_STIFF) {
    element_pass<D, NA, P, R, false, true, false>(ed, tb, coef, coef_f32, e, d1, V, d2, qual, bad);
#pragma unroll
    for (int u = 0; u < U; ++u) dst[slot * U + u] = (RS)V[u];
    ++slot;
  }
  if (which & LFEM_CMASS) {
    element_pass<D, NA, P, R, false, false, true>(ed, tb, coef, coef_f32, e, d1, d2, V, qual, bad);
#pragma unroll
    for (int u = 0; u < U; ++u) dst[slot * U + u] = (RS)V[u];
  }
}

// FAST: the rule is the compile-time one (float only; tables in fb).
template <int D, int NA, int P, typename R, bool FAST>
__global__ void __launch_bounds__(128) k_elem_local(const TwoPassArgs a, const __grid_constant__ FastBankTet fb) {
  constexpr int REF = Ref<D, P>::REF;
  constexpr int U = Ref<D, P>::U;
  const TabView<R> tb = tab_view<D, P, R>(a.tab);
  R* lb = static_cast<R*>(a.lbuf);
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < a.n_elem;
       e += (int64_t)gridDim.x * blockDim.x) {
    int32_t nodes[REF];
#pragma unroll
    for (int b = 0; b < REF; ++b) nodes[b] = __ldg(a.conn + e * REF + b);
    R* dst = lb + (size_t)e * a.nm * U;
    R qual = (R)1;
    bool bad = false;
    if constexpr (FAST && sizeof(R) == 4) {
      ElemData<D, NA, P, float> ed;
      const bool ok = load_element_data_split<D, NA, P>(a.coords, nodes, ed);
      constexpr int Q = FastLayout<D, P>::Q;
      const float* cs = (a.which & LFEM_CMASS) && a.coef_f32 ? static_cast<const float*>(a.coef) + e * Q : nullptr;
      const double* cd = (a.which & LFEM_CMASS) && !a.coef_f32 ? static_cast<const double*>(a.coef) + e * Q : nullptr;
      Checks ck;
      element_fast_store<D, NA, P>(ed, fb, cs, cd, a.qmin, a.which, dst, U, ck);
      // double recomputation of every requested matrix after a failed
      // finiteness or conditioning test (the float |det J| of a flat tet
      // loses about log2 cond(J) bits, so the mass-type matrices need it too)
      if (!ok || !ck.good || !ck.cond) {
        element_fp64_lean<D, NA, P, float>(a.coords, nodes, a.tab, a.coef, a.coef_f32, e, a.which, dst, U, bad);
        atomicAdd(a.fallback, 1ull);
      }
    } else if constexpr (sizeof(R) == 4) {
      ElemData<D, NA, P, float> ed;
      const bool ok = load_element_data_split<D, NA, P>(a.coords, nodes, ed);
      element_lean<D, NA, P, float, float>(ed, tb, a.coef, a.coef_f32, e, a.which, dst, qual, bad);
      if (!ok || (D > 1 && qual < (R)a.qmin) || bad) {
        bad = false;
        element_fp64_lean<D, NA, P, float>(a.coords, nodes, a.tab, a.coef, a.coef_f32, e, a.which, dst, U, bad);
        atomicAdd(a.fallback, 1ull);
      }
    } else {
      double X[REF][NA];
      gather_coords<D, NA, P>(a.coords, nodes, X);
      ElemData<D, NA, P, double> ed;
      load_element_data<D, NA, P, double>(X, ed);
      element_lean<D, NA, P, double, double>(ed, tb, a.coef, a.coef_f32, e, a.which, dst, qual, bad);
    }
    if (bad) atomicOr(a.status, ST_DEGENERATE);
  }
}

template <int U, typename R>
__global__ void __launch_bounds__(256) k_slot_gather(const TwoPassArgs a) {
  using Acc = typename AccOf<R>::T;
  const R* lb = static_cast<const R*>(a.lbuf);
  const int nm = a.nm;
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < a.nnz; s += (int64_t)gridDim.x * blockDim.x) {
    const int32_t k0 = __ldg(a.slot_off + s), k1 = __ldg(a.slot_off + s + 1);
    Acc c0, c1, c2;
    acc_zero(c0);
    acc_zero(c1);
    acc_zero(c2);
    for (int32_t k = k0; k < k1; ++k) {
      const uint32_t ent = (uint32_t)__ldg(a.slot_ent + k);
      const uint32_t e = ent / U, u = ent - e * U;
      const R* l = lb + (size_t)e * nm * U + u;
      acc_add(c0, l[0]);
      if (nm > 1) acc_add(c1, l[U]);
      if (nm > 2) acc_add(c2, l[2 * U]);
    }
    static_cast<R*>(a.out[0])[s] = (R)acc_final(c0);
    if (nm > 1) static_cast<R*>(a.out[1])[s] = (R)acc_final(c1);
    if (nm > 2) static_cast<R*>(a.out[2])[s] = (R)acc_final(c2);
  }
}

// Slot sums over the interleaved buffer: slot s adds buf[ent * NM + m] over its
// list, compensated, in list order (ascending (element, a, b)).
template <int NM>
__global__ void __launch_bounds__(256) k_slot_gather_il(const TwoPassArgs a) {
  const float* lb = static_cast<const float*>(a.lbuf);
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < a.nnz; s += (int64_t)gridDim.x * blockDim.x) {
    const int32_t k0 = __ldg(a.slot_off + s), k1 = __ldg(a.slot_off + s + 1);
    float2 c[NM];
#pragma unroll
    for (int m = 0; m < NM; ++m) acc_zero(c[m]);
    for (int32_t k = k0; k < k1; ++k) {
      const size_t ent = (uint32_t)__ldg(a.slot_ent + k);
      if constexpr (NM == 2) {
        const float2 v = __ldg(reinterpret_cast<const float2*>(lb) + ent);
        acc_add(c[0], v.x);
        acc_add(c[1], v.y);
      } else {
#pragma unroll
        for (int m = 0; m < NM; ++m) acc_add(c[m], __ldg(lb + ent * NM + m));
      }
    }
#pragma unroll
    for (int m = 0; m < NM; ++m) static_cast<float*>(a.out[m])[s] = acc_final(c[m]);
  }
}

template <int D, int NA, int P, typename R>
lfem_status launch_twopass(const TwoPassArgs& a, bool fast, const FastBankTet& fb, int sm_count, cudaStream_t st) {
  constexpr int U = Ref<D, P>::U;
  if (a.n_elem > 0) {
    int64_t g = (a.n_elem + 127) / 128;
    if (g > (int64_t)sm_count * 32) g = (int64_t)sm_count * 32;
    bool done = false;
    if constexpr (sizeof(R) == 4 && D == 3 && P <= 2) {
      if (fast) {
        k_elem_local<D, NA, P, R, true><<<(unsigned)g, 128, 0, st>>>(a, fb);
        done = true;
      }
    }
    if (!done) k_elem_local<D, NA, P, R, false><<<(unsigned)g, 128, 0, st>>>(a, fb);
    LFEM_CUDA(cudaGetLastError());
  }
  if (a.nnz > 0) {
    int64_t g = (a.nnz + 255) / 256;
    if (g > (int64_t)sm_count * 16) g = (int64_t)sm_count * 16;
    k_slot_gather<U, R><<<(unsigned)g, 256, 0, st>>>(a);
    LFEM_CUDA(cudaGetLastError());
  }
  return LFEM_OK;
}

}  // namespace lfem
