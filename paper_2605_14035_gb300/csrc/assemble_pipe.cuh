// Persistent, pipelined assembly kernel.
//
// Each CTA walks the work items k = blockIdx.x, blockIdx.x + gridDim.x, ...
// (a work item is one row tile of one mesh).  A tile's metadata block has two
// parts (see TileHdr): the front part (element ids, node list, local node
// indices) is needed from the start of the tile, the back part (the slots'
// contribution entries) only by phase 2.  The pipeline, per CTA:
//   front part of item k+2   TMA bulk copy issued at the start of item k
//                            (three front buffers)
//   node coordinates (and general-rule coefficients) of item k+1
//                            cp.async gathers issued at the start of item k,
//                            as soon as item k+1's front part is there
//                            (two node buffers)
//   back part of item k+1    TMA bulk copy issued when item k's phase 2 is
//                            done (one back buffer)
// so the global-memory latency of every copy hides behind a whole item of
// arithmetic.  Only the issuing thread touches the work-item records (a ring
// of four in shared memory, each fetched by cp.async three items ahead).
//
// Per tile (Sec. 3.2 / 3.3 of the paper; Eqs. reference_quadrature_mass,
// reference_quadrature_stiffness, M matrix, A matrix):
//   split    node coordinates -> float pairs (mixed) once per node, done for
//            item k+1 at the end of item k (no barrier of its own)
//   phase 1  geometry and local upper-triangle matrices of every element of
//            the tile -> shared memory (interleaved layout: one address per
//            entry serves M, A and MC)
//   phase 2  slots with more than two contributions are summed first, in
//            ascending element order with a compensated pair, into shared
//            memory; then every slot is the sum of its two entries (the second
//            may be the zero word), four consecutive slots per thread with
//            16-byte stores -- one writer per slot, fixed order, no atomics
//
// Every wait is bounded by the global timer; on timeout the CTA records
// ST_TIMEOUT in the status word, waits (bounded) for the copies it issued and
// returns, leaving the context usable.
#pragma once

#include "assemble_fast.cuh"
#include "assemble_impl.cuh"

namespace lfem {

constexpr int kPipeTPE = 2;  // threads per element in phase 1 (general rules)

// Launch shape: the float kernel fits 160 registers, so 192 threads and two
// CTAs per SM; the double kernel needs more registers: 256 threads, one CTA.
template <typename R>
struct PipeOcc;
template <>
struct PipeOcc<float> {
  static constexpr int THREADS = 192;
  static constexpr int MIN_BLOCKS = 2;
};
template <>
struct PipeOcc<double> {
  static constexpr int THREADS = 256;
  static constexpr int MIN_BLOCKS = 1;
};

// One mesh of a launch: its inputs, outputs and tables.
struct MeshRec {
  const double* coords;
  const void* coef;
  void* out[3];
  TabRef tab;
  int type;  // element type id (elem_type_id)
  int na, ref, entb, coef_f32;
  int c16;  // coords is 16-byte aligned: node runs arrive by bulk copies
};

__host__ __device__ constexpr int elem_type_id(int d, int na, int p) { return d * 100 + na * 10 + p; }
constexpr int kFastTypeOffset = 1000;

// Arguments of a persistent launch over work items.  Item k is items[k]: the
// block of one tile and the index of its mesh (meshes[mesh], or one).
struct PipeArgs {
  MeshRec one;              // the mesh when meshes is NULL
  const MeshRec* meshes;    // device table of a batch, or NULL
  const ItemRef* items;     // [n_items]
  int64_t n_items;
  int nm;
  unsigned which;
  int chunk;       // elements per phase-1 round (threads / kPipeTPE)
  int cap_front;   // largest front part
  int cap_back;    // largest back part
  int cap_nodes;   // most nodes in a tile
  int cap_nel;     // most elements in a tile
  int max_u;       // largest local upper triangle among the meshes
  int64_t cap_lsm; // local-matrix words: 3 nel UP + 6 (nl + 1), largest over the tiles
  int max_q;       // most quadrature points among the meshes
  int coef_bytes;  // 4 or 8 if the weighted mass is requested, else 0
  int coef_smem;   // bytes per coefficient staged in shared memory: coef_bytes if a
                   // general-rule tile may need them, else 0 (compile-time-rule
                   // tiles read theirs from global memory)
  int vec_out;     // every output array is 16-byte aligned: phase 2 may store 16 bytes at once
  float qmin;
  int32_t* status;
  unsigned long long* fallback;
  unsigned int* next_item;  // tile tickets (0 at launch): items past the first gridDim.x
                                  // go to whichever CTA asks first
  int starve;         // test knob: CTA 0 skips its first front copy
  long long wait_ns;  // bound of every wait
};

// Local-matrix words of a tile with nel elements of upper size u and nl long
// slots, ns matrix slots per entry pair: the elements, 2 ns result words per
// long slot, 2 ns zero words.  The float kernels keep all three slots (the
// tile blocks' words address that layout directly); the double kernels keep
// the requested matrices only (ns = nm) and map each word W of the
// three-slot layout to 2 ns (W / 6) + W mod 6.
__host__ __device__ constexpr int64_t lsm_words(int64_t nel, int u, int64_t nl, int ns = kLsmSlots) {
  return (int64_t)ns * nel * lsm_stride(u) + 2ll * ns * (nl + 1);
}

struct PipeSmem {
  size_t mbar, refs, rec, front, back, node0, node1, coef0, coef1, lsm, flag, total;
  size_t front_stride;
};

template <typename R>
__host__ __device__ inline PipeSmem pipe_smem_layout(int na, int64_t cap_lsm, int cap_front, int cap_back,
                                                     int cap_nodes, int cap_nel, int q, int coef_bytes) {
  auto al = [](size_t b) { return (b + 127) / 128 * 128; };
  PipeSmem L;
  size_t o = 0;
  L.mbar = o;  // 6 mbarriers (3 front buffers, the back buffer, 2 node buffers), then flags
  o += 128;
  L.refs = o;  // ring of 4 work-item records
  o += al(4 * sizeof(ItemRef));
  L.rec = o;  // the MeshRec of each front buffer's item
  o += al(3 * sizeof(MeshRec));
  L.front = o;
  L.front_stride = al(cap_front);
  o += 3 * L.front_stride;
  L.back = o;
  o += al(cap_back);
  L.node0 = o;
  o += al((size_t)cap_nodes * na * 8);
  L.node1 = o;
  o += al((size_t)cap_nodes * na * 8);
  L.coef0 = o;
  o += al((size_t)cap_nel * q * coef_bytes);
  L.coef1 = o;
  o += al((size_t)cap_nel * q * coef_bytes);
  L.lsm = o;
  o += al(sizeof(R) * (size_t)cap_lsm);
  L.flag = o;  // phase 1: compacted list of the elements to redo in double
  o += al(sizeof(uint32_t) * (size_t)cap_nel);
  L.total = o;
  return L;
}

// ---- PTX helpers (TMA bulk copy, mbarrier, cp.async) -------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* mb, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(mb)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void tma_load_block(void* dst, const void* src, uint32_t bytes, uint64_t* mb) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(mb)), "r"(bytes) : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(mb))
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* mb, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(mb)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Bounded wait for phase `parity` of mb; true if it completed.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* mb, uint32_t parity, long long limit_ns) {
  if (mbar_try_wait(mb, parity)) return true;
  const uint64_t t0 = global_ns();
  while (true) {
    if (mbar_try_wait(mb, parity)) return true;
    if ((long long)(global_ns() - t0) > limit_ns) return false;
  }
}

__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Store to global memory by an explicitly global address (a generic store
// could alias shared memory and would pin later shared loads behind it).
__device__ __forceinline__ void st_global(float* p, float v) { __stcg(p, v); }
__device__ __forceinline__ void st_global(double* p, double v) { __stcg(p, v); }
// Four consecutive values at a 16-byte aligned address.
__device__ __forceinline__ void st_global4(float* p, const float (&v)[4]) {
  __stcg(reinterpret_cast<float4*>(p), make_float4(v[0], v[1], v[2], v[3]));
}
__device__ __forceinline__ void st_global4(double* p, const double (&v)[4]) {
  __stcg(reinterpret_cast<double2*>(p), make_double2(v[0], v[1]));
  __stcg(reinterpret_cast<double2*>(p) + 1, make_double2(v[2], v[3]));
}

// General-rule tiles: cp.async gathers of the tile's element coefficients
// from its front part (compile-time-rule tiles read theirs from global memory
// in phase 1).
__device__ __forceinline__ void issue_coef_gathers(const MeshRec& mr, bool want_coef, const uint8_t* front,
                                                   void* coef_dst) {
  if (!want_coef || mr.type >= kFastTypeOffset) return;
  const TileHdr h = *reinterpret_cast<const TileHdr*>(front);
  const TileLayout L = tile_layout(h, mr.ref, mr.entb);
  const int q = mr.tab.q;
  const int32_t* el = reinterpret_cast<const int32_t*>(front + L.elem);
  for (int j = threadIdx.x; j < h.nel; j += blockDim.x) {
    const int64_t g0 = (int64_t)el[j] * q;
    if (mr.coef_f32) {
      for (int qq = 0; qq < q; ++qq)
        cp_async4(static_cast<float*>(coef_dst) + j * q + qq, static_cast<const float*>(mr.coef) + g0 + qq);
    } else {
      for (int qq = 0; qq < q; ++qq)
        cp_async8(static_cast<double*>(coef_dst) + j * q + qq, static_cast<const double*>(mr.coef) + g0 + qq);
    }
  }
}

// Element data from split node coordinates held in shared memory (hi, lo pairs).
template <int D, int NA, int P>
__device__ __forceinline__ void element_data_from_pairs(const float2* __restrict__ xs, const uint16_t* __restrict__ en,
                                                        ElemData<D, NA, P, float>& ed) {
  constexpr int REF = Ref<D, P>::REF;
  float xh[REF][NA], xl[REF][NA];
#pragma unroll
  for (int b = 0; b < REF; ++b) {
    const int v = en[b];
#pragma unroll
    for (int i = 0; i < NA; ++i) {
      const float2 t = xs[v * NA + i];
      xh[b][i] = t.x;
      xl[b][i] = t.y;
    }
  }
#pragma unroll
  for (int m = 0; m < D; ++m)
#pragma unroll
    for (int i = 0; i < NA; ++i) ed.e[m][i] = (xh[m + 1][i] - xh[0][i]) + (xl[m + 1][i] - xl[0][i]);
#pragma unroll
  for (int k = 0; k < Ref<D, P>::NE; ++k) {
    const int I = edge_i<D>(k), J = edge_j<D>(k), Ed = D + 1 + k;
#pragma unroll
    for (int i = 0; i < NA; ++i) {
      // explicit multiply-add: one rounding order in every kernel
      const float dh = fmaf(-0.5f, xh[J][i] - xh[I][i], xh[Ed][i] - xh[I][i]);
      const float dlo = fmaf(-0.5f, xl[J][i] - xl[I][i], xl[Ed][i] - xl[I][i]);
      ed.dl[k][i] = dh + dlo;
    }
  }
}

// The same element data in double from the split pairs: each difference of
// hi parts and of lo parts is exact in double, so e and dl are the exact
// differences of the double coordinates up to one final rounding.
template <int D, int NA, int P>
__device__ __forceinline__ void element_data64_from_pairs(const float2* __restrict__ xs,
                                                          const uint16_t* __restrict__ en,
                                                          ElemData<D, NA, P, double>& ed) {
  constexpr int REF = Ref<D, P>::REF;
  double xh[REF][NA], xl[REF][NA];
#pragma unroll
  for (int b = 0; b < REF; ++b) {
    const int v = en[b];
#pragma unroll
    for (int i = 0; i < NA; ++i) {
      const float2 t = xs[v * NA + i];
      xh[b][i] = (double)t.x;
      xl[b][i] = (double)t.y;
    }
  }
#pragma unroll
  for (int m = 0; m < D; ++m)
#pragma unroll
    for (int i = 0; i < NA; ++i) ed.e[m][i] = (xh[m + 1][i] - xh[0][i]) + (xl[m + 1][i] - xl[0][i]);
#pragma unroll
  for (int k = 0; k < Ref<D, P>::NE; ++k) {
    const int I = edge_i<D>(k), J = edge_j<D>(k), Ed = D + 1 + k;
#pragma unroll
    for (int i = 0; i < NA; ++i)
      ed.dl[k][i] = ((xh[Ed][i] - xh[I][i]) + (xl[Ed][i] - xl[I][i])) -
                    0.5 * ((xh[J][i] - xh[I][i]) + (xl[J][i] - xl[I][i]));
  }
}

// A triangle that failed the conditioning test, again: per quadrature point
// the geometry in double -- J from the exact differences of the split
// coordinates and the rule's double tables, s = |det DF|, and the R^{-T}
// factors c1, c2, c3 (as in tri_fast2) -- rounded to float, then the float
// contraction, one point at a time (few registers: this rare path shares the
// kernel with the hot one).  Every factor is then accurate to float rounding,
// so the error no longer grows with the conditioning (the float |det DF| of
// nearly parallel edge vectors loses about log2 cond(J) bits).  Every
// requested matrix goes to dst (element block, slots M, A, MC of the
// requested ones).  Returns false on a zero or non-finite |det DF|.
template <int NA, int P>
__device__ __forceinline__ bool redo_geo64(const float2* xs, const uint16_t* en, TabRef tab, const FastBank& fb,
                                           const float* cs, const double* cd, unsigned which, float* dst) {
  constexpr int REF = Ref<2, P>::REF, U = Ref<2, P>::U, NE = Ref<2, P>::NE, UP = lsm_stride(U);
  constexpr int Q = FastQ<2, P>::Q;
  ElemData<2, NA, P, double> ed;
  element_data64_from_pairs<2, NA, P>(xs, en, ed);
  const TabView<double> tb = tab_view<2, P, double>(tab);
  float Ao[UP];
#pragma unroll
  for (int u = 0; u < UP; ++u) Ao[u] = 0.f;
  float sq[Q];
  bool good = true;
#pragma unroll 1
  for (int q = 0; q < Q; ++q) {
    double J[NA][2];
#pragma unroll
    for (int i = 0; i < NA; ++i)
#pragma unroll
      for (int m = 0; m < 2; ++m) {
        double acc = ed.e[m][i];
#pragma unroll
        for (int e = 0; e < NE; ++e) acc = fma(ed.dl[e][i], tb.dpsi[(q * NE + e) * 2 + m], acc);
        J[i][m] = acc;
      }
    double g11 = 0.0, g12 = 0.0;
#pragma unroll
    for (int i = 0; i < NA; ++i) {
      g11 = fma(J[i][0], J[i][0], g11);
      g12 = fma(J[i][0], J[i][1], g12);
    }
    double sd;
    if constexpr (NA == 2) {
      sd = fabs(J[0][0] * J[1][1] - J[0][1] * J[1][0]);
    } else {
      const double n0 = J[1][0] * J[2][1] - J[2][0] * J[1][1];
      const double n1 = J[2][0] * J[0][1] - J[0][0] * J[2][1];
      const double n2 = J[0][0] * J[1][1] - J[1][0] * J[0][1];
      sd = sqrt(n0 * n0 + n1 * n1 + n2 * n2);
    }
    good &= (sd > 0.0) & (sd <= 1.0e300);
    sq[q] = (float)sd;
    if (which & LFEM_STIFF) {
      const double c1d = sqrt(tb.w[q] * sd) / sqrt(g11), kd = c1d / sd;
      const float c1 = (float)c1d, c2 = (float)(kd * g11), c3 = (float)(kd * g12);
      float y0[REF], y1[REF];
#pragma unroll
      for (int b = 0; b < REF; ++b) {
        const float gb1 = (float)tb.dphi[(q * REF + b) * 2], gb2 = (float)tb.dphi[(q * REF + b) * 2 + 1];
        y0[b] = c1 * gb1;
        y1[b] = fmaf(c2, gb2, -(c3 * gb1));
      }
#pragma unroll
      for (int a = 0; a < REF; ++a)
#pragma unroll
        for (int b = a; b < REF; ++b) {
          const int u = upper_index(REF, a, b);
          Ao[u] = fmaf(y1[a], y1[b], fmaf(y0[a], y0[b], Ao[u]));
        }
    }
  }
  int slot = 0;
  if (which & LFEM_MASS) contract_mass2<2, P>(fb, sq, dst + 2 * slot++);
  if (which & LFEM_STIFF) {
    float* d = dst + 2 * slot++;
#pragma unroll
    for (int j = 0; j < UP / 2; ++j) *reinterpret_cast<float2*>(d + 6 * j) = make_float2(Ao[2 * j], Ao[2 * j + 1]);
  }
  if (which & LFEM_CMASS) {
    float sc[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) sc[q] = sq[q] * (cs ? __ldg(cs + q) : (float)__ldg(cd + q));
    contract_mass2<2, P>(fb, sc, dst + 2 * slot);
  }
  return good;
}

// Quadrature loop of one element over the points q = q0, q0 + qs, ... (a lane
// pair splits the points; the partial sums are combined by the caller).
template <int D, int NA, int P, typename R, bool DM, bool DA, bool DC>
__device__ __forceinline__ void element_pass_split(const ElemData<D, NA, P, R>& ed, const TabView<R>& tb,
                                                   const void* coef, int coef_f32, int q0, int qs,
                                                   R (&Mo)[Ref<D, P>::U], R (&Ao)[Ref<D, P>::U],
                                                   R (&Co)[Ref<D, P>::U], R& qual, bool& bad) {
  constexpr int U = Ref<D, P>::U;
#pragma unroll
  for (int u = 0; u < U; ++u) {
    if (DM) Mo[u] = 0;
    if (DA) Ao[u] = 0;
    if (DC) Co[u] = 0;
  }
#pragma unroll 1
  for (int q = q0; q < tb.q; q += qs) {
    const R wq = tb.w[q];
    QpGeom<D, NA, P, R> g;
    qp_geometry<D, NA, P, R>(ed, tb, q, wq, g);
    qual = fmin(qual, g.quality);
    bad |= !(g.s > (R)0) || !isfinite(g.s) || !(g.quality > (sizeof(R) == 8 ? (R)1e-28 : (R)1e-12));
    R cq = 0;
    if (DC) cq = coef_f32 ? (R)static_cast<const float*>(coef)[q] : (R)static_cast<const double*>(coef)[q];
    qp_accumulate<D, NA, P, R, DM, DA, DC>(g, tb, q, wq, cq, Mo, Ao, Co);
  }
}

template <typename R>
__device__ __forceinline__ R pair_sum(R v) {
  return v + __shfl_xor_sync(0xffffffffu, v, 1);
}

// Local matrices of one element by a lane pair, stored into the element's
// block of the interleaved tile layout (dst = element base; matrix slots im,
// ia, ic); stride_m is the number of matrix slots per entry pair (entry u of
// slot m at word 2 stride_m (u / 2) + 2 m + u mod 2).
template <int D, int NA, int P, typename R, bool DM, bool DA, bool DC>
__device__ __forceinline__ void element_pair(const ElemData<D, NA, P, R>& ed, const TabView<R>& tb, const void* coef,
                                             int coef_f32, int sub, bool store, R* dst, int stride_m, int im,
                                             int ia, int ic, R& qual, bool& bad) {
  constexpr int U = Ref<D, P>::U;
  R Mo[U], Ao[U], Co[U];
  element_pass_split<D, NA, P, R, DM, DA, DC>(ed, tb, coef, coef_f32, sub, kPipeTPE, Mo, Ao, Co, qual, bad);
#pragma unroll
  for (int u = 0; u < U; ++u) {
    if (DM) Mo[u] = pair_sum(Mo[u]);
    if (DA) Ao[u] = pair_sum(Ao[u]);
    if (DC) Co[u] = pair_sum(Co[u]);
  }
  // the even lane stores the mass-type matrices, the odd lane the stiffness
  // (when only one kind is computed, the even lane stores it)
  const bool lane_m = (DM || DC) && (sub == 0);
  const bool lane_a = DA && (sub == ((DM || DC) ? 1 : 0));
  if (store && lane_m) {
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (DM) dst[2 * stride_m * (u >> 1) + 2 * im + (u & 1)] = Mo[u];
      if (DC) dst[2 * stride_m * (u >> 1) + 2 * ic + (u & 1)] = Co[u];
    }
  }
  if (store && lane_a) {
#pragma unroll
    for (int u = 0; u < U; ++u) dst[2 * stride_m * (u >> 1) + 2 * ia + (u & 1)] = Ao[u];
  }
}

template <int D, int NA, int P, typename R>
__device__ __forceinline__ void element_pair_dispatch(const ElemData<D, NA, P, R>& ed, const TabView<R>& tb,
                                                      const void* coef, int coef_f32, int sub, bool store, R* dst,
                                                      int mstride, unsigned which, R& qual, bool& bad) {
  const bool wm = which & LFEM_MASS, wa = which & LFEM_STIFF, wc = which & LFEM_CMASS;
  const int im = 0, ia = wm ? 1 : 0, ic = (wm ? 1 : 0) + (wa ? 1 : 0);
  if constexpr (D == 3) {
    // one matrix per pass: 55 accumulators at most
    if (wm) element_pair<D, NA, P, R, true, false, false>(ed, tb, coef, coef_f32, sub, store, dst, mstride, im, ia, ic, qual, bad);
    if (wc) element_pair<D, NA, P, R, false, false, true>(ed, tb, coef, coef_f32, sub, store, dst, mstride, im, ia, ic, qual, bad);
    if (wa) element_pair<D, NA, P, R, false, true, false>(ed, tb, coef, coef_f32, sub, store, dst, mstride, im, ia, ic, qual, bad);
  } else {
    if (wm && wa && wc)
      element_pair<D, NA, P, R, true, true, true>(ed, tb, coef, coef_f32, sub, store, dst, mstride, im, ia, ic, qual, bad);
    else if (wm && wa)
      element_pair<D, NA, P, R, true, true, false>(ed, tb, coef, coef_f32, sub, store, dst, mstride, im, ia, ic, qual, bad);
    else if (wm && wc)
      element_pair<D, NA, P, R, true, false, true>(ed, tb, coef, coef_f32, sub, store, dst, mstride, im, ia, ic, qual, bad);
    else if (wa && wc)
      element_pair<D, NA, P, R, false, true, true>(ed, tb, coef, coef_f32, sub, store, dst, mstride, im, ia, ic, qual, bad);
    else if (wm)
      element_pair<D, NA, P, R, true, false, false>(ed, tb, coef, coef_f32, sub, store, dst, mstride, im, ia, ic, qual, bad);
    else if (wa)
      element_pair<D, NA, P, R, false, true, false>(ed, tb, coef, coef_f32, sub, store, dst, mstride, im, ia, ic, qual, bad);
    else
      element_pair<D, NA, P, R, false, false, true>(ed, tb, coef, coef_f32, sub, store, dst, mstride, im, ia, ic, qual, bad);
  }
}

// Node coordinates of a tile into its node buffer, by one warp.  With a
// 16-byte aligned coordinate array lane 0 first posts the byte count of the
// runs on the mbarrier, then every run is one TMA bulk copy (lane r issues
// run r) and the extras are loaded and stored by the lanes; otherwise the
// lanes load and store every position.  Lane 0 arrives on the mbarrier once
// the lanes' own stores are done, so the phase completes when both the bulk
// copies and the stores are in place.
__device__ __forceinline__ void issue_node_copies(const MeshRec& mr, const uint8_t* front, double* dst, uint64_t* mb,
                                                  int lane) {
  const TileHdr h = *reinterpret_cast<const TileHdr*>(front);
  const TileLayout L = tile_layout(h, mr.ref, mr.entb);
  const int na = mr.na;
  if (mr.c16) {
    const int4* runs = reinterpret_cast<const int4*>(front + L.runs);
    const int2* extras = reinterpret_cast<const int2*>(front + L.extras);
    uint32_t bytes = 0;
    for (int r = lane; r < h.nruns; r += 32) bytes += (uint32_t)runs[r].y * (uint32_t)na * 8u;
    for (int o = 16; o > 0; o >>= 1) bytes += __shfl_xor_sync(0xffffffffu, bytes, o);
    if (lane == 0)
      asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(mb)), "r"(bytes)
                   : "memory");
    __syncwarp();
    for (int r = lane; r < h.nruns; r += 32) {
      const int4 q = runs[r];
      asm volatile(
          "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
              smem_addr(dst + (size_t)q.z * na)),
          "l"(mr.coords + (int64_t)q.x * na), "r"((uint32_t)q.y * (uint32_t)na * 8u), "r"(smem_addr(mb))
          : "memory");
    }
    for (int x = lane; x < h.nextra; x += 32) {
      const int2 e = extras[x];
      for (int c = 0; c < na; ++c) dst[(size_t)e.y * na + c] = __ldg(mr.coords + (int64_t)e.x * na + c);
    }
  } else {
    const int32_t* nd = reinterpret_cast<const int32_t*>(front + L.nodes);
    for (int v = lane; v < h.nnodes; v += 32)
      for (int c = 0; c < na; ++c) dst[(size_t)v * na + c] = __ldg(mr.coords + (int64_t)nd[v] * na + c);
  }
  __threadfence_block();
  __syncwarp();
  if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(mb)) : "memory");
}

// Node coordinates of a tile -> (hi, lo) float pairs in place (float kernels;
// nothing for the double kernels), by every thread.
template <typename R>
__device__ __forceinline__ void split_nodes(double* xd, int nvals) {
  if constexpr (sizeof(R) == 4) {
    for (int i = threadIdx.x; i < nvals; i += blockDim.x) {
      float hi, lo;
      bool ok = true;
      split_f64(xd[i], hi, lo, ok);
      if (!ok) hi = __int_as_float(0x7fc00000);  // out of float range: NaN forces the double path
      reinterpret_cast<float2*>(xd)[i] = make_float2(hi, lo);
    }
  }
}

// Everything done for one tile whose front part, (split) node coordinates and
// coefficients are in shared memory: the next items' copies (issue_next),
// phase 1, then -- once wait_back() says the back part has landed -- the
// double fallback (if any element was flagged) and phase 2.  Returns false if
// that wait ran out (nothing is written then).
template <int D, int NA, int P, bool FAST, typename R, typename EntT, typename IssueNext, typename WaitBack>
__device__ __forceinline__ bool process_tile(const PipeArgs& a, const MeshRec& mr, const uint8_t* front,
                                             const uint8_t* back, double* xd, const void* coef_s, R* lsm,
                                             uint32_t* flist, int* nflag, const FastBank& fb, IssueNext&& issue_next,
                                             WaitBack&& wait_back) {
  constexpr int REF = Ref<D, P>::REF;
  constexpr int U = Ref<D, P>::U;
  constexpr int UP = lsm_stride(U);
  // matrix slots per entry pair: three (float), the requested ones (double)
  constexpr bool COMPACT = sizeof(R) == 8;
  const int NS = COMPACT ? a.nm : kLsmSlots;
  const int EW = NS * UP;  // words of one element's local matrices
  auto wconv = [&](uint32_t w) -> uint32_t {
    if constexpr (COMPACT) return 2u * (uint32_t)NS * (w / 6u) + w % 6u;
    else return w;
  };
  constexpr int ENTB = (int)sizeof(EntT);
  using Acc = typename AccOf<R>::T;
  const int nm = a.nm, Q = mr.tab.q;
  const int coef_bytes = a.coef_bytes;
  const TabView<R> tb = tab_view<D, P, R>(mr.tab);
  const TileHdr h = *reinterpret_cast<const TileHdr*>(front);
  const TileLayout TL = tile_layout(h, REF, ENTB);
  const int32_t* t_elem = reinterpret_cast<const int32_t*>(front + TL.elem);
  const int32_t* t_nodes = reinterpret_cast<const int32_t*>(front + TL.nodes);
  const uint16_t* t_en = reinterpret_cast<const uint16_t*>(front + TL.enodes);
  const EntT* t_pair = reinterpret_cast<const EntT*>(back + TL.pair);
  const int4* t_lrec = reinterpret_cast<const int4*>(back + TL.lrec);
  const EntT* t_lent = reinterpret_cast<const EntT*>(back + TL.lent);

  // (the node coordinates in xd are already split for the float kernels;
  // *nflag is 0 on entry)
  const int LB = NS * h.nel * UP;  // long-slot results after the elements, then 2 NS zero words
  if (threadIdx.x < 2 * NS) lsm[LB + 2 * NS * h.nl + threadIdx.x] = (R)0;
  // the copies of the next items, issued while phase 1 runs
  issue_next();

  if constexpr (FAST && sizeof(R) == 4) {
    // ---- phase 1, compile-time rule: one thread per element, every element of the tile
    for (int jt = threadIdx.x; jt < h.nel; jt += blockDim.x) {
      ElemData<D, NA, P, float> ed;
      element_data_from_pairs<D, NA, P>(reinterpret_cast<const float2*>(xd), t_en + (size_t)jt * REF, ed);
      // coefficients of the element from global memory (loaded first, used last)
      const int64_t cg = (int64_t)t_elem[jt] * Q;
      const float* cs = coef_bytes == 4 ? static_cast<const float*>(mr.coef) + cg : nullptr;
      const double* cd = coef_bytes == 8 ? static_cast<const double*>(mr.coef) + cg : nullptr;
      Checks ck;
      element_fast_store2<D, NA, P>(ed, fb, cs, cd, a.qmin, a.which, reinterpret_cast<float*>(lsm) + (size_t)jt * EW,
                                    ck);
      const uint32_t fl = !ck.good ? 2u : (ck.cond ? 0u : 1u);
      if (fl) flist[atomicAdd(nflag, 1)] = (uint32_t)jt | (fl << 30);
    }
  } else {
    // ---- phase 1: a lane pair per element, every element of the tile
    for (int c0 = 0; c0 < h.nel; c0 += a.chunk) {
      const int cn = min(a.chunk, h.nel - c0);
      const int jj = threadIdx.x / kPipeTPE, sub = threadIdx.x % kPipeTPE;
      const bool active = jj < cn;
      const int jt = c0 + (active ? jj : 0);
      const uint16_t* en = t_en + (size_t)jt * REF;
      const void* cf = coef_s;
      if (coef_bytes) cf = static_cast<const uint8_t*>(cf) + (size_t)jt * Q * coef_bytes;
      R qual = (R)1;
      bool bad = false;
      R* dst = lsm + (size_t)jt * EW;
      if constexpr (sizeof(R) == 4) {
        ElemData<D, NA, P, float> ed;
        element_data_from_pairs<D, NA, P>(reinterpret_cast<const float2*>(xd), en, ed);
        element_pair_dispatch<D, NA, P, float>(ed, tb, cf, mr.coef_f32, sub, active, dst, NS, a.which, qual, bad);
      } else {
        double X[REF][NA];
#pragma unroll
        for (int bb = 0; bb < REF; ++bb)
#pragma unroll
          for (int i = 0; i < NA; ++i) X[bb][i] = xd[en[bb] * NA + i];
        ElemData<D, NA, P, double> ed;
        load_element_data<D, NA, P, double>(X, ed);
        element_pair_dispatch<D, NA, P, double>(ed, tb, cf, mr.coef_f32, sub, active, dst, NS, a.which, qual, bad);
      }
      const R q2 = fmin(qual, __shfl_xor_sync(0xffffffffu, qual, 1));
      const bool bad2 = bad || __shfl_xor_sync(0xffffffffu, (int)bad, 1);
      if (active && sub == 0) {
        if constexpr (sizeof(R) == 4) {
          const uint32_t fl = bad2 ? 2u : ((D > 1 && q2 < (R)a.qmin) ? 1u : 0u);
          if (fl) flist[atomicAdd(nflag, 1)] = (uint32_t)jt | (fl << 30);
        } else {
          const int32_t n0 = t_nodes[en[0]];
          if (bad2 && n0 >= h.r0 && n0 < h.r0 + h.nrows) atomicOr(a.status, ST_DEGENERATE);
        }
      }
    }
  }
  // the back part (slot entries) must have landed; the barrier also
  // publishes phase 1's local matrices and the flag count
  if (!wait_back()) return false;
  if constexpr (sizeof(R) == 4) {
    const int nf = *nflag;  // the same in every thread after the barrier
    if (nf > 0) {
      // rare path: every requested matrix of a flagged element again, from a
      // compacted list so that whole warps work on it (the FP64 pipe costs
      // the same for a warp instruction with few active lanes).  An element
      // that failed the conditioning test (1): with the compile-time rule on
      // triangles its per-point geometry in double and the float contraction
      // (its float |det DF| and metric lose about log2 cond(J) bits, the
      // float contraction of double-accurate factors does not); otherwise,
      // and for an element that failed the finiteness test (2), everything
      // in double from the global coordinates.
      for (int i = threadIdx.x; i < nf; i += blockDim.x) {
        const uint32_t v = flist[i];
        const int j = (int)(v & 0x3FFFFFFFu), fl = (int)(v >> 30);
        const uint16_t* en = t_en + (size_t)j * REF;
        int32_t nd[REF];
#pragma unroll
        for (int bb = 0; bb < REF; ++bb) nd[bb] = t_nodes[en[bb]];
        bool bad = false;
        R* d = lsm + (size_t)j * EW;
        if constexpr (FAST && D == 2) {
          if (fl == 1) {
            const int64_t cg = (int64_t)t_elem[j] * Q;
            const float* cs = coef_bytes == 4 ? static_cast<const float*>(mr.coef) + cg : nullptr;
            const double* cd = coef_bytes == 8 ? static_cast<const double*>(mr.coef) + cg : nullptr;
            const bool good = redo_geo64<NA, P>(reinterpret_cast<const float2*>(xd), en, mr.tab, fb, cs, cd, a.which,
                                                reinterpret_cast<float*>(d));
            if (nd[0] >= h.r0 && nd[0] < h.r0 + h.nrows) {
              atomicAdd(a.fallback, 1ull);
              if (!good) atomicOr(a.status, ST_DEGENERATE);
            }
            continue;
          }
        }
        element_fp64_lean<D, NA, P, float, true>(mr.coords, nd, mr.tab, mr.coef, mr.coef_f32, (int64_t)t_elem[j],
                                                 a.which, d, 0, bad, 0);
        if (nd[0] >= h.r0 && nd[0] < h.r0 + h.nrows) {
          atomicAdd(a.fallback, 1ull);
          if (bad) atomicOr(a.status, ST_DEGENERATE);
        }
      }
      __syncthreads();
      if (threadIdx.x == 0) *nflag = 0;  // every thread has read it; the next tile's phase 1 follows a barrier
    }
  }

  // ---- phase 2a: slots with more than two contributions (vertex diagonals),
  // one thread each, summed in ascending (element, a, b) order with a
  // compensated pair into the long-result words; entries and values are
  // loaded four at a time so that only the additions form a chain
  for (int j = threadIdx.x; j < h.nl; j += blockDim.x) {
    const int4 r = t_lrec[j];
    Acc c0, c1, c2;
    bool first = true;
    for (int k0 = r.y; k0 < r.z; k0 += 4) {
      uint32_t ent[4];
      R v0[4], v1[4], v2[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        ent[i] = k0 + i < r.z ? wconv(t_lent[k0 + i]) : 0u;
        v0[i] = lsm[ent[i]];
        v1[i] = nm > 1 ? lsm[ent[i] + 2] : (R)0;
        v2[i] = nm > 2 ? lsm[ent[i] + 4] : (R)0;
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        if (k0 + i >= r.z) break;
        if (first) {
          acc_init(c0, v0[i]);
          acc_init(c1, v1[i]);
          acc_init(c2, v2[i]);
          first = false;
        } else {
          acc_add(c0, v0[i]);
          acc_add(c1, v1[i]);
          acc_add(c2, v2[i]);
        }
      }
    }
    R* lr = lsm + LB + 2 * NS * r.w;
    lr[0] = (R)acc_final(c0);
    if (nm > 1) lr[2] = (R)acc_final(c1);
    if (nm > 2) lr[4] = (R)acc_final(c2);
  }
  __syncthreads();

  // ---- phase 2b: every slot = its first entry + its second entry (the zero
  // word for a single contribution or a long result), four consecutive slots
  // per thread, one writer per slot -- fixed order, no atomics
  {
    R* o[3];
#pragma unroll
    for (int m = 0; m < 3; ++m) o[m] = reinterpret_cast<R*>(mr.out[m < nm ? m : 0]);
    const int64_t gs0 = h.s0 - h.apad;  // global slot of padded slot 0 (a multiple of 4)
    const int ng = TL.npad >> 2;
    const int lo = h.apad, hi = h.apad + h.ns;
    for (int g = threadIdx.x; g < ng; g += blockDim.x) {
      uint32_t x[4], y[4];
      if constexpr (ENTB == 2) {
        const uint4 w = reinterpret_cast<const uint4*>(t_pair)[g];
        x[0] = w.x & 0xFFFFu, y[0] = w.x >> 16;
        x[1] = w.y & 0xFFFFu, y[1] = w.y >> 16;
        x[2] = w.z & 0xFFFFu, y[2] = w.z >> 16;
        x[3] = w.w & 0xFFFFu, y[3] = w.w >> 16;
      } else {
        const uint4 w0 = reinterpret_cast<const uint4*>(t_pair)[2 * g];
        const uint4 w1 = reinterpret_cast<const uint4*>(t_pair)[2 * g + 1];
        x[0] = w0.x, y[0] = w0.y, x[1] = w0.z, y[1] = w0.w;
        x[2] = w1.x, y[2] = w1.y, x[3] = w1.z, y[3] = w1.w;
      }
      R v[3][4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        x[i] = wconv(x[i]);
        y[i] = wconv(y[i]);
        v[0][i] = lsm[x[i]] + lsm[y[i]];
        if (nm > 1) v[1][i] = lsm[x[i] + 2] + lsm[y[i] + 2];
        if (nm > 2) v[2][i] = lsm[x[i] + 4] + lsm[y[i] + 4];
      }
      const int p0 = 4 * g;
      const int64_t gs = gs0 + p0;
      if (a.vec_out && p0 >= lo && p0 + 4 <= hi) {
#pragma unroll
        for (int m = 0; m < 3; ++m)
          if (m < nm) st_global4(o[m] + gs, v[m]);
      } else {
#pragma unroll
        for (int i = 0; i < 4; ++i)
          if (p0 + i >= lo && p0 + i < hi) {
#pragma unroll
            for (int m = 0; m < 3; ++m)
              if (m < nm) st_global(o[m] + gs + i, v[m][i]);
          }
      }
    }
  }
  return true;
}

// Element type of a launch; the compile-time-rule variant has its own id, so a
// batch can hold meshes of one type with and without the usual rule.
template <int D_, int NA_, int P_, bool FAST_ = false>
struct EType {
  static constexpr int D = D_, NA = NA_, P = P_;
  static constexpr bool FAST = FAST_;
  static constexpr int id = elem_type_id(D_, NA_, P_) + (FAST_ ? kFastTypeOffset : 0);
};

template <typename R, typename EntT, typename T0, typename... Ts, typename IssueNext, typename WaitBack>
__device__ __forceinline__ bool dispatch_tile(int type, const PipeArgs& a, const MeshRec& mr, const uint8_t* front,
                                              const uint8_t* back, double* xd, const void* coef_s, R* lsm,
                                              uint32_t* flist, int* nflag, const FastBank& fb, IssueNext&& issue_next,
                                              WaitBack&& wait_back) {
  if (type == T0::id) {
    return process_tile<T0::D, T0::NA, T0::P, T0::FAST, R, EntT>(a, mr, front, back, xd, coef_s, lsm, flist, nflag,
                                                                 fb, issue_next, wait_back);
  } else {
    if constexpr (sizeof...(Ts) > 0) {
      return dispatch_tile<R, EntT, Ts...>(type, a, mr, front, back, xd, coef_s, lsm, flist, nflag, fb, issue_next,
                                           wait_back);
    } else {
      // no variant for this tile's type: report it, keep the pipeline's steps
      if (threadIdx.x == 0) atomicOr(a.status, ST_TYPE);
      issue_next();
      return wait_back();
    }
  }
}

// Persistent launch over work items; Types lists the element types the launch
// may meet (one for a single mesh, several for a batch).
template <typename R, typename EntT, typename... Types>
__global__ void __launch_bounds__(PipeOcc<R>::THREADS, PipeOcc<R>::MIN_BLOCKS)
    k_assemble_pipe(const PipeArgs a, const __grid_constant__ FastBank fb) {
  extern __shared__ __align__(128) unsigned char pipe_smem[];
  const bool want_coef = a.coef_bytes != 0;
  const PipeSmem L = pipe_smem_layout<R>(3, a.cap_lsm, a.cap_front, a.cap_back, a.cap_nodes, a.cap_nel, a.max_q,
                                         a.coef_smem);
  // mbarriers: [0..2] front buffers, [3] the back buffer, [4], [5] node buffers
  uint64_t* mbar = reinterpret_cast<uint64_t*>(pipe_smem + L.mbar);
  int* s_nflag = reinterpret_cast<int*>(pipe_smem + L.mbar + 68);
  ItemRef* s_ref = reinterpret_cast<ItemRef*>(pipe_smem + L.refs);
  MeshRec* s_rec = reinterpret_cast<MeshRec*>(pipe_smem + L.rec);
  // buffers as shared-memory base + offset (no pointer arrays: a pointer
  // loaded back from local memory would turn every access generic)
  auto front_of = [&](int f) { return pipe_smem + L.front + (size_t)f * L.front_stride; };
  uint8_t* s_back = pipe_smem + L.back;
  auto node_of = [&](int b) { return reinterpret_cast<double*>(pipe_smem + (b ? L.node1 : L.node0)); };
  auto coef_of = [&](int b) { return static_cast<void*>(pipe_smem + (b ? L.coef1 : L.coef0)); };
  R* lsm = reinterpret_cast<R*>(pipe_smem + L.lsm);
  uint32_t* flist = reinterpret_cast<uint32_t*>(pipe_smem + L.flag);

  const int64_t G = gridDim.x;
  const int64_t i0 = blockIdx.x;
  if (i0 >= a.n_items) return;
  // item index of the CTA's k-th work item in s_item[k & 3] (-1: none): the
  // first is blockIdx.x, every later one a ticket drawn three items ahead
  // (items past the first gridDim.x go to whichever CTA asks first)
  int* s_item = reinterpret_cast<int*>(pipe_smem + L.mbar + 80);
  auto item_of = [&](int64_t k) -> int { return s_item[k & 3]; };
  // the copies are issued by the last warp (it has the fewest phase-1
  // elements), the whole-block ones by its last thread, the producer
  const bool pwarp = threadIdx.x >= blockDim.x - 32;
  const bool producer = threadIdx.x == blockDim.x - 1;
  const int lane = threadIdx.x & 31;
  // copies in flight per mbarrier (bit b; the producer's record) and the
  // parity of each mbarrier's next phase (the same in every thread); each
  // mbarrier has at most one phase in flight
  uint32_t pend = 0, par = 0;

  // producer: a ticket for the CTA's item k into s_item[k & 3] and its record
  // into s_ref[k & 3] (cp.async, landed by the next cp.async wait); the ticket
  // was drawn at the previous call, so the atomic's latency is not waited for
  unsigned int tk = 0;
  auto draw = [&](int64_t k) {
    const int64_t idx = G + (int64_t)tk;
    tk = atomicAdd(a.next_item, 1u);
    const int it = idx < a.n_items ? (int)idx : -1;
    s_item[k & 3] = it;
    if (it >= 0) {
      const ItemRef* src = a.items + it;
      ItemRef* dst = s_ref + (k & 3);
      cp_async16(dst, src);
      cp_async16(reinterpret_cast<uint8_t*>(dst) + 16, reinterpret_cast<const uint8_t*>(src) + 16);
    }
  };
  // a record is used only if its copies fit the buffers and meet the bulk
  // copies' 16-byte rules; otherwise the producer flags it (s_bad, ST_ITEM),
  // issues nothing, and the CTA stops at its next barrier
  int* s_bad = reinterpret_cast<int*>(pipe_smem + L.mbar + 72);
  auto rec_ok = [&](const ItemRef& r) {
    const bool ok = r.front != nullptr && ((reinterpret_cast<uintptr_t>(r.front) & 15) == 0) &&
                    r.front_bytes >= (int)sizeof(TileHdr) && r.front_bytes <= a.cap_front &&
                    (r.front_bytes & 15) == 0 && r.back_bytes >= 16 && r.back_bytes <= a.cap_back &&
                    (r.back_bytes & 15) == 0 && (!a.meshes || r.mesh >= 0);
    if (!ok) {
      *s_bad = 1;
      atomicOr(a.status, ST_ITEM);
    }
    return ok;
  };
  // producer: mesh record of item k (a batch's by cp.async: read from the next
  // item on, after a cp.async wait) and the TMA copy of its front part into
  // front buffer k % 3
  auto load_front = [&](int64_t k) {
    const int f = (int)(k % 3);
    const ItemRef& r = s_ref[k & 3];
    if (!rec_ok(r)) return;
    if (a.meshes) {
      static_assert(sizeof(MeshRec) % 16 == 0, "mesh records are copied in 16-byte pieces");
      const uint8_t* src = reinterpret_cast<const uint8_t*>(a.meshes + r.mesh);
      uint8_t* dst = reinterpret_cast<uint8_t*>(s_rec + f);
      for (int o = 0; o < (int)sizeof(MeshRec); o += 16) cp_async16(dst + o, src + o);
    } else {
      s_rec[f] = a.one;
    }
    tma_load_block(front_of(f), r.front, (uint32_t)r.front_bytes, &mbar[f]);
    pend |= 1u << f;
  };
  // producer: TMA copy of item k's back part into the back buffer
  auto load_back = [&](int64_t k) {
    const ItemRef& r = s_ref[k & 3];
    if (!rec_ok(r)) return;
    tma_load_block(s_back, r.front + r.front_bytes, (uint32_t)r.back_bytes, &mbar[3]);
    pend |= 1u << 3;
  };
  // last warp: node coordinates of the item whose front part is in buffer f, into node buffer b
  auto load_nodes = [&](int f, int b) {
    fence_proxy_async();
    issue_node_copies(s_rec[f], front_of(f), node_of(b), &mbar[4 + b], lane);
    pend |= 1u << (4 + b);
  };
  // one thread's bounded wait for the next phase of mbarrier b (each thread
  // waits for itself; the outcome is agreed on at the next barrier)
  auto wait_one = [&](int b) -> bool { return mbar_wait_bounded(&mbar[b], (par >> b) & 1u, a.wait_ns); };
  auto passed = [&](int b) {
    par ^= 1u << b;
    pend &= ~(1u << b);
  };
  // item k+1's node coordinates: wait for them, split them (every thread)
  auto nodes_ready = [&](int f, int b) -> bool {
    if (!wait_one(4 + b)) return false;
    const TileHdr h = *reinterpret_cast<const TileHdr*>(front_of(f));
    split_nodes<R>(node_of(b), h.nnodes * s_rec[f].na);
    return true;
  };
  // a wait ran out: report it, give every copy still in flight one more
  // bounded wait (so that none lands in the shared memory of a later CTA), stop
  auto bail = [&]() {
    if (producer) {
      atomicOr(a.status, ST_TIMEOUT);
      for (int b = 0; b < 6; ++b)
        if (pend & (1u << b)) mbar_wait_bounded(&mbar[b], (par >> b) & 1u, a.wait_ns);
    }
    cp_async_wait_all();
  };

  if (threadIdx.x == 0) {
    for (int b = 0; b < 6; ++b) mbar_init(&mbar[b], 1);
    fence_mbar_init();
    *s_nflag = 0;
    *s_bad = 0;
    s_item[0] = (int)i0;
    const ItemRef* src = a.items + i0;
    cp_async16(s_ref, src);
    cp_async16(reinterpret_cast<uint8_t*>(s_ref) + 16, reinterpret_cast<const uint8_t*>(src) + 16);
  }
  if (producer) {
    tk = atomicAdd(a.next_item, 1u);
    draw(1);
    draw(2);
  }
  cp_async_commit();  // (wait_group waits for committed groups only)
  cp_async_wait_all();
  __syncthreads();
  if (producer) {
    if (!(a.starve && blockIdx.x == 0)) load_front(0);
    if (item_of(1) >= 0) load_front(1);
  }
  cp_async_commit();  // (the mesh records of a batch)
  cp_async_wait_all();
  {
    const bool ok = (*s_bad == 0) && wait_one(0);
    if (__syncthreads_or(!ok)) {
      bail();
      return;
    }
    passed(0);
  }
  // item 0's node coordinates and coefficients
  if (pwarp) load_nodes(0, 0);
  issue_coef_gathers(s_rec[0], want_coef, front_of(0), coef_of(0));
  cp_async_commit();
  bool carry = nodes_ready(0, 0);

  for (int64_t k = 0; item_of(k) >= 0; ++k) {
    const int f = (int)(k % 3), nb = (int)(k & 1);
    const bool has1 = item_of(k + 1) >= 0;
    const int f1 = (int)((k + 1) % 3);
    // item k's node coordinates (split), coefficients and item k+3's record
    // have landed, item k+1's front part is here, item k-1 has left every
    // buffer (one barrier)
    cp_async_wait_all();
    {
      bool ok = carry && *s_bad == 0;
      if (has1 && ok) ok = wait_one(f1);
      if (__syncthreads_or(!ok)) {
        bail();
        return;
      }
      passed(4 + nb);
      if (has1) passed(f1);
    }
    // the copies for items k+1 .. k+3 (called by every thread at the start of
    // item k's phase 1, so that their issue overlaps it)
    auto issue_next = [&]() {
      if (producer) {
        fence_proxy_async();
        load_back(k);
        if (item_of(k + 2) >= 0) {
          load_front(k + 2);
          draw(k + 3);
        } else {
          s_item[(k + 3) & 3] = -1;
        }
      }
      if (has1) {
        if (pwarp) load_nodes(f1, nb ^ 1);
        issue_coef_gathers(s_rec[f1], want_coef, front_of(f1), coef_of(nb ^ 1));
      }
      cp_async_commit();
    };
    auto wait_back = [&]() -> bool {
      const bool ok = *s_bad == 0 && wait_one(3);
      if (__syncthreads_or(!ok)) return false;
      passed(3);
      return true;
    };
    const MeshRec& mr = s_rec[f];
    if (!dispatch_tile<R, EntT, Types...>(mr.type, a, mr, front_of(f), s_back, node_of(nb), coef_of(nb), lsm, flist,
                                          s_nflag, fb, issue_next, wait_back)) {
      bail();
      return;
    }
    carry = has1 ? nodes_ready(f1, nb ^ 1) : true;
  }
  cp_async_wait_all();
}

template <typename R, typename EntT, typename... Types>
lfem_status launch_pipe_types(const PipeArgs& a, const FastBank& fb, int sm_count, cudaStream_t st) {
  if (a.n_items == 0) return LFEM_OK;
  if (a.n_items >= 0x7FFFFFFF) return fail(LFEM_E_TOO_LARGE, "more than 2^31 - 1 tiles in one launch");
  const size_t smem = pipe_smem_layout<R>(3, a.cap_lsm, a.cap_front, a.cap_back, a.cap_nodes, a.cap_nel, a.max_q,
                                          a.coef_smem)
                          .total;
  if (smem > 227 * 1024) {
    const PipeSmem L = pipe_smem_layout<R>(3, a.cap_lsm, a.cap_front, a.cap_back, a.cap_nodes, a.cap_nel, a.max_q,
                                           a.coef_smem);
    return fail(LFEM_E_TOO_LARGE,
                "pipelined tile needs " + std::to_string(smem / 1024) + " KB of shared memory (more than 227 KB): " +
                    "local matrices " + std::to_string((L.flag - L.lsm) / 1024) + " KB for " +
                    std::to_string(a.cap_nel) + " elements, node buffers " +
                    std::to_string((L.coef0 - L.node0) / 1024) + " KB for " + std::to_string(a.cap_nodes) +
                    " nodes, front parts " + std::to_string((L.back - L.front) / 1024) + " KB, back part " +
                    std::to_string((L.node0 - L.back) / 1024) + " KB; use a smaller tile capacity");
  }
  auto kern = k_assemble_pipe<R, EntT, Types...>;
  LFEM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  LFEM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, PipeOcc<R>::THREADS, smem));
  if (per_sm < 1) return fail(LFEM_E_TOO_LARGE, "pipelined kernel does not fit on an SM");
  int64_t grid = (int64_t)per_sm * sm_count;
  if (grid > a.n_items) grid = a.n_items;
  kern<<<(unsigned)grid, PipeOcc<R>::THREADS, smem, st>>>(a, fb);
  LFEM_CUDA(cudaGetLastError());
  return LFEM_OK;
}

// Single mesh of type (D, NA, P); fast: the rule is the compile-time one (float only).
template <int D, int NA, int P, typename R>
lfem_status launch_pipe(const PipeArgs& a, int ent_bytes, bool fast, const FastBank& fb, int sm_count,
                        cudaStream_t st) {
  using T = EType<D, NA, P>;
  if constexpr (sizeof(R) == 4 && D <= 2) {
    using TF = EType<D, NA, P, true>;
    if (fast) {
      PipeArgs af = a;
      af.one.type = TF::id;  // the tile dispatch matches the variant's id
      af.coef_smem = 0;      // coefficients are read from global memory
      return ent_bytes == 2 ? launch_pipe_types<R, uint16_t, TF>(af, fb, sm_count, st)
                            : launch_pipe_types<R, uint32_t, TF>(af, fb, sm_count, st);
    }
  }
  return ent_bytes == 2 ? launch_pipe_types<R, uint16_t, T>(a, fb, sm_count, st)
                        : launch_pipe_types<R, uint32_t, T>(a, fb, sm_count, st);
}

template <typename R>
size_t pipe_smem_bytes(const PipeArgs& a) {
  return pipe_smem_layout<R>(3, a.cap_lsm, a.cap_front, a.cap_back, a.cap_nodes, a.cap_nel, a.max_q, a.coef_smem)
      .total;
}

}  // namespace lfem
