// Persistent, pipelined assembly kernel.
//
// Each CTA walks the row tiles t = blockIdx.x, blockIdx.x + gridDim.x, ...
// For every tile it needs one contiguous metadata block (see TileHdr: element
// ids, row/incidence offsets, column positions, the tile's node list and the
// local node indices of its elements), the coordinates of the tile's nodes and
// the coefficients of its elements.  While tile t is computed, the next tile's
// block is copied by the tensor memory accelerator (one cp.async.bulk with an
// mbarrier) into the other buffer, and as soon as it lands the next tile's
// node coordinates and coefficients are gathered with cp.async into that
// buffer as well: the global-memory latency of tile t+grid hides behind the
// arithmetic of tile t.
//
// Per tile (Sec. 3.2 / 3.3 of the paper; Eqs. reference_quadrature_mass,
// reference_quadrature_stiffness, M matrix, A matrix):
//   split    node coordinates -> float pairs (mixed) once per node
//   phase 1  two threads per element (quadrature points split between them):
//            geometry and local upper-triangle matrices of every element of
//            the tile -> shared memory
//   phase 2  one writer per CSR slot: slots with one or two contributions
//            take a thread each (plain sum, coalesced stores); longer lists
//            are summed in ascending element order with a compensated pair --
//            fixed order, no atomics
//
// Every mbarrier wait is bounded by the global timer; on timeout the CTA
// records ST_TIMEOUT in the status word, waits (bounded) for its own copy and
// returns, leaving the context usable.
#pragma once

#include "assemble_fast.cuh"
#include "assemble_impl.cuh"

namespace lfem {

constexpr int kPipeTPE = 2;  // threads per element in phase 1

// Launch shape: the float kernel fits 170 registers, so 192 threads and two
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

// One mesh of a launch: its inputs, outputs, tables and tile blocks.
struct MeshRec {
  const double* coords;
  const void* coef;
  const uint8_t* meta;
  const int64_t* meta_off;
  void* out[3];
  TabRef tab;
  int type;  // element type id (elem_type_id)
  int na, ref, entb, coef_f32, pad;
};

__host__ __device__ constexpr int elem_type_id(int d, int na, int p) { return d * 100 + na * 10 + p; }
constexpr int kFastTypeOffset = 1000;

// Arguments of a persistent launch over work items (mesh, tile).  With one
// mesh and no item list, item i is tile i of mesh 0.
struct PipeArgs {
  MeshRec one;              // the mesh when meshes is NULL
  const MeshRec* meshes;    // device table of a batch, or NULL
  const int2* items;  // (mesh, tile), or NULL
  int64_t n_items;
  int nm;
  unsigned which;
  int chunk;       // elements per phase-1 round (threads / kPipeTPE)
  int cap_bytes;   // largest metadata block
  int cap_nodes;   // most nodes in a tile
  int cap_nel;     // most elements in a tile
  int max_u;       // largest local upper triangle among the meshes
  int64_t cap_lsm; // largest nel * nm * lsm_stride(U) over the meshes (local-matrix words)
  int max_q;       // most quadrature points among the meshes
  int coef_bytes;  // 4 or 8 if the weighted mass is requested, else 0
  float qmin;
  int32_t* status;
  unsigned long long* fallback;
  int starve;         // test knob: CTA 0 skips its first metadata copy
  long long wait_ns;  // bound of every mbarrier wait
};

struct PipeSmem {
  size_t mbar, rec, meta0, meta1, node0, node1, coef0, coef1, lsm, flag, total;
};

template <typename R>
__host__ __device__ inline PipeSmem pipe_smem_layout(int na, int64_t cap_lsm, int cap_bytes, int cap_nodes,
                                                     int cap_nel, int q, int coef_bytes) {
  auto al = [](size_t b) { return (b + 127) / 128 * 128; };
  PipeSmem L;
  size_t o = 0;
  L.mbar = o;
  o += 128;
  L.rec = o;  // the MeshRec of the current and of the next item
  o += al(2 * sizeof(MeshRec));
  L.meta0 = o;
  o += al(cap_bytes);
  L.meta1 = o;
  o += al(cap_bytes);
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
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

template <typename PosT, int REF>
__device__ __forceinline__ void load_pos_smem(const uint8_t* base, int k, int (&pos)[REF]) {
  constexpr int BYTES = pos_stride(REF) * (int)sizeof(PosT);
  const uint8_t* p = base + (size_t)k * BYTES;
  uint32_t w[BYTES >= 4 ? BYTES / 4 : 1];
  if constexpr (BYTES == 2) {
    w[0] = *reinterpret_cast<const unsigned short*>(p);
  } else if constexpr (BYTES == 4) {
    w[0] = *reinterpret_cast<const unsigned int*>(p);
  } else if constexpr (BYTES == 8) {
    const uint2 v = *reinterpret_cast<const uint2*>(p);
    w[0] = v.x;
    w[1] = v.y;
  } else {
#pragma unroll
    for (int h = 0; h < BYTES / 16; ++h) {
      const uint4 v = reinterpret_cast<const uint4*>(p)[h];
      w[4 * h + 0] = v.x;
      w[4 * h + 1] = v.y;
      w[4 * h + 2] = v.z;
      w[4 * h + 3] = v.w;
    }
  }
#pragma unroll
  for (int b = 0; b < REF; ++b) {
    if constexpr (sizeof(PosT) == 1) pos[b] = (w[b >> 2] >> (8 * (b & 3))) & 0xFF;
    else pos[b] = (w[b >> 1] >> (16 * (b & 1))) & 0xFFFF;
  }
}

// Store to global memory by an explicitly global address (a generic store
// could alias shared memory and would pin later shared loads behind it).
__device__ __forceinline__ void st_global(float* p, float v) { __stcg(p, v); }
__device__ __forceinline__ void st_global(double* p, double v) { __stcg(p, v); }

// Issue the gathers of a tile's node coordinates and element coefficients.
__device__ __forceinline__ void issue_gathers(const MeshRec& mr, bool want_coef, const uint8_t* meta,
                                              double* nodes_dst, void* coef_dst) {
  const TileHdr h = *reinterpret_cast<const TileHdr*>(meta);
  const TileLayout L = tile_layout(h.nel, h.ns, h.nl, h.nle, h.nnodes, mr.ref, mr.entb);
  const int32_t* nd = reinterpret_cast<const int32_t*>(meta + L.nodes);
  const int na = mr.na;
  // a thread per node (no division by the runtime sizes)
  for (int v = threadIdx.x; v < h.nnodes; v += blockDim.x) {
    const double* src = mr.coords + (int64_t)nd[v] * na;
    for (int c = 0; c < na; ++c) cp_async8(nodes_dst + v * na + c, src + c);
  }
  // compile-time-rule tiles read their coefficients straight from global memory
  if (want_coef && mr.type < kFastTypeOffset) {
    const int q = mr.tab.q;
    const int32_t* el = reinterpret_cast<const int32_t*>(meta + L.elem);
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
  cp_async_commit();
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

// Local matrices of one element by a lane pair; the even lane stores the
// first half of the entries, the odd lane the second half.
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
      if (DM) dst[im * stride_m + u] = Mo[u];
      if (DC) dst[ic * stride_m + u] = Co[u];
    }
  }
  if (store && lane_a) {
#pragma unroll
    for (int u = 0; u < U; ++u) dst[ia * stride_m + u] = Ao[u];
  }
}

template <int D, int NA, int P, typename R>
__device__ __forceinline__ void element_pair_dispatch(const ElemData<D, NA, P, R>& ed, const TabView<R>& tb,
                                                      const void* coef, int coef_f32, int sub, bool store, R* dst,
                                                      int mstride, unsigned which, R& qual, bool& bad) {
  constexpr int U = Ref<D, P>::U;
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

// Everything done for one tile whose block, node coordinates and coefficients
// are in shared memory: split, phase 1 (+ the double fallback), the prefetch
// hook of the next item after the first phase-1 round, phase 2.
template <int D, int NA, int P, bool FAST, typename R, typename EntT, typename Prefetch>
__device__ __forceinline__ void process_tile(const PipeArgs& a, const MeshRec& mr, const uint8_t* mb, double* xd,
                                             const void* coef_s, R* lsm, uint32_t* flist, int* nflag,
                                             const FastBank& fb,
                                             Prefetch&& prefetch) {
  constexpr int REF = Ref<D, P>::REF;
  constexpr int U = Ref<D, P>::U;
  constexpr int UP = lsm_stride(U);
  constexpr int ENTB = (int)sizeof(EntT);
  using Acc = typename AccOf<R>::T;
  const int nm = a.nm, Q = mr.tab.q;
  const int coef_bytes = a.coef_bytes;
  const TabView<R> tb = tab_view<D, P, R>(mr.tab);
  const TileHdr h = *reinterpret_cast<const TileHdr*>(mb);
  // local matrices matrix-major: lsm[m * nel * UP + e * UP + u] (row stride U
  // rounded up to even); a contribution entry is the word offset e * UP + u
  const int mstride = h.nel * UP;
  const TileLayout TL = tile_layout(h.nel, h.ns, h.nl, h.nle, h.nnodes, REF, ENTB);
  const int32_t* t_elem = reinterpret_cast<const int32_t*>(mb + TL.elem);
  const int32_t* t_nodes = reinterpret_cast<const int32_t*>(mb + TL.nodes);
  const uint16_t* t_en = reinterpret_cast<const uint16_t*>(mb + TL.enodes);
  const EntT* t_pair = reinterpret_cast<const EntT*>(mb + TL.pair);
  const int4* t_lrec = reinterpret_cast<const int4*>(mb + TL.lrec);
  const EntT* t_lent = reinterpret_cast<const EntT*>(mb + TL.lent);

  if (threadIdx.x == 0) *nflag = 0;  // visible after the next barrier (split, or the one after phase 1)
  // node coordinates -> (hi, lo) float pairs in place (mixed)
  if constexpr (sizeof(R) == 4) {
    for (int i = threadIdx.x; i < h.nnodes * NA; i += blockDim.x) {
      float hi, lo;
      bool ok = true;
      split_f64(xd[i], hi, lo, ok);
      if (!ok) hi = __int_as_float(0x7fc00000);  // out of float range: NaN forces the double path
      reinterpret_cast<float2*>(xd)[i] = make_float2(hi, lo);
    }
    __syncthreads();
  }

  bool prefetched = false;
  if constexpr (FAST && sizeof(R) == 4) {
    // ---- phase 1, compile-time rule: one thread per element, every element of the tile
    for (int c0 = 0; c0 < h.nel; c0 += (int)blockDim.x) {
      const int jt = c0 + (int)threadIdx.x;
      if (jt < h.nel) {
        ElemData<D, NA, P, float> ed;
        element_data_from_pairs<D, NA, P>(reinterpret_cast<const float2*>(xd), t_en + (size_t)jt * REF, ed);
        // coefficients of the element from global memory (loaded first, used last)
        const int64_t cg = (int64_t)t_elem[jt] * Q;
        const float* cs = coef_bytes == 4 ? static_cast<const float*>(mr.coef) + cg : nullptr;
        const double* cd = coef_bytes == 8 ? static_cast<const double*>(mr.coef) + cg : nullptr;
        Checks ck;
        element_fast_store2<D, NA, P>(ed, fb, cs, cd, a.qmin, a.which, reinterpret_cast<float*>(lsm) + (size_t)jt * UP,
                                      mstride, ck);
        const uint32_t fl = !ck.good ? 2u : (ck.cond ? 0u : 1u);
        if (fl) flist[atomicAdd(nflag, 1)] = (uint32_t)jt | (fl << 30);
      }
      if (!prefetched) {
        prefetch();
        prefetched = true;
      }
    }
  } else
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
    R* dst = lsm + (size_t)jt * UP;
    if constexpr (sizeof(R) == 4) {
      ElemData<D, NA, P, float> ed;
      element_data_from_pairs<D, NA, P>(reinterpret_cast<const float2*>(xd), en, ed);
      element_pair_dispatch<D, NA, P, float>(ed, tb, cf, mr.coef_f32, sub, active, dst, mstride, a.which, qual, bad);
    } else {
      double X[REF][NA];
#pragma unroll
      for (int bb = 0; bb < REF; ++bb)
#pragma unroll
        for (int i = 0; i < NA; ++i) X[bb][i] = xd[en[bb] * NA + i];
      ElemData<D, NA, P, double> ed;
      load_element_data<D, NA, P, double>(X, ed);
      element_pair_dispatch<D, NA, P, double>(ed, tb, cf, mr.coef_f32, sub, active, dst, mstride, a.which, qual, bad);
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
    if (!prefetched) {
      prefetch();
      prefetched = true;
    }
  }
  if constexpr (sizeof(R) == 4) {
    __syncthreads();
    // rare path: double recomputation of flagged elements from global
    // coordinates -- every requested matrix for an element that failed the
    // finiteness test (2), the stiffness alone for one that failed only the
    // conditioning test (1): mass-type matrices need s, not G^{-1}
    // (a compacted list, so that whole warps work on it: the FP64 pipe costs
    // the same for a warp instruction with few active lanes)
    const int ia = (a.which & LFEM_MASS) ? 1 : 0;
    const int nf = *nflag;
    for (int i = threadIdx.x; i < nf; i += blockDim.x) {
      const uint32_t v = flist[i];
      const int j = (int)(v & 0x3FFFFFFFu), fl = (int)(v >> 30);
      const unsigned fw = fl == 2 ? a.which : (a.which & LFEM_STIFF);
      if (!fw) continue;
      const uint16_t* en = t_en + (size_t)j * REF;
      int32_t nd[REF];
#pragma unroll
      for (int bb = 0; bb < REF; ++bb) nd[bb] = t_nodes[en[bb]];
      bool bad = false;
      R* d = lsm + (size_t)j * UP + (fl == 2 ? 0 : ia * mstride);
      element_fp64_lean<D, NA, P, float>(mr.coords, nd, mr.tab, mr.coef, mr.coef_f32, (int64_t)t_elem[j], fw, d,
                                         mstride, bad);
      if (nd[0] >= h.r0 && nd[0] < h.r0 + h.nrows) {
        atomicAdd(a.fallback, 1ull);
        if (bad) atomicOr(a.status, ST_DEGENERATE);
      }
    }
  }
  if (!prefetched) prefetch();
  __syncthreads();

  // ---- phase 2: one writer per CSR slot, each slot's contributions summed
  // in ascending (element, a, b) order -- fixed order, no atomics.  Slots with
  // one or two contributions (nearly all of them on surfaces) take a thread
  // each, consecutive slots on consecutive threads (coalesced stores, no
  // loop); the few longer lists (the diagonal of a node of high valence) are
  // summed with a compensated pair from the long list.
  {
    constexpr EntT NONE = (EntT)~(EntT)0;
    R* o0 = reinterpret_cast<R*>(mr.out[0]) + h.s0;
    R* o1 = nm > 1 ? reinterpret_cast<R*>(mr.out[1]) + h.s0 : o0;
    R* o2 = nm > 2 ? reinterpret_cast<R*>(mr.out[2]) + h.s0 : o0;
    const R* l1 = lsm + mstride;
    const R* l2 = lsm + 2 * mstride;
#pragma unroll 2
    for (int s = threadIdx.x; s < h.ns; s += blockDim.x) {
      const EntT x = t_pair[2 * s], y = t_pair[2 * s + 1];
      if (x == NONE) continue;
      R v0 = lsm[x], v1 = nm > 1 ? l1[x] : (R)0, v2 = nm > 2 ? l2[x] : (R)0;
      if (y != NONE) {
        v0 += lsm[y];
        if (nm > 1) v1 += l1[y];
        if (nm > 2) v2 += l2[y];
      }
      st_global(o0 + s, v0);
      if (nm > 1) st_global(o1 + s, v1);
      if (nm > 2) st_global(o2 + s, v2);
    }
    for (int j = threadIdx.x; j < h.nl; j += blockDim.x) {
      const int4 r = t_lrec[j];
      uint32_t ent = t_lent[r.y];
      Acc c0, c1, c2;
      acc_init(c0, lsm[ent]);
      if (nm > 1) acc_init(c1, l1[ent]);
      if (nm > 2) acc_init(c2, l2[ent]);
      for (int k = r.y + 1; k < r.z; ++k) {
        ent = t_lent[k];
        acc_add(c0, lsm[ent]);
        if (nm > 1) acc_add(c1, l1[ent]);
        if (nm > 2) acc_add(c2, l2[ent]);
      }
      st_global(o0 + r.x, (R)acc_final(c0));
      if (nm > 1) st_global(o1 + r.x, (R)acc_final(c1));
      if (nm > 2) st_global(o2 + r.x, (R)acc_final(c2));
    }
  }
}

// Element type of a launch; the compile-time-rule variant has its own id, so a
// batch can hold meshes of one type with and without the usual rule.
template <int D_, int NA_, int P_, bool FAST_ = false>
struct EType {
  static constexpr int D = D_, NA = NA_, P = P_;
  static constexpr bool FAST = FAST_;
  static constexpr int id = elem_type_id(D_, NA_, P_) + (FAST_ ? kFastTypeOffset : 0);
};

template <typename R, typename EntT, typename T0, typename... Ts, typename Prefetch>
__device__ __forceinline__ void dispatch_tile(int type, const PipeArgs& a, const MeshRec& mr, const uint8_t* mb,
                                              double* xd, const void* coef_s, R* lsm, uint32_t* flist, int* nflag,
                                              const FastBank& fb, Prefetch&& prefetch) {
  if (type == T0::id) {
    process_tile<T0::D, T0::NA, T0::P, T0::FAST, R, EntT>(a, mr, mb, xd, coef_s, lsm, flist, nflag, fb, prefetch);
  } else {
    if constexpr (sizeof...(Ts) > 0) {
      dispatch_tile<R, EntT, Ts...>(type, a, mr, mb, xd, coef_s, lsm, flist, nflag, fb, prefetch);
    } else {
      // no variant for this tile's type: report it, keep the pipeline's steps
      if (threadIdx.x == 0) atomicOr(a.status, ST_TYPE);
      prefetch();
      __syncthreads();
    }
  }
}

// Persistent launch over work items; Types lists the element types the launch
// may meet (one for a single mesh, several for a batch).
template <typename R, typename EntT, typename... Types>
__global__ void __launch_bounds__(PipeOcc<R>::THREADS, PipeOcc<R>::MIN_BLOCKS) k_assemble_pipe(const PipeArgs a, const __grid_constant__ FastBank fb) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const bool want_coef = a.coef_bytes != 0;
  const PipeSmem L =
      pipe_smem_layout<R>(3, a.cap_lsm, a.cap_bytes, a.cap_nodes, a.cap_nel, a.max_q, a.coef_bytes);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem_raw + L.mbar);
  int* s_flag = reinterpret_cast<int*>(smem_raw + L.mbar + 64);
  // buffers as shared-memory base + offset (no pointer arrays: a pointer
  // loaded back from local memory would turn every access generic)
  MeshRec* s_rec = reinterpret_cast<MeshRec*>(smem_raw + L.rec);
  auto meta_of = [&](int buf) { return smem_raw + (buf ? L.meta1 : L.meta0); };
  auto node_of = [&](int buf) { return reinterpret_cast<double*>(smem_raw + (buf ? L.node1 : L.node0)); };
  auto coef_of = [&](int buf) { return static_cast<void*>(smem_raw + (buf ? L.coef1 : L.coef0)); };
  R* lsm = reinterpret_cast<R*>(smem_raw + L.lsm);
  uint32_t* flist = reinterpret_cast<uint32_t*>(smem_raw + L.flag);
  int* s_nflag = reinterpret_cast<int*>(smem_raw + L.mbar + 68);

  int64_t i = blockIdx.x;
  if (i >= a.n_items) return;
  if (threadIdx.x == 0) {
    mbar_init(&mbar[0], 1);
    mbar_init(&mbar[1], 1);
    fence_mbar_init();
    *s_flag = 0;
  }
  __syncthreads();

  auto item = [&](int64_t k, int& mesh, int64_t& tile) {
    if (a.items) {
      const int2 v = a.items[k];
      mesh = v.x;
      tile = v.y;
    } else {
      mesh = 0;
      tile = k;
    }
  };
  // thread 0: item k's MeshRec into s_rec[buf] (read by all after the next
  // barrier) and one bulk copy of its metadata block
  auto load_block = [&](int64_t k, int buf) {
    int mesh;
    int64_t tile;
    item(k, mesh, tile);
    MeshRec& r = s_rec[buf];
    if (a.meshes) r = a.meshes[mesh];
    else r = a.one;
    const uint32_t bytes = (uint32_t)(r.meta_off[tile + 1] - r.meta_off[tile]);
    tma_load_block(meta_of(buf), r.meta + r.meta_off[tile], bytes, &mbar[buf]);
  };
  // prologue: item i into buffer 0
  const bool issued0 = !(a.starve && blockIdx.x == 0);
  if (threadIdx.x == 0 && issued0) load_block(i, 0);
  {
    const bool ok = mbar_wait_bounded(&mbar[0], 0, a.wait_ns);
    if (__syncthreads_or(!ok)) {
      // the copy (if one was issued) did not land within the bound: report, and
      // give it one more bounded wait so that it does not write into the shared
      // memory of a CTA that starts here after this one returns
      if (threadIdx.x == 0) {
        atomicOr(a.status, ST_TIMEOUT);
        if (issued0) mbar_wait_bounded(&mbar[0], 0, a.wait_ns);
      }
      return;
    }
  }
  issue_gathers(s_rec[0], want_coef, meta_of(0), node_of(0), coef_of(0));

  for (int it = 0; i < a.n_items; i += gridDim.x, ++it) {
    const int b = it & 1, nb = b ^ 1;
    const int64_t in = i + gridDim.x;
    // next item's metadata block: one bulk copy into the other buffer
    if (in < a.n_items && threadIdx.x == 0) {
      fence_proxy_async();
      load_block(in, nb);
    }
    cp_async_wait_all();
    __syncthreads();

    auto prefetch_next = [&]() {
      // all threads: wait for the next block (bounded), then gather its nodes and coefficients
      if (in < a.n_items) {
        const bool ok = mbar_wait_bounded(&mbar[nb], (uint32_t)(((it + 1) >> 1) & 1), a.wait_ns);
        if (__syncthreads_or(!ok)) {
          if (threadIdx.x == 0) *s_flag = 1;
        } else {
          issue_gathers(s_rec[nb], want_coef, meta_of(nb), node_of(nb), coef_of(nb));
        }
      }
    };
    const MeshRec& mr = s_rec[b];
    dispatch_tile<R, EntT, Types...>(mr.type, a, mr, meta_of(b), node_of(b), coef_of(b), lsm, flist, s_nflag, fb,
                                     prefetch_next);
    if (*s_flag) {
      // the next block never arrived: report, wait (bounded) for the copy, stop
      if (threadIdx.x == 0) atomicOr(a.status, ST_TIMEOUT);
      if (in < a.n_items) mbar_wait_bounded(&mbar[nb], (uint32_t)(((it + 1) >> 1) & 1), a.wait_ns);
      cp_async_wait_all();
      return;
    }
    __syncthreads();
  }
  cp_async_wait_all();
}

template <typename R, typename EntT, typename... Types>
lfem_status launch_pipe_types(const PipeArgs& a, const FastBank& fb, int sm_count, cudaStream_t st) {
  if (a.n_items == 0) return LFEM_OK;
  const size_t smem =
      pipe_smem_layout<R>(3, a.cap_lsm, a.cap_bytes, a.cap_nodes, a.cap_nel, a.max_q, a.coef_bytes).total;
  if (smem > 227 * 1024) return fail(LFEM_E_TOO_LARGE, "pipelined tile needs more than 227 KB of shared memory");
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

// Single mesh of type (D, NA, P).
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
      return ent_bytes == 2 ? launch_pipe_types<R, uint16_t, TF>(af, fb, sm_count, st)
                            : launch_pipe_types<R, uint32_t, TF>(af, fb, sm_count, st);
    }
  }
  return ent_bytes == 2 ? launch_pipe_types<R, uint16_t, T>(a, fb, sm_count, st)
                        : launch_pipe_types<R, uint32_t, T>(a, fb, sm_count, st);
}

template <typename R>
size_t pipe_smem_bytes(const PipeArgs& a) {
  return pipe_smem_layout<R>(3, a.cap_lsm, a.cap_bytes, a.cap_nodes, a.cap_nel, a.max_q, a.coef_bytes).total;
}

}  // namespace lfem
