// Internal declarations of the lfem CUDA library (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "lfem.h"

namespace lfem {

// ----------------------------------------------------------------------------
// Host-side error plumbing
// ----------------------------------------------------------------------------
void set_error(const std::string& msg);
lfem_status fail(lfem_status s, const std::string& msg);
lfem_status cuda_fail(cudaError_t e, const char* what);

// Every device allocation of the library goes through dev_malloc, which counts
// the successful ones (lfem_debug_alloc_count).
cudaError_t dev_malloc(void** p, size_t bytes);

#define LFEM_CUDA(call)                                   \
  do {                                                    \
    cudaError_t _e = (call);                              \
    if (_e != cudaSuccess) return ::lfem::cuda_fail(_e, #call); \
  } while (0)

// Device status bits (pattern status word).
enum : int32_t { ST_DEGENERATE = 1, ST_INDEX = 2, ST_TIMEOUT = 4, ST_TYPE = 8, ST_ITEM = 16 };

// Tile limits.
constexpr int kMaxTileIncidences = 4096;  // incidences (e, a) per tile; local index fits 12 bits
constexpr int kMaxDegree = 2048;          // elements meeting at one node
constexpr int kMaxSegSort = 16384;        // longest row of raw column entries sorted in one block
constexpr int kMaxTileRows = 4096;        // rows per tile (row offsets are 16-bit)
constexpr int kMaxTileEntries = 16384;    // incidences x ref per tile (node-list sort in one block)

// ----------------------------------------------------------------------------
// Element types
// ----------------------------------------------------------------------------
// C(p + d, d) local nodes: P1, P2 on every simplex; orders 3 and 4 on curves and triangles.
__host__ __device__ constexpr int n_ref(int d, int p) {
  return p == 1 ? d + 1
                : (p == 2 ? (d + 1) * (d + 2) / 2
                          : (d == 1 ? p + 1 : (d == 2 ? (p + 1) * (p + 2) / 2 : (p + 1) * (p + 2) * (p + 3) / 6)));
}
__host__ __device__ constexpr int n_upper(int ref) { return ref * (ref + 1) / 2; }
__host__ __device__ constexpr int n_edges(int d, int p) { return p == 2 ? n_ref(d, 2) - (d + 1) : 0; }

bool supported(int dim, int ambient, int order);
// The degree-2 rule that makes order-1 M and A exact (used when no rule is given).
const lfem_quad* exact_p1_rule(int dim);

// Reference tables (Lagrange basis, Sec. 3.1; quadrature rule, Sec. 3.2.2) in
// constant memory.  One 64 KB bank per device, append-only registry keyed by
// (dim, order, rule).  Layout of one entry (precision T = float or double):
//   w[Q], phi[Q][REF], dphi[Q][REF][D], dpsi[Q][NE][D]
// dpsi are the gradients of the edge bubbles 4 l_i l_j, used to build the
// Jacobian in hierarchical form (corner edge vectors + edge-node deviations).
struct TabRef {
  int q = 0;
  int off32 = 0;  // offset in floats into the bank
  int off64 = 0;  // offset in doubles into the bank
};
lfem_status get_tables(int dim, int order, const lfem_quad* quad, cudaStream_t st, TabRef* out);

// One bank per translation unit (no relocatable device code); every unit's
// copy receives the same uploads (see bank_upload_d*).
static __constant__ double c_bank[8192];

template <typename T>
__device__ __forceinline__ const T* bank();
template <>
__device__ __forceinline__ const float* bank<float>() {
  return reinterpret_cast<const float*>(c_bank);
}
template <>
__device__ __forceinline__ const double* bank<double>() {
  return c_bank;
}

template <int D, int P>
struct Ref {
  static constexpr int REF = n_ref(D, P);
  static constexpr int U = n_upper(REF);
  static constexpr int NE = n_edges(D, P);
};

// Edge k of the P2 element joins corners (edge_i(k), edge_j(k)).
template <int D>
__host__ __device__ constexpr int edge_i(int k) {
  return D == 1 ? 0 : (D == 2 ? (k == 2 ? 2 : k) : (k < 3 ? (k == 2 ? 2 : k) : k - 3));
}
template <int D>
__host__ __device__ constexpr int edge_j(int k) {
  return D == 1 ? 1 : (D == 2 ? (k == 2 ? 0 : k + 1) : (k < 3 ? (k == 2 ? 0 : k + 1) : 3));
}

// Column positions of one incidence are stored padded to a power of two so a
// single vector load fetches them (ref 2 -> 2, 3/4 -> 4, 6 -> 8, 10 -> 16).
__host__ __device__ constexpr int pos_stride(int ref) {
  return ref <= 2 ? 2 : (ref <= 4 ? 4 : (ref <= 8 ? 8 : (ref + 15) / 16 * 16));
}

template <typename PosT, int REF>
__device__ __forceinline__ void load_pos(const uint8_t* __restrict__ base, int64_t k, int (&pos)[REF]) {
  constexpr int BYTES = pos_stride(REF) * (int)sizeof(PosT);
  const uint8_t* p = base + k * BYTES;
  uint32_t w[BYTES >= 4 ? BYTES / 4 : 1];
  if constexpr (BYTES == 2) {
    w[0] = __ldg(reinterpret_cast<const unsigned short*>(p));
  } else if constexpr (BYTES == 4) {
    w[0] = __ldg(reinterpret_cast<const unsigned int*>(p));
  } else if constexpr (BYTES == 8) {
    const uint2 v = __ldg(reinterpret_cast<const uint2*>(p));
    w[0] = v.x;
    w[1] = v.y;
  } else {
#pragma unroll
    for (int h = 0; h < BYTES / 16; ++h) {
      const uint4 v = __ldg(reinterpret_cast<const uint4*>(p) + h);
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

// Upper-triangle index of local pair (a, b), a <= b.
__host__ __device__ constexpr int upper_index(int ref, int a, int b) {
  return a * ref - a * (a - 1) / 2 + (b - a);
}
__host__ __device__ constexpr int sym_index(int ref, int a, int b) {
  return a <= b ? upper_index(ref, a, b) : upper_index(ref, b, a);
}

template <typename T>
struct TabView {
  const T* w;
  const T* phi;
  const T* dphi;
  const T* dpsi;
  int q;
};

template <int D, int P, typename T>
__device__ __forceinline__ TabView<T> tab_view(const TabRef& t) {
  constexpr int REF = Ref<D, P>::REF, NE = Ref<D, P>::NE;
  const T* base = bank<T>() + (sizeof(T) == 4 ? t.off32 : t.off64);
  TabView<T> v;
  v.q = t.q;
  v.w = base;
  v.phi = v.w + t.q;
  v.dphi = v.phi + t.q * REF;
  v.dpsi = v.dphi + t.q * REF * D;
  (void)NE;
  return v;
}

// ----------------------------------------------------------------------------
// Per-element geometry and local matrices (Sec. 3.2), compute precision R.
//
//   J   = [x_1 - x_0, ..., x_D - x_0] + sum_k delta_k (grad psi_k)^T
//         (delta_k = x_{edge k} - (x_i + x_j)/2; equal to sum_a x_a grad phi_a^T
//          for the Lagrange P2 map, Eq. F_map, with the affine part exact)
//   s   = |det DF|: |det J| (D = n), |t1 x t2| (D=2, n=3), |t| (D=1)
//   H   = w s G^{-1} = (w / s) adj(G),  G = J^T J
//   M_ab  += w s phi_a phi_b,  MC_ab += w s c phi_a phi_b,
//   A_ab  += grad^phi_a . (H grad^phi_b)
// ----------------------------------------------------------------------------
template <int D, int NA, int P>
struct ElemGeom {
  static constexpr int REF = Ref<D, P>::REF;
  static constexpr int NE = Ref<D, P>::NE;
};

template <int D, int NA, int P, typename R>
struct ElemData {
  static constexpr int REF = Ref<D, P>::REF;
  static constexpr int NE = Ref<D, P>::NE;
  R e[D][NA];                      // corner edge vectors x_{m+1} - x_0
  R dl[NE > 0 ? NE : 1][NA];       // edge-node deviations
  R rel[P >= 3 ? REF : 1][NA];     // orders 3, 4: every node relative to node 0
};

template <int D, int NA, int P, typename R>
__device__ __forceinline__ void load_element_data(const double (&X)[Ref<D, P>::REF][NA], ElemData<D, NA, P, R>& ed) {
#pragma unroll
  for (int m = 0; m < D; ++m)
#pragma unroll
    for (int i = 0; i < NA; ++i) ed.e[m][i] = (R)(X[m + 1][i] - X[0][i]);
  if constexpr (P >= 3) {
#pragma unroll
    for (int a = 1; a < Ref<D, P>::REF; ++a)
#pragma unroll
      for (int i = 0; i < NA; ++i) ed.rel[a][i] = (R)(X[a][i] - X[0][i]);
  }
#pragma unroll
  for (int k = 0; k < Ref<D, P>::NE; ++k)
#pragma unroll
    for (int i = 0; i < NA; ++i)
      ed.dl[k][i] = (R)(X[D + 1 + k][i] - 0.5 * (X[edge_i<D>(k)][i] + X[edge_j<D>(k)][i]));
}

// Geometry at quadrature point q: J (NA x D), s, H (D x D sym, stored full), metric quality.
template <int D, int NA, int P, typename R>
struct QpGeom {
  R J[NA][D];
  R s;
  R H[D][D];      // w s G^{-1}
  R quality;      // det G / (tr G / D)^D in (0, 1]; 1 for D = 1
};

// s = sqrt(s2) and 1/s.  Float: one hardware reciprocal square root (about
// 1 ulp), no division sequence; double: IEEE square root and division.
__device__ __forceinline__ void norm_inv(float s2, float& s, float& inv) {
  inv = rsqrtf(s2);
  s = s2 * inv;
}
__device__ __forceinline__ void norm_inv(double s2, double& s, double& inv) {
  s = sqrt(s2);
  inv = 1.0 / s;
}
// 1/x: float hardware reciprocal (about 1 ulp); double IEEE.
__device__ __forceinline__ float rcp_(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double rcp_(double x) { return 1.0 / x; }

template <int D, int NA, int P, typename R>
__device__ __forceinline__ void qp_geometry(const ElemData<D, NA, P, R>& ed, const TabView<R>& tb, int q, R wq,
                                            QpGeom<D, NA, P, R>& g) {
  constexpr int NE = Ref<D, P>::NE;
  if constexpr (P >= 3) {
    // orders 3, 4: J = sum_a (x_a - x_0) grad^phi_a^T (Eq. F_map differentiated)
    constexpr int REF = Ref<D, P>::REF;
#pragma unroll
    for (int i = 0; i < NA; ++i)
#pragma unroll
      for (int m = 0; m < D; ++m) {
        R acc = 0;
#pragma unroll
        for (int a = 1; a < REF; ++a) acc = fma(ed.rel[a][i], tb.dphi[(q * REF + a) * D + m], acc);
        g.J[i][m] = acc;
      }
  } else {
#pragma unroll
    for (int i = 0; i < NA; ++i)
#pragma unroll
      for (int m = 0; m < D; ++m) {
        R acc = ed.e[m][i];
#pragma unroll
        for (int k = 0; k < NE; ++k) acc = fma(ed.dl[k][i], tb.dpsi[(q * NE + k) * D + m], acc);
        g.J[i][m] = acc;
      }
  }
  if constexpr (D == 1) {
    R tt = 0;
#pragma unroll
    for (int i = 0; i < NA; ++i) tt = fma(g.J[i][0], g.J[i][0], tt);
    R s, inv;
    norm_inv(tt, s, inv);
    g.s = s;
    g.H[0][0] = wq * inv;
    g.quality = (R)1;
  } else if constexpr (D == 2) {
    R g11 = 0, g12 = 0, g22 = 0;
#pragma unroll
    for (int i = 0; i < NA; ++i) {
      g11 = fma(g.J[i][0], g.J[i][0], g11);
      g12 = fma(g.J[i][0], g.J[i][1], g12);
      g22 = fma(g.J[i][1], g.J[i][1], g22);
    }
    R s, inv;
    if constexpr (NA == 2) {
      s = fabs(g.J[0][0] * g.J[1][1] - g.J[0][1] * g.J[1][0]);
      inv = rcp_(s);
    } else {
      R n0 = g.J[1][0] * g.J[2][1] - g.J[2][0] * g.J[1][1];
      R n1 = g.J[2][0] * g.J[0][1] - g.J[0][0] * g.J[2][1];
      R n2 = g.J[0][0] * g.J[1][1] - g.J[1][0] * g.J[0][1];
      norm_inv(n0 * n0 + n1 * n1 + n2 * n2, s, inv);
    }
    g.s = s;
    R ws_inv = wq * inv;
    g.H[0][0] = ws_inv * g22;
    g.H[1][1] = ws_inv * g11;
    g.H[0][1] = g.H[1][0] = -ws_inv * g12;
    R tr = (R)0.5 * (g11 + g22);
    g.quality = (s * s) * rcp_(tr * tr);
  } else {
    // D = NA = 3: cofactor vectors c_m = t_{m+1} x t_{m+2}; adj(G)_mk = c_m . c_k
    R c[3][3];
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      const int m1 = (m + 1) % 3, m2 = (m + 2) % 3;
      c[m][0] = g.J[1][m1] * g.J[2][m2] - g.J[2][m1] * g.J[1][m2];
      c[m][1] = g.J[2][m1] * g.J[0][m2] - g.J[0][m1] * g.J[2][m2];
      c[m][2] = g.J[0][m1] * g.J[1][m2] - g.J[1][m1] * g.J[0][m2];
    }
    R det = g.J[0][0] * c[0][0] + g.J[1][0] * c[0][1] + g.J[2][0] * c[0][2];
    R s = fabs(det);
    g.s = s;
    R ws_inv = wq * rcp_(s);
#pragma unroll
    for (int m = 0; m < 3; ++m)
#pragma unroll
      for (int k = m; k < 3; ++k) {
        R dot = c[m][0] * c[k][0] + c[m][1] * c[k][1] + c[m][2] * c[k][2];
        g.H[m][k] = g.H[k][m] = ws_inv * dot;
      }
    R tr = 0;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int m = 0; m < 3; ++m) tr = fma(g.J[i][m], g.J[i][m], tr);
    tr *= (R)(1.0 / 3.0);
    g.quality = (s * s) * rcp_(tr * tr * tr);
  }
}

// Accumulate one quadrature point's contributions into the local upper-triangle
// accumulators (compile-time selection of which matrices this pass computes).
template <int D, int NA, int P, typename R, bool DO_M, bool DO_A, bool DO_C>
__device__ __forceinline__ void qp_accumulate(const QpGeom<D, NA, P, R>& g, const TabView<R>& tb, int q, R wq, R cq,
                                              R (&Mo)[Ref<D, P>::U], R (&Ao)[Ref<D, P>::U],
                                              R (&Co)[Ref<D, P>::U]) {
  constexpr int REF = Ref<D, P>::REF;
  const R* ph = tb.phi + q * REF;
  const R* dph = tb.dphi + q * REF * D;
  const R ws = wq * g.s;
  if constexpr (DO_M || DO_C) {
#pragma unroll
    for (int a = 0; a < REF; ++a) {
      R wpa = ws * ph[a];
      R wca = wpa * cq;
#pragma unroll
      for (int b = a; b < REF; ++b) {
        const int u = upper_index(REF, a, b);
        if constexpr (DO_M) Mo[u] = fma(wpa, ph[b], Mo[u]);
        if constexpr (DO_C) Co[u] = fma(wca, ph[b], Co[u]);
      }
    }
  }
  if constexpr (DO_A) {
#pragma unroll
    for (int b = 0; b < REF; ++b) {
      R y[D];
#pragma unroll
      for (int m = 0; m < D; ++m) {
        R acc = 0;
#pragma unroll
        for (int k = 0; k < D; ++k) acc = fma(g.H[m][k], dph[b * D + k], acc);
        y[m] = acc;
      }
#pragma unroll
      for (int a = 0; a <= b; ++a) {
        const int u = upper_index(REF, a, b);
        R acc = Ao[u];
#pragma unroll
        for (int m = 0; m < D; ++m) acc = fma(dph[a * D + m], y[m], acc);
        Ao[u] = acc;
      }
    }
  }
}

// Load the REF x NA coordinates of element e (FP64, read-only path).
template <int D, int NA, int P>
__device__ __forceinline__ void gather_coords(const double* __restrict__ coords, const int32_t* __restrict__ cn,
                                              double (&X)[Ref<D, P>::REF][NA]) {
#pragma unroll
  for (int a = 0; a < Ref<D, P>::REF; ++a) {
    const double* p = coords + (int64_t)cn[a] * NA;
#pragma unroll
    for (int i = 0; i < NA; ++i) X[a][i] = __ldg(p + i);
  }
}

// ----------------------------------------------------------------------------
// Per-tile metadata block (built once per topology).  Two contiguous parts,
// each staged by one TMA bulk copy:
//   front (needed from the start of a tile: triple-buffered)
//     header   TileHdr (48 B)
//     elem     int32  [nel]          element ids, ascending
//     nodes    int32  [nnodes]       global node id of every position of the tile's
//                                    node buffer (runs, then extras)
//     enodes   uint16 [nel][ref]     node-buffer position of each element node
//     runs     int4   [nruns]        {first node, count, position, 0}: the node buffer
//                                    is these runs of consecutive node ids (first node,
//                                    count and position even, so that each run is one
//                                    16-byte aligned bulk copy of the coordinates), the
//                                    tile's nodes plus gaps of at most kRunGap nodes
//     extras   int2   [nextra]       {node, position}: nodes copied one by one (the
//                                    mesh's last node when an even run would pass it)
//   back (needed by phase 2 only: single-buffered)
//     pair     EntT   [npad][2]      the two contribution entries of every slot, in
//                                    padded slot order p = slot + apad (apad = s0 mod 4,
//                                    so that slot groups of four are 16-byte aligned in
//                                    the output); npad = apad + ns rounded up to 4
//     lrec     int4   [nl]           slots with more than two contributions:
//                                    {slot, first, end, long index li}
//     lent     EntT   [nle]          their entries, each run in ascending (e, a, b)
// every section starts on a 16-byte boundary; each part's size is a multiple of 16.
//
// Entries address the tile's local matrices in shared memory, laid out with
// the three matrix slots of an entry pair side by side:
//   word(e, u, m) = 6 (e UP/2 + u/2) + 2 m + (u mod 2)      (UP = U rounded up to even)
// so one address serves M, A and MC (offsets 0, 2, 4 words).  After the nel
// elements (3 nel UP words) come the long-list results, 6 words per long slot
// (word LB + 6 li + 2 m, LB = 3 nel UP), then six zero words: ZERO = LB + 6 nl.
// A slot with one contribution has ZERO as its second entry; a long slot has
// its result as the first and ZERO as the second.
// ----------------------------------------------------------------------------
struct TileHdr {
  int64_t s0;
  int32_t r0, nrows, ns, nruns, nel, nnodes;  // nnodes: positions of the node buffer
  int32_t nl, nle;  // slots with more than two contributions, and their entries
  int32_t apad;     // s0 mod 4: padded slot p = slot + apad
  int32_t nextra;
  int32_t pad[4];
};
static_assert(sizeof(TileHdr) == 64, "tile header");
constexpr int kRunGap = 2;  // node-id gaps up to this length are copied inside a run

__host__ __device__ constexpr int al16(int64_t b) { return (int)((b + 15) / 16 * 16); }

// Local-matrix row stride of an element: U rounded up to even, so that entry
// pairs are 8-byte aligned (64-bit stores).
__host__ __device__ constexpr int lsm_stride(int u) { return u + (u & 1); }
constexpr int kLsmSlots = 3;  // matrix slots per local entry in shared memory
__host__ __device__ constexpr int lsm_word(int u, int m) { return 6 * (u >> 1) + 2 * m + (u & 1); }

struct TileLayout {
  int elem, nodes, enodes, runs, extras, front;  // front part: offsets from its start; front = its size
  int pair, lrec, lent, back;                    // back part: offsets from its start; back = its size
  int npad;
};
__host__ __device__ inline TileLayout tile_layout(int nel, int ns, int nl, int nle, int nnodes, int ref, int entb,
                                                  int apad, int nruns, int nextra) {
  TileLayout L;
  int o = (int)sizeof(TileHdr);
  L.elem = o;
  o += al16(4ll * nel);
  L.nodes = o;
  o += al16(4ll * nnodes);
  L.enodes = o;
  o += al16(2ll * ref * nel);
  L.runs = o;
  o += 16 * nruns;
  L.extras = o;
  o += al16(8ll * nextra);
  L.front = o;
  L.npad = (apad + ns + 3) / 4 * 4;
  if (L.npad < 4) L.npad = 4;
  o = 0;
  L.pair = o;
  o += al16(2ll * entb * L.npad);
  L.lrec = o;
  o += 16 * nl;
  L.lent = o;
  o += al16((int64_t)entb * nle);
  L.back = o;
  return L;
}
__host__ __device__ inline TileLayout tile_layout(const TileHdr& h, int ref, int entb) {
  return tile_layout(h.nel, h.ns, h.nl, h.nle, h.nnodes, ref, entb, h.apad, h.nruns, h.nextra);
}

// One work item of a persistent launch: the tile block of a mesh.
struct ItemRef {
  const uint8_t* front;  // device address of the block (front part, then back part)
  int32_t front_bytes, back_bytes;
  int32_t mesh, tile;
  int32_t pad[2];
};
static_assert(sizeof(ItemRef) == 32, "item record");

// ----------------------------------------------------------------------------
// Pattern handle
// ----------------------------------------------------------------------------
// Vector assembly (load vector, mean-curvature-flow non-linear vectors).
struct VecArgs {
  const int32_t* conn;
  const double* coords;
  const double* u;  // nodal [N][nc]: f (nc = 1) or (nu, H) (nc = 4)
  double* loc;      // [nE][ref][nc]
  const int32_t* inc_ptr;
  const int32_t* inc_key;
  double* out;      // [nc][N]
  int64_t n_elem;
  int32_t n_nodes;
  int key_shift;    // incidence key (e << key_shift) | a
  TabRef tab;
};

// Blocks of every reducing kernel of the flow step's solver (fixed, so every
// dot product is the same sum on every run); its partials take
// 4 x kMcfBlocks x 3 doubles of scratch.
constexpr int kMcfBlocks = 608;

// The solver's 8-iteration block as an instantiated CUDA graph, and the
// scratch layout it was captured for.
struct McfGraph {
  cudaGraphExec_t exec = nullptr;
  const void* buf = nullptr;
  const void* K = nullptr;
  int32_t n = 0;
  int nc = 0;
};

// Device scalars of the solve, per column.
struct McfScalars {
  double rz[3], pq[3], rz_new[3], rr[3], bb[3];
};

// One mean-curvature-flow step (mcf.cu): the pattern's CSR arrays, the
// assembled M and A, and the solver's work vectors ([n][nc], nc = ambient).
struct McfSolveArgs {
  const int64_t* row_ptr;
  const int32_t* col_idx;
  const double* M;
  const double* A;
  double tau;
  int32_t n;
  double* K;
  double* dinv;
  const double* X0;
  double* X;
  double* B;
  double* Q;
  double* R;
  double* Z;
  double* P;
  double* part;  // [4][kMcfBlocks][nc]: <p, q>, <r, r> / <b, b>, two sets of <r, z>
  McfScalars* scalars;
  McfGraph* graph;
  double* X_out;
  double rtol;
  int max_iter;
};

struct PatternDev {
  int32_t* conn = nullptr;       // [nE][ref] device copy
  int64_t* row_ptr = nullptr;    // [N+1]
  int32_t* col_idx = nullptr;    // [nnz]
  int32_t* inc_ptr = nullptr;    // [N+1] node-incidence offsets
  int32_t* inc_key = nullptr;    // [nInc] (e << key_shift) | a, ascending per node
  uint8_t* inc_pos = nullptr;    // [nInc][ref] column position of conn[e][b] in row conn[e][a] (u8 or u16)
  int32_t* elem_inc = nullptr;   // [nE][ref] incidence index of (e, a)
  int32_t* tile_row0 = nullptr;  // [T+1]
  int32_t* tile_elem_ptr = nullptr;  // [T+1]
  int32_t* tile_elem = nullptr;  // [sum] ascending element ids per tile
  uint16_t* inc_local = nullptr; // [nInc] (index of e in its tile's list) << 4 | a
  int32_t* status = nullptr;     // [4]: status bits, pad, fallback count (int64 at [2])
  int32_t* slot_off = nullptr;   // [nnz+1] element-major path: start of each slot's contributions
  int32_t* slot_ent = nullptr;   // [nInc*ref] e * U + u, per slot in ascending (e, a, b)
  void* elem_buf = nullptr;      // element-major path: local matrices [nE][nm][U] (scratch)
  size_t elem_buf_bytes = 0;
  double* vec_buf = nullptr;     // vector assembly: local vectors [nE][ref][nc] (scratch)
  size_t vec_buf_bytes = 0;
  void* mcf_buf = nullptr;       // mean-curvature-flow step: matrices and solver vectors (scratch)
  size_t mcf_buf_bytes = 0;
  McfGraph mcf_graph;            // its captured solver iterations
  uint8_t* tile_meta = nullptr;  // per-tile metadata blocks (see TileHdr)
  int64_t* tile_meta_off = nullptr;  // [T+1] byte offsets, multiples of 16
  ItemRef* tile_refs = nullptr;  // [T] block address and part sizes per tile
};

}  // namespace lfem

struct lfem_pattern_s {
  int device = 0;
  int dim = 0, order = 0, ref = 0;
  int64_t n_elem = 0;
  int32_t n_nodes = 0;
  int64_t nnz = 0;
  int64_t n_inc = 0;
  int32_t max_row = 0, max_deg = 0;
  int pos_bytes = 1;
  int key_shift = 4;     // incidence key (e << key_shift) | a: 4 bits of local index up to 16 nodes, else 6
  int32_t tile_slots = 3072;
  int64_t n_tiles = 0;
  int64_t tile_elems_total = 0;
  int32_t max_tile_nel = 0, max_tile_nodes = 0, max_tile_front = 0, max_tile_back = 0, max_tile_nl = 0;
  int ent_bytes = 2;     // 2 or 4: contribution entry width in the tile blocks
  int min_ent_bytes = 2; // batches may ask for the wider entries
  int debug_starve = 0;  // test knob: the first CTA skips its first metadata copy (bounded wait runs out)
  int32_t chunk = 0;    // elements per chunk (0 = default)
  int32_t threads = 0;  // threads per block (0 = default)
  // LFEM_MIXED: metric quality below which an element is redone in double;
  // 4k/(1+k)^2 at k = 64, the largest quality of a metric with cond(G) = 64
  float qmin = 256.0f / 4225.0f;
  lfem::PatternDev d;
};

namespace lfem {
lfem_status build_tiles(lfem_pattern_s* p, int32_t tile_slots, cudaStream_t st);
// Element buffer of the element-major paths for nm matrices (grown, never shrunk).
size_t elem_buf_local_bytes(const lfem_pattern_s* p, int nm, bool mixed);
lfem_status reserve_elem_buf(lfem_pattern_s* p, int nm, bool mixed, int q);
}
