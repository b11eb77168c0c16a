// C ABI of the library: argument checks, reference tables, dispatch.
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <sstream>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "dispatch.cuh"

namespace lfem {

static thread_local std::string g_err;

void set_error(const std::string& msg) { g_err = msg; }

static std::atomic<long long> g_alloc_count{0};
cudaError_t dev_malloc(void** p, size_t bytes) {
  const cudaError_t e = cudaMalloc(p, bytes);
  if (e == cudaSuccess) g_alloc_count.fetch_add(1, std::memory_order_relaxed);
  return e;
}
lfem_status fail(lfem_status s, const std::string& msg) {
  g_err = msg;
  return s;
}
lfem_status cuda_fail(cudaError_t e, const char* what) {
  g_err = std::string(what) + ": " + cudaGetErrorString(e);
  return LFEM_E_CUDA;
}

bool supported(int dim, int ambient, int order) {
  if (order < 1 || order > 4) return false;
  if (dim < 1 || dim > 3 || ambient < dim || ambient > 3) return false;
  if (dim == 2 && ambient == 3) return true;
  if (dim == ambient) return true;
  return dim == 1;
}

// ---------------------------------------------------------------------------
// Reference tables: Lagrange P1/P2 basis (corner functions l_a, or
// l_a (2 l_a - 1) and edge functions 4 l_i l_j) with their reference gradients
// at the quadrature points, and the gradients of the edge bubbles 4 l_i l_j.
// ---------------------------------------------------------------------------
static void edge_nodes(int dim, int k, int& i, int& j) {
  static const int E1[1][2] = {{0, 1}};
  static const int E2[3][2] = {{0, 1}, {1, 2}, {2, 0}};
  static const int E3[6][2] = {{0, 1}, {1, 2}, {2, 0}, {0, 3}, {1, 3}, {2, 3}};
  const int(*E)[2] = dim == 1 ? E1 : (dim == 2 ? E2 : E3);
  i = E[k][0];
  j = E[k][1];
}

// Orders 3, 4 (curves, triangles): barycentric multi-indices of the nodes in
// the library's order -- corners; per edge (i, j) of the P2 edge order the
// nodes (p-k) e_i + k e_j, k = 1..p-1; interior nodes by increasing
// (alpha_1, alpha_2) -- and the Lagrange basis prod_i l_{alpha_i}(lambda_i),
// l_k(t) = prod_{j<k} (p t - j) / (j + 1).
static int high_order_nodes(int dim, int p, int al[][4]) {
  int n = 0;
  for (int i = 0; i <= dim; ++i) {
    for (int c = 0; c < 4; ++c) al[n][c] = c == i ? p : 0;
    ++n;
  }
  const int ne = dim == 1 ? 1 : 3;
  for (int k = 0; k < ne; ++k) {
    int i, j;
    edge_nodes(dim, k, i, j);
    for (int t = 1; t < p; ++t) {
      for (int c = 0; c < 4; ++c) al[n][c] = 0;
      al[n][i] = p - t;
      al[n][j] = t;
      ++n;
    }
  }
  if (dim == 2)
    for (int a1 = 1; a1 < p; ++a1)
      for (int a2 = 1; a1 + a2 < p; ++a2) {
        al[n][0] = p - a1 - a2;
        al[n][1] = a1;
        al[n][2] = a2;
        al[n][3] = 0;
        ++n;
      }
  return n;
}

static void lagrange_factor(int p, int k, double t, double& v, double& dv) {
  v = 1.0;
  dv = 0.0;
  for (int j = 0; j < k; ++j) {
    const double f = (p * t - j) / (j + 1);
    dv = dv * f + v * ((double)p / (j + 1));
    v *= f;
  }
}

static void host_tables(int dim, int order, const lfem_quad* quad, std::vector<double>& out) {
  const int Q = quad->n_pts, REF = n_ref(dim, order), NE = n_edges(dim, order);
  if (dim == 3 && order >= 3) {
    // order-3/4 tets tabulate their basis on the device: the rule alone, w[Q] then xi[Q][3]
    out.assign((size_t)Q * 4, 0.0);
    for (int q = 0; q < Q; ++q) {
      out[q] = quad->w[q];
      for (int m = 0; m < 3; ++m) out[Q + q * 3 + m] = quad->xi[q * 3 + m];
    }
    return;
  }
  out.assign((size_t)Q * (1 + REF + REF * dim + NE * dim), 0.0);
  double* w = out.data();
  double* phi = w + Q;
  double* dphi = phi + Q * REF;
  double* dpsi = dphi + Q * REF * dim;
  for (int q = 0; q < Q; ++q) {
    w[q] = quad->w[q];
    double lam[4], dlam[4][3];
    double sum = 0.0;
    for (int m = 0; m < dim; ++m) sum += quad->xi[q * dim + m];
    lam[0] = 1.0 - sum;
    for (int m = 0; m < dim; ++m) lam[m + 1] = quad->xi[q * dim + m];
    for (int i = 0; i <= dim; ++i)
      for (int m = 0; m < dim; ++m) dlam[i][m] = (i == 0) ? -1.0 : (i == m + 1 ? 1.0 : 0.0);
    if (order >= 3) {
      int al[16][4];
      const int n = high_order_nodes(dim, order, al);
      for (int a = 0; a < n; ++a) {
        double v[4], dv[4];
        for (int i = 0; i <= dim; ++i) lagrange_factor(order, al[a][i], lam[i], v[i], dv[i]);
        double prod = 1.0;
        for (int i = 0; i <= dim; ++i) prod *= v[i];
        phi[q * REF + a] = prod;
        for (int m = 0; m < dim; ++m) {
          double g = 0.0;
          for (int i = 0; i <= dim; ++i) {
            double t = dv[i] * dlam[i][m];
            for (int l = 0; l <= dim; ++l)
              if (l != i) t *= v[l];
            g += t;
          }
          dphi[(q * REF + a) * dim + m] = g;
        }
      }
      continue;
    }
    for (int a = 0; a <= dim; ++a) {
      phi[q * REF + a] = order == 1 ? lam[a] : lam[a] * (2.0 * lam[a] - 1.0);
      for (int m = 0; m < dim; ++m) dphi[(q * REF + a) * dim + m] = order == 1 ? dlam[a][m] : (4.0 * lam[a] - 1.0) * dlam[a][m];
    }
    for (int k = 0; k < NE; ++k) {
      int i, j;
      edge_nodes(dim, k, i, j);
      phi[q * REF + dim + 1 + k] = 4.0 * lam[i] * lam[j];
      for (int m = 0; m < dim; ++m) {
        double g = 4.0 * (lam[i] * dlam[j][m] + lam[j] * dlam[i][m]);
        dphi[(q * REF + dim + 1 + k) * dim + m] = g;
        dpsi[(q * NE + k) * dim + m] = g;
      }
    }
  }
}

// Compile-time-quadrature tables: packed pairs (FastLayout2) for curves and
// triangles, the per-point layout (FastLayout) for tetrahedra.  Edge bubble
// gradients, reference gradients, weights and weighted basis products.
int fast_table_size(int dim, int order) {
  if (dim == 1) return order == 1 ? FastLayout2<1, 1>::SIZE : FastLayout2<1, 2>::SIZE;
  if (dim == 2) return order == 1 ? FastLayout2<2, 1>::SIZE : FastLayout2<2, 2>::SIZE;
  return order == 1 ? FastLayout<3, 1>::SIZE : FastLayout<3, 2>::SIZE;
}

bool fast_tables_host(int dim, int order, const lfem_quad* quad, float* dst) {
  const int REF = n_ref(dim, order), NE = n_edges(dim, order), U = n_upper(REF), NK = dim * (dim + 1) / 2;
  const int QF = dim == 1 ? 3 : (dim == 2 ? (order == 1 ? 3 : 7) : (order == 1 ? 4 : 14));
  if (!quad || quad->n_pts != QF || (order != 1 && order != 2)) return false;
  std::vector<double> t;
  host_tables(dim, order, quad, t);
  const int Q = QF;
  const double* w = t.data();
  const double* phi = w + Q;
  const double* dphi = phi + Q * REF;
  const double* dpsi = dphi + Q * REF * dim;
  auto tm = [&](int q, int u) -> double {  // w_q phi_a phi_b of upper entry u (0 past the end)
    for (int a = 0; a < REF; ++a)
      for (int b = a; b < REF; ++b)
        if (upper_index(REF, a, b) == u) return w[q] * phi[q * REF + a] * phi[q * REF + b];
    return 0.0;
  };
  if (dim <= 2) {
    // packed layout (FastLayout2): point pairs (2k, 2k+1); with Q odd the last
    // pair is point Q-1 twice with half its weight in each half
    const int QP = (Q + 1) / 2, UH = (U + 1) / 2;
    const int per_pair = 2 * NE * dim + (dim == 2 ? 2 * REF * dim + 2 : 2 * U);
    for (int k = 0; k < QP; ++k) {
      float* d = dst + (size_t)k * per_pair;
      for (int h = 0; h < 2; ++h) {
        const int q = std::min(2 * k + h, Q - 1);
        const double wq = (2 * k + 1 >= Q) ? 0.5 * w[q] : w[q];
        for (int e = 0; e < NE; ++e)
          for (int m = 0; m < dim; ++m) d[2 * (e * dim + m) + h] = (float)dpsi[(q * NE + e) * dim + m];
        float* r = d + 2 * NE * dim;
        if (dim == 2) {
          for (int b = 0; b < REF; ++b)
            for (int m = 0; m < dim; ++m) r[2 * (b * dim + m) + h] = (float)dphi[(q * REF + b) * dim + m];
          r[2 * REF * dim + h] = (float)wq;
        } else {
          for (int a = 0; a < REF; ++a)
            for (int b = a; b < REF; ++b)
              r[2 * upper_index(REF, a, b) + h] = (float)(wq * dphi[q * REF + a] * dphi[q * REF + b]);
        }
      }
    }
    float* mass = dst + (size_t)QP * per_pair;
    for (int q = 0; q < Q; ++q)
      for (int j = 0; j < UH; ++j) {
        mass[2 * (q * UH + j)] = (float)tm(q, 2 * j);
        mass[2 * (q * UH + j) + 1] = (float)tm(q, 2 * j + 1);
      }
    return true;
  }
  const int per_q = NE * dim + U + REF * dim + 1;
  for (int q = 0; q < Q; ++q) {
    float* d = dst + (size_t)q * per_q;
    for (int k = 0; k < NE; ++k)
      for (int m = 0; m < dim; ++m) d[k * dim + m] = (float)dpsi[(q * NE + k) * dim + m];
    float* tmq = d + NE * dim;
    for (int u = 0; u < U; ++u) tmq[u] = (float)tm(q, u);
    // tetrahedra: reference gradients and the weight (stiffness point by point)
    float* ta = tmq + U;
    for (int b = 0; b < REF; ++b)
      for (int m = 0; m < dim; ++m) ta[b * dim + m] = (float)dphi[(q * REF + b) * dim + m];
    ta[REF * dim] = (float)w[q];
  }
  (void)NK;
  return true;
}

struct TabKey {
  int dev, dim, order, q;
  std::vector<double> data;
  bool operator<(const TabKey& o) const {
    return std::tie(dev, dim, order, q, data) < std::tie(o.dev, o.dim, o.order, o.q, o.data);
  }
};

static std::mutex g_tab_mu;
static std::map<TabKey, TabRef> g_tabs;
static std::map<int, size_t> g_bank_used;  // bytes per device

// Order 1 without a rule: the paper's P1 precomputation (Sec. 4.2) uses the exact
// reference mass matrix and stiffness building blocks.  On affine order-1
// elements the mass integrand is a polynomial of degree 2 and the stiffness
// integrand a constant, so any rule exact to degree 2 returns exactly those
// matrices; these are the degree-2 rules of each element (3-point Gauss on the
// interval, the interior 3-point triangle rule, the 4-point tet rule with
// a = (5 - sqrt 5) / 20), which the compile-time kernels also take.
const lfem_quad* exact_p1_rule(int dim) {
  static double xi1[3], w1[3], xi2[6], w2[3], xi3[12], w3[4];
  static lfem_quad q1{3, xi1, w1}, q2{3, xi2, w2}, q3{4, xi3, w3};
  static std::once_flag once;
  std::call_once(once, [] {
    const double h = std::sqrt(15.0) / 10.0;
    xi1[0] = 0.5 - h;
    xi1[1] = 0.5;
    xi1[2] = 0.5 + h;
    w1[0] = w1[2] = 5.0 / 18.0;
    w1[1] = 8.0 / 18.0;
    const double t[6] = {1.0 / 6.0, 1.0 / 6.0, 2.0 / 3.0, 1.0 / 6.0, 1.0 / 6.0, 2.0 / 3.0};
    for (int k = 0; k < 6; ++k) xi2[k] = t[k];
    w2[0] = w2[1] = w2[2] = 1.0 / 6.0;
    const double a = (5.0 - std::sqrt(5.0)) / 20.0, b = 1.0 - 3.0 * a;
    for (int q = 0; q < 4; ++q)
      for (int m = 0; m < 3; ++m) xi3[q * 3 + m] = (q == m + 1) ? b : a;
    for (int q = 0; q < 4; ++q) w3[q] = 1.0 / 24.0;
  });
  return dim == 1 ? &q1 : (dim == 2 ? &q2 : (dim == 3 ? &q3 : nullptr));
}

// The rule an entry point uses: the caller's, or for order 1 without one the exact rule.
static const lfem_quad* resolve_rule(const lfem_quad* quad, int dim, int order) {
  return quad ? quad : (order == 1 ? exact_p1_rule(dim) : nullptr);
}

lfem_status get_tables(int dim, int order, const lfem_quad* quad, cudaStream_t st, TabRef* out) {
  if (!quad || quad->n_pts <= 0 || !quad->xi || !quad->w) return fail(LFEM_E_ARG, "quadrature rule missing");
  if (quad->n_pts > LFEM_MAX_QPTS) return fail(LFEM_E_UNSUPPORTED, "more than LFEM_MAX_QPTS quadrature points");
  int dev = 0;
  LFEM_CUDA(cudaGetDevice(&dev));
  TabKey key{dev, dim, order, quad->n_pts, {}};
  key.data.assign(quad->xi, quad->xi + (size_t)quad->n_pts * dim);
  key.data.insert(key.data.end(), quad->w, quad->w + quad->n_pts);
  std::lock_guard<std::mutex> lk(g_tab_mu);
  auto it = g_tabs.find(key);
  if (it != g_tabs.end()) {
    *out = it->second;
    return LFEM_OK;
  }
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (st) cudaStreamIsCapturing(st, &cs);
  if (cs != cudaStreamCaptureStatusNone)
    return fail(LFEM_E_ARG, "first use of a quadrature rule inside stream capture; call once before capturing");
  std::vector<double> t64;
  host_tables(dim, order, quad, t64);
  std::vector<float> t32(t64.begin(), t64.end());
  const size_t b64 = t64.size() * sizeof(double);
  const size_t b32 = ((t32.size() * sizeof(float) + 7) / 8) * 8;
  size_t& used = g_bank_used[dev];
  if (used + b64 + b32 > sizeof(double) * 8192) {
    // bank full: start over (kernels in flight may still read old entries)
    LFEM_CUDA(cudaDeviceSynchronize());
    for (auto i = g_tabs.begin(); i != g_tabs.end();) i = (i->first.dev == dev) ? g_tabs.erase(i) : std::next(i);
    used = 0;
    if (b64 + b32 > sizeof(double) * 8192) return fail(LFEM_E_TOO_LARGE, "reference tables exceed constant memory");
  }
  std::vector<unsigned char> blob(b64 + b32, 0);
  memcpy(blob.data(), t64.data(), b64);
  memcpy(blob.data() + b64, t32.data(), t32.size() * sizeof(float));
  for (auto up : {bank_upload_d1, bank_upload_d2, bank_upload_d3, bank_upload_batch, bank_upload_vec,
                  bank_upload_high, bank_upload_tet_high, bank_upload_adj_high}) {
    lfem_status us = up(blob.data(), blob.size(), used);
    if (us != LFEM_OK) return us;
  }
  TabRef r;
  r.q = quad->n_pts;
  r.off64 = (int)(used / sizeof(double));
  r.off32 = (int)((used + b64) / sizeof(float));
  used += blob.size();
  g_tabs[key] = r;
  *out = r;
  return LFEM_OK;
}

lfem_status build_pattern(lfem_pattern_s* p, const int32_t* conn_in, cudaStream_t st);

static lfem_status run_stage(int dim, int NA, int P, int kind, const StageArgs& s, cudaStream_t st) {
  if (P >= 3) {
    // order-3/4 tets keep their basis tables on the device (the rule alone is in the bank)
    if (dim == 3) return fail(LFEM_E_UNSUPPORTED, "the element stages cover order-3/4 curves and triangles, not tets");
    return run_stage_high(dim, NA, P, kind, s, st);
  }
  if (dim == 1) return run_stage_d1(NA, P, kind, s, st);
  if (dim == 2) return run_stage_d2(NA, P, kind, s, st);
  return run_stage_d3(NA, P, kind, s, st);
}
static lfem_status run_adjoint(int dim, int NA, int P, const AdjArgs& a, int64_t T, int pb, cudaStream_t st) {
  if (dim == 1) return run_adjoint_d1(NA, P, a, T, pb, st);
  if (dim == 2) return run_adjoint_d2(NA, P, a, T, pb, st);
  return run_adjoint_d3(NA, P, a, T, pb, st);
}
static lfem_status run_pipe(int dim, int NA, int P, bool mixed, const PipeArgs& a, int pb, bool fast,
                            const FastBank& fb, int sms, cudaStream_t st) {
  if (dim == 1) return run_pipe_d1(NA, P, mixed, a, pb, fast, fb, sms, st);
  if (dim == 2) return run_pipe_d2(NA, P, mixed, a, pb, fast, fb, sms, st);
  return run_pipe_d3(NA, P, mixed, a, pb, fast, fb, sms, st);
}

static void destroy_dev(PatternDev& d) {
  void* ptrs[] = {d.conn,      d.row_ptr,       d.col_idx,   d.inc_ptr,   d.inc_key, d.inc_pos,    d.elem_inc,
                  d.tile_row0, d.tile_elem_ptr, d.tile_elem, d.inc_local, d.status,  d.tile_meta, d.tile_meta_off, d.tile_refs,
                  d.slot_off,  d.slot_ent,      d.elem_buf,  d.vec_buf,   d.mcf_buf};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (d.mcf_graph.exec) cudaGraphExecDestroy(d.mcf_graph.exec);
  d = PatternDev{};
}


}  // namespace lfem

using namespace lfem;

extern "C" {

const char* lfem_last_error(void) { return g_err.c_str(); }

const char* lfem_status_string(lfem_status s) {
  switch (s) {
    case LFEM_OK: return "ok";
    case LFEM_E_ARG: return "invalid argument";
    case LFEM_E_INDEX: return "node index out of range";
    case LFEM_E_UNSUPPORTED: return "unsupported element or rule";
    case LFEM_E_TOO_LARGE: return "size limit exceeded";
    case LFEM_E_NOMEM: return "out of device memory";
    case LFEM_E_CUDA: return "CUDA error";
    case LFEM_E_DEGENERATE: return "degenerate element";
    case LFEM_E_TIMEOUT: return "device wait timed out";
  }
  return "unknown status";
}

lfem_status lfem_pattern(const int32_t* conn, int64_t n_elem, int32_t n_nodes, int dim, int order, void* cuda_stream,
                         lfem_pattern_t* out) {
  if (!out) return fail(LFEM_E_ARG, "out is NULL");
  *out = nullptr;
  if (n_elem < 0 || n_nodes < 0) return fail(LFEM_E_ARG, "negative size");
  if (n_elem > 0 && !conn) return fail(LFEM_E_ARG, "conn is NULL");
  if (dim < 1 || dim > 3 || order < 1 || order > 4) return fail(LFEM_E_UNSUPPORTED, "dim/order");
  const int ref = n_ref(dim, order);
  const int ksh = ref > 16 ? 6 : 4;
  if (n_elem >= (1ll << (31 - ksh)) || n_elem * ref >= (1ll << 31)) return fail(LFEM_E_TOO_LARGE, "too many elements");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  lfem_pattern_s* p = new lfem_pattern_s();
  cudaGetDevice(&p->device);
  p->dim = dim;
  p->order = order;
  p->ref = ref;
  p->key_shift = ksh;
  p->n_elem = n_elem;
  p->n_nodes = n_nodes;
  // default tile capacity: all of a tile's local matrices stay in shared memory
  p->tile_slots = ref >= 10 ? 1024 : 2048;
  lfem_status s = build_pattern(p, conn, st);
  if (s != LFEM_OK) {
    std::string keep = g_err;
    destroy_dev(p->d);
    delete p;
    g_err = keep;
    return s;
  }
  *out = p;
  return LFEM_OK;
}

lfem_status lfem_pattern_csr(lfem_pattern_t p, int64_t* n_rows, int64_t* nnz, const int64_t** row_ptr,
                             const int32_t** col_idx) {
  if (!p) return fail(LFEM_E_ARG, "pattern is NULL");
  if (n_rows) *n_rows = p->n_nodes;
  if (nnz) *nnz = p->nnz;
  if (row_ptr) *row_ptr = p->d.row_ptr;
  if (col_idx) *col_idx = p->d.col_idx;
  return LFEM_OK;
}

lfem_status lfem_pattern_copy_csr(lfem_pattern_t p, int64_t* row_ptr, int32_t* col_idx, void* cuda_stream) {
  if (!p || !row_ptr || (!col_idx && p->nnz > 0)) return fail(LFEM_E_ARG, "NULL argument");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  LFEM_CUDA(cudaMemcpyAsync(row_ptr, p->d.row_ptr, sizeof(int64_t) * ((size_t)p->n_nodes + 1), cudaMemcpyDeviceToDevice, st));
  if (p->nnz > 0)
    LFEM_CUDA(cudaMemcpyAsync(col_idx, p->d.col_idx, sizeof(int32_t) * (size_t)p->nnz, cudaMemcpyDeviceToDevice, st));
  return LFEM_OK;
}

lfem_status lfem_pattern_info(lfem_pattern_t p, int64_t* n_tiles, int64_t* recompute_x1000, int32_t* max_row,
                              int32_t* tile_slots) {
  if (!p) return fail(LFEM_E_ARG, "pattern is NULL");
  if (n_tiles) *n_tiles = p->n_tiles;
  if (recompute_x1000) *recompute_x1000 = p->n_elem ? (p->tile_elems_total * 1000) / p->n_elem : 0;
  if (max_row) *max_row = p->max_row;
  if (tile_slots) *tile_slots = p->tile_slots;
  return LFEM_OK;
}

lfem_status lfem_pattern_retile(lfem_pattern_t p, int32_t tile_slots, void* cuda_stream) {
  if (!p) return fail(LFEM_E_ARG, "pattern is NULL");
  return build_tiles(p, tile_slots, (cudaStream_t)cuda_stream);
}

void lfem_pattern_destroy(lfem_pattern_t p) {
  if (!p) return;
  destroy_dev(p->d);
  delete p;
}

lfem_status lfem_set_launch(lfem_pattern_t p, int32_t elems_per_chunk, int32_t threads) {
  if (!p) return fail(LFEM_E_ARG, "pattern is NULL");
  if (elems_per_chunk < 0 || threads < 0 || (threads && (threads % 32 || threads > 256)))
    return fail(LFEM_E_ARG, "launch configuration");
  if (elems_per_chunk) p->chunk = elems_per_chunk;
  if (threads) p->threads = threads;
  return LFEM_OK;
}

lfem_status lfem_set_mixed_kappa(lfem_pattern_t p, double kappa_max) {
  if (!p) return fail(LFEM_E_ARG, "pattern is NULL");
  if (!(kappa_max >= 1.0)) return fail(LFEM_E_ARG, "kappa_max must be >= 1");
  // q = 4 k / (1 + k)^2, the largest metric quality of a metric with condition number k
  p->qmin = std::isinf(kappa_max) ? 0.0f : (float)(4.0 * kappa_max / ((1.0 + kappa_max) * (1.0 + kappa_max)));
  return LFEM_OK;
}

lfem_status lfem_debug_wide_entries(lfem_pattern_t p, int wide, void* cuda_stream) {
  if (!p) return fail(LFEM_E_ARG, "pattern is NULL");
  p->min_ent_bytes = wide ? 4 : 2;
  if (p->ref > 16) return LFEM_OK;  // no row tiles
  return build_tiles(p, p->tile_slots, (cudaStream_t)cuda_stream);
}

long long lfem_debug_alloc_count(void) { return lfem::g_alloc_count.load(std::memory_order_relaxed); }

lfem_status lfem_debug_starve_wait(lfem_pattern_t p, int starve) {
  if (!p) return fail(LFEM_E_ARG, "pattern is NULL");
  p->debug_starve = starve ? 1 : 0;
  return LFEM_OK;
}

}  // extern "C"

namespace lfem {

size_t elem_buf_local_bytes(const lfem_pattern_s* p, int nm, bool mixed) {
  return ((size_t)p->n_elem * nm * n_upper(p->ref) * (mixed ? 4 : 8) + 255) / 256 * 256;
}

// The element-major paths (tets, orders 3 and 4): the local matrices, then the
// order-3/4 tet tables and list, or the P2 tets' redo list.
lfem_status reserve_elem_buf(lfem_pattern_s* p, int nm, bool mixed, int q) {
  const bool tet_high = p->dim == 3 && p->order >= 3;
  const size_t redo_bytes = (size_t)p->n_elem * sizeof(int32_t);
  const size_t need =
      elem_buf_local_bytes(p, nm, mixed) + (tet_high ? tet_high_scratch_bytes(p->order, q, p->n_elem) : redo_bytes);
  if (need > p->d.elem_buf_bytes) {
    if (p->d.elem_buf) cudaFree(p->d.elem_buf);
    p->d.elem_buf = nullptr;
    p->d.elem_buf_bytes = 0;
    if (dev_malloc(&p->d.elem_buf, need ? need : 16) != cudaSuccess) {
      cudaGetLastError();
      return fail(LFEM_E_NOMEM, "element buffer allocation failed");
    }
    p->d.elem_buf_bytes = need;
  }
  return LFEM_OK;
}

}  // namespace lfem

extern "C" {

lfem_status lfem_assemble(lfem_pattern_t p, const double* coords, int ambient, const lfem_quad* quad,
                          const void* coef, int coef_is_fp32, unsigned which, lfem_precision prec, void* M, void* A,
                          void* MC, void* cuda_stream) {
  if (!p) return fail(LFEM_E_ARG, "pattern is NULL");
  if (!supported(p->dim, ambient, p->order)) return fail(LFEM_E_UNSUPPORTED, "(dim, ambient, order)");
  if (which == 0 || (which & ~7u)) return fail(LFEM_E_ARG, "which");
  if (prec != LFEM_FP64 && prec != LFEM_MIXED) return fail(LFEM_E_ARG, "precision");
  if ((which & LFEM_MASS) && !M) return fail(LFEM_E_ARG, "M is NULL");
  if ((which & LFEM_STIFF) && !A) return fail(LFEM_E_ARG, "A is NULL");
  if ((which & LFEM_CMASS) && (!MC || !coef)) return fail(LFEM_E_ARG, "MC or coef is NULL");
  if ((which & LFEM_CMASS) && !quad) return fail(LFEM_E_ARG, "LFEM_CMASS needs a quadrature rule");
  if (p->n_elem > 0 && !coords) return fail(LFEM_E_ARG, "coords is NULL");
  quad = resolve_rule(quad, p->dim, p->order);
  cudaStream_t st = (cudaStream_t)cuda_stream;
  TabRef tab;
  lfem_status s = get_tables(p->dim, p->order, quad, st, &tab);
  if (s != LFEM_OK) return s;
  const bool mixed = prec == LFEM_MIXED;
  AsmArgs a{};
  a.conn = p->d.conn;
  a.coords = coords;
  a.coef = coef;
  a.coef_f32 = coef_is_fp32 ? 1 : 0;
  a.row_ptr = p->d.row_ptr;
  a.inc_ptr = p->d.inc_ptr;
  a.inc_pos = p->d.inc_pos;
  a.inc_local = p->d.inc_local;
  a.tile_row0 = p->d.tile_row0;
  a.tile_elem_ptr = p->d.tile_elem_ptr;
  a.tile_elem = p->d.tile_elem;
  a.which = which;
  int nm = 0;
  if (which & LFEM_MASS) { a.out[nm] = M; a.mat[nm++] = 0; }
  if (which & LFEM_STIFF) { a.out[nm] = A; a.mat[nm++] = 1; }
  if (which & LFEM_CMASS) { a.out[nm] = MC; a.mat[nm++] = 2; }
  a.nm = nm;
  a.tab = tab;
  a.slots_cap = p->tile_slots;
  a.qmin = p->qmin;
  a.status = p->d.status;
  a.fallback = reinterpret_cast<unsigned long long*>(p->d.status + 2);
  if (p->dim == 3 || p->order >= 3) {
    // bulk tets and orders 3, 4: element-major two passes (local-matrix buffer owned by the pattern;
    // order-3/4 tets keep their basis tables and recomputation list behind the local matrices)
    const bool tet_high = p->dim == 3 && p->order >= 3;
    const size_t lbytes = elem_buf_local_bytes(p, nm, mixed);
    if ((s = reserve_elem_buf(p, nm, mixed, tab.q)) != LFEM_OK) return s;
    TwoPassArgs ta{};
    ta.conn = p->d.conn;
    ta.coords = coords;
    ta.coef = coef;
    ta.coef_f32 = a.coef_f32;
    ta.n_elem = p->n_elem;
    ta.nnz = p->nnz;
    ta.slot_off = p->d.slot_off;
    ta.slot_ent = p->d.slot_ent;
    ta.lbuf = p->d.elem_buf;
    for (int m = 0; m < 3; ++m) ta.out[m] = a.out[m];
    ta.nm = nm;
    ta.which = which;
    ta.tab = tab;
    ta.qmin = a.qmin;
    ta.status = p->d.status;
    ta.fallback = a.fallback;
    ta.redo = reinterpret_cast<int32_t*>(static_cast<char*>(p->d.elem_buf) + lbytes);
    int sms3 = 0;
    LFEM_CUDA(cudaDeviceGetAttribute(&sms3, cudaDevAttrMultiProcessorCount, p->device));
    if (mixed) LFEM_CUDA(cudaMemsetAsync(p->d.status + 2, 0, sizeof(unsigned long long), st));
    if (p->dim != 3) return run_twopass_high(p->dim, ambient, p->order, mixed, ta, sms3, st);
    if (tet_high) return run_tet_high(p->order, mixed, ta, static_cast<char*>(p->d.elem_buf) + lbytes, sms3, st);
    FastBankTet fbt;
    const bool fast3 = mixed && fast_tables_host(3, p->order, quad, fbt.v + (p->order == 1 ? FastBankTet::OFF31
                                                                                          : FastBankTet::OFF32));
    return run_twopass_d3(p->order, mixed, fast3, fbt, ta, sms3, st);
  }
  // persistent pipelined kernel: a lane pair per element, so 96 (float) or
  // 128 (double) elements per phase-1 round; all of a tile's local matrices
  // stay in shared memory
  PipeArgs pa{};
  MeshRec& mr = pa.one;
  mr.coords = coords;
  mr.coef = coef;
  for (int m = 0; m < 3; ++m) mr.out[m] = a.out[m];
  mr.tab = tab;
  mr.type = elem_type_id(p->dim, ambient, p->order);
  mr.na = ambient;
  mr.ref = p->ref;
  mr.entb = p->ent_bytes;
  mr.coef_f32 = a.coef_f32;
  mr.c16 = reinterpret_cast<uintptr_t>(coords) % 16 == 0 ? 1 : 0;
  pa.meshes = nullptr;
  pa.items = p->d.tile_refs;
  pa.n_items = p->n_tiles;
  pa.nm = nm;
  pa.which = which;
  pa.chunk = (mixed ? PipeOcc<float>::THREADS : PipeOcc<double>::THREADS) / kPipeTPE;
  pa.cap_front = p->max_tile_front;
  pa.cap_back = p->max_tile_back;
  pa.cap_nodes = p->max_tile_nodes;
  pa.cap_nel = p->max_tile_nel;
  pa.max_u = n_upper(p->ref);
  pa.cap_lsm = lsm_words(p->max_tile_nel, n_upper(p->ref), p->max_tile_nl, mixed ? kLsmSlots : nm);
  pa.vec_out = 1;
  for (int m = 0; m < nm; ++m)
    if (reinterpret_cast<uintptr_t>(a.out[m]) % 16) pa.vec_out = 0;
  pa.max_q = tab.q;
  pa.coef_bytes = (which & LFEM_CMASS) ? (coef_is_fp32 ? 4 : 8) : 0;
  pa.coef_smem = pa.coef_bytes;
  pa.qmin = a.qmin;
  pa.status = p->d.status;
  pa.next_item = reinterpret_cast<unsigned int*>(p->d.status + 4);
  pa.fallback = a.fallback;
  pa.starve = p->debug_starve;
  pa.wait_ns = 2000000000ll;  // 2 s bound on every mbarrier wait
  int sms = 0;
  LFEM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device));
  if (mixed) LFEM_CUDA(cudaMemsetAsync(p->d.status + 2, 0, sizeof(unsigned long long), st));
  LFEM_CUDA(cudaMemsetAsync(p->d.status + 4, 0, sizeof(unsigned long long), st));  // tile tickets
  // the usual rules run with compile-time quadrature (tables as kernel parameters)
  FastBank fb;
  bool fast = false;
  if (mixed && p->dim <= 2) {
    const int off = p->dim == 1 ? (p->order == 1 ? FastBank::OFF11 : FastBank::OFF12)
                                : (p->order == 1 ? FastBank::OFF21 : FastBank::OFF22);
    fast = fast_tables_host(p->dim, p->order, quad, fb.v + off);
  }
  return run_pipe(p->dim, ambient, p->order, mixed, pa, p->ent_bytes, fast, fb, sms, st);
}

static lfem_status adjoint_common(lfem_pattern_t p, const double* coords, int ambient, const lfem_quad* quad,
                                  const double* coef, const double* gM, const double* gA, const double* gMC,
                                  double* g_coords, double* g_coef, bool mixed, void* cuda_stream);

lfem_status lfem_assemble_adjoint(lfem_pattern_t p, const double* coords, int ambient, const lfem_quad* quad,
                                  const double* coef, const double* gM, const double* gA, const double* gMC,
                                  double* g_coords, double* g_coef, void* cuda_stream) {
  return adjoint_common(p, coords, ambient, quad, coef, gM, gA, gMC, g_coords, g_coef, false, cuda_stream);
}

lfem_status lfem_assemble_adjoint_mixed(lfem_pattern_t p, const double* coords, int ambient, const lfem_quad* quad,
                                        const double* coef, const double* gM, const double* gA, const double* gMC,
                                        double* g_coords, double* g_coef, void* cuda_stream) {
  return adjoint_common(p, coords, ambient, quad, coef, gM, gA, gMC, g_coords, g_coef, true, cuda_stream);
}

}  // extern "C"

static lfem_status adjoint_common(lfem_pattern_t p, const double* coords, int ambient, const lfem_quad* quad,
                                  const double* coef, const double* gM, const double* gA, const double* gMC,
                                  double* g_coords, double* g_coef, bool mixed, void* cuda_stream) {
  if (!p) return fail(LFEM_E_ARG, "pattern is NULL");
  if (!supported(p->dim, ambient, p->order)) return fail(LFEM_E_UNSUPPORTED, "(dim, ambient, order)");
  if (!g_coords && p->n_nodes > 0) return fail(LFEM_E_ARG, "g_coords is NULL");
  if (p->n_elem > 0 && !coords) return fail(LFEM_E_ARG, "coords is NULL");
  if (gMC && !coef) return fail(LFEM_E_ARG, "gMC given without coef");
  if (!quad && (gMC || g_coef)) return fail(LFEM_E_ARG, "coefficient gradients need a quadrature rule");
  quad = resolve_rule(quad, p->dim, p->order);
  cudaStream_t st = (cudaStream_t)cuda_stream;
  TabRef tab;
  lfem_status s = get_tables(p->dim, p->order, quad, st, &tab);
  if (s != LFEM_OK) return s;
  AdjArgs a{};
  a.conn = p->d.conn;
  a.coords = coords;
  a.coef = coef;
  a.gM = gM;
  a.gA = gA;
  a.gC = gMC;
  a.g_coords = g_coords;
  a.g_coef = g_coef;
  a.row_ptr = p->d.row_ptr;
  a.inc_ptr = p->d.inc_ptr;
  a.inc_pos = p->d.inc_pos;
  a.inc_local = p->d.inc_local;
  a.elem_inc = p->d.elem_inc;
  a.tile_row0 = p->d.tile_row0;
  a.tile_elem_ptr = p->d.tile_elem_ptr;
  a.tile_elem = p->d.tile_elem;
  a.tab = tab;
  a.chunk = 128;
  a.mixed = mixed ? 1 : 0;
  // G^{-1} enters the adjoint twice (d(s G^{-1})), so its conditioning test
  // uses sqrt(kappa_max): q >= 4k'/(1+k')^2 with k' = sqrt(k), k from qmin
  {
    const double q = p->qmin;
    const double k = q > 0.0 ? (2.0 - q + 2.0 * std::sqrt(1.0 - q)) / q : 0.0;  // inverse of q = 4k/(1+k)^2
    const double ka = k > 1.0 ? std::sqrt(k) : 1.0;
    a.qmin = q > 0.0 ? (float)(4.0 * ka / ((1.0 + ka) * (1.0 + ka))) : 0.0f;
  }
  a.fallback = reinterpret_cast<unsigned long long*>(p->d.status + 2);
  if (mixed) LFEM_CUDA(cudaMemsetAsync(p->d.status + 2, 0, sizeof(unsigned long long), st));
  if (g_coef && !gMC && p->n_elem > 0) {
    // dL/dc is zero without gMC
    LFEM_CUDA(cudaMemsetAsync(g_coef, 0, sizeof(double) * p->n_elem * quad->n_pts, st));
    a.g_coef = nullptr;
  }
  if (p->order >= 3) {
    // warp per element in double, element node gradients in the pattern's
    // element buffer, then a per-node pass over the incidences
    const size_t need = adjoint_high_scratch_bytes(p->dim, p->order, tab.q, ambient, p->n_elem);
    if (need > p->d.elem_buf_bytes) {
      if (p->d.elem_buf) cudaFree(p->d.elem_buf);
      p->d.elem_buf = nullptr;
      p->d.elem_buf_bytes = 0;
      if (dev_malloc(&p->d.elem_buf, need ? need : 16) != cudaSuccess) {
        cudaGetLastError();
        return fail(LFEM_E_NOMEM, "element buffer allocation failed");
      }
      p->d.elem_buf_bytes = need;
    }
    a.inc_key = p->d.inc_key;
    a.key_shift = p->key_shift;
    a.n_elem = p->n_elem;
    a.n_nodes = p->n_nodes;
    int sms = 0;
    LFEM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device));
    return run_adjoint_high(p->dim, ambient, p->order, a, p->pos_bytes, p->d.elem_buf, sms, st);
  }
  return run_adjoint(p->dim, ambient, p->order, a, p->n_tiles, p->pos_bytes, st);
}

extern "C" {

static lfem_status stage_common(int kind, const int32_t* conn, int64_t n_elem, int dim, int order,
                                const double* coords, int ambient, const lfem_quad* quad, const double* coef,
                                unsigned which, double* o0, double* o1, double* o2, void* cuda_stream) {
  if (n_elem < 0) return fail(LFEM_E_ARG, "negative size");
  if (!supported(dim, ambient, order)) return fail(LFEM_E_UNSUPPORTED, "(dim, ambient, order)");
  if (n_elem > 0 && (!conn || !coords)) return fail(LFEM_E_ARG, "conn or coords is NULL");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  TabRef tab;
  lfem_status s = get_tables(dim, order, quad, st, &tab);
  if (s != LFEM_OK) return s;
  StageArgs a{conn, n_elem, coords, tab, coef, which, o0, o1, o2};
  return run_stage(dim, ambient, order, kind, a, st);
}

lfem_status lfem_eval_points(const int32_t* conn, int64_t n_elem, int dim, int order, const double* coords,
                             int ambient, const lfem_quad* quad, double* out, void* cuda_stream) {
  if (!out && n_elem > 0) return fail(LFEM_E_ARG, "out is NULL");
  return stage_common(0, conn, n_elem, dim, order, coords, ambient, quad, nullptr, 0, out, nullptr, nullptr,
                      cuda_stream);
}

lfem_status lfem_geometry(const int32_t* conn, int64_t n_elem, int dim, int order, const double* coords,
                          int ambient, const lfem_quad* quad, double* J, double* s, double* Ginv,
                          void* cuda_stream) {
  return stage_common(1, conn, n_elem, dim, order, coords, ambient, quad, nullptr, 0, J, s, Ginv, cuda_stream);
}

lfem_status lfem_local(const int32_t* conn, int64_t n_elem, int dim, int order, const double* coords, int ambient,
                       const lfem_quad* quad, const double* coef, double* Mloc, double* Aloc, double* MCloc,
                       void* cuda_stream) {
  unsigned which = (Mloc ? LFEM_MASS : 0) | (Aloc ? LFEM_STIFF : 0) | (MCloc ? LFEM_CMASS : 0);
  if (!which) return fail(LFEM_E_ARG, "no output requested");
  if (MCloc && !coef) return fail(LFEM_E_ARG, "MCloc requested without coef");
  return stage_common(2, conn, n_elem, dim, order, coords, ambient, quad, coef, which, Mloc, Aloc, MCloc,
                      cuda_stream);
}

lfem_status lfem_sync_status(lfem_pattern_t p, void* cuda_stream) {
  if (!p) return fail(LFEM_E_ARG, "pattern is NULL");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int32_t h = 0;
  LFEM_CUDA(cudaMemcpyAsync(&h, p->d.status, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  LFEM_CUDA(cudaMemsetAsync(p->d.status, 0, sizeof(int32_t), st));
  LFEM_CUDA(cudaStreamSynchronize(st));
  if (h & ST_TIMEOUT) return fail(LFEM_E_TIMEOUT, "a bounded device wait ran out");
  if (h & ST_ITEM) return fail(LFEM_E_CUDA, "a work-item record failed its size or alignment check");
  if (h & ST_INDEX) return fail(LFEM_E_INDEX, "node index out of range");
  if (h & ST_TYPE) return fail(LFEM_E_UNSUPPORTED, "a tile met a kernel without its element type");
  if (h & ST_DEGENERATE) return fail(LFEM_E_DEGENERATE, "zero or non-finite |det DF| at a quadrature point");
  return LFEM_OK;
}

}  // extern "C"

static lfem_status vectors_common(lfem_pattern_t p, const double* coords, int ambient, const lfem_quad* quad,
                                  const double* u, double* out, int kind, cudaStream_t st) {
  if (!p) return fail(LFEM_E_ARG, "pattern is NULL");
  if (!supported(p->dim, ambient, p->order)) return fail(LFEM_E_UNSUPPORTED, "(dim, ambient, order)");
  if (kind == 1 && !(p->dim == 2 && ambient == 3))
    return fail(LFEM_E_UNSUPPORTED, "the non-linear vectors need a surface (dim 2 in R^3)");
  if (p->n_elem > 0 && (!coords || !u)) return fail(LFEM_E_ARG, "coords or nodal values are NULL");
  if (p->n_nodes > 0 && !out) return fail(LFEM_E_ARG, "output is NULL");
  quad = resolve_rule(quad, p->dim, p->order);
  TabRef tab;
  lfem_status s = get_tables(p->dim, p->order, quad, st, &tab);
  if (s != LFEM_OK) return s;
  const int nc = kind == 0 ? 1 : 4;
  // order-3/4 tets keep their device basis tables behind the local vectors
  const bool tet_high = p->dim == 3 && p->order >= 3;
  const size_t lbytes = ((size_t)p->n_elem * p->ref * nc * sizeof(double) + 255) / 256 * 256;
  const size_t need = lbytes + (tet_high ? tet_high_scratch_bytes(p->order, tab.q, 0) : 0);
  if (need > p->d.vec_buf_bytes) {
    if (p->d.vec_buf) cudaFree(p->d.vec_buf);
    p->d.vec_buf = nullptr;
    p->d.vec_buf_bytes = 0;
    if (dev_malloc((void**)&p->d.vec_buf, need ? need : 16) != cudaSuccess) {
      cudaGetLastError();
      return fail(LFEM_E_NOMEM, "local-vector buffer allocation failed");
    }
    p->d.vec_buf_bytes = need;
  }
  VecArgs a{};
  a.conn = p->d.conn;
  a.coords = coords;
  a.u = u;
  a.loc = p->d.vec_buf;
  a.inc_ptr = p->d.inc_ptr;
  a.inc_key = p->d.inc_key;
  a.out = out;
  a.n_elem = p->n_elem;
  a.n_nodes = p->n_nodes;
  a.key_shift = p->key_shift;
  a.tab = tab;
  if (tet_high) {
    int sms = 0;
    LFEM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device));
    return run_tet_high_load(p->order, a, reinterpret_cast<char*>(p->d.vec_buf) + lbytes, sms, st);
  }
  return run_vectors(p->dim, ambient, p->order, kind, a, st);
}

extern "C" {

lfem_status lfem_assemble_load(lfem_pattern_t p, const double* coords, int ambient, const lfem_quad* quad,
                               const double* f, double* b, void* cuda_stream) {
  return vectors_common(p, coords, ambient, quad, f, b, 0, (cudaStream_t)cuda_stream);
}

lfem_status lfem_mcf_step(lfem_pattern_t p, const double* coords, int ambient, const lfem_quad* quad, double tau,
                          double rtol, int max_iter, double* coords_out, int* iterations, void* cuda_stream) {
  if (!p) return fail(LFEM_E_ARG, "pattern is NULL");
  if (!supported(p->dim, ambient, p->order) || ambient != p->dim + 1)
    return fail(LFEM_E_UNSUPPORTED, "mean curvature flow needs a curve in R^2 or a surface in R^3");
  if (!(tau >= 0.0) || !(rtol > 0.0) || max_iter <= 0) return fail(LFEM_E_ARG, "tau, rtol or max_iter");
  if (!iterations || (p->n_nodes > 0 && (!coords || !coords_out))) return fail(LFEM_E_ARG, "NULL argument");
  quad = resolve_rule(quad, p->dim, p->order);
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const int nc = ambient;
  const size_t nnz = (size_t)p->nnz, n = (size_t)p->n_nodes;
  auto al = [](size_t b) { return (b + 255) / 256 * 256; };
  const size_t b_mat = al(sizeof(double) * nnz), b_vec = al(sizeof(double) * n * nc), b_dg = al(sizeof(double) * n);
  const size_t b_part = al(sizeof(double) * 4 * kMcfBlocks * 3), b_sc = al(sizeof(McfScalars));
  const size_t need = 3 * b_mat + b_dg + 6 * b_vec + b_part + b_sc;
  if (need > p->d.mcf_buf_bytes) {
    if (p->d.mcf_buf) cudaFree(p->d.mcf_buf);
    p->d.mcf_buf = nullptr;
    p->d.mcf_buf_bytes = 0;
    if (dev_malloc(&p->d.mcf_buf, need) != cudaSuccess) {
      cudaGetLastError();
      return fail(LFEM_E_NOMEM, "flow-step scratch allocation failed");
    }
    p->d.mcf_buf_bytes = need;
  }
  char* base = static_cast<char*>(p->d.mcf_buf);
  auto take = [&](size_t b) {
    char* r = base;
    base += b;
    return r;
  };
  McfSolveArgs s{};
  double* M = reinterpret_cast<double*>(take(b_mat));
  double* A = reinterpret_cast<double*>(take(b_mat));
  s.K = reinterpret_cast<double*>(take(b_mat));
  s.dinv = reinterpret_cast<double*>(take(b_dg));
  s.X = reinterpret_cast<double*>(take(b_vec));
  s.B = reinterpret_cast<double*>(take(b_vec));
  s.Q = reinterpret_cast<double*>(take(b_vec));
  s.R = reinterpret_cast<double*>(take(b_vec));
  s.Z = reinterpret_cast<double*>(take(b_vec));
  s.P = reinterpret_cast<double*>(take(b_vec));
  s.part = reinterpret_cast<double*>(take(b_part));
  s.scalars = reinterpret_cast<McfScalars*>(take(b_sc));
  s.graph = &p->d.mcf_graph;
  lfem_status e = lfem_assemble(p, coords, ambient, quad, nullptr, 0, LFEM_MASS | LFEM_STIFF, LFEM_FP64, M, A,
                                nullptr, cuda_stream);
  if (e != LFEM_OK) return e;
  s.row_ptr = p->d.row_ptr;
  s.col_idx = p->d.col_idx;
  s.M = M;
  s.A = A;
  s.tau = tau;
  s.n = p->n_nodes;
  s.X0 = coords;
  s.X_out = coords_out;
  s.rtol = rtol;
  s.max_iter = max_iter;
  return run_mcf_solve(nc, s, st, iterations);
}

lfem_status lfem_assemble_mcf_nonlinear(lfem_pattern_t p, const double* coords, const lfem_quad* quad,
                                        const double* u, double* out, void* cuda_stream) {
  return vectors_common(p, coords, 3, quad, u, out, 1, (cudaStream_t)cuda_stream);
}

lfem_status lfem_mixed_fallback_count(lfem_pattern_t p, void* cuda_stream, int64_t* n_fp64_elements) {
  if (!p || !n_fp64_elements) return fail(LFEM_E_ARG, "NULL argument");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  unsigned long long h = 0;
  LFEM_CUDA(cudaMemcpyAsync(&h, p->d.status + 2, sizeof(h), cudaMemcpyDeviceToHost, st));
  LFEM_CUDA(cudaStreamSynchronize(st));
  *n_fp64_elements = (int64_t)h;
  return LFEM_OK;
}

static std::string tune_key(lfem_pattern_t p, int ambient, const lfem_quad* quad, lfem_precision prec, unsigned which) {
  cudaDeviceProp prop;
  std::string name = "gpu";
  if (cudaGetDeviceProperties(&prop, p->device) == cudaSuccess) name = prop.name;
  for (auto& c : name)
    if (c == ' ') c = '_';
  int bucket = 0;
  for (int64_t n = p->n_elem; n > 1; n >>= 1) ++bucket;
  std::ostringstream k;
  k << "d" << p->dim << "_n" << ambient << "_p" << p->order << "_q" << quad->n_pts << "_prec" << (int)prec << "_w"
    << which << "_e2^" << bucket << "_" << name;
  return k.str();
}

lfem_status lfem_autotune(lfem_pattern_t p, const double* coords, int ambient, const lfem_quad* quad, const void* coef,
                          int coef_is_fp32, unsigned which, lfem_precision prec, void* M, void* A, void* MC,
                          const char* cache_path, void* cuda_stream, int32_t* best_slots) {
  if (!p) return fail(LFEM_E_ARG, "NULL argument");
  if (!quad && (which & LFEM_CMASS)) return fail(LFEM_E_ARG, "LFEM_CMASS needs a quadrature rule");
  quad = resolve_rule(quad, p->dim, p->order);
  if (!quad) return fail(LFEM_E_ARG, "quadrature rule missing");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const std::string key = tune_key(p, ambient, quad, prec, which);
  int best = 0;
  if (cache_path) {
    std::ifstream in(cache_path);
    std::string k;
    int v;
    while (in >> k >> v)
      if (k == key) best = v;
  }
  if (!best) {
    // finer steps around the capacities where a tile's elements still fit one
    // phase-1 round of the mixed kernel and two CTAs share an SM
    const int cand[] = {512, 1024, 1536, 2048, 2304, 2560, 2816, 3072, 3328, 3584, 4096, 6144, 8192};
    float best_ms = 1e30f;
    cudaEvent_t e0, e1;
    LFEM_CUDA(cudaEventCreate(&e0));
    LFEM_CUDA(cudaEventCreate(&e1));
    for (int c : cand) {
      if (c < p->max_row) continue;
      if (build_tiles(p, c, st) != LFEM_OK) continue;
      // one warm-up; configurations whose shared memory does not fit are skipped
      if (lfem_assemble(p, coords, ambient, quad, coef, coef_is_fp32, which, prec, M, A, MC, st) != LFEM_OK) continue;
      LFEM_CUDA(cudaEventRecord(e0, st));
      const int reps = 3;
      for (int r = 0; r < reps; ++r) {
        lfem_status s = lfem_assemble(p, coords, ambient, quad, coef, coef_is_fp32, which, prec, M, A, MC, st);
        if (s != LFEM_OK) return s;
      }
      LFEM_CUDA(cudaEventRecord(e1, st));
      LFEM_CUDA(cudaEventSynchronize(e1));
      float ms = 0.f;
      LFEM_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      if (ms < best_ms) {
        best_ms = ms;
        best = c;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!best) return fail(LFEM_E_TOO_LARGE, "no tile capacity fits this configuration");
    if (cache_path) {
      std::ofstream out(cache_path, std::ios::app);
      out << key << " " << best << "\n";
    }
  }
  if (p->tile_slots != best) {
    lfem_status s = build_tiles(p, best, st);
    if (s != LFEM_OK) return s;
  }
  LFEM_CUDA(cudaStreamSynchronize(st));
  if (best_slots) *best_slots = best;
  return LFEM_OK;
}

}  // extern "C"

