// Batched assembly: one persistent launch over the row tiles of many meshes
// (the batchwise processing of Sec. 3.3, Remark "Batch computations", done as
// a single work list on the GPU), optionally captured once into a CUDA graph
// and replayed.
#include <algorithm>
#include <cstring>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>

#include "dispatch.cuh"

namespace lfem {

#define TRY_STATUS(x)                   \
  do {                                  \
    lfem_status _s = (x);               \
    if (_s != LFEM_OK) return _s;       \
  } while (0)

__global__ void k_set_item_mesh(ItemRef* refs, int64_t n, int mesh) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) refs[t].mesh = mesh;
}

static bool batch_type_ok(int d, int na) { return (d == 1 && na == 2) || (d == 2 && (na == 2 || na == 3)); }

lfem_status bank_upload_batch(const void* src, size_t bytes, size_t offset) {
  LFEM_CUDA(cudaMemcpyToSymbol(c_bank, src, bytes, offset, cudaMemcpyHostToDevice));
  return LFEM_OK;
}

}  // namespace lfem

using namespace lfem;

struct lfem_batch_s {
  int device = 0;
  PipeArgs args{};
  MeshRec* d_meshes = nullptr;
  ItemRef* d_items = nullptr;
  int32_t* d_status = nullptr;  // [0] status bits, [2..3] fallback count, [4..5] tile tickets
  int ent_bytes = 2;
  int64_t n_elements = 0;
  FastBank fb{};  // compile-time-rule tables, one per (dim, order)
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  // orders 3, 4: assembled by their element-major path on the batch's stream,
  // after the persistent launch (and captured with it); rule copied here
  struct Side {
    lfem_pattern_s* p;
    const double* coords;
    int ambient;
    std::vector<double> xi, w;
    lfem_quad quad;
    const void* coef;
    void* M;
    void* A;
    void* MC;
  };
  std::vector<Side> side;
  // runs of the work list with one element type (the list is sorted by
  // family), each launched as its own persistent single-type kernel with the
  // shared-memory caps of its meshes: one kernel over every type spills
  struct Seg {
    int dim, na, order;
    bool fast;
    PipeArgs args;
  };
  std::vector<Seg> segs;
  unsigned which = 0;
  int coef_f32 = 0;
};

static lfem_status batch_launch(lfem_batch_s* b, cudaStream_t st) {
  int sms = 0;
  LFEM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device));
  LFEM_CUDA(cudaMemsetAsync(b->d_status + 2, 0, sizeof(unsigned long long), st));
  for (const auto& g : b->segs) {
    LFEM_CUDA(cudaMemsetAsync(b->d_status + 4, 0, sizeof(unsigned long long), st));  // tile tickets
    const lfem_status s = g.dim == 1 ? run_pipe_d1(g.na, g.order, true, g.args, b->ent_bytes, g.fast, b->fb, sms, st)
                                     : run_pipe_d2(g.na, g.order, true, g.args, b->ent_bytes, g.fast, b->fb, sms, st);
    if (s != LFEM_OK) return s;
  }
  for (auto& sd : b->side) {
    const lfem_status s = lfem_assemble(sd.p, sd.coords, sd.ambient, &sd.quad, sd.coef, b->coef_f32, b->which,
                                        LFEM_MIXED, sd.M, sd.A, sd.MC, st);
    if (s != LFEM_OK) return s;
  }
  return LFEM_OK;
}

extern "C" {

lfem_status lfem_batch_create(const lfem_batch_item* items_in, int n_items, unsigned which, int coef_is_fp32,
                              void* cuda_stream, lfem_batch_t* out) {
  if (!out || !items_in || n_items <= 0) return fail(LFEM_E_ARG, "batch arguments");
  *out = nullptr;
  // items without a rule: order 1 takes the exact rule, anything else is an error
  std::vector<lfem_batch_item> items_v(items_in, items_in + n_items);
  for (auto& it : items_v) {
    if (it.quad || !it.pattern) continue;
    if (it.pattern->order != 1 || (which & LFEM_CMASS)) return fail(LFEM_E_ARG, "batch item without a quadrature rule");
    it.quad = exact_p1_rule(it.pattern->dim);
  }
  if (which == 0 || (which & ~7u)) return fail(LFEM_E_ARG, "which");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  // orders 3, 4 run beside the persistent launch: check them, register their
  // rule and reserve their element buffer now (nothing allocates in a launch)
  std::vector<lfem_batch_item> pipe_v;
  std::vector<lfem_batch_s::Side> side_v;
  int nm_all = 0;
  for (unsigned bit = 1; bit <= 4; bit <<= 1) nm_all += (which & bit) ? 1 : 0;
  for (const auto& it : items_v) {
    lfem_pattern_s* p = it.pattern;
    if (!p) return fail(LFEM_E_ARG, "batch item without pattern");
    if (p->order <= 2) {
      pipe_v.push_back(it);
      continue;
    }
    if (!supported(p->dim, it.ambient, p->order) || !batch_type_ok(p->dim, it.ambient))
      return fail(LFEM_E_UNSUPPORTED, "element type not supported in batches");
    if ((which & LFEM_MASS) && !it.M) return fail(LFEM_E_ARG, "batch item M is NULL");
    if ((which & LFEM_STIFF) && !it.A) return fail(LFEM_E_ARG, "batch item A is NULL");
    if ((which & LFEM_CMASS) && (!it.MC || !it.coef)) return fail(LFEM_E_ARG, "batch item MC or coef is NULL");
    if (p->n_elem > 0 && !it.coords) return fail(LFEM_E_ARG, "batch item coords is NULL");
    lfem_batch_s::Side sd{p, it.coords, it.ambient, {}, {}, {}, it.coef, it.M, it.A, it.MC};
    sd.xi.assign(it.quad->xi, it.quad->xi + (size_t)it.quad->n_pts * p->dim);
    sd.w.assign(it.quad->w, it.quad->w + it.quad->n_pts);
    TabRef tab;
    lfem_status s = get_tables(p->dim, p->order, it.quad, st, &tab);
    if (s != LFEM_OK) return s;
    if ((s = reserve_elem_buf(p, nm_all, true, tab.q)) != LFEM_OK) return s;
    side_v.push_back(std::move(sd));
  }
  // the work list holds the meshes family by family (dim, order, ambient), so
  // neighbouring CTAs run the same element code (one type's phase 1 at a time
  // in the instruction cache); every tile owns its rows, so the order changes
  // no result
  std::stable_sort(pipe_v.begin(), pipe_v.end(), [](const lfem_batch_item& x, const lfem_batch_item& y) {
    const int kx = (x.pattern->dim * 8 + x.pattern->order) * 4 + x.ambient;
    const int ky = (y.pattern->dim * 8 + y.pattern->order) * 4 + y.ambient;
    return kx < ky;
  });
  const lfem_batch_item* items = pipe_v.data();
  n_items = (int)pipe_v.size();
  std::vector<MeshRec> recs(n_items);
  std::vector<int64_t> item_off(n_items + 1, 0);  // first work item of each mesh
  int cap_front = 0, cap_back = 0, cap_nodes = 0, cap_nel = 0, max_u = 0, max_q = 0, ent_bytes = 2;
  int64_t cap_lsm = 0;
  int64_t n_el = 0;
  int vec_out = 1;
  int nm = 0;
  for (unsigned bit = 1; bit <= 4; bit <<= 1) nm += (which & bit) ? 1 : 0;
  for (int i = 0; i < n_items; ++i) {
    const lfem_batch_item& it = items[i];
    lfem_pattern_s* p = it.pattern;
    if (!p) return fail(LFEM_E_ARG, "batch item without pattern");
    if (!supported(p->dim, it.ambient, p->order) || !batch_type_ok(p->dim, it.ambient))
      return fail(LFEM_E_UNSUPPORTED, "element type not supported in batches");
    if ((which & LFEM_MASS) && !it.M) return fail(LFEM_E_ARG, "batch item M is NULL");
    if ((which & LFEM_STIFF) && !it.A) return fail(LFEM_E_ARG, "batch item A is NULL");
    if ((which & LFEM_CMASS) && (!it.MC || !it.coef)) return fail(LFEM_E_ARG, "batch item MC or coef is NULL");
    if (p->n_elem > 0 && !it.coords) return fail(LFEM_E_ARG, "batch item coords is NULL");
    ent_bytes = std::max(ent_bytes, p->ent_bytes);
  }
  // all blocks of a batch are read with one entry width: widen where needed
  for (int i = 0; i < n_items; ++i) {
    lfem_pattern_s* p = items[i].pattern;
    if (p->ent_bytes != ent_bytes) {
      p->min_ent_bytes = ent_bytes;
      lfem_status s = build_tiles(p, p->tile_slots, st);
      if (s != LFEM_OK) return s;
    }
  }
  for (int i = 0; i < n_items; ++i) {
    const lfem_batch_item& it = items[i];
    lfem_pattern_s* p = it.pattern;
    TabRef tab;
    lfem_status s = get_tables(p->dim, p->order, it.quad, st, &tab);
    if (s != LFEM_OK) return s;
    MeshRec& r = recs[i];
    r.coords = it.coords;
    r.coef = it.coef;
    int m = 0;
    if (which & LFEM_MASS) r.out[m++] = it.M;
    if (which & LFEM_STIFF) r.out[m++] = it.A;
    if (which & LFEM_CMASS) r.out[m++] = it.MC;
    for (int k = 0; k < m; ++k)
      if (reinterpret_cast<uintptr_t>(r.out[k]) % 16) vec_out = 0;
    r.tab = tab;
    r.type = elem_type_id(p->dim, it.ambient, p->order);
    r.na = it.ambient;
    r.ref = p->ref;
    r.entb = p->ent_bytes;
    r.coef_f32 = coef_is_fp32 ? 1 : 0;
    r.c16 = reinterpret_cast<uintptr_t>(it.coords) % 16 == 0 ? 1 : 0;
    cap_front = std::max(cap_front, p->max_tile_front);
    cap_back = std::max(cap_back, p->max_tile_back);
    cap_nodes = std::max(cap_nodes, p->max_tile_nodes);
    cap_nel = std::max(cap_nel, p->max_tile_nel);
    max_u = std::max(max_u, n_upper(p->ref));
    cap_lsm = std::max(cap_lsm, lsm_words(p->max_tile_nel, n_upper(p->ref), p->max_tile_nl));
    max_q = std::max(max_q, tab.q);
    n_el += p->tile_elems_total;
    item_off[i + 1] = item_off[i] + p->n_tiles;
  }
  lfem_batch_s* b = new lfem_batch_s();
  cudaGetDevice(&b->device);
  // compile-time rules: an item runs the compile-time variant of its type when
  // its rule has the fixed size and the same points and weights as the first
  // such item of its (dim, order) (one table per (dim, order) in the launch)
  {
    bool seen[2][2] = {{false, false}, {false, false}};
    std::vector<float> tab;
    for (int i = 0; i < n_items; ++i) {
      const lfem_pattern_s* p = items[i].pattern;
      const int d = p->dim, o = p->order;
      const int off = d == 1 ? (o == 1 ? FastBank::OFF11 : FastBank::OFF12) : (o == 1 ? FastBank::OFF21 : FastBank::OFF22);
      const int size = fast_table_size(d, o);
      tab.assign(size, 0.f);
      bool fast = fast_tables_host(d, o, items[i].quad, tab.data());
      if (fast && seen[d - 1][o - 1]) {
        fast = memcmp(tab.data(), b->fb.v + off, sizeof(float) * size) == 0;
      } else if (fast) {
        memcpy(b->fb.v + off, tab.data(), sizeof(float) * size);
        seen[d - 1][o - 1] = true;
      }
      if (fast) recs[i].type += kFastTypeOffset;
    }
  }
  b->ent_bytes = ent_bytes;
  b->n_elements = n_el;
  b->which = which;
  b->coef_f32 = coef_is_fp32 ? 1 : 0;
  for (auto& sd : side_v) {
    b->n_elements += sd.p->n_elem;
    b->side.push_back(std::move(sd));
  }
  for (auto& sd : b->side) sd.quad = lfem_quad{(int)sd.w.size(), sd.xi.data(), sd.w.data()};
  auto cleanup = [&]() {
    if (b->d_meshes) cudaFree(b->d_meshes);
    if (b->d_items) cudaFree(b->d_items);
    if (b->d_status) cudaFree(b->d_status);
    delete b;
  };
  if (dev_malloc((void**)&b->d_meshes, sizeof(MeshRec) * std::max(1, n_items)) != cudaSuccess ||
      dev_malloc((void**)&b->d_items, sizeof(ItemRef) * std::max<int64_t>(1, item_off[n_items])) != cudaSuccess ||
      dev_malloc((void**)&b->d_status, 6 * sizeof(int32_t)) != cudaSuccess) {
    cudaGetLastError();
    cleanup();
    return fail(LFEM_E_NOMEM, "batch allocation failed");
  }
  if (n_items > 0) cudaMemcpyAsync(b->d_meshes, recs.data(), sizeof(MeshRec) * n_items, cudaMemcpyHostToDevice, st);
  // work items: every mesh's tile records, mesh by mesh, tagged with the mesh index
  for (int i = 0; i < n_items; ++i) {
    const int64_t n = item_off[i + 1] - item_off[i];
    if (n == 0) continue;
    cudaMemcpyAsync(b->d_items + item_off[i], items[i].pattern->d.tile_refs, sizeof(ItemRef) * n,
                    cudaMemcpyDeviceToDevice, st);
    k_set_item_mesh<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(b->d_items + item_off[i], n, i);
  }
  cudaMemsetAsync(b->d_status, 0, 6 * sizeof(int32_t), st);
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cleanup();
    return cuda_fail(e, "batch upload");
  }
  PipeArgs& a = b->args;
  a.meshes = b->d_meshes;
  a.items = b->d_items;
  a.n_items = item_off[n_items];
  a.nm = nm;
  a.which = which;
  a.chunk = PipeOcc<float>::THREADS / kPipeTPE;
  a.cap_front = cap_front;
  a.cap_back = cap_back;
  a.cap_nodes = cap_nodes;
  a.cap_nel = cap_nel;
  a.max_u = max_u;
  a.cap_lsm = cap_lsm;
  a.vec_out = vec_out;
  a.max_q = max_q;
  a.coef_bytes = (which & LFEM_CMASS) ? (coef_is_fp32 ? 4 : 8) : 0;
  a.coef_smem = 0;  // staged only for general-rule items
  for (int i = 0; i < n_items; ++i)
    if (recs[i].type < kFastTypeOffset) a.coef_smem = a.coef_bytes;
  a.qmin = 0.0f;
  for (int i = 0; i < n_items; ++i) a.qmin = std::max(a.qmin, items[i].pattern->qmin);
  a.status = b->d_status;
  a.fallback = reinterpret_cast<unsigned long long*>(b->d_status + 2);
  a.next_item = reinterpret_cast<unsigned int*>(b->d_status + 4);
  a.starve = 0;
  a.wait_ns = 2000000000ll;
  for (int i = 0; i < n_items;) {
    int j = i;
    while (j < n_items && recs[j].type == recs[i].type) ++j;
    lfem_batch_s::Seg g{items[i].pattern->dim, items[i].ambient, items[i].pattern->order,
                        recs[i].type >= kFastTypeOffset, a};
    PipeArgs& sa = g.args;
    sa.items = b->d_items + item_off[i];
    sa.n_items = item_off[j] - item_off[i];
    sa.cap_front = sa.cap_back = sa.cap_nodes = sa.cap_nel = sa.max_u = sa.max_q = 0;
    sa.cap_lsm = 0;
    sa.qmin = 0.0f;
    for (int k = i; k < j; ++k) {
      const lfem_pattern_s* p = items[k].pattern;
      sa.cap_front = std::max(sa.cap_front, p->max_tile_front);
      sa.cap_back = std::max(sa.cap_back, p->max_tile_back);
      sa.cap_nodes = std::max(sa.cap_nodes, p->max_tile_nodes);
      sa.cap_nel = std::max(sa.cap_nel, p->max_tile_nel);
      sa.max_u = std::max(sa.max_u, n_upper(p->ref));
      sa.cap_lsm = std::max(sa.cap_lsm, lsm_words(p->max_tile_nel, n_upper(p->ref), p->max_tile_nl));
      sa.max_q = std::max(sa.max_q, recs[k].tab.q);
      sa.qmin = std::max(sa.qmin, p->qmin);
    }
    sa.coef_smem = g.fast ? 0 : a.coef_bytes;
    if (pipe_smem_bytes<float>(sa) > 227 * 1024) {
      cleanup();
      return fail(LFEM_E_TOO_LARGE, "largest tile of the batch needs more than 227 KB of shared memory");
    }
    if (sa.n_items > 0) b->segs.push_back(g);
    i = j;
  }
  *out = b;
  return LFEM_OK;
}

lfem_status lfem_batch_assemble(lfem_batch_t b, void* cuda_stream) {
  if (!b) return fail(LFEM_E_ARG, "batch is NULL");
  return batch_launch(b, (cudaStream_t)cuda_stream);
}

lfem_status lfem_batch_graph_launch(lfem_batch_t b, void* cuda_stream) {
  if (!b) return fail(LFEM_E_ARG, "batch is NULL");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  if (!b->exec) {
    if (!st) return fail(LFEM_E_ARG, "graph capture needs a non-default stream");
    LFEM_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    lfem_status s = batch_launch(b, st);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(st, &g);
    if (s != LFEM_OK) {
      if (g) cudaGraphDestroy(g);
      return s;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&b->exec, g, 0);
    if (e != cudaSuccess) {
      cudaGraphDestroy(g);
      return cuda_fail(e, "cudaGraphInstantiate");
    }
    b->graph = g;
  }
  LFEM_CUDA(cudaGraphLaunch(b->exec, st));
  return LFEM_OK;
}

lfem_status lfem_batch_sync_status(lfem_batch_t b, void* cuda_stream) {
  if (!b) return fail(LFEM_E_ARG, "batch is NULL");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int32_t h = 0;
  LFEM_CUDA(cudaMemcpyAsync(&h, b->d_status, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  LFEM_CUDA(cudaMemsetAsync(b->d_status, 0, sizeof(int32_t), st));
  LFEM_CUDA(cudaStreamSynchronize(st));
  if (h & ST_TIMEOUT) return fail(LFEM_E_TIMEOUT, "a bounded device wait ran out");
  if (h & ST_ITEM) return fail(LFEM_E_CUDA, "a work-item record failed its size or alignment check");
  if (h & ST_TYPE) return fail(LFEM_E_UNSUPPORTED, "a tile met a kernel without its element type");
  if (h & ST_DEGENERATE) return fail(LFEM_E_DEGENERATE, "zero or non-finite |det DF| at a quadrature point");
  for (auto& sd : b->side) {
    const lfem_status s = lfem_sync_status(sd.p, cuda_stream);
    if (s != LFEM_OK) return s;
  }
  return LFEM_OK;
}

lfem_status lfem_batch_info(lfem_batch_t b, int64_t* n_work_items, int64_t* n_elements, int32_t* cap_elements) {
  if (!b) return fail(LFEM_E_ARG, "batch is NULL");
  if (n_work_items) *n_work_items = b->args.n_items;
  if (n_elements) *n_elements = b->n_elements;
  if (cap_elements) *cap_elements = b->args.cap_nel;
  return LFEM_OK;
}

void lfem_batch_destroy(lfem_batch_t b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->d_meshes) cudaFree(b->d_meshes);
  if (b->d_items) cudaFree(b->d_items);
  if (b->d_status) cudaFree(b->d_status);
  delete b;
}

lfem_status lfem_batch_autotune(const lfem_batch_item* items, int n_items, unsigned which, int coef_is_fp32,
                                const char* cache_path, void* cuda_stream, int32_t* best_slots) {
  if (!items || n_items <= 0) return fail(LFEM_E_ARG, "batch arguments");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  // the distinct patterns of each element family: (dim, order) = curves P1,
  // curves P2, triangles P1, triangles P2 (a P1 triangle tile holds about six
  // times the elements of a P2 one of the same capacity)
  std::vector<lfem_pattern_s*> fam[4];
  int64_t n_el = 0;
  int counts[3][4][3] = {};  // (dim, ambient, order) histogram for the cache key
  for (int i = 0; i < n_items; ++i) {
    lfem_pattern_s* p = items[i].pattern;
    if (!p) return fail(LFEM_E_ARG, "batch item without pattern");
    if (!batch_type_ok(p->dim, items[i].ambient))
      return fail(LFEM_E_UNSUPPORTED, "element type not supported in batches");
    if (p->order > 2) continue;  // element-major, no row tiles to tune
    auto& v = fam[2 * (p->dim - 1) + (p->order - 1)];
    if (std::find(v.begin(), v.end(), p) == v.end()) v.push_back(p);
    n_el += p->n_elem;
    ++counts[p->dim][items[i].ambient][p->order];
  }
  std::string name = "gpu";
  {
    int dev = 0;
    cudaDeviceProp prop;
    if (cudaGetDevice(&dev) == cudaSuccess && cudaGetDeviceProperties(&prop, dev) == cudaSuccess) name = prop.name;
    for (auto& c : name)
      if (c == ' ') c = '_';
  }
  int bucket = 0;
  for (int64_t n = n_el; n > 1; n >>= 1) ++bucket;
  std::ostringstream k;
  k << "batch_w" << which << "_f" << coef_is_fp32;
  for (int d = 1; d <= 2; ++d)
    for (int a = 2; a <= 3; ++a)
      for (int o = 1; o <= 2; ++o)
        if (counts[d][a][o]) k << "_d" << d << "n" << a << "p" << o << "x" << counts[d][a][o];
  k << "_e2^" << bucket << "_" << name;
  const std::string key = k.str();
  int best[4] = {0, 0, 0, 0};
  bool cached = false;
  if (cache_path) {
    std::ifstream in(cache_path);
    std::string kk;
    int v[4];
    while (in >> kk >> v[0] >> v[1] >> v[2] >> v[3])
      if (kk == key) {
        for (int f = 0; f < 4; ++f) best[f] = v[f];
        cached = true;
      }
  }
  auto retile = [&](int f, int slots) -> lfem_status {
    for (lfem_pattern_s* p : fam[f])
      if (p->tile_slots != slots) {
        lfem_status s = build_tiles(p, std::max(slots, (int)p->max_row), st);
        if (s != LFEM_OK) return s;
      }
    return LFEM_OK;
  };
  if (!cached) {
    // one family at a time (P2 triangles first: they carry most of the work),
    // the others held at their current (or already tuned) capacities; a
    // candidate whose launch does not fit is skipped
    const int cand[] = {1024, 1536, 2048, 2304, 2560, 3072};
    cudaEvent_t e0, e1;
    LFEM_CUDA(cudaEventCreate(&e0));
    LFEM_CUDA(cudaEventCreate(&e1));
    for (int f : {3, 2, 1, 0}) {
      if (fam[f].empty()) continue;
      float best_ms = 1e30f;
      for (int c : cand) {
        if (retile(f, c) != LFEM_OK) continue;
        lfem_batch_t b = nullptr;
        if (lfem_batch_create(items, n_items, which, coef_is_fp32, cuda_stream, &b) != LFEM_OK) continue;
        lfem_status s = lfem_batch_assemble(b, cuda_stream);  // warm-up
        if (s == LFEM_OK) s = lfem_batch_sync_status(b, cuda_stream);
        if (s != LFEM_OK) {
          lfem_batch_destroy(b);
          continue;
        }
        const int reps = 3;
        cudaEventRecord(e0, st);
        for (int r = 0; r < reps && s == LFEM_OK; ++r) s = lfem_batch_assemble(b, cuda_stream);
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (s == LFEM_OK) s = lfem_batch_sync_status(b, cuda_stream);
        lfem_batch_destroy(b);
        if (s == LFEM_OK && ms < best_ms) {
          best_ms = ms;
          best[f] = c;
        }
      }
      if (!best[f]) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return fail(LFEM_E_TOO_LARGE, "no tile capacity fits this batch");
      }
      TRY_STATUS(retile(f, best[f]));
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (cache_path) {
      std::ofstream out(cache_path, std::ios::app);
      out << key << " " << best[0] << " " << best[1] << " " << best[2] << " " << best[3] << "\n";
    }
  } else {
    for (int f = 0; f < 4; ++f)
      if (!fam[f].empty() && best[f]) TRY_STATUS(retile(f, best[f]));
  }
  LFEM_CUDA(cudaStreamSynchronize(st));
  if (best_slots)
    for (int f = 0; f < 4; ++f) best_slots[f] = best[f];
  return LFEM_OK;
}

}  // extern "C"
