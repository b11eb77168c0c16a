// Pattern builder (once per topology): integer sort / unique of the element
// index pairs (E[e,a], E[e,b]) into CSR, plus the maps the assembly kernels
// use.  All integer work; the CSR pattern and every contribution list are
// bit-exact and independent of thread scheduling (atomics only count, every
// list is sorted before use).  The one exception is the order of a tile's
// long-slot work list, which atomics hand out; it decides which thread sums a
// slot, never how.
//
// This replaces the per-assembly sort inside sparse(I, J, V) (Sec. 3.3: the
// log-linear cost comes from sorting and merging duplicates; precomputing the
// sparsity structure removes it from the assembly).
#include <algorithm>
#include <climits>
#include <cstdio>
#include <mutex>
#include <vector>

#include "lfem_internal.cuh"

namespace lfem {

// ----------------------------------------------------------------------------
// Exclusive scan (3 phases, recursive on block sums).
// ----------------------------------------------------------------------------
constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

template <typename TI, typename TO>
__global__ void k_scan_tiles(const TI* __restrict__ in, TO* __restrict__ out, int64_t n, TO* __restrict__ tile_sums) {
  __shared__ TO warp_tot[kScanThreads / 32];
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  TO v[kScanItems];
  TO run = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    TO x = (base + i < n) ? (TO)in[base + i] : (TO)0;
    v[i] = run;
    run += x;
  }
  // inclusive scan of per-thread totals within the block
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  TO t = run;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    TO y = __shfl_up_sync(0xffffffffu, t, o);
    if (lane >= o) t += y;
  }
  if (lane == 31) warp_tot[wid] = t;
  __syncthreads();
  if (wid == 0) {
    TO w = (lane < kScanThreads / 32) ? warp_tot[lane] : (TO)0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      TO y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < kScanThreads / 32) warp_tot[lane] = w;
  }
  __syncthreads();
  TO excl = t - run + (wid > 0 ? warp_tot[wid - 1] : (TO)0);
#pragma unroll
  for (int i = 0; i < kScanItems; ++i)
    if (base + i < n) out[base + i] = v[i] + excl;
  if (threadIdx.x == kScanThreads - 1) tile_sums[blockIdx.x] = excl + run;
}

template <typename TO>
__global__ void k_scan_add(TO* __restrict__ out, int64_t n, const TO* __restrict__ tile_off) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] += tile_off[i / kScanTile];
}

// out[0..n] = exclusive scan of in[0..n) with out[n] = total.  `scratch` needs
// scan_scratch_elems(n) elements of TO.
inline int64_t scan_scratch_elems(int64_t n) {
  int64_t tot = 0;
  int64_t m = n + 1;
  while (true) {
    int64_t tiles = (m + kScanTile - 1) / kScanTile;
    tot += tiles;
    if (tiles <= 1) break;
    m = tiles;
  }
  return tot + 8;
}

template <typename TI, typename TO>
void scan_exclusive(const TI* in, TO* out, int64_t n, TO* scratch, cudaStream_t st) {
  // treat the input as n+1 items with a trailing zero so out[n] is the total
  int64_t m = n + 1;
  int64_t tiles = (m + kScanTile - 1) / kScanTile;
  TO* sums = scratch;
  // in[n] is out of range: scan n items then write the total from the tile sums
  k_scan_tiles<TI, TO><<<(unsigned)tiles, kScanThreads, 0, st>>>(in, out, n, sums);
  if (tiles > 1) {
    TO* sums_scanned = scratch + tiles;
    scan_exclusive<TO, TO>(sums, sums_scanned, tiles, scratch + 2 * tiles + 1, st);
    k_scan_add<TO><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(out, n, sums_scanned);
    cudaMemcpyAsync(out + n, sums_scanned + tiles, sizeof(TO), cudaMemcpyDeviceToDevice, st);
  } else {
    cudaMemcpyAsync(out + n, sums, sizeof(TO), cudaMemcpyDeviceToDevice, st);
  }
}

static int64_t scan_scratch_bytes(int64_t n, size_t elem) {
  // generous: 3 levels of tile sums plus recursion
  int64_t t = (n + 1 + kScanTile - 1) / kScanTile;
  return (4 * t + 64) * (int64_t)elem;
}

// ----------------------------------------------------------------------------
// Segmented sort of int32 keys: segment i is [off[i]*scale, off[i+1]*scale).
// Bitonic networks in shared memory: a warp per segment up to 1024 keys, a
// block per segment up to kMaxSegSort keys.
// ----------------------------------------------------------------------------
template <bool BLOCK>
__device__ void bitonic_smem(int32_t* s, int n, int tid, int nthr) {
  for (int k = 2; k <= n; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = tid; i < n; i += nthr) {
        int ixj = i ^ j;
        if (ixj > i) {
          int32_t a = s[i], b = s[ixj];
          bool up = (i & k) == 0;
          if ((a > b) == up) {
            s[i] = b;
            s[ixj] = a;
          }
        }
      }
      if (BLOCK) __syncthreads();
      else __syncwarp();
    }
  }
}

__device__ __forceinline__ int next_pow2(int n) {
  int p = 1;
  while (p < n) p <<= 1;
  return p;
}

constexpr int kWarpSegMax = 1024;
constexpr int kSegWarps = 4;

__global__ void k_segsort_warp(int32_t* __restrict__ keys, const int32_t* __restrict__ off, int64_t nseg, int scale,
                               int32_t* __restrict__ long_list, int32_t* __restrict__ long_count) {
  __shared__ int32_t buf[kSegWarps][kWarpSegMax];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t seg = (int64_t)blockIdx.x * kSegWarps + w;
  if (seg >= nseg) return;
  const int64_t b = (int64_t)off[seg] * scale, e = (int64_t)off[seg + 1] * scale;
  const int len = (int)(e - b);
  if (len <= 1) return;
  if (len > kWarpSegMax) {
    if (lane == 0) long_list[atomicAdd(long_count, 1)] = (int32_t)seg;
    return;
  }
  const int n = next_pow2(len);
  for (int i = lane; i < n; i += 32) buf[w][i] = i < len ? keys[b + i] : INT_MAX;
  __syncwarp();
  bitonic_smem<false>(buf[w], n, lane, 32);
  for (int i = lane; i < len; i += 32) keys[b + i] = buf[w][i];
}

__global__ void k_segsort_block(int32_t* __restrict__ keys, const int32_t* __restrict__ off, int scale,
                                const int32_t* __restrict__ long_list) {
  extern __shared__ int32_t sbuf[];
  const int32_t seg = long_list[blockIdx.x];
  const int64_t b = (int64_t)off[seg] * scale, e = (int64_t)off[seg + 1] * scale;
  const int len = (int)(e - b);
  const int n = next_pow2(len);
  for (int i = threadIdx.x; i < n; i += blockDim.x) sbuf[i] = i < len ? keys[b + i] : INT_MAX;
  __syncthreads();
  bitonic_smem<true>(sbuf, n, threadIdx.x, blockDim.x);
  for (int i = threadIdx.x; i < len; i += blockDim.x) keys[b + i] = sbuf[i];
}

static lfem_status segsort(int32_t* keys, const int32_t* off, int64_t nseg, int scale, int max_len,
                           int32_t* scratch /* nseg + 1 ints */, cudaStream_t st) {
  if (max_len > kMaxSegSort) return fail(LFEM_E_TOO_LARGE, "segment longer than the sort limit");
  int32_t* count = scratch;
  int32_t* list = scratch + 1;
  LFEM_CUDA(cudaMemsetAsync(count, 0, sizeof(int32_t), st));
  if (nseg > 0) {
    unsigned grid = (unsigned)((nseg + kSegWarps - 1) / kSegWarps);
    k_segsort_warp<<<grid, 32 * kSegWarps, 0, st>>>(keys, off, nseg, scale, list, count);
    LFEM_CUDA(cudaGetLastError());
  }
  if (max_len > kWarpSegMax) {
    int32_t h = 0;
    LFEM_CUDA(cudaMemcpyAsync(&h, count, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    LFEM_CUDA(cudaStreamSynchronize(st));
    if (h > 0) {
      int np2 = 1;
      while (np2 < max_len) np2 <<= 1;
      size_t smem = (size_t)np2 * sizeof(int32_t);
      LFEM_CUDA(cudaFuncSetAttribute(k_segsort_block, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      k_segsort_block<<<h, 512, smem, st>>>(keys, off, scale, list);
      LFEM_CUDA(cudaGetLastError());
    }
  }
  return LFEM_OK;
}

// ----------------------------------------------------------------------------
// Pattern kernels
// ----------------------------------------------------------------------------
__global__ void k_count_degree(const int32_t* __restrict__ conn, int64_t total, int32_t n_nodes,
                               int32_t* __restrict__ deg, int32_t* __restrict__ status) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < total; k += (int64_t)gridDim.x * blockDim.x) {
    int32_t v = conn[k];
    if (v < 0 || v >= n_nodes) {
      atomicOr(status, ST_INDEX);
      continue;
    }
    atomicAdd(&deg[v], 1);
  }
}

__global__ void k_max_i32(const int32_t* __restrict__ a, int64_t n, int32_t* __restrict__ out) {
  int32_t m = 0;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    m = max(m, a[k]);
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_down_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

__global__ void k_fill_incidence(const int32_t* __restrict__ conn, int64_t n_elem, int ref, int ksh,
                                 const int32_t* __restrict__ inc_ptr, int32_t* __restrict__ cursor,
                                 int32_t* __restrict__ inc_key) {
  const int64_t total = n_elem * ref;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < total; k += (int64_t)gridDim.x * blockDim.x) {
    int32_t v = conn[k];
    int64_t e = k / ref;
    int a = (int)(k - e * ref);
    int32_t slot = inc_ptr[v] + atomicAdd(&cursor[v], 1);
    inc_key[slot] = (int32_t)((e << ksh) | a);
  }
}

__global__ void k_elem_inc_and_raw(const int32_t* __restrict__ conn, int ref, int ksh,
                                   const int32_t* __restrict__ inc_key, int64_t n_inc, int32_t* __restrict__ elem_inc,
                                   int32_t* __restrict__ raw) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n_inc; k += (int64_t)gridDim.x * blockDim.x) {
    int32_t key = inc_key[k];
    int64_t e = key >> ksh;
    int a = key & ((1 << ksh) - 1);
    elem_inc[e * ref + a] = (int32_t)k;
    for (int b = 0; b < ref; ++b) raw[k * ref + b] = conn[e * ref + b];
  }
}

__global__ void k_row_unique_count(const int32_t* __restrict__ raw, const int32_t* __restrict__ inc_ptr, int ref,
                                   int32_t n_nodes, int32_t* __restrict__ rowlen) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_nodes; i += (int64_t)gridDim.x * blockDim.x) {
    int64_t b = (int64_t)inc_ptr[i] * ref, e = (int64_t)inc_ptr[i + 1] * ref;
    int32_t cnt = 0;
    int32_t prev = -1;
    for (int64_t k = b; k < e; ++k) {
      int32_t v = raw[k];
      cnt += (v != prev);
      prev = v;
    }
    rowlen[i] = cnt;
  }
}

__global__ void k_row_compact(const int32_t* __restrict__ raw, const int32_t* __restrict__ inc_ptr, int ref,
                              int32_t n_nodes, const int64_t* __restrict__ row_ptr, int32_t* __restrict__ col_idx) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_nodes; i += (int64_t)gridDim.x * blockDim.x) {
    int64_t b = (int64_t)inc_ptr[i] * ref, e = (int64_t)inc_ptr[i + 1] * ref;
    int64_t o = row_ptr[i];
    int32_t prev = -1;
    for (int64_t k = b; k < e; ++k) {
      int32_t v = raw[k];
      if (v != prev) col_idx[o++] = v;
      prev = v;
    }
  }
}

template <typename PosT>
__global__ void k_positions(const int32_t* __restrict__ conn, int ref, int ksh, const int32_t* __restrict__ inc_key,
                            const int32_t* __restrict__ inc_ptr, int32_t n_nodes, const int64_t* __restrict__ row_ptr,
                            const int32_t* __restrict__ col_idx, PosT* __restrict__ pos) {
  // one thread per node; each incidence of the node gets the positions of its element's nodes in the row
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_nodes; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t rb = row_ptr[i], re = row_ptr[i + 1];
    for (int32_t k = inc_ptr[i]; k < inc_ptr[i + 1]; ++k) {
      int64_t e = inc_key[k] >> ksh;
      for (int b = 0; b < ref; ++b) {
        int32_t c = conn[e * ref + b];
        int64_t lo = rb, hi = re;
        while (lo < hi) {
          int64_t mid = (lo + hi) >> 1;
          if (col_idx[mid] < c) lo = mid + 1;
          else hi = mid;
        }
        pos[(int64_t)k * pos_stride(ref) + b] = (PosT)(lo - rb);
      }
    }
  }
}

// Element-major contribution lists: for every CSR slot, the (element, upper
// index) pairs that add into it, in ascending (e, a, b) order; a row's lists
// are contiguous (ref entries per incidence of the row).
template <typename PosT>
__global__ void k_slot_lists(const int32_t* __restrict__ inc_ptr, const int32_t* __restrict__ inc_key,
                             const PosT* __restrict__ inc_pos, const int64_t* __restrict__ row_ptr, int32_t n_nodes,
                             int ref, int ksh, int32_t* __restrict__ slot_off, int32_t* __restrict__ slot_ent) {
  const int U = ref * (ref + 1) / 2;
  const int ps = pos_stride(ref);
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n_nodes; r += (int64_t)gridDim.x * blockDim.x) {
    const int32_t kb = inc_ptr[r], ke = inc_ptr[r + 1];
    const int64_t s0 = row_ptr[r];
    const int len = (int)(row_ptr[r + 1] - s0);
    int32_t run = kb * ref;
    for (int j = 0; j < len; ++j) {
      slot_off[s0 + j] = run;
      for (int32_t k = kb; k < ke; ++k) {
        const int32_t key = inc_key[k];
        const int32_t e = key >> ksh;
        const int a = key & ((1 << ksh) - 1);
        for (int b = 0; b < ref; ++b) {
          if ((int)inc_pos[(int64_t)k * ps + b] != j) continue;
          const int u = a <= b ? a * ref - a * (a - 1) / 2 + (b - a) : b * ref - b * (b - 1) / 2 + (a - b);
          slot_ent[run++] = e * U + u;
        }
      }
    }
  }
}

// Per-tile element lists: sort + unique the elements of the tile's incidences;
// local index of every incidence; count.
__global__ void k_tile_elements(const int32_t* __restrict__ tile_row0, const int32_t* __restrict__ inc_ptr,
                                const int32_t* __restrict__ inc_key, int32_t* __restrict__ tmp,
                                int32_t* __restrict__ counts, uint16_t* __restrict__ inc_local) {
  __shared__ int32_t s[kMaxTileIncidences];
  __shared__ int32_t wsum[32];
  const int t = blockIdx.x;
  const int32_t i0 = inc_ptr[tile_row0[t]], i1 = inc_ptr[tile_row0[t + 1]];
  const int n = i1 - i0;
  if (n == 0) {
    if (threadIdx.x == 0) counts[t] = 0;
    return;
  }
  int np2 = 1;
  while (np2 < n) np2 <<= 1;
  for (int i = threadIdx.x; i < np2; i += blockDim.x) s[i] = i < n ? (inc_key[i0 + i] >> 4) : INT_MAX;
  __syncthreads();
  bitonic_smem<true>(s, np2, threadIdx.x, blockDim.x);
  // unique: flags -> block scan (sequential per thread chunk)
  const int per = (n + blockDim.x - 1) / blockDim.x;
  const int beg = threadIdx.x * per, end = min(n, beg + per);
  int cnt = 0;
  for (int i = beg; i < end; ++i) cnt += (i == 0 || s[i] != s[i - 1]);
  // block exclusive scan of cnt
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int x = cnt;
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int v = lane < (int)(blockDim.x >> 5) ? wsum[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += y;
    }
    wsum[lane] = v;
  }
  __syncthreads();
  int excl = x - cnt + (wid > 0 ? wsum[wid - 1] : 0);
  const int total = wsum[(blockDim.x >> 5) - 1];
  // unique values in place: write to tmp at offset i0
  for (int i = beg; i < end; ++i) {
    if (i == 0 || s[i] != s[i - 1]) tmp[i0 + excl++] = s[i];
  }
  __syncthreads();
  // local index of each incidence: binary search in tmp (unique, ascending)
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    int32_t key = inc_key[i0 + k];
    int32_t e = key >> 4;
    int lo = 0, hi = total;
    while (lo < hi) {
      int mid = (lo + hi) >> 1;
      if (tmp[i0 + mid] < e) lo = mid + 1;
      else hi = mid;
    }
    inc_local[i0 + k] = (uint16_t)((lo << 4) | (key & 15));
  }
  if (threadIdx.x == 0) counts[t] = total;
}

__global__ void k_tile_compact(const int32_t* __restrict__ tile_row0, const int32_t* __restrict__ inc_ptr,
                               const int32_t* __restrict__ tmp, const int32_t* __restrict__ tile_elem_ptr,
                               int32_t* __restrict__ tile_elem) {
  const int t = blockIdx.x;
  const int32_t i0 = inc_ptr[tile_row0[t]];
  const int32_t o = tile_elem_ptr[t], n = tile_elem_ptr[t + 1] - o;
  for (int i = threadIdx.x; i < n; i += blockDim.x) tile_elem[o + i] = tmp[i0 + i];
}

// ----------------------------------------------------------------------------
// Host orchestration
// ----------------------------------------------------------------------------
static unsigned grid_for(int64_t n, int threads) {
  int64_t g = (n + threads - 1) / threads;
  if (g > 152 * 64) g = 152 * 64;
  if (g < 1) g = 1;
  return (unsigned)g;
}

template <typename T>
static lfem_status dalloc(T** p, int64_t n) {
  *p = nullptr;
  if (n <= 0) n = 1;
  cudaError_t e = dev_malloc((void**)p, (size_t)n * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return fail(LFEM_E_NOMEM, "device allocation failed");
  }
  return LFEM_OK;
}

#define TRY(x)                          \
  do {                                  \
    lfem_status _s = (x);               \
    if (_s != LFEM_OK) return _s;       \
  } while (0)

// Distinct nodes of each tile's elements (sorted).
__global__ void k_tile_nodes(const int32_t* __restrict__ conn, int ref, const int32_t* __restrict__ tile_elem_ptr,
                             const int32_t* __restrict__ tile_elem, int32_t* __restrict__ tmp_nodes,
                             int32_t* __restrict__ n_nodes_out) {
  extern __shared__ int32_t sn[];
  __shared__ int32_t wsum[32];
  const int t = blockIdx.x;
  const int32_t e0 = tile_elem_ptr[t];
  const int nel = tile_elem_ptr[t + 1] - e0;
  const int n = nel * ref;
  int np2 = 1;
  while (np2 < n) np2 <<= 1;
  for (int i = threadIdx.x; i < np2; i += blockDim.x)
    sn[i] = i < n ? conn[(int64_t)tile_elem[e0 + i / ref] * ref + (i % ref)] : INT_MAX;
  __syncthreads();
  if (n > 1) bitonic_smem<true>(sn, np2, threadIdx.x, blockDim.x);
  const int per = (n + blockDim.x - 1) / blockDim.x;
  const int beg = threadIdx.x * per, end = min(n, beg + per);
  int cnt = 0;
  for (int i = beg; i < end; ++i) cnt += (i == 0 || sn[i] != sn[i - 1]);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int x = cnt;
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int v = lane < (int)(blockDim.x >> 5) ? wsum[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += y;
    }
    wsum[lane] = v;
  }
  __syncthreads();
  int excl = x - cnt + (wid > 0 ? wsum[wid - 1] : 0);
  const int total = wsum[(blockDim.x >> 5) - 1];
  int32_t* out = tmp_nodes + (int64_t)e0 * ref;
  for (int i = beg; i < end; ++i)
    if (i == 0 || sn[i] != sn[i - 1]) out[excl++] = sn[i];
  if (threadIdx.x == 0) n_nodes_out[t] = total;
}

// Node buffer of each tile (one thread per tile, a serial pass over its sorted
// node list): runs of consecutive node ids, with gaps of up to kRunGap nodes
// copied along, each run widened to even first node and even count (a 16-byte
// aligned bulk copy of 2- or 3-component double coordinates); a run that
// would end past the mesh's last node N-1 stops one short and N-1 becomes an
// extra, copied on its own.  Per distinct node its buffer position; per tile
// the counts and the block's part sizes.
__global__ void k_tile_runs(const int32_t* __restrict__ tmp_nodes, const int32_t* __restrict__ n_nodes,
                            const int32_t* __restrict__ tile_elem_ptr, int ref, int32_t N,
                            const int32_t* __restrict__ tile_row0, const int64_t* __restrict__ row_ptr,
                            const int32_t* __restrict__ nl_in, const int32_t* __restrict__ nle_in, int entb, int64_t T,
                            int4* __restrict__ runs_tmp, int2* __restrict__ extras_tmp, int32_t* __restrict__ pos_tmp,
                            int32_t* __restrict__ nruns_out, int32_t* __restrict__ nextra_out,
                            int32_t* __restrict__ nbuf_out, int64_t* __restrict__ bytes_out,
                            int32_t* __restrict__ front_out) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= T) return;
  const int64_t base = (int64_t)tile_elem_ptr[t] * ref;
  const int32_t* tn = tmp_nodes + base;
  int32_t* pos = pos_tmp + base;
  int4* runs = runs_tmp + base;
  int2* extras = extras_tmp + base;
  const int nn = n_nodes[t];
  int nr = 0, nx = 0, P = 0;
  int x_node = -1, x_idx = -1;  // at most one extra: node N - 1
  int i = 0;
  while (i < nn) {
    const int a = tn[i] & ~1;
    int end = tn[i] + 1, j = i + 1;
    while (j < nn && tn[j] - end <= kRunGap) end = tn[j++] + 1;
    int b = (end + 1) & ~1;
    if (b > N) b -= 2;  // end == N, N odd: N - 1 is left out of the run
    if (b > a) {
      runs[nr++] = make_int4(a, b - a, P, 0);
      for (int k = i; k < j; ++k)
        if (tn[k] < b) pos[k] = P + (tn[k] - a);
      P += b - a;
    }
    for (int k = i; k < j; ++k)
      if (tn[k] >= b) {
        x_node = tn[k];
        x_idx = k;
      }
    i = j;
  }
  if (x_idx >= 0) {
    extras[nx++] = make_int2(x_node, P);
    pos[x_idx] = P;
  }
  const int nbuf = P + nx;
  nruns_out[t] = nr;
  nextra_out[t] = nx;
  nbuf_out[t] = nbuf;
  const int32_t nel = tile_elem_ptr[t + 1] - tile_elem_ptr[t];
  const int32_t r0 = tile_row0[t], r1 = tile_row0[t + 1];
  const int ns = (int)(row_ptr[r1] - row_ptr[r0]);
  const TileLayout L = tile_layout(nel, ns, nl_in[t], nle_in[t], nbuf, ref, entb, (int)(row_ptr[r0] & 3), nr, nx);
  bytes_out[t] = L.front + L.back;
  front_out[t] = L.front;
}

// Contributions of slot j of a row: local pairs (incidence k, node b) of the
// row's incidences kb..ke whose column position is j.
template <typename PosT>
__device__ __forceinline__ int slot_count(const PosT* __restrict__ inc_pos, int ps, int ref, int kb, int ke, int j) {
  int c = 0;
  for (int k = kb; k < ke; ++k)
    for (int b = 0; b < ref; ++b) c += ((int)inc_pos[(int64_t)k * ps + b] == j);
  return c;
}

// Per tile: number of slots with more than two contributions and their entries.
template <typename PosT>
__global__ void k_tile_long(int ref, const int32_t* __restrict__ tile_row0, const int64_t* __restrict__ row_ptr,
                            const int32_t* __restrict__ inc_ptr, const PosT* __restrict__ inc_pos,
                            int32_t* __restrict__ nl_out, int32_t* __restrict__ nle_out) {
  __shared__ int s_nl, s_nle;
  const int t = blockIdx.x;
  if (threadIdx.x == 0) s_nl = s_nle = 0;
  __syncthreads();
  const int32_t r0 = tile_row0[t], r1 = tile_row0[t + 1];
  const int ps = pos_stride(ref);
  int nl = 0, nle = 0;
  for (int r = r0 + (int)threadIdx.x; r < r1; r += blockDim.x) {
    const int kb = inc_ptr[r], ke = inc_ptr[r + 1];
    const int len = (int)(row_ptr[r + 1] - row_ptr[r]);
    for (int j = 0; j < len; ++j) {
      const int c = slot_count(inc_pos, ps, ref, kb, ke, j);
      if (c > 2) {
        ++nl;
        nle += c;
      }
    }
  }
  atomicAdd(&s_nl, nl);
  atomicAdd(&s_nle, nle);
  __syncthreads();
  if (threadIdx.x == 0) {
    nl_out[t] = s_nl;
    nle_out[t] = s_nle;
  }
}

// Fill one tile's block.  The contribution list of a slot holds, in ascending
// (element, a, b) order, every local pair of the tile's elements that adds into
// it, as the word offset e_local * U + u of that entry in a local-matrix
// array; a row's lists are contiguous (ref entries per incidence of the row).
template <typename PosT>
__global__ void k_tile_fill(const int32_t* __restrict__ conn, int ref, const int32_t* __restrict__ tile_row0,
                            const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ inc_ptr,
                            const uint16_t* __restrict__ inc_local, const PosT* __restrict__ inc_pos,
                            const int32_t* __restrict__ tile_elem_ptr, const int32_t* __restrict__ tile_elem,
                            const int32_t* __restrict__ tmp_nodes, const int32_t* __restrict__ n_nodes,
                            const int32_t* __restrict__ nl_in, const int32_t* __restrict__ nle_in,
                            const int64_t* __restrict__ off, int entb, uint8_t* __restrict__ meta,
                            const int4* __restrict__ runs_tmp, const int2* __restrict__ extras_tmp,
                            const int32_t* __restrict__ pos_tmp, const int32_t* __restrict__ nruns_in,
                            const int32_t* __restrict__ nextra_in, const int32_t* __restrict__ nbuf_in) {
  __shared__ int s_nl, s_nle;
  const int t = blockIdx.x;
  const int32_t r0 = tile_row0[t], r1 = tile_row0[t + 1];
  const int nrows = r1 - r0;
  const int32_t e0 = tile_elem_ptr[t];
  const int nel = tile_elem_ptr[t + 1] - e0;
  const int nn = n_nodes[t];                                // distinct nodes
  const int nbuf = nbuf_in[t], nr = nruns_in[t], nx = nextra_in[t];  // node-buffer positions, runs, extras
  const int64_t s0 = row_ptr[r0];
  const int ns = (int)(row_ptr[r1] - s0);
  // entries address the interleaved local-matrix layout (see TileHdr):
  // word(e, u) = 6 (e UP/2 + u/2) + (u mod 2); a long slot's first entry is
  // its result word LB + 6 li; zeros at ZERO
  const int U = ref * (ref + 1) / 2;
  const int UP = lsm_stride(U);
  const int ps = pos_stride(ref);
  uint8_t* blk = meta + off[t];
  const int nl_t = nl_in[t], nle_t = nle_in[t];
  const int apad = (int)(s0 & 3);
  const TileLayout L = tile_layout(nel, ns, nl_t, nle_t, nbuf, ref, entb, apad, nr, nx);
  const uint32_t LB = (uint32_t)(kLsmSlots * nel * UP), ZERO = LB + 6u * (uint32_t)nl_t;
  auto word = [&](int loc, int u) -> uint32_t { return 6u * (uint32_t)(loc * (UP / 2) + (u >> 1)) + (uint32_t)(u & 1); };
  for (int i = threadIdx.x; i < (L.front + L.back) / 4; i += blockDim.x) reinterpret_cast<uint32_t*>(blk)[i] = 0u;
  if (threadIdx.x == 0) s_nl = s_nle = 0;
  __syncthreads();
  uint8_t* bk = blk + L.front;
  for (int i = threadIdx.x; i < 2 * L.npad; i += blockDim.x) {
    if (entb == 2) reinterpret_cast<uint16_t*>(bk + L.pair)[i] = (uint16_t)ZERO;
    else reinterpret_cast<uint32_t*>(bk + L.pair)[i] = ZERO;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    TileHdr h;
    h.s0 = s0;
    h.r0 = r0;
    h.nrows = nrows;
    h.ns = ns;
    h.nruns = nr;
    h.nel = nel;
    h.nnodes = nbuf;
    h.nl = nl_t;
    h.nle = nle_t;
    h.apad = apad;
    h.nextra = nx;
    h.pad[0] = h.pad[1] = h.pad[2] = h.pad[3] = 0;
    *reinterpret_cast<TileHdr*>(blk) = h;
  }
  int32_t* el = reinterpret_cast<int32_t*>(blk + L.elem);
  int32_t* nd = reinterpret_cast<int32_t*>(blk + L.nodes);
  uint16_t* en = reinterpret_cast<uint16_t*>(blk + L.enodes);
  uint8_t* pr = bk + L.pair;
  int4* lrec = reinterpret_cast<int4*>(bk + L.lrec);
  uint8_t* lent = bk + L.lent;
  for (int i = threadIdx.x; i < nel; i += blockDim.x) el[i] = tile_elem[e0 + i];
  const int32_t* tn = tmp_nodes + (int64_t)e0 * ref;
  const int32_t* tpos = pos_tmp + (int64_t)e0 * ref;
  const int4* truns = runs_tmp + (int64_t)e0 * ref;
  const int2* textra = extras_tmp + (int64_t)e0 * ref;
  int4* runs = reinterpret_cast<int4*>(blk + L.runs);
  int2* extras = reinterpret_cast<int2*>(blk + L.extras);
  // global node id of every buffer position, the runs and the extras
  for (int r = 0; r < nr; ++r) {
    const int4 q = truns[r];
    for (int j = threadIdx.x; j < q.y; j += blockDim.x) nd[q.z + j] = q.x + j;
  }
  for (int r = threadIdx.x; r < nr; r += blockDim.x) runs[r] = truns[r];
  for (int x = threadIdx.x; x < nx; x += blockDim.x) {
    extras[x] = textra[x];
    nd[textra[x].y] = textra[x].x;
  }
  for (int i = threadIdx.x; i < nel * ref; i += blockDim.x) {
    const int32_t v = conn[(int64_t)tile_elem[e0 + i / ref] * ref + (i % ref)];
    int lo = 0, hi = nn;
    while (lo < hi) {
      int mid = (lo + hi) >> 1;
      if (tn[mid] < v) lo = mid + 1;
      else hi = mid;
    }
    en[i] = (uint16_t)tpos[lo];
  }
  auto put = [&](uint8_t* base, int64_t i, uint32_t v) {
    if (entb == 2) reinterpret_cast<uint16_t*>(base)[i] = (uint16_t)v;
    else reinterpret_cast<uint32_t*>(base)[i] = v;
  };
  // contribution lists, one thread per row; slots with one or two entries go
  // to the pair array, longer lists to the long list (its order is the order
  // the threads claim places in it; each run keeps ascending (e, a, b))
  for (int rl = threadIdx.x; rl < nrows; rl += blockDim.x) {
    const int r = r0 + rl;
    const int kb = inc_ptr[r], ke = inc_ptr[r + 1];
    const int slot0 = (int)(row_ptr[r] - s0), len = (int)(row_ptr[r + 1] - row_ptr[r]);
    for (int j = 0; j < len; ++j) {
      const int c = slot_count(inc_pos, ps, ref, kb, ke, j);
      const int slot = slot0 + j;
      const int pp = slot + apad;  // padded slot
      int w = 0, lbeg = 0;
      if (c > 2) {
        const int li = atomicAdd(&s_nl, 1);
        lbeg = atomicAdd(&s_nle, c);
        if (li < nl_t && lbeg + c <= nle_t) {
          lrec[li] = make_int4(slot, lbeg, lbeg + c, li);
          put(pr, 2ll * pp, LB + 6u * (uint32_t)li);  // second entry stays ZERO
        }
      }
      for (int k = kb; k < ke; ++k) {
        const int lk = inc_local[k];
        const int a = lk & 15, loc = lk >> 4;
        for (int b = 0; b < ref; ++b) {
          if ((int)inc_pos[(int64_t)k * ps + b] != j) continue;
          const int u = a <= b ? a * ref - a * (a - 1) / 2 + (b - a) : b * ref - b * (b - 1) / 2 + (a - b);
          const uint32_t ent = word(loc, u);
          if (c > 2) {
            if (lbeg + w < nle_t) put(lent, lbeg + w, ent);
          } else {
            put(pr, 2ll * pp + w, ent);
          }
          ++w;
        }
      }
    }
  }
}

__global__ void k_max_i64(const int64_t* __restrict__ a, int64_t n, int64_t* __restrict__ out) {
  long long m = 0;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    m = max(m, (long long)a[k]);
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_down_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax((unsigned long long*)out, (unsigned long long)m);
}

// Work-item records of a pattern's tiles: block address and part sizes.
__global__ void k_tile_refs(uint8_t* meta, const int64_t* __restrict__ off, const int64_t* __restrict__ bytes,
                            const int32_t* __restrict__ front, int64_t T, ItemRef* __restrict__ refs) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= T) return;
  ItemRef r;
  r.front = meta + off[t];
  r.front_bytes = front[t];
  r.back_bytes = (int32_t)(bytes[t] - front[t]);
  r.mesh = 0;
  r.tile = (int32_t)t;
  r.pad[0] = r.pad[1] = 0;
  refs[t] = r;
}

// Build the per-tile metadata blocks from the tile lists.
static lfem_status build_tile_blocks(lfem_pattern_s* p, cudaStream_t st) {
  PatternDev& d = p->d;
  const int64_t T = p->n_tiles;
  const int ref = p->ref;
  if (d.tile_meta) cudaFree(d.tile_meta);
  if (d.tile_meta_off) cudaFree(d.tile_meta_off);
  if (d.tile_refs) cudaFree(d.tile_refs);
  d.tile_meta = nullptr;
  d.tile_meta_off = nullptr;
  d.tile_refs = nullptr;
  std::vector<int32_t> hep(T + 1);
  LFEM_CUDA(cudaMemcpyAsync(hep.data(), d.tile_elem_ptr, sizeof(int32_t) * (T + 1), cudaMemcpyDeviceToHost, st));
  LFEM_CUDA(cudaStreamSynchronize(st));
  int32_t mnel = 0;
  for (int64_t t = 0; t < T; ++t) mnel = std::max(mnel, hep[t + 1] - hep[t]);
  int32_t *tmp_nodes = nullptr, *nn = nullptr, *nl = nullptr, *nle = nullptr, *front = nullptr;
  int32_t *pos_tmp = nullptr, *nruns = nullptr, *nextra = nullptr, *nbuf = nullptr;
  int4* runs_tmp = nullptr;
  int2* extras_tmp = nullptr;
  int64_t *bytes = nullptr, *scr = nullptr;
  TRY(dalloc(&tmp_nodes, p->tile_elems_total * ref));
  TRY(dalloc(&pos_tmp, p->tile_elems_total * ref));
  TRY(dalloc(&runs_tmp, p->tile_elems_total * ref));
  TRY(dalloc(&extras_tmp, p->tile_elems_total * ref));
  TRY(dalloc(&nruns, T + 1));
  TRY(dalloc(&nextra, T + 1));
  TRY(dalloc(&nbuf, T + 1));
  TRY(dalloc(&nn, T + 1));
  TRY(dalloc(&nl, T + 1));
  TRY(dalloc(&nle, T + 1));
  TRY(dalloc(&front, T + 1));
  TRY(dalloc(&bytes, T + 1));
  TRY(dalloc(&scr, scan_scratch_bytes(T, 8) / 8));
  TRY(dalloc(&d.tile_meta_off, T + 1));
  TRY(dalloc(&d.tile_refs, T));
  std::vector<int32_t> hnl(T);
  if (T > 0) {
    if (p->pos_bytes == 1)
      k_tile_long<uint8_t><<<(unsigned)T, 128, 0, st>>>(ref, d.tile_row0, d.row_ptr, d.inc_ptr, d.inc_pos, nl, nle);
    else
      k_tile_long<uint16_t><<<(unsigned)T, 128, 0, st>>>(ref, d.tile_row0, d.row_ptr, d.inc_ptr,
                                                          (const uint16_t*)d.inc_pos, nl, nle);
    LFEM_CUDA(cudaGetLastError());
    LFEM_CUDA(cudaMemcpyAsync(hnl.data(), nl, sizeof(int32_t) * T, cudaMemcpyDeviceToHost, st));
    LFEM_CUDA(cudaStreamSynchronize(st));
  }
  int32_t mnl = 0;
  for (int64_t t = 0; t < T; ++t) mnl = std::max(mnl, hnl[t]);
  // entries are words of the interleaved local-matrix layout; the largest is
  // the last zero word, 3 nel UP + 6 nl + 5
  const int64_t max_word = (int64_t)kLsmSlots * mnel * lsm_stride(n_upper(ref)) + 6ll * mnl + 5;
  const int entb = std::max(max_word <= 65535 ? 2 : 4, p->min_ent_bytes);
  if (T > 0) {
    const size_t smem = sizeof(int32_t) * kMaxTileEntries;
    LFEM_CUDA(cudaFuncSetAttribute(k_tile_nodes, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_tile_nodes<<<(unsigned)T, 512, smem, st>>>(d.conn, ref, d.tile_elem_ptr, d.tile_elem, tmp_nodes, nn);
    LFEM_CUDA(cudaGetLastError());
    k_tile_runs<<<grid_for(T, 128), 128, 0, st>>>(tmp_nodes, nn, d.tile_elem_ptr, ref, p->n_nodes, d.tile_row0,
                                                  d.row_ptr, nl, nle, entb, T, runs_tmp, extras_tmp, pos_tmp, nruns,
                                                  nextra, nbuf, bytes, front);
    LFEM_CUDA(cudaGetLastError());
  }
  scan_exclusive<int64_t, int64_t>(bytes, d.tile_meta_off, T, scr, st);
  int64_t total = 0;
  std::vector<int64_t> hbytes(T);
  std::vector<int32_t> hfront(T), hnn(T);
  LFEM_CUDA(cudaMemcpyAsync(&total, d.tile_meta_off + T, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  if (T > 0) {
    LFEM_CUDA(cudaMemcpyAsync(hbytes.data(), bytes, sizeof(int64_t) * T, cudaMemcpyDeviceToHost, st));
    LFEM_CUDA(cudaMemcpyAsync(hfront.data(), front, sizeof(int32_t) * T, cudaMemcpyDeviceToHost, st));
    LFEM_CUDA(cudaMemcpyAsync(hnn.data(), nbuf, sizeof(int32_t) * T, cudaMemcpyDeviceToHost, st));
  }
  LFEM_CUDA(cudaStreamSynchronize(st));
  TRY(dalloc(&d.tile_meta, total));
  if (T > 0) {
    if (p->pos_bytes == 1)
      k_tile_fill<uint8_t><<<(unsigned)T, 128, 0, st>>>(d.conn, ref, d.tile_row0, d.row_ptr, d.inc_ptr, d.inc_local,
                                                         d.inc_pos, d.tile_elem_ptr, d.tile_elem, tmp_nodes, nn,
                                                         nl, nle, d.tile_meta_off, entb, d.tile_meta, runs_tmp,
                                                         extras_tmp, pos_tmp, nruns, nextra, nbuf);
    else
      k_tile_fill<uint16_t><<<(unsigned)T, 128, 0, st>>>(d.conn, ref, d.tile_row0, d.row_ptr, d.inc_ptr,
                                                          d.inc_local, (const uint16_t*)d.inc_pos, d.tile_elem_ptr,
                                                          d.tile_elem, tmp_nodes, nn, nl, nle, d.tile_meta_off, entb,
                                                          d.tile_meta, runs_tmp, extras_tmp, pos_tmp, nruns, nextra,
                                                          nbuf);
    LFEM_CUDA(cudaGetLastError());
    k_tile_refs<<<grid_for(T, 256), 256, 0, st>>>(d.tile_meta, d.tile_meta_off, bytes, front, T, d.tile_refs);
    LFEM_CUDA(cudaGetLastError());
  }
  int32_t mnn = 0, mfront = 0, mback = 0;
  for (int64_t t = 0; t < T; ++t) {
    mnn = std::max(mnn, hnn[t]);
    mfront = std::max(mfront, hfront[t]);
    mback = std::max(mback, (int32_t)(hbytes[t] - hfront[t]));
  }
  p->max_tile_nel = mnel;
  p->max_tile_nodes = mnn;
  p->max_tile_front = mfront;
  p->max_tile_back = mback;
  p->max_tile_nl = mnl;
  p->ent_bytes = entb;
  LFEM_CUDA(cudaStreamSynchronize(st));
  cudaFree(tmp_nodes);
  cudaFree(pos_tmp);
  cudaFree(runs_tmp);
  cudaFree(extras_tmp);
  cudaFree(nruns);
  cudaFree(nextra);
  cudaFree(nbuf);
  cudaFree(nn);
  cudaFree(nl);
  cudaFree(nle);
  cudaFree(front);
  cudaFree(bytes);
  cudaFree(scr);
  return LFEM_OK;
}

lfem_status build_tiles(lfem_pattern_s* p, int32_t tile_slots, cudaStream_t st) {
  PatternDev& d = p->d;
  const int32_t N = p->n_nodes;
  if (tile_slots < 256 || tile_slots > 16384) return fail(LFEM_E_ARG, "tile_slots outside [256, 16384]");
  if (p->ref > 16) return fail(LFEM_E_UNSUPPORTED, "row tiles hold elements of at most 16 nodes");
  if (p->max_row > tile_slots) return fail(LFEM_E_TOO_LARGE, "a CSR row is longer than the tile capacity");
  // greedy contiguous packing of rows under the slot and incidence budgets
  std::vector<int64_t> rp(N + 1);
  std::vector<int32_t> ip(N + 1);
  LFEM_CUDA(cudaMemcpyAsync(rp.data(), d.row_ptr, sizeof(int64_t) * (N + 1), cudaMemcpyDeviceToHost, st));
  LFEM_CUDA(cudaMemcpyAsync(ip.data(), d.inc_ptr, sizeof(int32_t) * (N + 1), cudaMemcpyDeviceToHost, st));
  LFEM_CUDA(cudaStreamSynchronize(st));
  std::vector<int32_t> rows;
  rows.push_back(0);
  int32_t r0 = 0;
  for (int32_t i = 0; i < N; ++i) {
    const int64_t ninc = ip[i + 1] - ip[r0];
    bool over = (rp[i + 1] - rp[r0] > tile_slots) || (ninc > kMaxTileIncidences) ||
                (ninc * p->ref > kMaxTileEntries) || (i + 1 - r0 > kMaxTileRows);
    if (over && i > r0) {
      rows.push_back(i);
      r0 = i;
    }
  }
  if (N > 0 && rows.back() != N) rows.push_back(N);
  const int64_t T = (int64_t)rows.size() - 1;
  if (d.tile_row0) cudaFree(d.tile_row0);
  if (d.tile_elem_ptr) cudaFree(d.tile_elem_ptr);
  if (d.tile_elem) cudaFree(d.tile_elem);
  d.tile_row0 = d.tile_elem_ptr = d.tile_elem = nullptr;
  TRY(dalloc(&d.tile_row0, T + 1));
  TRY(dalloc(&d.tile_elem_ptr, T + 1));
  LFEM_CUDA(cudaMemcpyAsync(d.tile_row0, rows.data(), sizeof(int32_t) * (T + 1), cudaMemcpyHostToDevice, st));
  int32_t *tmp = nullptr, *counts = nullptr, *scr = nullptr;
  TRY(dalloc(&tmp, p->n_inc));
  TRY(dalloc(&counts, T + 1));
  TRY(dalloc(&scr, scan_scratch_bytes(T, sizeof(int32_t)) / 4));
  if (T > 0) {
    k_tile_elements<<<(unsigned)T, 512, 0, st>>>(d.tile_row0, d.inc_ptr, d.inc_key, tmp, counts, d.inc_local);
    LFEM_CUDA(cudaGetLastError());
  }
  scan_exclusive<int32_t, int32_t>(counts, d.tile_elem_ptr, T, scr, st);
  int32_t total = 0;
  LFEM_CUDA(cudaMemcpyAsync(&total, d.tile_elem_ptr + T, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  LFEM_CUDA(cudaStreamSynchronize(st));
  TRY(dalloc(&d.tile_elem, total));
  if (T > 0) {
    k_tile_compact<<<(unsigned)T, 256, 0, st>>>(d.tile_row0, d.inc_ptr, tmp, d.tile_elem_ptr, d.tile_elem);
    LFEM_CUDA(cudaGetLastError());
  }
  LFEM_CUDA(cudaStreamSynchronize(st));
  cudaFree(tmp);
  cudaFree(counts);
  cudaFree(scr);
  p->n_tiles = T;
  p->tile_slots = tile_slots;
  p->tile_elems_total = total;
  return build_tile_blocks(p, st);
}

lfem_status build_pattern(lfem_pattern_s* p, const int32_t* conn_in, cudaStream_t st) {
  PatternDev& d = p->d;
  const int ref = p->ref;
  const int64_t nE = p->n_elem;
  const int32_t N = p->n_nodes;
  const int64_t n_inc = nE * ref;
  p->n_inc = n_inc;
  TRY(dalloc(&d.status, 6));  // status bits, pad, fallback count (int64), tile ticket counter (int64)
  LFEM_CUDA(cudaMemsetAsync(d.status, 0, 6 * sizeof(int32_t), st));
  TRY(dalloc(&d.conn, n_inc));
  if (n_inc > 0)
    LFEM_CUDA(cudaMemcpyAsync(d.conn, conn_in, sizeof(int32_t) * n_inc, cudaMemcpyDeviceToDevice, st));
  int32_t *deg = nullptr, *scr = nullptr, *maxv = nullptr;
  TRY(dalloc(&deg, (int64_t)N + 1));
  TRY(dalloc(&d.inc_ptr, (int64_t)N + 1));
  TRY(dalloc(&scr, scan_scratch_bytes((int64_t)N + n_inc, sizeof(int64_t)) / 4 + (int64_t)N + 2));
  TRY(dalloc(&maxv, 2));
  LFEM_CUDA(cudaMemsetAsync(deg, 0, sizeof(int32_t) * ((int64_t)N + 1), st));
  LFEM_CUDA(cudaMemsetAsync(maxv, 0, 2 * sizeof(int32_t), st));
  if (n_inc > 0) k_count_degree<<<grid_for(n_inc, 256), 256, 0, st>>>(d.conn, n_inc, N, deg, d.status);
  LFEM_CUDA(cudaGetLastError());
  if (N > 0) k_max_i32<<<grid_for(N, 256), 256, 0, st>>>(deg, N, maxv);
  int32_t hst[2] = {0, 0};
  LFEM_CUDA(cudaMemcpyAsync(&hst[0], d.status, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  LFEM_CUDA(cudaMemcpyAsync(&hst[1], maxv, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  LFEM_CUDA(cudaStreamSynchronize(st));
  if (hst[0] & ST_INDEX) {
    cudaFree(deg);
    cudaFree(scr);
    cudaFree(maxv);
    return fail(LFEM_E_INDEX, "connectivity holds a node index outside [0, n_nodes)");
  }
  p->max_deg = hst[1];
  if (p->max_deg > kMaxDegree || (int64_t)p->max_deg * ref > kMaxSegSort) {
    cudaFree(deg);
    cudaFree(scr);
    cudaFree(maxv);
    return fail(LFEM_E_TOO_LARGE, "too many elements meet at one node");
  }
  scan_exclusive<int32_t, int32_t>(deg, d.inc_ptr, N, scr, st);
  TRY(dalloc(&d.inc_key, n_inc));
  LFEM_CUDA(cudaMemsetAsync(deg, 0, sizeof(int32_t) * ((int64_t)N + 1), st));
  if (n_inc > 0) k_fill_incidence<<<grid_for(n_inc, 256), 256, 0, st>>>(d.conn, nE, ref, p->key_shift, d.inc_ptr, deg,
                                                                       d.inc_key);
  LFEM_CUDA(cudaGetLastError());
  int32_t* sort_scr = nullptr;
  TRY(dalloc(&sort_scr, (int64_t)N + 2));
  TRY(segsort(d.inc_key, d.inc_ptr, N, 1, p->max_deg, sort_scr, st));
  // raw column lists per row and the (e, a) -> incidence map
  int32_t* raw = nullptr;
  TRY(dalloc(&raw, n_inc * ref));
  TRY(dalloc(&d.elem_inc, n_inc));
  if (n_inc > 0) k_elem_inc_and_raw<<<grid_for(n_inc, 256), 256, 0, st>>>(d.conn, ref, p->key_shift, d.inc_key, n_inc,
                                                                         d.elem_inc, raw);
  LFEM_CUDA(cudaGetLastError());
  TRY(segsort(raw, d.inc_ptr, N, ref, p->max_deg * ref, sort_scr, st));
  int32_t* rowlen = deg;  // reuse
  if (N > 0) k_row_unique_count<<<grid_for(N, 128), 128, 0, st>>>(raw, d.inc_ptr, ref, N, rowlen);
  LFEM_CUDA(cudaGetLastError());
  TRY(dalloc(&d.row_ptr, (int64_t)N + 1));
  int64_t* scr64 = nullptr;
  TRY(dalloc(&scr64, scan_scratch_bytes(N, sizeof(int64_t)) / 8));
  scan_exclusive<int32_t, int64_t>(rowlen, d.row_ptr, N, scr64, st);
  LFEM_CUDA(cudaMemsetAsync(maxv, 0, 2 * sizeof(int32_t), st));
  if (N > 0) k_max_i32<<<grid_for(N, 256), 256, 0, st>>>(rowlen, N, maxv);
  int64_t nnz = 0;
  LFEM_CUDA(cudaMemcpyAsync(&nnz, d.row_ptr + N, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  LFEM_CUDA(cudaMemcpyAsync(&hst[1], maxv, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  LFEM_CUDA(cudaStreamSynchronize(st));
  p->nnz = nnz;
  p->max_row = hst[1];
  if (nnz >= INT32_MAX) return fail(LFEM_E_TOO_LARGE, "nnz >= 2^31");
  TRY(dalloc(&d.col_idx, nnz));
  if (N > 0) k_row_compact<<<grid_for(N, 128), 128, 0, st>>>(raw, d.inc_ptr, ref, N, d.row_ptr, d.col_idx);
  LFEM_CUDA(cudaGetLastError());
  p->pos_bytes = p->max_row <= 256 ? 1 : 2;
  TRY(dalloc(&d.inc_pos, n_inc * pos_stride(ref) * p->pos_bytes));
  LFEM_CUDA(cudaMemsetAsync(d.inc_pos, 0, (size_t)n_inc * pos_stride(ref) * p->pos_bytes, st));
  if (N > 0) {
    if (p->pos_bytes == 1)
      k_positions<uint8_t><<<grid_for(N, 128), 128, 0, st>>>(d.conn, ref, p->key_shift, d.inc_key, d.inc_ptr, N,
                                                               d.row_ptr, d.col_idx, d.inc_pos);
    else
      k_positions<uint16_t><<<grid_for(N, 128), 128, 0, st>>>(d.conn, ref, p->key_shift, d.inc_key, d.inc_ptr, N,
                                                                d.row_ptr, d.col_idx, (uint16_t*)d.inc_pos);
  }
  LFEM_CUDA(cudaGetLastError());
  TRY(dalloc(&d.inc_local, n_inc));
  if (p->dim == 3 || p->order >= 3) {
    // bulk tets and orders 3, 4: element-major path (row tiles would recompute
    // most tets several times; high orders have large local matrices)
    if (n_inc * ref >= INT32_MAX || p->n_elem * n_upper(ref) >= INT32_MAX)
      return fail(LFEM_E_TOO_LARGE, "too many contributions for the element-major path");
    TRY(dalloc(&d.slot_off, nnz + 1));
    TRY(dalloc(&d.slot_ent, n_inc * ref));
    if (N > 0) {
      if (p->pos_bytes == 1)
        k_slot_lists<uint8_t><<<grid_for(N, 128), 128, 0, st>>>(d.inc_ptr, d.inc_key, d.inc_pos, d.row_ptr, N, ref,
                                                                 p->key_shift, d.slot_off, d.slot_ent);
      else
        k_slot_lists<uint16_t><<<grid_for(N, 128), 128, 0, st>>>(d.inc_ptr, d.inc_key, (const uint16_t*)d.inc_pos,
                                                                  d.row_ptr, N, ref, p->key_shift, d.slot_off,
                                                                  d.slot_ent);
      LFEM_CUDA(cudaGetLastError());
    }
    const int32_t tot = (int32_t)(n_inc * ref);
    LFEM_CUDA(cudaMemcpyAsync(d.slot_off + nnz, &tot, sizeof(int32_t), cudaMemcpyHostToDevice, st));
  }
  LFEM_CUDA(cudaStreamSynchronize(st));
  cudaFree(raw);
  cudaFree(deg);
  cudaFree(scr);
  cudaFree(scr64);
  cudaFree(maxv);
  cudaFree(sort_scr);
  // elements of more than 16 nodes (order-3/4 tets) use the element-major path only
  if (ref > 16) return LFEM_OK;
  return build_tiles(p, p->tile_slots, st);
}

// ----------------------------------------------------------------------------
// CSR pattern without device allocation (lfem_pattern_csr_noalloc).
//
// Some callers cannot allocate device memory while they run: programs whose
// allocator owns all device memory up front (a fixed arena or pool, a real-time
// loop that forbids cudaMalloc after start-up), or hosts that hand this library
// only the buffers they manage.  This path keeps its scratch in one file-scope
// device array instead.  Every GPU that loads the library holds the array until
// the process exits; all calls share it, so calls whose work overlaps on the
// GPU (different streams, threads or processes sharing a context) race.  The
// array keeps the last call's contents; every region a step needs at zero is
// cleared on the stream first.
// ----------------------------------------------------------------------------
constexpr int64_t kStaticScratchWords = 4ll << 20;  // 16 MiB of int32 words
static __device__ __align__(256) int32_t g_static_scratch[kStaticScratchWords];
static std::mutex g_static_mu;
static void* g_static_ptr[64];

// Device address of the array for the current device.  The first call on a
// device looks it up (cudaGetSymbolAddress); the host-side symbol itself is
// only a stand-in and must never be passed to a kernel.
static lfem_status static_scratch(int32_t** out) {
  int dev = 0;
  LFEM_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(LFEM_E_ARG, "device ordinal >= 64");
  std::lock_guard<std::mutex> lk(g_static_mu);
  if (!g_static_ptr[dev]) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(static scratch)");
    g_static_ptr[dev] = ptr;
  }
  *out = static_cast<int32_t*>(g_static_ptr[dev]);
  return LFEM_OK;
}

lfem_status pattern_csr_noalloc(const int32_t* conn, int64_t nE, int32_t N, int dim, int order, int64_t* row_ptr,
                                int32_t* col_idx, int64_t col_capacity, int64_t* nnz_out, cudaStream_t st) {
  const int ref = n_ref(dim, order);
  const int64_t I = nE * ref;
  // word budget, each region rounded up to 64 words (256 bytes)
  auto rnd = [](int64_t w) { return (w + 63) / 64 * 64; };
  const int64_t w_deg = rnd((int64_t)N + 2), w_ptr = rnd((int64_t)N + 2), w_misc = 64;
  const int64_t w_key = rnd(I), w_einc = rnd(I), w_raw = rnd(I * ref), w_sort = rnd((int64_t)N + 2);
  const int64_t w_s32 = rnd(scan_scratch_bytes(N, 4) / 4), w_s64 = rnd(scan_scratch_bytes(N, 8) / 4);
  const int64_t need = w_deg + w_ptr + w_misc + w_key + w_einc + w_raw + w_sort + w_s32 + w_s64;
  if (need > kStaticScratchWords)
    return fail(LFEM_E_TOO_LARGE, "mesh needs more than the 16 MiB static scratch of the no-allocation path");
  int32_t* base = nullptr;
  TRY(static_scratch(&base));
  int32_t* deg = base;
  int32_t* inc_ptr = deg + w_deg;
  int32_t* misc = inc_ptr + w_ptr;  // [0] status, [1] max degree, [2] max row length
  int32_t* key = misc + w_misc;
  int32_t* einc = key + w_key;
  int32_t* raw = einc + w_einc;
  int32_t* sort_scr = raw + w_raw;
  int32_t* s32 = sort_scr + w_sort;
  int64_t* s64 = reinterpret_cast<int64_t*>(s32 + w_s32);

  LFEM_CUDA(cudaMemsetAsync(deg, 0, sizeof(int32_t) * ((size_t)N + 1), st));
  LFEM_CUDA(cudaMemsetAsync(misc, 0, sizeof(int32_t) * 4, st));
  if (I > 0) k_count_degree<<<grid_for(I, 256), 256, 0, st>>>(conn, I, N, deg, misc);
  LFEM_CUDA(cudaGetLastError());
  if (N > 0) k_max_i32<<<grid_for(N, 256), 256, 0, st>>>(deg, N, misc + 1);
  LFEM_CUDA(cudaGetLastError());
  int32_t h[2] = {0, 0};
  LFEM_CUDA(cudaMemcpyAsync(h, misc, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  LFEM_CUDA(cudaStreamSynchronize(st));
  if (h[0] & ST_INDEX) return fail(LFEM_E_INDEX, "connectivity holds a node index outside [0, n_nodes)");
  if (h[1] > kMaxDegree || (int64_t)h[1] * ref > kMaxSegSort)
    return fail(LFEM_E_TOO_LARGE, "too many elements meet at one node");
  scan_exclusive<int32_t, int32_t>(deg, inc_ptr, N, s32, st);
  LFEM_CUDA(cudaMemsetAsync(deg, 0, sizeof(int32_t) * ((size_t)N + 1), st));
  // incidence key (e << ksh) | a, as in lfem_pattern: 4 bits of local index up to 16 nodes, else 6
  const int ksh = ref > 16 ? 6 : 4;
  if (I > 0) k_fill_incidence<<<grid_for(I, 256), 256, 0, st>>>(conn, nE, ref, ksh, inc_ptr, deg, key);
  LFEM_CUDA(cudaGetLastError());
  TRY(segsort(key, inc_ptr, N, 1, h[1], sort_scr, st));
  if (I > 0) k_elem_inc_and_raw<<<grid_for(I, 256), 256, 0, st>>>(conn, ref, ksh, key, I, einc, raw);
  LFEM_CUDA(cudaGetLastError());
  TRY(segsort(raw, inc_ptr, N, ref, h[1] * ref, sort_scr, st));
  if (N > 0) k_row_unique_count<<<grid_for(N, 128), 128, 0, st>>>(raw, inc_ptr, ref, N, deg);
  LFEM_CUDA(cudaGetLastError());
  scan_exclusive<int32_t, int64_t>(deg, row_ptr, N, s64, st);
  int64_t nnz = 0;
  LFEM_CUDA(cudaMemcpyAsync(&nnz, row_ptr + N, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  LFEM_CUDA(cudaStreamSynchronize(st));
  if (nnz_out) *nnz_out = nnz;
  if (nnz > col_capacity) return fail(LFEM_E_TOO_LARGE, "col_idx capacity smaller than nnz (nnz returned)");
  if (N > 0) k_row_compact<<<grid_for(N, 128), 128, 0, st>>>(raw, inc_ptr, ref, N, row_ptr, col_idx);
  LFEM_CUDA(cudaGetLastError());
  LFEM_CUDA(cudaStreamSynchronize(st));
  return LFEM_OK;
}

// ---------------------------------------------------------------------------
// Order-p nodes from an order-1 mesh (the node generation of the paper's
// preprocessing, Sec. 4).  Edges are the upper slots (i < j) of the P1
// pattern's rows, numbered in CSR order (row i ascending, then column j), so
// edge (i, j)'s number is up_start[i] + (position of j in row i) - (entries of
// row i with column <= i).  Tetrahedron faces are numbered in lexicographic
// order of their sorted vertex triples (g0 < g1 < g2): every face is keyed
// under g0 by the positions of g1 and g2 in row g0, the keys of each vertex
// are sorted and made unique, and a face's number is the count of distinct
// faces before it.  Node numbers: vertices, then p - 1 nodes per edge from its
// lower to its higher vertex, then the face nodes (tets; face by face, on the
// sorted vertices by increasing (alpha_1, alpha_2)) or the triangle interior
// nodes, then the tet interior nodes.  Positions are the straight ones,
// rounded in a fixed order (products, then sums left to right, face nodes
// over the sorted vertices; no multiply-add contraction).
// ---------------------------------------------------------------------------
__global__ void k_lift_count(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col_idx, int32_t n,
                             int32_t* __restrict__ up_cnt, int32_t* __restrict__ c_le) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    int64_t lo = row_ptr[i], hi = row_ptr[i + 1];
    const int64_t b = lo, e = hi;
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (col_idx[mid] <= i) lo = mid + 1;
      else hi = mid;
    }
    c_le[i] = (int32_t)(lo - b);
    up_cnt[i] = (int32_t)(e - lo);
  }
}

__global__ void k_lift_corners(const double* __restrict__ x, int64_t n_values, double* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_values; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = x[i];
}

// Local edges (0,1), (1,2), (2,0), (0,3), (1,3), (2,3); local faces (0,1,2),
// (0,1,3), (0,2,3), (1,2,3) -- face f leaves out corner 3 - f.
__device__ __forceinline__ int lift_edge_first(int k) { return k < 3 ? k : k - 3; }
__device__ __forceinline__ int lift_edge_second(int k) { return k < 3 ? (k + 1) % 3 : 3; }
__device__ __forceinline__ int lift_face_corner(int f, int k) { return k + (k >= 3 - f ? 1 : 0); }

// Position of column c in row r (offset from the row start), or -1.
__device__ __forceinline__ int64_t row_position(const int64_t* __restrict__ row_ptr,
                                                const int32_t* __restrict__ col_idx, int32_t r, int32_t c) {
  int64_t lo = row_ptr[r], hi = row_ptr[r + 1];
  const int64_t rb = lo, re = hi;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (col_idx[mid] < c) lo = mid + 1;
    else hi = mid;
  }
  return (lo < re && col_idx[lo] == c) ? lo - rb : -1;
}

// Local face f of a tet: its corners' global numbers sorted (g[0] < g[1] < g[2])
// and rank[k] = place of the face's k-th local corner among them.
__device__ __forceinline__ void tet_face_sorted(const int32_t (&v)[4], int f, int32_t (&g)[3], int (&rank)[3]) {
  const int32_t a = v[lift_face_corner(f, 0)], b = v[lift_face_corner(f, 1)], c = v[lift_face_corner(f, 2)];
  rank[0] = (a > b) + (a > c);
  rank[1] = (b > a) + (b > c);
  rank[2] = (c > a) + (c > b);
  g[rank[0]] = a;
  g[rank[1]] = b;
  g[rank[2]] = c;
}

__device__ __forceinline__ int32_t face_key(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col_idx,
                                            const int32_t (&g)[3]) {
  const int64_t p1 = row_position(row_ptr, col_idx, g[0], g[1]), p2 = row_position(row_ptr, col_idx, g[0], g[2]);
  if (p1 < 0 || p2 < 0 || p2 > 32767) return -1;
  return (int32_t)((p1 << 16) | p2);
}

__global__ void k_face_count(const int32_t* __restrict__ conn, int64_t n_elem, int32_t* __restrict__ cnt) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n_elem; e += (int64_t)gridDim.x * blockDim.x) {
    int32_t v[4];
    for (int a = 0; a < 4; ++a) v[a] = conn[e * 4 + a];
    for (int f = 0; f < 4; ++f) {
      int32_t g[3];
      int rank[3];
      tet_face_sorted(v, f, g, rank);
      atomicAdd(&cnt[g[0]], 1);
    }
  }
}

__global__ void k_face_fill(const int32_t* __restrict__ conn, int64_t n_elem, const int64_t* __restrict__ row_ptr,
                            const int32_t* __restrict__ col_idx, const int32_t* __restrict__ off,
                            int32_t* __restrict__ cursor, int32_t* __restrict__ keys, int32_t* status) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n_elem; e += (int64_t)gridDim.x * blockDim.x) {
    int32_t v[4];
    for (int a = 0; a < 4; ++a) v[a] = conn[e * 4 + a];
    for (int f = 0; f < 4; ++f) {
      int32_t g[3];
      int rank[3];
      tet_face_sorted(v, f, g, rank);
      int32_t key = face_key(row_ptr, col_idx, g);
      if (key < 0) {
        atomicOr(status, ST_INDEX);  // the pattern does not hold this face's edges
        key = INT_MAX;
      }
      keys[off[g[0]] + atomicAdd(&cursor[g[0]], 1)] = key;
    }
  }
}

// Per vertex: distinct-key number of every (sorted) key, and the distinct count.
__global__ void k_face_unique(const int32_t* __restrict__ keys, const int32_t* __restrict__ off, int32_t n,
                              int32_t* __restrict__ uid, int32_t* __restrict__ fcnt) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    int32_t d = -1, prev = -1;
    for (int32_t k = off[i]; k < off[i + 1]; ++k) {
      d += keys[k] != prev;
      prev = keys[k];
      uid[k] = d;
    }
    fcnt[i] = d + 1;
  }
}

struct LiftFaces {
  const int32_t* off = nullptr;    // [N + 1] per-vertex key ranges
  const int32_t* keys = nullptr;   // sorted face keys
  const int32_t* uid = nullptr;    // distinct number of each key within its vertex
  const int64_t* fbase = nullptr;  // [N + 1] first face number of each vertex
  int64_t n_faces = 0;
};

// Index of (p - a1 - a2, a1, a2) in the list of a triangle's interior
// multi-indices by increasing (a1, a2).
__device__ __forceinline__ int face_alpha_index(int p, int a1, int a2) {
  int t = 0;
  for (int b1 = 1; b1 < a1; ++b1) t += p - 1 - b1;
  return t + a2 - 1;
}

__global__ void k_lift_elements(const int32_t* __restrict__ conn, int64_t n_elem, int dim, int na, int order,
                                const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col_idx,
                                const int64_t* __restrict__ up_start, const int32_t* __restrict__ c_le,
                                int32_t n_vert, int64_t n_edges, const LiftFaces fc, const double* __restrict__ x,
                                int32_t* conn_out, double* coords_out, int32_t* status) {
  const int ref1 = dim + 1;
  const int n_le = dim == 1 ? 1 : (dim == 2 ? 3 : 6);
  const int nfi = (order - 1) * (order - 2) / 2;  // interior nodes of one triangle
  const int nci = dim == 3 ? (order - 1) * (order - 2) * (order - 3) / 6 : 0;
  const int refp = ref1 + n_le * (order - 1) + (dim == 2 ? nfi : (dim == 3 ? 4 * nfi + nci : 0));
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n_elem; e += (int64_t)gridDim.x * blockDim.x) {
    int32_t v[4];
    for (int a = 0; a < ref1; ++a) v[a] = conn[e * ref1 + a];
    int32_t* row = conn_out ? conn_out + e * refp : nullptr;
    if (row)
      for (int a = 0; a < ref1; ++a) row[a] = v[a];
    int slot = ref1;
    for (int le = 0; le < n_le; ++le) {
      const int32_t i = v[lift_edge_first(le)], j = v[lift_edge_second(le)];
      const int32_t lo_v = i < j ? i : j, hi_v = i < j ? j : i;
      const int64_t pos = row_position(row_ptr, col_idx, lo_v, hi_v);
      const int64_t eid = up_start[lo_v] + pos - c_le[lo_v];
      if (pos < 0 || eid < 0 || eid >= n_edges) {
        atomicOr(status, ST_INDEX);  // the pattern does not hold this edge: skip its nodes
        slot += order - 1;
        continue;
      }
      const int64_t first = (int64_t)n_vert + eid * (order - 1);
      for (int k = 1; k < order; ++k) {
        if (row) row[slot + k - 1] = (int32_t)(first + (i < j ? k : order - k) - 1);
        if (coords_out) {
          const double t = (double)k / (double)order, s = 1.0 - t;
          for (int c = 0; c < na; ++c)
            coords_out[(first + k - 1) * na + c] =
                __dadd_rn(__dmul_rn(x[(int64_t)lo_v * na + c], s), __dmul_rn(x[(int64_t)hi_v * na + c], t));
        }
      }
      slot += order - 1;
    }
    const int64_t base = (int64_t)n_vert + n_edges * (order - 1);
    if (dim == 2) {
      const int64_t first = base + e * nfi;
      int t = 0;
      for (int a1 = 1; a1 < order; ++a1)
        for (int a2 = 1; a1 + a2 < order; ++a2, ++t) {
          if (row) row[slot + t] = (int32_t)(first + t);
          if (coords_out) {
            const double l0 = (double)(order - a1 - a2) / order, l1 = (double)a1 / order, l2 = (double)a2 / order;
            for (int c = 0; c < na; ++c) {
              const double s01 = __dadd_rn(__dmul_rn(l0, x[(int64_t)v[0] * na + c]), __dmul_rn(l1, x[(int64_t)v[1] * na + c]));
              coords_out[(first + t) * na + c] = __dadd_rn(s01, __dmul_rn(l2, x[(int64_t)v[2] * na + c]));
            }
          }
        }
    }
    if (dim == 3 && nfi > 0) {
      for (int f = 0; f < 4; ++f, slot += nfi) {
        int32_t g[3];
        int rank[3];
        tet_face_sorted(v, f, g, rank);
        const int32_t key = face_key(row_ptr, col_idx, g);
        int32_t lo = fc.off[g[0]], hi = fc.off[g[0] + 1];
        const int32_t end = hi;
        while (lo < hi) {
          const int32_t mid = (lo + hi) >> 1;
          if (fc.keys[mid] < key) lo = mid + 1;
          else hi = mid;
        }
        const int64_t fid = key < 0 || lo >= end || fc.keys[lo] != key ? -1 : fc.fbase[g[0]] + fc.uid[lo];
        if (fid < 0 || fid >= fc.n_faces) {
          atomicOr(status, ST_INDEX);
          continue;
        }
        const int64_t first = base + fid * nfi;
        int t = 0;
        for (int aj = 1; aj < order; ++aj)
          for (int al = 1; aj + al < order; ++al, ++t) {
            // weights of the local corners (i, j, l), moved onto the sorted corners
            int w[3];
            w[rank[0]] = order - aj - al;
            w[rank[1]] = aj;
            w[rank[2]] = al;
            const int64_t node = first + face_alpha_index(order, w[1], w[2]);
            if (row) row[slot + t] = (int32_t)node;
            if (coords_out) {
              const double l0 = (double)w[0] / order, l1 = (double)w[1] / order, l2 = (double)w[2] / order;
              for (int c = 0; c < na; ++c) {
                const double s01 = __dadd_rn(__dmul_rn(l0, x[(int64_t)g[0] * na + c]), __dmul_rn(l1, x[(int64_t)g[1] * na + c]));
                coords_out[node * na + c] = __dadd_rn(s01, __dmul_rn(l2, x[(int64_t)g[2] * na + c]));
              }
            }
          }
      }
      const int64_t first = base + fc.n_faces * nfi + e * nci;
      int t = 0;
      for (int a1 = 1; a1 < order; ++a1)
        for (int a2 = 1; a1 + a2 < order; ++a2)
          for (int a3 = 1; a1 + a2 + a3 < order; ++a3, ++t) {
            if (row) row[slot + t] = (int32_t)(first + t);
            if (coords_out) {
              const double l[4] = {(double)(order - a1 - a2 - a3) / order, (double)a1 / order, (double)a2 / order,
                                   (double)a3 / order};
              for (int c = 0; c < na; ++c) {
                double acc = __dmul_rn(l[0], x[(int64_t)v[0] * na + c]);
                for (int k = 1; k < 4; ++k) acc = __dadd_rn(acc, __dmul_rn(l[k], x[(int64_t)v[k] * na + c]));
                coords_out[(first + t) * na + c] = acc;
              }
            }
          }
    }
  }
}

lfem_status lift_order(lfem_pattern_s* p, const double* coords, int na, int order, int32_t* conn_out,
                       double* coords_out, int64_t* n_nodes_out, cudaStream_t st) {
  PatternDev& d = p->d;
  const int32_t N = p->n_nodes;
  const int64_t nE = p->n_elem;
  const int nfi = (order - 1) * (order - 2) / 2;
  const int nci = p->dim == 3 ? (order - 1) * (order - 2) * (order - 3) / 6 : 0;
  std::vector<void*> owned;
  auto cleanup = [&]() {
    for (void* q : owned) cudaFree(q);
    owned.clear();
  };
  auto alloc32 = [&](int32_t** q, int64_t n) {
    lfem_status r = dalloc(q, n);
    if (r == LFEM_OK) owned.push_back(*q);
    return r;
  };
  auto alloc64 = [&](int64_t** q, int64_t n) {
    lfem_status r = dalloc(q, n);
    if (r == LFEM_OK) owned.push_back(*q);
    return r;
  };
#define LIFT_TRY(x)           \
  do {                        \
    lfem_status r_ = (x);     \
    if (r_ != LFEM_OK) {      \
      cleanup();              \
      return r_;              \
    }                         \
  } while (0)
  int32_t *cnt = nullptr, *cle = nullptr;
  int64_t *up = nullptr, *scr = nullptr;
  LIFT_TRY(alloc32(&cnt, (int64_t)N + 1));
  LIFT_TRY(alloc32(&cle, (int64_t)N + 1));
  LIFT_TRY(alloc64(&up, (int64_t)N + 1));
  LIFT_TRY(alloc64(&scr, scan_scratch_bytes((int64_t)N + 1, 8) / 8));
  cudaMemsetAsync(cnt, 0, sizeof(int32_t) * ((size_t)N + 1), st);
  if (N > 0) k_lift_count<<<grid_for(N, 256), 256, 0, st>>>(d.row_ptr, d.col_idx, N, cnt, cle);
  // up[0..N]: exclusive scan of the N row counts, up[N] = number of edges
  scan_exclusive<int32_t, int64_t>(cnt, up, (int64_t)N, scr, st);
  int64_t n_edges = 0;
  cudaMemcpyAsync(&n_edges, up + N, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
  cudaError_t ce = cudaStreamSynchronize(st);
  if (ce != cudaSuccess) {
    cleanup();
    return cuda_fail(ce, "order lifting");
  }
  LiftFaces fc;
  if (p->dim == 3 && nfi > 0 && nE > 0) {
    // faces: per lowest vertex, sorted unique keys (positions of the other two in its row)
    if (p->max_row > 32767) {
      cleanup();
      return fail(LFEM_E_TOO_LARGE, "a CSR row is too long for the face keys");
    }
    int32_t *fcnt = nullptr, *foff = nullptr, *fcur = nullptr, *fkeys = nullptr, *fuid = nullptr, *fscr = nullptr,
            *sort_scr = nullptr, *mx = nullptr;
    int64_t *fbase = nullptr, *fscr64 = nullptr;
    LIFT_TRY(alloc32(&fcnt, (int64_t)N + 1));
    LIFT_TRY(alloc32(&foff, (int64_t)N + 1));
    LIFT_TRY(alloc32(&fcur, (int64_t)N + 1));
    LIFT_TRY(alloc32(&fkeys, 4 * nE));
    LIFT_TRY(alloc32(&fuid, 4 * nE));
    LIFT_TRY(alloc32(&fscr, scan_scratch_bytes((int64_t)N + 1, 4) / 4));
    LIFT_TRY(alloc32(&sort_scr, (int64_t)N + 2));
    LIFT_TRY(alloc32(&mx, 2));
    LIFT_TRY(alloc64(&fbase, (int64_t)N + 1));
    LIFT_TRY(alloc64(&fscr64, scan_scratch_bytes((int64_t)N + 1, 8) / 8));
    cudaMemsetAsync(fcnt, 0, sizeof(int32_t) * ((size_t)N + 1), st);
    cudaMemsetAsync(fcur, 0, sizeof(int32_t) * ((size_t)N + 1), st);
    cudaMemsetAsync(mx, 0, 2 * sizeof(int32_t), st);
    k_face_count<<<grid_for(nE, 128), 128, 0, st>>>(d.conn, nE, fcnt);
    scan_exclusive<int32_t, int32_t>(fcnt, foff, (int64_t)N, fscr, st);
    k_face_fill<<<grid_for(nE, 128), 128, 0, st>>>(d.conn, nE, d.row_ptr, d.col_idx, foff, fcur, fkeys, d.status);
    if (N > 0) k_max_i32<<<grid_for(N, 256), 256, 0, st>>>(fcnt, N, mx);
    int32_t max_len = 0;
    cudaMemcpyAsync(&max_len, mx, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    ce = cudaStreamSynchronize(st);
    if (ce != cudaSuccess) {
      cleanup();
      return cuda_fail(ce, "order lifting");
    }
    LIFT_TRY(segsort(fkeys, foff, N, 1, max_len, sort_scr, st));
    if (N > 0) k_face_unique<<<grid_for(N, 128), 128, 0, st>>>(fkeys, foff, N, fuid, fcnt);
    scan_exclusive<int32_t, int64_t>(fcnt, fbase, (int64_t)N, fscr64, st);
    cudaMemcpyAsync(&fc.n_faces, fbase + N, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
    ce = cudaGetLastError();
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    if (ce != cudaSuccess) {
      cleanup();
      return cuda_fail(ce, "order lifting");
    }
    fc.off = foff;
    fc.keys = fkeys;
    fc.uid = fuid;
    fc.fbase = fbase;
  }
  const int64_t n_out = (int64_t)N + n_edges * (order - 1) + (p->dim == 2 ? nE * nfi : 0) +
                        (p->dim == 3 ? fc.n_faces * nfi + nE * nci : 0);
  *n_nodes_out = n_out;
  if (n_out >= INT32_MAX) {
    cleanup();
    return fail(LFEM_E_TOO_LARGE, "order-p mesh has too many nodes for int32 indices");
  }
  if (conn_out || coords_out) {
    if (coords_out && N > 0)
      k_lift_corners<<<grid_for((int64_t)N * na, 256), 256, 0, st>>>(coords, (int64_t)N * na, coords_out);
    if (nE > 0)
      k_lift_elements<<<grid_for(nE, 128), 128, 0, st>>>(d.conn, nE, p->dim, na, order, d.row_ptr, d.col_idx, up, cle,
                                                         N, n_edges, fc, coords, conn_out, coords_out, d.status);
    ce = cudaGetLastError();
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);  // scratch is freed below
    if (ce != cudaSuccess) {
      cleanup();
      return cuda_fail(ce, "order lifting");
    }
  }
#undef LIFT_TRY
  cleanup();
  return LFEM_OK;
}

}  // namespace lfem

extern "C" lfem_status lfem_lift_order(lfem_pattern_t p, const double* coords, int ambient, int order,
                                       int32_t* conn_out, double* coords_out, int64_t* n_nodes_out,
                                       void* cuda_stream) {
  if (!p || !n_nodes_out) return lfem::fail(LFEM_E_ARG, "NULL argument");
  if (p->order != 1 || order < 2 || order > 4)
    return lfem::fail(LFEM_E_UNSUPPORTED, "lifting needs an order-1 pattern and order 2..4");
  if (ambient < p->dim || ambient > 3) return lfem::fail(LFEM_E_ARG, "ambient");
  if (coords_out && p->n_nodes > 0 && !coords) return lfem::fail(LFEM_E_ARG, "coords is NULL");
  return lfem::lift_order(p, coords, ambient, order, conn_out, coords_out, n_nodes_out, (cudaStream_t)cuda_stream);
}

extern "C" lfem_status lfem_pattern_csr_noalloc(const int32_t* conn, int64_t n_elem, int32_t n_nodes, int dim,
                                                int order, int64_t* row_ptr, int32_t* col_idx, int64_t col_capacity,
                                                int64_t* nnz, void* cuda_stream) {
  if (n_elem < 0 || n_nodes < 0 || col_capacity < 0) return lfem::fail(LFEM_E_ARG, "negative size");
  if ((n_elem > 0 && !conn) || !row_ptr || (col_capacity > 0 && !col_idx))
    return lfem::fail(LFEM_E_ARG, "NULL argument");
  if (dim < 1 || dim > 3 || (order != 1 && order != 2)) return lfem::fail(LFEM_E_UNSUPPORTED, "dim/order");
  // the incidence key (e << ksh) | a must fit 31 bits (ksh = 4 up to 16 local nodes, else 6)
  const int ksh = lfem::n_ref(dim, order) > 16 ? 6 : 4;
  if (n_elem >= (1ll << (31 - ksh))) return lfem::fail(LFEM_E_TOO_LARGE, "too many elements");
  return lfem::pattern_csr_noalloc(conn, n_elem, n_nodes, dim, order, row_ptr, col_idx, col_capacity, nnz,
                                   (cudaStream_t)cuda_stream);
}

