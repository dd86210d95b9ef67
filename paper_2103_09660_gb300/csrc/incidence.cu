// Level construction: the star-expansion incidence of the input hypergraph
// (Section 1.1) as CSR (hyperedge -> nodes) and CSC (node -> hyperedges) with
// ascending, duplicate-free rows, plus the per-level arrays the refinement
// kernels read (weighted node degrees, 1/|e|, CSC weights) and the split-row
// work plans of both half-sweeps.
#include <algorithm>
#include <cmath>
#include <cstdlib>

#include "hnv_internal.cuh"

namespace hnv {

namespace {

constexpr unsigned FULL = 0xffffffffu;

__global__ void check_ptr_kernel(int32_t m, const int64_t* __restrict__ ptr,
                                 int32_t* __restrict__ err) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t d = ptr[e + 1] - ptr[e];
    if (d < 0) atomicOr(err, ERRBIT_BAD_PTR);
    if (d == 0) atomicOr(err, ERRBIT_EMPTY_EDGE);
    if (e == 0 && ptr[0] != 0) atomicOr(err, ERRBIT_BAD_PTR);
  }
}

// Largest edge_ptr[e+1] - edge_ptr[e] (clamped to 2^30), for choosing the sort.
__global__ void max_len_i64_kernel(int32_t m, const int64_t* __restrict__ ptr,
                                   int32_t* __restrict__ out) {
  int32_t mx = 0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t d = ptr[e + 1] - ptr[e];
    mx = max(mx, (int32_t)(d < ((int64_t)1 << 30) ? d : ((int64_t)1 << 30)));
  }
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0 && mx) atomicMax(out, mx);
}

__global__ void check_weights_kernel(int32_t m, const float* __restrict__ w,
                                     int32_t* __restrict__ err) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x) {
    const float x = w[e];
    if (!(x > 0.f) || !isfinite(x)) atomicOr(err, ERRBIT_BAD_WEIGHT);
  }
}

// key = (e << 32) | node, warp per hyperedge; an out-of-range node sets the
// error bit and is replaced by 0 so the sort stays in bounds.
__global__ void pack_input_keys(int32_t m, int32_t n, const int64_t* __restrict__ ptr,
                                const int32_t* __restrict__ nodes, uint64_t* __restrict__ keys,
                                int32_t* __restrict__ err) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t e = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); e < m;
       e += warps) {
    const int64_t b = ptr[e], end = ptr[e + 1];
    for (int64_t k = b + lane; k < end; k += 32) {
      int32_t v = nodes[k];
      if (v < 0 || v >= n) {
        atomicOr(err, ERRBIT_NODE_RANGE);
        v = 0;
      }
      keys[k] = ((uint64_t)(uint32_t)e << 32) | (uint32_t)v;
    }
  }
}

__global__ void first_flags(const uint64_t* __restrict__ keys, int64_t n, int32_t* __restrict__ f) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    f[k] = (k == 0 || keys[k] != keys[k - 1]) ? 1 : 0;
}

// Unique (row, col) keys -> CSR columns + per-row counts.
__global__ void csr_from_unique(const uint64_t* __restrict__ keys, int64_t n,
                                const int32_t* __restrict__ first, const int32_t* __restrict__ pos,
                                int32_t* __restrict__ cols, int32_t* __restrict__ row_cnt) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    if (!first[k]) continue;
    const uint64_t key = keys[k];
    cols[pos[k]] = (int32_t)(uint32_t)key;
    atomicAdd(&row_cnt[(uint32_t)(key >> 32)], 1);
  }
}

__global__ void iota_kernel(int32_t* p, int32_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = (int32_t)i;
}

__global__ void inv_size_kernel(int32_t m, const int32_t* __restrict__ e_ptr,
                                float* __restrict__ inv) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int32_t d = e_ptr[e + 1] - e_ptr[e];
    inv[e] = d > 0 ? 1.0f / (float)d : 0.0f;
  }
}

__global__ void csc_weights_kernel(int64_t nnz, const int32_t* __restrict__ v_edges,
                                   const float* __restrict__ w, float* __restrict__ v_w) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nnz;
       k += (int64_t)gridDim.x * blockDim.x)
    v_w[k] = w[v_edges[k]];
}

// deg_v[v] = sum of the CSC row's weights: lane-strided partial sums, then a
// fixed xor-shuffle tree (deterministic). Rows longer than kLongRow are
// appended to `long_rows` and left to deg_long_kernel (a warp on a row of
// 10^5 incidences would hold up the whole grid).
constexpr int32_t kLongRow = 4096;

__global__ void deg_kernel(int32_t n, const int32_t* __restrict__ v_ptr,
                           const float* __restrict__ v_w, float* __restrict__ deg,
                           float* __restrict__ inv_deg, int32_t* __restrict__ long_rows,
                           int32_t* __restrict__ n_long) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t v = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); v < n;
       v += warps) {
    const int64_t b = v_ptr[v], e = v_ptr[v + 1];
    if (e - b > kLongRow) {
      if (lane == 0) long_rows[atomicAdd(n_long, 1)] = (int32_t)v;
      continue;
    }
    float s = 0.f;
    for (int64_t k = b + lane; k < e; k += 32) s += v_w[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(FULL, s, o);
    if (lane == 0) {
      deg[v] = s;
      inv_deg[v] = (e > b) ? 1.0f / s : 0.0f;
    }
  }
}

// Block-wide sum in a fixed order: thread-strided partial sums, then a
// shared-memory tree. blockDim.x is kLongThreads.
constexpr int kLongThreads = 512;

__device__ float block_sum_fixed(float x, float* sm) {
  sm[threadIdx.x] = x;
  __syncthreads();
  for (int w = kLongThreads / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sm[threadIdx.x] += sm[threadIdx.x + w];
    __syncthreads();
  }
  const float r = sm[0];
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(kLongThreads)
deg_long_kernel(const int32_t* __restrict__ long_rows, const int32_t* __restrict__ n_long,
                const int32_t* __restrict__ v_ptr, const float* __restrict__ v_w,
                float* __restrict__ deg, float* __restrict__ inv_deg) {
  __shared__ float sm[kLongThreads];
  const int32_t count = *n_long;
  for (int32_t i = blockIdx.x; i < count; i += gridDim.x) {
    const int32_t v = long_rows[i];
    const int64_t b = v_ptr[v], e = v_ptr[v + 1];
    float s = 0.f;
    for (int64_t k = b + threadIdx.x; k < e; k += kLongThreads) s += v_w[k];
    s = block_sum_fixed(s, sm);
    if (threadIdx.x == 0) {
      deg[v] = s;
      inv_deg[v] = 1.0f / s;
    }
  }
}

// Row class for the refinement plan: 0 empty, 1 A (1..a_max), 2 B (..b_max),
// 3 C (..c_max), 4 D (..T), 5 split into at most mid_chunks chunks, 6 split
// into more.
constexpr int kClasses = 7;

__global__ void classify_rows(int32_t rows, const int32_t* __restrict__ ptr, int32_t T,
                              int32_t mid_chunks, PlanShape shape, uint64_t* __restrict__ keys,
                              int32_t* __restrict__ counts) {
  __shared__ int32_t h[kClasses];
  if (threadIdx.x < kClasses) h[threadIdx.x] = 0;
  __syncthreads();
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < rows;
       r += (int64_t)gridDim.x * blockDim.x) {
    const int32_t d = ptr[r + 1] - ptr[r];
    int c;
    if (d == 0) c = 0;
    else if (d <= shape.a_max) c = 1;
    else if (d <= shape.b_max) c = 2;
    else if (d <= shape.c_max) c = 3;
    else if (d <= T) c = 4;
    else c = ((d + T - 1) / T <= mid_chunks) ? 5 : 6;
    keys[r] = ((uint64_t)c << 32) | (uint32_t)r;
    atomicAdd(&h[c], 1);
  }
  __syncthreads();
  if (threadIdx.x < kClasses && h[threadIdx.x]) atomicAdd(&counts[threadIdx.x], h[threadIdx.x]);
}

__global__ void fill_row_items(const uint64_t* __restrict__ keys, int32_t begin, int32_t count,
                               const int32_t* __restrict__ ptr, int4* __restrict__ items) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t r = (int32_t)(uint32_t)keys[begin + i];
    const int32_t b = ptr[r];
    items[i] = make_int4(r, b, ptr[r + 1] - b, -1);
  }
}

// a_members[i] = the (at most 4) neighbours of class-A item i, 0-padded.
__global__ void pack_a_members(const int4* __restrict__ items, int32_t n_a,
                               const int32_t* __restrict__ idx, int4* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_a;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int4 it = items[i];
    const int32_t b = it.y, len = it.z;
    out[i] = make_int4(len > 0 ? idx[b] : 0, len > 1 ? idx[b + 1] : 0, len > 2 ? idx[b + 2] : 0,
                       len > 3 ? idx[b + 3] : 0);
  }
}

// out[16 i + j] = neighbour j of class-B item i (j < its length), else 0.
__global__ void pack_b_members(const int4* __restrict__ items, int32_t n_b,
                               const int32_t* __restrict__ idx, int32_t* __restrict__ out) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < (int64_t)n_b * 16;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t >> 4;
    const int32_t j = (int32_t)(t & 15);
    const int4 it = items[i];
    out[t] = j < it.z ? idx[it.y + j] : 0;
  }
}

__global__ void long_chunk_counts(const uint64_t* __restrict__ keys, int32_t begin, int32_t count,
                                  const int32_t* __restrict__ ptr, int32_t T,
                                  int32_t* __restrict__ nch) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t r = (int32_t)(uint32_t)keys[begin + i];
    nch[i] = (ptr[r + 1] - ptr[r] + T - 1) / T;
  }
}

__global__ void fill_long(const uint64_t* __restrict__ keys, int32_t begin, int32_t count,
                          const int32_t* __restrict__ ptr, int32_t T,
                          const int32_t* __restrict__ chunk_off, int4* __restrict__ long_desc,
                          int4* __restrict__ chunk_items) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t r = (int32_t)(uint32_t)keys[begin + i];
    const int32_t b = ptr[r], e = ptr[r + 1];
    const int32_t c0 = chunk_off[i];
    const int32_t nc = (e - b + T - 1) / T;
    long_desc[i] = make_int4(r, c0, nc, 0);
    for (int32_t j = 0; j < nc; ++j) {
      const int32_t s = b + j * T;
      chunk_items[c0 + j] = make_int4(r, s, min(T, e - s), c0 + j);
    }
  }
}

__global__ void key_rows(const uint64_t* __restrict__ keys, int32_t count, int32_t* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (int32_t)(uint32_t)keys[i];
}

}  // namespace

int level_alloc(Level* lv, void** p, size_t bytes, cudaStream_t s) {
  HNV_CHECK(dev_alloc(p, bytes, s));
  lv->owned.push_back(*p);
  return HNV_OK;
}

void free_level(Level* lv, cudaStream_t s) {
  for (void* p : lv->owned) dev_free(p, s);
  lv->owned.clear();
  for (int side = 0; side < 2; ++side) {
    for (void* p : lv->panel_owned[side]) dev_free(p, s);
    lv->panel_owned[side].clear();
  }
  *lv = Level();
}

int read_ints(hnv_graph* g, const int32_t* d_src, int count, int32_t* host_out, cudaStream_t s) {
  HNV_CUDA(cudaMemcpyAsync(g->h_buf, d_src, sizeof(int32_t) * count, cudaMemcpyDeviceToHost, s));
  HNV_CUDA(cudaStreamSynchronize(s));
  for (int i = 0; i < count; ++i) host_out[i] = g->h_buf[i];
  return HNV_OK;
}

int read_and_clear_err(hnv_graph* g, cudaStream_t s, int32_t* bits) {
  HNV_CHECK(read_ints(g, g->d_err, 1, bits, s));
  HNV_CUDA(cudaMemsetAsync(g->d_err, 0, sizeof(int32_t), s));
  return HNV_OK;
}

static int owned_alloc(std::vector<void*>* owned, void** p, size_t bytes, cudaStream_t s) {
  HNV_CHECK(dev_alloc(p, bytes, s));
  owned->push_back(*p);
  return HNV_OK;
}

int build_split_plan(hnv_graph* g, std::vector<void*>* owned, const int32_t* ptr, int32_t rows,
                     SplitPlan* plan, cudaStream_t s, const PlanShape& shape,
                     const int32_t* idx) {
  *plan = SplitPlan();
  const int32_t T = plan->T;
  if (rows == 0) return HNV_OK;
  TempPool pool(s);
  uint64_t *k0 = nullptr, *k1 = nullptr, *sorted = nullptr;
  HNV_CHECK(pool.get(&k0, (size_t)rows));
  HNV_CHECK(pool.get(&k1, (size_t)rows));
  int32_t* cnt = g->d_buf;
  HNV_CUDA(cudaMemsetAsync(cnt, 0, 16 * sizeof(int32_t), s));
  HNV_CHECK(launch("classify_rows", classify_rows, grid_for(rows, 256), 256, 0, s, rows, ptr, T,
                   kMidChunks, shape, k0, cnt));
  const int shift = 32;
  HNV_CHECK(radix_sort_u64(k0, k1, rows, &shift, 1, s, &sorted));   // stable: rows ascend per class
  int32_t c[kClasses];
  HNV_CHECK(read_ints(g, cnt, kClasses, c, s));
  int32_t off[kClasses + 1] = {0};
  for (int i = 0; i < kClasses; ++i) off[i + 1] = off[i] + c[i];
  plan->n_zero = c[0];
  plan->n_a = c[1];
  plan->n_b = c[2];
  plan->n_c = c[3];
  plan->n_d = c[4];
  plan->n_mid = c[5];
  plan->n_huge = c[6];
  const int32_t n_rows_items = c[1] + c[2] + c[3] + c[4];
  const int32_t n_long = c[5] + c[6];
  int32_t* chunk_off = nullptr;
  if (n_long > 0) {
    HNV_CHECK(pool.get(&chunk_off, (size_t)n_long));
    HNV_CHECK(launch("long_chunk_counts", long_chunk_counts, grid_for(n_long, 256), 256, 0, s,
                     (const uint64_t*)sorted, off[5], n_long, ptr, T, chunk_off));
    HNV_CHECK(exclusive_scan_i32(chunk_off, chunk_off, n_long, cnt + 8, s));
    HNV_CHECK(read_ints(g, cnt + 8, 1, &plan->n_chunks, s));
  }
  const int64_t n_items = (int64_t)n_rows_items + plan->n_chunks;
  if (n_items > 0)
    HNV_CHECK(owned_alloc(owned, (void**)&plan->items, sizeof(int4) * (size_t)n_items, s));
  if (n_rows_items > 0)
    HNV_CHECK(launch("fill_row_items", fill_row_items, grid_for(n_rows_items, 256), 256, 0, s,
                     (const uint64_t*)sorted, off[1], n_rows_items, ptr, plan->items));
  if (n_long > 0) {
    HNV_CHECK(owned_alloc(owned, (void**)&plan->long_desc, sizeof(int4) * (size_t)n_long, s));
    HNV_CHECK(launch("fill_long", fill_long, grid_for(n_long, 256), 256, 0, s,
                     (const uint64_t*)sorted, off[5], n_long, ptr, T, (const int32_t*)chunk_off,
                     plan->long_desc, plan->items + n_rows_items));
  }
  if (idx && shape.a_max <= 4 && plan->n_a > 0) {
    HNV_CHECK(owned_alloc(owned, (void**)&plan->a_members, sizeof(int4) * (size_t)plan->n_a, s));
    HNV_CHECK(launch("pack_a_members", pack_a_members, grid_for(plan->n_a, 256), 256, 0, s,
                     (const int4*)plan->items, plan->n_a, idx, plan->a_members));
  }
  if (idx && shape.b_max <= 16 && plan->n_b > 0) {
    HNV_CHECK(owned_alloc(owned, (void**)&plan->b_members,
                          sizeof(int32_t) * 16 * (size_t)plan->n_b, s));
    HNV_CHECK(launch("pack_b_members", pack_b_members, grid_for((int64_t)plan->n_b * 16, 256), 256,
                     0, s, (const int4*)(plan->items + plan->n_a), plan->n_b, idx,
                     plan->b_members));
  }
  if (plan->n_zero > 0) {
    HNV_CHECK(owned_alloc(owned, (void**)&plan->zero_rows, sizeof(int32_t) * (size_t)plan->n_zero, s));
    HNV_CHECK(launch("key_rows", key_rows, grid_for(plan->n_zero, 256), 256, 0, s,
                     (const uint64_t*)sorted, plan->n_zero, plan->zero_rows));
  }
  return HNV_OK;
}

// ---------------------------------------------------------------------------
// Panel plans
// ---------------------------------------------------------------------------

namespace {

// First position in idx[lo, hi) (ascending) whose value is >= key.
__device__ __forceinline__ int32_t lower_bound_i32(const int32_t* __restrict__ idx, int32_t lo,
                                                   int32_t hi, int64_t key) {
  while (lo < hi) {
    const int32_t mid = lo + ((hi - lo) >> 1);
    if ((int64_t)idx[mid] < key) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// Start of panel p of row [beg, end): panels split the neighbour IDs
// [0, cols) into P ranges [p*cols/P, (p+1)*cols/P).
__device__ __forceinline__ int32_t panel_cut(const int32_t* __restrict__ idx, int32_t beg,
                                             int32_t end, int32_t cols, int32_t P, int32_t p) {
  if (p <= 0) return beg;
  if (p >= P) return end;
  return lower_bound_i32(idx, beg, end, (int64_t)p * cols / P);
}

// The long rows of a plan (its D rows, then its split rows) as one list, and
// the sum of their lengths (atomically added to *total).
__global__ void long_rows_list(const int4* __restrict__ d_items, int32_t n_d,
                               const int4* __restrict__ long_desc, int32_t n_long,
                               const int32_t* __restrict__ ptr, int32_t* __restrict__ rows_out,
                               int32_t* __restrict__ total) {
  int32_t acc = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (int64_t)n_d + n_long;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t r = i < n_d ? d_items[i].x : long_desc[i - n_d].x;
    rows_out[i] = r;
    acc += ptr[r + 1] - ptr[r];
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0 && acc) atomicAdd(total, acc);
}

// Per listed row i (a warp each; lane p < P owns panel p, P <= 32): work
// items per panel (items_pr[p * R + i]), partial slots (row_chunks[i], 0
// for a row left whole) and whether it is split into at most mid_chunks
// pieces (flags[i]) or more (flags[R + i]).
__global__ void panel_rows(int32_t R, const int32_t* __restrict__ list,
                           const int32_t* __restrict__ ptr, const int32_t* __restrict__ idx,
                           int32_t cols, int32_t P, int32_t T, int32_t mid_chunks,
                           int32_t* __restrict__ items_pr, int32_t* __restrict__ row_chunks,
                           int32_t* __restrict__ flags) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < R;
       i += warps) {
    const int32_t r = list[i];
    const int32_t beg = ptr[r], end = ptr[r + 1];
    const int32_t hi = lane < P ? panel_cut(idx, beg, end, cols, P, lane + 1) : end;
    int32_t lo = __shfl_up_sync(0xffffffffu, hi, 1);
    if (lane == 0) lo = beg;
    const int32_t cp = lane < P ? (hi - lo + T - 1) / T : 0;
    const int32_t c = __reduce_add_sync(0xffffffffu, cp);
    if (lane < P) items_pr[(int64_t)lane * R + i] = cp;
    if (lane == 0) {
      const bool split = c > 1;
      row_chunks[i] = split ? c : 0;
      flags[i] = (split && c <= mid_chunks) ? 1 : 0;
      flags[(int64_t)R + i] = (split && c > mid_chunks) ? 1 : 0;
    }
  }
}

__global__ void panel_fill(int32_t R, const int32_t* __restrict__ list,
                           const int32_t* __restrict__ ptr, const int32_t* __restrict__ idx,
                           int32_t cols, int32_t P, int32_t T,
                           const int32_t* __restrict__ item_off, const int32_t* __restrict__ slot_off,
                           const int32_t* __restrict__ flag_off, int4* __restrict__ items,
                           int4* __restrict__ long_desc) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < R;
       i += warps) {
    const int32_t r = list[i];
    const int32_t beg = ptr[r], end = ptr[r + 1];
    const int32_t hi = lane < P ? panel_cut(idx, beg, end, cols, P, lane + 1) : end;
    int32_t lo = __shfl_up_sync(0xffffffffu, hi, 1);
    if (lane == 0) lo = beg;
    const int32_t cp = lane < P ? (hi - lo + T - 1) / T : 0;
    // pieces of the panels before this lane's (an inclusive scan, minus its own)
    int32_t pre = cp;
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t t = __shfl_up_sync(0xffffffffu, pre, o);
      if (lane >= o) pre += t;
    }
    const int32_t c = __shfl_sync(0xffffffffu, pre, 31);
    pre -= cp;
    const bool split = c > 1;
    if (lane < P && cp > 0) {
      int64_t at = item_off[(int64_t)lane * R + i];
      int32_t slot = split ? slot_off[i] + pre : -1;
      for (int32_t s0 = lo; s0 < hi; s0 += T) {
        items[at++] = make_int4(r, s0, min(T, hi - s0), slot);
        if (split) ++slot;
      }
    }
    if (lane == 0 && split) {
      // mid rows first, then the rest (flag_off[R + i] counts every mid row)
      const bool mid = flag_off[i + 1] != flag_off[i];
      const int64_t pos = mid ? (int64_t)flag_off[i] : (int64_t)flag_off[(int64_t)R + i];
      long_desc[pos] = make_int4(r, slot_off[i], c, 0);
    }
  }
}

// Panels worth cutting the long rows of `base` into, for a neighbour table
// of table_bytes: panels of about 64 MB (half of L2) so that a panel's rows
// stay in L2 while every row piece gathering from it runs, but no more than
// keep pieces at 32 incidences on average (each piece writes and reads one
// partial row), and none at all if the table mostly fits L2 or the panels
// would be larger than L2.
int forced_panels() {
  static int forced = -2;
  if (forced == -2) {
    const char* e = getenv("HNV_PANELS");
    forced = (e && atoi(e) >= 1) ? std::min(atoi(e), 32) : -1;   // a lane per panel
  }
  return forced;
}

constexpr int64_t kPanelMinTable = 96000000;   // below: the table mostly stays in L2

int choose_panels(int64_t table_bytes, int64_t long_rows, int64_t long_nnz) {
  if (long_rows == 0) return 1;
  if (forced_panels() > 0) return forced_panels();
  if (table_bytes <= kPanelMinTable) return 1;
  const int64_t target = (table_bytes + (int64_t)64e6 - 1) / (int64_t)64e6;
  const int64_t by_length = long_nnz / (32 * long_rows);
  const int64_t P = std::min<int64_t>(std::min(target, by_length), 32);
  if (P < 2 || table_bytes / P > (int64_t)160e6) return 1;
  return (int)P;
}

}  // namespace

int build_panel_plan(hnv_graph* g, std::vector<void*>* owned, const SplitPlan& base,
                     const int32_t* ptr, const int32_t* idx, int32_t cols, int64_t table_bytes,
                     SplitPlan* plan, int* panels, cudaStream_t s) {
  *panels = 1;
  const int32_t R = base.n_d + base.n_mid + base.n_huge;
  if (R == 0 || (forced_panels() < 1 && table_bytes <= kPanelMinTable)) return HNV_OK;
  const int32_t T = base.T;
  TempPool pool(s);
  int32_t* list = nullptr;
  HNV_CHECK(pool.get(&list, (size_t)R));
  int32_t* cnt = g->d_buf;
  HNV_CUDA(cudaMemsetAsync(cnt, 0, 4 * sizeof(int32_t), s));
  const int32_t n_short = base.n_a + base.n_b + base.n_c;
  HNV_CHECK(launch("long_rows_list", long_rows_list, grid_for(R, 256), 256, 0, s,
                   (const int4*)(base.items + n_short), base.n_d, (const int4*)base.long_desc,
                   base.n_mid + base.n_huge, ptr, list, cnt));
  int32_t long_nnz = 0;
  HNV_CHECK(read_ints(g, cnt, 1, &long_nnz, s));
  const int P = choose_panels(table_bytes, R, long_nnz);
  if (P <= 1) return HNV_OK;
  if ((int64_t)P * R + 1 > (int64_t)INT32_MAX)
    HNV_FAIL(HNV_ERR_TOO_LARGE, "panel plan: %d panels over %d rows", P, R);

  const int64_t npr = (int64_t)P * R;
  int32_t *items_pr = nullptr, *row_chunks = nullptr, *flags = nullptr;
  HNV_CHECK(pool.get(&items_pr, (size_t)npr));
  HNV_CHECK(pool.get(&row_chunks, (size_t)R));
  HNV_CHECK(pool.get(&flags, 2 * (size_t)R + 1));
  HNV_CHECK(launch("panel_rows", panel_rows, grid_for((int64_t)R * 32, 256), 256, 0, s, R, (const int32_t*)list,
                   ptr, idx, cols, P, T, kMidChunks, items_pr, row_chunks, flags));
  // each array becomes its exclusive prefix sums in place; totals to d_buf
  HNV_CHECK(exclusive_scan_i32(items_pr, items_pr, npr, cnt + 0, s));
  HNV_CHECK(exclusive_scan_i32(row_chunks, row_chunks, R, cnt + 1, s));
  HNV_CHECK(exclusive_scan_i32(flags, flags, 2 * (int64_t)R, cnt + 2, s));
  HNV_CUDA(cudaMemcpyAsync(cnt + 3, flags + R, sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
  int32_t c[4];
  HNV_CHECK(read_ints(g, cnt, 4, c, s));
  const int32_t n_panel_items = c[0], n_chunks = c[1], n_split = c[2], n_mid = c[3];

  *plan = SplitPlan();
  plan->T = T;
  plan->n_a = base.n_a;
  plan->n_b = base.n_b;
  plan->n_c = base.n_c;
  plan->n_d = n_panel_items - n_chunks;   // long rows left whole
  plan->n_chunks = n_chunks;
  plan->n_mid = n_mid;
  plan->n_huge = n_split - n_mid;
  plan->n_zero = base.n_zero;
  plan->zero_rows = base.zero_rows;       // shared with `base`, which outlives this plan
  plan->a_members = base.a_members;       // the class-A and B items are the base's, in order
  plan->b_members = base.b_members;
  HNV_CHECK(owned_alloc(owned, (void**)&plan->items,
                        sizeof(int4) * ((size_t)n_short + n_panel_items), s));
  if (n_short > 0)
    HNV_CUDA(cudaMemcpyAsync(plan->items, base.items, sizeof(int4) * (size_t)n_short,
                             cudaMemcpyDeviceToDevice, s));
  if (n_split > 0)
    HNV_CHECK(owned_alloc(owned, (void**)&plan->long_desc, sizeof(int4) * (size_t)n_split, s));
  HNV_CHECK(launch("panel_fill", panel_fill, grid_for((int64_t)R * 32, 256), 256, 0, s, R, (const int32_t*)list,
                   ptr, idx, cols, P, T, (const int32_t*)items_pr, (const int32_t*)row_chunks,
                   (const int32_t*)flags, plan->items + n_short, plan->long_desc));
  *panels = P;
  return HNV_OK;
}

int side_plan(hnv_graph* g, Level* lv, int side, size_t row_bytes, const SplitPlan** plan,
              cudaStream_t s) {
  const SplitPlan& base = side == 0 ? lv->planE : lv->planV;
  *plan = &base;
  const int32_t rows = side == 0 ? lv->m : lv->n;
  const int32_t cols = side == 0 ? lv->n : lv->m;
  if (rows == 0 || cols == 0) return HNV_OK;
  if (lv->panel_rb[side] != row_bytes) {
    for (void* p : lv->panel_owned[side]) dev_free(p, s);
    lv->panel_owned[side].clear();
    lv->panel_plan[side] = SplitPlan();
    lv->panel_P[side] = 1;
    int P = 1;
    HNV_CHECK(build_panel_plan(g, &lv->panel_owned[side], base, side == 0 ? lv->e_ptr : lv->v_ptr,
                               side == 0 ? lv->e_nodes : lv->v_edges, cols,
                               (int64_t)cols * (int64_t)row_bytes, &lv->panel_plan[side], &P, s));
    lv->panel_P[side] = P;
    lv->panel_rb[side] = row_bytes;
  }
  if (lv->panel_P[side] > 1) *plan = &lv->panel_plan[side];
  return HNV_OK;
}

int level_weight_arrays(Level* lv, cudaStream_t s) {
  HNV_CHECK(launch("csc_weights", csc_weights_kernel, grid_for(lv->nnz, 256), 256, 0, s, lv->nnz,
                   (const int32_t*)lv->v_edges, (const float*)lv->w, lv->v_w));
  TempPool pool(s);
  int32_t *long_rows = nullptr, *n_long = nullptr;
  HNV_CHECK(pool.get(&long_rows, (size_t)(lv->nnz / kLongRow + 1)));
  HNV_CHECK(pool.get(&n_long, 1));
  HNV_CUDA(cudaMemsetAsync(n_long, 0, sizeof(int32_t), s));
  HNV_CHECK(launch("deg", deg_kernel, grid_for((int64_t)lv->n * 32, 256), 256, 0, s, lv->n,
                   (const int32_t*)lv->v_ptr, (const float*)lv->v_w, lv->deg_v, lv->inv_deg_v,
                   long_rows, n_long));
  return launch("deg_long", deg_long_kernel, (unsigned)(2 * num_sms()), kLongThreads, 0, s,
                (const int32_t*)long_rows, (const int32_t*)n_long, (const int32_t*)lv->v_ptr,
                (const float*)lv->v_w, lv->deg_v, lv->inv_deg_v);
}

int finish_level(hnv_graph* g, Level* lv) {
  cudaStream_t s = g->stream;
  const int32_t n = lv->n, m = lv->m;
  const int64_t nnz = lv->nnz;
  HNV_CHECK(level_alloc(lv, (void**)&lv->v_ptr, sizeof(int32_t) * ((size_t)n + 1), s));
  HNV_CHECK(level_alloc(lv, (void**)&lv->v_edges, sizeof(int32_t) * (size_t)nnz, s));
  HNV_CHECK(transpose_csr(m, n, nnz, lv->e_ptr, lv->e_nodes, lv->v_ptr, lv->v_edges, s));
  HNV_CHECK(level_alloc(lv, (void**)&lv->inv_size_e, sizeof(float) * (size_t)m, s));
  HNV_CHECK(level_alloc(lv, (void**)&lv->v_w, sizeof(float) * (size_t)nnz, s));
  HNV_CHECK(level_alloc(lv, (void**)&lv->deg_v, sizeof(float) * (size_t)n, s));
  HNV_CHECK(level_alloc(lv, (void**)&lv->inv_deg_v, sizeof(float) * (size_t)n, s));
  HNV_CHECK(launch("inv_size", inv_size_kernel, grid_for(m, 256), 256, 0, s, m,
                   (const int32_t*)lv->e_ptr, lv->inv_size_e));
  HNV_CHECK(level_weight_arrays(lv, s));
  HNV_CHECK(build_split_plan(g, &lv->owned, lv->e_ptr, m, &lv->planE, s, PlanShape(),
                             lv->e_nodes));
  HNV_CHECK(build_split_plan(g, &lv->owned, lv->v_ptr, n, &lv->planV, s));
  return HNV_OK;
}

int build_level0(hnv_graph* g, int32_t n, int32_t m, const int64_t* d_edge_ptr,
                 const int32_t* d_edge_nodes, const float* d_w, Level* lv) {
  cudaStream_t s = g->stream;
  *lv = Level();
  lv->n = n;
  lv->m = m;
  // 1. the pointer array must be valid before anything indexes with it
  int64_t nnz_in = 0;
  {
    int64_t h[2] = {0, 0};
    HNV_CUDA(cudaMemcpyAsync(&h[0], d_edge_ptr, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    HNV_CUDA(cudaMemcpyAsync(&h[1], d_edge_ptr + m, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    HNV_CUDA(cudaStreamSynchronize(s));
    if (h[0] != 0) HNV_FAIL(HNV_ERR_INVALID_ARG, "edge_ptr[0] must be 0");
    nnz_in = h[1];
    if (nnz_in < 0) HNV_FAIL(HNV_ERR_INVALID_ARG, "edge_ptr[m] < 0");
    if (nnz_in > (int64_t)0x7fffff00) HNV_FAIL(HNV_ERR_TOO_LARGE, "nnz %lld >= 2^31", (long long)nnz_in);
  }
  HNV_CHECK(launch("check_ptr", check_ptr_kernel, grid_for(m, 256), 256, 0, s, m, d_edge_ptr,
                   g->d_err));
  if (d_w)
    HNV_CHECK(launch("check_weights", check_weights_kernel, grid_for(m, 256), 256, 0, s, m, d_w,
                     g->d_err));
  int32_t bits = 0;
  HNV_CHECK(read_and_clear_err(g, s, &bits));
  if (bits & ERRBIT_BAD_PTR) HNV_FAIL(HNV_ERR_INVALID_ARG, "edge_ptr is not non-decreasing from 0");
  if (bits & ERRBIT_EMPTY_EDGE) HNV_FAIL(HNV_ERR_INVALID_ARG, "a hyperedge has no members");
  if (bits & ERRBIT_BAD_WEIGHT) HNV_FAIL(HNV_ERR_INVALID_ARG, "weights must be finite and > 0");

  // 2. sort (hyperedge, node) keys and drop repeats
  TempPool pool(s);
  uint64_t *k0 = nullptr, *k1 = nullptr, *sorted = nullptr;
  int32_t *first = nullptr, *pos = nullptr, *cnt = nullptr;
  HNV_CHECK(pool.get(&k0, (size_t)nnz_in));
  HNV_CHECK(pool.get(&k1, (size_t)nnz_in));
  HNV_CHECK(launch("pack_input_keys", pack_input_keys, grid_for((int64_t)m * 32, 256), 256, 0, s,
                   m, n, d_edge_ptr, d_edge_nodes, k0, g->d_err));
  HNV_CHECK(read_and_clear_err(g, s, &bits));
  if (bits & ERRBIT_NODE_RANGE) HNV_FAIL(HNV_ERR_OUT_OF_RANGE, "a node ID is outside [0, n)");
  // the keys are grouped by hyperedge already: sorting every hyperedge's run
  // by node gives what a full sort by (e, node) would
  int32_t max_len = 0;
  HNV_CUDA(cudaMemsetAsync(g->d_buf + 40, 0, sizeof(int32_t), s));
  HNV_CHECK(launch("max_len", max_len_i64_kernel, grid_for(m, 256), 256, 0, s, m, d_edge_ptr,
                   g->d_buf + 40));
  HNV_CHECK(read_ints(g, g->d_buf + 40, 1, &max_len, s));
  if (max_len <= kSegSortMax) {
    HNV_CHECK(segmented_sort_low32(m, nullptr, d_edge_ptr, max_len, nnz_in, k0, s, (uint32_t)n));
    sorted = k0;
  } else {
    int shifts[16];
    const int np = radix_shifts(bits_for_count(n), bits_for_count(m), shifts);
    HNV_CHECK(radix_sort_u64(k0, k1, nnz_in, shifts, np, s, &sorted));
  }
  HNV_CHECK(pool.get(&first, (size_t)nnz_in));
  HNV_CHECK(pool.get(&pos, (size_t)nnz_in));
  HNV_CHECK(pool.get(&cnt, (size_t)m + 1));
  HNV_CHECK(launch("first_flags", first_flags, grid_for(nnz_in, 256), 256, 0, s,
                   (const uint64_t*)sorted, nnz_in, first));
  HNV_CHECK(exclusive_scan_i32(first, pos, nnz_in, g->d_buf, s));
  int32_t nnz = 0;
  HNV_CHECK(read_ints(g, g->d_buf, 1, &nnz, s));
  lv->nnz = nnz;
  HNV_CHECK(level_alloc(lv, (void**)&lv->e_ptr, sizeof(int32_t) * ((size_t)m + 1), s));
  HNV_CHECK(level_alloc(lv, (void**)&lv->e_nodes, sizeof(int32_t) * (size_t)nnz, s));
  HNV_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * ((size_t)m + 1), s));
  HNV_CHECK(launch("csr_from_unique", csr_from_unique, grid_for(nnz_in, 256), 256, 0, s,
                   (const uint64_t*)sorted, nnz_in, (const int32_t*)first, (const int32_t*)pos,
                   lv->e_nodes, cnt));
  HNV_CHECK(exclusive_scan_i32(cnt, lv->e_ptr, (int64_t)m + 1, nullptr, s));

  // 3. weights (copy, or all ones) and level-0 IDs
  HNV_CHECK(level_alloc(lv, (void**)&lv->w, sizeof(float) * (size_t)m, s));
  HNV_CHECK(level_alloc(lv, (void**)&lv->orig_e, sizeof(int32_t) * (size_t)m, s));
  if (m > 0) {
    if (d_w) {
      HNV_CUDA(cudaMemcpyAsync(lv->w, d_w, sizeof(float) * m, cudaMemcpyDeviceToDevice, s));
    } else {
      HNV_CHECK(fill_i32(reinterpret_cast<int32_t*>(lv->w), 0x3f800000, m, s));  // 1.0f
    }
    HNV_CHECK(launch("iota", iota_kernel, grid_for(m, 256), 256, 0, s, lv->orig_e, m));
  }
  return finish_level(g, lv);
}

}  // namespace hnv
