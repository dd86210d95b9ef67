// Level construction: the star-expansion incidence of the input hypergraph
// (Section 1.1) as CSR (hyperedge -> nodes) and CSC (node -> hyperedges) with
// ascending, duplicate-free rows, plus the per-level arrays the refinement
// kernels read (weighted node degrees, 1/|e|, CSC weights) and the split-row
// work plans of both half-sweeps.
#include <cmath>

#include "hnv_internal.cuh"

namespace hnv {

// Rows with more incidences than this are split into chunks (see SplitPlan).
constexpr int32_t kSplitT = 128;

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
// fixed xor-shuffle tree (deterministic).
__global__ void deg_kernel(int32_t n, const int32_t* __restrict__ v_ptr,
                           const float* __restrict__ v_w, float* __restrict__ deg,
                           float* __restrict__ inv_deg) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t v = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); v < n;
       v += warps) {
    const int64_t b = v_ptr[v], e = v_ptr[v + 1];
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

__global__ void long_flags_kernel(int32_t rows, const int32_t* __restrict__ ptr, int32_t T,
                                  int32_t* __restrict__ is_long, int32_t* __restrict__ nchunk) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < rows;
       r += (int64_t)gridDim.x * blockDim.x) {
    const int32_t d = ptr[r + 1] - ptr[r];
    const bool l = d > T;
    is_long[r] = l ? 1 : 0;
    nchunk[r] = l ? (d + T - 1) / T : 0;
  }
}

__global__ void fill_plan_kernel(int32_t rows, const int32_t* __restrict__ ptr, int32_t T,
                                 const int32_t* __restrict__ is_long,
                                 const int32_t* __restrict__ long_idx,
                                 const int32_t* __restrict__ chunk_off,
                                 int32_t* __restrict__ long_rows, int32_t* __restrict__ chunk_ptr,
                                 int2* __restrict__ ranges) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < rows;
       r += (int64_t)gridDim.x * blockDim.x) {
    if (!is_long[r]) continue;
    const int32_t i = long_idx[r];
    long_rows[i] = (int32_t)r;
    const int32_t c0 = chunk_off[r];
    chunk_ptr[i] = c0;
    const int32_t b = ptr[r], e = ptr[r + 1];
    int32_t c = c0;
    for (int32_t s = b; s < e; s += T, ++c) ranges[c] = make_int2(s, min(s + T, e));
  }
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

static int build_plan(hnv_graph* g, Level* lv, const int32_t* ptr, int32_t rows, SplitPlan* plan,
                      cudaStream_t s) {
  plan->T = kSplitT;
  TempPool pool(s);
  int32_t *is_long = nullptr, *nchunk = nullptr;
  HNV_CHECK(pool.get(&is_long, (size_t)rows + 1));
  HNV_CHECK(pool.get(&nchunk, (size_t)rows + 1));
  HNV_CHECK(launch("long_flags", long_flags_kernel, grid_for(rows, 256), 256, 0, s, rows, ptr,
                   kSplitT, is_long, nchunk));
  int32_t* tot = g->d_buf;
  HNV_CHECK(exclusive_scan_i32(is_long, is_long, rows, tot, s));   // is_long -> long index
  HNV_CHECK(exclusive_scan_i32(nchunk, nchunk, rows, tot + 1, s)); // nchunk -> chunk offset
  int32_t h[2];
  HNV_CHECK(read_ints(g, tot, 2, h, s));
  plan->n_long = h[0];
  plan->n_chunks = h[1];
  if (plan->n_long == 0) return HNV_OK;
  // the scans overwrote the flags; recompute them into a fresh buffer
  int32_t *flag = nullptr, *dummy = nullptr;
  HNV_CHECK(pool.get(&flag, (size_t)rows + 1));
  HNV_CHECK(pool.get(&dummy, (size_t)rows + 1));
  HNV_CHECK(launch("long_flags", long_flags_kernel, grid_for(rows, 256), 256, 0, s, rows, ptr,
                   kSplitT, flag, dummy));
  HNV_CHECK(level_alloc(lv, (void**)&plan->long_rows, sizeof(int32_t) * plan->n_long, s));
  HNV_CHECK(level_alloc(lv, (void**)&plan->chunk_ptr, sizeof(int32_t) * (plan->n_long + 1), s));
  HNV_CHECK(level_alloc(lv, (void**)&plan->chunk_range, sizeof(int2) * plan->n_chunks, s));
  HNV_CHECK(launch("fill_plan", fill_plan_kernel, grid_for(rows, 256), 256, 0, s, rows, ptr,
                   kSplitT, (const int32_t*)flag, (const int32_t*)is_long,
                   (const int32_t*)nchunk, plan->long_rows, plan->chunk_ptr, plan->chunk_range));
  HNV_CUDA(cudaMemcpyAsync(plan->chunk_ptr + plan->n_long, &tot[1], sizeof(int32_t),
                           cudaMemcpyDeviceToDevice, s));
  return HNV_OK;
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
  HNV_CHECK(launch("csc_weights", csc_weights_kernel, grid_for(nnz, 256), 256, 0, s, nnz,
                   (const int32_t*)lv->v_edges, (const float*)lv->w, lv->v_w));
  HNV_CHECK(launch("deg", deg_kernel, grid_for((int64_t)n * 32, 256), 256, 0, s, n,
                   (const int32_t*)lv->v_ptr, (const float*)lv->v_w, lv->deg_v, lv->inv_deg_v));
  HNV_CHECK(build_plan(g, lv, lv->e_ptr, m, &lv->planE, s));
  HNV_CHECK(build_plan(g, lv, lv->v_ptr, n, &lv->planV, s));
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
  int shifts[16];
  const int np = radix_shifts(bits_for_count(n), bits_for_count(m), shifts);
  HNV_CHECK(radix_sort_u64(k0, k1, nnz_in, shifts, np, s, &sorted));
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
