// One coarsening step (Algorithm 1, Section 3.1), integer only and
// bit-exact: every node picks a hyperedge, nodes that picked the same
// hyperedge merge into one coarse node, hyperedges whose members all merged
// into one coarse node are removed, the rest connect the coarse nodes of
// their members.
#include <cmath>

#include "hnv_internal.cuh"

namespace hnv {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;  // SplitMix64 increment

// SplitMix64 finaliser (Steele, Lea & Flood, OOPSLA 2014).
__host__ __device__ inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// prio_l(e) for the policies of hnv_assign (see hnv.h).
__global__ void priority_kernel(int32_t m, int32_t policy, uint64_t salt,
                                const int32_t* __restrict__ e_ptr, const float* __restrict__ w,
                                const int32_t* __restrict__ orig_e,
                                const uint64_t* __restrict__ explicit_tab,
                                uint64_t* __restrict__ prio) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t h = mix64((uint64_t)e ^ salt);
    uint64_t p = h;
    if (policy == HNV_ASSIGN_LOW_DEGREE) {
      uint64_t sz = (uint64_t)(e_ptr[e + 1] - e_ptr[e]);
      if (sz > 0xFFFFFFull) sz = 0xFFFFFFull;
      p = (sz << 40) | (h >> 24);
    } else if (policy == HNV_ASSIGN_HIGH_WEIGHT) {
      const uint64_t bits = (uint64_t)__float_as_uint(w[e]);
      p = ((0xFFFFFFFFull - bits) << 32) | (h >> 32);
    } else if (policy == HNV_ASSIGN_EXPLICIT) {
      p = explicit_tab[orig_e[e]];
    }
    prio[e] = p;
  }
}

// c(v) = argmin_{e in N(v)} (-score(v, e), prio(e), e), or -1; warp per
// node, lanes stride the CSC row, then a lexicographic min over the warp.
// score is the cosine of the feature rule (per CSC entry), or absent (all
// equal: the featureless rules). Rows longer than kLongRow go to
// `long_rows` for assign_long_kernel (block per row).
constexpr int32_t kLongRow = 4096;
constexpr int kLongThreads = 512;

__device__ __forceinline__ void lex_min(float& bs, uint64_t& bp, int32_t& be, float sc, uint64_t p,
                                        int32_t e) {
  if (sc > bs || (sc == bs && (p < bp || (p == bp && e < be)))) {
    bs = sc;
    bp = p;
    be = e;
  }
}

// ---------------------------------------------------------------------------
// Feature rule (Section 3.1, nodes with features). The cosine decides an
// argmax, so every float step is an explicitly rounded float32 operation
// (no fused multiply-add) in a fixed order; the oracle takes the same steps.
// ---------------------------------------------------------------------------

// out[r] = mean of X rows idx[ptr[r] .. ptr[r+1]) (one thread per (r, dim),
// added in list order, then divided by the count; an empty list gives 0).
__global__ void segment_mean_kernel(int32_t rows, int32_t k, const int32_t* __restrict__ ptr,
                                    const int32_t* __restrict__ idx, const float* __restrict__ X,
                                    float* __restrict__ out) {
  const int64_t total = (int64_t)rows * k;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = t / k;
    const int32_t i = (int32_t)(t - r * k);
    const int32_t b = ptr[r], e = ptr[r + 1];
    float acc = 0.f;
    for (int32_t j = b; j < e; ++j) acc = __fadd_rn(acc, X[(size_t)idx[j] * k + i]);
    out[t] = (e > b) ? __fdiv_rn(acc, (float)(e - b)) : 0.f;
  }
}

// |F[r]| = sqrt(sum_i F[r,i] * F[r,i]), squares added in dimension order.
__global__ void row_norm_kernel(int32_t rows, int32_t k, const float* __restrict__ F,
                                float* __restrict__ out) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < rows;
       r += (int64_t)gridDim.x * blockDim.x) {
    float acc = 0.f;
    for (int32_t i = 0; i < k; ++i) {
      const float x = F[(size_t)r * k + i];
      acc = __fadd_rn(acc, __fmul_rn(x, x));
    }
    out[r] = __fsqrt_rn(acc);
  }
}

// node_of[j] = the node of CSC entry j (warp per node).
__global__ void node_of_kernel(int32_t n, const int32_t* __restrict__ v_ptr,
                               int32_t* __restrict__ node_of) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t v = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); v < n;
       v += warps)
    for (int32_t j = v_ptr[v] + lane; j < v_ptr[v + 1]; j += 32) node_of[j] = (int32_t)v;
}

// score[j] = cos(f(e), f(v)) for CSC entry j = (v, e): f(e).f(v) with the
// products added in dimension order, over |f(e)| |f(v)|; 0 where that
// product is 0 (an undefined cosine).
__global__ void cosine_score_kernel(int64_t nnz, int32_t k, const int32_t* __restrict__ node_of,
                                    const int32_t* __restrict__ v_edges,
                                    const float* __restrict__ X, const float* __restrict__ FE,
                                    const float* __restrict__ nv, const float* __restrict__ ne,
                                    float* __restrict__ score) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < nnz;
       j += (int64_t)gridDim.x * blockDim.x) {
    const int32_t v = node_of[j], e = v_edges[j];
    const float* fv = X + (size_t)v * k;
    const float* fe = FE + (size_t)e * k;
    float dot = 0.f;
    for (int32_t i = 0; i < k; ++i) dot = __fadd_rn(dot, __fmul_rn(fe[i], fv[i]));
    const float den = __fmul_rn(ne[e], nv[v]);
    score[j] = (den > 0.f) ? __fdiv_rn(dot, den) : 0.f;
  }
}

__global__ void assign_kernel(int32_t n, const int32_t* __restrict__ v_ptr,
                              const int32_t* __restrict__ v_edges,
                              const uint64_t* __restrict__ prio, const float* __restrict__ score,
                              int32_t* __restrict__ c, int32_t* __restrict__ long_rows,
                              int32_t* __restrict__ n_long) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t v = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); v < n;
       v += warps) {
    const int64_t b = v_ptr[v], end = v_ptr[v + 1];
    if (end - b > kLongRow) {
      if (lane == 0) long_rows[atomicAdd(n_long, 1)] = (int32_t)v;
      continue;
    }
    float bs = -INFINITY;
    uint64_t bp = ~0ull;
    int32_t be = 0x7fffffff;
    for (int64_t k = b + lane; k < end; k += 32) {
      const int32_t e = v_edges[k];
      lex_min(bs, bp, be, score ? score[k] : 0.f, prio[e], e);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float os = __shfl_xor_sync(FULL, bs, o);
      const uint64_t op = __shfl_xor_sync(FULL, bp, o);
      const int32_t oe = __shfl_xor_sync(FULL, be, o);
      lex_min(bs, bp, be, os, op, oe);
    }
    if (lane == 0) c[v] = (end > b) ? be : -1;
  }
}

__global__ void __launch_bounds__(kLongThreads)
assign_long_kernel(const int32_t* __restrict__ long_rows, const int32_t* __restrict__ n_long,
                   const int32_t* __restrict__ v_ptr, const int32_t* __restrict__ v_edges,
                   const uint64_t* __restrict__ prio, const float* __restrict__ score,
                   int32_t* __restrict__ c) {
  __shared__ float ss[kLongThreads / 32];
  __shared__ uint64_t sp[kLongThreads / 32];
  __shared__ int32_t se[kLongThreads / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int32_t count = *n_long;
  for (int32_t i = blockIdx.x; i < count; i += gridDim.x) {
    const int32_t v = long_rows[i];
    const int64_t b = v_ptr[v], end = v_ptr[v + 1];
    float bs = -INFINITY;
    uint64_t bp = ~0ull;
    int32_t be = 0x7fffffff;
    // four incidences per step keep four independent load chains in flight
    // (the minimum of a total order does not depend on the visiting order)
    int64_t k = b + threadIdx.x;
    for (; k + 3 * kLongThreads < end; k += 4 * kLongThreads) {
      int32_t e[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) e[u] = v_edges[k + u * kLongThreads];
      uint64_t pr[4];
      float sc[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        pr[u] = prio[e[u]];
        sc[u] = score ? score[k + u * kLongThreads] : 0.f;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) lex_min(bs, bp, be, sc[u], pr[u], e[u]);
    }
    for (; k < end; k += kLongThreads) {
      const int32_t e = v_edges[k];
      lex_min(bs, bp, be, score ? score[k] : 0.f, prio[e], e);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float os = __shfl_xor_sync(FULL, bs, o);
      const uint64_t op = __shfl_xor_sync(FULL, bp, o);
      const int32_t oe = __shfl_xor_sync(FULL, be, o);
      lex_min(bs, bp, be, os, op, oe);
    }
    if (lane == 0) {
      ss[w] = bs;
      sp[w] = bp;
      se[w] = be;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int q = 1; q < kLongThreads / 32; ++q) lex_min(bs, bp, be, ss[q], sp[q], se[q]);
      c[v] = be;
    }
    __syncthreads();
  }
}

__global__ void iota_kernel(int64_t n, int32_t* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (int32_t)i;
}

// key(v) = c(v) or m + v; flags[key] = 1 (all writers store the same value).
__global__ void mark_keys_kernel(int32_t n, int32_t m, const int32_t* __restrict__ c,
                                 int32_t* __restrict__ flags) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t cv = c[v];
    flags[cv >= 0 ? (int64_t)cv : (int64_t)m + v] = 1;
  }
}

__global__ void rep_v_kernel(int32_t n, int32_t m, const int32_t* __restrict__ c,
                             const int32_t* __restrict__ rank, int32_t* __restrict__ rep_v) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t cv = c[v];
    rep_v[v] = rank[cv >= 0 ? (int64_t)cv : (int64_t)m + v];
  }
}

// key = (e << 32) | rep_v[member], warp per hyperedge.
__global__ void pack_image_keys(int32_t m, const int32_t* __restrict__ e_ptr,
                                const int32_t* __restrict__ e_nodes,
                                const int32_t* __restrict__ rep_v, uint64_t* __restrict__ keys) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t e = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); e < m;
       e += warps) {
    const int64_t b = e_ptr[e], end = e_ptr[e + 1];
    for (int64_t k = b + lane; k < end; k += 32)
      keys[k] = ((uint64_t)(uint32_t)e << 32) | (uint32_t)rep_v[e_nodes[k]];
  }
}

__global__ void max_row_len(int32_t rows, const int32_t* __restrict__ ptr, int32_t* __restrict__ out) {
  int32_t mx = 0;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < rows;
       r += (int64_t)gridDim.x * blockDim.x)
    mx = max(mx, ptr[r + 1] - ptr[r]);
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(FULL, mx, o));
  if ((threadIdx.x & 31) == 0 && mx) atomicMax(out, mx);
}

__global__ void image_first_kernel(const uint64_t* __restrict__ keys, int64_t n,
                                   int32_t* __restrict__ first, int32_t* __restrict__ img_size) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    const bool f = (k == 0 || keys[k] != keys[k - 1]);
    first[k] = f ? 1 : 0;
    if (f) atomicAdd(&img_size[(uint32_t)(keys[k] >> 32)], 1);
  }
}

__global__ void keep_kernel(int32_t m, const int32_t* __restrict__ img_size,
                            int32_t* __restrict__ keep) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x)
    keep[e] = img_size[e] >= 2 ? 1 : 0;
}

// Entries of surviving hyperedges: flag2 = first && keep[row]. Removed
// hyperedges (image of size 1) record -1 - c in rep_e.
__global__ void survivor_entries(const uint64_t* __restrict__ keys, int64_t n,
                                 const int32_t* __restrict__ first, const int32_t* __restrict__ keep,
                                 int32_t* __restrict__ flag2, int32_t* __restrict__ rep_e) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t key = keys[k];
    const uint32_t e = (uint32_t)(key >> 32);
    const int32_t f = first[k];
    const int32_t kp = keep[e];
    flag2[k] = (f && kp) ? 1 : 0;
    if (f && !kp) rep_e[e] = -1 - (int32_t)(uint32_t)key;
  }
}

__global__ void scatter_survivors(const uint64_t* __restrict__ keys, int64_t n,
                                  const int32_t* __restrict__ flag2, const int32_t* __restrict__ pos,
                                  int32_t* __restrict__ e_nodes2) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    if (flag2[k]) e_nodes2[pos[k]] = (int32_t)(uint32_t)keys[k];
}

// Per fine hyperedge: survivors get their new ID in rep_e and carry their
// size, weight and level-0 ID to the coarse level.
__global__ void survivor_rows(int32_t m, const int32_t* __restrict__ keep,
                              const int32_t* __restrict__ new_id,
                              const int32_t* __restrict__ img_size, const float* __restrict__ w,
                              const int32_t* __restrict__ orig_e, int32_t* __restrict__ rep_e,
                              int32_t* __restrict__ size2, float* __restrict__ w2,
                              int32_t* __restrict__ orig2) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x) {
    if (!keep[e]) continue;
    const int32_t r = new_id[e];
    rep_e[e] = r;
    size2[r] = img_size[e];
    w2[r] = w[e];
    orig2[r] = orig_e[e];
  }
}

}  // namespace

int coarsen_step(hnv_graph* g, int level, const hnv_coarsen_params* p,
                 const uint64_t* d_explicit, Level* fine, Level* coarse) {
  NvtxRange nvtx("hnv coarsen level %d", level);
  cudaStream_t s = g->stream;
  const int32_t n = fine->n, m = fine->m;
  const int64_t nnz = fine->nnz;
  TempPool pool(s);

  // 1. AssignHyperedge for every node
  uint64_t* prio = nullptr;
  int32_t* c = nullptr;
  HNV_CHECK(pool.get(&prio, (size_t)m));
  HNV_CHECK(pool.get(&c, (size_t)n));
  const uint64_t salt = mix64(p->seed + (uint64_t)level * kGamma);
  HNV_CHECK(launch("priority", priority_kernel, grid_for(m, 256), 256, 0, s, m, p->policy, salt,
                   (const int32_t*)fine->e_ptr, (const float*)fine->w,
                   (const int32_t*)fine->orig_e, d_explicit, prio));
  // the feature rule: a cosine per CSC entry
  float* score = nullptr;
  const int32_t k = fine->feat_k;
  if (p->policy == HNV_ASSIGN_COSINE) {
    if (!fine->feat || k < 1) HNV_FAIL(HNV_ERR_STATE, "level %d has no node features", level);
    float *fe = nullptr, *nv = nullptr, *ne = nullptr;
    int32_t* node_of = nullptr;
    HNV_CHECK(pool.get(&fe, (size_t)m * k));
    HNV_CHECK(pool.get(&nv, (size_t)n));
    HNV_CHECK(pool.get(&ne, (size_t)m));
    HNV_CHECK(pool.get(&node_of, (size_t)nnz));
    HNV_CHECK(pool.get(&score, (size_t)nnz));
    HNV_CHECK(launch("edge_features", segment_mean_kernel, grid_for((int64_t)m * k, 256), 256, 0,
                     s, m, k, (const int32_t*)fine->e_ptr, (const int32_t*)fine->e_nodes,
                     (const float*)fine->feat, fe));
    HNV_CHECK(launch("node_norms", row_norm_kernel, grid_for(n, 256), 256, 0, s, n, k,
                     (const float*)fine->feat, nv));
    HNV_CHECK(launch("edge_norms", row_norm_kernel, grid_for(m, 256), 256, 0, s, m, k,
                     (const float*)fe, ne));
    HNV_CHECK(launch("node_of", node_of_kernel, grid_for((int64_t)n * 32, 256), 256, 0, s, n,
                     (const int32_t*)fine->v_ptr, node_of));
    HNV_CHECK(launch("cosine_score", cosine_score_kernel, grid_for(nnz, 256), 256, 0, s, nnz, k,
                     (const int32_t*)node_of, (const int32_t*)fine->v_edges,
                     (const float*)fine->feat, (const float*)fe, (const float*)nv,
                     (const float*)ne, score));
  }
  int32_t *long_rows = nullptr, *n_long = nullptr;
  HNV_CHECK(pool.get(&long_rows, (size_t)(nnz / kLongRow + 1)));
  HNV_CHECK(pool.get(&n_long, 1));
  HNV_CUDA(cudaMemsetAsync(n_long, 0, sizeof(int32_t), s));
  HNV_CHECK(launch("assign", assign_kernel, grid_for((int64_t)n * 32, 256), 256, 0, s, n,
                   (const int32_t*)fine->v_ptr, (const int32_t*)fine->v_edges,
                   (const uint64_t*)prio, (const float*)score, c, long_rows, n_long));
  HNV_CHECK(launch("assign_long", assign_long_kernel, (unsigned)(2 * num_sms()), kLongThreads, 0,
                   s, (const int32_t*)long_rows, (const int32_t*)n_long,
                   (const int32_t*)fine->v_ptr, (const int32_t*)fine->v_edges,
                   (const uint64_t*)prio, (const float*)score, c));

  // 2. Merge: coarse IDs are the ranks of the keys c(v) / m + v
  int32_t* rank = nullptr;
  const int64_t nkeys = (int64_t)m + n;
  HNV_CHECK(pool.get(&rank, (size_t)nkeys));
  HNV_CUDA(cudaMemsetAsync(rank, 0, sizeof(int32_t) * nkeys, s));
  HNV_CHECK(launch("mark_keys", mark_keys_kernel, grid_for(n, 256), 256, 0, s, n, m,
                   (const int32_t*)c, rank));
  HNV_CHECK(exclusive_scan_i32(rank, rank, nkeys, g->d_buf, s));
  HNV_CUDA(cudaMemsetAsync(g->d_buf + 1, 0, sizeof(int32_t), s));
  HNV_CHECK(launch("max_row_len", max_row_len, grid_for(m, 256), 256, 0, s, m,
                   (const int32_t*)fine->e_ptr, g->d_buf + 1));
  int32_t nm[2];
  HNV_CHECK(read_ints(g, g->d_buf, 2, nm, s));
  const int32_t n2 = nm[0], max_e_len = nm[1];
  HNV_CHECK(level_alloc(fine, (void**)&fine->rep_v, sizeof(int32_t) * (size_t)n, s));
  HNV_CHECK(level_alloc(fine, (void**)&fine->rep_e, sizeof(int32_t) * (size_t)m, s));
  HNV_CHECK(launch("rep_v", rep_v_kernel, grid_for(n, 256), 256, 0, s, n, m, (const int32_t*)c,
                   (const int32_t*)rank, fine->rep_v));

  // 3. Images of the hyperedges: sorted distinct rep_v of the members
  uint64_t *k0 = nullptr, *k1 = nullptr, *sorted = nullptr;
  int32_t *first = nullptr, *img_size = nullptr, *keep = nullptr, *new_id = nullptr;
  HNV_CHECK(pool.get(&k0, (size_t)nnz));
  HNV_CHECK(pool.get(&k1, (size_t)nnz));
  HNV_CHECK(launch("pack_image_keys", pack_image_keys, grid_for((int64_t)m * 32, 256), 256, 0, s,
                   m, (const int32_t*)fine->e_ptr, (const int32_t*)fine->e_nodes,
                   (const int32_t*)fine->rep_v, k0));
  // the keys were packed hyperedge by hyperedge: sorting every hyperedge's
  // run by its low word gives what a full sort by (e, rep) would
  if (max_e_len <= kSegSortMax) {
    HNV_CHECK(segmented_sort_low32(m, fine->e_ptr, (const int64_t*)nullptr, max_e_len, nnz, k0, s,
                                   (uint32_t)n2));
    sorted = k0;
  } else {
    int shifts[16];
    const int np = radix_shifts(bits_for_count(n2), bits_for_count(m), shifts);
    HNV_CHECK(radix_sort_u64(k0, k1, nnz, shifts, np, s, &sorted));
  }
  HNV_CHECK(pool.get(&first, (size_t)nnz));
  HNV_CHECK(pool.get(&img_size, (size_t)m + 1));
  HNV_CHECK(pool.get(&keep, (size_t)m + 1));
  HNV_CHECK(pool.get(&new_id, (size_t)m + 1));
  HNV_CUDA(cudaMemsetAsync(img_size, 0, sizeof(int32_t) * ((size_t)m + 1), s));
  HNV_CHECK(launch("image_first", image_first_kernel, grid_for(nnz, 256), 256, 0, s,
                   (const uint64_t*)sorted, nnz, first, img_size));

  // 4. addHedge: survivors have >= 2 distinct coarse members
  HNV_CHECK(launch("keep", keep_kernel, grid_for(m, 256), 256, 0, s, m,
                   (const int32_t*)img_size, keep));
  HNV_CHECK(exclusive_scan_i32(keep, new_id, m, g->d_buf, s));
  int32_t* flag2 = nullptr;
  int32_t* pos = nullptr;
  HNV_CHECK(pool.get(&flag2, (size_t)nnz));
  HNV_CHECK(pool.get(&pos, (size_t)nnz));
  HNV_CHECK(launch("survivor_entries", survivor_entries, grid_for(nnz, 256), 256, 0, s,
                   (const uint64_t*)sorted, nnz, (const int32_t*)first, (const int32_t*)keep,
                   flag2, fine->rep_e));
  HNV_CHECK(exclusive_scan_i32(flag2, pos, nnz, g->d_buf + 1, s));
  int32_t h[2];
  HNV_CHECK(read_ints(g, g->d_buf, 2, h, s));
  const int32_t m2 = h[0];
  const int32_t nnz2 = h[1];

  // 5. addNode/addEdge: the coarse level's CSR, weights and level-0 IDs
  *coarse = Level();
  coarse->n = n2;
  coarse->m = m2;
  coarse->nnz = nnz2;
  int32_t* size2 = nullptr;
  HNV_CHECK(pool.get(&size2, (size_t)m2 + 1));
  HNV_CHECK(level_alloc(coarse, (void**)&coarse->e_ptr, sizeof(int32_t) * ((size_t)m2 + 1), s));
  HNV_CHECK(level_alloc(coarse, (void**)&coarse->e_nodes, sizeof(int32_t) * (size_t)nnz2, s));
  HNV_CHECK(level_alloc(coarse, (void**)&coarse->w, sizeof(float) * (size_t)m2, s));
  HNV_CHECK(level_alloc(coarse, (void**)&coarse->orig_e, sizeof(int32_t) * (size_t)m2, s));
  HNV_CHECK(launch("scatter_survivors", scatter_survivors, grid_for(nnz, 256), 256, 0, s,
                   (const uint64_t*)sorted, nnz, (const int32_t*)flag2, (const int32_t*)pos,
                   coarse->e_nodes));
  HNV_CUDA(cudaMemsetAsync(size2, 0, sizeof(int32_t) * ((size_t)m2 + 1), s));
  HNV_CHECK(launch("survivor_rows", survivor_rows, grid_for(m, 256), 256, 0, s, m,
                   (const int32_t*)keep, (const int32_t*)new_id, (const int32_t*)img_size,
                   (const float*)fine->w, (const int32_t*)fine->orig_e, fine->rep_e, size2,
                   coarse->w, coarse->orig_e));
  HNV_CHECK(exclusive_scan_i32(size2, coarse->e_ptr, (int64_t)m2 + 1, nullptr, s));

  // 6. The coarse node features (feature rule): the mean of the merged
  // nodes' features, in ascending fine-node order (the CSC of rep_v).
  if (p->policy == HNV_ASSIGN_COSINE) {
    int32_t *iota = nullptr, *ch_ptr = nullptr, *ch_idx = nullptr;
    HNV_CHECK(pool.get(&iota, (size_t)n + 1));
    HNV_CHECK(pool.get(&ch_ptr, (size_t)n2 + 1));
    HNV_CHECK(pool.get(&ch_idx, (size_t)n));
    HNV_CHECK(launch("iota", iota_kernel, grid_for((int64_t)n + 1, 256), 256, 0, s, n + 1, iota));
    HNV_CHECK(transpose_csr(n, n2, n, iota, fine->rep_v, ch_ptr, ch_idx, s));
    HNV_CHECK(level_alloc(coarse, (void**)&coarse->feat, sizeof(float) * (size_t)n2 * k, s));
    coarse->feat_k = k;
    HNV_CHECK(launch("merge_features", segment_mean_kernel, grid_for((int64_t)n2 * k, 256), 256, 0,
                     s, n2, k, (const int32_t*)ch_ptr, (const int32_t*)ch_idx,
                     (const float*)fine->feat, coarse->feat));
  }
  return HNV_OK;
}

}  // namespace hnv
