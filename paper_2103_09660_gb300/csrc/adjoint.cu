// Reverse mode of the two-phase V-cycle (float32): gradients of a loss with
// respect to the level-0 hyperedge weights and the coarsest embedding, given
// the gradient with respect to the level-0 output rows.
//
// Forward, per sweep (Algorithm 2, Section 3.3, two-phase order):
//   z_e^i = (1-w) z_e^{i-1} + w (1/|e|) sum_{v in e} z_v^{i-1}
//   z_v^i = (1-w) z_v^{i-1} + w s_v / D_v,  s_v = sum_{e ∋ v} w_e z_e^i,
//                                           D_v = sum_{e ∋ v} w_e.
// Reverse, sweep i = k..1 (G_V, G_E: gradients w.r.t. z_v^i, z_e^i):
//   node half-sweep:  a_v = G_V / D_v,  A_e = sum_{v in e} a_v,
//                     dw_e += w (<A_e, z_e^i> - sum_{v in e} <a_v, z~_v>)
//                     (d(s_v/D_v)/dw_e = (z_e - z~_v)/D_v, z~_v = s_v/D_v),
//                     G_E += w w_e A_e,   G_V *= (1-w) on rows with D_v > 0;
//   hyperedge half:   G_V += w sum_{e ∋ v} G_E[e] / |e|,   G_E *= (1-w).
// Projection (a fine row copies a coarse row) reverses to a segmented sum of
// the fine gradients into their coarse row; a level's weights are the level-0
// weights of their hyperedges (orig_e), so dw accumulates into dw0.
// Per level, the forward iterates are recomputed from the level's starting
// rows saved by hnv_vcycle_save (per-level checkpointing). The replay keeps,
// per sweep, z_e^i and z~_v = s_v / D_v itself (the node half-sweep's gather
// before the blend), so z~ is never recovered by dividing by w. The factor
// (1-w) of G_E is applied lazily: the next reversed sweep's update of G_E
// takes it as its keep factor, and the level's last one by a scaling pass.
#include <algorithm>
#include <memory>

#include "hnv_internal.cuh"

namespace hnv {

namespace {

constexpr unsigned FULL = 0xffffffffu;

__global__ void table_at_kernel(int64_t nnz, const int32_t* __restrict__ idx,
                                const float* __restrict__ table, float* __restrict__ out) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nnz;
       k += (int64_t)gridDim.x * blockDim.x)
    out[k] = table[idx[k]];
}

__global__ void propagate_weights(int32_t m, const int32_t* __restrict__ orig_e,
                                  const float* __restrict__ w0, float* __restrict__ w) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x)
    w[e] = w0[orig_e[e]];
}

__global__ void check_w_kernel(int32_t m, const float* __restrict__ w, int32_t* __restrict__ err) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x) {
    const float x = w[e];
    if (!(x > 0.f) || !isfinite(x)) atomicOr(err, ERRBIT_BAD_WEIGHT);
  }
}

__global__ void collapsed_flags(int32_t m, const int32_t* __restrict__ rep_e,
                                int32_t* __restrict__ flag) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x)
    flag[e] = rep_e[e] < 0 ? 1 : 0;
}

// keys of the children lists: (coarse node << 32) | child, child = v for a
// fine node, n_f + e for a hyperedge that collapsed into the coarse node
__global__ void children_keys(int32_t n_f, int32_t m_f, const int32_t* __restrict__ rep_v,
                              const int32_t* __restrict__ rep_e, const int32_t* __restrict__ pos,
                              uint64_t* __restrict__ keys) {
  const int64_t total = (int64_t)n_f + m_f;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (i < n_f) {
      keys[i] = ((uint64_t)(uint32_t)rep_v[i] << 32) | (uint32_t)i;
    } else {
      const int64_t e = i - n_f;
      const int32_t r = rep_e[e];
      if (r < 0) keys[n_f + pos[e]] = ((uint64_t)(uint32_t)(-1 - r) << 32) | (uint32_t)i;
    }
  }
}

__global__ void key_counts(const uint64_t* __restrict__ keys, int64_t n, int32_t* __restrict__ cnt,
                           int32_t* __restrict__ low) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    atomicAdd(&cnt[(uint32_t)(keys[i] >> 32)], 1);
    low[i] = (int32_t)(uint32_t)keys[i];
  }
}

// a[v] = inv_deg[v] * G_V[v] and c[v] = <a_v, z~_v>; rows without
// incidences get a = 0, c = 0 (their z~ rows are never written).   (G lanes
// per row, G = 8, 16 or 32; lane-strided partial sums, then a fixed xor tree)
template <int G>
__global__ void node_dot_kernel(int32_t n, int32_t d4, const float4* __restrict__ gv,
                                const float4* __restrict__ zt, const float* __restrict__ inv_deg,
                                float4* __restrict__ a, float* __restrict__ c) {
  const int lane = threadIdx.x & 31;
  const int lg = lane & (G - 1);
  const unsigned mask = G == 32 ? FULL : (((1u << G) - 1u) << (lane & (32 - G)));
  const int64_t groups = (int64_t)gridDim.x * (blockDim.x / G);
  for (int64_t r = (int64_t)blockIdx.x * (blockDim.x / G) + threadIdx.x / G; r < n;
       r += groups) {
    const float s = inv_deg[r];
    float acc = 0.f;
    for (int k = lg; k < d4; k += G) {
      const size_t o = (size_t)r * d4 + k;
      float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
      if (s != 0.f) {
        x = gv[o];
        x = make_float4(s * x.x, s * x.y, s * x.z, s * x.w);
        const float4 y = zt[o];
        acc = fmaf(x.x, y.x, acc);
        acc = fmaf(x.y, y.y, acc);
        acc = fmaf(x.z, y.z, acc);
        acc = fmaf(x.w, y.w, acc);
      }
      a[o] = x;
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(mask, acc, o);
    if (lg == 0) c[r] = acc;
  }
}

// Per hyperedge e (G lanes per row, G = 8, 16 or 32), after A_e = sum_{v in e} a_v:
//   dw[e]  += w (<A_e, z_e> - sum_{v in e} c[v])
//   G_E[e]  = keep * G_E[e] + w w_e A_e
// Hyperedges longer than T take their sum of c from csum (long_csum_kernel):
// a group would otherwise walk thousands of members alone.
template <int G>
__global__ void edge_update_kernel(int32_t m, int32_t d4, const float4* __restrict__ A,
                                   const float4* __restrict__ ze, float4* __restrict__ ge,
                                   const float* __restrict__ w_e, float keep, float omega,
                                   const int32_t* __restrict__ e_ptr,
                                   const int32_t* __restrict__ e_nodes,
                                   const float* __restrict__ c, int32_t T,
                                   const float* __restrict__ csum, float* __restrict__ dw) {
  const int lane = threadIdx.x & 31;
  const int lg = lane & (G - 1);
  const unsigned mask = G == 32 ? FULL : (((1u << G) - 1u) << (lane & (32 - G)));
  const int64_t groups = (int64_t)gridDim.x * (blockDim.x / G);
  for (int64_t e = (int64_t)blockIdx.x * (blockDim.x / G) + threadIdx.x / G; e < m;
       e += groups) {
    const float f = omega * w_e[e];
    float dot = 0.f;
    for (int k = lg; k < d4; k += G) {
      const size_t o = (size_t)e * d4 + k;
      const float4 a = A[o], z = ze[o];
      float4 g = ge[o];
      dot = fmaf(a.x, z.x, dot);
      dot = fmaf(a.y, z.y, dot);
      dot = fmaf(a.z, z.z, dot);
      dot = fmaf(a.w, z.w, dot);
      g.x = fmaf(f, a.x, keep * g.x);
      g.y = fmaf(f, a.y, keep * g.y);
      g.z = fmaf(f, a.z, keep * g.z);
      g.w = fmaf(f, a.w, keep * g.w);
      ge[o] = g;
    }
    const int32_t beg = e_ptr[e], end = e_ptr[e + 1];
    float cs = 0.f;
    if (end - beg > T) {
      if (lg == 0) cs = csum[e];
    } else {
      for (int32_t k = beg + lg; k < end; k += G) cs += c[e_nodes[k]];
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
      dot += __shfl_xor_sync(mask, dot, o);
      cs += __shfl_xor_sync(mask, cs, o);
    }
    if (lg == 0) dw[e] += omega * (dot - cs);
  }
}

// csum[r] = sum_{v in r} c[v] for the split (longer than T) hyperedges of a
// plan: one block per row, thread-strided partial sums, then a fixed tree.
__global__ void long_csum_kernel(const int4* __restrict__ long_desc,
                                 const int32_t* __restrict__ e_ptr,
                                 const int32_t* __restrict__ e_nodes,
                                 const float* __restrict__ c, float* __restrict__ csum) {
  __shared__ float red[32];
  const int32_t r = long_desc[blockIdx.x].x;
  const int32_t beg = e_ptr[r], end = e_ptr[r + 1];
  float acc = 0.f;
  for (int32_t k = beg + (int32_t)threadIdx.x; k < end; k += blockDim.x) acc += c[e_nodes[k]];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    acc = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o);
    if (threadIdx.x == 0) csum[r] = acc;
  }
}

// Z[r] = (1-w) Z[r] + w Zt[r] where cond[r] != 0 (the node half-sweep's
// blend, with z~ kept apart)
__global__ void row_blend_kernel(int32_t rows, int32_t d4, float4* __restrict__ Z,
                                 const float4* __restrict__ Zt, float omega,
                                 const float* __restrict__ cond) {
  const float keep = 1.f - omega;
  const int64_t total = (int64_t)rows * d4;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (cond[i / d4] == 0.f) continue;
    const float4 t = Zt[i];
    float4 z = Z[i];
    z.x = fmaf(keep, z.x, omega * t.x);
    z.y = fmaf(keep, z.y, omega * t.y);
    z.z = fmaf(keep, z.z, omega * t.z);
    z.w = fmaf(keep, z.w, omega * t.w);
    Z[i] = z;
  }
}

// Y[r] *= factor where cond[r] != 0
__global__ void row_scale_kernel(int32_t rows, int32_t d4, float4* __restrict__ Y, float factor,
                                 const float* __restrict__ cond) {
  const int64_t total = (int64_t)rows * d4;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (cond[i / d4] == 0.f) continue;
    float4 y = Y[i];
    y.x *= factor;
    y.y *= factor;
    y.z *= factor;
    y.w *= factor;
    Y[i] = y;
  }
}

// dw0[orig_e[e]] += dw[e]  (orig_e is one-to-one within a level)
__global__ void scatter_orig_kernel(int32_t m, const int32_t* __restrict__ orig_e,
                                    const float* __restrict__ dw, float* __restrict__ dw0) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x)
    dw0[orig_e[e]] += dw[e];
}

// gc_e[rep_e[e]] = ge_f[e] for every surviving fine hyperedge (one-to-one)
__global__ void scatter_kept_kernel(int32_t m_f, int32_t d4, const int32_t* __restrict__ rep_e,
                                    const float4* __restrict__ ge_f, float4* __restrict__ gc_e) {
  const int64_t total = (int64_t)m_f * d4;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = i / d4;
    const int32_t r = rep_e[e];
    if (r >= 0) gc_e[(size_t)r * d4 + (i - e * d4)] = ge_f[i];
  }
}

// Algorithmic bytes of one level of the backward pass, per phase (every
// array a kernel reads or writes counted once per kernel, float32 rows of d):
//   replay, per sweep: the hyperedge gather (node table, previous and new
//     hyperedge rows, CSR indices), the node gather keeping z~ (hyperedge
//     table, z~ rows, CSC indices and weights, 1/D_v), the blend (two reads,
//     one write; all sweeps but the last); once: the checkpoint's node rows
//     copied to the running rows;
//   reverse, per sweep: node_dot (G_V, z~ and a rows; 1/D_v, c), the gather of
//     a (node table, A rows, CSR indices), edge_update (A, z_e, G_E read, G_E
//     written; w, offsets, the members' c, dw read and written), the node-side
//     gather (G_E table, G_V read and written, CSC indices and 1/|e|);
//   projection: G_E's last (1-w), the weight-gradient scatter, and for a level
//     with a coarser one the cleared coarse rows, the children gather and the
//     surviving hyperedges' copy.
struct AdjointBytes {
  double replay = 0, reverse = 0, project = 0;
};

AdjointBytes adjoint_bytes(const Level& lv, const Level* cv, int d, int k) {
  const double r = 4.0 * d, n = lv.n, m = lv.m, nnz = (double)lv.nnz;
  AdjointBytes b;
  if (k > 0) {
    const double gE = r * (n + 2 * m) + 4 * (nnz + 2 * m + 1);
    const double gV = r * (m + n) + 4 * (2 * nnz + 2 * n + 1);
    b.replay = k * (gE + gV) + (k - 1) * (3 * r * n + 4 * n) + 2 * r * n;
    const double dot = 3 * r * n + 8 * n;
    const double gA = r * (n + m) + 4 * (nnz + 2 * m + 1);
    const double upd = 4 * r * m + 4 * (nnz + 5 * m + n);
    const double gN = r * (m + 2 * n) + 4 * (2 * nnz + 2 * n + 1);
    b.reverse = k * (dot + gA + upd + gN) + 4 * m;
    b.project = 2 * r * m + 4 * m;
  }
  b.project += 12 * m;
  if (cv) {
    const double nc = cv->n, mc = cv->m, ch = (double)lv.ch_total;
    b.project += r * (nc + mc) + r * (ch + nc) + 4 * (ch + nc + 1) + 2 * r * mc + 4 * m;
  } else {
    b.project += 2 * r * (n + m);
  }
  return b;
}

// Lanes per row of the row-and-reduction kernels: two float4 of a row per
// lane up to d = 128, so that more rows, and their dependent loads, are in
// flight per SM (measured on the 200K-node differentiation workload at d = 64:
// backward 10.83 ms with 8 lanes per hyperedge against 11.19 ms with 16).
int row_lanes(int d4) { return d4 <= 16 ? 8 : (d4 <= 32 ? 16 : 32); }

int launch_edge_update(int d4, int32_t m, const float4* A, const float4* ze, float4* ge,
                       const float* w, float keep, float omega, const int32_t* e_ptr,
                       const int32_t* e_nodes, const float* c, int32_t T, const float* csum,
                       float* dw, cudaStream_t s) {
  const int G = row_lanes(d4);
  const unsigned grid = grid_for((int64_t)m * G, 256);
  if (G == 8)
    return launch("edge_update", edge_update_kernel<8>, grid, 256, 0, s, m, d4, A, ze, ge, w,
                  keep, omega, e_ptr, e_nodes, c, T, csum, dw);
  if (G == 16)
    return launch("edge_update", edge_update_kernel<16>, grid, 256, 0, s, m, d4, A, ze, ge, w,
                  keep, omega, e_ptr, e_nodes, c, T, csum, dw);
  return launch("edge_update", edge_update_kernel<32>, grid, 256, 0, s, m, d4, A, ze, ge, w, keep,
                omega, e_ptr, e_nodes, c, T, csum, dw);
}

int launch_node_dot(int d4, int32_t n, const float4* gv, const float4* zt, const float* inv_deg,
                    float4* a, float* c, cudaStream_t s) {
  const int G = row_lanes(d4);
  const unsigned grid = grid_for((int64_t)n * G, 256);
  if (G == 8)
    return launch("node_dot", node_dot_kernel<8>, grid, 256, 0, s, n, d4, gv, zt, inv_deg, a, c);
  if (G == 16)
    return launch("node_dot", node_dot_kernel<16>, grid, 256, 0, s, n, d4, gv, zt, inv_deg, a, c);
  return launch("node_dot", node_dot_kernel<32>, grid, 256, 0, s, n, d4, gv, zt, inv_deg, a, c);
}

// Per-level arrays of the adjoint: per-incidence 1/|e| (CSC order; the sizes
// do not depend on the weights), and the children lists of the next level's
// nodes.
int prepare_level_adjoint(hnv_graph* g, int level, cudaStream_t s) {
  Level& lv = g->levels[level];
  if (!lv.v_invsize_w) {
    HNV_CHECK(level_alloc(&lv, (void**)&lv.v_invsize_w, sizeof(float) * (size_t)(lv.nnz + 1), s));
    HNV_CHECK(launch("table_at", table_at_kernel, grid_for(lv.nnz, 256), 256, 0, s, lv.nnz,
                     (const int32_t*)lv.v_edges, (const float*)lv.inv_size_e, lv.v_invsize_w));
  }
  if (lv.adj_ready || level + 1 >= (int)g->levels.size()) return HNV_OK;
  const int32_t n_f = lv.n, m_f = lv.m, n_c = g->levels[level + 1].n;
  TempPool pool(s);
  int32_t* pos = nullptr;
  HNV_CHECK(pool.get(&pos, (size_t)m_f + 1));
  HNV_CHECK(launch("collapsed_flags", collapsed_flags, grid_for(m_f, 256), 256, 0, s, m_f,
                   (const int32_t*)lv.rep_e, pos));
  HNV_CHECK(exclusive_scan_i32(pos, pos, m_f, g->d_buf, s));
  int32_t n_col = 0;
  HNV_CHECK(read_ints(g, g->d_buf, 1, &n_col, s));
  const int64_t total = (int64_t)n_f + n_col;
  lv.ch_total = total;
  uint64_t *k0 = nullptr, *k1 = nullptr, *sorted = nullptr;
  int32_t* cnt = nullptr;
  HNV_CHECK(pool.get(&k0, (size_t)total));
  HNV_CHECK(pool.get(&k1, (size_t)total));
  HNV_CHECK(pool.get(&cnt, (size_t)n_c + 1));
  HNV_CHECK(launch("children_keys", children_keys, grid_for((int64_t)n_f + m_f, 256), 256, 0, s,
                   n_f, m_f, (const int32_t*)lv.rep_v, (const int32_t*)lv.rep_e,
                   (const int32_t*)pos, k0));
  int shifts[16];
  const int np = radix_shifts(0, bits_for_count(n_c), shifts);
  HNV_CHECK(radix_sort_u64(k0, k1, total, shifts, np, s, &sorted));
  HNV_CHECK(level_alloc(&lv, (void**)&lv.ch_ptr, sizeof(int32_t) * ((size_t)n_c + 1), s));
  HNV_CHECK(level_alloc(&lv, (void**)&lv.ch_idx, sizeof(int32_t) * (size_t)total, s));
  HNV_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * ((size_t)n_c + 1), s));
  HNV_CHECK(launch("key_counts", key_counts, grid_for(total, 256), 256, 0, s,
                   (const uint64_t*)sorted, total, cnt, lv.ch_idx));
  HNV_CHECK(exclusive_scan_i32(cnt, lv.ch_ptr, (int64_t)n_c + 1, nullptr, s));
  HNV_CHECK(build_split_plan(g, &lv.owned, lv.ch_ptr, n_c, &lv.planC, s));
  lv.adj_ready = true;
  return HNV_OK;
}

int ensure_partials(hnv_graph* g, int d, cudaStream_t s) {
  int64_t chunks = 1;
  for (const Level& lv : g->levels)
    chunks = std::max<int64_t>(chunks, std::max({(int64_t)lv.planE.n_chunks,
                                                 (int64_t)lv.planV.n_chunks,
                                                 (int64_t)lv.planC.n_chunks}));
  const size_t need = sizeof(float) * (size_t)chunks * d;
  if (g->partials && g->partials_bytes >= need) return HNV_OK;
  if (g->partials) dev_free(g->partials, s);
  g->partials = nullptr;
  g->partials_bytes = 0;
  void* p = nullptr;
  HNV_CHECK(dev_alloc(&p, need, s));
  g->partials = static_cast<float*>(p);
  g->partials_bytes = need;
  return HNV_OK;
}

}  // namespace

int set_weights_impl(hnv_graph* g, const float* d_w0, cudaStream_t s) {
  const int32_t m0 = g->levels[0].m;
  if (m0 == 0) return HNV_OK;
  HNV_CHECK(launch("check_w", check_w_kernel, grid_for(m0, 256), 256, 0, s, m0, d_w0, g->d_err));
  int32_t bits = 0;
  HNV_CHECK(read_and_clear_err(g, s, &bits));
  if (bits & ERRBIT_BAD_WEIGHT) HNV_FAIL(HNV_ERR_INVALID_ARG, "weights must be finite and > 0");
  for (Level& lv : g->levels) {
    if (lv.m > 0)
      HNV_CHECK(launch("propagate_weights", propagate_weights, grid_for(lv.m, 256), 256, 0, s, lv.m,
                       (const int32_t*)lv.orig_e, d_w0, lv.w));
    HNV_CHECK(level_weight_arrays(&lv, s));
  }
  return HNV_OK;
}

int vcycle_backward_impl(hnv_graph* g, const float* ckpt, const float* g_v0, const float* g_e0,
                         float* grad_w0, float* grad_zc, int d, float omega, int sweeps,
                         cudaStream_t s) {
  const int L = (int)g->levels.size() - 1;
  const int d4 = d / 4;
  const size_t row = sizeof(float) * (size_t)d;
  for (int l = 0; l <= L; ++l) HNV_CHECK(prepare_level_adjoint(g, l, s));
  HNV_CHECK(ensure_partials(g, d, s));
  // omega == 0: every sweep is the identity, and so is its reverse
  const int rsweeps = omega == 0.f ? 0 : sweeps;
  // checkpoint offsets (floats)
  std::vector<size_t> off(L + 2, 0);
  for (int l = 0; l <= L; ++l)
    off[l + 1] = off[l] + ((size_t)g->levels[l].n + g->levels[l].m) * d;

  TempPool pool(s);
  size_t maxrows = 0, maxm = 1, maxn = 1;
  for (const Level& lv : g->levels) {
    maxrows = std::max(maxrows, (size_t)lv.n + lv.m);
    maxm = std::max(maxm, (size_t)lv.m);
    maxn = std::max(maxn, (size_t)lv.n);
  }
  // states: per sweep i, z~^i (n rows) then z_e^i (m rows); zv: the running
  // node rows of the replay
  float *G = nullptr, *GC = nullptr, *states = nullptr, *zv = nullptr, *A = nullptr, *c = nullptr,
        *dwl = nullptr, *csum = nullptr, *av = nullptr;
  HNV_CHECK(pool.get(&G, maxrows * d));
  HNV_CHECK(pool.get(&GC, maxrows * d));
  HNV_CHECK(pool.get(&states, (size_t)(rsweeps > 0 ? rsweeps : 1) * maxrows * d));
  HNV_CHECK(pool.get(&zv, maxn * d));
  HNV_CHECK(pool.get(&av, maxn * d));
  HNV_CHECK(pool.get(&A, maxm * d));
  HNV_CHECK(pool.get(&c, maxn));
  HNV_CHECK(pool.get(&dwl, maxm));
  HNV_CHECK(pool.get(&csum, maxm));
  const Level& l0 = g->levels[0];
  if (l0.n > 0) {
    if (g_v0) HNV_CUDA(cudaMemcpyAsync(G, g_v0, row * l0.n, cudaMemcpyDeviceToDevice, s));
    else HNV_CUDA(cudaMemsetAsync(G, 0, row * l0.n, s));
  }
  if (l0.m > 0) {
    float* ge = G + (size_t)l0.n * d;
    if (g_e0) HNV_CUDA(cudaMemcpyAsync(ge, g_e0, row * l0.m, cudaMemcpyDeviceToDevice, s));
    else HNV_CUDA(cudaMemsetAsync(ge, 0, row * l0.m, s));
  }
  if (l0.m > 0) HNV_CUDA(cudaMemsetAsync(grad_w0, 0, sizeof(float) * l0.m, s));

  for (int l = 0; l <= L; ++l) {
    const Level& lv = g->levels[l];
    const int32_t n = lv.n, m = lv.m;
    const size_t rows = (size_t)n + m;
    float* gv = G;
    float* ge = G + (size_t)n * d;
    const AdjointBytes by = adjoint_bytes(lv, l < L ? &g->levels[l + 1] : nullptr, d, rsweeps);
    // forward iterates of this level from its checkpoint
    const float* ck_e = ckpt + off[l] + (size_t)n * d;
    std::unique_ptr<PhaseScope> ps(new PhaseScope(HNV_PHASE_ADJOINT_REPLAY, s, by.replay));
    if (rsweeps > 0 && n > 0)
      HNV_CUDA(cudaMemcpyAsync(zv, ckpt + off[l], row * n, cudaMemcpyDeviceToDevice, s));
    for (int i = 1; i <= rsweeps; ++i) {
      float* zt_i = states + (size_t)(i - 1) * rows * d;
      float* ze_i = zt_i + (size_t)n * d;
      if (m > 0)  // z_e^i = (1-w) z_e^{i-1} + w (1/|e|) sum_{v in e} z_v^{i-1}
        HNV_CHECK(gather_rows_f32(lv.planE, lv.e_nodes, nullptr, lv.inv_size_e, zv,
                                  i == 1 ? ck_e : ze_i - rows * d, ze_i, d, 1.f - omega, omega,
                                  g->partials, s, g));
      if (n > 0 && m > 0) {  // z~^i = s_v / D_v, then z_v^i = (1-w) z_v^{i-1} + w z~^i
        HNV_CHECK(gather_rows_f32(lv.planV, lv.v_edges, lv.v_w, lv.inv_deg_v, ze_i, zt_i, zt_i, d,
                                  0.f, 1.f, g->partials, s, g));
        if (i < rsweeps)
          HNV_CHECK(launch("row_blend", row_blend_kernel, grid_for((int64_t)n * d4, 256), 256, 0,
                           s, n, d4, (float4*)zv, (const float4*)zt_i, omega,
                           (const float*)lv.inv_deg_v));
      }
    }
    ps.reset();
    ps.reset(new PhaseScope(HNV_PHASE_ADJOINT_REVERSE, s, by.reverse));
    if (m > 0) HNV_CUDA(cudaMemsetAsync(dwl, 0, sizeof(float) * m, s));
    for (int i = rsweeps; i >= 1; --i) {
      const float* zt_i = states + (size_t)(i - 1) * rows * d;
      const float* ze_i = zt_i + (size_t)n * d;
      // G_E still lacks the (1-w) of the reversed sweep after this one
      const float keep_e = i == rsweeps ? 1.f : 1.f - omega;
      // node half-sweep, reversed
      if (n > 0)  // a_v = G_V/D_v, c_v = <a_v, z~_v>
        HNV_CHECK(launch_node_dot(d4, n, (const float4*)gv, (const float4*)zt_i, lv.inv_deg_v,
                                  (float4*)av, c, s));
      if (m > 0) {
        // the long rows' sums of c run on a side stream, under the gather
        const int32_t n_long = lv.planE.n_mid + lv.planE.n_huge;
        const bool side = n_long > 0 && g->aux[0] && g->aux[1];
        cudaStream_t ls = s;
        if (side) {
          HNV_CUDA(cudaEventRecord(g->fork_ev, s));
          HNV_CUDA(cudaStreamWaitEvent(g->aux[0], g->fork_ev, 0));
          ls = g->aux[0];
        }
        if (n_long > 0)
          HNV_CHECK(launch("long_csum", long_csum_kernel, n_long, 256, 0, ls,
                           (const int4*)lv.planE.long_desc, (const int32_t*)lv.e_ptr,
                           (const int32_t*)lv.e_nodes, (const float*)c, csum));
        // A_e = sum_{v in e} a_v: an unweighted gather, like the forward
        // hyperedge half-sweep (short rows take the packed kernels)
        HNV_CHECK(gather_rows_f32(lv.planE, lv.e_nodes, nullptr, nullptr, av, A, A, d, 0.f, 1.f,
                                  g->partials, s, g));
        if (side) {
          HNV_CUDA(cudaEventRecord(g->join_ev[0], g->aux[0]));
          HNV_CUDA(cudaStreamWaitEvent(s, g->join_ev[0], 0));
        }
        HNV_CHECK(launch_edge_update(d4, m, (const float4*)A, (const float4*)ze_i, (float4*)ge,
                                     lv.w, keep_e, omega, lv.e_ptr, lv.e_nodes, c, lv.planE.T,
                                     csum, dwl, s));
      }
      // G_V *= (1-w) on rows with D_v > 0, then the hyperedge half-sweep,
      // reversed: G_V += w sum_{e ∋ v} G_E[e] / |e|. Rows with D_v > 0 are
      // exactly the rows with incidences, the rows the gather writes.
      if (n > 0 && m > 0)
        HNV_CHECK(gather_rows_f32(lv.planV, lv.v_edges, lv.v_invsize_w, nullptr, ge, gv, gv, d,
                                  1.f - omega, omega, g->partials, s, g));
    }
    ps.reset();
    ps.reset(new PhaseScope(HNV_PHASE_ADJOINT_PROJECT, s, by.project));
    if (rsweeps > 0 && m > 0)  // the last reversed sweep's G_E *= (1-w)
      HNV_CHECK(launch("row_scale", row_scale_kernel, grid_for((int64_t)m * d4, 256), 256, 0, s,
                       m, d4, (float4*)ge, 1.f - omega, (const float*)lv.inv_size_e));
    if (m > 0)
      HNV_CHECK(launch("scatter_orig", scatter_orig_kernel, grid_for(m, 256), 256, 0, s, m,
                       (const int32_t*)lv.orig_e, (const float*)dwl, grad_w0));
    if (l == L) break;
    // projection, reversed: coarse rows collect their children's gradients
    const Level& cv = g->levels[l + 1];
    const size_t crow = (size_t)cv.n + cv.m;
    HNV_CUDA(cudaMemsetAsync(GC, 0, row * crow, s));
    if (cv.n > 0)
      HNV_CHECK(gather_rows_f32(lv.planC, lv.ch_idx, nullptr, nullptr, G, GC, GC, d, 0.f, 1.f,
                                g->partials, s, g));
    if (m > 0)
      HNV_CHECK(launch("scatter_kept", scatter_kept_kernel, grid_for((int64_t)m * d4, 256), 256, 0,
                       s, m, d4, (const int32_t*)lv.rep_e, (const float4*)ge,
                       (float4*)(GC + (size_t)cv.n * d)));
    std::swap(G, GC);
  }
  const Level& top = g->levels[L];
  if ((size_t)top.n + top.m > 0)
    HNV_CUDA(cudaMemcpyAsync(grad_zc, G, row * ((size_t)top.n + top.m), cudaMemcpyDeviceToDevice,
                             s));
  return HNV_OK;
}

}  // namespace hnv
