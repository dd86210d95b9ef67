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
// z~_v is recovered from the stored iterates as (z_v^i - (1-w) z_v^{i-1})/w.
// Projection (a fine row copies a coarse row) reverses to a segmented sum of
// the fine gradients into their coarse row; a level's weights are the level-0
// weights of their hyperedges (orig_e), so dw accumulates into dw0.
// Per level, the forward iterates are recomputed from the level's starting
// rows saved by hnv_vcycle_save (per-level checkpointing).
#include <algorithm>

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

// out[r] = s[r] * <X[r], a1 * Y1[r] + a2 * Y2[r]>   (warp per row; Y2, s may
// be null; lane-strided partial sums, then a fixed xor tree)
__global__ void row_dot_kernel(int32_t rows, int32_t d4, const float4* __restrict__ X,
                               const float4* __restrict__ Y1, float a1,
                               const float4* __restrict__ Y2, float a2,
                               const float* __restrict__ s, float* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < rows;
       r += warps) {
    float acc = 0.f;
    for (int c = lane; c < d4; c += 32) {
      const size_t o = (size_t)r * d4 + c;
      const float4 x = X[o];
      float4 y = Y1[o];
      y = make_float4(a1 * y.x, a1 * y.y, a1 * y.z, a1 * y.w);
      if (Y2) {
        const float4 z = Y2[o];
        y = make_float4(fmaf(a2, z.x, y.x), fmaf(a2, z.y, y.y), fmaf(a2, z.z, y.z),
                        fmaf(a2, z.w, y.w));
      }
      acc = fmaf(x.x, y.x, acc);
      acc = fmaf(x.y, y.y, acc);
      acc = fmaf(x.z, y.z, acc);
      acc = fmaf(x.w, y.w, acc);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o);
    if (lane == 0) out[r] = s ? s[r] * acc : acc;
  }
}

// dw[e] += omega * (dotA[e] - sum_{v in e} c[v])   (warp per hyperedge)
__global__ void weight_grad_kernel(int32_t m, const int32_t* __restrict__ e_ptr,
                                   const int32_t* __restrict__ e_nodes, const float* __restrict__ c,
                                   const float* __restrict__ dotA, float omega,
                                   float* __restrict__ dw) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t e = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); e < m;
       e += warps) {
    float acc = 0.f;
    for (int64_t k = e_ptr[e] + lane; k < e_ptr[e + 1]; k += 32) acc += c[e_nodes[k]];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o);
    if (lane == 0) dw[e] += omega * (dotA[e] - acc);
  }
}

// Y[r] += alpha * s[r] * X[r]
__global__ void row_axpy_kernel(int32_t rows, int32_t d4, float4* __restrict__ Y,
                                const float4* __restrict__ X, float alpha,
                                const float* __restrict__ s) {
  const int64_t total = (int64_t)rows * d4;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float f = alpha * s[i / d4];
    const float4 x = X[i];
    float4 y = Y[i];
    y.x = fmaf(f, x.x, y.x);
    y.y = fmaf(f, x.y, y.y);
    y.z = fmaf(f, x.z, y.z);
    y.w = fmaf(f, x.w, y.w);
    Y[i] = y;
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

// Per-level arrays of the adjoint: per-incidence 1/D_v (CSR order) and 1/|e|
// (CSC order), and the children lists of the next level's nodes.
int prepare_level_adjoint(hnv_graph* g, int level, cudaStream_t s) {
  Level& lv = g->levels[level];
  if (!lv.e_invdeg_w) {
    HNV_CHECK(level_alloc(&lv, (void**)&lv.e_invdeg_w, sizeof(float) * (size_t)(lv.nnz + 1), s));
    HNV_CHECK(level_alloc(&lv, (void**)&lv.v_invsize_w, sizeof(float) * (size_t)(lv.nnz + 1), s));
  }
  // 1/D_v depends on the weights: refreshed on every call
  HNV_CHECK(launch("table_at", table_at_kernel, grid_for(lv.nnz, 256), 256, 0, s, lv.nnz,
                   (const int32_t*)lv.e_nodes, (const float*)lv.inv_deg_v, lv.e_invdeg_w));
  HNV_CHECK(launch("table_at", table_at_kernel, grid_for(lv.nnz, 256), 256, 0, s, lv.nnz,
                   (const int32_t*)lv.v_edges, (const float*)lv.inv_size_e, lv.v_invsize_w));
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
  // omega == 0: every sweep is the identity (and z~ cannot be recovered by
  // dividing by omega); the gradients pass through the sweeps unchanged
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
  float *G = nullptr, *GC = nullptr, *states = nullptr, *A = nullptr, *c = nullptr,
        *dotA = nullptr, *dwl = nullptr;
  HNV_CHECK(pool.get(&G, maxrows * d));
  HNV_CHECK(pool.get(&GC, maxrows * d));
  HNV_CHECK(pool.get(&states, (size_t)(sweeps + 1) * maxrows * d));
  HNV_CHECK(pool.get(&A, maxm * d));
  HNV_CHECK(pool.get(&c, maxn));
  HNV_CHECK(pool.get(&dotA, maxm));
  HNV_CHECK(pool.get(&dwl, maxm));
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
    // forward iterates of this level from its checkpoint
    HNV_CUDA(cudaMemcpyAsync(states, ckpt + off[l], row * rows, cudaMemcpyDeviceToDevice, s));
    for (int i = 1; i <= rsweeps; ++i) {
      float* si = states + (size_t)i * rows * d;
      HNV_CUDA(cudaMemcpyAsync(si, si - rows * d, row * rows, cudaMemcpyDeviceToDevice, s));
      HNV_CHECK(refine_level(g, l, si, si + (size_t)n * d, HNV_F32, d, omega, 1,
                             HNV_SWEEP_TWO_PHASE, s));
    }
    if (m > 0) HNV_CUDA(cudaMemsetAsync(dwl, 0, sizeof(float) * m, s));
    for (int i = rsweeps; i >= 1; --i) {
      const float* zv_i = states + (size_t)i * rows * d;
      const float* ze_i = zv_i + (size_t)n * d;
      const float* zv_p = zv_i - rows * d;
      // node half-sweep, reversed
      if (m > 0) {
        HNV_CHECK(gather_rows_f32(lv.planE, lv.e_nodes, lv.e_invdeg_w, nullptr, gv, A, A, d, 0.f,
                                  1.f, g->partials, s));  // A_e = sum_{v in e} G_V[v] / D_v
        HNV_CHECK(launch("row_dot", row_dot_kernel, grid_for((int64_t)m * 32, 256), 256, 0, s, m,
                         d4, (const float4*)A, (const float4*)ze_i, 1.f, (const float4*)nullptr,
                         0.f, (const float*)nullptr, dotA));
      }
      if (n > 0)
        HNV_CHECK(launch("row_dot", row_dot_kernel, grid_for((int64_t)n * 32, 256), 256, 0, s, n,
                         d4, (const float4*)gv, (const float4*)zv_i, 1.f / omega,
                         (const float4*)zv_p, -(1.f - omega) / omega,
                         (const float*)lv.inv_deg_v, c));  // c_v = <G_V/D_v, z~_v>
      if (m > 0) {
        HNV_CHECK(launch("weight_grad", weight_grad_kernel, grid_for((int64_t)m * 32, 256), 256, 0,
                         s, m, (const int32_t*)lv.e_ptr, (const int32_t*)lv.e_nodes,
                         (const float*)c, (const float*)dotA, omega, dwl));
        HNV_CHECK(launch("row_axpy", row_axpy_kernel, grid_for((int64_t)m * d4, 256), 256, 0, s,
                         m, d4, (float4*)ge, (const float4*)A, omega, (const float*)lv.w));
      }
      if (n > 0)
        HNV_CHECK(launch("row_scale", row_scale_kernel, grid_for((int64_t)n * d4, 256), 256, 0, s,
                         n, d4, (float4*)gv, 1.f - omega, (const float*)lv.inv_deg_v));
      // hyperedge half-sweep, reversed: G_V += w sum_{e ∋ v} G_E[e] / |e|
      if (n > 0 && m > 0)
        HNV_CHECK(gather_rows_f32(lv.planV, lv.v_edges, lv.v_invsize_w, nullptr, ge, gv, gv, d,
                                  1.f, omega, g->partials, s));
      if (m > 0)
        HNV_CHECK(launch("row_scale", row_scale_kernel, grid_for((int64_t)m * d4, 256), 256, 0, s,
                         m, d4, (float4*)ge, 1.f - omega, (const float*)lv.inv_size_e));
    }
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
                                g->partials, s));
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
