// The extern "C" entry points of libhnv.so (declared in include/hnv.h) and
// the V-cycle driver (Section 3, Fig. 1): coarsen level by level, refine the
// coarsest level, then project and refine every finer level.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "hnv_internal.cuh"

using namespace hnv;

namespace {

// Makes the graph's device current for the duration of a call.
struct DeviceGuard {
  int prev = -1;
  bool ok = true;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

void destroy_graph(hnv_graph* g) {
  if (!g) return;
  cudaStream_t s = g->stream;
  for (auto& lv : g->levels) free_level(&lv, s);
  g->levels.clear();
  dev_free(g->partials, s);
  dev_free(g->jacobi_tmp, s);
  dev_free(g->d_err, s);
  dev_free(g->d_buf, s);
  cudaStreamSynchronize(s);
  for (int i = 0; i < 2; ++i) {
    if (g->aux[i]) {
      cudaStreamSynchronize(g->aux[i]);
      cudaStreamDestroy(g->aux[i]);
    }
    if (g->join_ev[i]) cudaEventDestroy(g->join_ev[i]);
  }
  if (g->fork_ev) cudaEventDestroy(g->fork_ev);
  if (g->h_buf) cudaFreeHost(g->h_buf);
  delete g;
}

int check_embedding_args(hnv_dtype dt, int d) {
  if (dt == HNV_F32) {
    if (d < 4 || d > 1024 || d % 4 != 0)
      HNV_FAIL(HNV_ERR_UNSUPPORTED_D, "d = %d: need 4 <= d <= 1024 and d %% 4 == 0 for F32", d);
    return HNV_OK;
  }
  if (dt == HNV_BF16) {
    if (d < 8 || d > 1024 || d % 8 != 0)
      HNV_FAIL(HNV_ERR_UNSUPPORTED_D, "d = %d: need 8 <= d <= 1024 and d %% 8 == 0 for BF16", d);
    return HNV_OK;
  }
  HNV_FAIL(HNV_ERR_INVALID_ARG, "unknown dtype %d", (int)dt);
}

size_t dtype_size(hnv_dtype dt) { return dt == HNV_BF16 ? 2 : 4; }

__global__ void check_features_kernel(int64_t count, const float* __restrict__ x,
                                      int32_t* __restrict__ err) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float v = x[i];
    if (!(fabsf(v) <= 1e15f)) atomicOr(err, (int32_t)ERRBIT_BAD_FEATURE);   // also NaN
  }
}

int check_buf(const void* p, int64_t rows, const char* name) {
  if (rows > 0 && p == nullptr) HNV_FAIL(HNV_ERR_INVALID_ARG, "%s is NULL", name);
  if (p && (reinterpret_cast<uintptr_t>(p) & 15u))
    HNV_FAIL(HNV_ERR_INVALID_ARG, "%s is not 16-byte aligned", name);
  return HNV_OK;
}

// Frees one pointer a level owns (used to drop stale rep maps).
void drop_owned(Level* lv, void* p, cudaStream_t s) {
  if (!p) return;
  auto it = std::find(lv->owned.begin(), lv->owned.end(), p);
  if (it != lv->owned.end()) lv->owned.erase(it);
  dev_free(p, s);
}

void drop_maps(Level* lv, cudaStream_t s) {
  drop_owned(lv, lv->rep_v, s);
  drop_owned(lv, lv->rep_e, s);
  lv->rep_v = nullptr;
  lv->rep_e = nullptr;
}

// ckpt (optional, device, float32 only): every level's starting rows (node
// rows then hyperedge rows) at float offset sum_{j<l} (n_j + m_j) * d.
int vcycle_impl(hnv_graph* g, const void* z_coarsest, void* z_v_out, void* z_e_out, int dtype,
                int d, float omega, int sweeps, int mode, int on_device, cudaStream_t s,
                float* ckpt = nullptr) {
  NvtxRange nvtx("hnv vcycle (%d levels)", (int)g->levels.size());
  const int L = (int)g->levels.size() - 1;
  const size_t row_bytes = dtype_size((hnv_dtype)dtype) * (size_t)d;
  TempPool pool(s);
  size_t maxrows = 0;
  for (int l = 1; l <= L; ++l)
    maxrows = std::max(maxrows, (size_t)g->levels[l].n + (size_t)g->levels[l].m);
  uint8_t* buf[2] = {nullptr, nullptr};
  if (L >= 1) {
    HNV_CHECK(pool.get(&buf[0], maxrows * row_bytes));
    HNV_CHECK(pool.get(&buf[1], maxrows * row_bytes));
  }
  const Level& l0 = g->levels[0];
  uint8_t* out_v = static_cast<uint8_t*>(z_v_out);
  uint8_t* out_e = static_cast<uint8_t*>(z_e_out);
  if (!on_device) {
    HNV_CHECK(pool.get(&out_v, (size_t)l0.n * row_bytes));
    HNV_CHECK(pool.get(&out_e, (size_t)l0.m * row_bytes));
  }
  auto zv = [&](int l) { return l == 0 ? out_v : buf[l & 1]; };
  auto ze = [&](int l) {
    return l == 0 ? out_e : buf[l & 1] + (size_t)g->levels[l].n * row_bytes;
  };
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  const Level& top = g->levels[L];
  const uint8_t* zc = static_cast<const uint8_t*>(z_coarsest);
  if (top.n > 0) HNV_CUDA(cudaMemcpyAsync(zv(L), zc, row_bytes * top.n, kind, s));
  if (top.m > 0)
    HNV_CUDA(cudaMemcpyAsync(ze(L), zc + (size_t)top.n * row_bytes, row_bytes * top.m, kind, s));
  std::vector<size_t> off(L + 2, 0);
  for (int l = 0; l <= L; ++l)
    off[l + 1] = off[l] + ((size_t)g->levels[l].n + g->levels[l].m) * row_bytes;
  auto save = [&](int l) -> int {
    if (!ckpt) return HNV_OK;
    uint8_t* c = reinterpret_cast<uint8_t*>(ckpt) + off[l];
    const Level& lv = g->levels[l];
    if (lv.n > 0)
      HNV_CUDA(cudaMemcpyAsync(c, zv(l), row_bytes * lv.n, cudaMemcpyDeviceToDevice, s));
    if (lv.m > 0)
      HNV_CUDA(cudaMemcpyAsync(c + row_bytes * lv.n, ze(l), row_bytes * lv.m,
                               cudaMemcpyDeviceToDevice, s));
    return HNV_OK;
  };
  HNV_CHECK(save(L));
  HNV_CHECK(refine_level(g, L, zv(L), ze(L), dtype, d, omega, sweeps, mode, s));
  for (int l = L - 1; l >= 0; --l) {
    HNV_CHECK(project_level(g, l, zv(l + 1), ze(l + 1), zv(l), ze(l), dtype, d, s));
    HNV_CHECK(save(l));
    HNV_CHECK(refine_level(g, l, zv(l), ze(l), dtype, d, omega, sweeps, mode, s));
  }
  if (!on_device) {
    if (l0.n > 0)
      HNV_CUDA(cudaMemcpyAsync(z_v_out, out_v, row_bytes * l0.n, cudaMemcpyDeviceToHost, s));
    if (l0.m > 0)
      HNV_CUDA(cudaMemcpyAsync(z_e_out, out_e, row_bytes * l0.m, cudaMemcpyDeviceToHost, s));
    HNV_CUDA(cudaStreamSynchronize(s));
    int32_t bits = 0;
    HNV_CHECK(read_and_clear_err(g, s, &bits));
    if (bits & ERRBIT_TIMEOUT)
      HNV_FAIL(HNV_ERR_TIMEOUT, "a bounded wait of a refinement kernel gave up");
  }
  return HNV_OK;
}

}  // namespace

extern "C" {

int hnv_build_incidence(int32_t n_nodes, int32_t n_edges, const int64_t* edge_ptr,
                        const int32_t* edge_nodes, const float* edge_w, int inputs_on_device,
                        hnv_stream_t stream, hnv_graph** out) {
  NvtxRange nvtx("hnv build incidence");
  clear_error_detail();
  if (!out) HNV_FAIL(HNV_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (n_nodes < 1 || n_edges < 0) HNV_FAIL(HNV_ERR_INVALID_ARG, "need n >= 1 and m >= 0");
  if (!edge_ptr) HNV_FAIL(HNV_ERR_INVALID_ARG, "edge_ptr is NULL");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int64_t nnz_host = -1;
  if (!inputs_on_device) {
    if (edge_ptr[0] != 0) HNV_FAIL(HNV_ERR_INVALID_ARG, "edge_ptr[0] must be 0");
    nnz_host = edge_ptr[n_edges];
    if (nnz_host < 0) HNV_FAIL(HNV_ERR_INVALID_ARG, "edge_ptr[m] < 0");
    if (nnz_host > (int64_t)0x7fffff00) HNV_FAIL(HNV_ERR_TOO_LARGE, "nnz >= 2^31");
  }
  if (!edge_nodes && (inputs_on_device || nnz_host > 0))
    HNV_FAIL(HNV_ERR_INVALID_ARG, "edge_nodes is NULL");

  hnv_graph* g = new (std::nothrow) hnv_graph();
  if (!g) HNV_FAIL(HNV_ERR_OOM, "host allocation failed");
  cudaGetDevice(&g->device);
  g->stream = s;
  int rc = HNV_OK;
  do {
    if (cudaMallocHost((void**)&g->h_buf, 64 * sizeof(int32_t)) != cudaSuccess) {
      g->h_buf = nullptr;
      set_error_detail("cudaMallocHost failed");
      rc = HNV_ERR_OOM;
      break;
    }
    if ((rc = dev_alloc((void**)&g->d_err, sizeof(int32_t), s)) != HNV_OK) break;
    if ((rc = dev_alloc((void**)&g->d_buf, 64 * sizeof(int32_t), s)) != HNV_OK) break;
    {
      cudaError_t e = cudaEventCreateWithFlags(&g->fork_ev, cudaEventDisableTiming);
      for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
        e = cudaStreamCreateWithFlags(&g->aux[i], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g->join_ev[i], cudaEventDisableTiming);
      }
      if (e != cudaSuccess) {
        rc = cuda_status(e, "side streams");
        break;
      }
    }
    if (cudaMemsetAsync(g->d_err, 0, sizeof(int32_t), s) != cudaSuccess) {
      rc = cuda_status(cudaGetLastError(), "cudaMemsetAsync");
      break;
    }
    TempPool pool(s);
    const int64_t* d_ptr = edge_ptr;
    const int32_t* d_nodes = edge_nodes;
    const float* d_w = edge_w;
    if (!inputs_on_device) {
      int64_t* p1 = nullptr;
      int32_t* p2 = nullptr;
      float* p3 = nullptr;
      if ((rc = pool.get(&p1, (size_t)n_edges + 1)) != HNV_OK) break;
      if ((rc = pool.get(&p2, (size_t)nnz_host)) != HNV_OK) break;
      cudaError_t e = cudaMemcpyAsync(p1, edge_ptr, sizeof(int64_t) * ((size_t)n_edges + 1),
                                      cudaMemcpyHostToDevice, s);
      if (e == cudaSuccess && nnz_host > 0)
        e = cudaMemcpyAsync(p2, edge_nodes, sizeof(int32_t) * (size_t)nnz_host,
                            cudaMemcpyHostToDevice, s);
      if (e == cudaSuccess && edge_w && n_edges > 0) {
        if ((rc = pool.get(&p3, (size_t)n_edges)) != HNV_OK) break;
        e = cudaMemcpyAsync(p3, edge_w, sizeof(float) * (size_t)n_edges, cudaMemcpyHostToDevice, s);
      }
      if (e != cudaSuccess) {
        rc = cuda_status(e, "cudaMemcpyAsync (inputs)");
        break;
      }
      d_ptr = p1;
      d_nodes = p2;
      d_w = edge_w ? p3 : nullptr;
    }
    g->levels.resize(1);
    PhaseScope ps(HNV_PHASE_BUILD, s, 0.0);
    rc = build_level0(g, n_nodes, n_edges, d_ptr, d_nodes, d_w, &g->levels[0]);
  } while (0);
  if (rc == HNV_OK) {
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) rc = cuda_status(e, "cudaStreamSynchronize (build)");
  }
  if (rc != HNV_OK) {
    char keep[512];
    strncpy(keep, hnv_last_error_detail(), sizeof(keep) - 1);
    keep[sizeof(keep) - 1] = 0;
    destroy_graph(g);
    set_error_detail("%s", keep);
    return rc;
  }
  *out = g;
  return HNV_OK;
}

int hnv_coarsen(hnv_graph* g, const hnv_coarsen_params* p, int32_t* n_levels) {
  clear_error_detail();
  if (!g || !p) HNV_FAIL(HNV_ERR_INVALID_ARG, "graph or params is NULL");
  if (p->policy < HNV_ASSIGN_HASH || p->policy > HNV_ASSIGN_COSINE)
    HNV_FAIL(HNV_ERR_INVALID_ARG, "unknown policy %d", p->policy);
  if (p->policy == HNV_ASSIGN_COSINE && !g->levels[0].feat)
    HNV_FAIL(HNV_ERR_STATE, "the cosine policy needs node features (hnv_set_node_features)");
  if (p->max_levels < 0) HNV_FAIL(HNV_ERR_INVALID_ARG, "max_levels < 0");
  if (p->policy == HNV_ASSIGN_EXPLICIT && !p->explicit_prio && p->max_levels > 0)
    HNV_FAIL(HNV_ERR_INVALID_ARG, "EXPLICIT policy needs explicit_prio");
  DeviceGuard dg(g->device);
  cudaStream_t s = g->stream;
  ++g->generation;   // anything built on the old hierarchy (a batch) is stale now
  // drop any previous hierarchy above level 0
  while (g->levels.size() > 1) {
    free_level(&g->levels.back(), s);
    g->levels.pop_back();
  }
  drop_maps(&g->levels[0], s);
  const int32_t m0 = g->levels[0].m;
  {
    PhaseScope ps(HNV_PHASE_COARSEN, s, 0.0);
    TempPool pool(s);
    uint64_t* d_tab = nullptr;
    if (p->policy == HNV_ASSIGN_EXPLICIT) HNV_CHECK(pool.get(&d_tab, (size_t)m0 + 1));
    for (;;) {
      const int ell = (int)g->levels.size() - 1;
      Level* cur = &g->levels[ell];
      if (!(cur->n > p->min_nodes && ell < p->max_levels && cur->m > 0)) break;
      if (d_tab && m0 > 0)
        HNV_CUDA(cudaMemcpyAsync(d_tab, p->explicit_prio + (size_t)ell * m0,
                                 sizeof(uint64_t) * m0, cudaMemcpyHostToDevice, s));
      Level nxt;
      int rc = coarsen_step(g, ell, p, d_tab, cur, &nxt);
      if (rc != HNV_OK) {
        free_level(&nxt, s);
        drop_maps(cur, s);
        return rc;
      }
      if (nxt.n == cur->n) {   // nothing merged: discard the step
        free_level(&nxt, s);
        drop_maps(cur, s);
        break;
      }
      rc = finish_level(g, &nxt);
      if (rc != HNV_OK) {
        free_level(&nxt, s);
        drop_maps(cur, s);
        return rc;
      }
      g->levels.push_back(nxt);
    }
  }
  HNV_CUDA(cudaStreamSynchronize(s));
  if (n_levels) *n_levels = (int32_t)g->levels.size();
  return HNV_OK;
}

int hnv_num_levels(const hnv_graph* g, int32_t* n_levels) {
  if (!g || !n_levels) HNV_FAIL(HNV_ERR_INVALID_ARG, "NULL argument");
  *n_levels = (int32_t)g->levels.size();
  return HNV_OK;
}

int hnv_level_info(const hnv_graph* g, int level, int32_t* n, int32_t* m, int64_t* nnz) {
  if (!g) HNV_FAIL(HNV_ERR_INVALID_ARG, "graph is NULL");
  if (level < 0 || level >= (int)g->levels.size())
    HNV_FAIL(HNV_ERR_OUT_OF_RANGE, "level %d not in [0, %d)", level, (int)g->levels.size());
  const Level& lv = g->levels[level];
  if (n) *n = lv.n;
  if (m) *m = lv.m;
  if (nnz) *nnz = lv.nnz;
  return HNV_OK;
}

int hnv_get_level_arrays(const hnv_graph* g, int level, const int32_t** e_ptr,
                         const int32_t** e_nodes, const int32_t** v_ptr, const int32_t** v_edges,
                         const float** w, const int32_t** rep_v, const int32_t** rep_e) {
  if (!g) HNV_FAIL(HNV_ERR_INVALID_ARG, "graph is NULL");
  if (level < 0 || level >= (int)g->levels.size())
    HNV_FAIL(HNV_ERR_OUT_OF_RANGE, "level %d not in [0, %d)", level, (int)g->levels.size());
  const Level& lv = g->levels[level];
  if (e_ptr) *e_ptr = lv.e_ptr;
  if (e_nodes) *e_nodes = lv.e_nodes;
  if (v_ptr) *v_ptr = lv.v_ptr;
  if (v_edges) *v_edges = lv.v_edges;
  if (w) *w = lv.w;
  if (rep_v) *rep_v = lv.rep_v;
  if (rep_e) *rep_e = lv.rep_e;
  return HNV_OK;
}

int hnv_copy_level_array(const hnv_graph* g, int level, int which, void* dst,
                         size_t capacity_bytes, int dst_on_device, hnv_stream_t stream) {
  if (!g) HNV_FAIL(HNV_ERR_INVALID_ARG, "graph is NULL");
  if (level < 0 || level >= (int)g->levels.size())
    HNV_FAIL(HNV_ERR_OUT_OF_RANGE, "level %d not in [0, %d)", level, (int)g->levels.size());
  const Level& lv = g->levels[level];
  const void* src = nullptr;
  size_t bytes = 0;
  switch (which) {
    case HNV_ARR_E_PTR: src = lv.e_ptr; bytes = 4 * ((size_t)lv.m + 1); break;
    case HNV_ARR_E_NODES: src = lv.e_nodes; bytes = 4 * (size_t)lv.nnz; break;
    case HNV_ARR_V_PTR: src = lv.v_ptr; bytes = 4 * ((size_t)lv.n + 1); break;
    case HNV_ARR_V_EDGES: src = lv.v_edges; bytes = 4 * (size_t)lv.nnz; break;
    case HNV_ARR_W: src = lv.w; bytes = 4 * (size_t)lv.m; break;
    case HNV_ARR_REP_V: src = lv.rep_v; bytes = 4 * (size_t)lv.n; break;
    case HNV_ARR_REP_E: src = lv.rep_e; bytes = 4 * (size_t)lv.m; break;
    case HNV_ARR_DEG_V: src = lv.deg_v; bytes = 4 * (size_t)lv.n; break;
    default: HNV_FAIL(HNV_ERR_INVALID_ARG, "unknown array %d", which);
  }
  if ((which == HNV_ARR_REP_V || which == HNV_ARR_REP_E) && !src)
    HNV_FAIL(HNV_ERR_STATE, "level %d is the coarsest: it has no rep maps", level);
  if (bytes > capacity_bytes) HNV_FAIL(HNV_ERR_INVALID_ARG, "destination too small (%zu < %zu)", capacity_bytes, bytes);
  if (bytes == 0) return HNV_OK;
  if (!dst) HNV_FAIL(HNV_ERR_INVALID_ARG, "dst is NULL");
  DeviceGuard dgd(g->device);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  HNV_CUDA(cudaMemcpyAsync(dst, src, bytes,
                           dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
  HNV_CUDA(cudaStreamSynchronize(s));
  return HNV_OK;
}

int hnv_set_node_features(hnv_graph* g, const float* x, int32_t k, int x_on_device,
                          hnv_stream_t stream) {
  clear_error_detail();
  if (!g) HNV_FAIL(HNV_ERR_INVALID_ARG, "graph is NULL");
  if (k < 1 || k > 4096) HNV_FAIL(HNV_ERR_INVALID_ARG, "k = %d not in [1, 4096]", k);
  Level& l0 = g->levels[0];
  if (l0.n > 0 && !x) HNV_FAIL(HNV_ERR_INVALID_ARG, "features are NULL");
  DeviceGuard dgd(g->device);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const size_t bytes = sizeof(float) * (size_t)l0.n * k;
  float* feat = nullptr;
  HNV_CHECK(dev_alloc((void**)&feat, bytes ? bytes : 16, s));
  int rc = HNV_OK;
  if (bytes) {
    const cudaError_t e = cudaMemcpyAsync(feat, x, bytes,
                                          x_on_device ? cudaMemcpyDeviceToDevice
                                                      : cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) rc = cuda_status(e, "cudaMemcpyAsync");
  }
  if (rc == HNV_OK && bytes)
    rc = launch("check_features", check_features_kernel, grid_for((int64_t)l0.n * k, 256), 256, 0,
                s, (int64_t)l0.n * k, (const float*)feat, g->d_err);
  int32_t bits = 0;
  if (rc == HNV_OK) rc = read_and_clear_err(g, s, &bits);
  if (rc == HNV_OK && (bits & ERRBIT_BAD_FEATURE)) {
    rc = HNV_ERR_INVALID_ARG;
    set_error_detail("features must be finite with |x| <= 1e15");
  }
  if (rc != HNV_OK) {
    dev_free(feat, s);
    return rc;
  }
  drop_owned(&l0, l0.feat, s);
  l0.feat = feat;
  l0.feat_k = k;
  l0.owned.push_back(feat);
  return HNV_OK;
}

int hnv_copy_level_features(const hnv_graph* g, int level, float* dst, size_t capacity_bytes,
                            int dst_on_device, hnv_stream_t stream) {
  clear_error_detail();
  if (!g) HNV_FAIL(HNV_ERR_INVALID_ARG, "graph is NULL");
  if (level < 0 || level >= (int)g->levels.size())
    HNV_FAIL(HNV_ERR_OUT_OF_RANGE, "level %d not in [0, %d)", level, (int)g->levels.size());
  const Level& lv = g->levels[level];
  if (!lv.feat) HNV_FAIL(HNV_ERR_STATE, "level %d has no node features", level);
  const size_t bytes = sizeof(float) * (size_t)lv.n * lv.feat_k;
  if (bytes > capacity_bytes)
    HNV_FAIL(HNV_ERR_INVALID_ARG, "destination too small (%zu < %zu)", capacity_bytes, bytes);
  if (bytes == 0) return HNV_OK;
  if (!dst) HNV_FAIL(HNV_ERR_INVALID_ARG, "dst is NULL");
  DeviceGuard dgd(g->device);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  HNV_CUDA(cudaMemcpyAsync(dst, lv.feat, bytes,
                           dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
  HNV_CUDA(cudaStreamSynchronize(s));
  return HNV_OK;
}

int hnv_level_feature_dim(const hnv_graph* g, int level, int32_t* k) {
  if (!g || !k) HNV_FAIL(HNV_ERR_INVALID_ARG, "NULL argument");
  if (level < 0 || level >= (int)g->levels.size())
    HNV_FAIL(HNV_ERR_OUT_OF_RANGE, "level %d not in [0, %d)", level, (int)g->levels.size());
  *k = g->levels[level].feat ? g->levels[level].feat_k : 0;
  return HNV_OK;
}

int hnv_project(const hnv_graph* g, int fine_level, const void* zc_v, const void* zc_e,
                void* zf_v, void* zf_e, hnv_dtype dt, int d, hnv_stream_t stream) {
  clear_error_detail();
  if (!g) HNV_FAIL(HNV_ERR_INVALID_ARG, "graph is NULL");
  if (fine_level < 0 || fine_level + 1 >= (int)g->levels.size())
    HNV_FAIL(HNV_ERR_OUT_OF_RANGE, "fine_level %d not in [0, %d)", fine_level,
             (int)g->levels.size() - 1);
  HNV_CHECK(check_embedding_args(dt, d));
  const Level& f = g->levels[fine_level];
  const Level& c = g->levels[fine_level + 1];
  HNV_CHECK(check_buf(zc_v, c.n, "zc_v"));
  HNV_CHECK(check_buf(zc_e, c.m, "zc_e"));
  HNV_CHECK(check_buf(zf_v, f.n, "zf_v"));
  HNV_CHECK(check_buf(zf_e, f.m, "zf_e"));
  DeviceGuard dgd(g->device);
  return project_level(g, fine_level, zc_v, zc_e, zf_v, zf_e, (int)dt, d,
                       reinterpret_cast<cudaStream_t>(stream));
}

int hnv_refine(hnv_graph* g, int level, void* z_v, void* z_e, hnv_dtype dt, int d, float omega,
               int sweeps, hnv_sweep mode, hnv_stream_t stream) {
  clear_error_detail();
  if (!g) HNV_FAIL(HNV_ERR_INVALID_ARG, "graph is NULL");
  if (level < 0 || level >= (int)g->levels.size())
    HNV_FAIL(HNV_ERR_OUT_OF_RANGE, "level %d not in [0, %d)", level, (int)g->levels.size());
  HNV_CHECK(check_embedding_args(dt, d));
  if (!(omega >= 0.f && omega <= 1.f)) HNV_FAIL(HNV_ERR_INVALID_ARG, "omega must be in [0, 1]");
  if (sweeps < 0) HNV_FAIL(HNV_ERR_INVALID_ARG, "sweeps < 0");
  if (mode != HNV_SWEEP_TWO_PHASE && mode != HNV_SWEEP_JACOBI)
    HNV_FAIL(HNV_ERR_INVALID_ARG, "unknown sweep mode %d", (int)mode);
  const Level& lv = g->levels[level];
  HNV_CHECK(check_buf(z_v, lv.n, "z_v"));
  HNV_CHECK(check_buf(z_e, lv.m, "z_e"));
  DeviceGuard dgd(g->device);
  return refine_level(g, level, z_v, z_e, (int)dt, d, omega, sweeps, (int)mode,
                      reinterpret_cast<cudaStream_t>(stream));
}

int hnv_refine_until(hnv_graph* g, int level, void* z_v, void* z_e, hnv_dtype dt, int d,
                     float omega, int max_sweeps, float eps, hnv_sweep mode,
                     int32_t* sweeps_done, float* last_delta, hnv_stream_t stream) {
  clear_error_detail();
  if (!g) HNV_FAIL(HNV_ERR_INVALID_ARG, "graph is NULL");
  if (!sweeps_done || !last_delta) HNV_FAIL(HNV_ERR_INVALID_ARG, "NULL output");
  if (level < 0 || level >= (int)g->levels.size())
    HNV_FAIL(HNV_ERR_OUT_OF_RANGE, "level %d not in [0, %d)", level, (int)g->levels.size());
  HNV_CHECK(check_embedding_args(dt, d));
  if (!(omega >= 0.f && omega <= 1.f)) HNV_FAIL(HNV_ERR_INVALID_ARG, "omega must be in [0, 1]");
  if (max_sweeps < 0) HNV_FAIL(HNV_ERR_INVALID_ARG, "max_sweeps < 0");
  if (eps != eps) HNV_FAIL(HNV_ERR_INVALID_ARG, "eps is NaN");
  if (mode != HNV_SWEEP_TWO_PHASE && mode != HNV_SWEEP_JACOBI)
    HNV_FAIL(HNV_ERR_INVALID_ARG, "unknown sweep mode %d", (int)mode);
  const Level& lv = g->levels[level];
  HNV_CHECK(check_buf(z_v, lv.n, "z_v"));
  HNV_CHECK(check_buf(z_e, lv.m, "z_e"));
  DeviceGuard dgd(g->device);
  return refine_level_until(g, level, z_v, z_e, (int)dt, d, omega, max_sweeps, eps, (int)mode,
                            sweeps_done, last_delta, reinterpret_cast<cudaStream_t>(stream));
}

int hnv_vcycle(hnv_graph* g, const void* z_coarsest, void* z_v_out, void* z_e_out, hnv_dtype dt,
               int d, float omega, int sweeps_per_level, hnv_sweep mode, int buffers_on_device,
               hnv_stream_t stream) {
  clear_error_detail();
  if (!g) HNV_FAIL(HNV_ERR_INVALID_ARG, "graph is NULL");
  HNV_CHECK(check_embedding_args(dt, d));
  if (!(omega >= 0.f && omega <= 1.f)) HNV_FAIL(HNV_ERR_INVALID_ARG, "omega must be in [0, 1]");
  if (sweeps_per_level < 0) HNV_FAIL(HNV_ERR_INVALID_ARG, "sweeps_per_level < 0");
  if (mode != HNV_SWEEP_TWO_PHASE && mode != HNV_SWEEP_JACOBI)
    HNV_FAIL(HNV_ERR_INVALID_ARG, "unknown sweep mode %d", (int)mode);
  const Level& top = g->levels.back();
  const Level& l0 = g->levels[0];
  if (buffers_on_device) {
    HNV_CHECK(check_buf(z_coarsest, (int64_t)top.n + top.m, "z_coarsest"));
    HNV_CHECK(check_buf(z_v_out, l0.n, "z_v_out"));
    HNV_CHECK(check_buf(z_e_out, l0.m, "z_e_out"));
  } else {
    if ((top.n + (int64_t)top.m > 0 && !z_coarsest) || (l0.n > 0 && !z_v_out) ||
        (l0.m > 0 && !z_e_out))
      HNV_FAIL(HNV_ERR_INVALID_ARG, "NULL host buffer");
  }
  DeviceGuard dgd(g->device);
  return vcycle_impl(g, z_coarsest, z_v_out, z_e_out, (int)dt, d, omega, sweeps_per_level,
                     (int)mode, buffers_on_device, reinterpret_cast<cudaStream_t>(stream));
}

int hnv_set_weights(hnv_graph* g, const float* w0, int on_device, hnv_stream_t stream) {
  clear_error_detail();
  if (!g) HNV_FAIL(HNV_ERR_INVALID_ARG, "graph is NULL");
  const int32_t m0 = g->levels[0].m;
  if (m0 > 0 && !w0) HNV_FAIL(HNV_ERR_INVALID_ARG, "w0 is NULL");
  DeviceGuard dgd(g->device);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  TempPool pool(s);
  const float* d_w0 = w0;
  if (!on_device && m0 > 0) {
    float* t = nullptr;
    HNV_CHECK(pool.get(&t, (size_t)m0));
    HNV_CUDA(cudaMemcpyAsync(t, w0, sizeof(float) * m0, cudaMemcpyHostToDevice, s));
    d_w0 = t;
  }
  return set_weights_impl(g, d_w0, s);
}

int hnv_checkpoint_floats(const hnv_graph* g, int d, int64_t* floats) {
  if (!g || !floats) HNV_FAIL(HNV_ERR_INVALID_ARG, "NULL argument");
  int64_t t = 0;
  for (const Level& lv : g->levels) t += ((int64_t)lv.n + lv.m) * d;
  *floats = t;
  return HNV_OK;
}

int hnv_vcycle_save(hnv_graph* g, const float* z_coarsest, float* z_v_out, float* z_e_out, int d,
                    float omega, int sweeps_per_level, float* checkpoints, hnv_stream_t stream) {
  clear_error_detail();
  if (!g) HNV_FAIL(HNV_ERR_INVALID_ARG, "graph is NULL");
  HNV_CHECK(check_embedding_args(HNV_F32, d));
  if (!(omega >= 0.f && omega <= 1.f)) HNV_FAIL(HNV_ERR_INVALID_ARG, "omega must be in [0, 1]");
  if (sweeps_per_level < 0) HNV_FAIL(HNV_ERR_INVALID_ARG, "sweeps_per_level < 0");
  const Level& top = g->levels.back();
  const Level& l0 = g->levels[0];
  HNV_CHECK(check_buf(z_coarsest, (int64_t)top.n + top.m, "z_coarsest"));
  HNV_CHECK(check_buf(z_v_out, l0.n, "z_v_out"));
  HNV_CHECK(check_buf(z_e_out, l0.m, "z_e_out"));
  HNV_CHECK(check_buf(checkpoints, 1, "checkpoints"));
  DeviceGuard dgd(g->device);
  return vcycle_impl(g, z_coarsest, z_v_out, z_e_out, HNV_F32, d, omega, sweeps_per_level,
                     HNV_SWEEP_TWO_PHASE, 1, reinterpret_cast<cudaStream_t>(stream), checkpoints);
}

int hnv_vcycle_backward(hnv_graph* g, const float* checkpoints, const float* g_v0,
                        const float* g_e0, float* grad_w0, float* grad_z_coarsest, int d,
                        float omega, int sweeps_per_level, hnv_stream_t stream) {
  clear_error_detail();
  if (!g) HNV_FAIL(HNV_ERR_INVALID_ARG, "graph is NULL");
  HNV_CHECK(check_embedding_args(HNV_F32, d));
  if (!(omega >= 0.f && omega <= 1.f)) HNV_FAIL(HNV_ERR_INVALID_ARG, "omega must be in [0, 1]");
  if (sweeps_per_level < 0) HNV_FAIL(HNV_ERR_INVALID_ARG, "sweeps_per_level < 0");
  const Level& top = g->levels.back();
  const Level& l0 = g->levels[0];
  HNV_CHECK(check_buf(checkpoints, 1, "checkpoints"));
  HNV_CHECK(check_buf(g_v0, 0, "g_v0"));
  HNV_CHECK(check_buf(g_e0, 0, "g_e0"));
  HNV_CHECK(check_buf(grad_w0, l0.m, "grad_w0"));
  HNV_CHECK(check_buf(grad_z_coarsest, (int64_t)top.n + top.m, "grad_z_coarsest"));
  DeviceGuard dgd(g->device);
  return vcycle_backward_impl(g, checkpoints, g_v0, g_e0, grad_w0, grad_z_coarsest, d, omega,
                              sweeps_per_level, reinterpret_cast<cudaStream_t>(stream));
}

int hnv_sync_status(hnv_graph* g, hnv_stream_t stream) {
  if (!g) HNV_FAIL(HNV_ERR_INVALID_ARG, "graph is NULL");
  DeviceGuard dgd(g->device);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  HNV_CUDA(cudaStreamSynchronize(s));
  int32_t bits = 0;
  HNV_CHECK(read_and_clear_err(g, s, &bits));
  if (bits & ERRBIT_TIMEOUT)
    HNV_FAIL(HNV_ERR_TIMEOUT, "a bounded wait of a refinement kernel gave up");
  if (bits & ERRBIT_BAD_ITEM)
    HNV_FAIL(HNV_ERR_STATE, "a batched work item lay outside its graph's arrays and was skipped");
  return HNV_OK;
}

int hnv_selftest_wait_timeout(hnv_graph* g, uint32_t limit_us, hnv_stream_t stream) {
  clear_error_detail();
  if (!g) HNV_FAIL(HNV_ERR_INVALID_ARG, "graph is NULL");
  if (limit_us < 1 || limit_us > 1000000)
    HNV_FAIL(HNV_ERR_INVALID_ARG, "limit_us = %u: need 1 .. 1000000", limit_us);
  DeviceGuard dgd(g->device);
  return wait_selftest(g->d_err, (uint64_t)limit_us * 1000ull,
                       reinterpret_cast<cudaStream_t>(stream));
}

void hnv_graph_free(hnv_graph* g) {
  if (!g) return;
  DeviceGuard dgd(g->device);
  destroy_graph(g);
}

}  // extern "C"
