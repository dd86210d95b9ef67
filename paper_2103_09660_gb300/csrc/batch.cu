// Batched V-cycle: many independent hypergraphs refined together.
//
// Every graph keeps its own hierarchy (built and coarsened as usual). The
// batch lines the graphs up by level index: at step s (from the deepest
// level down to 0) every graph whose coarsest level is >= s projects onto
// level s (or, at its own coarsest level, starts from its input rows) and
// refines it. The work of one half-sweep of one step, over all graphs, is a
// single list of items {row, first incidence, length, partial slot} with a
// graph index per item; batched_gather_kernel runs the same per-item gather
// as the single-graph path (refine_device.cuh) with that graph's pointers,
// looping over the list with a grid of a few blocks per SM. One launch per
// row class and side replaces one launch per class, side and graph; the
// whole V-cycle (all steps, sweeps, projections) is captured once into a
// CUDA graph and replayed.
//
// Two half-sweep kernels: one launch per row class (classes on concurrent
// streams, lanes per row chosen per class), or one persistent launch over
// every item of the half-sweep (warps take tasks from a counter; see
// batched_persistent_kernel). Both are followed by the split-row reduction.
//
// Autotuner: the row-class boundaries (PlanShape) and the lanes per row of
// the short classes of the per-class kernel, and the persistent kernel, are
// timed on a whole V-cycle of the batch with one sweep per level (the coarse
// levels dominate a batch of many small graphs, so a level-0 sweep alone
// picks badly), and the fastest is kept and cached per (dtype, d, level-0
// length histogram).
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "refine_device.cuh"

namespace hnv {

namespace {

// HNV_TRACE=1: host-side progress of the batch calls on stderr.
bool trace_on() {
  static int on = -1;
  if (on < 0) {
    const char* e = getenv("HNV_TRACE");
    on = (e && e[0] == '1') ? 1 : 0;
  }
  return on == 1;
}

#define BTRACE(...)                        \
  do {                                     \
    if (trace_on()) {                      \
      fprintf(stderr, "[hnv_batch] ");     \
      fprintf(stderr, __VA_ARGS__);        \
      fprintf(stderr, "\n");               \
      fflush(stderr);                      \
    }                                      \
  } while (0)

struct GraphSide {
  const int32_t* idx;
  const float* inc_w;
  const float* inv_norm;
  const uint4* src;
  const uint4* self_in;
  uint4* out;
  float* partials;
  // bounds every item of this graph must respect (checked per item; an item
  // outside them is skipped and flagged in err)
  int32_t self_rows = 0;
  int64_t nnz = 0;
  int64_t n_slots = 0;
  int32_t* err = nullptr;
};

struct ProjDesc {
  const int32_t* rep_v;
  const int32_t* rep_e;
  int32_t n_f, m_f;
  const uint4* zc_v;
  const uint4* zc_e;
  uint4* zf_v;
  uint4* zf_e;
};

struct CopyDesc {
  const uint4* src;
  uint4* dst;
};

template <typename T, int G, int VPL, bool W>
__global__ void __launch_bounds__(256)
batched_gather_kernel(const int4* __restrict__ items, const int32_t* __restrict__ item_g,
                      int32_t n_items, const GraphSide* __restrict__ sides, int32_t n_graphs,
                      int32_t dv, float keep, float scale) {
  constexpr int R = 32 / G;
  const int lane = threadIdx.x & 31;
  const int grp = lane / G;
  const int lg = lane & (G - 1);
  const int64_t warps_total = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t wbase = ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * R;
       wbase < n_items; wbase += warps_total * R) {
    const int64_t item = wbase + grp;
    int4 it = make_int4(-1, 0, 0, -1);
    int32_t gi = 0;
    bool bad = false;
    if (item < n_items) {
      it = __ldg(items + item);
      gi = __ldg(item_g + item);
      if (gi < 0 || gi >= n_graphs) {
        gi = 0;
        bad = true;
      }
    }
    const GraphSide sd = sides[gi];
    if (item < n_items) {
      bad = bad || it.x < -1 || it.x >= sd.self_rows || it.y < 0 || it.z < 0 ||
            (int64_t)it.y + it.z > sd.nnz || it.w >= sd.n_slots || (it.x < 0 && it.w < 0);
      if (bad) {
        if (sd.err) atomicOr(sd.err, (int32_t)ERRBIT_BAD_ITEM);
        it = make_int4(-1, 0, 0, -1);
      }
    }
    dev::gather_item<T, G, VPL, W>(it, lg, sd.idx, sd.inc_w, sd.inv_norm, sd.src, sd.self_in,
                                   sd.out, dv, keep, scale, sd.partials);
  }
}

// Persistent half-sweep: one launch runs every item of one side of one step,
// over all graphs and all row classes. A warp takes a task (kTaskPasses
// passes over items of one class) from a counter in device memory until
// none is left. The long rows and chunks (the last class) come first, then
// class B, then class A, so the short rows fill the tail. Classes B and the
// rest use one lane per 16-byte vector of the row (GL lanes); the rows of
// class A (1..a_max incidences) use GA = GL/4 lanes with 4 vectors each, so
// a warp has four times as many of these short rows in flight. The sums run
// in the same order as in the per-class kernels: the results are the same
// bits.
constexpr int kTaskPasses = 8;
constexpr int kPersistThreads = 64;
constexpr int kCountersPerHalf = 1;   // task counters of one persistent launch

template <typename T, int G, int VPL, bool W>
__device__ __forceinline__ void persistent_task(const int4* __restrict__ items,
                                                const int32_t* __restrict__ item_g,
                                                int32_t lo, int32_t hi,
                                                const GraphSide* __restrict__ sides,
                                                int32_t n_graphs, int32_t dv, float keep,
                                                float scale) {
  constexpr int R = 32 / G;
  const int lane = threadIdx.x & 31;
  const int grp = lane / G;
  const int lg = lane & (G - 1);
#pragma unroll 1
  for (int k = 0; k < kTaskPasses; ++k) {
    const int32_t base = lo + k * R;
    if (base >= hi) break;                                     // warp-uniform
    const int32_t item = base + grp;
    int4 it = make_int4(-1, 0, 0, -1);
    int32_t gi = 0;
    bool bad = false;
    if (item < hi) {
      it = __ldg(items + item);
      gi = __ldg(item_g + item);
      if (gi < 0 || gi >= n_graphs) {
        gi = 0;
        bad = true;
      }
    }
    const GraphSide sd = sides[gi];
    if (item < hi) {
      bad = bad || it.x < -1 || it.x >= sd.self_rows || it.y < 0 || it.z < 0 ||
            (int64_t)it.y + it.z > sd.nnz || it.w >= sd.n_slots || (it.x < 0 && it.w < 0);
      if (bad) {
        if (sd.err) atomicOr(sd.err, (int32_t)ERRBIT_BAD_ITEM);
        it = make_int4(-1, 0, 0, -1);
      }
    }
    dev::gather_item<T, G, VPL, W>(it, lg, sd.idx, sd.inc_w, sd.inv_norm, sd.src, sd.self_in,
                                   sd.out, dv, keep, scale, sd.partials);
  }
}

template <typename T, int GA, int VA, int GL, int VL, bool W>
__global__ void __launch_bounds__(256)
batched_persistent_kernel(const int4* __restrict__ items, const int32_t* __restrict__ item_g,
                          int32_t n_a, int32_t n_b, int32_t n_rest,
                          const GraphSide* __restrict__ sides, int32_t n_graphs, int32_t dv,
                          float keep, float scale, int32_t* __restrict__ counter) {
  constexpr int32_t kPerA = (32 / GA) * kTaskPasses;   // items per task
  constexpr int32_t kPerL = (32 / GL) * kTaskPasses;
  const int lane = threadIdx.x & 31;
  // tasks: the rest (items [n_a + n_b, n)), then B, then A, each from its end
  const int32_t t_rest = (int32_t)(((int64_t)n_rest + kPerL - 1) / kPerL);
  const int32_t t_b = (int32_t)(((int64_t)n_b + kPerL - 1) / kPerL);
  const int32_t t_a = (int32_t)(((int64_t)n_a + kPerA - 1) / kPerA);
  const int32_t n_tasks = t_rest + t_b + t_a;
  while (true) {
    int32_t t = 0;
    if (lane == 0) t = atomicAdd(counter, 1);
    t = __shfl_sync(dev::kFull, t, 0);
    if (t >= n_tasks) break;                                   // warp-uniform
    if (t < t_rest + t_b) {
      const bool rest = t < t_rest;
      const int32_t base = rest ? n_a + n_b : n_a;             // the class's items
      const int32_t end = rest ? n_a + n_b + n_rest : n_a + n_b;
      const int32_t tt = rest ? t : t - t_rest;
      const int32_t hi = end - tt * kPerL;
      const int32_t lo = hi - kPerL > base ? hi - kPerL : base;
      persistent_task<T, GL, VL, W>(items, item_g, lo, hi, sides, n_graphs, dv, keep, scale);
    } else {
      const int32_t tt = t - t_rest - t_b;
      const int32_t hi = n_a - tt * kPerA;
      const int32_t lo = hi - kPerA > 0 ? hi - kPerA : 0;
      persistent_task<T, GA, VA, W>(items, item_g, lo, hi, sides, n_graphs, dv, keep, scale);
    }
  }
}

constexpr int kFinThreads = 1024;

template <typename T>
__global__ void __launch_bounds__(kFinThreads)
batched_finalize_kernel(const int4* __restrict__ long_desc, const int32_t* __restrict__ long_g,
                        int32_t n_mid, int32_t n_huge, int32_t mid_blocks,
                        const GraphSide* __restrict__ sides, int32_t n_graphs, int32_t dv,
                        float keep, float scale) {
  extern __shared__ float4 sm4[];
  const bool mid = (int32_t)blockIdx.x < mid_blocks;
  const int32_t k = mid ? (int32_t)(blockIdx.x * (kFinThreads / 32) + (threadIdx.x >> 5))
                        : n_mid + (int32_t)blockIdx.x - mid_blocks;
  if (k >= (mid ? n_mid : n_mid + n_huge)) return;
  const int32_t gi = long_g[k];
  if (gi < 0 || gi >= n_graphs) return;   // (cannot be flagged without a graph)
  const GraphSide sd = sides[gi];
  const int4 ds = long_desc[k];
  // self-check: the row and its chunk run must lie inside the graph's arrays
  if (ds.x < 0 || ds.x >= sd.self_rows || ds.z < 1 || ds.y < 0 ||
      (int64_t)ds.y + ds.z > sd.n_slots || (mid && ds.z > kMidChunks)) {
    if (sd.err && (threadIdx.x & 31) == 0) atomicOr(sd.err, (int32_t)ERRBIT_BAD_ITEM);
    return;   // uniform per warp (mid) or per block (huge)
  }
  if (mid) {
    dev::finalize_mid<T>(ds, threadIdx.x & 31, sd.partials, sd.inv_norm, sd.self_in, sd.out, dv,
                         keep, scale);
    return;
  }
  dev::finalize_huge<T>(ds, reinterpret_cast<float*>(sm4), sd.partials, sd.inv_norm, sd.self_in,
                        sd.out, dv, keep, scale);
}

// index of the segment of `prefix` (n+1 ascending offsets) holding i
__device__ __forceinline__ int32_t segment_of(const int64_t* __restrict__ prefix, int32_t n,
                                              int64_t i) {
  int32_t lo = 0, hi = n;   // prefix[lo] <= i < prefix[hi]
  while (hi - lo > 1) {
    const int32_t mid = (lo + hi) >> 1;
    if (prefix[mid] <= i) lo = mid;
    else hi = mid;
  }
  return lo;
}

__global__ void batched_project_kernel(const ProjDesc* __restrict__ pd,
                                       const int64_t* __restrict__ prefix, int32_t n,
                                       int64_t total, int32_t dv) {
  if (prefix[n] != total) return;   // self-check: the table is the one the host built
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t g = segment_of(prefix, n, i);
    const ProjDesc p = pd[g];
    const int64_t local = i - prefix[g];
    const int64_t row = local / dv;
    const int32_t col = (int32_t)(local - row * dv);
    if (row < p.n_f) {
      p.zf_v[local] = p.zc_v[(size_t)p.rep_v[row] * dv + col];
    } else {
      const int64_t e = row - p.n_f;
      const int32_t r = p.rep_e[e];
      const uint4* s = (r >= 0) ? p.zc_e + (size_t)r * dv : p.zc_v + (size_t)(-1 - r) * dv;
      p.zf_e[e * dv + col] = s[col];
    }
  }
}

__global__ void batched_copy_kernel(const CopyDesc* __restrict__ cd,
                                    const int64_t* __restrict__ prefix, int32_t n,
                                    int64_t total) {
  if (prefix[n] != total) return;   // self-check: the table is the one the host built
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t g = segment_of(prefix, n, i);
    cd[g].dst[i - prefix[g]] = cd[g].src[i - prefix[g]];
  }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------

struct BSide {
  int4* items = nullptr;
  int32_t* item_g = nullptr;
  int32_t n_cls[3] = {0, 0, 0};   // A rows, B rows, the rest (C, D rows and chunks)
  int4* long_desc = nullptr;
  int32_t* long_g = nullptr;
  int32_t n_mid = 0, n_huge = 0;
  GraphSide* sides = nullptr;     // device, indexed by graph
  int32_t n_graphs = 0;
  bool weighted = false;
};

struct BStep {
  BSide side[2];                  // 0: hyperedge rows, 1: node rows
  ProjDesc* proj = nullptr;
  int64_t* proj_prefix = nullptr;
  int32_t n_proj = 0;
  CopyDesc* copies = nullptr;
  int64_t* copy_prefix = nullptr;
  int32_t n_copies = 0;
  int64_t proj_total = 0, copy_total = 0;   // vectors to move
};

int next_pow2(int x) {
  int p = 1;
  while (p < x) p <<= 1;
  return p;
}

}  // namespace
}  // namespace hnv

using namespace hnv;

struct hnv_batch {
  std::vector<hnv_graph*> graphs;
  std::vector<uint64_t> generation;   // each graph's hierarchy generation at creation
  int device = 0;
  cudaStream_t cap_stream = nullptr;
  // side streams: a half-sweep's row classes run concurrently (see enqueue_half)
  cudaStream_t aux[2] = {nullptr, nullptr};
  cudaEvent_t fork_ev = nullptr;
  cudaEvent_t join_ev[2] = {nullptr, nullptr};
  std::vector<int> top;            // coarsest level of each graph
  int Lmax = 0;
  PlanShape shape;
  int lanes[3] = {0, 0, 0};        // lanes per row of classes A, B, rest (0: default)
  // per-graph plans for `shape`: plans[side][graph][level]
  std::vector<std::vector<SplitPlan>> plans[2];
  std::vector<void*> plan_owned;
  bool plans_ready = false;
  size_t plans_row_bytes = 0;
  // step structures for one (dtype, d, buffers)
  std::vector<BStep> steps;
  std::vector<void*> step_owned;
  float* partials = nullptr;
  uint8_t* arena[2] = {nullptr, nullptr};
  int built_dt = -1, built_d = -1;
  const void* built_zc = nullptr;
  const void* built_zv = nullptr;
  const void* built_ze = nullptr;
  // captured V-cycle
  cudaGraphExec_t exec = nullptr;
  float exec_omega = -1.f;
  int exec_sweeps = -1;
  int64_t exec_kernels = 0;        // kernel nodes of the captured V-cycle
  int exec_kernel = -1;            // the half-sweep kernel it was captured with
  // half-sweep kernel: 0 one launch per row class, 1 one persistent launch
  int kernel = HNV_BATCH_KERNEL_PER_CLASS;
  // task counters of the persistent launches, one per half-sweep of a V-cycle
  int32_t* counters = nullptr;
  int64_t counters_n = 0;
  std::vector<int64_t> coarse_off, v_off, e_off;   // row offsets (count + 1)
};

namespace hnv {
namespace {

std::mutex g_tune_mu;
std::map<std::vector<int64_t>, std::pair<PlanShape, std::vector<int>>> g_tune_cache;

void free_list(std::vector<void*>& v, cudaStream_t s) {
  for (void* p : v) dev_free(p, s);
  v.clear();
}

int alloc_into(std::vector<void*>& owned, void** p, size_t bytes, cudaStream_t s) {
  HNV_CHECK(dev_alloc(p, bytes ? bytes : 16, s));
  owned.push_back(*p);
  return HNV_OK;
}

// Row-class plans of every graph and level. Where the single-graph path
// cuts long rows into panels (a neighbour table far larger than L2), the
// batch builds the same panel plan from the level's own regular plan, so
// both sum every row in the same order; elsewhere it uses its tuned shape.
int build_plans(hnv_batch* b, size_t row_bytes, cudaStream_t s, int only_level = -1) {
  BTRACE("build_plans row_bytes=%zu only_level=%d", row_bytes, only_level);
  free_list(b->plan_owned, s);
  for (int side = 0; side < 2; ++side) b->plans[side].assign(b->graphs.size(), {});
  for (size_t i = 0; i < b->graphs.size(); ++i) {
    hnv_graph* g = b->graphs[i];
    const int L = (int)g->levels.size();
    for (int side = 0; side < 2; ++side) b->plans[side][i].assign(L, SplitPlan());
    for (int l = 0; l < L; ++l) {
      if (only_level >= 0 && l != only_level) continue;
      Level& lv = g->levels[l];
      for (int side = 0; side < 2; ++side) {
        const int32_t rows = side == 0 ? lv.m : lv.n, cols = side == 0 ? lv.n : lv.m;
        const int32_t* ptr = side == 0 ? lv.e_ptr : lv.v_ptr;
        SplitPlan& out = b->plans[side][i][l];
        int P = 1;
        if (rows > 0 && cols > 0)
          HNV_CHECK(build_panel_plan(g, &b->plan_owned, side == 0 ? lv.planE : lv.planV, ptr,
                                     side == 0 ? lv.e_nodes : lv.v_edges, cols,
                                     (int64_t)cols * (int64_t)row_bytes, &out, &P, s));
        if (P <= 1) HNV_CHECK(build_split_plan(g, &b->plan_owned, ptr, rows, &out, s, b->shape));
        BTRACE("plan graph %zu level %d side %d: P=%d a=%d b=%d c=%d d=%d chunks=%d mid=%d huge=%d",
               i, l, side, P, out.n_a, out.n_b, out.n_c, out.n_d, out.n_chunks, out.n_mid,
               out.n_huge);
      }
    }
  }
  b->plans_ready = only_level < 0;
  b->plans_row_bytes = row_bytes;
  return HNV_OK;
}

void free_steps(hnv_batch* b, cudaStream_t s) {
  free_list(b->step_owned, s);
  b->steps.clear();
  b->partials = nullptr;
  b->arena[0] = b->arena[1] = nullptr;
  b->built_dt = b->built_d = -1;
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
}

// Work lists, pointer tables and buffers of every step for (dt, d) and the
// caller's buffers. `only_step` >= 0 builds that step only (the autotuner
// times step 0).
int build_steps(hnv_batch* b, int dt, int d, const uint8_t* zc, uint8_t* zv0, uint8_t* ze0,
                cudaStream_t s, int only_step = -1) {
  BTRACE("build_steps dt=%d d=%d only_step=%d Lmax=%d", dt, d, only_step, b->Lmax);
  free_steps(b, s);
  const size_t rb = (dt == HNV_BF16 ? 2 : 4) * (size_t)d;
  const int32_t dv = (int32_t)(rb / 16);
  const size_t G = b->graphs.size();
  b->steps.assign(b->Lmax + 1, BStep());
  // arenas for levels >= 1 (parity of the level)
  size_t arena_rows = 0;
  for (int st = 1; st <= b->Lmax; ++st) {
    size_t rows = 0;
    for (size_t i = 0; i < G; ++i)
      if (b->top[i] >= st) rows += (size_t)b->graphs[i]->levels[st].n + b->graphs[i]->levels[st].m;
    arena_rows = std::max(arena_rows, rows);
  }
  if (arena_rows > 0 && only_step != 0) {
    HNV_CHECK(alloc_into(b->step_owned, (void**)&b->arena[0], arena_rows * rb, s));
    HNV_CHECK(alloc_into(b->step_owned, (void**)&b->arena[1], arena_rows * rb, s));
  }
  // row pointers of graph i at level st
  std::vector<std::vector<uint8_t*>> zvp(b->Lmax + 1, std::vector<uint8_t*>(G, nullptr));
  std::vector<std::vector<uint8_t*>> zep = zvp;
  for (int st = 0; st <= b->Lmax; ++st) {
    size_t off = 0;
    for (size_t i = 0; i < G; ++i) {
      if (b->top[i] < st) continue;
      const Level& lv = b->graphs[i]->levels[st];
      if (st == 0) {
        zvp[st][i] = zv0 + (size_t)b->v_off[i] * rb;
        zep[st][i] = ze0 + (size_t)b->e_off[i] * rb;
      } else {
        zvp[st][i] = b->arena[st & 1] + off * rb;
        zep[st][i] = zvp[st][i] + (size_t)lv.n * rb;
        off += (size_t)lv.n + lv.m;
      }
    }
  }
  // partials: the largest step-side total
  size_t max_chunks = 1;
  for (int st = 0; st <= b->Lmax; ++st)
    for (int side = 0; side < 2; ++side) {
      size_t c = 0;
      for (size_t i = 0; i < G; ++i)
        if (b->top[i] >= st) c += b->plans[side][i][st].n_chunks;
      max_chunks = std::max(max_chunks, c);
    }
  HNV_CHECK(alloc_into(b->step_owned, (void**)&b->partials, max_chunks * sizeof(float) * d, s));

  for (int st = 0; st <= b->Lmax; ++st) {
    if (only_step >= 0 && st != only_step) continue;
    BStep& S = b->steps[st];
    for (int side = 0; side < 2; ++side) {
      BSide& B = S.side[side];
      B.weighted = side == 1;
      std::vector<GraphSide> hs(G);
      B.n_graphs = (int32_t)G;
      int64_t n_items = 0, n_long = 0, chunk_base = 0;
      for (size_t i = 0; i < G; ++i) {
        if (b->top[i] < st) continue;
        const Level& lv = b->graphs[i]->levels[st];
        const SplitPlan& p = b->plans[side][i][st];
        GraphSide& gs = hs[i];
        if (side == 0) {
          gs.idx = lv.e_nodes;
          gs.inc_w = nullptr;
          gs.inv_norm = lv.inv_size_e;
          gs.src = (const uint4*)zvp[st][i];
          gs.self_in = (const uint4*)zep[st][i];
          gs.out = (uint4*)zep[st][i];
          gs.self_rows = lv.m;
        } else {
          gs.idx = lv.v_edges;
          gs.inc_w = lv.v_w;
          gs.inv_norm = lv.inv_deg_v;
          gs.src = (const uint4*)zep[st][i];
          gs.self_in = (const uint4*)zvp[st][i];
          gs.out = (uint4*)zvp[st][i];
          gs.self_rows = lv.n;
        }
        gs.nnz = lv.nnz;
        gs.n_slots = p.n_chunks;
        gs.err = b->graphs[i]->d_err;
        gs.partials = b->partials + (size_t)chunk_base * d;
        chunk_base += p.n_chunks;
        n_items += (int64_t)p.n_a + p.n_b + p.n_c + p.n_d + p.n_chunks;
        n_long += (int64_t)p.n_mid + p.n_huge;
      }
      HNV_CHECK(alloc_into(b->step_owned, (void**)&B.sides, sizeof(GraphSide) * G, s));
      HNV_CUDA(cudaMemcpyAsync(B.sides, hs.data(), sizeof(GraphSide) * G, cudaMemcpyHostToDevice, s));
      HNV_CHECK(alloc_into(b->step_owned, (void**)&B.items, sizeof(int4) * (size_t)n_items, s));
      HNV_CHECK(alloc_into(b->step_owned, (void**)&B.item_g, sizeof(int32_t) * (size_t)n_items, s));
      HNV_CHECK(alloc_into(b->step_owned, (void**)&B.long_desc, sizeof(int4) * (size_t)n_long, s));
      HNV_CHECK(alloc_into(b->step_owned, (void**)&B.long_g, sizeof(int32_t) * (size_t)n_long, s));
      std::vector<int32_t> hg_items, hg_long;
      hg_items.reserve(n_items);
      hg_long.reserve(n_long);
      int64_t pos = 0;
      for (int cls = 0; cls < 3; ++cls) {
        int64_t cls_count = 0;
        for (size_t i = 0; i < G; ++i) {
          if (b->top[i] < st) continue;
          const SplitPlan& p = b->plans[side][i][st];
          int64_t first = 0, count = 0;
          if (cls == 0) { first = 0; count = p.n_a; }
          else if (cls == 1) { first = p.n_a; count = p.n_b; }
          else { first = (int64_t)p.n_a + p.n_b; count = (int64_t)p.n_c + p.n_d + p.n_chunks; }
          if (count == 0) continue;
          HNV_CUDA(cudaMemcpyAsync(B.items + pos, p.items + first, sizeof(int4) * count,
                                   cudaMemcpyDeviceToDevice, s));
          hg_items.insert(hg_items.end(), count, (int32_t)i);
          pos += count;
          cls_count += count;
        }
        B.n_cls[cls] = (int32_t)cls_count;
      }
      int64_t lpos = 0;
      for (int part = 0; part < 2; ++part) {   // rows with few chunks first, then the rest
        int64_t cnt_part = 0;
        for (size_t i = 0; i < G; ++i) {
          if (b->top[i] < st) continue;
          const SplitPlan& p = b->plans[side][i][st];
          const int64_t first = part == 0 ? 0 : p.n_mid;
          const int64_t count = part == 0 ? p.n_mid : p.n_huge;
          if (count == 0) continue;
          HNV_CUDA(cudaMemcpyAsync(B.long_desc + lpos, p.long_desc + first, sizeof(int4) * count,
                                   cudaMemcpyDeviceToDevice, s));
          hg_long.insert(hg_long.end(), count, (int32_t)i);
          lpos += count;
          cnt_part += count;
        }
        if (part == 0) B.n_mid = (int32_t)cnt_part;
        else B.n_huge = (int32_t)cnt_part;
      }
      if (n_items)
        HNV_CUDA(cudaMemcpyAsync(B.item_g, hg_items.data(), sizeof(int32_t) * n_items,
                                 cudaMemcpyHostToDevice, s));
      if (n_long)
        HNV_CUDA(cudaMemcpyAsync(B.long_g, hg_long.data(), sizeof(int32_t) * n_long,
                                 cudaMemcpyHostToDevice, s));
      HNV_CUDA(cudaStreamSynchronize(s));   // the host vectors above die here
      BTRACE("step %d side %d: items %lld (A %d B %d rest %d) long %lld (mid %d huge %d)", st,
             side, (long long)n_items, B.n_cls[0], B.n_cls[1], B.n_cls[2], (long long)n_long,
             B.n_mid, B.n_huge);
    }
    // projections onto level st and starting rows at level st
    std::vector<ProjDesc> pd;
    std::vector<int64_t> ppre{0};
    std::vector<CopyDesc> cd;
    std::vector<int64_t> cpre{0};
    for (size_t i = 0; i < G; ++i) {
      if (b->top[i] < st) continue;
      const Level& lv = b->graphs[i]->levels[st];
      if (b->top[i] > st) {
        pd.push_back(ProjDesc{lv.rep_v, lv.rep_e, lv.n, lv.m, (const uint4*)zvp[st + 1][i],
                              (const uint4*)zep[st + 1][i], (uint4*)zvp[st][i],
                              (uint4*)zep[st][i]});
        ppre.push_back(ppre.back() + ((int64_t)lv.n + lv.m) * dv);
      } else {
        const uint8_t* src = zc + (size_t)b->coarse_off[i] * rb;
        if (lv.n > 0) {
          cd.push_back(CopyDesc{(const uint4*)src, (uint4*)zvp[st][i]});
          cpre.push_back(cpre.back() + (int64_t)lv.n * dv);
        }
        if (lv.m > 0) {
          cd.push_back(CopyDesc{(const uint4*)(src + (size_t)lv.n * rb), (uint4*)zep[st][i]});
          cpre.push_back(cpre.back() + (int64_t)lv.m * dv);
        }
      }
    }
    S.n_proj = (int32_t)pd.size();
    S.n_copies = (int32_t)cd.size();
    S.proj_total = ppre.back();
    S.copy_total = cpre.back();
    if (S.n_proj) {
      HNV_CHECK(alloc_into(b->step_owned, (void**)&S.proj, sizeof(ProjDesc) * pd.size(), s));
      HNV_CHECK(alloc_into(b->step_owned, (void**)&S.proj_prefix, sizeof(int64_t) * ppre.size(), s));
      HNV_CUDA(cudaMemcpyAsync(S.proj, pd.data(), sizeof(ProjDesc) * pd.size(), cudaMemcpyHostToDevice, s));
      HNV_CUDA(cudaMemcpyAsync(S.proj_prefix, ppre.data(), sizeof(int64_t) * ppre.size(),
                               cudaMemcpyHostToDevice, s));
    }
    if (S.n_copies) {
      HNV_CHECK(alloc_into(b->step_owned, (void**)&S.copies, sizeof(CopyDesc) * cd.size(), s));
      HNV_CHECK(alloc_into(b->step_owned, (void**)&S.copy_prefix, sizeof(int64_t) * cpre.size(), s));
      HNV_CUDA(cudaMemcpyAsync(S.copies, cd.data(), sizeof(CopyDesc) * cd.size(), cudaMemcpyHostToDevice, s));
      HNV_CUDA(cudaMemcpyAsync(S.copy_prefix, cpre.data(), sizeof(int64_t) * cpre.size(),
                               cudaMemcpyHostToDevice, s));
    }
    HNV_CUDA(cudaStreamSynchronize(s));
  }
  b->built_dt = dt;
  b->built_d = d;
  return HNV_OK;
}

// lanes per row of class c (0: A, 1: B, 2: rest) for rows of dv vectors
int class_lanes(const hnv_batch* b, int c, int dv) {
  const int natural[3] = {16, 16, 32};   // the single-graph defaults
  int g = b->lanes[c] > 0 ? b->lanes[c] : natural[c];
  g = std::min(g, next_pow2(dv));
  g = std::max(g, next_pow2((dv + 7) / 8));
  return std::min(g, 32);
}

template <typename T, int G, int VPL, bool W>
int launch_batched_items(const BSide& B, int64_t first, int32_t count, int dv, float keep,
                         float scale, cudaStream_t s) {
  if (count <= 0) return HNV_OK;
  constexpr int R = 32 / G;
  auto kern = batched_gather_kernel<T, G, VPL, W>;
  const int64_t warps = ((int64_t)count + R - 1) / R;
  // one pass per warp in two-warp blocks, as the single-graph gathers. A
  // resident grid of 256-thread blocks looping over the list measured 7.5%
  // (FP32) and 8% (BF16) slower on the 256-graph batch in one process
  // (V-cycle 322.6 against 298.4 ms, 208.9 against 191.8 ms, direct
  // launches, with the row classes and lanes tuned for these launches).
  const int64_t blocks = (warps + 1) / 2;
  BTRACE("launch gather G=%d VPL=%d W=%d first=%lld count=%d blocks=%lld", G, VPL, (int)W,
         (long long)first, count, (long long)blocks);
  return launch("batched_gather", kern, (unsigned)blocks, 64, 0, s,
                (const int4*)(B.items + first), (const int32_t*)(B.item_g + first), count,
                (const GraphSide*)B.sides, B.n_graphs, dv, keep, scale);
}

template <typename T, bool W>
int launch_batched_dispatch(int G, int VPL, const BSide& B, int64_t first, int32_t count, int dv,
                            float keep, float scale, cudaStream_t s) {
#define HNV_BCASE(g, v)                                                                      \
  if (G == g && VPL == v)                                                                    \
    return launch_batched_items<T, g, v, W>(B, first, count, dv, keep, scale, s);
  HNV_BCASE(1, 1) HNV_BCASE(2, 1) HNV_BCASE(2, 2) HNV_BCASE(2, 4) HNV_BCASE(2, 8)
  HNV_BCASE(4, 1) HNV_BCASE(4, 2) HNV_BCASE(4, 4) HNV_BCASE(4, 8)
  HNV_BCASE(8, 1) HNV_BCASE(8, 2) HNV_BCASE(8, 4) HNV_BCASE(8, 8)
  HNV_BCASE(16, 1) HNV_BCASE(16, 2) HNV_BCASE(16, 4) HNV_BCASE(16, 8)
  HNV_BCASE(32, 1) HNV_BCASE(32, 2) HNV_BCASE(32, 4) HNV_BCASE(32, 8)
#undef HNV_BCASE
  HNV_FAIL(HNV_ERR_UNSUPPORTED_D, "no batched gather variant for G=%d VPL=%d", G, VPL);
}

// The three row classes touch disjoint rows (chunks write only partials):
// classes B and the rest run on the batch's side streams, forked from s and
// joined back (inside a capture these become parallel branches of the
// graph); the split-row reduction follows the last class on its stream.
template <typename T, int GA, int VA, int GL, int VL, bool W>
int launch_persistent(const BSide& B, int dv, float keep, float scale, int32_t* counter,
                      cudaStream_t s) {
  const int32_t n = B.n_cls[0] + B.n_cls[1] + B.n_cls[2];
  if (n <= 0) return HNV_OK;
  auto kern = batched_persistent_kernel<T, GA, VA, GL, VL, W>;
  int per_sm = 0;
  HNV_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kPersistThreads, 0));
  if (per_sm < 1) per_sm = 1;
  const int64_t tasks = ((int64_t)B.n_cls[0] + (32 / GA) * kTaskPasses - 1) / ((32 / GA) * kTaskPasses) +
                        ((int64_t)B.n_cls[1] + B.n_cls[2] + 2 * (32 / GL) * kTaskPasses) /
                            ((32 / GL) * kTaskPasses);
  const int64_t wpb = kPersistThreads / 32;
  const int64_t blocks = std::min<int64_t>((tasks + wpb - 1) / wpb, (int64_t)num_sms() * per_sm);
  BTRACE("launch persistent GA=%d VA=%d GL=%d VL=%d W=%d items=%d tasks<=%lld blocks=%lld", GA,
         VA, GL, VL, (int)W, n, (long long)tasks, (long long)blocks);
  return launch("batched_persistent", kern, (unsigned)blocks, kPersistThreads, 0, s,
                (const int4*)B.items, (const int32_t*)B.item_g, B.n_cls[0], B.n_cls[1],
                B.n_cls[2], (const GraphSide*)B.sides, B.n_graphs, dv, keep, scale, counter);
}

// GL = one lane per row vector (at most 32); GA = GL / 4 (at least 1) with
// the vectors that makes per lane.
template <typename T, bool W>
int launch_persistent_dispatch(const BSide& B, int dv, float keep, float scale, int32_t* counter,
                               cudaStream_t s) {
  const int GL = std::min(next_pow2(dv), 32);
  const int VL = next_pow2((dv + GL - 1) / GL);
#define HNV_PCASE(ga, va, gl, vl)                                                            \
  if (GL == gl && VL == vl)                                                                  \
    return launch_persistent<T, ga, va, gl, vl, W>(B, dv, keep, scale, counter, s);
  HNV_PCASE(1, 1, 1, 1) HNV_PCASE(1, 2, 2, 1) HNV_PCASE(1, 4, 4, 1) HNV_PCASE(2, 4, 8, 1)
  HNV_PCASE(4, 4, 16, 1) HNV_PCASE(8, 4, 32, 1) HNV_PCASE(8, 8, 32, 2) HNV_PCASE(16, 8, 32, 4)
  HNV_PCASE(32, 8, 32, 8)
#undef HNV_PCASE
  HNV_FAIL(HNV_ERR_UNSUPPORTED_D, "no persistent variant for %d lanes x %d vectors", GL, VL);
}

template <typename T>
int enqueue_finalize(const BSide& B, int dv, float keep, float omega, cudaStream_t s);

template <typename T>
int enqueue_half(const hnv_batch* b, const BSide& B, int dv, float omega, int32_t* counter,
                 cudaStream_t s) {
  const float keep = 1.0f - omega;
  if (b->kernel == HNV_BATCH_KERNEL_PERSISTENT) {
    if (B.weighted)
      HNV_CHECK((launch_persistent_dispatch<T, true>(B, dv, keep, omega, counter, s)));
    else
      HNV_CHECK((launch_persistent_dispatch<T, false>(B, dv, keep, omega, counter, s)));
    return enqueue_finalize<T>(B, dv, keep, omega, s);
  }
  const bool conc = b->aux[0] && b->aux[1] && B.n_cls[1] > 0 && B.n_cls[2] > 0;
  cudaStream_t cs[3] = {s, s, s};
  if (conc) {
    HNV_CUDA(cudaEventRecord(b->fork_ev, s));
    for (int i = 0; i < 2; ++i) {
      HNV_CUDA(cudaStreamWaitEvent(b->aux[i], b->fork_ev, 0));
      cs[i + 1] = b->aux[i];
    }
  }
  int64_t first = 0;
  for (int c = 0; c < 3; ++c) {
    const int G = class_lanes(b, c, dv);
    const int VPL = next_pow2((dv + G - 1) / G);
    if (B.weighted)
      HNV_CHECK((launch_batched_dispatch<T, true>(G, VPL, B, first, B.n_cls[c], dv, keep, omega, cs[c])));
    else
      HNV_CHECK((launch_batched_dispatch<T, false>(G, VPL, B, first, B.n_cls[c], dv, keep, omega, cs[c])));
    first += B.n_cls[c];
  }
  // the reduction follows the chunks' class
  HNV_CHECK(enqueue_finalize<T>(B, dv, keep, omega, cs[2]));
  if (conc) {
    cudaStream_t origin = cs[0];
    for (int i = 0; i < 2; ++i) {
      HNV_CUDA(cudaEventRecord(b->join_ev[i], b->aux[i]));
      HNV_CUDA(cudaStreamWaitEvent(origin, b->join_ev[i], 0));
    }
  }
  return HNV_OK;
}

template <typename T>
int enqueue_finalize(const BSide& B, int dv, float keep, float omega, cudaStream_t s) {
  if (B.n_mid + B.n_huge <= 0) return HNV_OK;
  constexpr int N = dev::VecT<T>::N;
  const int32_t mid_blocks = (B.n_mid + kFinThreads / 32 - 1) / (kFinThreads / 32);
  const size_t smem = sizeof(float) * (size_t)(kFinThreads / dv) * dv * N;
  BTRACE("launch finalize mid=%d huge=%d smem=%zu", B.n_mid, B.n_huge, smem);
  return launch("batched_finalize", batched_finalize_kernel<T>, (unsigned)(mid_blocks + B.n_huge),
                kFinThreads, smem, s, (const int4*)B.long_desc, (const int32_t*)B.long_g,
                B.n_mid, B.n_huge, mid_blocks, (const GraphSide*)B.sides, B.n_graphs, dv, keep,
                omega);
}

// Counter slots the persistent launches of one V-cycle use: kCountersPerHalf
// per half-sweep (2 half-sweeps per sweep of every step). Grows the batch's array if needed;
// a V-cycle already queued on `user` may still use the old array, so that
// stream is drained before the array is released.
int ensure_counters(hnv_batch* b, int64_t n, cudaStream_t s, cudaStream_t user) {
  if (n <= b->counters_n && b->counters) return HNV_OK;
  if (b->counters) {
    HNV_CUDA(cudaStreamSynchronize(user));
    dev_free(b->counters, s);
  }
  b->counters = nullptr;
  b->counters_n = 0;
  HNV_CHECK(dev_alloc((void**)&b->counters, sizeof(int32_t) * (size_t)(n > 0 ? n : 1), s));
  b->counters_n = n > 0 ? n : 1;
  return HNV_OK;
}

template <typename T>
int enqueue_vcycle(const hnv_batch* b, int d, float omega, int sweeps, cudaStream_t s) {
  const int dv = (int)(d * sizeof(T) / 16);
  int32_t* counter = b->counters;
  if (b->kernel == HNV_BATCH_KERNEL_PERSISTENT) {
    const int64_t need = (int64_t)(b->Lmax + 1) * sweeps * 2 * kCountersPerHalf;
    if (need > b->counters_n) HNV_FAIL(HNV_ERR_STATE, "persistent counters not allocated");
    if (need > 0) HNV_CUDA(cudaMemsetAsync(counter, 0, sizeof(int32_t) * (size_t)need, s));
  }
  for (int st = b->Lmax; st >= 0; --st) {
    const BStep& S = b->steps[st];
    BTRACE("enqueue step %d copies %d proj %d", st, S.n_copies, S.n_proj);
    if (S.n_copies) {
      BTRACE("launch copy step %d n=%d total=%lld", st, S.n_copies, (long long)S.copy_total);
      HNV_CHECK(launch("batched_copy", batched_copy_kernel, (unsigned)(num_sms() * 8), 256, 0, s,
                       (const CopyDesc*)S.copies, (const int64_t*)S.copy_prefix, S.n_copies,
                       S.copy_total));
    }
    if (S.n_proj) {
      BTRACE("launch project step %d n=%d total=%lld", st, S.n_proj, (long long)S.proj_total);
      HNV_CHECK(launch("batched_project", batched_project_kernel, (unsigned)(num_sms() * 8), 256, 0,
                       s, (const ProjDesc*)S.proj, (const int64_t*)S.proj_prefix, S.n_proj,
                       S.proj_total, dv));
    }
    for (int it = 0; it < sweeps; ++it) {
      HNV_CHECK(enqueue_half<T>(b, S.side[0], dv, omega, counter, s));
      HNV_CHECK(enqueue_half<T>(b, S.side[1], dv, omega, counter + kCountersPerHalf, s));
      if (b->kernel == HNV_BATCH_KERNEL_PERSISTENT) counter += 2 * kCountersPerHalf;
    }
  }
  return HNV_OK;
}

int enqueue(const hnv_batch* b, int dt, int d, float omega, int sweeps, cudaStream_t s) {
  return dt == HNV_BF16 ? enqueue_vcycle<__nv_bfloat16>(b, d, omega, sweeps, s)
                        : enqueue_vcycle<float>(b, d, omega, sweeps, s);
}

// milliseconds of one V-cycle of the batch with one sweep per level (median
// of the timed repetitions; the first run warms the caches)
int time_vcycle1(const hnv_batch* b, int dt, int d, float omega, cudaStream_t s, float* ms) {
  cudaEvent_t e0, e1;
  HNV_CUDA(cudaEventCreate(&e0));
  HNV_CUDA(cudaEventCreate(&e1));
  std::vector<float> t;
  int rc = HNV_OK;
  for (int r = 0; r < 4 && rc == HNV_OK; ++r) {
    cudaEventRecord(e0, s);
    rc = enqueue(b, dt, d, omega, 1, s);
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    float x = 0.f;
    cudaEventElapsedTime(&x, e0, e1);
    if (r > 0) t.push_back(x);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  HNV_CHECK(rc);
  std::sort(t.begin(), t.end());
  *ms = t[t.size() / 2];
  return HNV_OK;
}

std::vector<int64_t> tune_key(const hnv_batch* b, int dt, int d) {
  std::vector<int64_t> k{dt, d, (int64_t)b->graphs.size()};
  int64_t hist[2][24] = {{0}};
  for (hnv_graph* g : b->graphs) {
    const Level& lv = g->levels[0];
    std::vector<int32_t> e(lv.m + 1), v(lv.n + 1);
    cudaMemcpy(e.data(), lv.e_ptr, sizeof(int32_t) * (lv.m + 1), cudaMemcpyDeviceToHost);
    cudaMemcpy(v.data(), lv.v_ptr, sizeof(int32_t) * (lv.n + 1), cudaMemcpyDeviceToHost);
    for (int side = 0; side < 2; ++side) {
      const std::vector<int32_t>& p = side == 0 ? e : v;
      for (size_t r = 0; r + 1 < p.size(); ++r) {
        int len = p[r + 1] - p[r], bkt = 0;
        while (bkt < 23 && (1 << bkt) < len) ++bkt;
        ++hist[side][bkt];
      }
    }
  }
  // coarse signature: the share of rows per length bucket, in percent
  for (int side = 0; side < 2; ++side) {
    int64_t tot = 0;
    for (int64_t x : hist[side]) tot += x;
    for (int64_t x : hist[side]) k.push_back(tot ? (100 * x) / tot : 0);
  }
  return k;
}

}  // namespace
}  // namespace hnv

extern "C" {

int hnv_batch_create(hnv_graph* const* graphs, int32_t count, hnv_batch** out) {
  clear_error_detail();
  if (!out) HNV_FAIL(HNV_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!graphs || count < 1) HNV_FAIL(HNV_ERR_INVALID_ARG, "need at least one graph");
  int dev0 = -1;
  for (int32_t i = 0; i < count; ++i) {
    if (!graphs[i]) HNV_FAIL(HNV_ERR_INVALID_ARG, "graph %d is NULL", i);
    if (dev0 < 0) dev0 = graphs[i]->device;
    if (graphs[i]->device != dev0) HNV_FAIL(HNV_ERR_INVALID_ARG, "graphs on different devices");
  }
  // the graphs' arrays are read on the batch's own stream from here on
  for (int32_t i = 0; i < count; ++i) {
    const cudaError_t e = cudaStreamSynchronize(graphs[i]->stream);
    if (e != cudaSuccess) return cuda_status(e, "cudaStreamSynchronize");
  }
  BTRACE("create: %d graphs synchronised", count);
  hnv_batch* b = new (std::nothrow) hnv_batch();
  if (!b) HNV_FAIL(HNV_ERR_OOM, "host allocation failed");
  b->graphs.assign(graphs, graphs + count);
  for (int32_t i = 0; i < count; ++i) b->generation.push_back(graphs[i]->generation);
  b->device = dev0;
  b->coarse_off.assign(count + 1, 0);
  b->v_off.assign(count + 1, 0);
  b->e_off.assign(count + 1, 0);
  for (int32_t i = 0; i < count; ++i) {
    const hnv_graph* g = graphs[i];
    const int L = (int)g->levels.size() - 1;
    b->top.push_back(L);
    b->Lmax = std::max(b->Lmax, L);
    b->coarse_off[i + 1] = b->coarse_off[i] + g->levels[L].n + g->levels[L].m;
    b->v_off[i + 1] = b->v_off[i] + g->levels[0].n;
    b->e_off[i + 1] = b->e_off[i] + g->levels[0].m;
  }
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(dev0);
  cudaError_t e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork_ev, cudaEventDisableTiming);
  for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
    e = cudaStreamCreateWithFlags(&b->aux[i], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join_ev[i], cudaEventDisableTiming);
  }
  if (prev >= 0) cudaSetDevice(prev);
  if (e != cudaSuccess) {
    hnv_batch_free(b);
    return cuda_status(e, "cudaStreamCreate");
  }
  *out = b;
  return HNV_OK;
}

int hnv_batch_offsets(const hnv_batch* b, int64_t* coarsest_rows, int64_t* node_rows,
                      int64_t* edge_rows) {
  if (!b) HNV_FAIL(HNV_ERR_INVALID_ARG, "batch is NULL");
  const size_t n = b->coarse_off.size();
  if (coarsest_rows) std::memcpy(coarsest_rows, b->coarse_off.data(), n * sizeof(int64_t));
  if (node_rows) std::memcpy(node_rows, b->v_off.data(), n * sizeof(int64_t));
  if (edge_rows) std::memcpy(edge_rows, b->e_off.data(), n * sizeof(int64_t));
  return HNV_OK;
}

int hnv_batch_autotune(hnv_batch* b, hnv_dtype dt, int d, float omega, hnv_batch_tuning* chosen) {
  clear_error_detail();
  if (!b) HNV_FAIL(HNV_ERR_INVALID_ARG, "batch is NULL");
  if (dt != HNV_F32 && dt != HNV_BF16) HNV_FAIL(HNV_ERR_INVALID_ARG, "unknown dtype");
  if (d < 8 || d > 1024 || d % 8) HNV_FAIL(HNV_ERR_UNSUPPORTED_D, "d must be a multiple of 8 in [8, 1024]");
  for (size_t i = 0; i < b->graphs.size(); ++i)
    if (b->graphs[i]->generation != b->generation[i])
      HNV_FAIL(HNV_ERR_STATE, "graph %zu was coarsened again after the batch was created", i);
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(b->device);
  cudaStream_t s = b->cap_stream;
  int rc = HNV_OK;
  const std::vector<int64_t> key = tune_key(b, dt, d);
  PlanShape best_shape = b->shape;
  std::vector<int> best_lanes(4, 0);   // lanes of classes A, B, rest; [3]: kernel
  float best_ms = -1.f, persistent_ms = -1.f;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      best_shape = it->second.first;
      best_lanes = it->second.second;
    }
  }
  const bool cached = best_lanes[0] != 0 || best_lanes[3] == HNV_BATCH_KERNEL_PERSISTENT;
  const size_t rb = (dt == HNV_BF16 ? 2 : 4) * (size_t)d;
  const int dv = (int)(rb / 16);
  uint8_t* zbuf = nullptr;
  if (!cached) {
    // scratch rows for level 0 of every graph, also read as the coarsest
    // rows (no graph's coarsest level has more rows than its level 0;
    // contents do not affect timing)
    const size_t rows = (size_t)b->v_off.back() + b->e_off.back();
    rc = dev_alloc((void**)&zbuf, rows * rb, s);
    if (rc == HNV_OK) {
      const cudaError_t e = cudaMemsetAsync(zbuf, 0, rows * rb, s);
      if (e != cudaSuccess) rc = cuda_status(e, "cudaMemsetAsync");
    }
    const PlanShape shapes[3] = {{4, 16, 64}, {2, 8, 32}, {8, 32, 64}};
    if (rc == HNV_OK) rc = ensure_counters(b, (int64_t)(b->Lmax + 1) * 2 * kCountersPerHalf, s, s);
    for (int si = 0; si < 3 && rc == HNV_OK; ++si) {
      // plans and work lists depend on the class boundaries only; the lanes
      // per row and the kernel only change the launches
      b->shape = shapes[si];
      std::fill(b->lanes, b->lanes + 3, 0);
      rc = build_plans(b, rb, s);
      if (rc == HNV_OK)
        rc = build_steps(b, dt, d, zbuf, zbuf, zbuf + (size_t)b->v_off.back() * rb, s);
      b->kernel = HNV_BATCH_KERNEL_PER_CLASS;
      const int cand_a[3] = {2, 4, 8}, cand_b[3] = {4, 8, 16};
      for (int ia = 0; ia < 3 && rc == HNV_OK; ++ia)
        for (int ib = 0; ib < 3 && rc == HNV_OK; ++ib) {
          b->lanes[0] = cand_a[ia];
          b->lanes[1] = cand_b[ib];
          b->lanes[2] = 0;
          if (class_lanes(b, 0, dv) != cand_a[ia] || class_lanes(b, 1, dv) != cand_b[ib]) continue;
          float ms = 0.f;
          rc = time_vcycle1(b, dt, d, omega, s, &ms);
          if (rc == HNV_OK && (best_ms < 0.f || ms < best_ms)) {
            best_ms = ms;
            best_shape = shapes[si];
            best_lanes = {cand_a[ia], cand_b[ib], 0, HNV_BATCH_KERNEL_PER_CLASS};
          }
        }
      // the persistent kernel (its own lanes; the default class boundaries)
      if (si == 0 && rc == HNV_OK) {
        std::fill(b->lanes, b->lanes + 3, 0);
        b->kernel = HNV_BATCH_KERNEL_PERSISTENT;
        rc = time_vcycle1(b, dt, d, omega, s, &persistent_ms);
        if (rc == HNV_OK && (best_ms < 0.f || persistent_ms < best_ms)) {
          best_ms = persistent_ms;
          best_shape = shapes[si];
          best_lanes = {0, 0, 0, HNV_BATCH_KERNEL_PERSISTENT};
        }
      }
    }
    if (zbuf) dev_free(zbuf, s);
    if (rc == HNV_OK) {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      g_tune_cache[key] = {best_shape, best_lanes};
    }
  }
  if (rc == HNV_OK) {
    b->shape = best_shape;
    for (int c = 0; c < 3; ++c) b->lanes[c] = best_lanes[c];
    b->kernel = best_lanes[3];
    free_steps(b, s);
    b->plans_ready = false;
    if (chosen) {
      chosen->kernel = best_lanes[3];
      chosen->persistent_ms = persistent_ms;
      chosen->a_max = best_shape.a_max;
      chosen->b_max = best_shape.b_max;
      chosen->c_max = best_shape.c_max;
      chosen->lanes_a = class_lanes(b, 0, dv);
      chosen->lanes_b = class_lanes(b, 1, dv);
      chosen->lanes_rest = class_lanes(b, 2, dv);
      chosen->best_ms = best_ms;
      chosen->from_cache = cached ? 1 : 0;
    }
  }
  cudaStreamSynchronize(s);
  if (prev >= 0) cudaSetDevice(prev);
  return rc;
}

int hnv_batch_vcycle(hnv_batch* b, const void* z_coarsest, void* z_v_out, void* z_e_out,
                     hnv_dtype dt, int d, float omega, int sweeps_per_level, int use_cuda_graph,
                     hnv_stream_t stream) {
  NvtxRange nvtx("hnv batch vcycle");
  clear_error_detail();
  if (!b) HNV_FAIL(HNV_ERR_INVALID_ARG, "batch is NULL");
  if (dt != HNV_F32 && dt != HNV_BF16) HNV_FAIL(HNV_ERR_INVALID_ARG, "unknown dtype");
  if (d < 8 || d > 1024 || d % 8)
    HNV_FAIL(HNV_ERR_UNSUPPORTED_D, "batched d must be a multiple of 8 in [8, 1024]");
  if (!(omega >= 0.f && omega <= 1.f)) HNV_FAIL(HNV_ERR_INVALID_ARG, "omega must be in [0, 1]");
  if (sweeps_per_level < 0) HNV_FAIL(HNV_ERR_INVALID_ARG, "sweeps_per_level < 0");
  if (!z_coarsest || !z_v_out || !z_e_out) HNV_FAIL(HNV_ERR_INVALID_ARG, "NULL buffer");
  if ((reinterpret_cast<uintptr_t>(z_coarsest) | reinterpret_cast<uintptr_t>(z_v_out) |
       reinterpret_cast<uintptr_t>(z_e_out)) & 15u)
    HNV_FAIL(HNV_ERR_INVALID_ARG, "buffers must be 16-byte aligned");
  for (size_t i = 0; i < b->graphs.size(); ++i)
    if (b->graphs[i]->generation != b->generation[i])
      HNV_FAIL(HNV_ERR_STATE, "graph %zu was coarsened again after the batch was created", i);
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(b->device);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaStream_t cs = b->cap_stream;
  int rc = HNV_OK;
  do {
    const size_t rb = (dt == HNV_BF16 ? 2 : 4) * (size_t)d;
    if (!b->plans_ready || b->plans_row_bytes != rb) {
      if ((rc = build_plans(b, rb, cs)) != HNV_OK) break;
      free_steps(b, cs);
    }
    if (b->built_dt != (int)dt || b->built_d != d || b->built_zc != z_coarsest ||
        b->built_zv != z_v_out || b->built_ze != z_e_out || b->steps.empty()) {
      if ((rc = build_steps(b, dt, d, (const uint8_t*)z_coarsest, (uint8_t*)z_v_out,
                            (uint8_t*)z_e_out, cs)) != HNV_OK)
        break;
      b->built_zc = z_coarsest;
      b->built_zv = z_v_out;
      b->built_ze = z_e_out;
    }
    if (b->kernel == HNV_BATCH_KERNEL_PERSISTENT &&
        (rc = ensure_counters(b, (int64_t)(b->Lmax + 1) * sweeps_per_level * 2 * kCountersPerHalf,
                              cs, s)) != HNV_OK)
      break;
    // the caller's stream must see the set-up work done on the batch stream
    {
      const cudaError_t e = cudaStreamSynchronize(cs);
      if (e != cudaSuccess) {
        rc = cuda_status(e, "cudaStreamSynchronize");
        break;
      }
    }
    if (!use_cuda_graph) {
      rc = enqueue(b, (int)dt, d, omega, sweeps_per_level, s);
      BTRACE("direct enqueue rc=%d", rc);
      break;
    }
    if (!b->exec || b->exec_omega != omega || b->exec_sweeps != sweeps_per_level ||
        b->exec_kernel != b->kernel) {
      if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
      }
      cudaGraph_t graph = nullptr;
      cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) { rc = cuda_status(e, "cudaStreamBeginCapture"); break; }
      const int64_t before = hnv_kernel_launch_count();
      const int erc = enqueue(b, (int)dt, d, omega, sweeps_per_level, cs);
      // captured launches run at replay: count them there, not here
      b->exec_kernels = hnv_kernel_launch_count() - before;
      note_launches(-b->exec_kernels);
      e = cudaStreamEndCapture(cs, &graph);
      if (erc != HNV_OK) { if (graph) cudaGraphDestroy(graph); rc = erc; break; }
      if (e != cudaSuccess) { rc = cuda_status(e, "cudaStreamEndCapture"); break; }
      e = cudaGraphInstantiate(&b->exec, graph, 0);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess) { b->exec = nullptr; rc = cuda_status(e, "cudaGraphInstantiate"); break; }
      b->exec_omega = omega;
      b->exec_sweeps = sweeps_per_level;
      b->exec_kernel = b->kernel;
    }
    BTRACE("graph launch (%lld kernels)", (long long)b->exec_kernels);
    cudaError_t e = cudaGraphLaunch(b->exec, s);
    if (e != cudaSuccess) rc = cuda_status(e, "cudaGraphLaunch");
    else note_launches(b->exec_kernels);
  } while (0);
  if (prev >= 0) cudaSetDevice(prev);
  return rc;
}

int hnv_batch_set_kernel(hnv_batch* b, int kernel) {
  clear_error_detail();
  if (!b) HNV_FAIL(HNV_ERR_INVALID_ARG, "batch is NULL");
  if (kernel != HNV_BATCH_KERNEL_PER_CLASS && kernel != HNV_BATCH_KERNEL_PERSISTENT)
    HNV_FAIL(HNV_ERR_INVALID_ARG, "unknown half-sweep kernel %d", kernel);
  b->kernel = kernel;   // a captured V-cycle of the other kernel is re-captured on next use
  return HNV_OK;
}

int hnv_batch_get_kernel(const hnv_batch* b) { return b ? b->kernel : HNV_ERR_INVALID_ARG; }

void hnv_batch_free(hnv_batch* b) {
  if (!b) return;
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(b->device);
  if (b->cap_stream) {
    free_steps(b, b->cap_stream);
    free_list(b->plan_owned, b->cap_stream);
    if (b->counters) dev_free(b->counters, b->cap_stream);
    cudaStreamSynchronize(b->cap_stream);
    cudaStreamDestroy(b->cap_stream);
  }
  for (int i = 0; i < 2; ++i) {
    if (b->aux[i]) {
      cudaStreamSynchronize(b->aux[i]);
      cudaStreamDestroy(b->aux[i]);
    }
    if (b->join_ev[i]) cudaEventDestroy(b->join_ev[i]);
  }
  if (b->fork_ev) cudaEventDestroy(b->fork_ev);
  if (prev >= 0) cudaSetDevice(prev);
  delete b;
}

}  // extern "C"
