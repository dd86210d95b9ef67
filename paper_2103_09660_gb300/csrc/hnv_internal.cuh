// Internal declarations shared by the translation units of libhnv.so.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <utility>
#include <vector>

#include "hnv.h"

namespace hnv {

// ---------------------------------------------------------------------------
// Errors
// ---------------------------------------------------------------------------

// Records a one-line message for hnv_last_error_detail() (thread-local).
void set_error_detail(const char* fmt, ...);
void clear_error_detail();
int cuda_status(cudaError_t e, const char* what);

#define HNV_FAIL(code, ...)                 \
  do {                                      \
    ::hnv::set_error_detail(__VA_ARGS__);   \
    return (code);                          \
  } while (0)

#define HNV_CHECK(expr)                     \
  do {                                      \
    int hnv_s_ = (expr);                    \
    if (hnv_s_ != HNV_OK) return hnv_s_;    \
  } while (0)

#define HNV_CUDA(call)                                             \
  do {                                                             \
    cudaError_t hnv_e_ = (call);                                   \
    if (hnv_e_ != cudaSuccess) return ::hnv::cuda_status(hnv_e_, #call); \
  } while (0)

// Bits of the per-graph device error word (set with atomicOr by kernels that
// validate input; read back by the host after a synchronising step).
enum : int32_t {
  ERRBIT_NODE_RANGE = 1,    // an input node ID outside [0, n)
  ERRBIT_EMPTY_EDGE = 2,    // an input hyperedge with no members
  ERRBIT_BAD_WEIGHT = 4,    // a weight that is not finite and > 0
  ERRBIT_BAD_PTR = 8,       // edge_ptr not starting at 0 / decreasing
  ERRBIT_TIMEOUT = 16,      // a bounded device wait gave up (refinement)
  ERRBIT_BAD_ITEM = 32,     // a batched work item outside its graph's arrays (skipped)
  ERRBIT_BAD_FEATURE = 64   // a node feature that is not finite or exceeds 1e15 in magnitude
};

// ---------------------------------------------------------------------------
// Kernel launches
// ---------------------------------------------------------------------------

void note_launch();
void note_launches(int64_t k);   // k kernels at once (a replayed CUDA graph)
int num_sms();

// Launches kernel<<<grid, block, smem, s>>>(args...) and counts it. A launch
// with no blocks is skipped.
template <typename... KArgs, typename... Args>
int launch(const char* name, void (*kernel)(KArgs...), unsigned grid, unsigned block,
           size_t smem, cudaStream_t s, Args&&... args) {
  if (grid == 0) return HNV_OK;
  kernel<<<grid, block, smem, s>>>(static_cast<KArgs>(std::forward<Args>(args))...);
  note_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_status(e, name);
  return HNV_OK;
}

// Blocks for a grid-stride loop over `items` with `per_block` items per
// block, capped at `waves` blocks per SM.
unsigned grid_for(int64_t items, int64_t per_block, int waves = 8);

// ---------------------------------------------------------------------------
// Device memory (stream-ordered; replaceable through hnv_set_allocator)
// ---------------------------------------------------------------------------

int dev_alloc(void** p, size_t bytes, cudaStream_t s);
void dev_free(void* p, cudaStream_t s);

// Temporary device buffers released (stream-ordered) when the pool dies.
class TempPool {
 public:
  explicit TempPool(cudaStream_t s) : s_(s) {}
  ~TempPool() {
    for (void* p : ptrs_) dev_free(p, s_);
  }
  TempPool(const TempPool&) = delete;
  TempPool& operator=(const TempPool&) = delete;
  template <typename T>
  int get(T** out, size_t count) {
    void* p = nullptr;
    HNV_CHECK(dev_alloc(&p, (count ? count : 1) * sizeof(T), s_));
    ptrs_.push_back(p);
    *out = static_cast<T*>(p);
    return HNV_OK;
  }

 private:
  cudaStream_t s_;
  std::vector<void*> ptrs_;
};

// ---------------------------------------------------------------------------
// Phase timing (CUDA events on the launching stream)
// ---------------------------------------------------------------------------

bool timing_on();
// Records the start event of a phase; returns an opaque slot or -1.
int timing_begin(int phase, cudaStream_t s, double alg_bytes);
void timing_end(int slot, cudaStream_t s);

// An NVTX range (named in profiler timelines) for the scope's lifetime.
// NVTX is header-only: without a tool attached a range costs a check.
struct NvtxRange {
  explicit NvtxRange(const char* fmt, ...);
  ~NvtxRange();
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

struct PhaseScope {
  int slot;
  cudaStream_t s;
  PhaseScope(int phase, cudaStream_t st, double bytes) : slot(-1), s(st) {
    if (timing_on()) slot = timing_begin(phase, st, bytes);
  }
  ~PhaseScope() {
    if (slot >= 0) timing_end(slot, s);
  }
};

// ---------------------------------------------------------------------------
// Primitives (prims.cu)
// ---------------------------------------------------------------------------

// out[i] = sum_{j<i} in[i]; in == out allowed. If total != nullptr the sum of
// all n inputs is written to *total (device). n may be 0.
int exclusive_scan_i32(const int32_t* in, int32_t* out, int64_t n, int32_t* total,
                       cudaStream_t s);

// Stable LSD radix sort of 64-bit keys, one pass of 8 bits per entry of
// `shifts` (digit = (key >> shift) & 255), ping-ponging between keys and alt.
// *result receives whichever buffer holds the sorted keys.
int radix_sort_u64(uint64_t* keys, uint64_t* alt, int64_t n, const int* shifts,
                   int npasses, cudaStream_t s, uint64_t** result);

// Shifts for the passes that sort the low `low_bits` bits, then bits
// [32, 32 + high_bits). Returns the number of passes.
int radix_shifts(int low_bits, int high_bits, int* shifts);

// Number of bits needed to hold values in [0, count).
int bits_for_count(int64_t count);

// Visits every entry k of the rows [0, rows) of a CSR with offsets ptr as
// f(row, k). A warp takes 32 consecutive rows, whose entries are contiguous,
// and walks them 32 at a time (coalesced, every lane busy whatever the row
// lengths), finding each entry's row by a binary search over the 32 row
// starts held one per lane. Launch with one thread per row (any grid).
template <typename P, typename F>
__device__ __forceinline__ void csr_rows_warp_visit(int64_t rows, const P* __restrict__ ptr,
                                                    F f) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t r0 = ((int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32;
       r0 < rows; r0 += warps * 32) {
    const int64_t last = r0 + 32 < rows ? r0 + 32 : rows;
    const int64_t mine = r0 + lane < last ? r0 + lane : last;
    const int64_t start = (int64_t)ptr[mine];  // lanes past the last row hold the end
    const int64_t first = __shfl_sync(0xffffffffu, start, 0);
    const int64_t end = (int64_t)ptr[last];
    for (int64_t base = first; base < end; base += 32) {
      const int64_t k = base + lane;
      int j = 0;
#pragma unroll
      for (int step = 16; step > 0; step >>= 1) {
        const int64_t sc = __shfl_sync(0xffffffffu, start, j + step);
        if (sc <= k) j += step;
      }
      if (k < end) f(r0 + j, k);
    }
  }
}

// Sorts keys[ptr[i] .. ptr[i+1]) of every segment i < segs by their low 32
// bits (stable is irrelevant: keys within a segment share their high word).
// ptr is int32 (ptr32) or int64 (ptr64, when ptr32 is null); max_len bounds
// the segment lengths and must be <= kSegSortMax.
// distinct_range > 0 promises that every low word is < distinct_range and
// that the caller needs only each segment's sorted distinct values: segments
// of more than 256 keys then hold their distinct values ascending followed by
// copies of the largest (still sorted; only the multiplicities differ), when
// a bitmap of distinct_range bits fits kSegBitmapBytes of shared memory.
constexpr int32_t kSegSortMax = 8192;
constexpr size_t kSegBitmapBytes = 160 * 1024;
int segmented_sort_low32(int32_t segs, const int32_t* ptr32, const int64_t* ptr64,
                         int32_t max_len, int64_t total_keys, uint64_t* keys, cudaStream_t s,
                         uint32_t distinct_range = 0);

int fill_i32(int32_t* p, int32_t value, int64_t n, cudaStream_t s);

// CSC (transpose) of a CSR with ascending rows: col_ptr[n_cols+1] and
// col_rows[nnz] with ascending entries per column.
int transpose_csr(int32_t n_rows, int32_t n_cols, int64_t nnz, const int32_t* row_ptr,
                  const int32_t* cols, int32_t* col_ptr, int32_t* col_rows, cudaStream_t s);

// ---------------------------------------------------------------------------
// The hierarchy
// ---------------------------------------------------------------------------

// Work plan of one half-sweep (one side of the star expansion).
// Rows are put in classes by length: A (1..4 incidences), B (5..16),
// C (17..64), D (65..T); longer rows are cut into chunks of T consecutive
// incidences whose partial sums a second kernel reduces in chunk order.
// `items` holds one descriptor per work item {row, first incidence, length,
// partial slot or -1}: the A rows, then B, C, D, then every chunk. Split
// rows are listed in `long_desc` {row, first chunk, chunk count, 0}: those
// with at most kMidChunks chunks first, then the rest. Rows of length 0 are
// in zero_rows.
constexpr int32_t kSplitT = 128;
constexpr int32_t kMidChunks = 32;

// Class boundaries of a plan (lengths: A <= a_max < B <= b_max < C <= c_max
// < D <= T). The single-graph path uses the defaults; the batched path takes
// them from its autotuner.
struct PlanShape {
  int32_t a_max = 4;
  int32_t b_max = 16;
  int32_t c_max = 64;
};

struct SplitPlan {
  int32_t T = kSplitT;
  int32_t n_a = 0, n_b = 0, n_c = 0, n_d = 0;  // rows per class
  int32_t n_chunks = 0;                        // chunk items (after the D rows)
  int32_t n_mid = 0, n_huge = 0;               // split rows by chunk count
  int32_t n_zero = 0;
  int4* items = nullptr;              // [n_a + n_b + n_c + n_d + n_chunks]
  int4* long_desc = nullptr;          // [n_mid + n_huge]
  int32_t* zero_rows = nullptr;       // [n_zero]
  // the neighbours of the class-A rows (at most 4; unused slots 0), one
  // int4 per class-A item in item order, or null (see build_split_plan)
  int4* a_members = nullptr;          // [n_a]
  // the same for the class-B rows (at most 16 neighbours, 16 slots each)
  int32_t* b_members = nullptr;       // [n_b * 16]
};

struct Level {
  int32_t n = 0, m = 0;
  int64_t nnz = 0;
  int32_t* e_ptr = nullptr;      // [m+1]
  int32_t* e_nodes = nullptr;    // [nnz]
  int32_t* v_ptr = nullptr;      // [n+1]
  int32_t* v_edges = nullptr;    // [nnz]
  float* w = nullptr;            // [m]
  float* v_w = nullptr;          // [nnz] w of each CSC entry
  float* deg_v = nullptr;        // [n] sum_{e ∋ v} w_e
  float* inv_deg_v = nullptr;    // [n] 1/deg_v (0 if no hyperedge)
  float* inv_size_e = nullptr;   // [m] 1/|e|
  int32_t* orig_e = nullptr;     // [m] level-0 ID
  int32_t* rep_v = nullptr;      // [n] -> level+1 (null on the coarsest)
  int32_t* rep_e = nullptr;      // [m] -> level+1 or -1-c
  float* feat = nullptr;         // [n x feat_k] node features (cosine policy), or null
  int32_t feat_k = 0;
  SplitPlan planE, planV;
  // adjoint (built on first use; freed with the level)
  bool adj_ready = false;
  float* v_invsize_w = nullptr;  // [nnz] CSC order: 1/|e| of each hyperedge
  int32_t* ch_ptr = nullptr;     // [n_{l+1}+1] children of each coarse node:
  int32_t* ch_idx = nullptr;     //   fine nodes v, then collapsed hyperedges n + e
  int64_t ch_total = 0;          // entries of ch_idx
  SplitPlan planC;
  std::vector<void*> owned;      // every device allocation of this level
  // panel plans of the two sides (0 hyperedge rows, 1 node rows) for the
  // row size they were chosen for (side_plan); kept apart from `owned` so
  // that they can be rebuilt for another row size
  SplitPlan panel_plan[2];
  int32_t panel_P[2] = {1, 1};
  size_t panel_rb[2] = {0, 0};
  std::vector<void*> panel_owned[2];
};

}  // namespace hnv

struct hnv_graph {
  int device = 0;
  cudaStream_t stream = nullptr;
  std::vector<hnv::Level> levels;
  int32_t* d_err = nullptr;      // device error word
  int32_t* h_buf = nullptr;      // pinned host scratch (64 ints)
  int32_t* d_buf = nullptr;      // device scratch (64 ints)
  float* partials = nullptr;     // split-row partial sums
  size_t partials_bytes = 0;
  float* jacobi_tmp = nullptr;   // Jacobi: next hyperedge rows
  size_t jacobi_bytes = 0;
  uint64_t generation = 0;       // bumped whenever the hierarchy is rebuilt
  // side streams on which a half-sweep's row classes run concurrently
  // (forked from and joined back into the caller's stream)
  cudaStream_t aux[2] = {nullptr, nullptr};
  cudaEvent_t fork_ev = nullptr;
  cudaEvent_t join_ev[2] = {nullptr, nullptr};
};

namespace hnv {

// incidence.cu: level-0 construction, derived arrays and split plans.
int build_level0(hnv_graph* g, int32_t n, int32_t m, const int64_t* d_edge_ptr,
                 const int32_t* d_edge_nodes, const float* d_w, Level* out);
int finish_level(hnv_graph* g, Level* lv);   // derived arrays + plans
// Weight-dependent arrays of a level (v_w, deg_v, inv_deg_v) from lv->w.
int level_weight_arrays(Level* lv, cudaStream_t s);
// Split-row work plan of a CSR with `rows` rows; its device allocations are
// appended to `owned` (freed by whoever owns that list).
// With idx (the CSR's neighbour lists) and a_max <= 4 (b_max <= 16) the
// plan also packs the class-A (class-B) rows' neighbours next to their items
// (a_members, b_members), so that a gather reads a short row's descriptor
// and neighbours in one step.
int build_split_plan(hnv_graph* g, std::vector<void*>* owned, const int32_t* ptr, int32_t rows,
                     SplitPlan* plan, cudaStream_t s, const PlanShape& shape = PlanShape(),
                     const int32_t* idx = nullptr);
// Panel plan: the rows of `base` no longer than its class C bound keep their
// classes and items; the longer rows (listed ascending neighbour IDs in
// [0, cols)) are cut where their neighbours cross a panel boundary (P equal
// ranges of IDs) and into chunks of at most T incidences, and their items
// are listed panel by panel after the short classes, so that the launch
// over them works through the neighbour table one panel at a time (a
// panel's rows are read from DRAM about once and then hit L2). A long row
// left in one piece is a row item (n_d counts them); the pieces of a cut
// row are reduced in order (panel, then position) by the split-row
// reduction. P is chosen from table_bytes (the neighbour table's size) and
// the long rows' lengths; *panels = 1 means no panel plan (plan untouched).
int build_panel_plan(hnv_graph* g, std::vector<void*>* owned, const SplitPlan& base,
                     const int32_t* ptr, const int32_t* idx, int32_t cols, int64_t table_bytes,
                     SplitPlan* plan, int* panels, cudaStream_t s);
// The plan of one side of a level (0 hyperedge rows, 1 node rows) for
// neighbour rows of row_bytes: its panel plan (built on first use) or the
// regular one. HNV_PANELS=<k> forces k panels wherever there are long rows.
int side_plan(hnv_graph* g, Level* lv, int side, size_t row_bytes, const SplitPlan** plan,
              cudaStream_t s);
void free_level(Level* lv, cudaStream_t s);
int level_alloc(Level* lv, void** p, size_t bytes, cudaStream_t s);

// coarsen.cu: one step of Algorithm 1.
int coarsen_step(hnv_graph* g, int level, const hnv_coarsen_params* p, const uint64_t* d_explicit,
                 Level* fine, Level* coarse);

// refine.cu
// dtype: HNV_F32 or HNV_BF16 row storage (sums in float32 either way).
int refine_level(hnv_graph* g, int level, void* z_v, void* z_e, int dtype, int d, float omega,
                 int sweeps, int mode, cudaStream_t s);
int project_level(const hnv_graph* g, int fine_level, const void* zc_v, const void* zc_e,
                  void* zf_v, void* zf_e, int dtype, int d, cudaStream_t s);
// Sweeps until the largest change of any coordinate in a sweep is <= eps, or
// max_sweeps (synchronises after every sweep to read that change).
int refine_level_until(hnv_graph* g, int level, void* z_v, void* z_e, int dtype, int d,
                       float omega, int max_sweeps, float eps, int mode, int32_t* sweeps_done,
                       float* last_delta, cudaStream_t s);
// adjoint.cu: weights from a level-0 weight vector (device) to every level,
// and the reverse mode of the two-phase float32 V-cycle.
int set_weights_impl(hnv_graph* g, const float* d_w0, cudaStream_t s);
int vcycle_backward_impl(hnv_graph* g, const float* ckpt, const float* g_v0, const float* g_e0,
                         float* grad_w0, float* grad_zc, int d, float omega, int sweeps,
                         cudaStream_t s);

// tma_refine.cu: TMA-gather half-sweep for d in {32, 64, 128, 256}.
bool tma_supported(int d);
// One bounded mbarrier wait that nothing completes; sets ERRBIT_TIMEOUT in
// *err once it gives up after limit_ns.
int wait_selftest(int32_t* err, uint64_t limit_ns, cudaStream_t s);
int tma_half_sweep(const SplitPlan& plan, const int32_t* idx, const float* inc_w,
                   const float* inv_norm, const float* src, int64_t src_rows, const float* self_in,
                   float* out, int64_t self_rows, int d, float omega, float* partials,
                   int32_t* err, cudaStream_t s);

// General float32 row gather over a plan (used by the adjoint):
// out[r] = keep * self[r] + scale * norm[r] * sum_k wgt[k] * src[idx[k]];
// norm / wgt may be null (1); with keep == 0 self is not read. With conc, a
// graph with side streams, the plan's row classes run concurrently on them.
int gather_rows_f32(const SplitPlan& plan, const int32_t* idx, const float* wgt,
                    const float* norm, const float* src, const float* self_in, float* out, int d,
                    float keep, float scale, float* partials, cudaStream_t s,
                    const hnv_graph* conc = nullptr);

// Two-phase sweeps whose split-row partial sums go to caller-provided
// scratch (at least max(planE.n_chunks, planV.n_chunks) * d floats); no
// allocation and no timing events.
int refine_two_phase_with_partials(const hnv_graph* g, int level, float* z_v, float* z_e, int d,
                                   float omega, int sweeps, float* partials, cudaStream_t s);

// Reads the device error word (synchronising s) and clears it.
int read_and_clear_err(hnv_graph* g, cudaStream_t s, int32_t* bits);
// Copies `count` device ints into the graph's pinned buffer and synchronises.
int read_ints(hnv_graph* g, const int32_t* d_src, int count, int32_t* host_out, cudaStream_t s);

}  // namespace hnv
