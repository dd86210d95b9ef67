/*
 * hnv.h -- C ABI of the GB300 HyperNetVec V-cycle library (libhnv.so).
 *
 * The library computes the multilevel hypergraph embedding of HyperNetVec
 * (Maleki, Saless, Wall, Pingali, "HyperNetVec: Fast and Scalable
 * Hierarchical Embedding for Hypergraphs"): coarsening (Algorithm 1,
 * Section 3.1), projection and refinement (Algorithm 2, Section 3.3) over the
 * star expansion of the hypergraph (Section 1.1), run as a V-cycle from the
 * coarsest level back to the original hypergraph (Section 3, Fig. 1).
 *
 * Conventions
 *  - Every call returns an int: HNV_OK (0) or a negative HNV_ERR_* code.
 *    Nothing throws across the ABI. hnv_error_string() names a code and
 *    hnv_last_error_detail() gives a one-line message for the calling
 *    thread's last failure.
 *  - Streams are cudaStream_t values passed as hnv_stream_t (ABI-identical;
 *    NULL = the legacy default stream). Calls are asynchronous on that stream
 *    unless stated otherwise.
 *  - Embedding buffers are caller-owned device memory (e.g. torch tensors):
 *    row-major [rows x d], contiguous, 16-byte aligned, row stride d
 *    elements. HNV_F32 needs d % 4 == 0; HNV_BF16 needs d % 8 == 0;
 *    4 <= d <= 1024.
 *  - The hierarchy (all levels' incidence arrays and maps) is owned by an
 *    opaque hnv_graph and released by hnv_graph_free(). Its device memory
 *    is allocated stream-ordered from a memory pool of the library's own
 *    (one per device, keeping freed memory for reuse; see
 *    hnv_release_cached_memory) unless an allocator is installed with
 *    hnv_set_allocator().
 *  - IDs are int32: n, m < 2^31 and every level's incidence count
 *    nnz < 2^31 (HNV_ERR_TOO_LARGE otherwise).
 *  - One graph (or one batch) holds scratch that its calls share (split-row
 *    partials, a small device word buffer, two side streams on which a
 *    half-sweep's row classes run, forked from and joined back into the
 *    caller's stream). Calls on the same graph or batch must therefore not
 *    run concurrently from several host threads, or on streams whose work
 *    overlaps; different graphs are independent.
 */
#ifndef HNV_H_
#define HNV_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ABI-identical to cudaStream_t. */
typedef struct CUstream_st* hnv_stream_t;

/* Error codes. */
enum {
  HNV_OK = 0,
  HNV_ERR_INVALID_ARG = -1,   /* bad pointer, size, weight, enum or layout */
  HNV_ERR_OUT_OF_RANGE = -2,  /* a node ID >= n in the input, or a level index */
  HNV_ERR_TOO_LARGE = -3,     /* a count would not fit the int32 index space */
  HNV_ERR_OOM = -4,           /* device allocation failed */
  HNV_ERR_CUDA = -5,          /* a CUDA runtime call or kernel launch failed */
  HNV_ERR_TIMEOUT = -6,       /* a bounded device wait gave up */
  HNV_ERR_UNSUPPORTED_D = -7, /* embedding width not supported for the dtype */
  HNV_ERR_STATE = -8          /* call made in the wrong state (e.g. no hierarchy) */
};

typedef enum { HNV_F32 = 0, HNV_BF16 = 1 } hnv_dtype;

/* Update order of one refinement sweep (Algorithm 2, Section 3.3).
 * TWO_PHASE: every hyperedge from the current node embeddings, then every
 *   node from the new hyperedge embeddings (the text's "hyperedges are
 *   updated using the nodes, and nodes using the hyperedges").
 * JACOBI: both sides from the previous iterate (Algorithm 2 as printed). */
typedef enum { HNV_SWEEP_TWO_PHASE = 0, HNV_SWEEP_JACOBI = 1 } hnv_sweep;

/* How a node picks its hyperedge during coarsening (Section 3.1; the paper
 * uses "weights or degrees of a hyperedge" when there are no node features
 * and breaks ties at random). Every policy minimises a 64-bit priority
 * prio_l(e) over the node's hyperedges, ties going to the smaller ID:
 *   HASH        prio = mix64(e ^ mix64(seed + l * 0x9E3779B97F4A7C15)),
 *               mix64 = the SplitMix64 finaliser (default);
 *   LOW_DEGREE  prio = (min(|e|, 2^24-1) << 40) | (hash >> 24);
 *   HIGH_WEIGHT prio = ((2^32-1 - float_bits(w_e)) << 32) | (hash >> 32);
 *   EXPLICIT    prio = explicit_prio[l * m0 + orig(e)], where orig(e) is the
 *               level-0 ID of hyperedge e (test policy). */
typedef enum {
  HNV_ASSIGN_HASH = 0,
  HNV_ASSIGN_LOW_DEGREE = 1,
  HNV_ASSIGN_HIGH_WEIGHT = 2,
  HNV_ASSIGN_EXPLICIT = 3,
  /* Feature rule of Section 3.1 (nodes with features): f(e) = mean of its
   * members' features, c(v) = argmax_{e in N(v)} cos(f(e), f(v)), ties to
   * the smallest (hash priority, e) as under HNV_ASSIGN_HASH; a zero norm
   * gives score 0. The cosines are float32 with every operation rounded
   * separately (no fused multiply-add), sums in a fixed order: products
   * and squares added in dimension order, members in ascending node order.
   * Merged nodes take the mean of their nodes' features (ascending node
   * order), which the next level uses. Needs hnv_set_node_features. */
  HNV_ASSIGN_COSINE = 4
} hnv_assign;

typedef struct {
  int32_t policy;                 /* hnv_assign */
  int32_t min_nodes;              /* coarsen while n_l > min_nodes ...        */
  int32_t max_levels;             /* ... and l < max_levels and m_l > 0        */
  int32_t reserved;
  uint64_t seed;                  /* hash seed                                 */
  const uint64_t* explicit_prio;  /* EXPLICIT only: HOST array, max_levels*m0  */
} hnv_coarsen_params;

typedef struct hnv_graph hnv_graph;

/* ---------------------------------------------------------------------------
 * hnv_build_incidence -- level 0 of the hierarchy.
 * The hypergraph H = (V, E, w) (Section 1.1) as hyperedge member lists:
 * members of hyperedge e are edge_nodes[edge_ptr[e] .. edge_ptr[e+1]).
 * Builds the star-expansion incidence CSR (hyperedge -> nodes) and CSC
 * (node -> hyperedges) with ascending, duplicate-free rows, the weighted
 * node degrees sum_{e ∋ v} w_e (float32, summed in a fixed order) and 1/|e|.
 *   n_nodes, n_edges   : |V| >= 1, |E| >= 0
 *   edge_ptr [m+1]     : int64, edge_ptr[0] = 0, non-decreasing; every
 *                        hyperedge non-empty (the paper's hyperedges are
 *                        non-empty sets) -> else HNV_ERR_INVALID_ARG
 *   edge_nodes [nnz]   : int32 node IDs in [0, n); repeats are removed;
 *                        an ID outside -> HNV_ERR_OUT_OF_RANGE
 *   edge_w [m] or NULL : float32 weights, finite and > 0 (NULL = all 1)
 *   inputs_on_device   : 1 = the three arrays are device pointers;
 *                        0 = host pointers (copied by the call)
 * Synchronises the stream (sizes are read back). On success *out owns the
 * hierarchy (one level); on failure *out is NULL.
 * ------------------------------------------------------------------------- */
int hnv_build_incidence(int32_t n_nodes, int32_t n_edges, const int64_t* edge_ptr,
                        const int32_t* edge_nodes, const float* edge_w,
                        int inputs_on_device, hnv_stream_t stream, hnv_graph** out);

/* ---------------------------------------------------------------------------
 * hnv_coarsen -- Algorithm 1 (Section 3.1), level by level, on the graph's
 * stream. Per level l: every node v picks c(v) = argmin_{e in N(v)}
 * (prio_l(e), e); nodes with equal c(v) merge into one coarse node, a node
 * in no hyperedge stays alone; coarse IDs are the ranks of c(v) (or m_l + v
 * for a lone node). A hyperedge survives iff its members map to >= 2
 * distinct coarse nodes; survivors keep their order and weight and get the
 * sorted distinct images of their members. rep_v[l][v] is v's coarse node;
 * rep_e[l][e] is e's coarse hyperedge, or -1 - c when e collapsed into
 * coarse node c. Stops when n_l <= min_nodes, l == max_levels or m_l == 0;
 * a step that merges nothing is discarded and ends the loop.
 * Replaces any previous hierarchy above level 0. *n_levels (out) counts
 * levels including level 0. Synchronises the stream once per level.
 * ------------------------------------------------------------------------- */
int hnv_coarsen(hnv_graph* g, const hnv_coarsen_params* p, int32_t* n_levels);

/* Number of levels currently held (>= 1). */
int hnv_num_levels(const hnv_graph* g, int32_t* n_levels);

/* Sizes of one level. */
int hnv_level_info(const hnv_graph* g, int level, int32_t* n, int32_t* m, int64_t* nnz);

/* Device pointers of one level's arrays (owned by g, valid until the
 * hierarchy is rebuilt or freed). Any out pointer may be NULL. rep_v/rep_e
 * are NULL on the coarsest level. */
int hnv_get_level_arrays(const hnv_graph* g, int level, const int32_t** e_ptr,
                         const int32_t** e_nodes, const int32_t** v_ptr,
                         const int32_t** v_edges, const float** w,
                         const int32_t** rep_v, const int32_t** rep_e);

/* Which array hnv_copy_level_array() copies, and its element count. */
typedef enum {
  HNV_ARR_E_PTR = 0,    /* int32 [m+1]  */
  HNV_ARR_E_NODES = 1,  /* int32 [nnz]  */
  HNV_ARR_V_PTR = 2,    /* int32 [n+1]  */
  HNV_ARR_V_EDGES = 3,  /* int32 [nnz]  */
  HNV_ARR_W = 4,        /* float [m]    */
  HNV_ARR_REP_V = 5,    /* int32 [n]    (not on the coarsest level) */
  HNV_ARR_REP_E = 6,    /* int32 [m]    (not on the coarsest level) */
  HNV_ARR_DEG_V = 7     /* float [n]    weighted degree sum_{e ∋ v} w_e */
} hnv_array;

/* Copies one array of a level into dst (device pointer if dst_on_device,
 * else host) and synchronises the stream. capacity_bytes guards dst. */
int hnv_copy_level_array(const hnv_graph* g, int level, int which, void* dst,
                         size_t capacity_bytes, int dst_on_device, hnv_stream_t stream);

/* ---------------------------------------------------------------------------
 * Node features for the feature rule (HNV_ASSIGN_COSINE, Section 3.1: the
 * node feature matrix X of Algorithm 1's input and its coarse version X').
 *
 * hnv_set_node_features: copies X [n_0 x k] (row-major float32, host or
 * device per x_on_device) into the graph as level 0's features, replacing
 * any earlier ones. Every value must be finite with |x| <= 1e15 (so no sum
 * of squares can overflow): otherwise HNV_ERR_INVALID_ARG and nothing
 * changes. 1 <= k <= 4096. Synchronises the stream. A later hnv_coarsen
 * with HNV_ASSIGN_COSINE computes every coarse level's features.
 *
 * hnv_copy_level_features: copies level `level`'s features [n_l x k] to
 * dst (host or device); HNV_ERR_STATE if that level has none.
 * hnv_level_feature_dim: k of that level's features, 0 if none.
 * ------------------------------------------------------------------------- */
int hnv_set_node_features(hnv_graph* g, const float* x, int32_t k, int x_on_device,
                          hnv_stream_t stream);
int hnv_copy_level_features(const hnv_graph* g, int level, float* dst, size_t capacity_bytes,
                            int dst_on_device, hnv_stream_t stream);
int hnv_level_feature_dim(const hnv_graph* g, int level, int32_t* k);

/* ---------------------------------------------------------------------------
 * hnv_project -- initial embedding of level fine_level from level
 * fine_level + 1 (Section 3.3: a coarse node's embedding goes to every node
 * it merged). zf_v[v] = zc_v[rep_v[v]]; zf_e[e] = zc_e[rep_e[e]] if e
 * survived, else zc_v[c] for the coarse node c it collapsed into (the mean
 * of its projected members). Bitwise row copies.
 *   zc_v [n_{l+1} x d], zc_e [m_{l+1} x d] : device, read
 *   zf_v [n_l x d],     zf_e [m_l x d]     : device, written
 * ------------------------------------------------------------------------- */
int hnv_project(const hnv_graph* g, int fine_level, const void* zc_v, const void* zc_e,
                void* zf_v, void* zf_e, hnv_dtype dt, int d, hnv_stream_t stream);

/* ---------------------------------------------------------------------------
 * hnv_refine -- Algorithm 2 (Section 3.3) on one level, in place:
 * `sweeps` iterations of
 *   z~_e = (1/|e|) sum_{v in e} z_v,
 *   z~_v = sum_{e ∋ v} w_e z_e / sum_{e ∋ v} w_e,
 *   z <- (1 - omega) z + omega z~,
 * in the given update order; rows with no neighbours are left unchanged.
 * Sums are float32 in a fixed order (results are deterministic). Where one
 * side's neighbour table (rows x d x element size) is far larger than L2,
 * that side's long rows are summed in pieces, one per range of neighbour
 * IDs (panels), and the pieces added in order: the first call for a new
 * row size builds that plan (allocating; HNV_PANELS=<k> in the environment
 * forces k panels).
 *   z_v [n_l x d], z_e [m_l x d] : device, read and written
 *   omega in [0, 1]; sweeps >= 0
 * ------------------------------------------------------------------------- */
int hnv_refine(hnv_graph* g, int level, void* z_v, void* z_e, hnv_dtype dt, int d,
               float omega, int sweeps, hnv_sweep mode, hnv_stream_t stream);

/* ---------------------------------------------------------------------------
 * hnv_refine_until -- hnv_refine with the stopping rule the experiments of
 * Section 4 name as the alternative to a fixed iteration count: stop once
 * two consecutive iterates differ by at most eps. The difference of a sweep
 * is the largest |change| of any coordinate of any node or hyperedge row
 * (as stored). Runs at most max_sweeps sweeps; eps < 0 never stops early.
 *   sweeps_done [out] : sweeps run; last_delta [out] : the last difference
 * Synchronises the stream after every sweep (to read the difference) and
 * allocates two row buffers of the level for the previous iterate.
 * ------------------------------------------------------------------------- */
int hnv_refine_until(hnv_graph* g, int level, void* z_v, void* z_e, hnv_dtype dt, int d,
                     float omega, int max_sweeps, float eps, hnv_sweep mode,
                     int32_t* sweeps_done, float* last_delta, hnv_stream_t stream);

/* ---------------------------------------------------------------------------
 * hnv_vcycle -- the refinement half of the V-cycle (Section 3, Fig. 1):
 * refine the coarsest level L from z_coarsest, then for l = L-1 .. 0
 * project onto level l and refine it; write level 0's result.
 *   z_coarsest [(n_L + m_L) x d] : the coarsest level's initial embedding,
 *                                  node rows first, then hyperedge rows
 *   z_v_out [n_0 x d], z_e_out [m_0 x d]
 *   buffers_on_device : 1 = the three buffers are device pointers
 *                       (asynchronous on the stream);
 *                       0 = host pointers (copied in and out by the call,
 *                       which synchronises the stream before returning)
 * The per-level working buffers are allocated by the call.
 * ------------------------------------------------------------------------- */
int hnv_vcycle(hnv_graph* g, const void* z_coarsest, void* z_v_out, void* z_e_out,
               hnv_dtype dt, int d, float omega, int sweeps_per_level, hnv_sweep mode,
               int buffers_on_device, hnv_stream_t stream);

/* ---------------------------------------------------------------------------
 * hnv_refine_noalloc -- hnv_refine (HNV_SWEEP_TWO_PHASE, HNV_F32) for callers
 * that must not allocate device memory during the call. This is a library
 * service with no counterpart in the paper.
 * Some programs reserve their whole device-memory budget up front (a serving
 * process with a fixed pool, a deployment under a hard memory cap) and treat
 * any later cudaMalloc as an error: it can fail under memory pressure and may
 * stall the device while it synchronises. hnv_refine allocates its split-row
 * scratch on first use; this call uses a fixed device array compiled into the
 * library instead (HNV_NOALLOC_SCRATCH_BYTES, held by every GPU that loads
 * the library until the process exits) and calls no allocator at all.
 *   Arguments and results are those of hnv_refine with mode TWO_PHASE; the
 *   graph (built earlier) and the embeddings stay caller-provided.
 *   Returns HNV_ERR_TOO_LARGE when the level needs more scratch than the
 *   array holds: max(chunks of either half-sweep) * d * 4 bytes, where a row
 *   with more than 128 incidences contributes ceil(len / 128) chunks.
 *   It always uses the regular row plan (building a panel plan would
 *   allocate): on a level where hnv_refine cuts rows into panels the two
 *   agree to float32 rounding, elsewhere bit for bit.
 *   The first call on a device looks up the array's device address (once per
 *   device, under a lock); make that first call outside any stream capture.
 *   The address stays cached for the life of the process: after a
 *   cudaDeviceReset of that device it is stale, so do not call this entry
 *   point on a device that has been reset. All calls share the one array and it keeps the
 *   last call's contents; calls whose kernels overlap on the GPU (other
 *   streams, other host threads) race on it, so serialise them.
 * ------------------------------------------------------------------------- */
#define HNV_NOALLOC_SCRATCH_BYTES (16u << 20)
int hnv_refine_noalloc(hnv_graph* g, int level, void* z_v, void* z_e, hnv_dtype dt, int d,
                       float omega, int sweeps, hnv_stream_t stream);

/* ---------------------------------------------------------------------------
 * Differentiation (reverse mode of the two-phase float32 V-cycle)
 *
 * The V-cycle maps (w0, Z^L) -> (Z_V^0, Z_E^0), where w0 are the level-0
 * hyperedge weights (a coarse hyperedge keeps the weight of the level-0
 * hyperedge it represents) and Z^L the coarsest rows. The weights enter the
 * node half-sweeps of Algorithm 2 through the weighted neighbour mean of
 * Section 3.3. The hierarchy itself does not depend on the weights under
 * HNV_ASSIGN_HASH / LOW_DEGREE / EXPLICIT (it does under HIGH_WEIGHT).
 * ------------------------------------------------------------------------- */

/* Replaces the level-0 weights (float32 [m0], finite and > 0; host or device)
 * and every level's weight-dependent arrays. Synchronises the stream. */
int hnv_set_weights(hnv_graph* g, const float* w0, int on_device, hnv_stream_t stream);

/* Size (in floats) of the checkpoint buffer hnv_vcycle_save writes for width
 * d: sum over levels of (n_l + m_l) * d. */
int hnv_checkpoint_floats(const hnv_graph* g, int d, int64_t* floats);

/* hnv_vcycle (two-phase, float32, device buffers) that also saves every
 * level's starting rows (after projection; the coarsest level's input) into
 * `checkpoints` (device, hnv_checkpoint_floats floats) for the backward pass. */
int hnv_vcycle_save(hnv_graph* g, const float* z_coarsest, float* z_v_out, float* z_e_out, int d,
                    float omega, int sweeps_per_level, float* checkpoints, hnv_stream_t stream);

/* Reverse mode of hnv_vcycle_save. Given dL/dZ_V^0 (g_v0 [n0 x d]) and
 * dL/dZ_E^0 (g_e0 [m0 x d]; either may be NULL = zero), writes dL/dw0
 * (grad_w0 [m0]) and dL/dZ^L (grad_z_coarsest [(n_L + m_L) x d]). Every
 * level's sweeps are recomputed from its checkpoint, then reversed:
 *   node half:      a_v = G_V/D_v, A_e = sum_{v in e} a_v,
 *                   dw_e += omega (<A_e, z_e> - sum_{v in e} <a_v, z~_v>),
 *                   G_E += omega w_e A_e, G_V *= 1 - omega;
 *   hyperedge half: G_V += omega sum_{e ∋ v} G_E[e]/|e|, G_E *= 1 - omega;
 * projection reverses to a segmented sum over each coarse row's copies. The
 * replay keeps z~_v = s_v/D_v of every sweep as the gather computes it, so no
 * step divides by omega. Working memory, from the library's pool: sweeps x
 * max_l (n_l + m_l) x d floats of replayed iterates, plus
 * 2 max_l (n_l + m_l) + 2 max_l n_l + max_l m_l rows of d floats. The weights, omega, d and sweeps must be those of the forward
 * call. All device buffers; asynchronous on the stream; deterministic. */
int hnv_vcycle_backward(hnv_graph* g, const float* checkpoints, const float* g_v0,
                        const float* g_e0, float* grad_w0, float* grad_z_coarsest, int d,
                        float omega, int sweeps_per_level, hnv_stream_t stream);

/* ---------------------------------------------------------------------------
 * Batched V-cycle: many independent hypergraphs refined together
 *
 * Each graph is built and coarsened as usual (its hierarchy does not change).
 * The batch lines the graphs up by level index: at step s (deepest level
 * first) every graph whose coarsest level is >= s projects onto its level s
 * (or starts from its input rows at its coarsest level) and runs the
 * two-phase sweeps of Algorithm 2 there. Per half-sweep, one launch per row
 * class (or one persistent launch) covers the rows of all graphs (a work
 * list with a graph index per item); the whole V-cycle can be captured once
 * into a CUDA graph and replayed. Results equal hnv_vcycle on each graph
 * (same per-row sums). The persistent launches use a small array of task
 * counters owned by the batch (one per half-sweep), cleared at the start of
 * every V-cycle; V-cycles of one batch must not overlap on the GPU.
 * ------------------------------------------------------------------------- */
typedef struct hnv_batch hnv_batch;

/* Half-sweep kernels of the batched V-cycle. PER_CLASS: one launch per row
 * class (rows of 1..a_max, a_max+1..b_max and longer rows with chunks), the
 * classes on concurrent streams. PERSISTENT: one launch per half-sweep over
 * every item of every class and graph; resident warps take fixed-size tasks
 * from a counter in device memory, the longest items first. Both are followed
 * by the split-row reduction and give the same bits. */
enum { HNV_BATCH_KERNEL_PER_CLASS = 0, HNV_BATCH_KERNEL_PERSISTENT = 1 };

/* Row-length classes, lanes per row and half-sweep kernel chosen by
 * hnv_batch_autotune. */
typedef struct {
  int32_t a_max, b_max, c_max;          /* class boundaries (incidences) */
  int32_t lanes_a, lanes_b, lanes_rest; /* lanes per row of the classes  */
  float best_ms;                        /* V-cycle, 1 sweep per level, ms (-1: cached) */
  int32_t from_cache;                   /* 1: taken from the tuning cache */
  int32_t kernel;                       /* HNV_BATCH_KERNEL_*              */
  float persistent_ms;                  /* the same with the persistent kernel (-1: cached) */
} hnv_batch_tuning;

/* A batch over `count` graphs (built and coarsened; all on one device). The
 * batch references the graphs (they must outlive it) and owns its own work
 * lists, buffers, streams and captured graph. Coarsening a graph again makes
 * the batch stale: its later calls return HNV_ERR_STATE.
 *   graphs [count] : host array of graph handles; count >= 1
 *   out            : receives the batch (NULL on failure)
 * Errors: HNV_ERR_INVALID_ARG (NULL, count < 1, graphs on different
 * devices), HNV_ERR_OOM, HNV_ERR_CUDA. Synchronises each graph's stream. */
int hnv_batch_create(hnv_graph* const* graphs, int32_t count, hnv_batch** out);

/* Row offsets of the batched buffers (each array count + 1 entries, host):
 * graph i's coarsest rows (its nodes, then its hyperedges) start at row
 * coarsest_rows[i] of z_coarsest; its level-0 node rows at node_rows[i] of
 * z_v_out; its level-0 hyperedge rows at edge_rows[i] of z_e_out. */
int hnv_batch_offsets(const hnv_batch* b, int64_t* coarsest_rows, int64_t* node_rows,
                      int64_t* edge_rows);

/* Times candidate row-class boundaries and lanes per row of the per-class
 * kernel, and the persistent kernel, on a whole V-cycle of the batch with one
 * sweep per level, and keeps the fastest (cached per dtype, d and the batch's
 * level-0 row-length histogram). Uses scratch rows of the batch's level-0
 * size while it runs. Synchronises. */
int hnv_batch_autotune(hnv_batch* b, hnv_dtype dt, int d, float omega, hnv_batch_tuning* chosen);

/* Selects the half-sweep kernel (HNV_BATCH_KERNEL_*) of later hnv_batch_vcycle
 * calls; a new batch starts with HNV_BATCH_KERNEL_PER_CLASS (measured faster
 * on the 256-graph batching workload), and hnv_batch_autotune sets the faster. Errors: HNV_ERR_INVALID_ARG (NULL batch,
 * unknown kernel). hnv_batch_get_kernel returns the current one (or
 * HNV_ERR_INVALID_ARG for NULL). */
int hnv_batch_set_kernel(hnv_batch* b, int kernel);
int hnv_batch_get_kernel(const hnv_batch* b);

/* The two-phase V-cycle of every graph of the batch (device buffers laid out
 * as hnv_batch_offsets says; d % 8 == 0). With use_cuda_graph the whole
 * cycle is captured once (per buffers, dtype, d, omega and sweeps) and
 * replayed on `stream`.
 *   z_coarsest [coarsest_rows[count] x d] : read
 *   z_v_out [node_rows[count] x d], z_e_out [edge_rows[count] x d] : written
 *   (device, 16-byte aligned, caller-owned; the batch keeps work lists built
 *   for these pointers until they change)
 * Errors: HNV_ERR_INVALID_ARG (NULL or misaligned buffer, omega outside
 * [0, 1], sweeps < 0), HNV_ERR_UNSUPPORTED_D, HNV_ERR_STATE (a graph was
 * coarsened again), HNV_ERR_OOM, HNV_ERR_CUDA. Device-side checks of the
 * work items report through hnv_sync_status of the graphs. Asynchronous on
 * `stream` after the first call for a set of buffers (which builds the work
 * lists and synchronises its own stream). */
int hnv_batch_vcycle(hnv_batch* b, const void* z_coarsest, void* z_v_out, void* z_e_out,
                     hnv_dtype dt, int d, float omega, int sweeps_per_level, int use_cuda_graph,
                     hnv_stream_t stream);

/* Releases the batch (its buffers, streams and captured graph; not the
 * graphs). Synchronises the batch's streams. NULL is a no-op. */
void hnv_batch_free(hnv_batch* b);

/* Synchronises `stream` and reports device-side failures of the graph's
 * asynchronous calls since the last check: HNV_ERR_TIMEOUT if a bounded
 * device wait of a refinement kernel gave up (its results are then invalid),
 * HNV_ERR_CUDA for a CUDA error, else HNV_OK. Clears the recorded failure. */
int hnv_sync_status(hnv_graph* g, hnv_stream_t stream);

/* Self-test of the device-side failure path (a library service; the paper
 * has no counterpart). Launches one bounded wait, the kind the TMA gather
 * kernels use, on an mbarrier that nothing completes (no memory copy is in
 * flight); after limit_us microseconds (1 .. 1000000) the wait gives up and
 * records a timeout for the graph, exactly as a refinement kernel would.
 * The next hnv_sync_status on that graph returns HNV_ERR_TIMEOUT (and
 * clears it); the context stays usable. Asynchronous on stream.
 * Errors: HNV_ERR_INVALID_ARG (NULL graph, limit out of range), HNV_ERR_CUDA. */
int hnv_selftest_wait_timeout(hnv_graph* g, uint32_t limit_us, hnv_stream_t stream);

/* Releases the hierarchy (stream-ordered on the graph's stream). NULL is a no-op. */
void hnv_graph_free(hnv_graph* g);

/* ---------------------------------------------------------------------------
 * Utilities
 * ------------------------------------------------------------------------- */
const char* hnv_error_string(int code);
/* One-line detail of the calling thread's last error ("" if none). */
const char* hnv_last_error_detail(void);

/* Replaces the device allocator (NULL, NULL restores the library's pool:
 * cudaMallocFromPoolAsync / cudaFreeAsync). alloc returns NULL on failure,
 * which the library reports as HNV_ERR_OOM. Not thread-safe with respect to
 * calls in flight. */
typedef void* (*hnv_alloc_fn)(size_t bytes, hnv_stream_t stream, void* ctx);
typedef void (*hnv_free_fn)(void* ptr, hnv_stream_t stream, void* ctx);
int hnv_set_allocator(hnv_alloc_fn alloc_fn, hnv_free_fn free_fn, void* ctx);

/* The library allocates from a stream-ordered memory pool of its own per
 * device whose freed memory stays mapped for the next call (a V-cycle step
 * at the 1M-node size allocates and frees about 1.5 GB; mapping it afresh on
 * every call costs time). This returns the pools' unused memory to the
 * system (memory still allocated stays). Errors: HNV_ERR_CUDA. */
int hnv_release_cached_memory(void);

/* Number of kernels this library has launched in the process so far. */
int64_t hnv_kernel_launch_count(void);

/* Per-phase device timing. When enabled, the library records CUDA events
 * around each phase's kernels on the launching stream. Phases: */
typedef enum {
  HNV_PHASE_BUILD = 0,
  HNV_PHASE_COARSEN = 1,
  HNV_PHASE_PROJECT = 2,
  HNV_PHASE_REFINE_E = 3,   /* hyperedge half-sweeps (gather node rows)   */
  HNV_PHASE_REFINE_V = 4,   /* node half-sweeps (gather hyperedge rows)   */
  /* hnv_vcycle_backward, per level: */
  HNV_PHASE_ADJOINT_REPLAY = 5,   /* the level's sweeps recomputed           */
  HNV_PHASE_ADJOINT_REVERSE = 6,  /* the sweeps reversed                     */
  HNV_PHASE_ADJOINT_PROJECT = 7,  /* weight gradients out, projection reversed */
  HNV_PHASE_COUNT = 8
} hnv_phase;
int hnv_timing_enable(int enable);
/* Clears the recorded events. */
int hnv_timing_reset(void);
/* Synchronises the recorded events and returns, for one phase, the summed
 * milliseconds, the number of recorded launches and the summed algorithmic
 * bytes (compulsory traffic: every input and output array touched once). */
int hnv_timing_read(int phase, double* total_ms, int64_t* launches, double* alg_bytes);

#ifdef __cplusplus
}
#endif
#endif /* HNV_H_ */
