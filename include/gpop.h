/*
 * gpop.h -- C ABI of the GB300 partition-centric scatter/gather engine.
 *
 * The engine follows GPOP (Lakhotia, Pati, Kannan, Prasanna): vertices are
 * split into index partitions of P consecutive IDs (Sec. 3.1.1); each
 * iteration scatters messages from every active partition p into bins
 * bin[p][q] (Sec. 3.1.2, Alg. 2), either source-centric (SC: only active
 * vertices, as (destination, value) pairs) or partition-centric (PC: one value
 * per PNG entry, destination lists laid out once at build, Alg. 3), with the
 * mode chosen per partition and iteration by the traffic model of Sec. 3.2
 * (Eq. (mode)); gather then drains bin[*][q] into q's vertex data without
 * locks or atomics on vertex data, and the filter step builds the next,
 * optionally continued, frontier (Sec. 4 user functions).
 *
 * Conventions for every entry point:
 *  - Vertex IDs are uint32 with num_vertices < 2^31; num_edges < 2^32.
 *  - Inputs are copied; the caller keeps ownership of everything it passes.
 *  - Outputs go to caller-allocated buffers of the stated length.
 *  - A pointer argument is device memory when the matching *_is_device flag is
 *    non-zero, host memory otherwise.  cuda_stream is a cudaStream_t (NULL =
 *    the legacy default stream); calls are synchronous with respect to it
 *    on return.
 *  - No call aborts or exits.  On failure a non-zero gpop_status is returned
 *    and gpop_last_error() describes it; outputs are then unspecified.
 *  - The library allocates device memory with cudaMalloc; all of it belongs
 *    to the gpop_graph handle and is released by gpop_graph_destroy.
 */
#ifndef GPOP_H
#define GPOP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GPOP_OK = 0,
    GPOP_ERR_INVALID_ARG = 1,    /* bad sizes, malformed CSR, unsupported option */
    GPOP_ERR_OOM = 2,            /* device or host allocation failed */
    GPOP_ERR_CUDA = 3,           /* a CUDA runtime call failed */
    GPOP_ERR_DEVICE_CHECK = 4,   /* a device-side consistency check failed */
    GPOP_ERR_TIMEOUT = 5,        /* a bounded device wait gave up */
    GPOP_ERR_NOT_CONVERGED = 6,  /* max_iters reached before tol_l1 (results valid) */
    GPOP_ERR_NO_SELECTOR = 7     /* learned mode requested but no trained selector */
} gpop_status;

/* Opaque graph handle; owns the partitioned layout and all device memory. */
typedef struct gpop_graph gpop_graph;

/*
 * Builds the partitioned layout from a CSR graph (pre-processing of Sec. 3.1:
 * index partitions, per-partition E^p and r^p, the PNG of Alg. 3 with its
 * destination-ID lists written once, and SC bin capacities).
 *   num_vertices   V, 1 <= V < 2^31
 *   num_edges      E, 0 <= E < 2^32
 *   row_ptr        V+1 offsets (uint64), row_ptr[0] = 0, non-decreasing, row_ptr[V] = E
 *   col            E destination IDs (< V); rows need not be sorted; self loops
 *                  and repeated edges are kept as parallel edges
 *   weights        E non-negative int32 edge weights (SSSP), or NULL
 *   partition_size P, a power of two in [32, 16384], or 0 for the default
 *                  (16384, clamped to V rounded up to a power of two); the
 *                  partition count k = ceil(V/P) must not exceed 65536
 *   mem_is_device  non-zero if row_ptr/col/weights are device pointers
 *   cuda_stream    stream for the build kernels
 *   out            receives the handle (unchanged on failure)
 * Errors: GPOP_ERR_INVALID_ARG for malformed input (checked on the device),
 * GPOP_ERR_OOM, GPOP_ERR_CUDA.
 */
gpop_status gpop_graph_build(uint32_t num_vertices, uint64_t num_edges, const uint64_t *row_ptr,
                             const uint32_t *col, const int32_t *weights, uint32_t partition_size,
                             int mem_is_device, void *cuda_stream, gpop_graph **out);

typedef struct {
    uint32_t num_vertices;
    uint32_t partition_size;      /* P */
    uint32_t num_partitions;      /* k */
    uint32_t weighted;            /* 1 if built with weights */
    uint64_t num_edges;           /* E */
    uint64_t num_bins;            /* non-empty bin[p][q] pairs */
    uint64_t num_png;             /* sum_p r^p E^p (PNG entries, unpadded) */
    uint64_t num_png_padded;      /* PNG slots including per-row padding to 8 */
    uint32_t num_gather_tasks;    /* static (column, destination range) tasks */
    uint32_t num_scatter_tasks;   /* static PC scatter chunks */
    uint32_t max_row_bins;        /* largest number of bins in one bin row */
    uint32_t reserved;
    uint64_t device_bytes;        /* device memory held by the handle */
    uint64_t num_pc_blocks;       /* staged message blocks of the PC gather */
    uint32_t num_pc_tasks;        /* PC gather tasks (column, block range) */
    uint32_t num_pc_partials;     /* partial result vectors of columns split over several tasks */
} gpop_graph_info;

/* Fills *info.  Errors: GPOP_ERR_INVALID_ARG on NULL arguments. */
gpop_status gpop_graph_get_info(const gpop_graph *g, gpop_graph_info *info);

/* Copies per-partition E^p (out-edges) and n_png^p = r^p E^p (Sec. 3.1.2) into
 * host arrays of k uint64 entries each (either may be NULL). */
gpop_status gpop_graph_partition_stats(const gpop_graph *g, uint64_t *edges, uint64_t *png);

/* Releases the handle and its device memory; NULL is ignored. */
void gpop_graph_destroy(gpop_graph *g);

typedef enum {
    GPOP_PAGERANK = 0,   /* Alg. 6: topological PageRank, all vertices always active */
    GPOP_BFS = 1,        /* Alg. 5: BFS levels and parents from a root */
    GPOP_CC = 2,         /* Sec. 5: min-label propagation (use a symmetrised graph) */
    GPOP_SSSP = 3,       /* Alg. 7: Bellman-Ford over non-negative integer weights */
    GPOP_PPR = 4,        /* seeded personalised PageRank, restart = 1 - damping */
    GPOP_NIBBLE = 5      /* Alg. 4: parallel Nibble from the seed `source` with threshold `epsilon`
                            (a vertex stays on the frontier while PR >= epsilon * outdeg; a sink never
                            stays on) */
} gpop_algo;

typedef enum {
    GPOP_MODE_ANALYTIC = 0,   /* Eq. (mode) per partition per iteration */
    GPOP_MODE_LEARNED = 1,    /* trained MLP selector, Eq. (mode) as fallback */
    GPOP_MODE_FORCE_SC = 2,   /* every scattered partition in SC mode */
    GPOP_MODE_FORCE_PC = 3,   /* every scattered partition in PC mode */
    GPOP_MODE_LOG_BOTH = 4    /* Eq. (mode) decides; both scatters run and are timed */
} gpop_mode_policy;

typedef struct {
    int32_t algo;              /* gpop_algo */
    uint32_t source;           /* BFS/SSSP root, PPR / Nibble seed (ignored by PageRank/CC) */
    double damping;            /* PageRank d (default 0.85); PPR continuation 1 - restart */
    uint32_t max_iters;        /* iteration cap (default 1000) */
    double tol_l1;             /* PageRank/PPR: stop once sum_v |x_{t+1}-x_t| < tol_l1; 0 = run max_iters */
    int32_t mode;              /* gpop_mode_policy */
    uint32_t bw_ratio_num;     /* BW_PC / BW_SC = num / den (Sec. 3.2 default 2/1) */
    uint32_t bw_ratio_den;
    int32_t msg_bf16;          /* PageRank / PPR only: non-zero sends messages through the bins as BF16
                                  (round to nearest even), gathered in FP32; other algorithms: must be 0 */
    int32_t profile_kernels;   /* non-zero: time every kernel launch with CUDA events (stats.kernel_*) */
    void *cuda_stream;         /* stream for all kernels of the run */
    uint8_t *trace_modes;      /* optional HOST buffer of max_iters * k bytes: per iteration and
                                  partition 0 = not scattered, 1 = SC, 2 = PC */
    uint64_t *trace_frontier;  /* optional HOST buffer of max_iters * 2: V_a and E_a entering each iteration */
    float *log_buffer;         /* optional HOST buffer for GPOP_MODE_LOG_BOTH timing records,
                                  log_capacity records of GPOP_LOG_RECORD_FLOATS floats */
    uint64_t log_capacity;
    double epsilon;            /* Nibble threshold (default 1e-9, Sec. 5's setting); >= 0, finite */
    int32_t resume;            /* non-zero: continue the state the graph holds (the last successful run of
                                  this algorithm on it, or gpop_state_import) instead of starting afresh:
                                  no initial frontier, iterations numbered on from the saved ones (BFS
                                  levels), max_iters counts this call's iterations, and the first plan
                                  tests the saved L1 change, so a run split at any iteration gives the
                                  same results as one uninterrupted run.  source is not used.  Not for
                                  gpop_run_msbfs.  GPOP_ERR_INVALID_ARG when no state of the algorithm
                                  is held. */
    uint32_t isg_waves;        /* CC and SSSP: interleaved scatter-gather (Sec. 3.3) with this many waves
                                  (0 or 1: bulk-synchronous).  Iteration i scatters only the active
                                  partitions p with p mod isg_waves == (i - 1) mod isg_waves; its gather
                                  updates every destination, and active vertices of the partitions that did
                                  not scatter stay active.  A partition thus scatters the values its vertices
                                  received from the waves before it in the same sweep, the paper's "gather
                                  the messages already received, then scatter" with the wave order in place
                                  of thread timing.  Results are the same fixed point; iteration counts (one
                                  wave each) change.  GPOP_ERR_INVALID_ARG for other algorithms. */
} gpop_run_opts;

/* Floats per LOG_BOTH record: 8 selector features, t_PC (us), t_SC (us),
 * chosen mode (2 PC / 1 SC), partition id, iteration. */
#define GPOP_LOG_RECORD_FLOATS 13

typedef struct {
    uint32_t iterations;          /* scatter/gather rounds executed */
    int32_t converged;            /* 1 if the frontier emptied or tol_l1 was met */
    double residual;              /* last L1 change (PageRank/PPR), else 0 */
    uint64_t edges_scattered;     /* sum over iterations of E_a (active out-edges) */
    uint64_t vertices_scattered;  /* sum over iterations of V_a */
    uint64_t pc_partition_steps;  /* partition-iterations scattered in PC mode */
    uint64_t sc_partition_steps;  /* partition-iterations scattered in SC mode */
    double model_bytes;           /* sum of Sec. 3.2 bytes of the chosen modes */
    double device_ms;             /* CUDA-event time of the iteration loop */
    uint64_t log_records;         /* LOG_BOTH records written */
    /* with opts.profile_kernels: per kernel kind (0 plan (+ learned selection), 1 PC scatter,
       2 SC scatter (with its per-segment active-edge counts), 3 task gather + filter, 4 PC gather, 5 merge of split columns' PC partials) the
       summed CUDA-event duration and the number of launches (a kind the plan gives nothing to do in
       an iteration is not launched) */
    double kernel_ms[6];
    uint64_t kernel_launches[6];
    uint64_t sc_vertices_scattered;  /* sum over iterations of V_a of the partitions scattered in SC mode */
    uint64_t sc_edges_scattered;     /* sum over iterations of E_a of the partitions scattered in SC mode */
    uint64_t gathered_vertices;      /* sum over iterations of the destinations the task gather visited
                                        (every vertex of each gather task whose column had messages or
                                        active vertices) */
} gpop_run_stats;

/* Fills opts with defaults: PageRank, d = 0.85, max_iters 1000, tol 0,
 * analytic mode, BW ratio 2/1, NULL stream and buffers. */
void gpop_run_opts_default(gpop_run_opts *opts);

/*
 * Runs one application on the graph (Alg. 2 iterations until the frontier is
 * empty, max_iters is reached, or for PageRank/PPR the L1 change drops below
 * tol_l1).
 *   out_values  V elements: float PageRank / PPR / Nibble values; uint32 BFS level,
 *               SSSP distance or CC label (0xFFFFFFFF = unreached)
 *   out_parent  BFS only: V uint32 parents (root's parent is the root,
 *               0xFFFFFFFF = unreached), or NULL
 *   out_is_device  non-zero if out_values/out_parent are device pointers
 *   stats       optional, filled on return
 * Errors: GPOP_ERR_INVALID_ARG (bad source, weights missing for SSSP, ...),
 * GPOP_ERR_NO_SELECTOR, GPOP_ERR_CUDA, GPOP_ERR_OOM.  Reaching max_iters is
 * not an error (stats->converged tells).
 */
gpop_status gpop_run(gpop_graph *g, const gpop_run_opts *opts, void *out_values, uint32_t *out_parent,
                     int out_is_device, gpop_run_stats *stats);

/*
 * Multi-source BFS: the levels of Alg. 5 from every source in one call, up to
 * 32 sources per pass through the engine.  A pass carries, per vertex, the set
 * of its sources that reached the vertex (bit j = sources[b + j]); a vertex's
 * message in SC and PC bins is the complement of the sources that reached it
 * in the previous iteration, combined with bitwise AND, so the NULL of an
 * inactive source (all ones) is the identity and every pass keeps the single
 * BFS's exact results.  Partition modes follow opts.mode as in gpop_run, from
 * the union frontier of the pass.
 *   sources      HOST array of num_sources vertex IDs (< V; repeats allowed)
 *   out_levels   num_sources x V uint32, row j = levels from sources[j]
 *                (0xFFFFFFFF = unreached), caller-owned; device memory if
 *                out_is_device, else host memory (staged through a 32 x V
 *                device buffer owned by the graph)
 *   opts         mode, bw ratio, max_iters (per pass), profile_kernels and
 *                cuda_stream are used; algo, source and damping are ignored;
 *                msg_bf16 and resume must be 0; trace buffers hold the last pass
 *   stats        optional: sums over the passes (iterations, device_ms,
 *                kernel times, ...), converged = every pass converged
 * No parents are produced.  Errors: GPOP_ERR_INVALID_ARG (NULL pointers with
 * num_sources > 0, a source >= V, msg_bf16), GPOP_ERR_NO_SELECTOR,
 * GPOP_ERR_OOM, GPOP_ERR_CUDA, GPOP_ERR_TIMEOUT.  num_sources = 0 returns
 * GPOP_OK without work.
 */
gpop_status gpop_run_msbfs(gpop_graph *g, const gpop_run_opts *opts, const uint32_t *sources, uint32_t num_sources,
                           uint32_t *out_levels, int out_is_device, gpop_run_stats *stats);

/*
 * Many graphs at once.  gpop_graph_build_union builds num_graphs graphs as one graph, their disjoint union
 * (graph i's vertices follow graph i-1's, its edges shifted with them), so that the partitions, bins and
 * gather tasks of Sec. 3.1 span graphs of uneven size and one traversal of the scatter / gather serves all
 * of them.  Arguments per graph, HOST arrays: num_vertices[i] (> 0), num_edges[i], row_ptrs[i] (V_i + 1
 * offsets starting at 0), cols[i] (E_i local destinations < V_i), weights NULL or weights[i] (E_i values,
 * for every graph with edges); partition_size as gpop_graph_build.  The union must have fewer than 2^31
 * vertices and 2^32 edges.  The caller keeps its arrays; the result is a gpop_graph like any other (any
 * application can run on the union), which also knows its graphs' first vertices:
 *   gpop_graph_union_offsets   writes num_graphs + 1 offsets (graph i = vertices [offsets[i], offsets[i+1])
 *                              of the union) into the caller's HOST array, or only *num_graphs when
 *                              offsets is NULL; *num_graphs = 0 for a graph not built as a union.
 *   gpop_run_bfs_union         the BFS levels (Alg. 5) of every graph from its own source: sources[i] is a
 *                              LOCAL vertex of graph i; out_levels (V of the union, caller-owned, device
 *                              memory if out_is_device) receives graph i's levels at offsets[i] ..
 *                              (0xFFFFFFFF = unreached).  Up to 32 graphs per traversal: one source each in
 *                              the multi-source BFS of gpop_run_msbfs, whose levels inside a graph are that
 *                              graph's BFS because no edge leaves it.  opts as gpop_run_msbfs.
 * Errors: GPOP_ERR_INVALID_ARG (a graph without vertices, a destination outside its graph, too large a
 * union, weights for some graphs only, a source outside its graph, a graph not built as a union),
 * GPOP_ERR_OOM, GPOP_ERR_CUDA, and those of gpop_graph_build and gpop_run_msbfs.
 */
gpop_status gpop_graph_build_union(uint32_t num_graphs, const uint32_t *num_vertices, const uint64_t *num_edges,
                                   const uint64_t *const *row_ptrs, const uint32_t *const *cols,
                                   const int32_t *const *weights, uint32_t partition_size, void *cuda_stream,
                                   gpop_graph **out);
gpop_status gpop_graph_union_offsets(const gpop_graph *g, uint32_t *offsets, uint32_t *num_graphs);
gpop_status gpop_run_bfs_union(gpop_graph *g, const gpop_run_opts *opts, const uint32_t *sources, uint32_t *out_levels,
                               int out_is_device, gpop_run_stats *stats);

/*
 * Batched seeded personalized PageRank: the PPR vector of every seed (restart 1 - damping, the iteration
 * of gpop_run's GPOP_PPR) in passes of up to 32 seeds, each pass one traversal of the partition-centric
 * scatter / gather in which a message carries one FP32 value per seed of the pass (Alg. 2 with Alg. 3's
 * PC layout; the single-seed application's scatter, gather and filter functions applied per seed).  Every
 * partition holding a vertex active for some seed of the pass (the union frontier) is scattered in PC mode.
 *   seeds        HOST array of num_seeds vertex IDs (< V; repeats allowed)
 *   out_values   num_seeds x V floats, row j = the PPR vector of seeds[j], caller-owned; device memory if
 *                out_is_device, else host memory
 *   opts         damping (restart alpha = 1 - damping), max_iters (per pass), tol_l1 (a pass stops once
 *                every one of its seeds' L1 change is below it; 0: run max_iters), cuda_stream,
 *                profile_kernels; msg_bf16 and resume must be 0; mode, bw ratio and trace buffers are
 *                not used
 *   stats        iterations summed over passes, converged = every pass met tol_l1, residual = the largest
 *                L1 change of the last iteration of the last pass, device_ms, edges_scattered (out-edges
 *                of the partitions scattered, summed over iterations and passes)
 * The combined message of 32 seeds per destination is kept in shared memory, so the graph's partition
 * size must be at most 1024.  All working memory (about 3 x 128 B per vertex and 128 B per PNG slot) is
 * allocated by the call and released before it returns.  Sums are taken in a fixed order: results do
 * not change from run to run.
 * Errors: GPOP_ERR_INVALID_ARG (seed out of range, partition size above 1024, damping outside (0, 1),
 * msg_bf16 or resume set), GPOP_ERR_OOM, GPOP_ERR_CUDA.  num_seeds = 0 returns GPOP_OK without work.
 */
gpop_status gpop_run_ppr_batch(gpop_graph *g, const gpop_run_opts *opts, const uint32_t *seeds, uint32_t num_seeds,
                               float *out_values, int out_is_device, gpop_run_stats *stats);

/*
 * Checkpoint of a run (all applications but multi-source BFS): the vertex values, BFS levels, next
 * messages and frontier bitmap the last successful gpop_run on this graph left, with its algorithm, the
 * number of iterations behind it and the L1 change of its last gather.
 *   gpop_state_export  writes the checkpoint into the caller's HOST buffer of `capacity` bytes and its
 *                      size into *size; with buffer NULL only the size is returned.
 *   gpop_state_import  loads a checkpoint of the same graph (vertex and edge counts, partition size and a
 *                      fingerprint of its edges and weights must match) into this graph, for a following
 *                      gpop_run with opts.resume set.  That run must repeat the saved run's options that
 *                      shape the result (source, damping, epsilon, msg_bf16, where the algorithm uses them);
 *                      otherwise it returns GPOP_ERR_INVALID_ARG.
 * The layout is an 80-byte header (magic "GPST", version 2, algorithm, V, iterations, frontier words,
 * L1 change, E, graph fingerprint, P, msg_bf16, source, damping, epsilon) then V words each of values,
 * levels and messages and the frontier words, little endian.
 * Errors: GPOP_ERR_INVALID_ARG (no state held, buffer too small, header or size that does not match,
 * another graph or partition size), GPOP_ERR_OOM, GPOP_ERR_CUDA.
 */
gpop_status gpop_state_export(const gpop_graph *g, void *buffer, uint64_t capacity, uint64_t *size);
gpop_status gpop_state_import(gpop_graph *g, const void *buffer, uint64_t size);

/*
 * Diagnostics of the bounded device waits (every mbarrier wait of the PC gather and the PC scatter gives
 * up after a fixed number of polls, raises the run's error word and lets the run return
 * GPOP_ERR_TIMEOUT, leaving the CUDA context usable).  This call runs the same wait, on the current
 * device, against a barrier phase that nothing completes, with at most `tries` polls, and sets
 * *gave_up = 1 when the wait ran out and raised the error word as it must.  Errors:
 * GPOP_ERR_INVALID_ARG (gave_up NULL), GPOP_ERR_CUDA, GPOP_ERR_DEVICE_CHECK (the phase reported
 * completion, which would be a defect).
 */
gpop_status gpop_probe_bounded_wait(uint32_t tries, uint32_t *gave_up);

/*
 * Learned SC/PC selector (replaces Eq. (mode) per partition per iteration when
 * opts.mode = GPOP_MODE_LEARNED).  An MLP 8 -> 32 -> 32 -> 1 with ReLU,
 * FP32, predicting y = log(t_PC / t_SC); PC is chosen iff y <= 0.  Features
 * are standardised with the stored mean/std; a partition whose features fall
 * outside the training range [fmin, fmax] falls back to Eq. (mode).
 * Parameter layout (GPOP_SELECTOR_PARAMS floats): W1[32][8], b1[32],
 * W2[32][32], b2[32], W3[32], b3, then mean[8], std[8], fmin[8], fmax[8].
 * The paper has no learned selector; the traffic model it replaces is Sec. 3.2.
 */
#define GPOP_SELECTOR_FEATURES 8
#define GPOP_SELECTOR_HIDDEN 32
#define GPOP_SELECTOR_WEIGHTS (32 * 8 + 32 + 32 * 32 + 32 + 32 + 1)
#define GPOP_SELECTOR_PARAMS (GPOP_SELECTOR_WEIGHTS + 4 * 8)

/* Installs selector parameters (host array of GPOP_SELECTOR_PARAMS floats)
 * process-wide, or removes them when params is NULL. */
gpop_status gpop_selector_set(const float *params);

/* Copies the installed parameters to a host array; GPOP_ERR_NO_SELECTOR if none. */
gpop_status gpop_selector_get(float *params);

/*
 * Trains the selector on the GPU with the library's own forward, backward and
 * Adam kernels (mean squared error on y), full-batch.
 *   features  n x 8 host floats (raw features as logged by LOG_BOTH)
 *   targets   n host floats, y = log(t_PC / t_SC)
 *   epochs, lr  Adam steps and step size; seed  initialisation stream
 *   params_out  GPOP_SELECTOR_PARAMS host floats (trained weights + feature statistics)
 *   loss_out    optional, final MSE
 */
gpop_status gpop_selector_train(const float *features, const float *targets, uint32_t n, uint32_t epochs,
                                float lr, uint64_t seed, void *cuda_stream, float *params_out,
                                float *loss_out);

/*
 * Forward pass and parameter gradients of the MSE loss on one batch (device
 * kernels), for checking against a CPU reference.
 *   params  GPOP_SELECTOR_WEIGHTS host floats (weights only)
 *   x       n x 8 host floats, already standardised;  y  n host floats
 *   pred_out n host floats;  grad_out GPOP_SELECTOR_WEIGHTS host floats;  loss_out optional
 */
gpop_status gpop_selector_grad(const float *params, const float *x, const float *y, uint32_t n,
                               void *cuda_stream, float *pred_out, float *grad_out, float *loss_out);

/*
 * Allocation-free variant of gpop_selector_grad for callers that cannot call cudaMalloc: code running
 * while a stream is captured into a CUDA graph, code whose device memory belongs to another allocator
 * (a framework's caching allocator or a fixed arena), and loops where an allocation would synchronise
 * the device.  The paper has no counterpart; this is a convenience of this library.
 *   params   GPOP_SELECTOR_WEIGHTS device floats;  x  n x 8 device floats (standardised);  y  n device floats
 *   n        1 <= n <= 16384 (GPOP_ERR_INVALID_ARG otherwise)
 *   pred_out n device floats or NULL;  grad_out GPOP_SELECTOR_WEIGHTS device floats;  loss_out 1 device float or NULL
 * The call only enqueues two kernels on cuda_stream and returns; results are ready when the stream
 * reaches them.  Its scratch is one fixed 1.4 MB device array inside the library, held by every GPU that
 * loads the library until the process exits; nothing in it needs clearing between calls, and calls whose
 * kernels overlap on the GPU (different streams, or different host threads) race on it.  The first call
 * on each device looks up that array's device address with the device current; make that first call
 * before any stream capture begins.  No cudaMalloc, cudaFree or other allocating routine is called.
 */
gpop_status gpop_selector_grad_noalloc(const float *params, const float *x, const float *y, uint32_t n,
                                       void *cuda_stream, float *pred_out, float *grad_out, float *loss_out);

/* Description of the last error on the calling thread ("" if none). */
const char *gpop_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* GPOP_H */
