/*
 * bp_gb300.h - C ABI of the GB300 (sm_103a) frontier-scheduled loopy belief
 * propagation library (libbp_gb300.so).
 *
 * The library runs sum-product belief propagation on discrete pairwise Markov
 * random fields (Section II-A, Eq. 1) with the frontier loop of Algorithm 1:
 * every round it evaluates candidate messages (Eq. 2) and their residuals
 * (Eq. 4), tests eps-convergence, selects a frontier and commits it. Four
 * frontier generators are provided: synchronous LBP (Section II-B, III-A),
 * top-k Residual BP (Section III-A, III-D), Residual Splash (Section II-B, III-A)
 * and Randomized BP (Section IV-A). Beliefs follow Eq. 3.
 *
 * Conventions shared by every entry point
 *  - All pointers are HOST pointers unless stated otherwise; the library copies
 *    what it needs to the GPU, so the caller keeps ownership of every input and
 *    provides every output buffer.
 *  - Return value: BP_OK (0) or a negative bp_status code; bp_last_error()
 *    returns a message describing the most recent failure of the calling thread.
 *  - A handle is not thread-safe: use one handle per host thread.
 *  - Graph layout: CSR of directed edges. Directed edge e = (i -> j) is stored in
 *    row i (row_ptr[i] <= e < row_ptr[i+1]) with col[e] = j; rev[e] is the id of
 *    the opposite edge (j -> i). Both directions of every undirected edge must be
 *    present; self-loops are rejected.
 *  - Non-convergence within max_rounds is not an error: the run's stats say
 *    converged = 0 and the beliefs come from the last committed state.
 */
#ifndef BP_GB300_H
#define BP_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bp_graph bp_graph;

typedef enum {
    BP_OK = 0,
    BP_ERR_INVALID_ARG = -1,   /* a NULL pointer, a size or a parameter out of range */
    BP_ERR_BAD_GRAPH = -2,     /* CSR not monotone, col out of range, rev not an involution,
                                  col[rev[e]] != source(e), self-loop, or an edge that
                                  leaves its graph in a batch */
    BP_ERR_NO_POTENTIALS = -3, /* bp_run before bp_set_potentials */
    BP_ERR_NONFINITE = -4,     /* NaN/Inf potential, or an asymmetric pairwise table */
    BP_ERR_CUDA = -5,          /* a CUDA runtime call failed (see bp_last_error) */
    BP_ERR_TIMEOUT = -6,       /* the wall-clock budget of bp_run ran out */
    BP_ERR_OOM = -7,           /* device or host allocation failed */
    BP_ERR_UNSUPPORTED = -8,   /* combination not implemented (e.g. k > 32) */
    BP_ERR_NO_RESULT = -9,     /* results requested before any bp_run */
    BP_ERR_INTERNAL = -10      /* an internal consistency check failed (a library bug;
                                  see bp_last_error) */
} bp_status;

/* Frontier generators (Algorithm 1, GenerateFrontier). */
typedef enum {
    BP_LBP = 0,   /* every message, every round (Section II-B) */
    BP_RBP = 1,   /* top-k messages by residual, k = clamp(ceil(p*M), 1, M) (Section III-A) */
    BP_RS = 2,    /* top-k vertices by vertex residual + depth-h splash (Section II-B) */
    BP_RNBP = 3   /* residual >= eps, then a Philox Bernoulli(p) filter (Section IV-A) */
} bp_schedule;

/* Storage type of the log-domain messages (arithmetic is FP32, or FP64 for BP_F64).
 * Binary Ising messages (k = 2, BP_PAIR_ISING_BETA) are stored as one log-odds
 * value u = log m(1) - log m(0); other messages as k values log m(x).
 * BP_BF16: k-state logs are rounded to bfloat16. A binary Ising log-odds is
 * stored in the exponent of a bfloat16 word: the word nearest to
 * w = 2^(|u| / b - 125) with the sign of u, b = the smallest power of two
 * >= 2 max_e |beta_e| / 250.
 * An Ising message satisfies |u| <= 2 |beta|, so w stays in [2^-125, 2^125],
 * and the word's exponent and mantissa bits form a logarithmic code of |u|
 * whose step is at most b / 128 (a plain bfloat16 log-odds would have a
 * relative step of 2^-7 |u|, too coarse for beliefs within 2e-3).
 * BP_Q16 (binary Ising only) stores u as a signed 16-bit integer q with
 * u = q * s, s = (float)(2 max_e |beta_e| / 32767); the step is uniform.
 * bp_storage_scale returns b and s. With BF16 and Q16 a residual compares
 * rounded candidates with the stored messages, so an unchanged stored value
 * has residual 0. */
typedef enum { BP_F64 = 0, BP_F32 = 1, BP_BF16 = 2, BP_Q16 = 3 } bp_msg_dtype;

/* Pairwise potential layouts, as natural logs theta = log psi (Eq. 1). */
typedef enum {
    BP_PAIR_ISING_BETA = 0, /* k = 2; beta per directed edge [M]:
                               theta(x_i, x_j) = beta * s(x_i) * s(x_j), s(0) = -1, s(1) = +1;
                               beta[rev[e]] must equal beta[e] */
    BP_PAIR_TABLE = 1,      /* [M * k * k], entry (e, a, b) = theta(x_src = a, x_dst = b);
                               table(rev[e]) must be the transpose of table(e) */
    BP_PAIR_SHARED = 2      /* one symmetric [k * k] table for every edge (Potts-like) */
} bp_pair_kind;

/* Per-run (or per-graph) statistics. */
typedef struct {
    int32_t converged;          /* 1 if max residual < eps at the final evaluation */
    int32_t rounds;             /* committing rounds (Algorithm 1 loop iterations) */
    int64_t committed_updates;  /* sum of frontier sizes (RS: messages updated in splashes) */
    int64_t candidate_evals;    /* message evaluations (Eq. 2) performed */
    double final_max_residual;  /* max residual at the final evaluation */
    int64_t final_unconverged;  /* messages with residual >= eps at the final evaluation */
    int32_t status;             /* BP_OK, or BP_ERR_TIMEOUT when stopped by the budget */
    int32_t n_graphs;           /* graphs summarised by this record */
    double device_ms;           /* device time of the whole bp_run call */
} bp_run_stats;

/* Options of bp_run; bp_default_options fills the defaults noted here. */
typedef struct {
    uint64_t seed;            /* Philox key for RnBP (default 0) */
    double high_p;            /* RnBP HighP (default 1.0, Section IV-D) */
    double ratio_threshold;   /* RnBP EdgeRatio switch (default 0.9, Section IV-A) */
    int32_t splash_depth;     /* RS splash depth h (default 2, Section III-D) */
    int32_t rs_roots_mode;    /* RS roots: 0 = clamp(ceil(p*M), 1, n) (default), 1 = ceil(p*n) */
    int32_t msg_dtype;        /* bp_msg_dtype (default BP_F32) */
    int32_t record_trace;     /* 1: record each round's frontier as a bitmask (default 0) */
    int32_t trace_capacity;   /* rounds the trace can hold (default 0) */
    int32_t rounds_per_launch;/* rounds per CUDA-graph replay between host polls (0 = auto) */
    void *cuda_stream;        /* cudaStream_t to run on (NULL = the legacy default stream) */
    double time_budget_ms;    /* wall-clock budget of bp_run, 0 = none */
    uint32_t graph_id_base;   /* Philox graph id of graph 0 of the handle (default 0) */
    int32_t kernel_variant;   /* binary Ising update mapping (every mapping computes the
                                 same bits): 0 = automatic (the choice bp_autotune
                                 recorded for the handle's size class; else, for
                                 messages that are not FP64, 6 for RnBP when the
                                 streamed tiles apply, 4 when no vertex has more
                                 than 4 edges and 6 when the streamed tiles apply; 1
                                 otherwise), 1 =
                                 per-round kernels, one thread per vertex, 3 = persistent
                                 batch kernel: one thread-block cluster per graph runs all
                                 of its rounds in a single launch, 4 = one thread per
                                 vertex with the graph arrays of 4 edges prefetched in
                                 parallel with the graph's status, 6 = streamed tiles: warp tiles of <= 128 edges staged in
                                 shared memory by bulk copies from a producer warp, one
                                 lane per edge (FP32 / BF16 / Q16 messages, vertices with
                                 <= 128 out-edges; BP_ERR_UNSUPPORTED otherwise); 2 and 5
                                 (two mappings that never measured fastest) are retired
                                 and rejected (BP_ERR_INVALID_ARG) */
    int32_t profile;          /* 1: time every round's phases with CUDA events (default 0) */
    int32_t potts_path;       /* shared-table (BP_PAIR_SHARED) update, FP32/BF16 storage,
                                 k <= 32, tiles of <= 128 edges: 0 = automatic (3 for
                                 16 <= k <= 32, else the per-vertex k-state kernel), 1 = tiles on the
                                 CUDA cores, 2 = tiles on the tensor cores with BF16
                                 products, 3 = tensor cores with the BF16 residual
                                 products added (close to FP32) */
    int32_t select_path;      /* RBP / RS top-k selection (same frontier either way):
                                 0 = automatic (by an occupancy-based time estimate), 1 =
                                 one thread-block cluster per graph, 2 = grid-wide
                                 kernels (for a few large graphs) */
    int32_t splash_sweep;     /* RS sweeps (binary messages, splash_depth <= 3): 0 =
                                 automatic, 1 = one launch per sub-step over the
                                 batch-wide level lists, one list entry per thread (the
                                 only form; 0 selects it). Any other value is
                                 BP_ERR_INVALID_ARG. */
    int32_t overlap_launches; /* programmatic dependent launches of the per-round update,
                                 decision and RnBP commit kernels (each grid may be
                                 scheduled while the previous kernel drains; it waits
                                 for it before reading run state; the sweep steps
                                 always launch without it): 0 = automatic (on), 1 =
                                 on, 2 = off */
    int32_t dynamic_p;        /* RBP and RS: 1 = switch the frontier fraction every round
                                 by the EdgeRatio rule that RnBP uses (Section IV-A; the
                                 paper tried the same for RBP / RS and dropped it for its
                                 overhead): HighP = high_p in round 1, then
                                 parallelism (LowP) when the count of messages with
                                 residual >= eps grew by more than ratio_threshold
                                 relative to the previous round, else high_p; 0 = the
                                 fixed fraction parallelism (default) */
} bp_options;

/* Phase timings and launch counts of the last bp_run. The timings are filled
 * only when the run had profile = 1: the rounds are then launched directly
 * (not through a captured CUDA graph) with CUDA events on the run's stream
 * between the evaluation kernel (Eq. 2 + Eq. 4 + convergence reduction), the
 * per-graph decision and the frontier work (selection, splash, commit);
 * rounds after every graph had stopped are left out. A profiled run pays the
 * direct-launch overhead, so its wall time is above an unprofiled run's; the
 * kernel durations themselves are unaffected. */
typedef struct {
    int64_t kernel_launches;   /* kernels launched by bp_run (graph nodes replayed + direct) */
    int64_t eval_launches;     /* timed full-evaluation launches (profile = 1) */
    int64_t full_evals;        /* messages evaluated by those launches */
    int64_t active_vertices;   /* vertices processed by those launches */
    double eval_ms;            /* summed duration of those launches */
    double decide_ms;          /* summed duration of the per-graph decisions */
    double frontier_ms;        /* summed duration of selection / splash / commit */
    double batch_kernel_ms;    /* duration of the persistent batch kernel (always recorded
                                  when that kernel ran; 0 otherwise) */
    double select_ms;          /* part of frontier_ms: selection, RnBP commit, splash levels */
    double sweep_ms;           /* part of frontier_ms: the Residual Splash sweeps */
    int64_t sweep_launches;    /* fused sweep-step launches (binary RS), counted with sweep_ms */
    int32_t select_ctas[2];    /* RBP, RS selection of the run: CTAs per graph of the cluster
                                  kernels (0 when the grid-wide kernels ran; always filled) */
    int32_t kernel_variant;    /* the binary update mapping the run used (always filled) */
    int32_t sweep_ctas;        /* always 0 (the RS sweeps run one launch per sub-step) */
    int32_t sweep_form;        /* always 0: RS sweeps as per-sub-step launches */
    int32_t overlap_launches;  /* 1 when the run used programmatic dependent launches */
    int32_t fused_commit;      /* 1 when the RnBP rounds committed inside the streamed update
                                  (kernel_variant 6 without a recorded trace: both EdgeRatio
                                  outcomes written, no commit kernel; always filled) */
} bp_profile;

/* Fills *opt with the defaults listed above. */
void bp_default_options(bp_options *opt);

/* Result of bp_autotune. */
typedef struct {
    int32_t kernel_variant;    /* the fastest mapping measured (1, 3, 4 or 6) */
    int32_t size_class;        /* the key it was recorded under: schedule (bits 0-1), msg_dtype
                                  (2-3), floor(log2(n_vars / n_graphs)) (4-8),
                                  floor(log2(n_graphs)) (9-13), largest vertex degree
                                  <= 4 / <= 8 / more (14-15) */
    double ms_per_round[8];    /* measured device ms per round, index = mapping; 0 = not tried */
    int32_t select_path;       /* RBP / RS: the faster selection path measured (1 cluster, 2
                                  grid-wide; bp_options.select_path), 0 for other schedules */
    double ms_per_round_select[3]; /* device ms per round with the chosen mapping, index =
                                  selection path; 0 = not tried */
} bp_tune_result;

/*
 * Creates a handle for one graph: the structure of the pairwise MRF of Eq. 1
 * (Section II-A), one variable per vertex and one pairwise factor per
 * undirected edge, stored as the adjacency list with edge and vertex ids that
 * Section III-B describes. n_states = k (uniform over vertices,
 * 2 <= k <= 128). row_ptr has n_vars + 1 entries (row_ptr[0] = 0,
 * row_ptr[n_vars] = n_dir_edges), col and rev have n_dir_edges entries.
 * The CSR is validated (BP_ERR_BAD_GRAPH) and copied to the device.
 * n_dir_edges must be below 2^31. *out receives the handle.
 */
int bp_create_graph(int32_t n_vars, int32_t n_states, int64_t n_dir_edges,
                    const int64_t *row_ptr, const int32_t *col, const int32_t *rev,
                    bp_graph **out);

/*
 * Creates a handle for a batch of independent graphs given as one disjoint
 * union: graph g owns vertices [graph_var_offsets[g], graph_var_offsets[g+1])
 * and every edge of those rows, which must stay inside the graph. Each graph
 * is tested for convergence, counts its rounds and stops on its own; graph g
 * draws RnBP randomness with graph id graph_id_base + g.
 */
int bp_create_batch(int32_t n_graphs, const int64_t *graph_var_offsets, int32_t n_states,
                    int64_t n_dir_edges, const int64_t *row_ptr, const int32_t *col,
                    const int32_t *rev, bp_graph **out);

/*
 * Sets the log-potentials of Eq. 1. unary_log is [n_vars * k] (row = vertex);
 * pair_log is laid out per bp_pair_kind (see above). Inputs are validated for
 * finiteness and for the symmetry the kind requires (BP_ERR_NONFINITE) and
 * copied to the device; any previous result of the handle is discarded.
 * Variable state counts (the paper's protein-folding graphs, Section IV-E,
 * have 2 to 81 states per vertex): a unary log-potential of -inf marks that
 * state of that vertex absent, so vertex v has k_v <= k present states. A
 * message into v is then a distribution over v's present states (uniform at
 * the start of a run, no mass on the absent ones) and absent states get
 * belief 0. Needs BP_PAIR_TABLE (BP_ERR_UNSUPPORTED otherwise; table entries
 * may also be -inf) and at least one present state per vertex
 * (BP_ERR_NONFINITE). NaN and +inf are rejected everywhere. Binary Ising
 * couplings (BP_PAIR_ISING_BETA) are copied as they are and checked and
 * turned into the update's arrays on the device (the call returns when that
 * work is done); after a rejected call the handle has no potentials until the
 * next successful one.
 */
int bp_set_potentials(bp_graph *g, const float *unary_log, int32_t pair_kind,
                      const float *pair_log);

/*
 * Runs Algorithm 1 from uniform messages (Section II-A) until every graph of
 * the handle has max residual < eps (converged) or has committed max_rounds
 * rounds. parallelism = p for RBP and RS, LowP for RnBP (HighP in opt),
 * ignored for LBP; 0 < parallelism, eps > 0, max_rounds >= 0. opt may be NULL
 * (defaults). stats (nullable) receives the whole-handle summary: converged =
 * 1 only if all graphs converged, rounds = the largest round count, counters
 * summed. On return the beliefs (Eq. 3) are ready for bp_get_beliefs.
 * Device memory: the handle keeps two message buffers of the storage format
 * (n_dir_edges x elements per message), residuals, and per-graph state from
 * the first run on; an RnBP run on the streamed mapping (kernel_variant 6)
 * without a recorded trace adds a third message buffer (it writes both
 * EdgeRatio outcomes of a round, Section IV-A), kept until the storage format
 * changes or the handle is destroyed. A failed allocation returns BP_ERR_OOM.
 */
int bp_run(bp_graph *g, int32_t schedule, double parallelism, double eps, int32_t max_rounds,
           const bp_options *opt, bp_run_stats *stats);

/* Copies the beliefs of the last bp_run (Eq. 3: b_i(x) proportional to
 * psi_i(x) times the product of the incoming messages, normalised in FP64),
 * [n_vars * k] float64 (row = vertex), rows summing to 1. The caller owns out. */
int bp_get_beliefs(const bp_graph *g, double *out);

/* Copies the final messages of the last bp_run (the committed state of the
 * Eq. 2 updates, each normalised to sum 1 as Section II-A requires) in the
 * probability domain, [n_dir_edges * k] float64 (row e = message on directed
 * edge e); a 16-bit stored value is decoded exactly as the kernels decode it.
 * The caller owns out. */
int bp_get_messages(const bp_graph *g, double *out);

/* Copies the residuals (Eq. 4: max-norm of the probability-domain change) of
 * the evaluation that ended the last bp_run, out[n_dir_edges] float64: for a
 * run stopped by max_rounds = t these are the residuals the frontier of round
 * t + 1 would be selected from. RnBP, RBP and RS runs (LBP keeps none:
 * BP_ERR_UNSUPPORTED); in a batch, a graph that stopped earlier keeps its own
 * final evaluation's values. */
int bp_get_residuals(const bp_graph *g, double *out);

/* Copies per-graph statistics of the last bp_run into out[n_graphs]. */
int bp_get_graph_stats(const bp_graph *g, bp_run_stats *out);

/*
 * Copies the recorded frontiers of the last bp_run (record_trace = 1). Round t
 * (1-based) occupies words [(t-1) * W, t * W) with W = ceil(count / 32), count =
 * n_dir_edges (LBP, RBP, RnBP: bit e = message e committed) or n_vars (RS: bit
 * v = vertex v chosen as splash root); bit b of a word is (word >> b) & 1.
 * *rounds_out receives the number of recorded rounds; fails with
 * BP_ERR_INVALID_ARG when capacity_words is too small.
 */
int bp_get_trace(const bp_graph *g, uint32_t *out, int64_t capacity_words, int32_t *rounds_out);

/*
 * bp_lbp_run_noalloc - synchronous LBP (FP32 messages) on one binary Ising
 * graph without allocating any memory. The paper has no counterpart: this is a
 * service entry point for callers that cannot allocate device memory, such as
 * code running under another framework's caching allocator that has already
 * reserved the GPU, latency-critical paths where cudaMalloc/cudaFree would
 * synchronise the device, or plug-ins that must leave the allocation state
 * alone.
 *
 * Every pointer argument except rounds_out and converged_out is a DEVICE
 * pointer owned by the caller: row_ptr [n_vars + 1] (int32), col and rev
 * [n_dir_edges], unary_log [n_vars * 2], beta [n_dir_edges] (layouts as for
 * bp_create_graph / BP_PAIR_ISING_BETA), beliefs [n_vars * 2] float64 output.
 * rounds_out / converged_out are optional HOST outputs. The run evaluates with
 * the thread-per-vertex update mapping (bp_options.kernel_variant = 1) in
 * direct launches, with the same arithmetic, rounds and convergence test as
 * bp_run(BP_LBP) with msg_dtype BP_F32 and that mapping, and writes the same
 * beliefs bit for bit.
 *
 * Scratch: one static device array of about 5.0 MiB in the library, held on
 * every GPU where it has been set up until the process exits. It bounds the
 * graph to at most 131072 vertices and 262144 directed edges (larger graphs
 * fail with BP_ERR_UNSUPPORTED before anything is launched). The CUDA runtime
 * loads the library's device code lazily, so the FIRST call on each device does
 * the set-up: it loads this entry point's module, which places the array (and
 * the module's code) in device memory, and looks up the array's device address
 * with that device current. Make that first call (a small graph will do) before
 * a framework reserves the GPU's memory and before any stream capture; later
 * calls on that device allocate nothing. Each call clears the scratch it reads
 * and runs on cuda_stream (NULL = legacy default stream), synchronising it.
 * Every call on a device shares the one array: calls whose work overlaps on
 * the GPU race on it, so callers must serialise them. Inputs are validated on
 * the device (BP_ERR_BAD_GRAPH, BP_ERR_NONFINITE). A launch error is reported
 * as BP_ERR_CUDA with the failing step; an error that earlier CUDA work of the
 * calling thread left pending is consumed at entry and not reported.
 */
int bp_lbp_run_noalloc(int32_t n_vars, int64_t n_dir_edges, const int32_t *row_ptr, const int32_t *col,
                       const int32_t *rev, const float *unary_log, const float *beta, double eps,
                       int32_t max_rounds, double *beliefs, int32_t *rounds_out, int32_t *converged_out,
                       void *cuda_stream);

/*
 * bp_autotune - picks the binary Ising update mapping (bp_options.kernel_variant)
 * for the handle's size class by measurement. The paper has no counterpart
 * (it runs one kernel design); the batch configuration of arbitrary graph
 * sizes calls for a tuned choice per size class.
 *
 * For each mapping (1, 4, 6 where the streamed tiles apply, and 3 when the
 * handle holds more than one graph) it runs bp_run(schedule, parallelism, eps, trial_rounds, opt) twice
 * (the first run captures the rounds; the second is timed by its device_ms)
 * and records the mapping with the least device time per round in a
 * process-wide table under the size class (see bp_tune_result); for RBP and
 * RS it then times both selection paths with that mapping and records the
 * faster. Later runs with kernel_variant = 0 (select_path = 0) on any handle
 * of that size class, schedule and msg_dtype use them. Every mapping gives the same results, so tuning changes
 * speed only. The trial runs leave no result (bp_get_beliefs fails with
 * BP_ERR_NO_RESULT until the next bp_run). Binary Ising handles only
 * (BP_ERR_UNSUPPORTED otherwise); trial_rounds >= 1; errors of bp_run pass
 * through. The table is guarded by a mutex; the handle itself is not
 * thread-safe.
 */
int bp_autotune(bp_graph *g, int32_t schedule, double parallelism, double eps, const bp_options *opt,
                int32_t trial_rounds, bp_tune_result *out);

/*
 * bp_set_graph_parallelism - per-graph parallelism for the graphs of a batch:
 * p[q] (host array of n_graphs values, each > 0 and finite) replaces bp_run's
 * parallelism argument for graph q: its RnBP LowP (Section IV-A), or its RBP /
 * RS frontier fraction (Section III-D). p = NULL returns to the run's single
 * value. The values are copied to the device and stay until changed. The
 * paper runs one p per experiment; a batch of graphs of different sizes can
 * use a p per size class (bp_autotune_parallelism).
 */
int bp_set_graph_parallelism(bp_graph *g, const double *p);

/*
 * bp_autotune_parallelism - picks the parallelism of every size class of the
 * batch's graphs (class = floor(log2(vertices of the graph))) among
 * candidates[0 .. n_candidates) (each > 0, at most 64 candidates) for RnBP,
 * RBP or RS. For each candidate it runs bp_run(schedule, candidate, eps,
 * max_rounds, opt) on the whole batch and scores each class by the rounds its
 * graphs took to converge, a graph that did not converge counting
 * 2 * max_rounds; the lowest score wins (ties: the earlier candidate). The
 * choice is installed with bp_set_graph_parallelism and, when graph_p_out is
 * not NULL, copied to graph_p_out[n_graphs] (host). The trial runs leave no
 * result. Errors of bp_run pass through.
 */
int bp_autotune_parallelism(bp_graph *g, int32_t schedule, const double *candidates, int32_t n_candidates,
                            double eps, int32_t max_rounds, const bp_options *opt, double *graph_p_out);

/*
 * bp_time_update - device time of the message-update kernel (Eq. 2 + Eq. 4 +
 * convergence reduction) alone, for rooflines: the kernel that bp_run(schedule,
 * parallelism, opt) would launch every round (same mapping, storage format and
 * shared-table path) is launched `launches` times back to back on
 * opt->cuda_stream from uniform messages, between two CUDA events;
 * *ms_per_launch receives the mean. Every launch evaluates every message of
 * every graph (no graph stops), so launches do identical work. The handle's
 * previous result is discarded (bp_get_beliefs fails with BP_ERR_NO_RESULT
 * until the next bp_run). BP_ERR_UNSUPPORTED for the persistent batch mapping
 * (3), which has no separate update launch; launches >= 1. The paper has no
 * counterpart (measurement support).
 */
int bp_time_update(bp_graph *g, int32_t schedule, double parallelism, const bp_options *opt, int32_t launches,
                   double *ms_per_launch);

/*
 * bp_storage_scale - the scale of a 16-bit message format on the handle's
 * binary Ising potentials (see bp_msg_dtype), with B = max_e |beta_e|:
 * BP_Q16: the log-odds per integer unit, s = (float)(2 B / 32767);
 * BP_BF16: the log-odds per unit of log2 of the stored word, b = the
 * smallest power of two >= 2 B / 250. When every beta is 0, B = 1/2 is used. *out (host)
 * receives it. BP_ERR_INVALID_ARG for other formats, BP_ERR_UNSUPPORTED for
 * other potential layouts, BP_ERR_NO_POTENTIALS before bp_set_potentials. The
 * paper has no counterpart (the formats are this library's message storage;
 * the scale is exported so that checkers emulate the same grid).
 */
int bp_storage_scale(const bp_graph *g, int32_t msg_dtype, float *out);

/* Copies the phase profile of the last bp_run (see bp_profile). */
int bp_get_profile(const bp_graph *g, bp_profile *out);

/* Sizes of a handle (any pointer may be NULL). */
int bp_graph_info(const bp_graph *g, int32_t *n_vars, int32_t *n_states, int64_t *n_dir_edges,
                  int32_t *n_graphs);

/* Frees the handle and its device memory. NULL is ignored. */
void bp_destroy_graph(bp_graph *g);

/* Static description of a status code. */
const char *bp_status_string(int status);

/* Message of the last failure on the calling thread ("" if none). */
const char *bp_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* BP_GB300_H */
