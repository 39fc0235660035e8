/*
 * im.h — C ABI of a GB300-native (sm_103a) sketch-based influence-maximisation library.
 *
 * The library implements the hot path of HyperFuseR (Goktürk & Kaya, arXiv 2105.04023): hash-based fused sampling
 * of independent-cascade simulations (Section 3.1, Eq. 4-5), Flajolet-Martin sketch registers per vertex and
 * simulation (Section 2.2, Eq. 1-3) diffused to a fixpoint by pull-based sweeps (Algorithm 2), and greedy seed
 * selection with error-adaptive sketch rebuilding (Algorithm 1, Section 3.2.1).  Every step runs in the library's
 * own CUDA kernels on one GPU.
 *
 * Conventions for every call:
 *   - Each call returns an im_status; IM_OK (0) means success.  A non-zero status leaves every output untouched
 *     and the reason is available from im_last_error(ctx) until the next call on that context.  No call aborts.
 *   - A context is used by one host thread at a time.  All device work of a context is issued on its CUDA stream
 *     (the one given to im_ctx_create, or a stream the context creates); calls return after that work completes.
 *   - Graph arrays are owned by the caller and are read only; with IM_MEM_DEVICE they are device pointers that
 *     must stay valid for the lifetime of every sketch built from them, with IM_MEM_HOST the library copies them
 *     into its own device memory during the call.
 *   - Sketches, contexts and batches are owned by the library and freed by their *_destroy call.
 *   - Output pointers are HOST pointers unless stated otherwise.
 *
 * Readings of the paper that fix the results (shared with the CPU oracle used by the tests):
 *   edge hash h(u,v) = fmix32(lo32(u*n+v) XOR fmix32(hi32(u*n+v))) (MurmurHash3 finaliser, Eq. 4), h_max = 2^32;
 *   simulation words X_r, Y_r = high halves of splitmix64 outputs 2r and 2r+1 from the seed;
 *   edge (u,v) is live in simulation r iff (h XOR X_r) <= ceil(p * 2^32) - 1 (Eq. 5, "P < w"), p = 1/indeg(v)
 *   for the weighted cascade, never for p <= 0;
 *   initial register M_v[j] = clz32(fmix32(v XOR 0x9E3779B9) XOR Y_j) (Algorithm 1 initialisation);
 *   u pulls from its out-neighbour v: M_u[j] = max(M_u[j], M_v[j]) over live edges (Algorithm 2);
 *   estimate e = 2^(mean_j M[j]) / 0.77351 (Eq. 2); greedy argmax over v not in S, ties to the smallest id.
 */
#ifndef IM_H_
#define IM_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    IM_OK = 0,
    IM_EINVAL = 1,     /* invalid argument: malformed CSR, out-of-range id, bad R, K or probability */
    IM_ENOMEM = 2,     /* the footprint does not fit the device memory or the given HBM budget */
    IM_ECUDA = 3,      /* a CUDA runtime call failed (including "no device") */
    IM_ETIMEOUT = 4,   /* a diffusion or search exceeded its sweep limit (im_params.max_sweeps) */
    IM_ECANCELED = 5,  /* the request was cancelled before it ran */
    IM_ENOTREADY = 6   /* a batch or served request has not finished yet */
} im_status;

typedef enum {
    IM_IC_CONST = 0, /* independent cascade, the same probability p on every edge (Section 2.1) */
    IM_WC = 1,       /* weighted cascade, p(u,v) = 1 / indeg(v) (Section 2.1, Fig. 1b) */
    IM_PER_EDGE = 2  /* one probability per edge, p_edge[e] for the e-th entry of adj */
} im_model;

typedef enum {
    IM_MEM_DEVICE = 0, /* xadj / adj / p_edge are device pointers of the context's device */
    IM_MEM_HOST = 1    /* they are host pointers (pinned or pageable); the library copies them */
} im_memory;

/*
 * A directed graph as an out-neighbour CSR (Section 3.3): the targets of vertex u are adj[xadj[u] .. xadj[u+1]-1].
 * Requirements (checked, IM_EINVAL otherwise): n >= 1, xadj[0] = 0, xadj non-decreasing, xadj[n] = m, every target
 * in [0, n), n < 2^31.  Self-loops and parallel edges should be merged beforehand (Section 2.1); they are accepted
 * and treated as ordinary edges.
 * undirected = 1 marks an undirected input (six of the paper's graphs, Section 4) stored with both directions of
 * every edge: each row sorted by target and every (u, v) matched by (v, u) (checked, IM_EINVAL otherwise).  Both
 * directions then take the hash of the key (min(u, v), max(u, v)) and are sampled in the same simulations, so with
 * one probability for both directions a sampled graph reaches exactly a connected component; the weighted cascade
 * keeps 1/indeg of the target per direction.  im_influence_mc does not take undirected inputs.
 */
typedef struct {
    int64_t n;             /* vertices */
    int64_t m;             /* edges */
    const int64_t *xadj;   /* n + 1 row offsets */
    const int32_t *adj;    /* m target ids */
    im_model model;
    double p;              /* IM_IC_CONST: the edge probability, in [0, 1] */
    const float *p_edge;   /* IM_PER_EDGE: m probabilities in [0, 1]; NULL otherwise */
    im_memory memory;
    int32_t undirected;    /* 0: directed; 1: undirected input stored with both directions (see above) */
} im_graph;

typedef enum {
    IM_BLOCK_RESIDUAL = 0, /* a rebuild sketches the residual samples: registers of vertices S reaches are 0 and never
                              updated (Section 3.2.1) */
    IM_BLOCK_LITERAL = 1   /* Algorithms 1 and 2 as printed: a rebuild re-initialises every register and Simulate
                              never updates a blocked (u, j), which keeps its rank and passes it to unblocked
                              in-neighbours */
} im_blocking;

/*
 * Parameters of one influence-maximisation run (Algorithm 1).
 * R: simulations = FM registers per vertex (the paper's J): 64, 128, 256, 512 or 1024.
 * K: seeds to select, 1 <= K <= n.
 * eps_g, eps_l: global and local error thresholds of Section 3.2.1 (the paper uses 0.01 and 0.3); 0 rebuilds the
 *   sketch after every seed, +infinity never rebuilds.
 * eps_c: the diffusion stops after the first sweep whose set of changed vertices has at most eps_c * n members
 *   (Section 3.2; 0 runs to the fixpoint).
 * seed: run seed of the per-simulation words.
 * max_sweeps: limit on sweeps of one diffusion and levels of one reachability search; 0 means n + 2 (always
 *   enough for a fixpoint).  Exceeding it returns IM_ETIMEOUT.
 * blocking: an im_blocking value, how a rebuild treats the registers of vertices S reaches (default residual).
 */
typedef struct {
    int32_t R;
    int32_t K;
    double eps_g;
    double eps_l;
    double eps_c;
    uint64_t seed;
    int64_t max_sweeps;
    int32_t blocking;
} im_params;

/* Per-step record of a seed selection (Algorithm 1); every array has K entries and may be NULL. */
typedef struct {
    int32_t *seeds;     /* chosen seed of step k */
    double *sigma;      /* sigma after step k: mean over the R samples of |R_{G_j}(S)| */
    double *estimate;   /* e of step k: Estimate(Merge(M_S', M_s)) */
    uint64_t *gsum;     /* integer register sum behind e: sum_j max(M_S'[j], M_s[j]) */
    uint8_t *rebuilt;   /* 1 if the error check of step k asked for a rebuild */
} im_trace;

/* Counters of the last completed call on a context. */
typedef struct {
    uint64_t visits;          /* edge-simulation visits: sum over sweeps of |{(u,v): v in L}| * R */
    uint64_t prop_bytes;      /* bytes the propagation kernels must move: per visited row 16 (offsets) + R (own
                                 row) + R if written; per scanned edge 4 (target id) + the threshold bytes of edges
                                 to live-set vertices (4 weighted cascade, 5 per-edge); R per neighbour row read;
                                 R per partial row written and read back for split rows */
    int64_t sweeps;           /* diffusion sweeps */
    int64_t builds;           /* diffusions run (initial build + rebuilds) */
    int64_t bfs_levels;       /* reachability-search levels */
    int64_t kernel_launches;  /* kernels launched by the call */
    int64_t prop_launches;    /* launches of the propagation kernel (one per sweep and R class) */
    double prop_ms;           /* summed CUDA-event time of the propagation kernels of every sweep (the row kernel
                                 and the merge of split rows; 0 unless timing is enabled) */
    double total_ms;          /* device time of the whole call (CUDA events around it) */
    double sweep_ms;          /* with timing enabled: all kernels of the diffusion sweeps */
    double scan_ms;           /* with timing enabled: gain scans and seed choice */
    double bfs_ms;            /* with timing enabled: reachability-search levels */
    double init_ms;           /* with timing enabled: register (re)initialisation and M_S' merges */
    uint64_t live_pairs;      /* sparse (edge, simulation) pairs the propagation kernels examined: the live pairs
                                 behind `visits` that the sweeps actually touch (edges live in many simulations,
                                 merged as whole rows, are not counted) */
    uint64_t first_bytes;     /* of prop_bytes, those of the first sweep of every diffusion (its own kernel) */
    double first_ms;          /* with timing enabled: CUDA-event time of the first-sweep kernel's launches */
    int64_t first_launches;   /* its launches */
} im_stats;

typedef struct im_ctx im_ctx;
typedef struct im_sketch im_sketch;

/* Creates a context on CUDA device `device`.  `cuda_stream` is a cudaStream_t to issue work on, or NULL for a
 * stream owned by the context.  Returns IM_ECUDA if the device cannot be used. */
im_status im_ctx_create(int device, void *cuda_stream, im_ctx **out);
im_status im_ctx_destroy(im_ctx *ctx);

/* Last error message of the context (never NULL); valid until the next call on the context. */
const char *im_last_error(const im_ctx *ctx);

/*
 * Autotuning of launch shapes (no counterpart in the paper; the results never depend on it).  For the graph's
 * shape class (R and the mean out-degree class floor(log2(m / n)) + 1, or 0 when m < n) the call times the first
 * diffusion of `graph` with `params` under each candidate configuration (the register budget of the first-sweep
 * kernel, 3, 4 or 6 resident blocks per SM, and whether push sweeps over a large frontier stream every in-pair),
 * checks that every candidate reaches the same registers, sweeps and visits (IM_ECUDA otherwise), and keeps the
 * fastest for all later calls on the context with graphs of that class.  out (nullable) receives the choice.
 */
typedef struct {
    int32_t first_sweep_blocks; /* chosen register budget of the first-sweep kernel (resident blocks per SM) */
    int32_t stream_push;        /* 1: push sweeps over a large frontier stream every in-pair */
    int32_t candidates;         /* configurations timed */
    int32_t degree_class;
    double best_ms;             /* diffusion time under the chosen configuration (best of two) */
    double default_ms;          /* and under the default one */
} im_tuning;

im_status im_autotune(im_ctx *ctx, const im_graph *graph, const im_params *params, im_tuning *out);

/* Enables (1) or disables (0) per-launch CUDA-event timing of the propagation kernel, reported in im_stats. */
im_status im_ctx_set_timing(im_ctx *ctx, int enable);

/* Copies the counters of the last completed call. */
im_status im_ctx_stats(const im_ctx *ctx, im_stats *out);

/*
 * Builds the sketch of a graph: initial registers (Algorithm 1) then Simulate (Algorithm 2) to the fixpoint (or
 * the eps_c stop).  Uses params R, seed, eps_c and max_sweeps.  The sketch keeps pointers to the caller's device
 * graph arrays (IM_MEM_DEVICE) or its own copy (IM_MEM_HOST).
 */
im_status im_build_sketches(im_ctx *ctx, const im_graph *graph, const im_params *params, im_sketch **out);

/*
 * Influence estimate of a seed set on a built sketch: the registers of the k seeds are merged (Eq. 3) and
 * estimated (Eq. 2) into *est_out.  If sigma_out is not NULL the exact mean reach of the set over the sketch's R
 * hash-sampled graphs is also computed (Algorithm 1's Monte-Carlo step).  seeds is a host array of k ids in
 * [0, n); k >= 1.
 */
im_status im_estimate(im_ctx *ctx, const im_sketch *sketch, const int32_t *seeds, int32_t k, double *est_out,
                      double *sigma_out);

/* Copies the n*R registers of a sketch, row-major (vertex-major, simulation-minor), to host memory. */
im_status im_sketch_registers(im_ctx *ctx, const im_sketch *sketch, uint8_t *host_out);

/* Number of sweeps and edge-simulation visits of the sketch's diffusion; frontier_log (may be NULL) receives
 * |L| at the start of each sweep for the first log_cap sweeps. */
im_status im_sketch_info(im_ctx *ctx, const im_sketch *sketch, int64_t *sweeps, uint64_t *visits,
                         int64_t *frontier_log, int64_t log_cap);

im_status im_sketch_destroy(im_sketch *sketch);

/*
 * Export and import of a built sketch, so that one build serves later runs with the same (graph, R, seed, eps_c,
 * max_sweeps) outside a server (Section 3's sketch is a pure function of them).  The exported bytes are an
 * im_sketch_header, then the R sampling words X_r and the R initialisation words Y_r (uint32 each), then the n*R
 * registers, row-major.  The header carries the parameters, the diffusion's sweep and visit counts, and a 64-bit
 * fingerprint of the graph (its edges and per-edge thresholds) that an import must match.
 */
#define IM_SKETCH_MAGIC 0x314354454B534D49ull /* the bytes "IMSKETC1" */
typedef struct {
    uint64_t magic;      /* IM_SKETCH_MAGIC */
    int64_t n, m;
    int32_t R;
    int32_t model;       /* im_model */
    double p;            /* the graph's p */
    uint64_t seed;
    double eps_c;
    int64_t max_sweeps;
    int64_t sweeps;      /* sweeps of the diffusion */
    uint64_t visits;     /* its edge-simulation visits */
    uint64_t graph_hash;
    int32_t undirected;
    int32_t reserved;
} im_sketch_header;

/* Writes the sketch to host_buf (HOST pointer, capacity cap bytes) and its size to *size_out; with host_buf NULL only
 * the size is reported.  IM_EINVAL if cap is too small. */
im_status im_sketch_export(im_ctx *ctx, const im_sketch *sketch, void *host_buf, uint64_t cap, uint64_t *size_out);

/*
 * Recreates a sketch from exported bytes (HOST pointer, size bytes) on `graph`, which must be the graph it was built
 * on (same n, m, model, p, undirected flag and fingerprint; IM_EINVAL otherwise).  The sampling of the graph is
 * redone (it is deterministic) and its words must equal the exported ones.  The imported sketch answers
 * im_estimate, im_sketch_registers and im_select_seeds_from like the original; im_sketch_info reports its sweep
 * and visit counts but no frontier sizes (zeros).
 */
im_status im_sketch_import(im_ctx *ctx, const im_graph *graph, const void *host_buf, uint64_t size,
                           im_sketch **out);

/*
 * im_select_seeds starting from a built (or imported) sketch instead of running the first diffusion: params must
 * have the sketch's R, seed, eps_c and max_sweeps (IM_EINVAL otherwise); K, eps_g, eps_l and blocking are free.
 * The results are those of im_select_seeds with the same graph and parameters.  The sketch is not modified.
 */
im_status im_select_seeds_from(im_ctx *ctx, const im_sketch *sketch, const im_params *params, int32_t *seeds_out,
                               double *sigma_out, int32_t *rebuilds_out, im_trace *trace);

/*
 * Selects K seeds with Algorithm 1: build, then K greedy steps; each step picks the argmax of the merged-sketch
 * estimate, computes the exact reach of S over the R samples, and either merges the seed into M_S' or rebuilds
 * the sketch on the residual samples (registers of vertices reached by S set to 0) when both the local and the
 * global estimation error reach their thresholds.  seeds_out: host array of K ids.  sigma_out (nullable): final
 * sigma.  rebuilds_out (nullable): number of steps whose check asked for a rebuild.  trace (nullable): per step.
 */
im_status im_select_seeds(im_ctx *ctx, const im_graph *graph, const im_params *params, int32_t *seeds_out,
                          double *sigma_out, int32_t *rebuilds_out, im_trace *trace);

/*
 * Runs nq independent seed selections (one graph and parameter set each) together: every kernel launch serves
 * all problems that are in the same phase, so many small graphs share the GPU.  seeds_out[q] is a host array of
 * params[q].K ids; sigma_out (nullable) receives nq final sigmas; rebuilds_out (nullable) nq counts.  Results are
 * identical to nq separate im_select_seeds calls.
 */
im_status im_select_seeds_batch(im_ctx *ctx, int32_t nq, const im_graph *graphs, const im_params *params,
                                int32_t *const *seeds_out, double *sigma_out, int32_t *rebuilds_out);

/*
 * Serving.  A server keeps a pool of graphs prepared on the device and answers seed-selection queries on them.
 * Queries wait in a first-come-first-served queue and are admitted while a batch slot is free and the device bytes
 * of all running queries stay within the HBM budget; each admitted query's footprint (registers 2 n R bytes, reach
 * bits 3 n R / 8, and lists of O(n + m / 64) words) is allocated on admission and freed when it finishes.  Every
 * im_server_step admits what fits and then advances all running queries by one engine tick, in which each phase
 * (sweeps, gain scans, reachability searches) is one launch for all of them, so queries that arrive while others
 * run join the batch at the next step (continuous batching).  Results are identical to im_select_seeds on the
 * same graph and parameters.  A server and its context are used by one host thread.
 */
typedef struct im_server im_server;

/* Creates a server on ctx with an HBM budget for running queries and at most max_active (1..4096) of them. */
im_status im_server_create(im_ctx *ctx, uint64_t hbm_budget_bytes, int32_t max_active, im_server **out);
im_status im_server_destroy(im_server *srv);

/* Prepares a graph on the device (copied if IM_MEM_HOST) and adds it to the pool; *graph_id names it. */
im_status im_server_add_graph(im_server *srv, const im_graph *graph, int32_t *graph_id);

/* Queues a query (Algorithm 1 with these parameters on graph graph_id); *ticket identifies it.  IM_ENOMEM if the
 * query alone needs more than the budget. */
im_status im_server_submit(im_server *srv, int32_t graph_id, const im_params *params, uint64_t *ticket);

/* Device bytes a query with these parameters on graph graph_id is charged against the budget on admission. */
im_status im_server_footprint(im_server *srv, int32_t graph_id, const im_params *params, uint64_t *bytes);

/* Admits queued queries that fit and advances every running query by one tick; reports how many queries are
 * running and queued afterwards (either pointer may be NULL).
 * A query's first diffusion depends only on (graph, R, seed, eps_c, max_sweeps): the server keeps the sampled
 * graph and the registers of each first diffusion it runs, within the budget, and a later query with the same five
 * starts from them (same results: the diffusion is deterministic).  Kept diffusions are dropped, least recently
 * used first, when an admission needs their room. */
im_status im_server_step(im_server *srv, int32_t *active_out, int32_t *queued_out);

/* Budget use of a server (HOST pointers, each may be NULL): bytes charged (running queries' reservations plus kept
 * diffusions), kept diffusions, and queries started from a kept diffusion so far. */
im_status im_server_info(const im_server *srv, uint64_t *used_bytes, int32_t *kept_builds, uint64_t *build_hits);

/* Result of a ticket: IM_ENOTREADY while queued or running; IM_OK with seeds_out (params.K ids), sigma_out and
 * rebuilds_out (each may be NULL) once done, after which the ticket is forgotten; IM_ECANCELED for a cancelled
 * query; a query that failed returns its error status. */
im_status im_server_poll(im_server *srv, uint64_t ticket, int32_t *seeds_out, double *sigma_out,
                         int32_t *rebuilds_out);

/* Cancels a queued or running query (its memory is freed at once). */
im_status im_server_cancel(im_server *srv, uint64_t ticket);

/* Largest seed count and register count accepted by im_estimate_static. */
#define IM_STATIC_MAX_SEEDS 4096
#define IM_STATIC_MAX_R 1024

/*
 * Estimate of a seed set that allocates no device memory.  The paper has no counterpart: this is an interface
 * addition for callers that must not allocate at call time, such as a serving thread on a latency budget
 * (cudaMalloc can synchronise the whole device and serialises on a process-wide lock) or a host process that
 * accounts for every device byte through its own allocator and does not let a library allocate behind its back.
 *
 * It returns what im_estimate returns without sigma: *est_out = 2^(g / R) / 0.77351 (Eq. 2), where g (also stored
 * in *gsum_out when it is not NULL) is the sum over the R simulations of the largest register of the k seeds
 * (Eq. 3).  The caller passes the data and owns it:
 *   registers: DEVICE pointer (device of ctx), 4-byte aligned, to an n x R uint8 register matrix, row-major (row v =
 *              the R registers of vertex v), for example the output of im_sketch_registers copied to the device.
 *              Any byte values are accepted (the library's own registers are at most 32);
 *   seeds:     DEVICE pointer, 4-byte aligned, to k vertex ids;
 *   est_out, gsum_out: HOST pointers, written only on IM_OK.
 * Limits: R is 64, 128, 256, 512 or 1024; 1 <= k <= IM_STATIC_MAX_SEEDS; n >= 1.  Other values, and unaligned
 * pointers, return IM_EINVAL, and so does a seed id outside [0, n) (checked on the device, the row is then not read).
 * Scratch: one static device array of about 64 KiB defined in the library, which every device that runs this
 * call keeps until the process exits.  The first call on a device looks up the array's address (once per device,
 * with that device current); make that first call before any stream capture on the device.  All calls share the
 * array and each call clears what it needs cleared, so calls that overlap on the GPU (from several threads or
 * streams) race and can return wrong results: serialise them.  Work runs on the context's stream with the
 * context's device current; the calling thread's current device is restored before the call returns, which is
 * after the work completes.
 */
im_status im_estimate_static(im_ctx *ctx, const uint8_t *registers, int64_t n, int32_t R, const int32_t *seeds,
                             int32_t k, double *est_out, uint64_t *gsum_out);

/*
 * Influence score of a seed set by plain sample-then-diffuse Monte Carlo, the way the paper's experiments score
 * every method's seed sets (Section 4, "Performance Metrics": a separate oracle that samples with mt19937 and then
 * diffuses, independent of the hash-based sampling of Section 3.1).  In each of nsamples samples every edge is
 * drawn live or not with mt19937, and the vertices the k seeds reach over the live edges are counted:
 *   sample s draws edge e's value as output (e mod 8192) of its own mt19937 stream for the chunk of 8192 edges
 *   holding e (out-CSR order), seeded by init_genrand with the high 32 bits of output s * ceil(m / 8192) +
 *   floor(e / 8192) of the splitmix64 sequence of `seed`; the edge is live iff the draw is <= its threshold
 *   T = ceil(p * 2^32) - 1 (weighted cascade: floor((2^32 - 1) / indeg(v)); p <= 0 never live).
 * graph: as for im_select_seeds (device or host arrays).  seeds: HOST array of k ids in [0, n), k >= 1 (repeats
 * count once).  nsamples: a multiple of 64 in [64, 2^24].  sigma_out: HOST pointer, receives the mean reach over
 * the samples.  reach_out: HOST array of nsamples counts (nullable), receives each sample's reach.  Outputs are
 * written only on IM_OK; IM_EINVAL for bad arguments or an invalid graph.  Device memory: one 1024-sample batch
 * (about m * 128 + n * 640 bytes) at a time, freed before the call returns.
 */
im_status im_influence_mc(im_ctx *ctx, const im_graph *graph, const int32_t *seeds, int32_t k, int64_t nsamples,
                          uint64_t seed, double *sigma_out, uint64_t *reach_out);

#ifdef __cplusplus
}
#endif

#endif /* IM_H_ */
