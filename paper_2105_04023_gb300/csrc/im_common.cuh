// Device-side data layout and helpers shared by the kernels and the host engine of the influence-maximisation
// library.  One DevProb describes one seed-selection problem (a graph, its sampling thresholds and every device
// buffer of its sketch); kernels take an array of them so that a single launch serves many problems.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace imk {

constexpr int kBlock = 256;          // threads per block of every kernel
constexpr int kWarpsPerBlock = kBlock / 32;
constexpr int kHeavyDeg = 64;        // rows with more out-edges are split into tasks (task_edges)
constexpr int kTaskEdges = 64;
constexpr int kBigTasks = 32;        // split rows with more tasks are merged by a whole block
constexpr int kMaxTaskEdges = 1024;

// Edges of each task of a split row with d out-edges: kTaskEdges, or for hubs (d > kTaskEdges * kBigTasks) a
// multiple of kTaskEdges near d / 512, at most kMaxTaskEdges, so that a hub has about 512 partial rows to merge
// (more only past 512 kMaxTaskEdges edges): the one block that merges a hub's partials was the critical path for
// hubs of 10^5 to 10^6 edges in 64-edge tasks.  The first sweep hands tasks out dynamically, so their unequal
// lengths do not unbalance it.
__host__ __device__ __forceinline__ int64_t task_edges(int64_t d) {
    if (d <= static_cast<int64_t>(kTaskEdges) * kBigTasks) return kTaskEdges;
    const int64_t t = ((d + 511) / 512 + kTaskEdges - 1) / kTaskEdges * kTaskEdges;
    return t < kMaxTaskEdges ? t : kMaxTaskEdges;
}
constexpr int kBfsTaskEdges = 32;    // out-edges per search task with R = 1024 (one warp, one edge a lane)
constexpr int kBfsTaskEdgesMin = 8;  // out-edges per search task with R <= 256 (four tasks a warp)
// Out-edges per search task for rows of W words: a group of that many lanes holds the task's delta row.
__host__ __device__ constexpr int bfs_task_edges(int W) { return W <= 8 ? 8 : (W <= 16 ? 16 : kBfsTaskEdges); }
constexpr int kPushChunk = 1024;     // a changed vertex pushes its in-edges in units of at most this many
constexpr int kMcChunk = 8192;      // edges per generator stream of the Monte-Carlo influence scorer
constexpr int kCasLimit = 1024;      // compare-and-swap tries of one register-word update before it counts as a fault
                                     // (the default of DevProb::cas_limit)

enum Model : int32_t { kIC = 0, kWC = 1, kPerEdge = 2 };

// Work of one sweep unit (a light row, or a task of task_edges(deg) edges of a split row): its sparse pairs
// [p0, p0 + np) and its dense edges dlist[d0, d0 + nd); hu is vertex_hash(u), the first sweep's seed of u's initial
// ranks (0 in push-unit descriptors).
struct UnitD {
    int64_t p0;
    int64_t d0;
    uint32_t np;
    uint32_t nd;
    int32_t u;
    uint32_t hu;
};

// Grid-wide barrier of the persistent (cooperatively launched) kernels: arrivals and a generation count; and the
// finished-block count of the frontier kernels.
struct GridBar {
    unsigned int count;
    unsigned int gen;
    unsigned int fail;   // a block gave up waiting (every block then leaves the kernel)
    unsigned int tail;   // blocks of a frontier launch that finished: the last one ends the sweep or level
};
constexpr uint32_t kBarrierLimit = 1u << 20;  // polls of one barrier wait (under a second in all) before giving up
                                              // (the default limit the persistent search is launched with)

// Counters of one problem, written by the kernels and read back by the host after each engine tick.
struct DevCtr {
    // diffusion (Algorithm 2) ----------------------------------------------------------------------------------
    uint32_t t;          // sweep index of the current diffusion
    uint32_t done;       // 1 once the diffusion reached its stop condition
    uint32_t timeout;    // 1 if it hit the sweep limit first
    uint32_t full;       // the current sweep pulls into every row; otherwise L pushes along its in-edges
    uint32_t res_par;    // register buffer (0/1) holding the diffusion's result
    uint32_t nchg;       // vertices whose registers changed in the current sweep (|L'|, counted after it)
    uint32_t nchg_list;  // entries written to chg_list (changed vertices with at most kPushChunk in-edges)
    uint32_t nchg_hc;    // entries written to chg_hc (chunks of the changed vertices with more)
    uint32_t npush_l;    // chg_list / chg_hc entries the current push sweep works on
    uint32_t npush_h;
    uint32_t stream;     // the current push sweep streams every in-pair (its L is large)
    uint32_t task_next;  // first sweep: tasks handed out so far (the tiles that finished their rows take the next)
    uint32_t fault;      // bit 0: a bulk copy did not complete in time; bit 1: a register update kept failing;
                         // bit 2: a grid barrier of a persistent kernel was not reached in time;
                         // bit 3: a pulling sweep reached the push-only kernel;
                         // bit 4: a row's kept register sum disagreed with its registers (check_sums only)
    unsigned long long chg_indeg;     // in-edges into the vertices changed in the current sweep
    unsigned long long visits;        // edge-simulation visits, running total
    unsigned long long bytes;         // algorithmic bytes of the propagation kernels, running total
    unsigned long long pairs;         // sparse (edge, simulation) pairs the propagation kernels examined
    unsigned long long first_bytes;   // of `bytes`, those of the first-sweep kernel
    unsigned long long sweeps_total;  // sweeps, running total
    // greedy step (Algorithm 1) --------------------------------------------------------------------------------
    unsigned long long best_key;      // max over candidates of (gain << 32 | ~v), gain = gsum - gms
    unsigned long long cand_key;      // lazy scan: max over candidates of (stale gain << 32 | ~v)
    unsigned long long tau_key;       // lazy scan: exact key of that candidate (the bound the others must beat)
    uint32_t s;          // seed chosen by the last step
    uint32_t gsum;       // sum_j max(M_S'[j], M_s[j]) of that seed
    uint32_t gms;        // sum_j M_S'[j] (the register sum every candidate's gsum is compared over)
    uint32_t pad_c;
    // reachability search ---------------------------------------------------------------------------------------
    uint32_t lvl;        // level of the current search
    uint32_t bdone;      // 1 once the search found no new vertex
    uint32_t btimeout;   // 1 if it hit the level limit first
    uint32_t lvl0;       // level at which the current search started
    uint32_t nT[2];      // search tasks by level parity
    uint32_t nVl[3];     // frontier vertices by level mod 3 (those of the next level are added during a level)
    unsigned long long reached;       // |{(v, j): v in R_{G_j}(S)}|
    unsigned long long levels_total;
};

// One problem.  Register rows are R bytes, 16-byte aligned; bit arrays are 32-bit words.
struct DevProb {
    int64_t n, m;
    const int64_t *xadj;       // out-CSR (Section 3.3)
    const int32_t *adj;
    const int64_t *xadj_in;    // in-CSR, used to list the rows a changed vertex feeds
    const int32_t *adj_in;
    const uint32_t *ein;       // per in-edge: its index in the out-CSR
    const uint32_t *heavy;     // bit per row: out-degree > kHeavyDeg
    const int64_t *task_off;   // n+1: first task of each row (tasks only for heavy rows)
    const int32_t *task_row;   // per task: its row
    const int32_t *light_list; // rows with 1 .. kHeavyDeg out-edges
    const int32_t *hsmall;     // split rows with at most kBigTasks tasks
    const int32_t *hbig;       // split rows with more tasks
    int64_t n_tasks;
    int64_t n_light, n_hsmall, n_hbig;
    int32_t model;
    int32_t R;                 // simulations (registers per row), a power of two in [64, 1024]
    int32_t W;                 // R / 32: words per row of a bit array over simulations
    uint32_t T_const;          // IC threshold
    int32_t ic_ok;             // IC: p > 0
    int32_t undirected;        // both directions of an edge share one hash key (min, max): an undirected input
    const uint32_t *T_vert;    // WC: threshold per target vertex
    const uint32_t *T_edge;    // per-edge model: threshold per edge
    const uint8_t *ok_edge;    // per-edge model: p > 0
    const uint32_t *X;         // sampling words X_r (Eq. 5)
    const uint32_t *Y;         // initialisation words ("hash(j)" of Algorithm 1)
    uint8_t *M0, *M1;          // register buffers (Jacobi pair)
    uint8_t *part;             // n_tasks x R partial maxima of heavy-row tasks
    uint32_t *part_any;        // bit per task: the task merged at least one neighbour
    uint32_t *Lb0, *Lb1;       // frontier bits: vertices changed in the previous sweep
    uint16_t *dmask;           // n x R/16: per 16-simulation chunk of row v, the registers the previous sweep changed
                               // (written by the frontier pass for the rows it copies, read by the next push sweep)
    int32_t *chg_list;         // compacted changed vertices with at most kPushChunk in-edges
    uint64_t *chg_hc;          // (chunk << 32) | v for the changed vertices with more in-edges
    uint32_t *live;            // m x W: edge e is live in simulation j (Eq. 4-5 evaluated once per run)
    // Sparse form of the sampled edges.  An edge live in at most dense_min simulations contributes one pair
    // (target v, simulation j) per live simulation, pairs in edge order; an edge live in more is a dense edge,
    // merged with whole register rows.
    const int64_t *pofs;       // m+1: pairs before each edge
    const int64_t *dofs;       // m+1: dense edges before each edge
    const int32_t *pv;         // per pair: target vertex (NULL unless pulling sweeps follow the first, or a rebuild
                               // tests each pair's target: more than 2^32 pairs)
    const uint16_t *pj;        // per pair: simulation (NULL with pv)
    const uint16_t *pq;        // per pair, for the first sweep: sw_slot(simulation, 0) | initial rank of (target,
                               // simulation) << 10 (R <= 1024, ranks <= 32)
    const uint32_t *iop;       // per in-pair: the index of the same pair in out-CSR order
    const uint32_t *dlist;     // dense edge ids, in edge order
    // the same pairs and dense edges by target: per in-edge of the in-CSR
    const int64_t *ipofs;      // m+1: in-pairs before each in-edge
    const int64_t *idofs;      // m+1: dense in-edges before each in-edge
    const int32_t *iu;         // per in-pair: source vertex
    const int32_t *iv;         // per in-pair: target vertex (the in-CSR row holding it), for streamed push sweeps
    const uint16_t *ij;        // per in-pair: simulation
    const int32_t *idu;        // per dense in-edge, in in-CSR order: source vertex
    const uint32_t *ide;       //   and out-CSR edge id
    const UnitD *vdesc;        // n: push unit of each vertex (in-pairs, dense in-edges)
    const UnitD *rdesc;        // n: sweep unit of each row (used for light rows)
    const UnitD *tdesc;        // n_tasks: sweep unit of each task
    int32_t dense_min;
    uint32_t pull_sweeps;      // sweeps 0 .. pull_sweeps-1 pull into every row, later ones push
    unsigned long long stream_min;  // a push sweep whose L has at least this many in-edges streams every in-pair
                                    // instead of taking L's vertices one by one (~0: never)

    uint32_t *vis;             // n x W: v in R_{G_j}(S)
    uint32_t *rany;            // bit per vertex: reached by S in some simulation (set at a rebuild; NULL: no search)
    uint16_t *pqb;             // residual blocking: this problem's copy of pq with the ranks of blocked (v, j) at 0
    uint8_t *Mi;               // n x R: the initial registers (Algorithm 1's initialisation) the first sweep of a
                               // diffusion reads, with the blocked (v, j) at 0 under residual blocking
    uint32_t *vis_done;        // n x W: the blocked bits already applied to Mi and pqb
    uint32_t *rnew;            // bit per vertex: has bits in vis not yet in vis_done (set by k_init)
    uint32_t *del[3];          // n x W: bits newly reached at the previous level, by level mod 3
    uint32_t *lstamp;          // per vertex: 1 + the last level that listed it
    int4 *T[2];                // search tasks by level parity: {first edge (lo, hi), vertex, edge count}
    int32_t *V[3];             // frontier vertices by level mod 3
    uint32_t *inS;             // bit per vertex: in the seed set
    uint8_t *MS;               // R bytes: M_S'
    uint32_t *gst;             // n: a candidate's last evaluated gain sum_j max(M_S'[j], M_v[j]) - sum_j M_S'[j]; an
                               // upper bound of its gain until the sketch is rebuilt (M_S' only grows)
    DevCtr *ctr;
    uint32_t stop_thr;         // diffusion stops when |L'| <= stop_thr
    uint32_t max_sweeps;       // sweep / level limit
    int32_t flog_cap;
    int64_t *flog;             // |L| at the start of each sweep of the current diffusion
    uint32_t *step_seed;       // per greedy step k: seed (device trace)
    uint32_t *step_gsum;
    unsigned long long *step_reached;
    uint32_t cas_limit;        // compare-and-swap tries of one register-word update before the fault flag is raised
    uint32_t check_sums;       // the full scan checks that gst holds every row's register sum while M_S' is empty
    int32_t literal;           // blocked registers as Algorithms 1 and 2 print them: they keep their initial rank and
                               // are never updated (otherwise they are 0 in a rebuilt sketch)
};

// ------------------------------------------------------------------------------------------------------------
// Method arithmetic (independent restatement of the paper's Section 3.1 / Algorithm 1 readings)

// MurmurHash3's 32-bit finaliser.
__device__ __forceinline__ uint32_t fmix32(uint32_t x) {
    x ^= x >> 16;
    x *= 0x85EBCA6Bu;
    x ^= x >> 13;
    x *= 0xC2B2AE35u;
    x ^= x >> 16;
    return x;
}

// Eq. 4: hash of edge (u, v) from the 64-bit key u * n + v; an undirected input hashes both directions of an edge
// by the key of (min, max), so they are live in the same simulations.
__device__ __forceinline__ uint32_t edge_hash(uint64_t u, uint64_t v, uint64_t n, bool undirected) {
    if (undirected && v < u) {
        const uint64_t t = u;
        u = v;
        v = t;
    }
    const uint64_t key = u * n + v;
    return fmix32(static_cast<uint32_t>(key) ^ fmix32(static_cast<uint32_t>(key >> 32)));
}

// Initial FM rank of vertex v for simulation word y (Algorithm 1's initialisation).
__device__ __forceinline__ uint32_t vertex_hash(uint32_t v) { return fmix32(v ^ 0x9E3779B9u); }

__device__ __forceinline__ bool test_bit(const uint32_t *bits, int64_t i) {
    return (bits[i >> 5] >> (i & 31)) & 1u;
}

__device__ __forceinline__ void set_bit(uint32_t *bits, int64_t i) { atomicOr(&bits[i >> 5], 1u << (i & 31)); }

// Threshold of edge e = (u, v) and whether it can be live at all.
__device__ __forceinline__ void edge_threshold(const DevProb &P, int64_t e, int32_t v, uint32_t &T, bool &ok) {
    if (P.model == kIC) {
        T = P.T_const;
        ok = P.ic_ok != 0;
    } else if (P.model == kWC) {
        T = __ldg(&P.T_vert[v]);
        ok = true;
    } else {
        T = __ldg(&P.T_edge[e]);
        ok = __ldg(&P.ok_edge[e]) != 0;
    }
}

}  // namespace imk
