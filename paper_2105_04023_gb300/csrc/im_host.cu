// Host side of the library: contexts, graph preparation, per-problem device state, the engine that advances many
// seed-selection problems in lock step (one launch per phase serves all of them), and the C ABI of include/im.h.
//
// Host arithmetic that decides results (Algorithm 1's error check, Eq. 2) is done in double from the integers the
// kernels produce, with the same formula order as the paper states it; the file is compiled without floating
// contraction so the decisions do not depend on the compiler's use of fused multiply-add.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <deque>
#include <functional>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "../../include/im.h"
#include "im_common.cuh"
#include "im_launch.h"

using namespace imk;

namespace {

constexpr double kPhi = 0.77351;  // FM correction factor of Eq. 2

struct CudaError {
    cudaError_t code;
    const char *what;
};

inline void ck(cudaError_t e, const char *what) {
    if (e != cudaSuccess) throw CudaError{e, what};
}

struct ImError {
    im_status status;
    std::string msg;
};

[[noreturn]] inline void fail(im_status s, const std::string &msg) { throw ImError{s, msg}; }

}  // namespace

struct im_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::string err;
    im_stats stats{};
    bool timing = false;
    std::vector<cudaEvent_t> ev_free;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prop_ev;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> first_ev;  // the first-sweep kernel's launches
    int64_t first_launches = 0;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> phase_ev[4];  // sweeps, scans, searches, inits
    int64_t launches = 0;
    int64_t prop_launches = 0;
    DevCtr *h_ctr = nullptr;  // pinned staging for counter read-back
    size_t h_ctr_cap = 0;
    int32_t *h_act = nullptr;  // pinned staging for active lists
    size_t h_act_cap = 0;
    int32_t *d_act = nullptr;
    size_t d_act_cap = 0;
    int sweep_chunk = 8;   // sweeps enqueued per engine tick (the counters are read back once a tick)
    int level_chunk = 16;  // search levels enqueued per engine tick
    GridBar *d_gbar = nullptr;  // barrier of the persistent kernels
    int pull_sweeps = 1;        // sweeps of a diffusion that pull into every row before pushes take over
    // run whole searches in one cooperative launch (IM_PERSISTENT=1); measured no faster than level-by-level
    // launches on the R-MAT workloads, whose levels are dominated by their own dependent loads, so off by default
    bool persistent = false;
    // wait limits of the device-side waits; lowered only by the failure-detection tests (IM_TEST_CAS_LIMIT,
    // IM_TEST_BARRIER_LIMIT) to make a wait run out without any fault
    // lazy (CELF) argmax for greedy steps that keep the sketch (IM_CELF=0: a full scan every step; same results)
    bool celf = true;
    // the first step after a build scans every row and checks the register sums the sweeps kept
    // (IM_TEST_CHECK_SUMS=1); otherwise that step's argmax starts from those sums
    bool check_sums = false;
    // launch shapes chosen by im_autotune per (R, degree class): (first-sweep register budget, streamed pushes)
    std::map<std::pair<int, int>, std::pair<int, bool>> tuned;
    // push sweeps over a large L stream every in-pair (IM_STREAM=0: always vertex by vertex; same results)
    bool stream_push = true;
    uint32_t cas_limit = kCasLimit;
    uint32_t barrier_limit = kBarrierLimit;
};

namespace {

// ------------------------------------------------------------------------------------------------------------
// Device memory: stream-ordered allocations from the device's pool (kept reserved between calls).

struct DevMem {
    cudaStream_t s;
    std::vector<void *> ptrs;
    uint64_t bytes = 0;
    explicit DevMem(cudaStream_t st) : s(st) {}
    template <class T>
    T *alloc(size_t count, bool zero = false) {
        void *p = nullptr;
        const size_t bytes = std::max<size_t>(count * sizeof(T), 16);
        const cudaError_t e = cudaMallocAsync(&p, bytes, s);
        if (e == cudaErrorMemoryAllocation) {
            cudaGetLastError();
            fail(IM_ENOMEM, "device allocation of " + std::to_string(bytes) + " bytes failed");
        }
        ck(e, "cudaMallocAsync");
        ptrs.push_back(p);
        this->bytes += bytes;
        if (zero) ck(cudaMemsetAsync(p, 0, bytes, s), "cudaMemsetAsync");
        return static_cast<T *>(p);
    }
    // Returns a temporary allocation to the pool (stream-ordered: later work on s may reuse it).
    void release(void *p) {
        for (size_t i = 0; i < ptrs.size(); ++i)
            if (ptrs[i] == p) {
                cudaFreeAsync(p, s);
                ptrs.erase(ptrs.begin() + static_cast<std::ptrdiff_t>(i));
                return;
            }
    }
    ~DevMem() {
        for (void *p : ptrs) cudaFreeAsync(p, s);
    }
    DevMem(const DevMem &) = delete;
    DevMem &operator=(const DevMem &) = delete;
};

// Threshold of Eq. 5 for probability p: live iff (h XOR X_r) <= ceil(p * 2^32) - 1; p <= 0 is never live.
inline void ic_threshold(double p, uint32_t &T, int32_t &ok) {
    if (!(p > 0.0)) {
        T = 0;
        ok = 0;
        return;
    }
    T = static_cast<uint32_t>(std::ceil(p * 4294967296.0) - 1.0);
    ok = 1;
}

// A graph on the device with everything derived from it (in-CSR, thresholds, heavy-row tasks).
struct GraphDev {
    int64_t n = 0, m = 0;
    const int64_t *xadj = nullptr;
    const int32_t *adj = nullptr;
    const float *p_edge = nullptr;
    int32_t model = 0;
    int32_t undirected = 0;
    uint32_t T_const = 0;
    int32_t ic_ok = 0;
    int64_t *xadj_in = nullptr;
    int32_t *adj_in = nullptr;
    uint32_t *ein = nullptr;  // per in-edge: its index in the out-CSR
    uint32_t *T_vert = nullptr;
    uint32_t *T_edge = nullptr;
    uint8_t *ok_edge = nullptr;
    uint32_t *heavy = nullptr;
    int64_t *task_off = nullptr;
    int32_t *task_row = nullptr;
    int32_t *light_list = nullptr, *hsmall = nullptr, *hbig = nullptr;
    int64_t n_tasks = 0, n_light = 0, n_hsmall = 0, n_hbig = 0;
    std::unique_ptr<DevMem> mem;
    uint64_t bytes = 0;
};

}  // namespace

namespace imk {
void launch_validate(const int64_t *xadj, const int32_t *adj, int64_t n, int64_t m, unsigned int *flags,
                     cudaStream_t s);
void launch_edge_thresholds(const float *p, int64_t m, uint32_t *T, uint8_t *ok, unsigned int *flags,
                            cudaStream_t s);
void launch_validate_undirected(const int64_t *xadj, const int32_t *adj, int64_t n, unsigned int *flags,
                                cudaStream_t s);
}  // namespace imk

namespace {

void check_params(const im_params *pr, int64_t n, bool need_k) {
    if (!pr) fail(IM_EINVAL, "params is NULL");
    const int R = pr->R;
    if (R != 64 && R != 128 && R != 256 && R != 512 && R != 1024)
        fail(IM_EINVAL, "R must be one of 64, 128, 256, 512, 1024 (got " + std::to_string(R) + ")");
    if (need_k && (pr->K < 1 || pr->K > n)) fail(IM_EINVAL, "K must be in [1, n]");
    if (std::isnan(pr->eps_g) || std::isnan(pr->eps_l) || pr->eps_g < 0 || pr->eps_l < 0)
        fail(IM_EINVAL, "eps_g and eps_l must be >= 0");
    if (!(pr->eps_c >= 0.0 && pr->eps_c < 1.0)) fail(IM_EINVAL, "eps_c must be in [0, 1)");
    if (pr->max_sweeps < 0) fail(IM_EINVAL, "max_sweeps must be >= 0");
    if (pr->blocking != IM_BLOCK_RESIDUAL && pr->blocking != IM_BLOCK_LITERAL)
        fail(IM_EINVAL, "blocking must be IM_BLOCK_RESIDUAL or IM_BLOCK_LITERAL");
}

std::shared_ptr<GraphDev> prepare_graph(im_ctx *ctx, const im_graph *g) {
    if (!g) fail(IM_EINVAL, "graph is NULL");
    if (g->n < 1 || g->n >= (int64_t(1) << 31) - 1) fail(IM_EINVAL, "n must be in [1, 2^31 - 2]");
    if (g->m < 0 || g->m >= (int64_t(1) << 40)) fail(IM_EINVAL, "m out of range");
    if (!g->xadj || (g->m > 0 && !g->adj)) fail(IM_EINVAL, "xadj / adj is NULL");
    if (g->model != IM_IC_CONST && g->model != IM_WC && g->model != IM_PER_EDGE) fail(IM_EINVAL, "unknown model");
    if (g->model == IM_IC_CONST && !(g->p >= 0.0 && g->p <= 1.0)) fail(IM_EINVAL, "p must be in [0, 1]");
    if (g->model == IM_PER_EDGE && g->m > 0 && !g->p_edge) fail(IM_EINVAL, "p_edge is NULL");
    if (g->memory != IM_MEM_DEVICE && g->memory != IM_MEM_HOST) fail(IM_EINVAL, "unknown memory kind");
    if (g->undirected != 0 && g->undirected != 1) fail(IM_EINVAL, "undirected must be 0 or 1");
    cudaStream_t s = ctx->stream;
    auto G = std::make_shared<GraphDev>();
    G->mem = std::make_unique<DevMem>(s);
    DevMem &mem = *G->mem;
    G->n = g->n;
    G->m = g->m;
    G->model = g->model;
    G->undirected = g->undirected;
    const int64_t n = g->n, m = g->m;
    if (g->memory == IM_MEM_HOST) {
        if (g->xadj[0] != 0 || g->xadj[n] != m) fail(IM_EINVAL, "xadj[0] must be 0 and xadj[n] must be m");
        int64_t *x = mem.alloc<int64_t>(n + 1);
        ck(cudaMemcpyAsync(x, g->xadj, (n + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s), "copy xadj");
        int32_t *a = mem.alloc<int32_t>(m);
        if (m) ck(cudaMemcpyAsync(a, g->adj, m * sizeof(int32_t), cudaMemcpyHostToDevice, s), "copy adj");
        G->xadj = x;
        G->adj = a;
        if (g->model == IM_PER_EDGE) {
            float *pe = mem.alloc<float>(m);
            if (m) ck(cudaMemcpyAsync(pe, g->p_edge, m * sizeof(float), cudaMemcpyHostToDevice, s), "copy p");
            G->p_edge = pe;
        }
    } else {
        G->xadj = g->xadj;
        G->adj = g->adj;
        G->p_edge = g->p_edge;
    }
    // validation on the device: xadj[0] = 0, xadj[n] = m, non-decreasing, every target in [0, n)
    // (checked before any kernel indexes memory with these values)
    unsigned int *flags = mem.alloc<unsigned int>(8, true);
    launch_validate(G->xadj, G->adj, n, m, flags, s);
    ctx->launches += 1;
    {
        unsigned int f[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        ck(cudaMemcpyAsync(f, flags, sizeof(f), cudaMemcpyDeviceToHost, s), "read flags");
        ck(cudaStreamSynchronize(s), "sync");
        if (f[0]) fail(IM_EINVAL, "xadj[0] must be 0 and xadj[n] must be m");
        if (f[1]) fail(IM_EINVAL, "xadj must be non-decreasing");
        if (f[2]) fail(IM_EINVAL, "adj holds a vertex id outside [0, n)");
    }
    if (g->undirected) {  // (checked only once the offsets and ids are known to be in range)
        launch_validate_undirected(G->xadj, G->adj, n, flags, s);
        ctx->launches += 1;
        unsigned int f[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        ck(cudaMemcpyAsync(f, flags, sizeof(f), cudaMemcpyDeviceToHost, s), "read flags");
        ck(cudaStreamSynchronize(s), "sync");
        if (f[4]) fail(IM_EINVAL, "an undirected graph needs every row sorted by target without repeats");
        if (f[5]) fail(IM_EINVAL, "an undirected graph needs (v, u) for every edge (u, v)");
    }
    // in-degree, in-CSR
    int32_t *indeg = mem.alloc<int32_t>(n, true);
    launch_indeg(G->adj, m, indeg, s);
    const int64_t nb = scan_block_count(n) + 1;
    int64_t *bsums = mem.alloc<int64_t>(nb);
    G->xadj_in = mem.alloc<int64_t>(n + 1);
    ctx->launches += launch_exclusive_scan(indeg, n, G->xadj_in, bsums, s);
    unsigned long long *cursor = mem.alloc<unsigned long long>(n);
    ck(cudaMemcpyAsync(cursor, G->xadj_in, n * sizeof(int64_t), cudaMemcpyDeviceToDevice, s), "copy cursor");
    if (g->model == IM_WC) {
        G->T_vert = mem.alloc<uint32_t>(n);
        launch_wc_thresholds(indeg, n, G->T_vert, s);
        ctx->launches += 1;
    } else if (g->model == IM_PER_EDGE) {
        G->T_edge = mem.alloc<uint32_t>(m);
        G->ok_edge = mem.alloc<uint8_t>(m);
        launch_edge_thresholds(G->p_edge, m, G->T_edge, G->ok_edge, flags, s);
        ctx->launches += 1;
    } else {
        ic_threshold(g->p, G->T_const, G->ic_ok);
    }
    // heavy rows and their tasks
    const int64_t words = (n + 31) / 32;
    G->heavy = mem.alloc<uint32_t>(words, true);
    int32_t *ntask = mem.alloc<int32_t>(n);
    launch_row_tasks(G->xadj, n, ntask, G->heavy, s);
    G->task_off = mem.alloc<int64_t>(n + 1);
    ctx->launches += 1 + launch_exclusive_scan(ntask, n, G->task_off, bsums, s);
    // in-CSR, with the split-row task holding each in-edge
    G->adj_in = mem.alloc<int32_t>(m);
    G->ein = mem.alloc<uint32_t>(m);
    launch_transpose_fill(G->xadj, G->adj, n, m, cursor, G->adj_in, G->ein, s);
    ctx->launches += 2;
    int64_t h_tasks = 0;
    unsigned int h_flags[4] = {0, 0, 0, 0};
    ck(cudaMemcpyAsync(&h_tasks, G->task_off + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s), "read tasks");
    ck(cudaMemcpyAsync(h_flags, flags, sizeof(h_flags), cudaMemcpyDeviceToHost, s), "read flags");
    ck(cudaStreamSynchronize(s), "sync");
    if (h_flags[3]) fail(IM_EINVAL, "p_edge holds a value outside [0, 1]");
    if (n + h_tasks >= static_cast<int64_t>(0xFFFFFFFFll))  // the first sweep numbers rows and tasks in 32 bits
        fail(IM_EINVAL, "graph too large: vertices plus split-row tasks must stay below 2^32 - 1");
    G->n_tasks = h_tasks;
    G->task_row = mem.alloc<int32_t>(std::max<int64_t>(h_tasks, 1));
    G->light_list = mem.alloc<int32_t>(n);
    G->hsmall = mem.alloc<int32_t>(n);
    G->hbig = mem.alloc<int32_t>(n);
    unsigned int *counts = mem.alloc<unsigned int>(3, true);
    launch_classes(G->xadj, G->task_off, n, G->task_row, G->light_list, counts, G->hsmall, G->hbig, s);
    ctx->launches += 1;
    unsigned int h_counts[3] = {0, 0, 0};
    ck(cudaMemcpyAsync(h_counts, counts, sizeof(h_counts), cudaMemcpyDeviceToHost, s), "read classes");
    ck(cudaStreamSynchronize(s), "sync");
    G->n_light = h_counts[0];
    G->n_hsmall = h_counts[1];
    G->n_hbig = h_counts[2];
    return G;
}

// One seed-selection problem (or one sketch): its device state and the host side of Algorithm 1.
struct Prob {
    std::shared_ptr<GraphDev> G;
    im_params prm{};
    bool greedy = false;
    std::unique_ptr<DevMem> mem;
    std::shared_ptr<DevMem> smem;  // the sampled graph (live masks, pair lists, unit descriptors): read-only once
                                   // built, so queries with the same sample may share it
    DevProb dp{};
    DevProb *d_prob = nullptr;  // slot in the device descriptor array this problem was uploaded to
    DevCtr *d_ctr = nullptr;
    int64_t flog_cap = 0;
    // engine state
    enum Phase { kInit, kSweep, kScan, kBfs, kDone } phase = kInit;
    bool merge_pending = false;
    bool sums = false;  // gst holds every row's register sum, kept by the sweeps of the last build
    int step = 0;
    double varsigma = 0.0;
    std::vector<int32_t> seeds;
    std::vector<double> sigma, est;
    std::vector<uint64_t> gsum;
    std::vector<uint8_t> rebuilt;
    int64_t builds = 0;
    DevCtr last{};
    bool has_bfs = false;
    int64_t npairs = 0, ndense = 0;  // sparse pairs and dense edges of the sampled graph
    im_status status = IM_OK;  // failure of this problem when the engine keeps going (serving)
    std::string error;
    int variant = 0;  // register budget of the first-sweep kernel (resident blocks per SM; 0: default)
    // search levels: the counter at the start of the current search, and the length of the last finished one
    uint64_t levels_at_start = 0;
    uint32_t last_search_levels = 0;
};

// Shape class of a graph for the autotuner: floor(log2(mean out-degree)) + 1, 0 below one edge per vertex.
int degree_class(int64_t n, int64_t m) {
    if (m < n || n <= 0) return 0;
    int c = 1;
    for (int64_t d = m / n; d > 1; d >>= 1) ++c;
    return c;
}

// Buffers of the reachability searches (the per-edge live-simulation masks they read come from the sampling).
// The descriptor must be complete apart from its counters.
void alloc_bfs(Prob &P) {
    const int64_t n = P.G->n;
    const int W = P.prm.R / 32;
    DevMem &mem = *P.mem;
    const int64_t words = (n + 31) / 32;
    P.dp.vis = mem.alloc<uint32_t>(n * W, true);
    for (auto &d : P.dp.del) d = mem.alloc<uint32_t>(n * W, true);
    P.dp.lstamp = mem.alloc<uint32_t>(n, true);
    P.dp.inS = mem.alloc<uint32_t>(words, true);
    P.dp.rany = mem.alloc<uint32_t>(words, true);
    // tasks of a level: at most one per vertex plus one per kBfsTaskEdgesMin out-edges
    const size_t ntask = static_cast<size_t>(n + P.G->m / kBfsTaskEdgesMin + 1);
    for (auto &t : P.dp.T) t = mem.alloc<int4>(ntask);
    for (auto &v : P.dp.V) v = mem.alloc<int32_t>(n);
    P.has_bfs = true;
}

// An edge live in more simulations than this is merged as a dense edge (whole register rows), a sparser one as
// (target, simulation) pairs.
inline int32_t dense_min_for(int R) { return std::max(8, R / 8); }

// Eq. 4-5 for every edge and simulation, once per problem: the live masks (kept for the reachability searches)
// and from them the sparse pairs and the dense edge list of the sweeps.  Reads back the two totals to size the
// pair arrays (one stream synchronisation).
void sample_edges(im_ctx *ctx, Prob &P) {
    const int64_t m = P.G->m;
    const int W = P.prm.R / 32;
    P.smem = std::make_shared<DevMem>(ctx->stream);
    DevMem &mem = *P.smem;
    DevProb &d = P.dp;
    cudaStream_t s = ctx->stream;
    if (m >= (int64_t(1) << 32)) fail(IM_EINVAL, "graphs with 2^32 or more edges are not supported");
    d.dense_min = dense_min_for(P.prm.R);
    d.pull_sweeps = static_cast<uint32_t>(ctx->pull_sweeps);
    d.live = mem.alloc<uint32_t>(static_cast<size_t>(std::max<int64_t>(m, 1)) * W);
    int64_t *pofs = mem.alloc<int64_t>(m + 1, true);
    int64_t *dofs = mem.alloc<int64_t>(m + 1, true);
    d.pofs = pofs;
    d.dofs = dofs;
    UnitD *rdesc = mem.alloc<UnitD>(static_cast<size_t>(std::max<int64_t>(P.G->n, 1)));
    UnitD *tdesc = mem.alloc<UnitD>(static_cast<size_t>(std::max<int64_t>(P.G->n_tasks, 1)));
    d.rdesc = rdesc;
    d.tdesc = tdesc;
    if (m == 0) {
        d.pv = d.iu = d.iv = mem.alloc<int32_t>(1);
        d.stream_min = ~0ull;
        d.pj = d.ij = mem.alloc<uint16_t>(1);
        d.pq = mem.alloc<uint16_t>(1);
        d.dlist = d.ide = mem.alloc<uint32_t>(1);
        d.idu = mem.alloc<int32_t>(1);
        UnitD *vd0 = mem.alloc<UnitD>(static_cast<size_t>(std::max<int64_t>(P.G->n, 1)), true);
        d.vdesc = vd0;
        d.ipofs = pofs;
        d.idofs = dofs;
        // the first sweep of every diffusion visits every row through its descriptor (no pairs, no dense edges)
        launch_unit_desc(d, rdesc, tdesc, s);
        ctx->launches += 1;
        return;
    }
    int32_t *np = mem.alloc<int32_t>(m);
    int32_t *nd = mem.alloc<int32_t>(m);
    int64_t *bsums = mem.alloc<int64_t>(scan_block_count(m) + 1);
    launch_live_masks(d, np, nd, s);
    ctx->launches += 1 + launch_exclusive_scan(np, m, pofs, bsums, s);
    ctx->launches += launch_exclusive_scan(nd, m, dofs, bsums, s);
    // the same classes in in-CSR order (gathered from the out-edges'), for the pairs and dense edges of push sweeps
    int64_t *ipofs = mem.alloc<int64_t>(m + 1);
    int64_t *idofs = mem.alloc<int64_t>(m + 1);
    int32_t *inp = mem.alloc<int32_t>(m);
    int32_t *ind = mem.alloc<int32_t>(m);
    launch_inpair_counts(d, np, nd, inp, ind, s);
    ctx->launches += 1 + launch_exclusive_scan(inp, m, ipofs, bsums, s);
    ctx->launches += launch_exclusive_scan(ind, m, idofs, bsums, s);
    int64_t tot[2] = {0, 0};
    ck(cudaMemcpyAsync(&tot[0], pofs + m, sizeof(int64_t), cudaMemcpyDeviceToHost, s), "cudaMemcpyAsync");
    ck(cudaMemcpyAsync(&tot[1], dofs + m, sizeof(int64_t), cudaMemcpyDeviceToHost, s), "cudaMemcpyAsync");
    ck(cudaStreamSynchronize(s), "cudaStreamSynchronize");
    mem.release(inp);
    mem.release(ind);
    mem.release(np);
    mem.release(nd);
    mem.release(bsums);
    // targets and simulations of the out-pairs are read only by pulling sweeps after the first and by a rebuild
    // without the problem's own pair words (more than 2^32 pairs, no 32-bit in-pair -> out-pair index)
    const bool need_pv = ctx->pull_sweeps > 1 || tot[0] >= (int64_t(1) << 32);
    int32_t *pv = need_pv ? mem.alloc<int32_t>(static_cast<size_t>(std::max<int64_t>(tot[0], 1))) : nullptr;
    uint16_t *pj = need_pv ? mem.alloc<uint16_t>(static_cast<size_t>(std::max<int64_t>(tot[0], 1))) : nullptr;
    uint16_t *pq = mem.alloc<uint16_t>(static_cast<size_t>(std::max<int64_t>(tot[0], 1)));
    uint32_t *dlist = mem.alloc<uint32_t>(static_cast<size_t>(std::max<int64_t>(tot[1], 1)));
    launch_pair_fill(d, pv, pj, pq, dlist, s);
    launch_unit_desc(d, rdesc, tdesc, s);
    ctx->launches += 2;
    d.pv = pv;
    d.pj = pj;
    d.pq = pq;
    d.dlist = dlist;
    P.npairs = tot[0];
    P.ndense = tot[1];
    d.ipofs = ipofs;
    d.idofs = idofs;
    int32_t *iu = mem.alloc<int32_t>(static_cast<size_t>(std::max<int64_t>(tot[0], 1)));
    uint16_t *ij = mem.alloc<uint16_t>(static_cast<size_t>(std::max<int64_t>(tot[0], 1)));
    int32_t *iv = mem.alloc<int32_t>(static_cast<size_t>(std::max<int64_t>(tot[0], 1)));
    // in-pair -> out-pair index (32-bit), for residual blocking in a problem's copy of the pair words
    uint32_t *iop = tot[0] < (int64_t(1) << 32)
                        ? mem.alloc<uint32_t>(static_cast<size_t>(std::max<int64_t>(tot[0], 1)))
                        : nullptr;
    int32_t *idu = mem.alloc<int32_t>(static_cast<size_t>(std::max<int64_t>(tot[1], 1)));
    uint32_t *ide = mem.alloc<uint32_t>(static_cast<size_t>(std::max<int64_t>(tot[1], 1)));
    launch_inpair_fill(d, iu, ij, iop, iv, idu, ide, s);
    ctx->launches += 1;
    d.iop = iop;
    d.iv = iv;
    // push sweeps over a large L stream every in-pair (only without dense edges, which the stream leaves out)
    d.stream_min = (tot[1] == 0 && ctx->stream_push) ? static_cast<unsigned long long>(std::max<int64_t>(m / 2, 1))
                                                      : ~0ull;
    UnitD *vdesc = mem.alloc<UnitD>(static_cast<size_t>(std::max<int64_t>(P.G->n, 1)));
    launch_vertex_desc(d, vdesc, s);
    ctx->launches += 1;
    d.iu = iu;
    d.ij = ij;
    d.idu = idu;
    d.ide = ide;
    d.vdesc = vdesc;
}

// The descriptor fields sample_edges sets (everything the sampled graph consists of).
void copy_sample_fields(DevProb &d, const DevProb &src) {
    d.dense_min = src.dense_min;
    d.pull_sweeps = src.pull_sweeps;
    d.live = src.live;
    d.pofs = src.pofs;
    d.dofs = src.dofs;
    d.rdesc = src.rdesc;
    d.tdesc = src.tdesc;
    d.pv = src.pv;
    d.pj = src.pj;
    d.pq = src.pq;
    d.dlist = src.dlist;
    d.ipofs = src.ipofs;
    d.idofs = src.idofs;
    d.iu = src.iu;
    d.iv = src.iv;
    d.iop = src.iop;
    d.stream_min = src.stream_min;
    d.ij = src.ij;
    d.idu = src.idu;
    d.ide = src.ide;
    d.vdesc = src.vdesc;
}

// A problem built from a cached first diffusion: `sample` (whose sampled graph it shares) is any problem of the
// same graph, R, seed, eps_c and sweep limit; its own buffers are allocated and filled as make_prob would, except
// that the sampling is not redone.
std::unique_ptr<Prob> make_prob(im_ctx *ctx, std::shared_ptr<GraphDev> G, const im_params &prm, bool greedy,
                                const Prob *sample);

std::unique_ptr<Prob> make_prob(im_ctx *ctx, std::shared_ptr<GraphDev> G, const im_params &prm, bool greedy) {
    return make_prob(ctx, std::move(G), prm, greedy, nullptr);
}

std::unique_ptr<Prob> make_prob(im_ctx *ctx, std::shared_ptr<GraphDev> G, const im_params &prm, bool greedy,
                                const Prob *sample) {
    auto P = std::make_unique<Prob>();
    P->G = std::move(G);
    P->prm = prm;
    P->greedy = greedy;
    P->mem = std::make_unique<DevMem>(ctx->stream);
    DevMem &mem = *P->mem;
    const GraphDev &g = *P->G;
    const int64_t n = g.n;
    const int R = prm.R;
    DevProb &d = P->dp;
    d.n = n;
    d.m = g.m;
    d.xadj = g.xadj;
    d.adj = g.adj;
    d.xadj_in = g.xadj_in;
    d.adj_in = g.adj_in;
    d.ein = g.ein;
    d.heavy = g.heavy;
    d.task_off = g.task_off;
    d.task_row = g.task_row;
    d.light_list = g.light_list;
    d.hsmall = g.hsmall;
    d.hbig = g.hbig;
    d.n_tasks = g.n_tasks;
    d.n_light = g.n_light;
    d.n_hsmall = g.n_hsmall;
    d.n_hbig = g.n_hbig;
    d.model = g.model;
    d.R = R;
    d.W = R / 32;
    d.T_const = g.T_const;
    d.ic_ok = g.ic_ok;
    d.T_vert = g.T_vert;
    d.T_edge = g.T_edge;
    d.ok_edge = g.ok_edge;
    d.cas_limit = ctx->cas_limit;
    d.check_sums = ctx->check_sums ? 1u : 0u;
    d.undirected = g.undirected;
    d.literal = prm.blocking == IM_BLOCK_LITERAL ? 1 : 0;
    uint32_t *X = mem.alloc<uint32_t>(R);
    uint32_t *Y = mem.alloc<uint32_t>(R);
    launch_words(prm.seed, R, X, Y, ctx->stream);
    ctx->launches += 1;
    d.X = X;
    d.Y = Y;
    d.M0 = mem.alloc<uint8_t>(static_cast<size_t>(n) * R);
    d.M1 = mem.alloc<uint8_t>(static_cast<size_t>(n) * R);
    // the initial registers the first sweep of every diffusion reads (rebuilds zero the blocked ones in place)
    d.Mi = mem.alloc<uint8_t>(static_cast<size_t>(std::max<int64_t>(n, 1)) * R);
    if (n > 0) {
        launch_init_table(d, ctx->stream);
        ctx->launches += 1;
    }
    d.part = mem.alloc<uint8_t>(static_cast<size_t>(std::max<int64_t>(g.n_tasks, 1)) * R);
    d.part_any = mem.alloc<uint32_t>((g.n_tasks + 31) / 32 + 1, true);
    const int64_t words = (n + 31) / 32;
    d.Lb0 = mem.alloc<uint32_t>(words, true);
    d.Lb1 = mem.alloc<uint32_t>(words, true);
    d.dmask = mem.alloc<uint16_t>(static_cast<size_t>(n) * (R / 16));
    d.chg_list = mem.alloc<int32_t>(n);
    // chunks of changed vertices with more than kPushChunk in-edges: ceil(d / 1024) <= d / 512 for d > 1024
    d.chg_hc = mem.alloc<uint64_t>(static_cast<size_t>(g.m / 512 + 1));
    d.MS = mem.alloc<uint8_t>(R, true);
    const int64_t ms = prm.max_sweeps > 0 ? prm.max_sweeps : n + 2;
    d.max_sweeps = static_cast<uint32_t>(std::min<int64_t>(ms, 0x7FFFFFFF));
    // stop after the first sweep with |L'| <= eps_c * n: the largest integer count satisfying it
    const double thr = static_cast<double>(n) * prm.eps_c;
    d.stop_thr = static_cast<uint32_t>(std::floor(thr));
    P->flog_cap = 4096;
    d.flog_cap = static_cast<int32_t>(P->flog_cap);
    d.flog = mem.alloc<int64_t>(P->flog_cap, true);
    if (sample) {
        P->smem = sample->smem;
        copy_sample_fields(d, sample->dp);
        P->npairs = sample->npairs;
        P->ndense = sample->ndense;
    } else {
        sample_edges(ctx, *P);
    }
    // the autotuner's choice for this shape class, if any (the stream needs a sampled graph without dense edges)
    auto tn = ctx->tuned.find({R, degree_class(n, g.m)});
    if (tn != ctx->tuned.end()) {
        P->variant = tn->second.first;
        if (!tn->second.second) d.stream_min = ~0ull;
    }
    if (greedy) {
        alloc_bfs(*P);
        d.gst = mem.alloc<uint32_t>(static_cast<size_t>(n));
        // residual blocking applied at each rebuild to the initial registers and to a copy of the pair ranks (the
        // first sweep then tests nothing)
        if (prm.blocking == IM_BLOCK_RESIDUAL) {
            d.vis_done = mem.alloc<uint32_t>(static_cast<size_t>(n) * (R / 32), true);
            d.rnew = mem.alloc<uint32_t>(words, true);
            if (d.iop && P->npairs > 0) {
                d.pqb = mem.alloc<uint16_t>(static_cast<size_t>(P->npairs));
                ck(cudaMemcpyAsync(d.pqb, d.pq, static_cast<size_t>(P->npairs) * sizeof(uint16_t),
                                   cudaMemcpyDeviceToDevice, ctx->stream),
                   "copy pair words");
            }
        }
        d.step_seed = mem.alloc<uint32_t>(prm.K);
        d.step_gsum = mem.alloc<uint32_t>(prm.K);
    }
    P->seeds.reserve(greedy ? prm.K : 0);
    return P;
}

// ------------------------------------------------------------------------------------------------------------
// Engine

struct Engine {
    im_ctx *ctx;
    std::vector<Prob *> probs;
    DevProb *d_probs = nullptr;
    std::unique_ptr<DevMem> mem;

    DevCtr *d_ctrs = nullptr;
    bool soft_errors = false;  // record a failing problem and keep the others going instead of throwing

    // A slot table of `capacity` problems; the counters of all slots live in one array so one copy reads them back.
    Engine(im_ctx *c, size_t capacity) : ctx(c), probs(capacity, nullptr) {
        mem = std::make_unique<DevMem>(ctx->stream);
        d_probs = mem->alloc<DevProb>(capacity);
        d_ctrs = mem->alloc<DevCtr>(capacity, true);
        ensure_staging(capacity);
    }

    Engine(im_ctx *c, std::vector<Prob *> ps, const std::vector<DevCtr> *init_ctr = nullptr) : Engine(c, ps.size()) {
        for (size_t i = 0; i < ps.size(); ++i) attach(i, ps[i], init_ctr ? &(*init_ctr)[i] : nullptr);
        ck(cudaStreamSynchronize(ctx->stream), "sync");
    }

    // Puts problem p into slot i with the given (or zero) counters.
    void attach(size_t i, Prob *p, const DevCtr *c0) {
        probs[i] = p;
        p->dp.ctr = d_ctrs + i;
        p->d_ctr = d_ctrs + i;
        p->d_prob = d_probs + i;
        p->last = c0 ? *c0 : DevCtr{};
        ck(cudaMemcpyAsync(d_ctrs + i, &p->last, sizeof(DevCtr), cudaMemcpyHostToDevice, ctx->stream),
           "upload counters");
        ck(cudaMemcpyAsync(d_probs + i, &p->dp, sizeof(DevProb), cudaMemcpyHostToDevice, ctx->stream),
           "upload problem");
    }

    void detach(size_t i) { probs[i] = nullptr; }

    void ensure_staging(size_t np) {
        if (ctx->h_ctr_cap < np) {
            if (ctx->h_ctr) cudaFreeHost(ctx->h_ctr);
            ck(cudaMallocHost(&ctx->h_ctr, np * sizeof(DevCtr)), "cudaMallocHost");
            ctx->h_ctr_cap = np;
        }
        const size_t acap = 16 * np + 64;
        if (ctx->h_act_cap < acap) {
            if (ctx->h_act) cudaFreeHost(ctx->h_act);
            ck(cudaMallocHost(&ctx->h_act, acap * sizeof(int32_t)), "cudaMallocHost");
            ctx->h_act_cap = acap;
        }
        if (ctx->d_act_cap < acap) {
            if (ctx->d_act) cudaFree(ctx->d_act);
            ck(cudaMalloc(&ctx->d_act, acap * sizeof(int32_t)), "cudaMalloc");
            ctx->d_act_cap = acap;
        }
    }

    // Active lists of one tick live in one pinned array copied to the device once per tick.
    struct List {
        int off = 0, count = 0;
    };
    std::vector<int32_t> staging;

    List add_list(const std::vector<int32_t> &ids) {
        List l;
        l.off = static_cast<int>(staging.size());
        l.count = static_cast<int>(ids.size());
        staging.insert(staging.end(), ids.begin(), ids.end());
        return l;
    }

    const int32_t *dptr(const List &l) const { return ctx->d_act + l.off; }

    // One sweep's propagation launches (k_prop, then for a sweep that pulls into every row, k_combine for the split
    // rows), optionally between two events.
    void timed_prop(const std::vector<std::pair<int, List>> &byR, const std::vector<int> &variants, bool combine) {
        cudaStream_t s = ctx->stream;
        cudaEvent_t a = nullptr, b = nullptr;
        if (ctx->timing) {
            a = get_event();
            b = get_event();
            ck(cudaEventRecord(a, s), "event");
        }
        int64_t nl = 0;
        if (combine) {  // the first-sweep kernel, timed on its own as well
            cudaEvent_t fa = nullptr, fb = nullptr;
            if (ctx->timing) {
                fa = get_event();
                fb = get_event();
                ck(cudaEventRecord(fa, s), "event");
            }
            for (size_t i = 0; i < byR.size(); ++i)
                nl += launch_first(byR[i].first, d_probs, dptr(byR[i].second), byR[i].second.count, variants[i], s);
            if (ctx->timing) {
                ck(cudaEventRecord(fb, s), "event");
                ctx->first_ev.emplace_back(fa, fb);
            }
            ctx->first_launches += static_cast<int64_t>(byR.size());
        }
        for (size_t i = 0; i < byR.size(); ++i)
            nl += launch_prop(byR[i].first, d_probs, dptr(byR[i].second), byR[i].second.count, combine,
                              ctx->pull_sweeps > 1, s);
        if (combine) {
            for (auto &rl : byR) launch_combine(rl.first, d_probs, dptr(rl.second), rl.second.count, s);
            nl += 2 * static_cast<int64_t>(byR.size());  // the two combine kernels
        }
        if (ctx->timing) {
            ck(cudaEventRecord(b, s), "event");
            ctx->prop_ev.emplace_back(a, b);
        }
        ctx->launches += nl;
        ctx->prop_launches += static_cast<int64_t>(byR.size());
    }

    // Runs launch(); with timing enabled, brackets it with events counted for phase k.
    template <class F>
    void phase(int k, F &&launch) {
        if (!ctx->timing) {
            launch();
            return;
        }
        cudaEvent_t a = get_event(), b = get_event();
        ck(cudaEventRecord(a, ctx->stream), "event");
        launch();
        ck(cudaEventRecord(b, ctx->stream), "event");
        ctx->phase_ev[k].emplace_back(a, b);
    }

    cudaEvent_t get_event() {
        if (ctx->ev_free.empty()) {
            cudaEvent_t e;
            ck(cudaEventCreate(&e), "cudaEventCreate");
            return e;
        }
        cudaEvent_t e = ctx->ev_free.back();
        ctx->ev_free.pop_back();
        return e;
    }

    // chunk sweeps of the listed problems; with first_full, some of them start a diffusion (their sweep 0 pulls into
    // every row, later sweeps push and have no split rows to combine)
    void enqueue_sweeps(const std::vector<int32_t> &ids, int chunk, bool first_full) {
        if (ids.empty()) return;
        cudaStream_t s = ctx->stream;
        std::vector<std::pair<int, List>> byR;
        std::vector<int> variants;  // the first-sweep kernel's shape: that of the group's first problem
        for (int R : {64, 128, 256, 512, 1024}) {
            std::vector<int32_t> sub;
            for (int32_t i : ids)
                if (probs[i]->prm.R == R) sub.push_back(i);
            if (!sub.empty()) {
                byR.emplace_back(R, add_list(sub));
                variants.push_back(probs[sub[0]]->variant);
            }
        }
        const List all = add_list(ids);
        pending.push_back([this, byR, variants, all, chunk, first_full, s]() {
            phase(0, [&]() {
                for (int c = 0; c < chunk; ++c) {
                    timed_prop(byR, variants, first_full && c < ctx->pull_sweeps);
                    launch_frontier(d_probs, dptr(all), all.count, ctx->d_gbar, s);
                    ctx->launches += 1;
                }
            });
        });
    }

    void enqueue_bfs(const std::vector<int32_t> &ids, int chunk) {
        if (ids.empty()) return;
        std::vector<std::pair<int, List>> byR;
        for (int R : {64, 128, 256, 512, 1024}) {
            std::vector<int32_t> sub;
            for (int32_t i : ids)
                if (probs[i]->prm.R == R) sub.push_back(i);
            if (!sub.empty()) byR.emplace_back(R, add_list(sub));
        }
        cudaStream_t s = ctx->stream;
        pending.push_back([this, byR, chunk, s]() {
            phase(2, [&]() {
                // whole searches, one cooperative launch per R; the host reads the counters once they are done
                if (ctx->persistent) {
                    size_t done = 0;
                    for (auto &rl : byR) {
                        if (!launch_bfs_run(rl.first, d_probs, dptr(rl.second), rl.second.count, ctx->d_gbar,
                                            ctx->barrier_limit, s))
                            break;
                        ++done;
                    }
                    ctx->launches += static_cast<int64_t>(done);
                    if (done == byR.size()) return;
                    ctx->persistent = false;  // not available on this device: step the remaining levels
                }
                for (int c = 0; c < chunk; ++c) {
                    for (auto &rl : byR)
                        launch_bfs_level(rl.first, d_probs, dptr(rl.second), rl.second.count, ctx->d_gbar, s);
                    ctx->launches += static_cast<int64_t>(byR.size());
                }
            });
        });
    }

    // The argmax of a greedy step: the lazy scan (k_celf_*) for a step whose sketch was kept (the gains of its
    // previous scans still bound the current ones) and for the first step after a build, whose gains (M_S' is
    // empty) are the row sums the sweeps kept in gst; a full scan otherwise (an imported sketch, IM_CELF=0, or
    // IM_TEST_CHECK_SUMS, whose scan also checks those sums).
    void enqueue_scan(const std::vector<int32_t> &ids) {
        if (ids.empty()) return;
        cudaStream_t s = ctx->stream;
        std::vector<std::pair<int, List>> full, lazy;
        for (int R : {64, 128, 256, 512, 1024}) {
            std::vector<int32_t> fsub, lsub;
            for (int32_t i : ids) {
                if (probs[i]->prm.R != R) continue;
                (ctx->celf && (probs[i]->merge_pending || probs[i]->sums) ? lsub : fsub).push_back(i);
            }
            if (!fsub.empty()) full.emplace_back(R, add_list(fsub));
            if (!lsub.empty()) lazy.emplace_back(R, add_list(lsub));
        }
        // one choose launch per problem: each records its own step index
        std::vector<std::pair<List, int>> chooses;
        for (int32_t i : ids) chooses.emplace_back(add_list({i}), probs[i]->step);
        pending.push_back([this, full, lazy, chooses, s]() {
            int64_t nl = 0;
            phase(1, [&]() {
                for (auto &rl : full) launch_scan(rl.first, d_probs, dptr(rl.second), rl.second.count, s);
                for (auto &rl : lazy) nl += launch_celf(rl.first, d_probs, dptr(rl.second), rl.second.count, s);
                for (auto &c : chooses) launch_choose(d_probs, dptr(c.first), 1, c.second, s);
            });
            ctx->launches += nl + static_cast<int64_t>(full.size() + chooses.size());
        });
    }

    std::vector<std::function<void()>> pending;

    void flush() {
        if (!staging.empty()) {
            std::memcpy(ctx->h_act, staging.data(), staging.size() * sizeof(int32_t));
            ck(cudaMemcpyAsync(ctx->d_act, ctx->h_act, staging.size() * sizeof(int32_t), cudaMemcpyHostToDevice,
                               ctx->stream),
               "upload active lists");
        }
        for (auto &f : pending) f();
        pending.clear();
        staging.clear();
    }

    void read_counters() {
        cudaStream_t s = ctx->stream;
        ck(cudaMemcpyAsync(ctx->h_ctr, d_ctrs, probs.size() * sizeof(DevCtr), cudaMemcpyDeviceToHost, s),
           "read counters");
        ck(cudaStreamSynchronize(s), "sync");
        ck(cudaGetLastError(), "kernel launch");
        for (size_t i = 0; i < probs.size(); ++i)
            if (probs[i]) probs[i]->last = ctx->h_ctr[i];
    }

    // Algorithm 1's error check after step k of problem P (host, double, from device integers).
    void decide(Prob &P) {
        const DevCtr &C = P.last;
        const int R = P.prm.R;
        const double e = std::exp2(static_cast<double>(C.gsum) / static_cast<double>(R)) / kPhi;
        const double sigma = static_cast<double>(C.reached) / static_cast<double>(R);
        const double delta = sigma - P.varsigma;
        const double err_l = (delta == 0.0) ? INFINITY : std::fabs((e - delta) / delta);
        const double err_g = std::fabs((e - delta) / sigma);
        P.seeds.push_back(static_cast<int32_t>(C.s));
        P.sigma.push_back(sigma);
        P.est.push_back(e);
        P.gsum.push_back(C.gsum);
        const int k = P.step;
        P.step += 1;
        if (err_l < P.prm.eps_l || err_g < P.prm.eps_g) {
            P.rebuilt.push_back(0);
            P.merge_pending = true;
            P.phase = (P.step == P.prm.K) ? Prob::kDone : Prob::kScan;
        } else {
            P.rebuilt.push_back(1);
            P.varsigma = sigma;
            P.merge_pending = false;
            P.phase = (k + 1 < P.prm.K) ? Prob::kInit : Prob::kDone;
        }
    }

    void problem_error(Prob &P, im_status st, const char *msg) {
        if (!soft_errors) fail(st, msg);
        P.status = st;
        P.error = msg;
        P.phase = Prob::kDone;
    }

    // One engine tick: every active problem advances by one phase step (one launch per phase for all of them),
    // then the counters are read back once.  Returns false when no problem had work.
    bool tick() {
        cudaStream_t s = ctx->stream;
        std::vector<int32_t> init, sweep, scan, bfs, merge;
        bool any = false;
        for (size_t i = 0; i < probs.size(); ++i) {
            if (!probs[i]) continue;
            Prob &P = *probs[i];
            switch (P.phase) {
                case Prob::kInit: init.push_back(i); sweep.push_back(i); any = true; break;
                case Prob::kSweep: sweep.push_back(i); any = true; break;
                case Prob::kScan:
                    if (P.merge_pending) merge.push_back(i);
                    scan.push_back(i);
                    bfs.push_back(i);
                    P.levels_at_start = P.last.levels_total;  // this step's search starts in this tick
                    any = true;
                    break;
                case Prob::kBfs: bfs.push_back(i); any = true; break;
                default: break;
            }
        }
        if (!any) return false;
        if (!merge.empty()) {
            const List l = add_list(merge);
            pending.push_back([this, l, s]() {
                phase(3, [&]() { launch_merge(d_probs, dptr(l), l.count, s); });
                ctx->launches += 1;
            });
        }
        if (!init.empty()) {
            const List l = add_list(init);
            pending.push_back([this, l, s]() {
                int nl = 0;
                phase(3, [&]() { nl = launch_init(d_probs, dptr(l), l.count, s); });
                ctx->launches += nl;
            });
        }
        enqueue_sweeps(sweep, ctx->sweep_chunk, !init.empty());
        enqueue_scan(scan);
        // a search takes about as many levels as the problem's previous one (seeds of one selection reach alike), so
        // a tick enqueues that many and two more, up to level_chunk; a longer search takes another tick
        int lchunk = 0;
        for (int32_t i : bfs) {
            const Prob &P = *probs[i];
            lchunk = std::max(lchunk, P.last_search_levels ? static_cast<int>(P.last_search_levels) + 2 : ctx->level_chunk);
        }
        enqueue_bfs(bfs, std::min(std::max(lchunk, 1), ctx->level_chunk));
        flush();
        read_counters();
        for (int32_t i : init) {
            probs[i]->phase = Prob::kSweep;
            probs[i]->builds += 1;
            probs[i]->sums = probs[i]->dp.gst != nullptr && !ctx->check_sums;
        }
        for (int32_t i : merge) probs[i]->merge_pending = false;
        for (int32_t i : scan) probs[i]->phase = Prob::kBfs;
        for (size_t i = 0; i < probs.size(); ++i) {
            if (!probs[i]) continue;
            Prob &P = *probs[i];
            if (P.phase == Prob::kDone) continue;
            if (P.last.fault) {
                problem_error(P, IM_ECUDA, (P.last.fault & 1u)   ? "a bulk copy into shared memory did not complete"
                                           : (P.last.fault & 2u) ? "a register update did not settle"
                                           : (P.last.fault & 4u) ? "a grid barrier was not reached in time"
                                           : (P.last.fault & 16u) ? "a kept register row sum disagreed with the row"
                                                                 : "a pulling sweep was launched as a push sweep");
            } else if (P.phase == Prob::kSweep && P.last.done) {
                if (P.last.timeout)
                    problem_error(P, IM_ETIMEOUT, "diffusion exceeded max_sweeps");
                else
                    P.phase = P.greedy ? Prob::kScan : Prob::kDone;
            } else if (P.phase == Prob::kBfs && P.last.bdone) {
                P.last_search_levels = static_cast<uint32_t>(P.last.levels_total - P.levels_at_start);
                if (P.last.btimeout)
                    problem_error(P, IM_ETIMEOUT, "reachability search exceeded max_sweeps levels");
                else
                    decide(P);
            }
        }
        return true;
    }

    void run() {
        while (tick()) {
        }
    }
};

void set_err(im_ctx *ctx, const std::string &m) {
    if (ctx) ctx->err = m;
}

template <class F>
im_status guarded(im_ctx *ctx, F &&f) {
    try {
        f();
        if (ctx) ctx->err.clear();
        return IM_OK;
    } catch (const ImError &e) {
        set_err(ctx, e.msg);
        return e.status;
    } catch (const CudaError &e) {
        set_err(ctx, std::string(e.what) + ": " + cudaGetErrorString(e.code));
        cudaGetLastError();
        return IM_ECUDA;
    } catch (const std::bad_alloc &) {
        set_err(ctx, "host allocation failed");
        return IM_ENOMEM;
    }
}

void begin_call(im_ctx *ctx) {
    ck(cudaSetDevice(ctx->device), "cudaSetDevice");
    ctx->launches = 0;
    ctx->prop_launches = 0;
    for (auto &pe : ctx->prop_ev) {
        ctx->ev_free.push_back(pe.first);
        ctx->ev_free.push_back(pe.second);
    }
    ctx->prop_ev.clear();
    for (auto &pe : ctx->first_ev) {
        ctx->ev_free.push_back(pe.first);
        ctx->ev_free.push_back(pe.second);
    }
    ctx->first_ev.clear();
    ctx->first_launches = 0;
    for (auto &v : ctx->phase_ev) {
        for (auto &pe : v) {
            ctx->ev_free.push_back(pe.first);
            ctx->ev_free.push_back(pe.second);
        }
        v.clear();
    }
}

void end_call(im_ctx *ctx, const std::vector<Prob *> &probs, cudaEvent_t t0, cudaEvent_t t1) {
    im_stats st{};
    for (Prob *P : probs) {
        st.visits += P->last.visits;
        st.prop_bytes += P->last.bytes;
        st.live_pairs += P->last.pairs;
        st.first_bytes += P->last.first_bytes;
        st.sweeps += static_cast<int64_t>(P->last.sweeps_total);
        st.bfs_levels += static_cast<int64_t>(P->last.levels_total);
        st.builds += P->builds;
    }
    st.kernel_launches = ctx->launches;
    st.prop_launches = ctx->prop_launches;
    float ms = 0.f;
    ck(cudaEventElapsedTime(&ms, t0, t1), "elapsed");
    st.total_ms = ms;
    double pm = 0.0;
    for (auto &pe : ctx->prop_ev) {
        float x = 0.f;
        ck(cudaEventElapsedTime(&x, pe.first, pe.second), "elapsed");
        pm += x;
    }
    st.prop_ms = pm;
    double fm = 0.0;
    for (auto &pe : ctx->first_ev) {
        float x = 0.f;
        ck(cudaEventElapsedTime(&x, pe.first, pe.second), "elapsed");
        fm += x;
    }
    st.first_ms = fm;
    st.first_launches = ctx->first_launches;
    double ph[4] = {0, 0, 0, 0};
    for (int k = 0; k < 4; ++k)
        for (auto &pe : ctx->phase_ev[k]) {
            float x = 0.f;
            ck(cudaEventElapsedTime(&x, pe.first, pe.second), "elapsed");
            ph[k] += x;
        }
    st.sweep_ms = ph[0];
    st.scan_ms = ph[1];
    st.bfs_ms = ph[2];
    st.init_ms = ph[3];
    ctx->stats = st;
}

struct CallTimer {
    im_ctx *ctx;
    cudaEvent_t a, b;
    explicit CallTimer(im_ctx *c) : ctx(c) {
        ck(cudaEventCreate(&a), "event");
        ck(cudaEventCreate(&b), "event");
        ck(cudaEventRecord(a, ctx->stream), "event");
    }
    void stop() {
        ck(cudaEventRecord(b, ctx->stream), "event");
        ck(cudaEventSynchronize(b), "event");
    }
    ~CallTimer() {
        cudaEventDestroy(a);
        cudaEventDestroy(b);
    }
};

}  // namespace

struct im_sketch {
    std::unique_ptr<Prob> P;
    im_ctx *ctx = nullptr;
    double p = 0.0;  // the graph's p (recorded in exports)
};

// Context accessors for the allocation-free entry point (im_static.cu).
namespace imh {
cudaStream_t ctx_stream(const im_ctx *ctx) { return ctx->stream; }
int ctx_device(const im_ctx *ctx) { return ctx->device; }
void ctx_set_error(im_ctx *ctx, const char *msg) { ctx->err = msg; }
}  // namespace imh

extern "C" {

im_status im_ctx_create(int device, void *cuda_stream, im_ctx **out) {
    if (!out) return IM_EINVAL;
    *out = nullptr;
    auto *ctx = new (std::nothrow) im_ctx();
    if (!ctx) return IM_ENOMEM;
    int count = 0;
    cudaError_t e = cudaGetDeviceCount(&count);
    if (e != cudaSuccess || device < 0 || device >= count) {
        cudaGetLastError();
        delete ctx;
        return IM_ECUDA;
    }
    ctx->device = device;
    if (cudaSetDevice(device) != cudaSuccess || configure(device) != cudaSuccess) {
        cudaGetLastError();
        delete ctx;
        return IM_ECUDA;
    }
    // keep freed device memory reserved in the pool so repeated calls do not pay for fresh allocations
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    if (cuda_stream) {
        ctx->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
        if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            delete ctx;
            return IM_ECUDA;
        }
        ctx->own_stream = true;
    }
    if (const char *v = std::getenv("IM_SWEEP_CHUNK")) ctx->sweep_chunk = std::max(1, std::atoi(v));
    if (const char *v = std::getenv("IM_LEVEL_CHUNK")) ctx->level_chunk = std::max(1, std::atoi(v));
    if (const char *v = std::getenv("IM_PERSISTENT")) ctx->persistent = std::atoi(v) != 0;
    if (const char *v = std::getenv("IM_PULL_SWEEPS")) ctx->pull_sweeps = std::max(1, std::min(8, std::atoi(v)));
    if (const char *v = std::getenv("IM_CELF")) ctx->celf = std::atoi(v) != 0;
    if (const char *v = std::getenv("IM_TEST_CHECK_SUMS")) ctx->check_sums = std::atoi(v) != 0;
    if (const char *v = std::getenv("IM_STREAM")) ctx->stream_push = std::atoi(v) != 0;
    if (const char *v = std::getenv("IM_TEST_CAS_LIMIT")) ctx->cas_limit = static_cast<uint32_t>(std::atol(v));
    if (const char *v = std::getenv("IM_TEST_BARRIER_LIMIT"))
        ctx->barrier_limit = static_cast<uint32_t>(std::atol(v));
    // every pulling sweep of a diffusion falls in the tick that starts it (split rows are combined only there)
    ctx->pull_sweeps = std::min(ctx->pull_sweeps, ctx->sweep_chunk);
    if (cudaMalloc(&ctx->d_gbar, sizeof(GridBar)) != cudaSuccess ||
        cudaMemset(ctx->d_gbar, 0, sizeof(GridBar)) != cudaSuccess) {
        cudaGetLastError();
        if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
        delete ctx;
        return IM_ECUDA;
    }
    *out = ctx;
    return IM_OK;
}

im_status im_ctx_destroy(im_ctx *ctx) {
    if (!ctx) return IM_EINVAL;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    for (auto &pe : ctx->prop_ev) {
        cudaEventDestroy(pe.first);
        cudaEventDestroy(pe.second);
    }
    for (auto &v : ctx->phase_ev)
        for (auto &pe : v) {
            cudaEventDestroy(pe.first);
            cudaEventDestroy(pe.second);
        }
    for (cudaEvent_t e : ctx->ev_free) cudaEventDestroy(e);
    if (ctx->h_ctr) cudaFreeHost(ctx->h_ctr);
    if (ctx->h_act) cudaFreeHost(ctx->h_act);
    if (ctx->d_act) cudaFree(ctx->d_act);
    if (ctx->d_gbar) cudaFree(ctx->d_gbar);
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
    return IM_OK;
}

const char *im_last_error(const im_ctx *ctx) { return ctx ? ctx->err.c_str() : "context is NULL"; }

im_status im_ctx_set_timing(im_ctx *ctx, int enable) {
    if (!ctx) return IM_EINVAL;
    ctx->timing = enable != 0;
    return IM_OK;
}

im_status im_ctx_stats(const im_ctx *ctx, im_stats *out) {
    if (!ctx || !out) return IM_EINVAL;
    *out = ctx->stats;
    return IM_OK;
}

im_status im_build_sketches(im_ctx *ctx, const im_graph *graph, const im_params *params, im_sketch **out) {
    if (!ctx) return IM_EINVAL;
    return guarded(ctx, [&]() {
        if (!out) fail(IM_EINVAL, "out is NULL");
        begin_call(ctx);
        CallTimer tm(ctx);
        if (!graph) fail(IM_EINVAL, "graph is NULL");
        check_params(params, graph->n, false);
        auto G = prepare_graph(ctx, graph);
        auto sk = std::make_unique<im_sketch>();
        sk->ctx = ctx;
        sk->p = graph->p;
        sk->P = make_prob(ctx, G, *params, false);
        Engine eng(ctx, {sk->P.get()});
        eng.run();
        tm.stop();
        end_call(ctx, {sk->P.get()}, tm.a, tm.b);
        *out = sk.release();
    });
}

// ------------------------------------------------------------------------------------------------------------
// Influence scoring by plain sample-then-diffuse Monte Carlo (Section 4's separate influence oracle), on the
// device: live masks drawn with mt19937 streams (k_mc_live), then the seed set's reachability search over them
// with the search kernels of the greedy loop, in batches of up to 1024 samples.

// A search-only problem of R samples on graph G: thresholds, live masks and search buffers, nothing of a sketch.
std::unique_ptr<Prob> make_mc_prob(im_ctx *ctx, std::shared_ptr<GraphDev> G, int R) {
    auto P = std::make_unique<Prob>();
    P->G = std::move(G);
    P->prm.R = R;
    P->prm.K = 1;
    P->mem = std::make_unique<DevMem>(ctx->stream);
    const GraphDev &g = *P->G;
    DevProb &d = P->dp;
    d.n = g.n;
    d.m = g.m;
    d.xadj = g.xadj;
    d.adj = g.adj;
    d.model = g.model;
    d.R = R;
    d.W = R / 32;
    d.T_const = g.T_const;
    d.ic_ok = g.ic_ok;
    d.T_vert = g.T_vert;
    d.T_edge = g.T_edge;
    d.ok_edge = g.ok_edge;
    d.live = P->mem->alloc<uint32_t>(static_cast<size_t>(std::max<int64_t>(g.m, 1)) * d.W);
    d.max_sweeps = static_cast<uint32_t>(std::min<int64_t>(g.n + 2, 0x7FFFFFFF));
    alloc_bfs(*P);
    return P;
}

im_status im_influence_mc(im_ctx *ctx, const im_graph *graph, const int32_t *seeds, int32_t k, int64_t nsamples,
                          uint64_t seed, double *sigma_out, uint64_t *reach_out) {
    if (!ctx) return IM_EINVAL;
    return guarded(ctx, [&]() {
        if (!graph || !seeds || !sigma_out) fail(IM_EINVAL, "graph / seeds / sigma_out is NULL");
        if (k < 1) fail(IM_EINVAL, "k must be >= 1");
        if (graph->undirected) fail(IM_EINVAL, "the Monte-Carlo scorer draws per directed edge: no undirected input");
        if (nsamples < 64 || nsamples % 64 != 0 || nsamples > (int64_t{1} << 24))
            fail(IM_EINVAL, "nsamples must be a multiple of 64 in [64, 2^24]");
        for (int32_t i = 0; i < k; ++i)
            if (seeds[i] < 0 || seeds[i] >= graph->n) fail(IM_EINVAL, "seed id outside [0, n)");
        begin_call(ctx);
        CallTimer tm(ctx);
        auto G = prepare_graph(ctx, graph);
        cudaStream_t s = ctx->stream;
        DevMem tmp(s);
        int32_t *d_seeds = tmp.alloc<int32_t>(k);
        ck(cudaMemcpyAsync(d_seeds, seeds, k * sizeof(int32_t), cudaMemcpyHostToDevice, s), "copy seeds");
        unsigned long long *d_counts = tmp.alloc<unsigned long long>(1024);
        std::vector<unsigned long long> h_counts(1024);
        const int64_t n = G->n;
        const int64_t nchunks = (G->m + kMcChunk - 1) / kMcChunk;
        std::unique_ptr<Prob> full, last;  // the 1024-sample problem reused by every full batch, the remainder's
        std::vector<Prob *> used;
        std::vector<unsigned long long> reach(static_cast<size_t>(nsamples));  // written out only on success
        unsigned long long total = 0;
        for (int64_t s0 = 0; s0 < nsamples;) {
            const int64_t left = nsamples - s0;
            int R = 1024;
            while (R > 64 && R / 2 >= left) R /= 2;
            std::unique_ptr<Prob> &slot = R == 1024 ? full : last;
            if (!slot) {
                slot = make_mc_prob(ctx, G, R);
                used.push_back(slot.get());
            }
            Prob &P = *slot;
            const int W = R / 32;
            const int64_t nb = std::min<int64_t>(left, R);
            for (uint32_t *d : P.dp.del) ck(cudaMemsetAsync(d, 0, static_cast<size_t>(n) * W * 4, s), "memset");
            ck(cudaMemsetAsync(P.dp.vis, 0, static_cast<size_t>(n) * W * 4, s), "memset");
            ck(cudaMemsetAsync(P.dp.lstamp, 0, static_cast<size_t>(n) * 4, s), "memset");
            ck(cudaMemsetAsync(P.dp.inS, 0, ((n + 31) / 32) * 4, s), "memset");
            ck(cudaMemsetAsync(d_counts, 0, R * sizeof(unsigned long long), s), "memset");
            std::vector<DevCtr> c0(1);
            c0[0].levels_total = P.last.levels_total;  // this problem's levels so far, for the call's statistics
            Engine eng(ctx, {&P}, &c0);
            eng.phase(3, [&]() { launch_mc_live(R, eng.d_probs, seed, s0, nb, nchunks, s); });
            launch_seed_set(eng.d_probs, d_seeds, k, W, s);
            ctx->launches += 2;
            P.phase = Prob::kBfs;
            for (;;) {
                eng.enqueue_bfs({0}, ctx->level_chunk);
                eng.flush();
                eng.read_counters();
                if (P.last.bdone || P.last.fault) break;
            }
            P.phase = Prob::kDone;
            if (P.last.fault) fail(IM_ECUDA, "a grid barrier was not reached in time");
            if (P.last.btimeout) fail(IM_ETIMEOUT, "reachability search exceeded its level limit");
            launch_sample_counts(R, eng.d_probs, d_counts, s);
            ctx->launches += 1;
            ck(cudaMemcpyAsync(h_counts.data(), d_counts, R * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s),
               "read counts");
            ck(cudaStreamSynchronize(s), "sync");
            for (int64_t j = 0; j < nb; ++j) {
                total += h_counts[j];
                reach[static_cast<size_t>(s0 + j)] = h_counts[j];
            }
            s0 += nb;
        }
        tm.stop();
        end_call(ctx, used, tm.a, tm.b);
        *sigma_out = static_cast<double>(total) / static_cast<double>(nsamples);
        if (reach_out) std::copy(reach.begin(), reach.end(), reach_out);
    });
}

im_status im_sketch_destroy(im_sketch *sketch) {
    if (!sketch) return IM_EINVAL;
    cudaSetDevice(sketch->ctx->device);
    cudaStreamSynchronize(sketch->ctx->stream);
    delete sketch;
    return IM_OK;
}

im_status im_sketch_registers(im_ctx *ctx, const im_sketch *sketch, uint8_t *host_out) {
    if (!ctx) return IM_EINVAL;
    return guarded(ctx, [&]() {
        if (!sketch || !host_out) fail(IM_EINVAL, "sketch / host_out is NULL");
        begin_call(ctx);
        const Prob &P = *sketch->P;
        const uint8_t *M = P.last.res_par ? P.dp.M1 : P.dp.M0;
        ck(cudaMemcpyAsync(host_out, M, static_cast<size_t>(P.G->n) * P.prm.R, cudaMemcpyDeviceToHost, ctx->stream),
           "copy registers");
        ck(cudaStreamSynchronize(ctx->stream), "sync");
    });
}

im_status im_sketch_info(im_ctx *ctx, const im_sketch *sketch, int64_t *sweeps, uint64_t *visits,
                         int64_t *frontier_log, int64_t log_cap) {
    if (!ctx) return IM_EINVAL;
    return guarded(ctx, [&]() {
        if (!sketch) fail(IM_EINVAL, "sketch is NULL");
        const Prob &P = *sketch->P;
        if (sweeps) *sweeps = static_cast<int64_t>(P.last.sweeps_total);
        if (visits) *visits = P.last.visits;
        if (frontier_log && log_cap > 0) {
            const int64_t k = std::min<int64_t>({log_cap, P.flog_cap, static_cast<int64_t>(P.last.sweeps_total)});
            if (k > 0) {
                ck(cudaMemcpyAsync(frontier_log, P.dp.flog, k * sizeof(int64_t), cudaMemcpyDeviceToHost, ctx->stream),
                   "copy log");
                ck(cudaStreamSynchronize(ctx->stream), "sync");
            }
        }
    });
}

im_status im_estimate(im_ctx *ctx, const im_sketch *sketch, const int32_t *seeds, int32_t k, double *est_out,
                      double *sigma_out) {
    if (!ctx) return IM_EINVAL;
    return guarded(ctx, [&]() {
        if (!sketch || !seeds || !est_out) fail(IM_EINVAL, "sketch / seeds / est_out is NULL");
        if (k < 1) fail(IM_EINVAL, "k must be >= 1");
        Prob &P = *sketch->P;
        for (int32_t i = 0; i < k; ++i)
            if (seeds[i] < 0 || seeds[i] >= P.G->n) fail(IM_EINVAL, "seed id outside [0, n)");
        begin_call(ctx);
        CallTimer tm(ctx);
        cudaStream_t s = ctx->stream;
        DevMem tmp(s);
        int32_t *d_seeds = tmp.alloc<int32_t>(k);
        ck(cudaMemcpyAsync(d_seeds, seeds, k * sizeof(int32_t), cudaMemcpyHostToDevice, s), "copy seeds");
        unsigned long long *d_g = tmp.alloc<unsigned long long>(1, true);
        if (sigma_out && !P.has_bfs) alloc_bfs(P);
        std::vector<DevCtr> c0(1);
        c0[0].res_par = P.last.res_par;
        c0[0].sweeps_total = P.last.sweeps_total;
        c0[0].visits = P.last.visits;
        c0[0].bytes = P.last.bytes;
        Engine eng(ctx, {&P}, &c0);
        launch_estimate(eng.d_probs, d_seeds, k, d_g, s);
        ctx->launches += 1;
        unsigned long long g = 0;
        ck(cudaMemcpyAsync(&g, d_g, sizeof(g), cudaMemcpyDeviceToHost, s), "read sum");
        ck(cudaStreamSynchronize(s), "sync");
        const double e = std::exp2(static_cast<double>(g) / static_cast<double>(P.prm.R)) / kPhi;
        double sigma = 0.0;
        const DevCtr keep = P.last;
        if (sigma_out) {
            const int64_t n = P.G->n;
            const int W = P.prm.R / 32;
            ck(cudaMemsetAsync(P.dp.vis, 0, static_cast<size_t>(n) * W * 4, s), "memset");
            for (uint32_t *d : P.dp.del) ck(cudaMemsetAsync(d, 0, static_cast<size_t>(n) * W * 4, s), "memset");
            ck(cudaMemsetAsync(P.dp.lstamp, 0, static_cast<size_t>(n) * 4, s), "memset");
            ck(cudaMemsetAsync(P.dp.inS, 0, ((n + 31) / 32) * 4, s), "memset");
            launch_seed_set(eng.d_probs, d_seeds, k, W, s);
            ctx->launches += 1;
            P.phase = Prob::kBfs;
            for (;;) {
                eng.enqueue_bfs({0}, ctx->level_chunk);
                eng.flush();
                eng.read_counters();
                if (P.last.bdone) break;
            }
            P.phase = Prob::kDone;
            if (P.last.btimeout) fail(IM_ETIMEOUT, "reachability search exceeded max_sweeps levels");
            sigma = static_cast<double>(P.last.reached) / static_cast<double>(P.prm.R);
        }
        P.last = keep;
        tm.stop();
        end_call(ctx, {&P}, tm.a, tm.b);
        *est_out = e;
        if (sigma_out) *sigma_out = sigma;
    });
}

// ------------------------------------------------------------------------------------------------------------
// Serving: a resident pool of prepared graphs, a queue of seed-selection queries, admission by an HBM budget and a
// slot limit, and continuous batching (every engine tick launches each phase once for all admitted queries; a
// query leaves the batch, and frees its memory, as soon as it is done).

namespace {

// Device bytes make_prob + alloc_bfs allocate for a greedy query (each allocation rounded up to 256 bytes).
uint64_t query_footprint(const GraphDev &g, const im_params &prm) {
    auto r = [](uint64_t b) { return (std::max<uint64_t>(b, 16) + 255) / 256 * 256; };
    const uint64_t n = static_cast<uint64_t>(g.n), R = static_cast<uint64_t>(prm.R), W = R / 32;
    const uint64_t words = (n + 31) / 32, nt = std::max<int64_t>(g.n_tasks, 1);
    uint64_t b = 0;
    b += r(4 * R) * 2;                                       // X, Y
    b += r(n * R) * 3;                                       // register buffers, initial registers
    b += r(nt * R) + r(4 * (static_cast<uint64_t>(g.n_tasks) / 32 + 1));  // partial rows, their bits
    b += r(4 * words) * 2;                                   // L bits
    b += r(n * R / 8);                                       // changed-register masks of the push sweeps
    b += r(4 * n) + r(8 * (static_cast<uint64_t>(g.m) / 512 + 1));  // changed lists
    b += r(R) + r(8 * 4096);                                 // M_S', frontier log
    b += r(4 * n * W) * 4 + r(4 * words) * 2 + r(4 * n) * 4;  // reach and delta bits, seed-set and reached-vertex
                                                                 // bits, stamps, frontiers
    b += r(4 * n);                                           // bounds of the lazy argmax
    b += r(4 * n * W) + r(4 * words);                        // blocked bits applied to the pair words, new ones
    b += r(sizeof(int4) * (n + static_cast<uint64_t>(g.m) / kBfsTaskEdgesMin + 1)) * 2;  // search tasks
    const uint64_t m1 = std::max<uint64_t>(static_cast<uint64_t>(g.m), 1);
    b += r(4 * W * m1);                                      // live-simulation masks of the edges
    b += r(8 * (m1 + 1)) * 4;                                // pair and dense-edge offsets, out- and in-CSR order
    b += r(sizeof(UnitD) * std::max<uint64_t>(n, 1)) + r(sizeof(UnitD) * nt);  // sweep-unit descriptors
    // pairs: at most dense_min per edge, dense edges 4 bytes; the per-edge counts (out- and in-CSR order) and the
    // scan sums of the preparation are freed before the pairs are allocated, and are smaller
    const uint64_t pmax = m1 * static_cast<uint64_t>(dense_min_for(prm.R));
    b += (r(4 * pmax) + r(2 * pmax)) * 2 + r(2 * pmax) * 2 + r(4 * pmax) * 2 + r(4 * m1) * 3;  // pairs both ways
        // with the out-pairs' first-sweep words (and the query's copy), the in-pairs' targets and out-pair indices,
        // dense edges
    b += r(sizeof(UnitD) * std::max<uint64_t>(n, 1));       // push-unit descriptors
    b += r(4 * static_cast<uint64_t>(prm.K)) * 2;            // step records
    return b;
}

}  // namespace

struct im_server {
    im_ctx *ctx = nullptr;
    uint64_t budget = 0, used = 0;
    std::vector<std::shared_ptr<GraphDev>> graphs;
    std::unique_ptr<Engine> eng;
    struct Query {
        int32_t gid = 0;
        im_params prm{};
        std::unique_ptr<Prob> P;
        int64_t slot = -1;
        uint64_t bytes = 0;
        int state = 0;  // 0 queued, 1 running, 2 done, 3 cancelled, 4 failed
        std::vector<int32_t> seeds;
        double sigma = 0.0;
        int32_t rebuilds = 0;
        im_status status = IM_OK;
        std::string error;
        bool fill = false;  // keep this query's first diffusion for later queries with the same one
    };
    // First diffusions by (graph, R, seed, eps_c, sweep limit): the sampled graph and the registers the
    // diffusion reached, for later queries that would compute exactly the same (their K and error thresholds only
    // act after it).  Held within the budget; the least recently used go first when a query needs the room.
    struct Build {
        Prob sample;                   // the shared sampled graph (smem, the sampling fields of dp, pair counts)
        std::unique_ptr<DevMem> rmem;  // the registers
        uint8_t *M = nullptr;
        DevCtr ctr{};                  // the counters right after the diffusion
        uint64_t bytes = 0;
        uint64_t last_use = 0;
    };
    using BuildKey = std::tuple<int32_t, int32_t, uint64_t, double, int64_t>;
    std::map<BuildKey, Build> builds;
    uint64_t clock = 0, build_hits = 0;
    std::map<uint64_t, Query> q;
    std::deque<uint64_t> queue;
    std::vector<size_t> free_slots;
    std::vector<uint64_t> slot_ticket;
    uint64_t next = 1;
};

namespace {

im_server::BuildKey build_key(const im_server::Query &Q) {
    return {Q.gid, Q.prm.R, Q.prm.seed, Q.prm.eps_c, Q.prm.max_sweeps};
}

// Drops the least recently used kept diffusion other than `spare` (nullable); false if there is none.  The memory
// of a sampled graph that a running query still shares stays allocated until that query ends, inside its own
// reservation.
bool evict_build(im_server *srv, const im_server::BuildKey *spare) {
    auto lru = srv->builds.end();
    for (auto it = srv->builds.begin(); it != srv->builds.end(); ++it)
        if ((!spare || it->first != *spare) && (lru == srv->builds.end() || it->second.last_use < lru->second.last_use))
            lru = it;
    if (lru == srv->builds.end()) return false;
    srv->used -= lru->second.bytes;
    srv->builds.erase(lru);
    return true;
}

// Keeps query Q's first diffusion (just finished: its registers are the result buffer) if the budget has room.
void keep_build(im_server *srv, im_server::Query &Q) {
    Prob &P = *Q.P;
    const GraphDev &g = *srv->graphs[static_cast<size_t>(Q.gid)];
    const size_t regs = static_cast<size_t>(g.n) * static_cast<size_t>(Q.prm.R);
    const uint64_t bytes = P.smem->bytes + (std::max<size_t>(regs, 16) + 255) / 256 * 256;
    if (srv->used + bytes > srv->budget) return;
    im_server::Build b;
    b.sample.smem = P.smem;
    copy_sample_fields(b.sample.dp, P.dp);
    b.sample.npairs = P.npairs;
    b.sample.ndense = P.ndense;
    b.rmem = std::make_unique<DevMem>(srv->ctx->stream);
    try {
        b.M = b.rmem->alloc<uint8_t>(regs);
    } catch (const ImError &) {  // keeping is optional: without the room the queries just run the diffusion
        return;
    }
    ck(cudaMemcpyAsync(b.M, P.last.res_par ? P.dp.M1 : P.dp.M0, regs, cudaMemcpyDeviceToDevice, srv->ctx->stream),
       "keep registers");
    b.ctr = P.last;
    b.bytes = bytes;
    b.last_use = ++srv->clock;
    srv->used += b.bytes;
    srv->builds[build_key(Q)] = std::move(b);
}

void server_release(im_server *srv, im_server::Query &Q) {
    if (Q.slot >= 0) {
        srv->eng->detach(static_cast<size_t>(Q.slot));
        srv->free_slots.push_back(static_cast<size_t>(Q.slot));
        srv->slot_ticket[static_cast<size_t>(Q.slot)] = 0;
        Q.slot = -1;
    }
    if (Q.P) {
        srv->used -= Q.bytes;
        Q.P.reset();
    }
}

}  // namespace

static void select_many(im_ctx *ctx, int32_t nq, const im_graph *graphs, const im_params *params,
                        std::vector<std::unique_ptr<Prob>> &out) {
    std::vector<std::shared_ptr<GraphDev>> gd(nq);
    for (int32_t q = 0; q < nq; ++q) {
        check_params(&params[q], graphs[q].n, true);
        // problems given the very same graph description share one prepared device graph
        for (int32_t r = 0; r < q && !gd[q]; ++r)
            if (std::memcmp(&graphs[r], &graphs[q], sizeof(im_graph)) == 0) gd[q] = gd[r];
        if (!gd[q]) gd[q] = prepare_graph(ctx, &graphs[q]);
    }
    for (int32_t q = 0; q < nq; ++q) out.push_back(make_prob(ctx, gd[q], params[q], true));
    std::vector<Prob *> raw;
    for (auto &p : out) raw.push_back(p.get());
    Engine eng(ctx, raw);
    eng.run();
}

static void write_select_outputs(const Prob &P, int K, int32_t *seeds_out, double *sigma_out, int32_t *rebuilds_out,
                                 im_trace *trace) {
    std::copy(P.seeds.begin(), P.seeds.end(), seeds_out);
    if (sigma_out) *sigma_out = P.sigma.back();
    if (rebuilds_out) {
        int32_t r = 0;
        for (uint8_t b : P.rebuilt) r += b;
        *rebuilds_out = r;
    }
    if (trace) {
        for (int k = 0; k < K; ++k) {
            if (trace->seeds) trace->seeds[k] = P.seeds[k];
            if (trace->sigma) trace->sigma[k] = P.sigma[k];
            if (trace->estimate) trace->estimate[k] = P.est[k];
            if (trace->gsum) trace->gsum[k] = P.gsum[k];
            if (trace->rebuilt) trace->rebuilt[k] = P.rebuilt[k];
        }
    }
}

im_status im_select_seeds(im_ctx *ctx, const im_graph *graph, const im_params *params, int32_t *seeds_out,
                          double *sigma_out, int32_t *rebuilds_out, im_trace *trace) {
    if (!ctx) return IM_EINVAL;
    return guarded(ctx, [&]() {
        if (!graph || !params || !seeds_out) fail(IM_EINVAL, "graph / params / seeds_out is NULL");
        begin_call(ctx);
        CallTimer tm(ctx);
        std::vector<std::unique_ptr<Prob>> probs;
        select_many(ctx, 1, graph, params, probs);
        tm.stop();
        Prob &P = *probs[0];
        std::vector<Prob *> raw{&P};
        end_call(ctx, raw, tm.a, tm.b);
        write_select_outputs(P, params->K, seeds_out, sigma_out, rebuilds_out, trace);
    });
}

// ------------------------------------------------------------------------------------------------------------
// Autotuning of launch shapes: every candidate runs the same first diffusion (bit-identical results, checked) and
// the fastest is kept for the graph's (R, degree class).

im_status im_autotune(im_ctx *ctx, const im_graph *graph, const im_params *params, im_tuning *out) {
    if (!ctx) return IM_EINVAL;
    return guarded(ctx, [&]() {
        if (!graph || !params) fail(IM_EINVAL, "graph / params is NULL");
        check_params(params, graph->n, false);
        begin_call(ctx);
        auto G = prepare_graph(ctx, graph);
        const std::pair<int, int> key{params->R, degree_class(G->n, G->m)};
        ctx->tuned.erase(key);  // the base problem samples with the defaults
        auto base = make_prob(ctx, G, *params, false);
        const bool can_stream = base->dp.stream_min != ~0ull;
        struct Cand {
            int variant;
            bool stream;
            double ms;
        };
        std::vector<Cand> cands;
        for (int v : {4, 3, 6})
            for (int st = can_stream ? 1 : 0; st >= 0; --st) cands.push_back({v, st != 0, 1e30});
        const size_t regs = static_cast<size_t>(G->n) * params->R;
        DevMem tmp(ctx->stream);
        unsigned long long *d_sum = tmp.alloc<unsigned long long>(1);
        bool have_ref = false;
        DevCtr ref{};
        unsigned long long ref_sum = 0;
        for (int trial = 0; trial < 2; ++trial)
            for (Cand &c : cands) {
                auto P = make_prob(ctx, G, *params, false, base.get());
                P->variant = c.variant;
                P->dp.stream_min = c.stream ? base->dp.stream_min : ~0ull;
                Engine eng(ctx, {P.get()});
                cudaEvent_t a = eng.get_event(), b = eng.get_event();
                ck(cudaEventRecord(a, ctx->stream), "event");
                eng.run();
                ck(cudaEventRecord(b, ctx->stream), "event");
                ck(cudaEventSynchronize(b), "event");
                float ms = 0.f;
                ck(cudaEventElapsedTime(&ms, a, b), "elapsed");
                ctx->ev_free.push_back(a);
                ctx->ev_free.push_back(b);
                c.ms = std::min(c.ms, static_cast<double>(ms));
                ck(cudaMemsetAsync(d_sum, 0, sizeof(unsigned long long), ctx->stream), "memset");
                launch_checksum(P->last.res_par ? P->dp.M1 : P->dp.M0, regs, d_sum, ctx->stream);
                unsigned long long sum = 0;
                ck(cudaMemcpyAsync(&sum, d_sum, sizeof(sum), cudaMemcpyDeviceToHost, ctx->stream), "read sum");
                ck(cudaStreamSynchronize(ctx->stream), "sync");
                if (P->last.timeout) fail(IM_ETIMEOUT, "diffusion exceeded max_sweeps");
                if (!have_ref) {
                    have_ref = true;
                    ref = P->last;
                    ref_sum = sum;
                } else if (sum != ref_sum || P->last.sweeps_total != ref.sweeps_total || P->last.visits != ref.visits) {
                    fail(IM_ECUDA, "autotuning candidates reached different registers");
                }
            }
        const Cand *best = &cands[0];
        for (const Cand &c : cands)
            if (c.ms < best->ms) best = &c;
        ctx->tuned[key] = {best->variant, best->stream};
        if (out) {
            out->first_sweep_blocks = best->variant;
            out->stream_push = best->stream ? 1 : 0;
            out->candidates = static_cast<int32_t>(cands.size());
            out->degree_class = key.second;
            out->best_ms = best->ms;
            out->default_ms = cands[0].ms;
        }
    });
}

// ------------------------------------------------------------------------------------------------------------
// Sketch export / import and selections that start from a built sketch.

namespace {

uint64_t graph_fingerprint(im_ctx *ctx, const GraphDev &g) {
    DevMem tmp(ctx->stream);
    unsigned long long *d = tmp.alloc<unsigned long long>(1, true);
    launch_graph_hash(g.xadj, g.adj, g.n, g.T_edge, d, ctx->stream);
    ctx->launches += 1;
    unsigned long long h = 0;
    ck(cudaMemcpyAsync(&h, d, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream), "read fingerprint");
    ck(cudaStreamSynchronize(ctx->stream), "sync");
    return h;
}

uint64_t export_size(int64_t n, int32_t R) {
    return sizeof(im_sketch_header) + 8ull * static_cast<uint64_t>(R) + static_cast<uint64_t>(n) * R;
}

}  // namespace

im_status im_sketch_export(im_ctx *ctx, const im_sketch *sketch, void *host_buf, uint64_t cap, uint64_t *size_out) {
    if (!ctx) return IM_EINVAL;
    return guarded(ctx, [&]() {
        if (!sketch || !size_out) fail(IM_EINVAL, "sketch / size_out is NULL");
        const Prob &P = *sketch->P;
        const int64_t n = P.G->n;
        const int32_t R = P.prm.R;
        const uint64_t size = export_size(n, R);
        *size_out = size;
        if (!host_buf) return;
        if (cap < size) fail(IM_EINVAL, "the buffer is smaller than the exported sketch");
        begin_call(ctx);
        im_sketch_header h{};
        h.magic = IM_SKETCH_MAGIC;
        h.n = n;
        h.m = P.G->m;
        h.R = R;
        h.model = P.G->model;
        h.p = sketch->p;
        h.seed = P.prm.seed;
        h.eps_c = P.prm.eps_c;
        h.max_sweeps = P.prm.max_sweeps;
        h.sweeps = static_cast<int64_t>(P.last.sweeps_total);
        h.visits = P.last.visits;
        h.graph_hash = graph_fingerprint(ctx, *P.G);
        h.undirected = P.G->undirected;
        uint8_t *out = static_cast<uint8_t *>(host_buf);
        std::memcpy(out, &h, sizeof(h));
        cudaStream_t s = ctx->stream;
        ck(cudaMemcpyAsync(out + sizeof(h), P.dp.X, 4ull * R, cudaMemcpyDeviceToHost, s), "copy X");
        ck(cudaMemcpyAsync(out + sizeof(h) + 4ull * R, P.dp.Y, 4ull * R, cudaMemcpyDeviceToHost, s), "copy Y");
        ck(cudaMemcpyAsync(out + sizeof(h) + 8ull * R, P.last.res_par ? P.dp.M1 : P.dp.M0,
                           static_cast<size_t>(n) * R, cudaMemcpyDeviceToHost, s),
           "copy registers");
        ck(cudaStreamSynchronize(s), "sync");
    });
}

im_status im_sketch_import(im_ctx *ctx, const im_graph *graph, const void *host_buf, uint64_t size,
                           im_sketch **out) {
    if (!ctx) return IM_EINVAL;
    return guarded(ctx, [&]() {
        if (!graph || !host_buf || !out) fail(IM_EINVAL, "graph / host_buf / out is NULL");
        if (size < sizeof(im_sketch_header)) fail(IM_EINVAL, "too few bytes for a sketch");
        im_sketch_header h;
        std::memcpy(&h, host_buf, sizeof(h));
        if (h.magic != IM_SKETCH_MAGIC) fail(IM_EINVAL, "not an exported sketch");
        im_params prm{};
        prm.R = h.R;
        prm.K = 1;
        prm.eps_g = 0.01;
        prm.eps_l = 0.3;
        prm.eps_c = h.eps_c;
        prm.seed = h.seed;
        prm.max_sweeps = h.max_sweeps;
        check_params(&prm, graph->n, false);
        if (h.n != graph->n || h.m != graph->m) fail(IM_EINVAL, "the sketch was built on another graph (n, m)");
        if (size != export_size(h.n, h.R)) fail(IM_EINVAL, "the byte count does not match the header");
        if (h.model != graph->model || h.undirected != graph->undirected ||
            (graph->model == IM_IC_CONST && std::memcmp(&h.p, &graph->p, sizeof(double)) != 0))
            fail(IM_EINVAL, "the sketch was built with another diffusion model, probability or edge kind");
        begin_call(ctx);
        CallTimer tm(ctx);
        auto G = prepare_graph(ctx, graph);
        if (graph_fingerprint(ctx, *G) != h.graph_hash) fail(IM_EINVAL, "the sketch was built on another graph");
        auto sk = std::make_unique<im_sketch>();
        sk->ctx = ctx;
        sk->p = graph->p;
        sk->P = make_prob(ctx, G, prm, false);
        Prob &P = *sk->P;
        cudaStream_t s = ctx->stream;
        const uint8_t *in = static_cast<const uint8_t *>(host_buf);
        std::vector<uint32_t> xy(2 * static_cast<size_t>(h.R));
        ck(cudaMemcpyAsync(xy.data(), P.dp.X, 4ull * h.R, cudaMemcpyDeviceToHost, s), "read X");
        ck(cudaMemcpyAsync(xy.data() + h.R, P.dp.Y, 4ull * h.R, cudaMemcpyDeviceToHost, s), "read Y");
        ck(cudaMemcpyAsync(P.dp.M0, in + sizeof(h) + 8ull * h.R, static_cast<size_t>(h.n) * h.R,
                           cudaMemcpyHostToDevice, s),
           "copy registers");
        ck(cudaStreamSynchronize(s), "sync");
        if (std::memcmp(xy.data(), in + sizeof(h), 8ull * h.R) != 0)
            fail(IM_EINVAL, "the sketch's simulation words differ from this library's for its seed");
        P.last = DevCtr{};
        P.last.done = 1;
        P.last.res_par = 0;
        P.last.sweeps_total = static_cast<unsigned long long>(h.sweeps);
        P.last.visits = h.visits;
        P.builds = 1;
        tm.stop();
        end_call(ctx, {&P}, tm.a, tm.b);
        *out = sk.release();
    });
}

im_status im_select_seeds_from(im_ctx *ctx, const im_sketch *sketch, const im_params *params, int32_t *seeds_out,
                               double *sigma_out, int32_t *rebuilds_out, im_trace *trace) {
    if (!ctx) return IM_EINVAL;
    return guarded(ctx, [&]() {
        if (!sketch || !params || !seeds_out) fail(IM_EINVAL, "sketch / params / seeds_out is NULL");
        const Prob &S = *sketch->P;
        check_params(params, S.G->n, true);
        if (params->R != S.prm.R || params->seed != S.prm.seed || params->eps_c != S.prm.eps_c ||
            params->max_sweeps != S.prm.max_sweeps)
            fail(IM_EINVAL, "params must have the sketch's R, seed, eps_c and max_sweeps");
        begin_call(ctx);
        CallTimer tm(ctx);
        // share the sketch's sampled graph, start from a copy of its registers at the first greedy step
        auto P = make_prob(ctx, S.G, *params, true, &S);
        ck(cudaMemcpyAsync(S.last.res_par ? P->dp.M1 : P->dp.M0, S.last.res_par ? S.dp.M1 : S.dp.M0,
                           static_cast<size_t>(S.G->n) * S.prm.R, cudaMemcpyDeviceToDevice, ctx->stream),
           "copy registers");
        std::vector<DevCtr> c0(1);
        c0[0].res_par = S.last.res_par;
        c0[0].done = 1;
        c0[0].sweeps_total = S.last.sweeps_total;
        c0[0].visits = S.last.visits;
        c0[0].bytes = S.last.bytes;
        Engine eng(ctx, {P.get()}, &c0);
        P->phase = Prob::kScan;
        P->builds = 1;
        eng.run();
        tm.stop();
        end_call(ctx, {P.get()}, tm.a, tm.b);
        write_select_outputs(*P, params->K, seeds_out, sigma_out, rebuilds_out, trace);
    });
}

im_status im_select_seeds_batch(im_ctx *ctx, int32_t nq, const im_graph *graphs, const im_params *params,
                                int32_t *const *seeds_out, double *sigma_out, int32_t *rebuilds_out) {
    if (!ctx) return IM_EINVAL;
    return guarded(ctx, [&]() {
        if (nq < 1 || !graphs || !params || !seeds_out) fail(IM_EINVAL, "empty batch or NULL argument");
        begin_call(ctx);
        CallTimer tm(ctx);
        std::vector<std::unique_ptr<Prob>> probs;
        select_many(ctx, nq, graphs, params, probs);
        tm.stop();
        std::vector<Prob *> raw;
        for (auto &p : probs) raw.push_back(p.get());
        end_call(ctx, raw, tm.a, tm.b);
        for (int32_t q = 0; q < nq; ++q) {
            if (!seeds_out[q]) fail(IM_EINVAL, "seeds_out[q] is NULL");
            std::copy(probs[q]->seeds.begin(), probs[q]->seeds.end(), seeds_out[q]);
            if (sigma_out) sigma_out[q] = probs[q]->sigma.back();
            if (rebuilds_out) {
                int32_t r = 0;
                for (uint8_t b : probs[q]->rebuilt) r += b;
                rebuilds_out[q] = r;
            }
        }
    });
}


im_status im_server_create(im_ctx *ctx, uint64_t hbm_budget_bytes, int32_t max_active, im_server **out) {
    if (!ctx) return IM_EINVAL;
    return guarded(ctx, [&]() {
        if (!out) fail(IM_EINVAL, "out is NULL");
        if (max_active < 1 || max_active > 4096) fail(IM_EINVAL, "max_active must be in [1, 4096]");
        if (hbm_budget_bytes == 0) fail(IM_EINVAL, "the HBM budget must be positive");
        ck(cudaSetDevice(ctx->device), "cudaSetDevice");
        auto srv = std::make_unique<im_server>();
        srv->ctx = ctx;
        srv->budget = hbm_budget_bytes;
        srv->eng = std::make_unique<Engine>(ctx, static_cast<size_t>(max_active));
        srv->eng->soft_errors = true;
        srv->slot_ticket.assign(static_cast<size_t>(max_active), 0);
        for (int32_t i = max_active - 1; i >= 0; --i) srv->free_slots.push_back(static_cast<size_t>(i));
        *out = srv.release();
    });
}

im_status im_server_destroy(im_server *srv) {
    if (!srv) return IM_EINVAL;
    cudaSetDevice(srv->ctx->device);
    cudaStreamSynchronize(srv->ctx->stream);
    for (auto &kv : srv->q) kv.second.P.reset();
    srv->eng.reset();
    srv->graphs.clear();
    cudaStreamSynchronize(srv->ctx->stream);
    delete srv;
    return IM_OK;
}

im_status im_server_add_graph(im_server *srv, const im_graph *graph, int32_t *graph_id) {
    if (!srv) return IM_EINVAL;
    im_ctx *ctx = srv->ctx;
    return guarded(ctx, [&]() {
        if (!graph_id) fail(IM_EINVAL, "graph_id is NULL");
        ck(cudaSetDevice(ctx->device), "cudaSetDevice");
        srv->graphs.push_back(prepare_graph(ctx, graph));
        *graph_id = static_cast<int32_t>(srv->graphs.size() - 1);
    });
}

im_status im_server_submit(im_server *srv, int32_t graph_id, const im_params *params, uint64_t *ticket) {
    if (!srv) return IM_EINVAL;
    im_ctx *ctx = srv->ctx;
    return guarded(ctx, [&]() {
        if (!params || !ticket) fail(IM_EINVAL, "params / ticket is NULL");
        if (graph_id < 0 || graph_id >= static_cast<int32_t>(srv->graphs.size())) fail(IM_EINVAL, "unknown graph id");
        const GraphDev &g = *srv->graphs[static_cast<size_t>(graph_id)];
        check_params(params, g.n, true);
        if (query_footprint(g, *params) > srv->budget)
            fail(IM_ENOMEM, "the query needs more device memory than the whole HBM budget");
        const uint64_t t = srv->next++;
        im_server::Query &Q = srv->q[t];
        Q.gid = graph_id;
        Q.prm = *params;
        srv->queue.push_back(t);
        *ticket = t;
    });
}

im_status im_server_footprint(im_server *srv, int32_t graph_id, const im_params *params, uint64_t *bytes) {
    if (!srv) return IM_EINVAL;
    return guarded(srv->ctx, [&]() {
        if (!params || !bytes) fail(IM_EINVAL, "params / bytes is NULL");
        if (graph_id < 0 || graph_id >= static_cast<int32_t>(srv->graphs.size())) fail(IM_EINVAL, "unknown graph id");
        const GraphDev &g = *srv->graphs[static_cast<size_t>(graph_id)];
        check_params(params, g.n, true);
        *bytes = query_footprint(g, *params);
    });
}

im_status im_server_step(im_server *srv, int32_t *active_out, int32_t *queued_out) {
    if (!srv) return IM_EINVAL;
    im_ctx *ctx = srv->ctx;
    return guarded(ctx, [&]() {
        ck(cudaSetDevice(ctx->device), "cudaSetDevice");
        // admission: first come, first served, while a slot is free and the budget allows
        while (!srv->queue.empty() && !srv->free_slots.empty()) {
            const uint64_t t = srv->queue.front();
            im_server::Query &Q = srv->q[t];
            const GraphDev &g = *srv->graphs[static_cast<size_t>(Q.gid)];
            const uint64_t est = query_footprint(g, Q.prm);
            const auto key = build_key(Q);
            // room for the query comes first: kept diffusions go, the one this query could start from last
            while (srv->used + est > srv->budget && evict_build(srv, &key)) {
            }
            if (srv->used + est > srv->budget) evict_build(srv, nullptr);
            if (srv->used + est > srv->budget) break;
            auto hit = srv->builds.find(key);
            srv->queue.pop_front();
            const size_t slot = srv->free_slots.back();
            srv->free_slots.pop_back();
            if (hit != srv->builds.end()) {
                // the first diffusion is this kept one: share its sampled graph, copy its registers, and start
                // at the first greedy step with the counters it ended with
                im_server::Build &b = hit->second;
                b.last_use = ++srv->clock;
                Q.P = make_prob(ctx, srv->graphs[static_cast<size_t>(Q.gid)], Q.prm, true, &b.sample);
                Prob &P = *Q.P;
                ck(cudaMemcpyAsync(b.ctr.res_par ? P.dp.M1 : P.dp.M0, b.M,
                                   static_cast<size_t>(g.n) * static_cast<size_t>(Q.prm.R), cudaMemcpyDeviceToDevice,
                                   ctx->stream),
                   "copy kept registers");
                srv->eng->attach(slot, &P, &b.ctr);
                P.phase = Prob::kScan;
                P.builds = 1;
                Q.fill = false;
                srv->build_hits += 1;
            } else {
                Q.P = make_prob(ctx, srv->graphs[static_cast<size_t>(Q.gid)], Q.prm, true);
                srv->eng->attach(slot, Q.P.get(), nullptr);
                Q.fill = true;
            }
            Q.bytes = est;  // the reservation: the query's allocations stay within it
            srv->used += Q.bytes;
            srv->slot_ticket[slot] = t;
            Q.slot = static_cast<int64_t>(slot);
            Q.state = 1;
        }
        srv->eng->tick();
        // keep first diffusions that just finished, before the next tick's kernels run
        for (size_t slot = 0; slot < srv->slot_ticket.size(); ++slot) {
            const uint64_t t = srv->slot_ticket[slot];
            if (!t) continue;
            im_server::Query &Q = srv->q[t];
            const Prob &P = *Q.P;
            if (Q.fill && P.status == IM_OK && P.phase == Prob::kScan && P.step == 0 && P.builds == 1) {
                Q.fill = false;
                if (srv->builds.find(build_key(Q)) == srv->builds.end()) keep_build(srv, Q);
            }
        }
        // harvest finished queries and free their memory
        for (size_t slot = 0; slot < srv->slot_ticket.size(); ++slot) {
            const uint64_t t = srv->slot_ticket[slot];
            if (!t) continue;
            im_server::Query &Q = srv->q[t];
            Prob &P = *Q.P;
            if (P.phase != Prob::kDone) continue;
            if (P.status != IM_OK) {
                Q.state = 4;
                Q.status = P.status;
                Q.error = P.error;
            } else {
                Q.state = 2;
                Q.seeds = P.seeds;
                Q.sigma = P.sigma.back();
                Q.rebuilds = 0;
                for (uint8_t b : P.rebuilt) Q.rebuilds += b;
            }
            server_release(srv, Q);
        }
        int32_t active = 0;
        for (uint64_t t : srv->slot_ticket) active += t ? 1 : 0;
        if (active_out) *active_out = active;
        if (queued_out) *queued_out = static_cast<int32_t>(srv->queue.size());
    });
}

im_status im_server_info(const im_server *srv, uint64_t *used_bytes, int32_t *kept_builds, uint64_t *build_hits) {
    if (!srv) return IM_EINVAL;
    if (used_bytes) *used_bytes = srv->used;
    if (kept_builds) *kept_builds = static_cast<int32_t>(srv->builds.size());
    if (build_hits) *build_hits = srv->build_hits;
    return IM_OK;
}

im_status im_server_poll(im_server *srv, uint64_t ticket, int32_t *seeds_out, double *sigma_out,
                         int32_t *rebuilds_out) {
    if (!srv) return IM_EINVAL;
    im_ctx *ctx = srv->ctx;
    auto it = srv->q.find(ticket);
    if (it == srv->q.end()) {
        set_err(ctx, "unknown ticket");
        return IM_EINVAL;
    }
    im_server::Query &Q = it->second;
    if (Q.state == 0 || Q.state == 1) return IM_ENOTREADY;
    if (Q.state == 3) {
        srv->q.erase(it);
        return IM_ECANCELED;
    }
    if (Q.state == 4) {
        const im_status st = Q.status;
        set_err(ctx, Q.error);
        srv->q.erase(it);
        return st;
    }
    if (seeds_out) std::copy(Q.seeds.begin(), Q.seeds.end(), seeds_out);
    if (sigma_out) *sigma_out = Q.sigma;
    if (rebuilds_out) *rebuilds_out = Q.rebuilds;
    srv->q.erase(it);
    return IM_OK;
}

im_status im_server_cancel(im_server *srv, uint64_t ticket) {
    if (!srv) return IM_EINVAL;
    auto it = srv->q.find(ticket);
    if (it == srv->q.end()) {
        set_err(srv->ctx, "unknown ticket");
        return IM_EINVAL;
    }
    im_server::Query &Q = it->second;
    if (Q.state >= 2) return IM_OK;
    if (Q.state == 0) {
        for (auto qi = srv->queue.begin(); qi != srv->queue.end(); ++qi)
            if (*qi == ticket) {
                srv->queue.erase(qi);
                break;
            }
    } else {
        server_release(srv, Q);
    }
    Q.state = 3;
    return IM_OK;
}

}  // extern "C"
