// Host-side launchers of the library's kernels (defined in im_kernels.cu).  Every launcher enqueues on stream s and
// returns at once; problem descriptors and the active list live in device memory.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "im_common.cuh"

namespace imk {

cudaError_t configure(int device);
int grid_warp();

// Start of a diffusion (counters, bits, the vertices S reached, residual blocking in the problem's pair ranks).
// Returns the launches.
int launch_init(const DevProb *probs, const int32_t *act, int nact, cudaStream_t s);
// One sweep: when a listed problem may start a diffusion, launch_first (the fused first-sweep kernel) and then
// launch_prop with pulls (the push kernel beside it, or with pull_more the kernel that also pulls later sweeps);
// else launch_prop alone (the push-only kernel).  Each returns the number of kernels launched.
int launch_first(int R, const DevProb *probs, const int32_t *act, int nact, int variant, cudaStream_t s);
int launch_prop(int R, const DevProb *probs, const int32_t *act, int nact, bool pulls, bool pull_more,
                cudaStream_t s);
// Adds an order-free checksum of `bytes` bytes (a multiple of 8) at x to *out.
void launch_checksum(const void *x, uint64_t bytes, unsigned long long *out, cudaStream_t s);
void launch_combine(int R, const DevProb *probs, const int32_t *act, int nact, cudaStream_t s);
// Ends a sweep: frontier lists and row copies, then (last block) the stop test and counter resets.
void launch_frontier(const DevProb *probs, const int32_t *act, int nact, GridBar *gb, cudaStream_t s);
void launch_scan(int R, const DevProb *probs, const int32_t *act, int nact, cudaStream_t s);
// The lazy argmax of a greedy step that keeps the sketch (bound pass, exact key of the best bound, exact pass over
// the candidates whose bound beats it); every listed problem must have had a full scan since its last build.
// Returns the kernels launched.
int launch_celf(int R, const DevProb *probs, const int32_t *act, int nact, cudaStream_t s);
void launch_choose(const DevProb *probs, const int32_t *act, int nact, int32_t step, cudaStream_t s);
void launch_seed_set(const DevProb *prob, const int32_t *seeds, int k, int W, cudaStream_t s);
// One search level of each listed problem; its last block ends the level (stop test, counter resets).
void launch_bfs_level(int R, const DevProb *probs, const int32_t *act, int nact, GridBar *gb, cudaStream_t s);
// A whole search in one cooperative launch; false if the device cannot run it (the caller then steps levels).
// barrier_limit: polls of one grid-barrier wait before the kernel gives up (kBarrierLimit unless a test lowers it).
bool launch_bfs_run(int R, const DevProb *probs, const int32_t *act, int nact, GridBar *gb, uint32_t barrier_limit,
                    cudaStream_t s);
void launch_merge(const DevProb *probs, const int32_t *act, int nact, cudaStream_t s);
// Influence scorer: live masks of samples s0 .. s0 + R - 1 (those at or past nvalid left dead) into prob->live,
// and per-sample reach counts of prob->vis added into counts[R].
void launch_mc_live(int R, const DevProb *prob, uint64_t seed, int64_t s0, int64_t nvalid, int64_t nchunks,
                    cudaStream_t s);
void launch_sample_counts(int R, const DevProb *prob, unsigned long long *counts, cudaStream_t s);
void launch_estimate(const DevProb *prob, const int32_t *seeds, int k, unsigned long long *gsum, cudaStream_t s);

void launch_live_masks(const DevProb &P, int32_t *npairs, int32_t *ndense, cudaStream_t s);
void launch_init_table(const DevProb &P, cudaStream_t s);
void launch_pair_fill(const DevProb &P, int32_t *pv, uint16_t *pj, uint16_t *pq, uint32_t *dlist, cudaStream_t s);
void launch_inpair_counts(const DevProb &P, const int32_t *np_out, const int32_t *nd_out, int32_t *npairs,
                          int32_t *ndense, cudaStream_t s);
void launch_inpair_fill(const DevProb &P, int32_t *iu, uint16_t *ij, uint32_t *iop, int32_t *iv, int32_t *idu,
                        uint32_t *ide, cudaStream_t s);
void launch_vertex_desc(const DevProb &P, UnitD *vdesc, cudaStream_t s);
void launch_unit_desc(const DevProb &P, UnitD *rdesc, UnitD *tdesc, cudaStream_t s);
void launch_words(uint64_t seed, int R, uint32_t *X, uint32_t *Y, cudaStream_t s);
// Adds the graph's 64-bit fingerprint (edges and per-edge thresholds, if any) to *out.
void launch_graph_hash(const int64_t *xadj, const int32_t *adj, int64_t n, const uint32_t *T_edge,
                       unsigned long long *out, cudaStream_t s);
void launch_indeg(const int32_t *adj, int64_t m, int32_t *indeg, cudaStream_t s);
void launch_wc_thresholds(const int32_t *indeg, int64_t n, uint32_t *T, cudaStream_t s);
void launch_transpose_fill(const int64_t *xadj, const int32_t *adj, int64_t n, int64_t m, unsigned long long *cursor,
                           int32_t *adj_in, uint32_t *ein, cudaStream_t s);
void launch_row_tasks(const int64_t *xadj, int64_t n, int32_t *ntask, uint32_t *heavy, cudaStream_t s);
void launch_classes(const int64_t *xadj, const int64_t *task_off, int64_t n, int32_t *task_row, int32_t *light,
                    unsigned int *counts, int32_t *hsmall, int32_t *hbig, cudaStream_t s);
int64_t scan_block_count(int64_t n);
// Returns the number of kernels it launched.
int launch_exclusive_scan(const int32_t *in, int64_t n, int64_t *out, int64_t *block_sums, cudaStream_t s);

}  // namespace imk
