// CUDA kernels (sm_103a) of the sketch-based influence-maximisation library.
//
// Every kernel takes an array of problem descriptors plus a list of the active ones and treats the work of all of
// them as one flat index space striped over its warps (or blocks, or threads), so a single launch serves one large
// problem or hundreds of small ones.  Grids are sized once per device (a multiple of the SM count) and kernels read
// their work counts from device memory, so the host can enqueue sweeps ahead without reading anything back.
//
// Paper map:
//   k_init        Algorithm 1, register initialisation (and its re-initialisation with R_G(S) blocked)
//   k_first       Algorithm 1's initialisation fused into Algorithm 2's first sweep (L = V): every register it
//                 reads is an initial rank (the pair words carry their neighbour's, the problem's table Mi the
//                 row's own and the dense neighbours'); it writes every row of both register buffers.
//   k_init_table  the table Mi of initial ranks, once per problem (rebuilds zero its blocked entries in
//                 k_block_done)
//                 The sampling of Eq. 4-5 is evaluated once per run (k_live_masks) and kept as (target,
//                 simulation) pairs for edges live in few simulations (k_pair_fill, and in in-CSR order
//                 k_inpair_fill) and as live masks for the others
//   k_propg       Algorithm 2, a later sweep that pulls into every row (when more than one sweep pulls)
//   k_push        Algorithm 2, the later sweeps, pushed from the vertices L that changed in the previous one
//   k_combine     Algorithm 2, sweep 0 for rows split over several warps
//   k_frontier    Algorithm 2, the live sets L and L' (and the copy a push sweep needs); its last block applies
//                 the stop test (eps_c)
//   k_scan, k_choose             Algorithm 1, argmax of Estimate(Merge(M_S', M_v)) (Eq. 2-3)
//   k_bfs_level (k_bfs_run)      Algorithm 1, reachability set of S in every simulation, sigma
//   k_merge                      Algorithm 1, M_S' <- Merge(M_S', M_s)
#include <algorithm>
#include <cstdlib>

#include "im_common.cuh"
#include "im_launch.h"

namespace imk {

namespace {

constexpr unsigned kFull = 0xffffffffu;

// First index owned by `worker` among the units [base, base + count) of a flat space striped over `nworkers`.
__device__ __forceinline__ uint64_t first_owned(uint64_t worker, uint64_t nworkers, uint64_t base) {
    const uint64_t r = base % nworkers;
    return worker >= r ? worker - r : worker + nworkers - r;
}

template <int R>
struct Geo {
    static constexpr int CH = R / 16;               // 16-byte chunks per register row
    static constexpr int G = CH < 32 ? CH : 32;     // lanes that read one neighbour row together
    static constexpr int NG = 32 / G;               // neighbour rows a warp reads at once
    static constexpr int CPL = CH / G;              // chunks per lane
};

// Byte-wise max of registers.  Every register value is <= 32 < 128, so per byte a - b + 128 lies in [1, 255]: the
// word subtraction below never carries across bytes and bit 7 of each byte is (a >= b); prmt replicates it.
__device__ __forceinline__ uint32_t sign_bytes(uint32_t x, uint32_t y, uint32_t sel) {
    uint32_t r;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(r) : "r"(x), "r"(y), "r"(sel));
    return r;
}

__device__ __forceinline__ uint32_t vmax4(uint32_t a, uint32_t b) {
    const uint32_t ge = sign_bytes(a + 0x80808080u - b, 0u, 0xBA98u);
    return (a & ge) | (b & ~ge);
}

struct WarpStage {
    unsigned long long mbar;  // completion barrier of the warp's bulk copies
    int32_t v[32];            // task index of each partial row being gathered
};

template <int R>
__device__ __forceinline__ void reduce_groups(uint32_t (&acc)[Geo<R>::CPL][4]) {
#pragma unroll
    for (int off = Geo<R>::G; off < 32; off <<= 1)
#pragma unroll
        for (int c = 0; c < Geo<R>::CPL; ++c)
#pragma unroll
            for (int w = 0; w < 4; ++w) acc[c][w] = vmax4(acc[c][w], __shfl_xor_sync(kFull, acc[c][w], off));
}

__device__ __forceinline__ uint64_t thr_bytes(int32_t model) { return model == kWC ? 4 : (model == kPerEdge ? 5 : 0); }

__device__ __forceinline__ uint64_t in_degree(const DevProb &P, int64_t v) {
    return static_cast<uint64_t>(__ldg(&P.xadj_in[v + 1]) - __ldg(&P.xadj_in[v]));
}

struct Stats {
    unsigned long long bytes = 0;
    unsigned long long pairs = 0;  // sparse (edge, simulation) pairs examined
};

__device__ __forceinline__ void flush_stats(DevCtr *C, Stats &st, int lane) {
    if (lane == 0) {
        if (st.bytes) atomicAdd(&C->bytes, st.bytes);
        if (st.pairs) atomicAdd(&C->pairs, st.pairs);
    }
    st = Stats();
}

// ------------------------------------------------------------------------------------------------------------
// Gather form of the sweep (the default): as above, one warp per row, but the register rows of the sampled
// neighbours of each staged batch (and the row's own registers) are copied into a per-warp shared-memory buffer
// with cp.async before they are merged, so a warp keeps up to GSlots<R> rows in flight without holding them in
// registers.

template <int R>
struct GSlots {
    static constexpr int N = R <= 256 ? 16 : (R == 512 ? 8 : 4);
    static constexpr int kBytesPerWarp = (N + 1) * R;
    // the sweep kernel: one 32-bit accumulator per simulation and tile for the sparse pairs
    static constexpr int kPropBytesPerWarp = Geo<R>::NG * 4 * R;
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Per-warp completion barrier for bulk copies (TMA bulk copy engine, one instruction per row).
constexpr uint32_t kWaitLimit = 1u << 16;      // tries of mbarrier.try_wait before a copy counts as lost
constexpr uint32_t kWaitHintNs = 20000;        // each try may suspend the thread up to this long (about 1.3 s in all)

__device__ __forceinline__ void mbar_init(unsigned long long *m) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(m)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect(unsigned long long *m, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(m)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, unsigned long long *m) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(m))
                 : "memory");
}
__device__ __forceinline__ bool mbar_try(unsigned long long *m, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(m)), "r"(parity), "r"(kWaitHintNs)
        : "memory");
    return ok != 0;
}
// Waits (all lanes of the warp) for the barrier phase of the given parity.  After kWaitLimit tries the copies count
// as lost: the fault flag is raised for the host, a second bounded wait gives copies still in flight a chance to
// land, and the warp is marked aborted, after which it issues no copies and waits no more (its remaining work runs
// on whatever the buffers hold and the host discards the result).
__device__ __forceinline__ bool mbar_wait(unsigned long long *m, uint32_t parity, unsigned int *fault, bool &aborted) {
    if (aborted) return false;
    bool done = false;
    for (uint32_t it = 0; it < kWaitLimit && !done; ++it) done = mbar_try(m, parity);
    done = __all_sync(0xffffffffu, done);
    if (!done) {
        if ((threadIdx.x & 31) == 0) atomicOr(fault, 1u);
        for (uint32_t it = 0; it < kWaitLimit; ++it)
            if (mbar_try(m, parity)) break;
        aborted = true;
    }
    return done;
}
// Orders this warp's earlier generic reads of a buffer before bulk copies that overwrite it.
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Bit k set where byte k of a and b differ (four bits): one byte-compare, then the low bit of each byte moved to
// bit 24 + k by one multiply (the shifted copies land on distinct bits, so nothing carries into bits 24..27).
__device__ __forceinline__ uint32_t ne_bits4(uint32_t a, uint32_t b) {
    return (((__vcmpne4(a, b) & 0x01010101u) * 0x01020408u) >> 24) & 0xFu;
}
// Sixteen registers (one 16-byte chunk): bit k set where register k of the chunk differs.
__device__ __forceinline__ uint32_t ne_bits16(const uint4 &a, const uint4 &b) {
    return ne_bits4(a.x, b.x) | (ne_bits4(a.y, b.y) << 4) | (ne_bits4(a.z, b.z) << 8) | (ne_bits4(a.w, b.w) << 12);
}

// Sum of the 16 registers (bytes) of a chunk.
__device__ __forceinline__ uint32_t byte_sum16(const uint4 &a) {
    return __dp4a(a.x, 0x01010101u, __dp4a(a.y, 0x01010101u, __dp4a(a.z, 0x01010101u, __dp4a(a.w, 0x01010101u, 0u))));
}

// Byte masks of four simulations from four live bits (the low nibble of n): bit k is moved to bit 8k + 7 by one
// multiply (the shifted copies never overlap, so nothing carries) and prmt replicates each byte's top bit.
__device__ __forceinline__ uint32_t nibble_bytes(uint32_t n) { return sign_bytes(n * 0x10204080u, 0u, 0xBA98u); }

// The sweep kernel works in tiles of G = Geo<R>::G lanes (16 for R = 256): each tile owns one unit (a light row
// or a task) at a time, so a warp keeps 32 / G units in flight.  Lane li of a tile holds the 16-simulation chunks
// li + G * c of the row.
template <int R>
__device__ __forceinline__ unsigned tile_mask(int g) {
    return Geo<R>::G == 32 ? kFull : (((1u << Geo<R>::G) - 1u) << (g * Geo<R>::G));
}

// The first sweep of a diffusion reads every register before any sweep has changed it, so every register it
// reads is an initial rank (Algorithm 1's initialisation): M_v[j] = clz(hash(v) XOR Y_j), or 0 where v is in
// R_{G_j}(S) (a rebuild).  P.rany marks the vertices reached in some simulation (their blocked bits are then read
// from vis); it is NULL when there is no seed set.
__device__ __forceinline__ uint32_t blocked16(const DevProb &P, int64_t v, int ch) {
    if (!P.rany || !test_bit(P.rany, v)) return 0u;
    return (__ldg(&P.vis[static_cast<size_t>(v) * P.W + (ch >> 1)]) >> (16 * (ch & 1))) & 0xFFFFu;
}

// Initial registers of the 16 simulations of chunk ch (four bytes a word) of a vertex with hash hv, zero where
// blk (bit k: simulation 16 ch + k) is set.  Y: the problem's initialisation words (global, or a shared copy).
__device__ __forceinline__ uint4 init_chunk(const uint32_t *Y, uint32_t hv, int ch, uint32_t blk) {
    const uint4 *y = reinterpret_cast<const uint4 *>(Y) + 4 * ch;
    uint32_t w[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const uint4 q = y[k];
        const uint32_t x = __clz(hv ^ q.x) | (__clz(hv ^ q.y) << 8) | (__clz(hv ^ q.z) << 16) |
                           (__clz(hv ^ q.w) << 24);
        w[k] = x & ~nibble_bytes((blk >> (4 * k)) & 0xFu);
    }
    return make_uint4(w[0], w[1], w[2], w[3]);
}

// Shared-memory slot of simulation j in a per-simulation word array (a tile's accumulators, the staged Y words):
// the four 16-byte words of each 16-simulation chunk ch are permuted by XOR with (ch / 2 XOR 2 rot) mod 4.  A 16-byte
// load is served eight lanes at a time, and eight lanes reading word w of chunks ch .. ch + 7 (a 64-byte stride)
// then cover the eight 16-byte bank groups once each: ch mod 2 picks the half of the 128 bytes, the permutation the
// group within it (without it the eight lanes fall on two groups, a 4-way conflict).  2 rot separates the two
// 4-lane tiles that share a load when a tile is 4 lanes wide (R = 64).  The map is its own inverse, and
// sw_slot(j, rot) = sw_slot(j, 0) XOR sw_tile(rot).
__device__ __forceinline__ uint32_t sw_tile(uint32_t rot) { return ((2u * rot) & 3u) << 2; }
__device__ __forceinline__ uint32_t sw_slot(uint32_t j, uint32_t rot) {
    return j ^ (((j >> 5) & 3u) << 2) ^ sw_tile(rot);
}
// Position of word w of chunk ch among the chunk's four 16-byte words under sw_slot(., rot).
__device__ __forceinline__ int sw_pos(int w, int ch, int rot) { return (w ^ (ch >> 1) ^ (2 * rot)) & 3; }

// init_chunk over Y words staged in shared memory with sw_slot(j, 0); without BLK nothing is blocked (blk unused).
template <bool BLK = true>
__device__ __forceinline__ uint4 init_chunk_sw(const uint32_t *Ysw, uint32_t hv, int ch, uint32_t blk) {
    const uint4 *y = reinterpret_cast<const uint4 *>(Ysw + 16 * ch);
    uint32_t w[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const uint4 q = y[sw_pos(k, ch, 0)];
        const uint32_t x = __clz(hv ^ q.x) | (__clz(hv ^ q.y) << 8) | (__clz(hv ^ q.z) << 16) |
                           (__clz(hv ^ q.w) << 24);
        w[k] = BLK ? x & ~nibble_bytes((blk >> (4 * k)) & 0xFu) : x;
    }
    return make_uint4(w[0], w[1], w[2], w[3]);
}

// Initial register of (v, j), 0 if v is in R_{G_j}(S) (unless literal blocking keeps it).  Ysw: the Y words
// staged with sw_slot(j, 0).
__device__ __forceinline__ uint32_t init_reg(const DevProb &P, const uint32_t *Ysw, int32_t v, uint32_t j) {
    const uint32_t r = __clz(vertex_hash(static_cast<uint32_t>(v)) ^ Ysw[sw_slot(j, 0)]);
    if (!P.literal && P.rany && test_bit(P.rany, v) &&
        ((__ldg(&P.vis[static_cast<size_t>(v) * P.W + (j >> 5)]) >> (j & 31)) & 1u))
        return 0u;
    return r;
}

// Blocked bits of an initial row: those of v under residual blocking (its registers there are 0), none under
// literal blocking (a blocked register keeps its rank).
__device__ __forceinline__ uint32_t init_blocked16(const DevProb &P, int64_t v, int ch) {
    return P.literal ? 0u : blocked16(P, v, ch);
}

// Whether (u, j) is blocked under literal blocking, where such a register is never updated.  Under residual
// blocking nothing needs this test: a blocked (u, j) has only blocked live successors, whose registers are 0.
__device__ __forceinline__ bool literal_blocked(const DevProb &P, int64_t u, uint32_t j) {
    return P.literal && P.rany && test_bit(P.rany, u) &&
           ((__ldg(&P.vis[static_cast<size_t>(u) * P.W + (j >> 5)]) >> (j & 31)) & 1u);
}

// Dense edges dlist[d0, d1) of the tile's unit (edges live in many simulations), merged with whole register rows:
// the tile loads two neighbour rows per round (16 bytes per lane and chunk) when their v is in L, and max-merges
// them into acc through the edges' live masks (Eq. 4-5, sampled once per run).  Returns the merged rows.  In the
// first sweep (INIT) the rows are the neighbours' initial registers, computed.
template <int R, bool INIT>
__device__ __forceinline__ uint32_t dense_tile(const DevProb &P, int64_t d0, int64_t d1, bool allL,
                                               const uint32_t *__restrict__ Lcur, const uint8_t *__restrict__ Mcur,
                                               const uint32_t *Ys, bool chk, uint32_t (&acc)[Geo<R>::CPL][4],
                                               int li) {
    using Gm = Geo<R>;
    constexpr int W = R / 32;
    uint32_t taken = 0;
    for (int64_t i = d0; i < d1; i += 2) {
        uint4 row[2][Gm::CPL];
        uint32_t msk[2][Gm::CPL];
        bool in[2];
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            in[r] = false;
            int64_t e = 0;
            int32_t v = 0;
            if (i + r < d1) {
                e = static_cast<int64_t>(__ldg(&P.dlist[i + r]));
                v = __ldg(&P.adj[e]);
                in[r] = allL || test_bit(Lcur, v);
            }
#pragma unroll
            for (int c = 0; c < Gm::CPL; ++c) {
                const int ch = li + Gm::G * c;  // 16-simulation chunk: half (ch & 1) of mask word ch / 2
                if (INIT)  // the neighbour's initial registers (blocked ones 0 under residual blocking)
                    row[r][c] = in[r] ? __ldg(reinterpret_cast<const uint4 *>(P.Mi + static_cast<size_t>(v) * R) + ch)
                                      : make_uint4(0, 0, 0, 0);
                else
                    row[r][c] = in[r] ? __ldg(reinterpret_cast<const uint4 *>(Mcur + static_cast<size_t>(v) * R) + ch)
                                      : make_uint4(0, 0, 0, 0);
                msk[r][c] = in[r] ? (__ldg(&P.live[static_cast<size_t>(e) * W + (ch >> 1)]) >> (16 * (ch & 1))) : 0u;
            }
        }
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            taken += in[r] ? 1u : 0u;
#pragma unroll
            for (int c = 0; c < Gm::CPL; ++c) {
                const uint32_t m = msk[r][c];
                acc[c][0] = vmax4(acc[c][0], row[r][c].x & nibble_bytes(m & 0xFu));
                acc[c][1] = vmax4(acc[c][1], row[r][c].y & nibble_bytes((m >> 4) & 0xFu));
                acc[c][2] = vmax4(acc[c][2], row[r][c].z & nibble_bytes((m >> 8) & 0xFu));
                acc[c][3] = vmax4(acc[c][3], row[r][c].w & nibble_bytes((m >> 12) & 0xFu));
            }
        }
    }
    return taken;
}

// Sparse pairs [p0, p1) of the tile's unit: for every pair (v, j) with v in L, acc32[j] = max(acc32[j], M_v[j])
// (the max-merge of Algorithm 2 for one sampled simulation).  Lanes take pairs four at a time, and a pair's
// register is loaded together with its L bit (and dropped if v is not in L), so one round of dependent loads
// serves 4 G pairs (in the first sweep, INIT, the registers are initial ranks, computed).  Returns the number of
// pairs this lane merged.
template <int R, bool INIT>
__device__ __forceinline__ uint32_t sparse_tile(const DevProb &P, int64_t p0, int64_t p1, bool allL,
                                                const uint32_t *__restrict__ Lcur, const uint8_t *__restrict__ Mcur,
                                                const uint32_t *Ys, uint32_t *acc32, int li) {
    constexpr int G = Geo<R>::G;
    const uint32_t g = static_cast<uint32_t>((threadIdx.x & 31) / G);  // the tile: rotation of its slots
    uint32_t taken = 0;
    for (int64_t p = p0 + li; p < p1; p += 4 * G) {
        int32_t v[4];
        uint32_t j[4];
        bool ok[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int64_t q = p + G * k;
            ok[k] = q < p1;
            v[k] = ok[k] ? __ldg(&P.pv[q]) : 0;
            j[k] = ok[k] ? __ldg(&P.pj[q]) : 0u;
        }
        uint32_t x[4], lw[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (INIT)
                x[k] = ok[k] ? init_reg(P, Ys, v[k], j[k]) : 0u;
            else
                x[k] = ok[k] ? __ldg(&Mcur[static_cast<size_t>(v[k]) * R + j[k]]) : 0u;
            lw[k] = (ok[k] && !allL) ? Lcur[v[k] >> 5] : 0xFFFFFFFFu;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const bool in = ok[k] && ((lw[k] >> (v[k] & 31)) & 1u);
            taken += in ? 1u : 0u;
            if (in && x[k]) atomicMax(&acc32[sw_slot(j[k], g)], x[k]);
        }
    }
    return taken;
}

// The first sweep's sparse pairs [p0, p1): each pair's candidate is the initial rank of (v, j), kept per pair since
// sampling in one 16-bit word with the simulation's accumulator slot (pq, or the problem's copy pqb whose blocked
// pairs k_block_pairs set to rank 0), so one load serves a pair; a rank of 0 changes nothing.  Without pqb, a
// rebuild (chk) reads the pair's v too and a blocked (v, j) gives 0 (residual blocking; literal blocking keeps the
// rank).
template <int R, int NB = 4>
__device__ __forceinline__ void sparse_tile_init(const DevProb &P, int64_t p0, int64_t p1, bool chk,
                                                 uint32_t *acc32, int li) {
    constexpr int G = Geo<R>::G;
    const uint32_t tx = sw_tile(static_cast<uint32_t>((threadIdx.x & 31) / G));
    const uint16_t *pq = P.pqb ? P.pqb : P.pq;
    const bool test = chk && !P.literal && !P.pqb;
    for (int64_t p = p0 + li; p < p1; p += NB * G) {  // NB pair words a lane per round
        uint32_t x[NB];
#pragma unroll
        for (int k = 0; k < NB; ++k) {
            const int64_t q = p + G * k;
            x[k] = q < p1 ? __ldg(&pq[q]) : 0u;
        }
        if (test) {
#pragma unroll
            for (int k = 0; k < NB; ++k)
                if (x[k] >> 10) {
                    const int32_t v = __ldg(&P.pv[p + G * k]);
                    const uint32_t j = sw_slot(x[k] & 0x3FFu, 0);  // the slot map is its own inverse
                    if (test_bit(P.rany, v) && ((__ldg(&P.vis[static_cast<size_t>(v) * P.W + (j >> 5)]) >> (j & 31)) & 1u))
                        x[k] = 0;
                }
        }
#pragma unroll
        for (int k = 0; k < NB; ++k)
            if (x[k] >> 10) atomicMax(&acc32[(x[k] & 0x3FFu) ^ tx], x[k] >> 10);
    }
}

// Adds the tile's sparse accumulators into acc (ASSIGN: acc is still zero, so they are copied) and clears them:
// each lane clears exactly the chunks it read, so one barrier before (the tile's atomics are done) and one after
// (the zeros land before the next unit's atomics) suffice.
template <int R, bool ASSIGN = false>
__device__ __forceinline__ void fold_tile(uint32_t (&acc)[Geo<R>::CPL][4], uint32_t *acc32, unsigned tm, int li) {
    using Gm = Geo<R>;
    const int g = (threadIdx.x & 31) / Gm::G;
    __syncwarp(tm);
#pragma unroll
    for (int c = 0; c < Gm::CPL; ++c) {
        const int ch = li + Gm::G * c;
        uint4 *a = reinterpret_cast<uint4 *>(acc32 + 16 * ch);
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            const int pos = sw_pos(w, ch, g);  // slots laid out by sw_slot(j, g)
            const uint4 q = a[pos];
            const uint32_t x = q.x | (q.y << 8) | (q.z << 16) | (q.w << 24);
            acc[c][w] = ASSIGN ? x : vmax4(acc[c][w], x);
            a[pos] = make_uint4(0, 0, 0, 0);
        }
    }
    __syncwarp(tm);
}

// Literal blocking: a blocked (u, j) is never updated, so the merged registers lose u's blocked simulations.
template <int R>
__device__ __forceinline__ void drop_blocked(const DevProb &P, int64_t u, uint32_t (&acc)[Geo<R>::CPL][4], int li) {
    if (!P.literal || !P.rany || !test_bit(P.rany, u)) return;
#pragma unroll
    for (int c = 0; c < Geo<R>::CPL; ++c) {
        const uint32_t blk = blocked16(P, u, li + Geo<R>::G * c);
#pragma unroll
        for (int w = 0; w < 4; ++w) acc[c][w] &= ~nibble_bytes((blk >> (4 * w)) & 0xFu);
    }
}

// Row u's new registers max(M_u, acc) for a tile (every lane holds its chunks of acc and of the row's own
// registers in own): written to the next buffer if they changed or the row is in L, and u joins L'.  With Mother
// (the first sweep) the row is written to both buffers whatever it holds: nothing else initialises them.
template <int R>
__device__ __forceinline__ void finalize_tile(const DevProb &P, int64_t u, uint32_t (&acc)[Geo<R>::CPL][4],
                                              bool anyTaken, bool sync, const uint4 (&own)[Geo<R>::CPL],
                                              uint8_t *__restrict__ Mnext, uint8_t *__restrict__ Mother,
                                              uint32_t *__restrict__ Lnext, unsigned tm, int li, Stats &st) {
    using Gm = Geo<R>;
    if (!anyTaken && !sync && !Mother) return;
    bool diff = false;
    uint4 nw[Gm::CPL];
#pragma unroll
    for (int c = 0; c < Gm::CPL; ++c) {
        const uint4 o = own[c];
        nw[c] = make_uint4(vmax4(o.x, acc[c][0]), vmax4(o.y, acc[c][1]), vmax4(o.z, acc[c][2]),
                           vmax4(o.w, acc[c][3]));
        diff |= (nw[c].x != o.x) | (nw[c].y != o.y) | (nw[c].z != o.z) | (nw[c].w != o.w);
    }
    const bool changed = __any_sync(tm, diff);
    if (changed || sync || Mother) {
        uint4 *dst = reinterpret_cast<uint4 *>(Mnext + static_cast<size_t>(u) * R);
#pragma unroll
        for (int c = 0; c < Gm::CPL; ++c) dst[li + Gm::G * c] = nw[c];
    }
    if (P.gst && (changed || Mother)) {  // the row's register sum (its gain while M_S' is empty)
        uint32_t sum = 0;
#pragma unroll
        for (int c = 0; c < Gm::CPL; ++c) sum += byte_sum16(nw[c]);
        sum = __reduce_add_sync(tm, sum);
        if (li == 0) P.gst[u] = sum;
    }
    if (Mother) {  // the first sweep also records which registers it raised, for the push of the next sweep
        uint4 *dst = reinterpret_cast<uint4 *>(Mother + static_cast<size_t>(u) * R);
#pragma unroll
        for (int c = 0; c < Gm::CPL; ++c) {
            dst[li + Gm::G * c] = nw[c];
            P.dmask[static_cast<size_t>(u) * Gm::CH + li + Gm::G * c] =
                static_cast<uint16_t>(ne_bits16(nw[c], own[c]));
        }
    }
    if (changed && li == 0) set_bit(Lnext, u);
    st.bytes += Mother ? 2 * R + R / 8 : R + ((changed || sync) ? R : 0);
}

template <int R>
__device__ __forceinline__ void finalize_row_r(const DevProb &P, int64_t u, uint32_t (&acc)[Geo<R>::CPL][4],
                                               bool anyTaken, bool sync, const uint4 (&own)[Geo<R>::CPL],
                                               uint8_t *__restrict__ Mnext, uint8_t *__restrict__ Mother,
                                               uint32_t *__restrict__ Lnext, int lane, int g, int li, Stats &st) {
    using Gm = Geo<R>;
    if (!anyTaken && !sync && !Mother) return;
    bool diff = false;
    uint4 nw[Gm::CPL];
    if (g == 0) {
#pragma unroll
        for (int c = 0; c < Gm::CPL; ++c) {
            const uint4 o = own[c];
            nw[c] = make_uint4(vmax4(o.x, acc[c][0]), vmax4(o.y, acc[c][1]), vmax4(o.z, acc[c][2]),
                               vmax4(o.w, acc[c][3]));
            diff |= (nw[c].x != o.x) | (nw[c].y != o.y) | (nw[c].z != o.z) | (nw[c].w != o.w);
        }
    }
    const bool changed = __any_sync(kFull, diff);
    if (g == 0 && (changed || sync || Mother)) {
        uint4 *dst = reinterpret_cast<uint4 *>(Mnext + static_cast<size_t>(u) * R);
#pragma unroll
        for (int c = 0; c < Gm::CPL; ++c) dst[li + Gm::G * c] = nw[c];
    }
    if (P.gst && (changed || Mother)) {  // the row's register sum (its gain while M_S' is empty)
        uint32_t sum = 0;
        if (g == 0) {
#pragma unroll
            for (int c = 0; c < Gm::CPL; ++c) sum += byte_sum16(nw[c]);
        }
        sum = __reduce_add_sync(kFull, sum);
        if (lane == 0) P.gst[u] = sum;
    }
    if (g == 0 && Mother) {
        uint4 *dst = reinterpret_cast<uint4 *>(Mother + static_cast<size_t>(u) * R);
#pragma unroll
        for (int c = 0; c < Gm::CPL; ++c) {
            dst[li + Gm::G * c] = nw[c];
            P.dmask[static_cast<size_t>(u) * Gm::CH + li + Gm::G * c] =
                static_cast<uint16_t>(ne_bits16(nw[c], own[c]));
        }
    }
    if (changed && lane == 0) set_bit(Lnext, u);
    st.bytes += Mother ? 2 * R + R / 8 : R + ((changed || sync) ? R : 0);
}

// finalize_row_r with the row's own registers read from ownp, or, in the first sweep of a diffusion (init), formed
// as initial ranks and written to both buffers (Mother).
template <int R>
__device__ __forceinline__ void finalize_row_g(const DevProb &P, int64_t u, uint32_t (&acc)[Geo<R>::CPL][4],
                                               bool anyTaken, bool sync, const uint4 *ownp, bool init,
                                               uint8_t *__restrict__ Mnext, uint8_t *__restrict__ Mother,
                                               uint32_t *__restrict__ Lnext, int lane, int g, int li, Stats &st) {
    using Gm = Geo<R>;
    if (!anyTaken && !sync && !init) return;
    uint4 own[Gm::CPL];
    const uint32_t hv = vertex_hash(static_cast<uint32_t>(u));
#pragma unroll
    for (int c = 0; c < Gm::CPL; ++c) {
        const int ch = li + Gm::G * c;
        own[c] = g != 0 ? make_uint4(0, 0, 0, 0) : (init ? init_chunk(P.Y, hv, ch, init_blocked16(P, u, ch)) : ownp[ch]);
    }
    drop_blocked<R>(P, u, acc, li);
    finalize_row_r<R>(P, u, acc, anyTaken, sync, own, Mnext, init ? Mother : nullptr, Lnext, lane, g, li, st);
}

// Work of a full sweep: every light row that has out-edges (static list) and every task of every split row.
struct SweepWork {
    uint64_t nlight, ntask;
    const int32_t *rows;
};

__device__ __forceinline__ SweepWork sweep_work(const DevProb &P) {
    SweepWork w;
    w.nlight = static_cast<uint64_t>(P.n_light);
    w.ntask = static_cast<uint64_t>(P.n_tasks);
    w.rows = P.light_list;
    return w;
}

// Index of sweep unit l in the descriptor arrays: a row id (l < nlight) or a task id.
__device__ __forceinline__ int64_t unit_id(const SweepWork &W, uint64_t l) {
    return l < W.nlight ? (W.rows ? static_cast<int64_t>(W.rows[l]) : static_cast<int64_t>(l))
                        : static_cast<int64_t>(l - W.nlight);
}

// A pulling sweep of one problem over this tile's units.  INIT: the first sweep of a diffusion (t = 0), which
// forms the initial registers itself (Algorithm 1's initialisation fused into the first Simulate sweep) and writes
// every row to both register buffers.
template <int R, bool INIT>
__device__ void prop_problem_t(const DevProb &P, uint32_t t, const SweepWork &W, uint64_t cnt, uint64_t first,
                               uint64_t nworkers, unsigned tm, int li, uint32_t *acc32, const uint32_t *Ys) {
    using Gm = Geo<R>;
    const bool par = t & 1u;
    const uint8_t *Mcur = par ? P.M1 : P.M0;
    uint8_t *Mnext = par ? P.M0 : P.M1;
    uint8_t *Mother = INIT ? (par ? P.M1 : P.M0) : nullptr;
    const uint32_t *Lcur = par ? P.Lb1 : P.Lb0;
    uint32_t *Lnext = par ? P.Lb0 : P.Lb1;
    const bool allL = (t == 0);
    const uint64_t tb = thr_bytes(P.model);
    Stats st;
    // two-stage prefetch over this tile's units: the descriptor of the next unit and the id of the one after it
    // are loaded while the current unit is processed
    int64_t id_next = first + nworkers < cnt ? unit_id(W, first + nworkers) : 0;
    UnitD cur{};
    int64_t cur_id = 0;
    if (first < cnt) {
        cur_id = unit_id(W, first);
        cur = first < W.nlight ? P.rdesc[cur_id] : P.tdesc[cur_id];
    }
    for (uint64_t l = first; l < cnt; l += nworkers) {
        UnitD nxt{};
        const int64_t nxt_id = id_next;
        if (l + nworkers < cnt) nxt = l + nworkers < W.nlight ? P.rdesc[id_next] : P.tdesc[id_next];
        if (l + 2 * nworkers < cnt) id_next = unit_id(W, l + 2 * nworkers);
        const bool is_row = l < W.nlight;
        if (INIT && is_row && cur.u < 0) {  // a split row: its tasks and the combine kernels finish it
            cur = nxt;
            cur_id = nxt_id;
            continue;
        }
        const int64_t u = cur.u;
        uint4 own[Gm::CPL];
        const uint32_t hu = INIT ? vertex_hash(static_cast<uint32_t>(u)) : 0u;
#pragma unroll
        for (int c = 0; c < Gm::CPL; ++c) {
            const int ch = li + Gm::G * c;
            if (INIT)
                own[c] = is_row ? init_chunk_sw(Ys, hu, ch, init_blocked16(P, u, ch)) : make_uint4(0, 0, 0, 0);
            else
                own[c] = is_row ? __ldg(reinterpret_cast<const uint4 *>(Mcur + static_cast<size_t>(u) * R) + ch)
                                : make_uint4(0, 0, 0, 0);
        }
        uint32_t acc[Gm::CPL][4];
#pragma unroll
        for (int c = 0; c < Gm::CPL; ++c)
#pragma unroll
            for (int w = 0; w < 4; ++w) acc[c][w] = 0;
        // the first sweep of a rebuild tests its pairs' neighbours for blocked simulations (none before a search)
        const bool chk = INIT && P.rany && P.ctr->lvl != 0;
        uint32_t nPairs = 0;
        if (cur.np > 0) {
            if (INIT) {
                sparse_tile_init<R>(P, cur.p0, cur.p0 + cur.np, chk, acc32, li);
                nPairs = cur.np;
            } else {
                nPairs = sparse_tile<R, INIT>(P, cur.p0, cur.p0 + cur.np, allL, Lcur, Mcur, Ys, acc32, li);
                nPairs = __reduce_add_sync(tm, nPairs);
            }
            fold_tile<R, true>(acc, acc32, tm, li);
        }
        const uint32_t nTaken =
            cur.nd > 0 ? dense_tile<R, INIT>(P, cur.d0, cur.d0 + cur.nd, allL, Lcur, Mcur, Ys, chk, acc, li) : 0u;
        // modelled bytes: descriptor, pair records, the registers pairs read (computed in the first sweep), dense
        // edges (id, target, threshold) and their rows (masks only in the first sweep)
        if (li == 0)
            st.pairs += cur.np;
        if (li == 0)
            st.bytes += 32 + 6 * static_cast<uint64_t>(cur.np) + (INIT ? 0u : nPairs) +
                        (8 + tb + (INIT ? R / 8 : 0)) * static_cast<uint64_t>(cur.nd) +
                        (INIT ? 0u : static_cast<uint64_t>(nTaken) * R);
        const bool any = nPairs + nTaken > 0;
        if (is_row) {
            drop_blocked<R>(P, u, acc, li);
            finalize_tile<R>(P, u, acc, any, !INIT && test_bit(Lcur, u), own, Mnext, Mother, Lnext, tm, li, st);
        } else if (any) {
            const int64_t task = cur_id;
            uint4 *dst = reinterpret_cast<uint4 *>(P.part + static_cast<size_t>(task) * R);
#pragma unroll
            for (int c = 0; c < Gm::CPL; ++c)
                dst[li + Gm::G * c] = make_uint4(acc[c][0], acc[c][1], acc[c][2], acc[c][3]);
            if (li == 0) {
                set_bit(P.part_any, task);
                st.bytes += R;
            }
        }
        cur = nxt;
        cur_id = nxt_id;
    }
    flush_stats(P.ctr, st, li);
}

// Row u of the first sweep: M_u = max(initial ranks own, merged acc), written to both register buffers, with its
// change mask (the registers raised above their initial rank, which the next sweep pushes); u joins L' if any
// register rose.  Per byte, own + 128 - acc has bit 7 set exactly where own >= acc (every register is <= 32, so no
// byte borrows): one word gives both the max and the change bits.
template <int R>
__device__ __forceinline__ void finalize_first(const DevProb &P, int64_t u, const uint32_t (&acc)[Geo<R>::CPL][4],
                                               const uint4 (&own)[Geo<R>::CPL], uint32_t *__restrict__ Lnext,
                                               uint32_t *__restrict__ gst, unsigned tm, int li) {
    using Gm = Geo<R>;
    uint32_t any = 0, sum = 0;
#pragma unroll
    for (int c = 0; c < Gm::CPL; ++c) {
        const int ch = li + Gm::G * c;
        const uint32_t o[4] = {own[c].x, own[c].y, own[c].z, own[c].w};
        uint32_t nw[4], bits = 0;
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            const uint32_t x = o[w] + 0x80808080u - acc[c][w];
            const uint32_t ge = sign_bytes(x, 0u, 0xBA98u);
            nw[w] = (o[w] & ge) | (acc[c][w] & ~ge);
            bits |= ((((~x >> 7) & 0x01010101u) * 0x01020408u) >> 24) << (4 * w);
        }
        const uint4 v = make_uint4(nw[0], nw[1], nw[2], nw[3]);
        reinterpret_cast<uint4 *>(P.M1 + static_cast<size_t>(u) * R)[ch] = v;
        reinterpret_cast<uint4 *>(P.M0 + static_cast<size_t>(u) * R)[ch] = v;
        P.dmask[static_cast<size_t>(u) * Gm::CH + ch] = static_cast<uint16_t>(bits);
        any |= bits;
        sum += byte_sum16(v);
    }
    if (__any_sync(tm, any != 0u) && li == 0) set_bit(Lnext, u);
    if (gst) {  // the row's register sum (its gain while M_S' is empty)
        sum = __reduce_add_sync(tm, sum);
        if (li == 0) gst[u] = sum;
    }
}

// The first sweep of one problem over this tile's units, software-pipelined: while a unit is processed, the pair
// records and ranks of the next unit's first 4 G pairs and the descriptor of the unit after it are already in
// flight, so the chain descriptor -> pairs -> merge of one unit overlaps the previous one.  The tile takes the rows
// first, dealt round-robin from row `first` on (rows have at most kHeavyDeg out-edges, so the deal is even), then
// tasks from the problem's shared counter until none is left: tasks differ in length (a hub's tasks are up to
// kMaxTaskEdges edges), and whichever tile is free takes the next one.  The counter is read one unit ahead of the
// descriptor load it feeds.  The descriptors wait in a per-tile ring of three in shared memory (ring: 3 x 8 words,
// 16-byte aligned), loaded a word a lane, and each prefetched pair is its 16-bit word (slot, rank), to keep the
// registers few.  A row's own initial registers come from the problem's table Mi (loaded before the merges, used
// after them).
template <int R>
__device__ void first_problem_t(const DevProb &P, uint64_t first, uint64_t nworkers, unsigned tm, int li,
                                uint32_t *acc32, uint32_t *ring) {
    using Gm = Geo<R>;
    constexpr int G = Gm::G;
    constexpr int DW = sizeof(UnitD) / 4;  // descriptor words
    constexpr int NW = (DW + G - 1) / G;   // descriptor words a lane moves
    static_assert(DW == 8, "descriptor of 8 words");
    const uint64_t n = static_cast<uint64_t>(P.n);
    const uint64_t nt = static_cast<uint64_t>(P.n_tasks);
    // unit ids: x < n row x, n <= x < n + nt task x - n, kEnd none left (n + nt < 2^32 - 1, checked at graph set-up)
    constexpr uint32_t kEnd = 0xFFFFFFFFu;
    const int lead = static_cast<int>(threadIdx.x & 31) - li;  // the tile's first lane
    // the tile's unit sequence: the next row of its deal, then the counter's next task (its atomic issued by
    // issue(), its value read by resolve() one unit later)
    uint32_t sx = static_cast<uint32_t>(first);
    bool ended = false, dyn = false;
    uint32_t pend = 0;  // the issued unit: a row id, or (dyn) the counter's value in the tile's first lane
    auto issue = [&]() {
        dyn = false;
        pend = kEnd;
        if (sx < n) {
            pend = sx;
            sx += static_cast<uint32_t>(nworkers);
        } else if (!ended) {
            dyn = true;
            if (li == 0) pend = atomicAdd(&P.ctr->task_next, 1u);
        }
    };
    auto resolve = [&]() -> uint32_t {
        if (!dyn) return pend;
        const uint32_t k = __shfl_sync(tm, pend, lead);
        if (k >= nt) {
            ended = true;
            return kEnd;
        }
        return static_cast<uint32_t>(n) + k;
    };
    const uint64_t tb = thr_bytes(P.model);
    const uint16_t *pq = P.pqb ? P.pqb : P.pq;
    uint32_t *const gst = P.gst;
    const bool rebuild = P.rany && P.ctr->lvl != 0;  // some vertices are blocked
    // a rebuild without the problem's own blocked ranks tests each pair's neighbour (residual blocking only)
    const bool test = rebuild && !P.pqb && !P.literal;
    const bool keep_own = rebuild && P.literal;  // literal blocking: a blocked register is never raised
    const uint32_t tx = sw_tile(static_cast<uint32_t>((threadIdx.x & 31) / G));  // this tile's slot permutation
    unsigned long long pairs = 0, bytes = 0;  // counted by lane 0 of the tile
    // this lane's words (li, li + G, ...) of the descriptor of unit x (zeros for kEnd)
    auto load_desc = [&](uint32_t x, uint32_t (&w)[NW]) {
        const uint32_t *src = x != kEnd ? reinterpret_cast<const uint32_t *>(x < n ? P.rdesc + x : P.tdesc + (x - n))
                                        : nullptr;
#pragma unroll
        for (int k = 0; k < NW; ++k) {
            const int wi = li + G * k;
            w[k] = (src && wi < DW) ? __ldg(src + wi) : 0u;
        }
    };
    auto store_desc = [&](int slot, const uint32_t (&w)[NW]) {
#pragma unroll
        for (int k = 0; k < NW; ++k) {
            const int wi = li + G * k;
            if (wi < DW) ring[slot * DW + wi] = w[k];
        }
    };
    struct D {
        int64_t p0, d0;
        uint32_t np, nd;
        int32_t u;
        uint32_t hu;
    };
    auto read_desc = [&](int slot) {
        const uint4 *r = reinterpret_cast<const uint4 *>(ring + slot * DW);
        const uint4 a = r[0], b = r[1];
        D d;
        d.p0 = static_cast<int64_t>((static_cast<uint64_t>(a.y) << 32) | a.x);
        d.d0 = static_cast<int64_t>((static_cast<uint64_t>(a.w) << 32) | a.z);
        d.np = b.x;
        d.nd = b.y;
        d.u = static_cast<int32_t>(b.z);
        d.hu = b.w;
        return d;
    };
    // the first 4 G pair words of unit d, this lane's share (rank 0 past the unit's end)
    auto batch = [&](const D &d, uint32_t (&b)[4]) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const uint32_t o = li + G * k;
            b[k] = o < d.np ? static_cast<uint32_t>(__ldg(&pq[d.p0 + o])) : 0u;
        }
    };
    issue();
    uint32_t x0 = resolve();  // the current unit (row `first`)
    issue();
    uint32_t x1 = resolve();  // the next one
    issue();
    uint32_t x2 = resolve();  // the one after it
    issue();                  // and the one after that, resolved at the end of the first round
    {
        uint32_t w[NW];
        load_desc(x0, w);
        store_desc(0, w);
        load_desc(x1, w);
        store_desc(1, w);
    }
    __syncwarp(tm);
    int slot = 0;  // ring slot of the current unit; slot + 1 holds the next one
    uint32_t cb[4];
    batch(read_desc(0), cb);
    while (x0 != kEnd) {
        const int s1 = slot == 2 ? 0 : slot + 1, s2 = s1 == 2 ? 0 : s1 + 1;
        const D cur = read_desc(slot);
        uint32_t nb[4];
        batch(read_desc(s1), nb);                 // the next unit's first pairs
        uint32_t wn[NW];
        load_desc(x2, wn);                        // and the descriptor after it
        const uint32_t x = x0;
        const bool is_row = x < n;
        if (!(is_row && cur.u < 0)) {  // a split row is left to its tasks and the combine kernels
            // the row's initial registers (blocked ones 0 under residual blocking), loaded before the merges
            uint4 own[Gm::CPL];
#pragma unroll
            for (int c = 0; c < Gm::CPL; ++c)
                own[c] = is_row ? __ldg(reinterpret_cast<const uint4 *>(P.Mi + static_cast<size_t>(cur.u) * R) + li + G * c)
                                : make_uint4(0, 0, 0, 0);
            uint32_t acc[Gm::CPL][4];
#pragma unroll
            for (int c = 0; c < Gm::CPL; ++c)
#pragma unroll
                for (int w = 0; w < 4; ++w) acc[c][w] = 0;
            if (cur.np > 0) {
                // a unit's pairs past its first 4 G take 8 words a lane per round: hub tasks of hundreds of pairs
                // then wait for fewer rounds of loads
                if (test) {
                    sparse_tile_init<R, 8>(P, cur.p0, cur.p0 + cur.np, true, acc32, li);
                } else {
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        if (cb[k] >> 10) atomicMax(&acc32[(cb[k] & 0x3FFu) ^ tx], cb[k] >> 10);
                    if (cur.np > 4 * G) sparse_tile_init<R, 8>(P, cur.p0 + 4 * G, cur.p0 + cur.np, false, acc32, li);
                }
                fold_tile<R, true>(acc, acc32, tm, li);
            }
            if (cur.nd > 0)
                dense_tile<R, true>(P, cur.d0, cur.d0 + cur.nd, true, nullptr, nullptr, nullptr, rebuild, acc, li);
            // modelled bytes: descriptor, pair words (slot, rank), dense edges (id, target, threshold, mask, the
            // neighbour's initial row), and the row's initial registers read and the row written to both buffers
            // with its change mask and register sum (or a task's partial row)
            if (li == 0) {
                pairs += cur.np;
                bytes += 32 + 2 * static_cast<uint64_t>(cur.np) + (8 + tb + R / 8 + R) * static_cast<uint64_t>(cur.nd) +
                         (is_row ? 3 * R + R / 8 + (gst ? 4 : 0) : (cur.np + cur.nd > 0 ? R : 0));
            }
            if (is_row) {
                const int64_t u = cur.u;
                if (keep_own) drop_blocked<R>(P, u, acc, li);
                finalize_first<R>(P, u, acc, own, P.Lb1, gst, tm, li);
            } else if (cur.np + cur.nd > 0) {
                const int64_t task = static_cast<int64_t>(x - n);
                uint4 *dst = reinterpret_cast<uint4 *>(P.part + static_cast<size_t>(task) * R);
#pragma unroll
                for (int c = 0; c < Gm::CPL; ++c)
                    dst[li + G * c] = make_uint4(acc[c][0], acc[c][1], acc[c][2], acc[c][3]);
                if (li == 0) set_bit(P.part_any, task);
            }
        }
        store_desc(s2, wn);  // the unit after next goes to the free slot (read as the next unit from next round)
        __syncwarp(tm);
        slot = s1;
#pragma unroll
        for (int k = 0; k < 4; ++k) cb[k] = nb[k];
        x0 = x1;
        x1 = x2;
        x2 = resolve();
        issue();
    }
    if (li == 0 && bytes) {
        atomicAdd(&P.ctr->first_bytes, bytes);
        atomicAdd(&P.ctr->bytes, bytes);
        atomicAdd(&P.ctr->pairs, pairs);
    }
}

// The partial rows of tasks [a, b) (b - a <= 32) that merged something: their part_any bits are consumed and the
// rows are gathered into shared memory, N at a time, and max-merged into acc.  Returns whether any was present.
template <int R>
__device__ __forceinline__ bool merge_partials(const DevProb &P, int64_t a, int64_t b,
                                               uint32_t (&acc)[Geo<R>::CPL][4], int lane, int g, int li,
                                               WarpStage &sw, uint4 *buf, Stats &st, uint32_t &phase,
                                               bool &aborted) {
    using Gm = Geo<R>;
    constexpr int N = GSlots<R>::N;
    const int64_t k = a + lane;
    const bool mine = k < b && test_bit(P.part_any, k);
    const unsigned m = __ballot_sync(kFull, mine);
    if (m == 0) return false;
    if (mine) {
        atomicAnd(&P.part_any[k >> 5], ~(1u << (k & 31)));
        sw.v[__popc(m & ((1u << lane) - 1u))] = lane;
    }
    __syncwarp();
    const int cnt = __popc(m);
    for (int i0 = 0; i0 < cnt; i0 += N) {
        const int nb = min(N, cnt - i0);
        __syncwarp();
        fence_async_smem();
        if (aborted) return true;
        if (lane == 0) mbar_expect(&sw.mbar, static_cast<uint32_t>(nb * R));
        __syncwarp();
        if (lane < nb)
            bulk_g2s(&buf[lane * Gm::CH], P.part + static_cast<size_t>(a + sw.v[i0 + lane]) * R, R, &sw.mbar);
        if (!mbar_wait(&sw.mbar, phase, &P.ctr->fault, aborted)) return true;
        phase ^= 1u;
        for (int sl = g; sl < nb; sl += Gm::NG) {
#pragma unroll
            for (int c = 0; c < Gm::CPL; ++c) {
                const uint4 x = buf[sl * Gm::CH + li + Gm::G * c];
                acc[c][0] = vmax4(acc[c][0], x.x);
                acc[c][1] = vmax4(acc[c][1], x.y);
                acc[c][2] = vmax4(acc[c][2], x.z);
                acc[c][3] = vmax4(acc[c][3], x.w);
            }
        }
        __syncwarp();
    }
    if (lane == 0) st.bytes += static_cast<uint64_t>(cnt) * R;
    return true;
}

// Split rows of a full sweep with at most kBigTasks tasks (one warp each) or more (one block each); a push sweep
// has none.
__device__ __forceinline__ uint64_t heavy_count(const DevProb &P, const DevCtr &C, bool big, const int32_t *&list) {
    list = big ? P.hbig : P.hsmall;
    if (!C.full) return 0;
    return static_cast<uint64_t>(big ? P.n_hbig : P.n_hsmall);
}

}  // namespace

// Bytewise max-merge of cand into the register word at w, lock-free, starting from the value old read there:
// returns whether the word grew.  A failed compare-and-swap means another thread grew the word first; words only
// grow (four registers of at most 33 values), so the retries are few; after `limit` tries the fault flag is raised.
__device__ __forceinline__ bool word_max(uint32_t *w, uint32_t old, uint32_t cand, unsigned int *fault,
                                         uint32_t limit) {
    for (uint32_t it = 0; it < limit; ++it) {
        const uint32_t nw = vmax4(old, cand);
        if (nw == old) return false;
        const uint32_t prev = atomicCAS(w, old, nw);
        if (prev == old) return true;
        old = prev;
    }
    atomicOr(fault, 2u);
    return false;
}


// A push sweep (Algorithm 2 with a small L, in the other direction): every changed vertex v merges M_v into the
// rows of its in-neighbours u, M'_u[j] = max(M'_u[j], M_v[j]) for every sampled (u, v, j).  The next buffer already
// holds M_u for every row (rows of L were copied after the previous sweep), so it is updated in place with
// compare-and-swap; reads come from the current buffer only (Jacobi).  A whole warp takes one unit, a changed
// vertex or a chunk of kPushChunk in-edges of one with more (tiles of one warp busy with units of different shapes
// would run their divergent paths one after the other); the change mask of v is staged in shared memory (after R
// bytes of the warp's area, which this path leaves unused), and a lane holds its chunks of M_v in registers for the
// dense in-edges.  Pairs take all 32 lanes, four per lane in flight; dense in-edges are merged by the warp's NG lane
// groups, two per group a round.
template <int R>
__device__ void push_problem_w(const DevProb &P, uint32_t t, uint64_t cnt, uint64_t first, uint64_t nworkers,
                               int lane, uint32_t *warp_smem) {
    using Gm = Geo<R>;
    constexpr int G = Gm::G, NG = Gm::NG;
    constexpr int W = R / 32;
    const int g = lane / G, li = lane % G;
    const unsigned tm = tile_mask<R>(g);
    const bool par = t & 1u;
    const uint8_t *Mcur = par ? P.M1 : P.M0;
    uint8_t *Mnext = par ? P.M0 : P.M1;
    uint32_t *Lnext = par ? P.Lb0 : P.Lb1;
    uint16_t *sdel = reinterpret_cast<uint16_t *>(warp_smem + R / 4);  // M_v's changed registers, per chunk
    unsigned int *fault = &P.ctr->fault;
    const uint32_t lim = P.cas_limit;
    const uint64_t nl = P.ctr->npush_l;
    Stats st;
    // the vertex and descriptor of a light unit are loaded one unit ahead, so that the next unit's dependent loads
    // overlap this unit's work
    int64_t vn = 0;
    UnitD dn{};
    if (first < cnt && first < nl) {
        vn = P.chg_list[first];
        dn = P.vdesc[vn];
    }
    for (uint64_t l = first; l < cnt; l += nworkers) {
        int64_t v, p0, p1, d0, d1;
        if (l < nl) {
            v = vn;
            p0 = dn.p0;
            p1 = dn.p0 + dn.np;
            d0 = dn.d0;
            d1 = dn.d0 + dn.nd;
        } else {
            const uint64_t h = P.chg_hc[l - nl];
            v = static_cast<int64_t>(static_cast<uint32_t>(h));
            const int64_t k0 = __ldg(&P.xadj_in[v]) + static_cast<int64_t>(h >> 32) * kPushChunk;
            const int64_t end = __ldg(&P.xadj_in[v + 1]);
            const int64_t k1 = end - k0 > kPushChunk ? k0 + kPushChunk : end;
            p0 = __ldg(&P.ipofs[k0]);
            p1 = __ldg(&P.ipofs[k1]);
            d0 = __ldg(&P.idofs[k0]);
            d1 = __ldg(&P.idofs[k1]);
        }
        if (l + nworkers < cnt && l + nworkers < nl) {
            vn = P.chg_list[l + nworkers];
            dn = P.vdesc[vn];
        }
        // Stage the registers of v that the previous sweep changed (recorded by that sweep's first pass, or by the
        // frontier pass that copied the row): only those can raise an in-neighbour (M_u[j] >= the previous sweep's
        // M_v[j] holds for every live (u, v) after the first sweep), so pairs of other simulations are skipped and
        // a pair of a changed one reads M_v[j] itself.
        const uint8_t *vbytes = Mcur + static_cast<size_t>(v) * R;
        const uint4 *vrow = reinterpret_cast<const uint4 *>(vbytes);
        for (int c = lane; c < Gm::CH; c += 32) sdel[c] = __ldg(&P.dmask[static_cast<size_t>(v) * Gm::CH + c]);
        uint4 rowc[Gm::CPL];  // this lane's chunks of M_v, for the dense in-edges
        const bool dense = d1 > d0;
#pragma unroll
        for (int c = 0; c < Gm::CPL; ++c) rowc[c] = dense ? __ldg(vrow + li + G * c) : make_uint4(0, 0, 0, 0);
        __syncwarp();
        uint32_t nproc = 0;  // pairs of changed registers (the others cost only their record)
        for (int64_t p = p0 + lane; p < p1; p += 128) {
            uint32_t *addr[4];
            uint32_t jj[4], old[4], x[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int64_t q = p + 32 * k;
                addr[k] = nullptr;
                jj[k] = 0;
                if (q < p1) {
                    const int64_t u = __ldg(&P.iu[q]);
                    const uint32_t j = __ldg(&P.ij[q]);
                    if (((sdel[j >> 4] >> (j & 15)) & 1u) && !literal_blocked(P, u, j)) {
                        jj[k] = j;
                        addr[k] = reinterpret_cast<uint32_t *>(Mnext + static_cast<size_t>(u) * R + (j & ~3u));
                        ++nproc;
                    }
                }
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {  // the candidate register and the target word, loaded together
                x[k] = addr[k] ? __ldg(vbytes + jj[k]) : 0u;
                old[k] = addr[k] ? __ldcg(addr[k]) : 0u;
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const uint32_t cand = x[k] << (8 * (jj[k] & 3));
                if (cand && word_max(addr[k], old[k], cand, fault, lim))
                    set_bit(Lnext, (reinterpret_cast<uint8_t *>(addr[k]) - Mnext) / R);
            }
        }
        // dense in-edges: the warp fetches up to 32 of them at once; group g merges edges i + g and i + NG + g
        for (int64_t db = d0; db < d1; db += 32) {
            const int nb = d1 - db < 32 ? static_cast<int>(d1 - db) : 32;
            int32_t my_u = 0;
            uint32_t my_e = 0;
            if (lane < nb) {
                my_u = __ldg(&P.idu[db + lane]);
                my_e = __ldg(&P.ide[db + lane]);
            }
            for (int i = 0; i < nb; i += 2 * NG) {
                int32_t u[2];
                bool ok[2], grew[2] = {false, false};
                uint32_t m[2][Gm::CPL];
                uint4 o[2][Gm::CPL];
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    const int ii = i + g + r * NG;
                    ok[r] = ii < nb;
                    u[r] = __shfl_sync(kFull, my_u, ok[r] ? ii : 0);
                    const uint32_t e = __shfl_sync(kFull, my_e, ok[r] ? ii : 0);
#pragma unroll
                    for (int c = 0; c < Gm::CPL; ++c) {
                        const int ch = li + G * c;
                        m[r][c] = ok[r] ? (__ldg(&P.live[static_cast<size_t>(e) * W + (ch >> 1)]) >> (16 * (ch & 1))) &
                                              sdel[ch]
                                        : 0u;
                        if (m[r][c] && P.literal) m[r][c] &= ~blocked16(P, u[r], ch);
                        o[r][c] = m[r][c] ? __ldcg(reinterpret_cast<const uint4 *>(Mnext + static_cast<size_t>(u[r]) * R) +
                                                   ch)
                                          : make_uint4(0, 0, 0, 0);
                    }
                }
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    if (ok[r]) {
#pragma unroll
                        for (int c = 0; c < Gm::CPL; ++c) {
                            uint32_t *dst = reinterpret_cast<uint32_t *>(Mnext + static_cast<size_t>(u[r]) * R) +
                                            4 * (li + G * c);
                            const uint32_t mm = m[r][c];
                            grew[r] |= word_max(dst + 0, o[r][c].x, rowc[c].x & nibble_bytes(mm & 0xFu), fault,
                                                lim);
                            grew[r] |= word_max(dst + 1, o[r][c].y, rowc[c].y & nibble_bytes((mm >> 4) & 0xFu), fault,
                                                lim);
                            grew[r] |= word_max(dst + 2, o[r][c].z, rowc[c].z & nibble_bytes((mm >> 8) & 0xFu), fault,
                                                lim);
                            grew[r] |= word_max(dst + 3, o[r][c].w, rowc[c].w & nibble_bytes((mm >> 12) & 0xFu), fault,
                                                lim);
                        }
                    }
                    if (__any_sync(tm, grew[r]) && li == 0) set_bit(Lnext, u[r]);
                }
            }
        }
        nproc = __reduce_add_sync(kFull, nproc);
        // modelled bytes: list entry and descriptor, the change mask, pair records, per pair of a changed register
        // the register and the target word, and with dense in-edges M_v plus per edge its ids, mask and target row
        if (lane == 0)
            st.pairs += static_cast<uint64_t>(p1 - p0);
        if (lane == 0)
            st.bytes += 36 + R / 8 + 6 * static_cast<uint64_t>(p1 - p0) + 5 * static_cast<uint64_t>(nproc) +
                        (dense ? R : 0) + (12 + W * 4 + R) * static_cast<uint64_t>(d1 - d0);
        __syncwarp();
    }
    // the staged masks may share the sparse accumulators, which a pulling unit of another problem in the same
    // launch expects to find zero
    for (int k = lane; k < R / 4 + R / 32; k += 32) warp_smem[k] = 0u;
    __syncwarp();
    if (st.bytes) atomicAdd(&P.ctr->bytes, st.bytes);
    if (st.pairs) atomicAdd(&P.ctr->pairs, st.pairs);
}

// A push sweep over a large L as one stream of in-pairs (sampled graphs without dense edges): every in-pair
// (u, v, j) in in-CSR order, 128 a warp at a time, merges M_v[j] into the next buffer's M_u[j] when v is in L and
// the previous sweep changed (v, j) (the same skip as push_problem_w; dmask of every listed v, or of every row after
// the first sweep, is current).  The pair records and the change masks of consecutive pairs are coalesced, and
// consecutive pairs share v, so M_v[j] is read from a row the warp just touched.  Few pairs pass (a few percent in
// sweep 1), so each passing pair (u, j, M_v[j]) goes to a per-warp queue in shared memory, and the warp updates the
// target words 32 at a time, one a lane: the random read and compare-and-swap of each target word then run with
// the whole warp's in flight instead of one or two lanes' per item.
constexpr int kPushQueue = 64;  // queue entries a warp (at most 31 left over plus 32 of one record slot)

template <int R>
__device__ void push_stream_w(const DevProb &P, uint32_t t, uint64_t cnt, uint64_t first, uint64_t nworkers,
                              int lane, uint2 *queue) {
    constexpr int CH = R / 16;
    const bool par = t & 1u;
    const uint8_t *Mcur = par ? P.M1 : P.M0;
    uint8_t *Mnext = par ? P.M0 : P.M1;
    const uint32_t *Lcur = par ? P.Lb1 : P.Lb0;
    uint32_t *Lnext = par ? P.Lb0 : P.Lb1;
    unsigned int *fault = &P.ctr->fault;
    const uint32_t lim = P.cas_limit;
    const uint64_t npairs = static_cast<uint64_t>(P.ipofs[P.m]);
    const uint32_t lt = (1u << lane) - 1u;
    uint32_t nproc = 0, nrec = 0;
    uint32_t head = 0, count = 0;  // the queue's first entry and length (the same in every lane)
    // the 32 queued entries from head on, one a lane (or the first n of them): target word max-merge
    auto drain = [&](uint32_t n) {
        __syncwarp();
        if (static_cast<uint32_t>(lane) < n) {
            const uint2 e = queue[(head + lane) % kPushQueue];
            const int32_t u = static_cast<int32_t>(e.x);
            const uint32_t j = e.y & 0xFFFFu, x = e.y >> 16;
            if (!literal_blocked(P, u, j)) {
                ++nproc;
                uint32_t *addr = reinterpret_cast<uint32_t *>(Mnext + static_cast<size_t>(u) * R + (j & ~3u));
                if (word_max(addr, __ldcg(addr), x << (8 * (j & 3)), fault, lim)) set_bit(Lnext, u);
            }
        }
        head = (head + n) % kPushQueue;
        count -= n;
        __syncwarp();
    };
    // the records of the next item are loaded while this one is processed
    int32_t nv[4];
    uint32_t nj[4];
    auto fetch = [&](uint64_t l) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const uint64_t q = l * 128 + 32 * k + lane;
            const bool ok = l < cnt && q < npairs;
            nv[k] = ok ? __ldg(&P.iv[q]) : -1;
            nj[k] = ok ? __ldg(&P.ij[q]) : 0u;
        }
    };
    fetch(first);
    for (uint64_t l = first; l < cnt; l += nworkers) {
        int32_t cv[4];
        uint32_t cj[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            cv[k] = nv[k];
            cj[k] = nj[k];
        }
        fetch(l + nworkers);
        bool go[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            go[k] = false;
            if (cv[k] >= 0) {
                ++nrec;
                const int32_t v = cv[k];
                const uint32_t j = cj[k];
                const bool inL = t == 1 || test_bit(Lcur, v);
                go[k] = inL && ((__ldg(&P.dmask[static_cast<size_t>(v) * CH + (j >> 4)]) >> (j & 15)) & 1u);
            }
        }
        // a passing pair's source u and candidate register M_v[j] (a changed register is never 0)
        uint32_t cu[4], cx[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            cu[k] = go[k] ? static_cast<uint32_t>(__ldg(&P.iu[l * 128 + 32 * k + lane])) : 0u;
            cx[k] = go[k] ? static_cast<uint32_t>(__ldg(Mcur + static_cast<size_t>(cv[k]) * R + cj[k])) : 0u;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const unsigned m = __ballot_sync(kFull, go[k]);
            if (go[k]) queue[(head + count + __popc(m & lt)) % kPushQueue] = make_uint2(cu[k], cj[k] | (cx[k] << 16));
            count += __popc(m);
            if (count >= 32) drain(32);
        }
    }
    if (count) drain(count);
    // modelled bytes: per pair its target and simulation (6 bytes) and change-mask word (2), and per pair of a
    // changed register its source (4), the register and the target word (5)
    nproc = __reduce_add_sync(kFull, nproc);
    nrec = __reduce_add_sync(kFull, nrec);
    if (lane == 0 && nrec) {
        atomicAdd(&P.ctr->bytes, 8ull * nrec + 9ull * nproc);
        atomicAdd(&P.ctr->pairs, static_cast<unsigned long long>(nrec));
    }
}

// Per-tile shared-memory accumulators of the pulling sweep kernels: one 32-bit slot per simulation and tile.
template <int R>
__device__ __forceinline__ uint32_t *tile_acc(uint4 *smem, int wib, int g, int li) {
    using Gm = Geo<R>;
    uint32_t *acc32 = reinterpret_cast<uint32_t *>(smem) + (static_cast<size_t>(wib) * Gm::NG + g) * R;
    for (int k = li; k < R; k += Gm::G) acc32[k] = 0;
    return acc32;
}

// The first sweep of every listed problem that starts a diffusion (Algorithm 1's initialisation fused into
// Algorithm 2's first sweep, L = V): tiles of G lanes take rows and tasks; problems at other sweeps are left to the
// sweep kernel launched beside this one.
template <int R, int MINB>
__global__ void __launch_bounds__(kBlock, MINB) k_first(const DevProb *__restrict__ probs,
                                                        const int32_t *__restrict__ act, int nact) {
    using Gm = Geo<R>;
    extern __shared__ __align__(16) uint4 gather_smem[];
    __shared__ __align__(16) uint32_t sring[kWarpsPerBlock * Geo<R>::NG][3 * 8];  // per tile: three unit descriptors
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int g = lane / Gm::G, li = lane % Gm::G;
    const unsigned tm = tile_mask<R>(g);
    uint32_t *acc32 = tile_acc<R>(gather_smem, wib, g, li);
    __syncwarp(tm);
    const uint64_t worker = (static_cast<uint64_t>(blockIdx.x) * kWarpsPerBlock + wib) * Gm::NG + g;
    const uint64_t nworkers = static_cast<uint64_t>(gridDim.x) * kWarpsPerBlock * Gm::NG;
    uint64_t base = 0;
    for (int q = 0; q < nact; ++q) {
        const DevProb &P = probs[act[q]];
        const DevCtr &C = *P.ctr;
        if (C.done || !C.full || C.t != 0) continue;  // the same for every thread of the block
        // rows are dealt over the tiles; the tiles that got a row also share the problem's tasks
        const uint64_t first = first_owned(worker, nworkers, base);
        base += static_cast<uint64_t>(P.n);
        if (first >= static_cast<uint64_t>(P.n)) continue;
        first_problem_t<R>(P, first, nworkers, tm, li, acc32, sring[wib * Geo<R>::NG + g]);
    }
}

// A later sweep that pulls into every row (sweeps 1 .. pull_sweeps - 1), or pushes, for every listed problem that
// is not in its first sweep.
template <int R, int MINB>
__global__ void __launch_bounds__(kBlock, MINB) k_propg(const DevProb *__restrict__ probs,
                                                        const int32_t *__restrict__ act, int nact) {
    using Gm = Geo<R>;
    extern __shared__ __align__(16) uint4 gather_smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int g = lane / Gm::G, li = lane % Gm::G;
    const unsigned tm = tile_mask<R>(g);
    uint32_t *acc32 = tile_acc<R>(gather_smem, wib, g, li);
    __syncwarp(tm);
    const uint64_t wworker = static_cast<uint64_t>(blockIdx.x) * kWarpsPerBlock + wib;
    const uint64_t nwworkers = static_cast<uint64_t>(gridDim.x) * kWarpsPerBlock;
    const uint64_t worker = wworker * Gm::NG + g;  // tiles for pulls, whole warps for pushes
    const uint64_t nworkers = nwworkers * Gm::NG;
    uint64_t base = 0;
    for (int q = 0; q < nact; ++q) {
        const DevProb &P = probs[act[q]];
        const DevCtr &C = *P.ctr;
        if (C.done || (C.full && C.t == 0)) continue;
        const SweepWork W = sweep_work(P);
        const uint64_t cnt = C.full ? W.nlight + W.ntask : static_cast<uint64_t>(C.npush_l) + C.npush_h;
        const uint64_t first = C.full ? first_owned(worker, nworkers, base) : first_owned(wworker, nwworkers, base);
        base += cnt;
        if (first >= cnt) continue;
        if (C.full)
            prop_problem_t<R, false>(P, C.t, W, cnt, first, nworkers, tm, li, acc32, P.Y);
        else
            push_problem_w<R>(P, C.t, cnt, first, nwworkers, lane,
                              reinterpret_cast<uint32_t *>(gather_smem) + static_cast<size_t>(wib) * Gm::NG * R);
    }
}

constexpr int kPushMinBlocks = 4;  // resident blocks an SM the push kernel's register budget is set for

// A sweep in which every listed problem pushes (only the first pull_sweeps sweeps of a diffusion pull): the push
// path alone, with its own register budget and R bytes of shared memory a warp for the staged row.  skip_full:
// problems in their first sweep are pulled by k_first in the same sweep.
template <int R, int MINB>
__global__ void __launch_bounds__(kBlock, MINB) k_push(const DevProb *__restrict__ probs,
                                                       const int32_t *__restrict__ act, int nact, int skip_full) {
    // per warp: R bytes the push leaves unused, then v's change mask (padded to whole 16-byte words)
    __shared__ __align__(16) uint32_t srow[kWarpsPerBlock][R / 4 + ((R / 32 + 3) & ~3)];
    __shared__ uint2 squeue[kWarpsPerBlock][kPushQueue];  // the streamed push's queue of passing pairs
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const uint64_t wworker = static_cast<uint64_t>(blockIdx.x) * kWarpsPerBlock + wib;
    const uint64_t nwworkers = static_cast<uint64_t>(gridDim.x) * kWarpsPerBlock;
    uint64_t base = 0;
    for (int q = 0; q < nact; ++q) {
        const DevProb &P = probs[act[q]];
        const DevCtr &C = *P.ctr;
        if (C.done) continue;
        if (C.full) {  // pulled by k_first launched beside this kernel; otherwise a scheduling error, flagged
            if (!skip_full && blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&P.ctr->fault, 8u);
            continue;
        }
        if (C.stream) {  // a large L: every in-pair, 128 a warp item
            const uint64_t cnt = (static_cast<uint64_t>(P.ipofs[P.m]) + 127) / 128;
            const uint64_t first = first_owned(wworker, nwworkers, base);
            base += cnt;
            if (first >= cnt) continue;
            push_stream_w<R>(P, C.t, cnt, first, nwworkers, lane, squeue[wib]);
            continue;
        }
        const uint64_t cnt = static_cast<uint64_t>(C.npush_l) + C.npush_h;
        const uint64_t first = first_owned(wworker, nwworkers, base);
        base += cnt;
        if (first >= cnt) continue;
        push_problem_w<R>(P, C.t, cnt, first, nwworkers, lane, srow[wib]);
    }
}

// Split rows with at most kBigTasks tasks: one warp merges a row's partial rows and finishes the row.
template <int R>
__global__ void __launch_bounds__(kBlock) k_combine(const DevProb *__restrict__ probs,
                                                    const int32_t *__restrict__ act, int nact) {
    using Gm = Geo<R>;
    __shared__ WarpStage stage[kWarpsPerBlock];
    extern __shared__ __align__(16) uint4 gather_smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int g = lane / Gm::G, li = lane % Gm::G;
    uint4 *buf = gather_smem + static_cast<size_t>(wib) * (GSlots<R>::kBytesPerWarp / 16);
    if (lane == 0) mbar_init(&stage[wib].mbar);
    __syncwarp();
    uint32_t phase = 0;
    bool aborted = false;
    const uint64_t worker = static_cast<uint64_t>(blockIdx.x) * kWarpsPerBlock + wib;
    const uint64_t nworkers = static_cast<uint64_t>(gridDim.x) * kWarpsPerBlock;
    uint64_t base = 0;
    for (int q = 0; q < nact; ++q) {
        const DevProb &P = probs[act[q]];
        const DevCtr &C = *P.ctr;
        if (C.done) continue;
        const int32_t *list = nullptr;
        const uint64_t cnt = heavy_count(P, C, false, list);
        const uint64_t first = first_owned(worker, nworkers, base);
        base += cnt;
        if (first >= cnt) continue;
        const bool par = C.t & 1u;
        const bool init = C.t == 0;  // the first sweep: own registers are initial ranks, both buffers written
        const uint8_t *Mcur = par ? P.M1 : P.M0;
        uint8_t *Mnext = par ? P.M0 : P.M1;
        uint8_t *Mother = par ? P.M1 : P.M0;
        const uint32_t *Lcur = par ? P.Lb1 : P.Lb0;
        uint32_t *Lnext = par ? P.Lb0 : P.Lb1;
        Stats st;
        for (uint64_t l = first; l < cnt; l += nworkers) {
            const int64_t u = list[l];
            uint32_t acc[Gm::CPL][4];
#pragma unroll
            for (int c = 0; c < Gm::CPL; ++c)
#pragma unroll
                for (int w = 0; w < 4; ++w) acc[c][w] = 0;
            const bool any = merge_partials<R>(P, __ldg(&P.task_off[u]), __ldg(&P.task_off[u + 1]), acc, lane, g,
                                               li, stage[wib], buf, st, phase, aborted);
            reduce_groups<R>(acc);
            if (lane == 0) st.bytes += 16;
            finalize_row_g<R>(P, u, acc, any, !init && test_bit(Lcur, u),
                              reinterpret_cast<const uint4 *>(Mcur + static_cast<size_t>(u) * R), init, Mnext,
                              Mother, Lnext, lane, g, li, st);
            __syncwarp();
        }
        flush_stats(P.ctr, st, lane);
    }
}

// Split rows with more than kBigTasks tasks (hubs): the warps of one block share a row's partial rows, reduce
// through shared memory, and warp 0 finishes the row.
template <int R>
__global__ void __launch_bounds__(kBlock) k_combine_big(const DevProb *__restrict__ probs,
                                                        const int32_t *__restrict__ act, int nact) {
    using Gm = Geo<R>;
    __shared__ WarpStage stage[kWarpsPerBlock];
    __shared__ uint4 s_red[kWarpsPerBlock][Gm::CH];
    __shared__ int s_any[kWarpsPerBlock];
    extern __shared__ __align__(16) uint4 gather_smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int g = lane / Gm::G, li = lane % Gm::G;
    uint4 *buf = gather_smem + static_cast<size_t>(wib) * (GSlots<R>::kBytesPerWarp / 16);
    if (lane == 0) mbar_init(&stage[wib].mbar);
    __syncwarp();
    uint32_t phase = 0;
    bool aborted = false;
    uint64_t base = 0;
    for (int q = 0; q < nact; ++q) {
        const DevProb &P = probs[act[q]];
        const DevCtr &C = *P.ctr;
        if (C.done) continue;
        const int32_t *list = nullptr;
        const uint64_t cnt = heavy_count(P, C, true, list);
        const uint64_t first = first_owned(blockIdx.x, gridDim.x, base);
        base += cnt;
        if (first >= cnt) continue;
        const bool par = C.t & 1u;
        const bool init = C.t == 0;
        const uint8_t *Mcur = par ? P.M1 : P.M0;
        uint8_t *Mnext = par ? P.M0 : P.M1;
        uint8_t *Mother = par ? P.M1 : P.M0;
        const uint32_t *Lcur = par ? P.Lb1 : P.Lb0;
        uint32_t *Lnext = par ? P.Lb0 : P.Lb1;
        Stats st;
        for (uint64_t l = first; l < cnt; l += gridDim.x) {
            const int64_t u = list[l];
            const int64_t t0 = __ldg(&P.task_off[u]), t1 = __ldg(&P.task_off[u + 1]);
            uint32_t acc[Gm::CPL][4];
#pragma unroll
            for (int c = 0; c < Gm::CPL; ++c)
#pragma unroll
                for (int w = 0; w < 4; ++w) acc[c][w] = 0;
            bool any = false;
            for (int64_t a = t0 + 32 * wib; a < t1; a += 32 * kWarpsPerBlock)
                any |= merge_partials<R>(P, a, min(a + 32, t1), acc, lane, g, li, stage[wib], buf, st, phase, aborted);
            reduce_groups<R>(acc);
            if (g == 0) {
#pragma unroll
                for (int c = 0; c < Gm::CPL; ++c)
                    s_red[wib][li + Gm::G * c] = make_uint4(acc[c][0], acc[c][1], acc[c][2], acc[c][3]);
            }
            if (lane == 0) s_any[wib] = any ? 1 : 0;
            __syncthreads();
            if (wib == 0) {
                bool all_any = false;
                for (int w = 0; w < kWarpsPerBlock; ++w) {
                    all_any |= s_any[w] != 0;
#pragma unroll
                    for (int c = 0; c < Gm::CPL; ++c) {
                        const uint4 x = s_red[w][li + Gm::G * c];
                        acc[c][0] = vmax4(acc[c][0], x.x);
                        acc[c][1] = vmax4(acc[c][1], x.y);
                        acc[c][2] = vmax4(acc[c][2], x.z);
                        acc[c][3] = vmax4(acc[c][3], x.w);
                    }
                }
                if (lane == 0) st.bytes += 16;
                finalize_row_g<R>(P, u, acc, all_any, !init && test_bit(Lcur, u),
                                  reinterpret_cast<const uint4 *>(Mcur + static_cast<size_t>(u) * R), init, Mnext,
                                  Mother, Lnext, lane, g, li, st);
            }
            __syncthreads();
        }
        flush_stats(P.ctr, st, lane);
    }
}


namespace {

// Block-aggregated append of the set bits of one word per thread: ids (word_index*32 + bit) go to out[], the block
// reserves its range with one atomic on *count.  All threads of the block must call it.
__device__ __forceinline__ void block_append_bits(uint32_t w, int64_t word_index, int32_t *out, uint32_t *count,
                                                  uint32_t *seg_base = nullptr, uint32_t *seg_len = nullptr) {
    __shared__ uint32_t s_warp[kWarpsPerBlock];
    __shared__ uint32_t s_base, s_run;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const uint32_t c = __popc(w);
    uint32_t incl = c;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, incl, off);
        if (lane >= off) incl += y;
    }
    if (lane == 31) s_warp[wib] = incl;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t run = 0;
        for (int i = 0; i < kWarpsPerBlock; ++i) {
            const uint32_t x = s_warp[i];
            s_warp[i] = run;
            run += x;
        }
        s_base = run ? atomicAdd(count, run) : 0;
        s_run = run;
    }
    __syncthreads();
    uint32_t pos = s_base + s_warp[wib] + incl - c;
    if (seg_base) *seg_base = s_base;
    if (seg_len) *seg_len = s_run;
    while (w) {
        const int b = __ffs(w) - 1;
        w &= w - 1;
        out[pos++] = static_cast<int32_t>(word_index * 32 + b);
    }
    __syncthreads();
}

// The first pull_sweeps sweeps pull into every row (sweep 0 has L = V, and the next ones still have most of V in L);
// every later sweep pushes from L'.  Called after sweep C.t.
__device__ __forceinline__ bool next_is_push(const DevProb &P, const DevCtr &C) {
    return __ldcg(&C.t) + 1 >= P.pull_sweeps;
}

}  // namespace

// After sweep t: clear L_t's bits (the buffer L_{t+2} will be written to) and, when the next sweep is a push
// sweep, compact L_{t+1} into the changed-vertex lists (whole vertices, or kPushChunk-in-edge chunks of those
// with more) and copy each changed row into the buffer the next sweep writes, so that it holds every row.
__device__ __forceinline__ void advance_one(const DevProb &P);

// True in the last block of the launch to get here (after every block's writes are visible to it).
__device__ __forceinline__ bool last_block(GridBar *gb) {
    __shared__ int s_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(&gb->tail, 1u) == gridDim.x - 1;
        if (s_last) {
            gb->tail = 0;
            __threadfence();
        }
    }
    __syncthreads();
    return s_last != 0;
}

constexpr int kFrontChunk = 4 * kBlock;  // vertices of L_{t+1} a frontier block takes at a time (4 a thread)
constexpr int kFrontSuper = kBlock / 32;  // chunks a frontier block checks at once: one a warp, a word a lane
static_assert(4 * kWarpsPerBlock == 32, "one warp scans the frontier chunk's per-warp counts");

__global__ void __launch_bounds__(kBlock) k_frontier(const DevProb *__restrict__ probs,
                                                     const int32_t *__restrict__ act, int nact, GridBar *gb) {
    __shared__ uint32_t s_cnt[4 * kWarpsPerBlock];  // light vertices listed by (k, warp), then their offsets
    __shared__ uint32_t s_base, s_n;
    __shared__ int32_t s_v[kFrontChunk];            // the chunk's listed vertices, for the row copies
    __shared__ int s_nz[kFrontSuper];               // which of the block's current chunks have a bit of L_{t+1}
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    uint64_t base = 0;
    for (int q = 0; q < nact; ++q) {
        const DevProb &P = probs[act[q]];
        const DevCtr &C = *P.ctr;
        if (C.done) continue;
        const bool push_next = next_is_push(P, C);
        // the first sweep of a diffusion wrote every row to both buffers: nothing to copy after it
        const bool copy = C.t != 0;
        // after a push sweep the copies also raise the rows' register sums (a pulling sweep stored them itself)
        const bool rsum = P.gst && !C.full;
        const bool par = C.t & 1u;
        uint32_t *Lold = par ? P.Lb1 : P.Lb0;
        const uint32_t *Lnew = par ? P.Lb0 : P.Lb1;
        const uint8_t *Mw = par ? P.M0 : P.M1;  // written by sweep t
        uint8_t *Mr = par ? P.M1 : P.M0;        // read by sweep t, written by sweep t + 1
        const int64_t words = (P.n + 31) >> 5;
        const uint64_t chunks = (static_cast<uint64_t>(P.n) + kFrontChunk - 1) / kFrontChunk;
        const uint64_t first = first_owned(blockIdx.x, gridDim.x, base);
        base += chunks;
        unsigned long long indeg = 0;  // in-edges into L': the next sweep's work count
        uint32_t nchg = 0;             // |L'| (this thread's bits)
        // the block's chunks first, first + grid, ...: kFrontSuper of them at a time, warp w loading chunk w's 32
        // words of L_{t+1} (and clearing its words of L_t); a chunk without any bit costs nothing more, so a later
        // sweep's small L skips most chunks after one load and one barrier
        for (uint64_t cg = first; cg < chunks; cg += kFrontSuper * static_cast<uint64_t>(gridDim.x)) {
            {
                const uint64_t chw = cg + static_cast<uint64_t>(wib) * gridDim.x;  // this warp's chunk
                const int64_t wi = static_cast<int64_t>(chw) * 32 + lane;
                uint32_t w = 0;
                if (chw < chunks && wi < words) {
                    w = Lnew[wi];
                    Lold[wi] = 0;
                }
                const bool nz = __any_sync(kFull, w != 0u);
                if (lane == 0) s_nz[wib] = nz ? 1 : 0;
                if (!__syncthreads_or(nz)) continue;  // also orders s_nz before its reads
            }
            for (int sub = 0; sub < kFrontSuper; ++sub) {
                const uint64_t ch = cg + static_cast<uint64_t>(sub) * gridDim.x;
                if (ch >= chunks) break;
                if (!s_nz[sub]) continue;
                // vertex ch * kFrontChunk + k * kBlock + threadIdx.x: word (ch * 4 + k) * kWarpsPerBlock + wib,
                // bit lane
                bool light[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int64_t wi = (static_cast<int64_t>(ch) * 4 + k) * kWarpsPerBlock + wib;
                    uint32_t w = 0;
                    if (wi < words) {
                        w = Lnew[wi];
                        if (lane == 0) Lold[wi] = 0;
                    }
                    light[k] = false;
                    nchg += (w >> lane) & 1u;
                    if ((w >> lane) & 1u) {
                        const int64_t v = wi * 32 + lane;
                        const uint64_t d = in_degree(P, v);
                        indeg += d;
                        light[k] = true;
                        if (push_next && d > kPushChunk) {
                            light[k] = false;
                            const uint4 *src = reinterpret_cast<const uint4 *>(Mw + static_cast<size_t>(v) * P.R);
                            uint4 *dst = reinterpret_cast<uint4 *>(Mr + static_cast<size_t>(v) * P.R);
                            if (copy) {
                                const int CH = P.R / 16;
                                uint32_t rise = 0;  // how much sweep t raised the row's register sum
                                for (int c = 0; c < CH; ++c) {
                                    const uint4 a = src[c], b = dst[c];
                                    P.dmask[static_cast<size_t>(v) * CH + c] = static_cast<uint16_t>(ne_bits16(a, b));
                                    rise += byte_sum16(a) - byte_sum16(b);
                                    dst[c] = a;
                                }
                                if (rsum && rise) atomicAdd(&P.gst[v], rise);
                            }
                            const uint32_t nt = static_cast<uint32_t>((d + kPushChunk - 1) / kPushChunk);
                            const uint32_t at = atomicAdd(&P.ctr->nchg_hc, nt);
                            for (uint32_t c = 0; c < nt; ++c)
                                P.chg_hc[at + c] = (static_cast<uint64_t>(c) << 32) | static_cast<uint32_t>(v);
                        }
                    }
                }
                if (!push_next) continue;  // the next sweep pulls into every row: no list, no copies
                // list the chunk's light vertices (one reservation) and copy their rows into the next sweep's buffer.
                // This barrier also ends the previous chunk's use of the shared arrays.
                if (!__syncthreads_or(light[0] | light[1] | light[2] | light[3])) continue;
                unsigned mk[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    mk[k] = __ballot_sync(kFull, light[k]);
                    if (lane == 0) s_cnt[k * kWarpsPerBlock + wib] = __popc(mk[k]);
                }
                __syncthreads();
                if (wib == 0) {
                    const uint32_t c = s_cnt[lane];
                    uint32_t incl = c;
#pragma unroll
                    for (int off = 1; off < 32; off <<= 1) {
                        const uint32_t y = __shfl_up_sync(kFull, incl, off);
                        if (lane >= off) incl += y;
                    }
                    s_cnt[lane] = incl - c;
                    if (lane == 31) {
                        s_n = incl;
                        s_base = incl ? atomicAdd(&P.ctr->nchg_list, incl) : 0u;
                    }
                }
                __syncthreads();
                const uint32_t sn = s_n, sb = s_base;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    if (light[k]) {
                        const uint32_t at = s_cnt[k * kWarpsPerBlock + wib] + __popc(mk[k] & lt);
                        const int32_t v = static_cast<int32_t>(
                            ((static_cast<int64_t>(ch) * 4 + k) * kWarpsPerBlock + wib) * 32 + lane);
                        P.chg_list[sb + at] = v;
                        s_v[at] = v;
                    }
                }
                __syncthreads();
                if (!copy) continue;
                // consecutive threads on consecutive 16-byte chunks of the listed rows; the chunks' changed registers
                // (Mw against the previous sweep's Mr) go to dmask for the push sweep
                // and each row's register sum rises by what sweep t added (one atomic per row and warp: a row's CH
                // chunks are CH consecutive lanes, CH-aligned, when CH divides 32, or whole warps when 32 divides CH)
                const uint32_t CH = static_cast<uint32_t>(P.R / 16);
                const uint32_t seg = CH < 32 ? CH : 32;
                const uint32_t xend = (sn * CH + 31) & ~31u;  // whole warps, so that the sums' shuffles converge
#pragma unroll 4
                for (uint32_t x = threadIdx.x; x < xend; x += blockDim.x) {
                    const bool in = x < sn * CH;
                    const int64_t v = in ? s_v[x / CH] : 0;
                    uint32_t rise = 0;
                    if (in) {
                        uint4 *dst = reinterpret_cast<uint4 *>(Mr + static_cast<size_t>(v) * P.R) + x % CH;
                        const uint4 a = reinterpret_cast<const uint4 *>(Mw + static_cast<size_t>(v) * P.R)[x % CH];
                        const uint4 b = *dst;
                        P.dmask[static_cast<size_t>(v) * CH + x % CH] = static_cast<uint16_t>(ne_bits16(a, b));
                        rise = byte_sum16(a) - byte_sum16(b);
                        *dst = a;
                    }
                    if (rsum) {
                        const unsigned segmask = (seg == 32 ? kFull : (1u << seg) - 1u) << (lane & ~(seg - 1));
                        rise = __reduce_add_sync(segmask, rise);
                        if (in && (lane & (seg - 1)) == 0 && rise) atomicAdd(&P.gst[v], rise);
                    }
                }
            }
            __syncthreads();  // the chunks are done with s_nz before the next group writes it
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            indeg += __shfl_xor_sync(kFull, indeg, off);
            nchg += __shfl_xor_sync(kFull, nchg, off);
        }
        if (lane == 0 && nchg) {
            atomicAdd(&P.ctr->nchg, nchg);
            atomicAdd(&P.ctr->chg_indeg, indeg);
        }
    }
    if (last_block(gb))
        for (int q = threadIdx.x; q < nact; q += blockDim.x) advance_one(probs[act[q]]);
}

// Ends sweep t: stop test (|L'| <= eps_c |V| or the sweep limit), mode of the next sweep, counter resets.  Run by
// the last block of the frontier kernel to finish.
__device__ __forceinline__ void advance_one(const DevProb &P) {
    DevCtr &C = *P.ctr;
    if (__ldcg(&C.done)) return;
    const uint32_t t = __ldcg(&C.t);
    const uint32_t nchg = __ldcg(&C.nchg);
    if (static_cast<int32_t>(t + 1) < P.flog_cap) P.flog[t + 1] = nchg;
    C.sweeps_total += 1;
    const bool stop = nchg <= P.stop_thr;
    const bool lim = t + 1 >= P.max_sweeps;
    if (stop || lim) {
        C.done = 1;
        C.timeout = (!stop && lim) ? 1u : 0u;
        C.res_par = (t + 1) & 1u;
    }
    // visits of the next sweep (Algorithm 2's work count): every edge (u, v) with v in L_{t+1}, in every simulation
    if (!C.done) C.visits += __ldcg(&C.chg_indeg) * static_cast<unsigned long long>(P.R);
    C.full = next_is_push(P, C) ? 0u : 1u;
    C.stream = (!C.full && __ldcg(&C.chg_indeg) >= P.stream_min) ? 1u : 0u;
    C.npush_l = C.full ? 0u : __ldcg(&C.nchg_list);
    C.npush_h = C.full ? 0u : __ldcg(&C.nchg_hc);
    C.nchg = 0;
    C.nchg_list = 0;
    C.nchg_hc = 0;
    C.chg_indeg = 0;
    C.t = t + 1;
}

// Start of a diffusion (Algorithm 1's initialisation; the initial registers themselves are formed by the first
// sweep, which writes both register buffers): clears the frontier and task bits, resets the diffusion counters and
// M_S', and on a rebuild marks in rany the vertices R_G(S) reached in some simulation (their blocked registers are
// 0 in the rebuilt sketch).
__global__ void __launch_bounds__(kBlock) k_init(const DevProb *__restrict__ probs, const int32_t *__restrict__ act,
                                                 int nact) {
    const uint64_t tid = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    const uint64_t nthreads = static_cast<uint64_t>(gridDim.x) * blockDim.x;
    const int lane = threadIdx.x & 31;
    // rany / rnew words: a warp per 32 vertices, a lane per vertex row
    {
        const uint64_t worker = tid >> 5, nworkers = nthreads >> 5;
        uint64_t base = 0;
        for (int q = 0; q < nact; ++q) {
            const DevProb &P = probs[act[q]];
            if (!P.rany) continue;
            const uint64_t words = (static_cast<uint64_t>(P.n) + 31) >> 5;
            const uint64_t first = first_owned(worker, nworkers, base);
            base += words;
            // no search has run yet (levels count on over the searches of a problem): nothing is reached
            const bool searched = P.ctr->lvl != 0;
            for (uint64_t wi = first; wi < words; wi += nworkers) {
                const int64_t v = static_cast<int64_t>(wi) * 32 + lane;
                uint32_t any = 0, nw = 0;
                if (searched && v < P.n) {
                    const uint2 *row = reinterpret_cast<const uint2 *>(P.vis + static_cast<size_t>(v) * P.W);
                    const uint2 *done =
                        P.vis_done ? reinterpret_cast<const uint2 *>(P.vis_done + static_cast<size_t>(v) * P.W)
                                   : nullptr;
                    for (int k = 0; k < P.W / 2; ++k) {
                        const uint2 x = row[k];
                        any |= x.x | x.y;
                        if (done) {
                            const uint2 y = done[k];
                            nw |= (x.x & ~y.x) | (x.y & ~y.y);
                        }
                    }
                }
                const uint32_t bits = __ballot_sync(kFull, any != 0);
                const uint32_t fresh = __ballot_sync(kFull, nw != 0);
                if (lane == 0) {
                    P.rany[wi] = bits;
                    if (P.rnew) P.rnew[wi] = fresh;  // vertices with blocked bits not yet applied
                }
            }
        }
    }
    uint64_t base = 0;
    for (int q = 0; q < nact; ++q) {
        const DevProb &P = probs[act[q]];
        const int64_t words = (P.n + 31) >> 5;
        const int64_t twords = (P.n_tasks + 31) >> 5;
        // units: L bits (2 x words), task bits, counters
        const uint64_t cnt = 2 * static_cast<uint64_t>(words) + static_cast<uint64_t>(twords) + 1;
        const uint64_t first = first_owned(tid, nthreads, base);
        base += cnt;
        for (uint64_t l = first; l < cnt; l += nthreads) {
            if (l < 2 * static_cast<uint64_t>(words)) {
                (l < static_cast<uint64_t>(words) ? P.Lb0 : P.Lb1)[l % words] = 0;
            } else if (l < cnt - 1) {
                P.part_any[l - 2 * static_cast<uint64_t>(words)] = 0;
            } else {
                DevCtr &C = *P.ctr;
                C.t = 0;
                C.done = 0;
                C.timeout = 0;
                C.full = 1;
                C.res_par = 0;
                C.nchg = 0;
                C.nchg_list = 0;
                C.nchg_hc = 0;
                C.npush_l = 0;
                C.npush_h = 0;
                C.stream = 0;
                C.task_next = 0;
                C.chg_indeg = 0;
                C.gms = 0;  // M_S' is cleared below
                C.cand_key = 0;
                if (P.flog_cap > 0) P.flog[0] = P.n;
                C.visits += static_cast<unsigned long long>(P.m) * static_cast<unsigned long long>(P.R);  // L_0 = V
                for (int j = 0; j < P.R; ++j) P.MS[j] = 0;
            }
        }
    }
}

namespace {

template <int R>
__device__ void scan_problem(const DevProb &P, uint64_t cnt, uint64_t first, uint64_t nworkers, int lane) {
    using Gm = Geo<R>;
    const int g = lane / Gm::G, li = lane % Gm::G;
    const uint8_t *M = P.ctr->res_par ? P.M1 : P.M0;
    const uint32_t gms = P.ctr->gms;
    uint32_t ms[Gm::CPL][4];
    {
        const uint4 *p = reinterpret_cast<const uint4 *>(P.MS);
#pragma unroll
        for (int c = 0; c < Gm::CPL; ++c) {
            const uint4 x = p[li + Gm::G * c];
            ms[c][0] = x.x;
            ms[c][1] = x.y;
            ms[c][2] = x.z;
            ms[c][3] = x.w;
        }
    }
    // U rows a lane group in flight at once: their loads go out together, and apart from the seed-set test
    constexpr int U = Gm::CPL == 1 ? 4 : (Gm::CPL == 2 ? 2 : 1);
    unsigned long long best = 0;
    for (uint64_t l0 = first; l0 < cnt; l0 += U * nworkers) {
        int64_t v[U];
        bool ok[U];
        uint4 x[U][Gm::CPL];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint64_t l = l0 + static_cast<uint64_t>(u) * nworkers;
            v[u] = static_cast<int64_t>(l) * Gm::NG + g;
            ok[u] = l < cnt && v[u] < P.n;
            const uint4 *row = reinterpret_cast<const uint4 *>(M + static_cast<size_t>(ok[u] ? v[u] : 0) * R);
#pragma unroll
            for (int c = 0; c < Gm::CPL; ++c) x[u][c] = ok[u] ? __ldg(row + li + Gm::G * c) : make_uint4(0, 0, 0, 0);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) ok[u] = ok[u] && !test_bit(P.inS, v[u]);
#pragma unroll
        for (int u = 0; u < U; ++u) {
            uint32_t s = 0;
#pragma unroll
            for (int c = 0; c < Gm::CPL; ++c) {
                s = __dp4a(vmax4(x[u][c].x, ms[c][0]), 0x01010101u, s);
                s = __dp4a(vmax4(x[u][c].y, ms[c][1]), 0x01010101u, s);
                s = __dp4a(vmax4(x[u][c].z, ms[c][2]), 0x01010101u, s);
                s = __dp4a(vmax4(x[u][c].w, ms[c][3]), 0x01010101u, s);
            }
#pragma unroll
            for (int off = 1; off < Gm::G; off <<= 1) s += __shfl_xor_sync(kFull, s, off);
            if (ok[u]) {
                const uint32_t gain = s - gms;  // s >= sum_j M_S'[j]
                if (li == 0 && P.gst) {
                    // with M_S' empty every gain is the row's register sum, which the sweeps kept in gst
                    if (P.check_sums && gms == 0 && P.gst[v[u]] != gain) atomicOr(&P.ctr->fault, 16u);
                    P.gst[v[u]] = gain;
                }
                const unsigned long long key =
                    (static_cast<unsigned long long>(gain) << 32) | (0xFFFFFFFFu - static_cast<uint32_t>(v[u]));
                best = key > best ? key : best;
            }
        }
    }
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const unsigned long long o = __shfl_xor_sync(kFull, best, off);
        best = o > best ? o : best;
    }
    if (lane == 0 && best) atomicMax(&P.ctr->best_key, best);
}

}  // namespace

// Algorithm 1's argmax: for every v not in S, gsum_v = sum_j max(M_S'[j], M_v[j]) (Merge, Eq. 3; Estimate, Eq. 2 is
// increasing in it); the maximum of (gain_v << 32 | ~v), gain_v = gsum_v - sum_j M_S'[j], picks the largest sum,
// ties to the smallest id.  Every gain is also kept in gst for the lazy scans of the next steps.
template <int R>
__global__ void __launch_bounds__(kBlock) k_scan(const DevProb *__restrict__ probs, const int32_t *__restrict__ act,
                                                 int nact) {
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const uint64_t worker = static_cast<uint64_t>(blockIdx.x) * kWarpsPerBlock + wib;
    const uint64_t nworkers = static_cast<uint64_t>(gridDim.x) * kWarpsPerBlock;
    uint64_t base = 0;
    for (int q = 0; q < nact; ++q) {
        const DevProb &P = probs[act[q]];
        const uint64_t cnt = (static_cast<uint64_t>(P.n) + Geo<R>::NG - 1) / Geo<R>::NG;
        const uint64_t first = first_owned(worker, nworkers, base);
        base += cnt;
        if (first >= cnt) continue;
        scan_problem<R>(P, cnt, first, nworkers, lane);
    }
}

// The block's largest key, added to *dst by one atomic (every thread of the block calls it with its own key).
__device__ __forceinline__ void block_max_key(unsigned long long key, unsigned long long *dst) {
    __shared__ unsigned long long s_key[kWarpsPerBlock];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const unsigned long long o = __shfl_xor_sync(kFull, key, off);
        key = o > key ? o : key;
    }
    if (lane == 0) s_key[wib] = key;
    __syncthreads();
    if (wib == 0) {
        key = lane < kWarpsPerBlock ? s_key[lane] : 0ull;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const unsigned long long o = __shfl_xor_sync(kFull, key, off);
            key = o > key ? o : key;
        }
        if (lane == 0 && key) atomicMax(dst, key);
    }
    __syncthreads();  // s_key is free again
}

// ------------------------------------------------------------------------------------------------------------
// Lazy (CELF-style) argmax for the greedy steps that keep the sketch.  Between two builds M_S' only grows, so a
// candidate's gain gain_v = sum_j max(M_S'[j], M_v[j]) - sum_j M_S'[j] = sum_j (M_v[j] - M_S'[j])^+ only shrinks,
// and the gain last evaluated for v (gst[v]; right after a build, the row's register sum kept by the sweeps, which
// is its exact gain since M_S' is empty) bounds its current gain from above.  A step then
//   1. finds the candidate v1 with the largest bound key (gst[v] << 32 | ~v)            (k_celf_max),
//   2. evaluates v1 exactly: its exact key tau                                           (k_celf_tau),
//   3. evaluates exactly every other candidate whose bound key exceeds tau, and keeps the largest exact key
//                                                                                        (k_celf_eval).
// Every candidate left out has exact key <= bound key <= tau <= the result, so the result is the full argmax
// (largest gain, ties to the smallest id), with far fewer register rows read.

// A thread takes four consecutive candidates at a time (one 16-byte load of their bounds, one word of seed bits).
__global__ void __launch_bounds__(kBlock) k_celf_max(const DevProb *__restrict__ probs,
                                                     const int32_t *__restrict__ act, int nact) {
    const uint64_t tid = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    const uint64_t nthreads = static_cast<uint64_t>(gridDim.x) * blockDim.x;
    uint64_t base = 0;
    for (int q = 0; q < nact; ++q) {
        const DevProb &P = probs[act[q]];
        const uint64_t n = static_cast<uint64_t>(P.n);
        const uint64_t cnt = (n + 3) / 4;
        const uint64_t first = first_owned(tid, nthreads, base);
        base += cnt;
        unsigned long long best = 0;
        for (uint64_t g = first; g < cnt; g += nthreads) {
            const uint64_t v0 = g * 4;
            uint32_t b[4];
            if (v0 + 4 <= n) {
                const uint4 x = __ldg(reinterpret_cast<const uint4 *>(P.gst) + g);
                b[0] = x.x, b[1] = x.y, b[2] = x.z, b[3] = x.w;
            } else {
#pragma unroll
                for (int i = 0; i < 4; ++i) b[i] = v0 + i < n ? __ldg(&P.gst[v0 + i]) : 0u;
            }
            const uint32_t sb = __ldg(&P.inS[v0 >> 5]) >> (v0 & 31);  // the four candidates' seed bits
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                if (v0 + i < n && !((sb >> i) & 1u)) {
                    const unsigned long long key = (static_cast<unsigned long long>(b[i]) << 32) |
                                                   (0xFFFFFFFFu - static_cast<uint32_t>(v0 + i));
                    best = key > best ? key : best;
                }
            }
        }
        block_max_key(best, &P.ctr->cand_key);
    }
}

// The exact key of the best-bounded candidate (one block per problem); it also starts the step's best key.
__global__ void k_celf_tau(const DevProb *__restrict__ probs, const int32_t *__restrict__ act, int nact) {
    const int q = blockIdx.x;
    if (q >= nact) return;
    const DevProb &P = probs[act[q]];
    DevCtr &C = *P.ctr;
    const unsigned long long ck = C.cand_key;
    __shared__ uint32_t s_sum;
    if (threadIdx.x == 0) s_sum = 0;
    __syncthreads();
    if (ck == 0) {  // no candidate left: every vertex is a seed
        if (threadIdx.x == 0) C.tau_key = C.best_key = 0;
        return;
    }
    const uint32_t v = 0xFFFFFFFFu - static_cast<uint32_t>(ck & 0xFFFFFFFFull);
    const uint8_t *M = C.res_par ? P.M1 : P.M0;
    const uint32_t *row = reinterpret_cast<const uint32_t *>(M + static_cast<size_t>(v) * P.R);
    const uint32_t *ms = reinterpret_cast<const uint32_t *>(P.MS);
    uint32_t part = 0;
    for (int i = threadIdx.x; i < P.R / 4; i += blockDim.x) part = __dp4a(vmax4(row[i], ms[i]), 0x01010101u, part);
    atomicAdd(&s_sum, part);
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint32_t gain = s_sum - C.gms;
        const unsigned long long key = (static_cast<unsigned long long>(gain) << 32) | (0xFFFFFFFFu - v);
        P.gst[v] = gain;
        C.tau_key = key;
        C.best_key = key;
        C.cand_key = 0;
    }
}

// Exact evaluation of every candidate whose bound key exceeds tau: a warp takes 32 consecutive vertices, a lane
// tests one bound, and the warp evaluates the surviving rows one after the other (R / 4 register words over its
// lanes), storing each exact gain back into gst.
template <int R>
__global__ void __launch_bounds__(kBlock) k_celf_eval(const DevProb *__restrict__ probs,
                                                      const int32_t *__restrict__ act, int nact) {
    constexpr int WPL = R / 4 >= 32 ? R / 128 : 1;  // register words a lane holds
    constexpr int LANES = R / 4 >= 32 ? 32 : R / 4;   // lanes that hold words
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const uint64_t worker = static_cast<uint64_t>(blockIdx.x) * kWarpsPerBlock + wib;
    const uint64_t nworkers = static_cast<uint64_t>(gridDim.x) * kWarpsPerBlock;
    uint64_t base = 0;
    for (int q = 0; q < nact; ++q) {
        const DevProb &P = probs[act[q]];
        const DevCtr &C = *P.ctr;
        const uint64_t cnt = (static_cast<uint64_t>(P.n) + 31) / 32;
        const uint64_t first = first_owned(worker, nworkers, base);
        base += cnt;
        if (first >= cnt) continue;
        const unsigned long long tau = C.tau_key;
        const uint32_t gms = C.gms;
        const uint8_t *M = C.res_par ? P.M1 : P.M0;
        uint32_t ms[WPL];
#pragma unroll
        for (int k = 0; k < WPL; ++k)
            ms[k] = lane < LANES ? reinterpret_cast<const uint32_t *>(P.MS)[lane + LANES * k] : 0u;
        unsigned long long best = 0;
        for (uint64_t l = first; l < cnt; l += nworkers) {
            const uint64_t v = l * 32 + lane;
            bool cand = false;
            if (v < static_cast<uint64_t>(P.n) && !test_bit(P.inS, static_cast<int64_t>(v))) {
                const unsigned long long key = (static_cast<unsigned long long>(__ldg(&P.gst[v])) << 32) |
                                               (0xFFFFFFFFu - static_cast<uint32_t>(v));
                cand = key > tau;
            }
            for (unsigned m = __ballot_sync(kFull, cand); m; m &= m - 1u) {
                const uint32_t u = static_cast<uint32_t>(l * 32 + (__ffs(m) - 1));
                const uint32_t *row = reinterpret_cast<const uint32_t *>(M + static_cast<size_t>(u) * R);
                uint32_t sum = 0;
#pragma unroll
                for (int k = 0; k < WPL; ++k)
                    if (lane < LANES) sum = __dp4a(vmax4(__ldg(row + lane + LANES * k), ms[k]), 0x01010101u, sum);
                sum = __reduce_add_sync(kFull, sum);
                const uint32_t gain = sum - gms;
                if (lane == 0) P.gst[u] = gain;
                const unsigned long long key = (static_cast<unsigned long long>(gain) << 32) | (0xFFFFFFFFu - u);
                best = key > best ? key : best;
            }
        }
        if (lane == 0 && best) atomicMax(&P.ctr->best_key, best);
    }
}

namespace {
constexpr int kFirstTask = 0x100;  // flag in a task's edge-count field: the vertex's first task (it counts the row)

// Search task c of vertex v, whose out-edges start at edge e: te of them (fewer in the last task, none for a
// vertex without out-edges), so a level reads neither the task's vertex offsets nor its degree.
__device__ __forceinline__ int4 bfs_task(uint32_t v, int64_t e, int64_t deg, uint32_t c, int te) {
    const int64_t e0 = e + static_cast<int64_t>(c) * te;
    const int64_t left = deg - static_cast<int64_t>(c) * te;
    const int ne = static_cast<int>(left < te ? left : te);
    return make_int4(static_cast<int>(static_cast<uint32_t>(e0)), static_cast<int>(static_cast<uint64_t>(e0) >> 32),
                     static_cast<int>(v), ne | (c == 0 ? kFirstTask : 0));
}

// Tasks of a vertex: one per te out-edges, and one for a vertex without out-edges, whose first task still counts
// the bits its delta row newly reached.
__device__ __forceinline__ uint32_t bfs_ntasks(int64_t deg, int te) {
    return deg > 0 ? static_cast<uint32_t>((deg + te - 1) / te) : 1u;
}

// Appends the search tasks of vertex v.
__device__ __forceinline__ void bfs_tasks(int4 *T, uint32_t *count, uint32_t v, const int64_t *xadj, int te) {
    const int64_t e = xadj[v], deg = xadj[v + 1] - e;
    const uint32_t nt = bfs_ntasks(deg, te);
    const uint32_t at = atomicAdd(count, nt);
    for (uint32_t c = 0; c < nt; ++c) T[at + c] = bfs_task(v, e, deg, c, te);
}
}  // namespace

// Search state across levels.  Level numbers run on over the searches of a problem (a search starts at the level
// where the previous one ended), and level L uses
//   del[L % 3]        delta rows of its frontier F_L (bits newly reached at the previous level), read,
//   del[(L + 1) % 3]  delta rows of F_{L+1}, written,
//   del[(L + 2) % 3]  delta rows of F_{L-1}, cleared (so they are zero again when level L + 1 writes there),
// with the vertex lists V[.] in the same rotation, tasks T[L % 2] read and T[(L + 1) % 2] written, and the level
// stamp L + 1 marking the vertices listed into F_{L+1}.  Nothing has to be cleared between levels but those rows.

// Takes the argmax as seed s of step k, adds it to S and starts the reachability search from it: s is marked
// reached in every simulation where it was not yet, and those bits form the first frontier.
__global__ void k_choose(const DevProb *__restrict__ probs, const int32_t *__restrict__ act, int nact, int32_t step) {
    const int q = blockIdx.x;
    if (q >= nact) return;
    const DevProb &P = probs[act[q]];
    DevCtr &C = *P.ctr;
    const int lane = threadIdx.x;
    const unsigned long long key = C.best_key;
    const uint32_t s = 0xFFFFFFFFu - static_cast<uint32_t>(key & 0xFFFFFFFFull);
    const uint32_t gsum = static_cast<uint32_t>(key >> 32) + C.gms;
    if (key == 0 || s >= static_cast<uint64_t>(P.n)) {  // no candidate was scanned: nothing to search
        if (lane == 0) {
            C.bdone = 1;
            C.btimeout = 1;
        }
        return;
    }
    const uint32_t L = C.lvl;
    __syncthreads();  // every thread has read the counters before warp 0 updates them
    uint32_t *d0 = P.del[L % 3u];
    uint32_t added = 0;
    if (lane < 32) {
        for (int k = lane; k < P.W; k += 32) {
            const size_t at = static_cast<size_t>(s) * P.W + k;
            const uint32_t nb = ~P.vis[at];
            P.vis[at] = 0xFFFFFFFFu;
            d0[at] = nb;
            added += __popc(nb);
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) added += __shfl_xor_sync(kFull, added, off);
        __syncwarp();
    }
    if (lane == 0) {
        C.s = s;
        C.gsum = gsum;
        C.best_key = 0;
        set_bit(P.inS, s);
        C.nT[L & 1u] = 0;
        C.nT[(L & 1u) ^ 1u] = 0;
        C.nVl[L % 3u] = 1;
        C.nVl[(L + 1u) % 3u] = 0;
        P.V[L % 3u][0] = static_cast<int32_t>(s);
        C.lvl0 = L;
        C.bdone = added ? 0u : 1u;
        C.btimeout = 0;
        if (step >= 0) {
            P.step_seed[step] = s;
            P.step_gsum[step] = gsum;
        }
    }
    // the seed's search tasks for the first level, written by the whole block (a hub seed has 10^5 of them); the
    // task lists of this level were empty, so they start at 0
    const int te = bfs_task_edges(P.W);
    const int64_t e = P.xadj[s], deg = P.xadj[s + 1] - e;
    const uint32_t nt = bfs_ntasks(deg, te);
    for (uint32_t c = lane; c < nt; c += blockDim.x) P.T[L & 1u][c] = bfs_task(s, e, deg, c, te);
    if (lane == 0) C.nT[L & 1u] = nt;
}

// Starts a reachability search from a whole seed set (for an exact sigma of a given set).
__global__ void k_seed_set(const DevProb *__restrict__ prob, const int32_t *__restrict__ seeds, int k) {
    const DevProb &P = *prob;
    DevCtr &C = *P.ctr;
    const uint32_t L = C.lvl;
    uint32_t *d0 = P.del[L % 3u];
    if (blockIdx.x == 0 && threadIdx.x == 0) C.lvl0 = L;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < k * P.W; i += gridDim.x * blockDim.x) {
        const int32_t s = seeds[i / P.W];
        const int w = i % P.W;
        const size_t at = static_cast<size_t>(s) * P.W + w;
        const uint32_t old = atomicOr(&P.vis[at], 0xFFFFFFFFu);
        if (~old) atomicOr(&d0[at], ~old);
        if (w == 0) {
            const uint32_t prev = atomicOr(&P.inS[s >> 5], 1u << (s & 31));
            if (!((prev >> (s & 31)) & 1u)) {
                P.V[L % 3u][atomicAdd(&C.nVl[L % 3u], 1u)] = s;
                bfs_tasks(P.T[L & 1u], &C.nT[L & 1u], static_cast<uint32_t>(s), P.xadj, bfs_task_edges(P.W));
            }
        }
    }
}

// Loads VW consecutive words (VW = 2 or 4) with one vector load: through L1 for read-only data (ldg) or from L2 for
// data other blocks write during the launch (ldcg).
template <int VW>
__device__ __forceinline__ void ldg_words(const uint32_t *p, uint32_t *out) {
    if constexpr (VW == 4) {
        const uint4 q = __ldg(reinterpret_cast<const uint4 *>(p));
        out[0] = q.x, out[1] = q.y, out[2] = q.z, out[3] = q.w;
    } else {
        const uint2 q = __ldg(reinterpret_cast<const uint2 *>(p));
        out[0] = q.x, out[1] = q.y;
    }
}

template <int VW>
__device__ __forceinline__ void ldcg_words(const uint32_t *p, uint32_t *out) {
    if constexpr (VW == 4) {
        const uint4 q = __ldcg(reinterpret_cast<const uint4 *>(p));
        out[0] = q.x, out[1] = q.y, out[2] = q.z, out[3] = q.w;
    } else {
        const uint2 q = __ldcg(reinterpret_cast<const uint2 *>(p));
        out[0] = q.x, out[1] = q.y;
    }
}

constexpr int kStage = 32;  // vertices a warp lists before it reserves room for them in the global lists

// Moves a warp's staged vertices (c of them, one a lane) into F_{L+1}'s list and writes their tasks for level
// L + 1: one reservation per list for the whole batch, so the list counters see one atomic per kStage listed
// vertices rather than one per listing warp.
__device__ __forceinline__ void bfs_flush(const DevProb &P, const int32_t *stage, uint32_t c, int32_t *Vn,
                                          uint32_t *nV, int4 *Tn, uint32_t *nT, int lane, int te) {
    __syncwarp();
    int32_t v = 0;
    int64_t e = 0, deg = 0;
    uint32_t k = 0;
    if (lane < static_cast<int>(c)) {
        v = stage[lane];
        e = __ldg(&P.xadj[v]);
        deg = __ldg(&P.xadj[v + 1]) - e;
        k = bfs_ntasks(deg, te);
    }
    uint32_t incl = k;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, incl, off);
        if (lane >= off) incl += y;
    }
    const uint32_t total = __shfl_sync(kFull, incl, 31);
    uint32_t vb = 0, tb = 0;
    if (lane == 0) vb = atomicAdd(nV, c);
    if (lane == 31 && total) tb = atomicAdd(nT, total);
    vb = __shfl_sync(kFull, vb, 0);
    tb = __shfl_sync(kFull, tb, 31) + incl - k;
    if (lane < static_cast<int>(c)) Vn[vb + lane] = v;
    if (k <= 2)
        for (uint32_t t = 0; t < k; ++t) Tn[tb + t] = bfs_task(static_cast<uint32_t>(v), e, deg, t, te);
    // vertices with more tasks write them with the whole warp
    for (unsigned big = __ballot_sync(kFull, k > 2); big; big &= big - 1u) {
        const int f = __ffs(big) - 1;
        const uint32_t fv = static_cast<uint32_t>(__shfl_sync(kFull, v, f));
        const int64_t fe = __shfl_sync(kFull, e, f);
        const int64_t fd = __shfl_sync(kFull, deg, f);
        const uint32_t fn = __shfl_sync(kFull, k, f);
        const uint32_t fa = __shfl_sync(kFull, tb, f);
        for (uint32_t t = lane; t < fn; t += 32) Tn[fa + t] = bfs_task(fv, fe, fd, t, te);
    }
    __syncwarp();
}

// One level L of the bit-parallel reachability search of Algorithm 1, over all simulations at once: a lane group
// per task (TE out-edges of a frontier vertex u, one a lane, 32 / TE tasks a warp; TE = 8, 16 or 32 as R/32 words
// fit a group).  The delta d of u goes out over each edge
// e = (u, v) in the simulations where e is live; bits not yet reached at v are ORed into vis[v] and into v's next
// delta, and the thread that stamps v first lists it in F_{L+1} (staged per warp in `stage`, kStage entries, and
// moved to the global list with its tasks for level L + 1 in batches).  Pushers of one level may race on a bit:
// both OR it, the same result, so no OR needs a returned value; the newly reached (v, j) are counted from the
// delta rows, each by the first task of its vertex at the next level.  The same launch zeroes the delta rows of
// F_{L-1}.
// Phases of a search level are device functions so that the persistent kernel can run many levels in one launch;
// everything another block may have written during that launch is read past L1 (__ldcg).
template <int R>
__device__ __forceinline__ void bfs_level_phase(const DevProb *__restrict__ probs, const int32_t *__restrict__ act,
                                                int nact, int32_t *stage) {
    constexpr int W = R / 32;
    constexpr int VW = W < 4 ? W : 4;  // words per vector load of a row
    // Up to 8 words (one 32-byte sector) a live row is loaded whole, together with the delta row; longer rows load
    // only the vectors where the delta has a bit.
    constexpr bool kEager = W <= 8;
    constexpr int TE = bfs_task_edges(W);  // edges of a task, one a lane of its lane group
    constexpr int NH = 32 / TE;            // tasks a warp takes at a time
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int gl = lane % TE, g0 = lane - gl;  // this lane's place in its group, and the group's first lane
    const uint32_t lt = (1u << lane) - 1u;
    const uint64_t worker = static_cast<uint64_t>(blockIdx.x) * (blockDim.x >> 5) + wib;
    const uint64_t nworkers = static_cast<uint64_t>(gridDim.x) * (blockDim.x >> 5);
    uint64_t base = 0;
    for (int q = 0; q < nact; ++q) {
        const DevProb &P = probs[act[q]];
        DevCtr &C = *P.ctr;
        if (__ldcg(&C.bdone)) continue;
        const uint32_t L = __ldcg(&C.lvl);
        const uint32_t p2 = L & 1u, p3 = L % 3u, n3 = (L + 1u) % 3u, c3 = (L + 2u) % 3u;
        const uint64_t nt = __ldcg(&C.nT[p2]);
        const uint64_t ntw = (nt + NH - 1) / NH;  // warp items of tasks: tasks NH l .. NH l + NH - 1
        const uint64_t nclw = static_cast<uint64_t>(__ldcg(&C.nVl[c3])) * W;  // delta words of F_{L-1}
        const uint64_t cnt = ntw + (nclw + 31) / 32;
        const uint64_t first = first_owned(worker, nworkers, base);
        base += cnt;
        const int4 *T = P.T[p2];
        int4 *Tn = P.T[p2 ^ 1u];
        const uint32_t *dcur = P.del[p3];
        uint32_t *dnext = P.del[n3];
        int32_t *Vn = P.V[n3];
        const uint32_t stamp = L + 1u;
        unsigned long long added = 0;
        uint32_t ns = 0;  // staged vertices of this warp
        uint64_t l = first;
        const uint64_t hq = static_cast<uint64_t>(lane / TE);  // this lane group's task of the warp item
        int4 tn = l < ntw && l * NH + hq < nt ? __ldcg(&T[l * NH + hq]) : make_int4(0, 0, 0, 0);
        for (; l < ntw; l += nworkers) {
            const int4 t = tn;  // empty (no edges, not first) past the last task
            const uint64_t ln = l + nworkers;
            if (ln < ntw) tn = ln * NH + hq < nt ? __ldcg(&T[ln * NH + hq]) : make_int4(0, 0, 0, 0);  // prefetch
            const int64_t e = static_cast<int64_t>((static_cast<uint64_t>(static_cast<uint32_t>(t.y)) << 32) |
                                                   static_cast<uint32_t>(t.x)) + gl;
            const int64_t u = static_cast<uint32_t>(t.z);
            const bool has = gl < (t.w & (kFirstTask - 1));
            const uint32_t dl = gl < W ? __ldcg(&dcur[static_cast<size_t>(u) * W + gl]) : 0u;
            if (t.w & kFirstTask) added += __popc(dl);  // u's row: the bits newly reached at u, counted once
            const int32_t v = has ? __ldg(&P.adj[e]) : 0;
            const uint32_t *lrow = P.live + static_cast<size_t>(e) * W;
            uint32_t m[W];
            if (kEager) {
#pragma unroll
                for (int c = 0; c < W; c += VW) {
                    if (has) {
                        ldg_words<VW>(lrow + c, m + c);
                    } else {
#pragma unroll
                        for (int k = 0; k < VW; ++k) m[c + k] = 0u;
                    }
                }
            }
            uint32_t any = 0;
#pragma unroll
            for (int c = 0; c < W; c += VW) {
                uint32_t d[VW], dor = 0;
#pragma unroll
                for (int k = 0; k < VW; ++k) {
                    d[k] = __shfl_sync(kFull, dl, g0 + c + k);
                    dor |= d[k];
                }
                if (!kEager) {
                    if (has && dor) {
                        ldg_words<VW>(lrow + c, m + c);
                    } else {
#pragma unroll
                        for (int k = 0; k < VW; ++k) m[c + k] = 0u;
                    }
                }
#pragma unroll
                for (int k = 0; k < VW; ++k) {
                    m[c + k] &= d[k];
                    any |= m[c + k];
                }
            }
            bool fresh = false;
            if (__any_sync(kFull, any != 0)) {
                const uint32_t *vrow = P.vis + static_cast<size_t>(v) * W;
                uint32_t x[W];
#pragma unroll
                for (int c = 0; c < W; c += VW) {
                    uint32_t mor = 0;
#pragma unroll
                    for (int k = 0; k < VW; ++k) mor |= m[c + k];
                    if (mor) {
                        ldcg_words<VW>(vrow + c, x + c);
                    } else {
#pragma unroll
                        for (int k = 0; k < VW; ++k) x[c + k] = 0u;
                    }
                }
                bool nbits = false;
#pragma unroll
                for (int k = 0; k < W; ++k) {
                    const uint32_t nb = m[k] & ~x[k];
                    if (!nb) continue;
                    const size_t at = static_cast<size_t>(v) * W + k;
                    atomicOr(&P.vis[at], nb);
                    atomicOr(&dnext[at], nb);
                    nbits = true;
                }
                if (nbits) fresh = atomicExch(&P.lstamp[v], stamp) != stamp;
            }
            // the vertices this warp stamped first go to its stage
            const unsigned mf = __ballot_sync(kFull, fresh);
            if (mf) {
                if (ns + __popc(mf) > kStage) {
                    bfs_flush(P, stage, ns, Vn, &C.nVl[n3], Tn, &C.nT[p2 ^ 1u], lane, TE);
                    ns = 0;
                }
                if (fresh) stage[ns + __popc(mf & lt)] = v;
                ns += __popc(mf);
            }
        }
        if (ns) bfs_flush(P, stage, ns, Vn, &C.nVl[n3], Tn, &C.nT[p2 ^ 1u], lane, TE);
        // zero the delta rows of F_{L-1}: level L + 1 writes its new bits there
        const int32_t *Vc = P.V[c3];
        uint32_t *dclr = P.del[c3];
        for (; l < cnt; l += nworkers) {
            const uint64_t w = (l - ntw) * 32 + lane;
            if (w < nclw) dclr[static_cast<size_t>(__ldcg(&Vc[w / W])) * W + w % W] = 0u;
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) added += __shfl_xor_sync(kFull, added, off);
        if (lane == 0 && added) atomicAdd(&C.reached, added);
    }
}

// Ends level L of problem act[q]: the search stops when F_{L+1} is empty (or at the level limit), and the counters
// of the lists and tasks level L + 1 fills are reset.
__device__ __forceinline__ void bfs_advance_one(const DevProb *__restrict__ probs, const int32_t *__restrict__ act,
                                                int q) {
    const DevProb &P = probs[act[q]];
    DevCtr &C = *P.ctr;
    if (__ldcg(&C.bdone)) return;
    const uint32_t L = __ldcg(&C.lvl);
    C.levels_total += 1;
    const bool empty = __ldcg(&C.nVl[(L + 1u) % 3u]) == 0;
    const bool lim = L + 1u - __ldcg(&C.lvl0) >= P.max_sweeps;
    C.nT[L & 1u] = 0;
    C.nVl[(L + 2u) % 3u] = 0;
    C.lvl = L + 1u;
    if (empty || lim) {
        C.bdone = 1;
        C.btimeout = (!empty && lim) ? 1u : 0u;
    }
}

// Blocks per SM the register budget is set for (85 registers a thread: no spills up to R = 512; 4 blocks measured
// no faster with the spills they cost); R = 1024 rows need more.
template <int R>
constexpr int bfs_level_min_blocks() { return R <= 512 ? 3 : 2; }

template <int R>
__global__ void __launch_bounds__(kBlock, bfs_level_min_blocks<R>())
    k_bfs_level(const DevProb *__restrict__ probs, const int32_t *__restrict__ act, int nact, GridBar *gb) {
    __shared__ int32_t stage[(kBlock / 32) * kStage];
    bfs_level_phase<R>(probs, act, nact, stage + (threadIdx.x >> 5) * kStage);
    if (last_block(gb))
        for (int q = threadIdx.x; q < nact; q += blockDim.x) bfs_advance_one(probs, act, q);
}


namespace {
__device__ __forceinline__ unsigned int ld_acquire(const unsigned int *p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
}  // namespace

// Grid-wide barrier for a cooperatively launched kernel (every block resident).  Each wait is bounded: a block that
// gives up raises gb->fail, and every block leaves the kernel at its next barrier (returns false) instead of waiting
// again, so a lost block cannot hang the device.
__device__ __forceinline__ bool grid_sync(GridBar *gb, uint32_t limit) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = ld_acquire(&gb->fail) == 0;
        if (ok) {
            const unsigned int gen = ld_acquire(&gb->gen);
            __threadfence();
            if (atomicAdd(&gb->count, 1u) == gridDim.x - 1) {
                atomicExch(&gb->count, 0u);
                __threadfence();
                atomicAdd(&gb->gen, 1u);
            } else {
                // spin first (a barrier normally opens within microseconds), then poll with short sleeps
                for (uint32_t it = 0; ld_acquire(&gb->gen) == gen; ++it) {
                    if (it >= limit || ld_acquire(&gb->fail)) {
                        atomicExch(&gb->fail, 1u);
                        ok = 0;
                        break;
                    }
                    if (it >= 4096) __nanosleep(128);
                }
            }
            __threadfence();
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// A whole reachability search (every level until every listed problem is done) in one cooperative launch: level,
// barrier, advance (block 0), barrier, stop test.
// Marks every listed problem as failed by a lost barrier (bit 2 of its fault word).
__device__ __forceinline__ void barrier_lost(const DevProb *__restrict__ probs, const int32_t *__restrict__ act,
                                             int nact) {
    for (int q = threadIdx.x; q < nact; q += blockDim.x) atomicOr(&probs[act[q]].ctr->fault, 4u);
}

constexpr int kRunBlock = 1024;  // threads per block of the persistent kernels (one block per SM: few barrier arrivals)

template <int R>
__global__ void __launch_bounds__(kRunBlock) k_bfs_run(const DevProb *__restrict__ probs,
                                                       const int32_t *__restrict__ act, int nact, GridBar *gb,
                                                       uint32_t barrier_limit) {
    __shared__ int32_t stage[(kRunBlock / 32) * kStage];
    for (;;) {
        bfs_level_phase<R>(probs, act, nact, stage + (threadIdx.x >> 5) * kStage);
        if (!grid_sync(gb, barrier_limit)) return barrier_lost(probs, act, nact);
        if (blockIdx.x == 0)
            for (int q = threadIdx.x; q < nact; q += blockDim.x) bfs_advance_one(probs, act, q);
        if (!grid_sync(gb, barrier_limit)) return barrier_lost(probs, act, nact);
        bool all = true;
        for (int q = 0; q < nact && all; ++q) all = __ldcg(&probs[act[q]].ctr->bdone) != 0;
        if (all) return;
    }
}

// M_S' <- Merge(M_S', M_s) (Eq. 3).
__global__ void k_merge(const DevProb *__restrict__ probs, const int32_t *__restrict__ act, int nact) {
    const int q = blockIdx.x;
    if (q >= nact) return;
    const DevProb &P = probs[act[q]];
    const DevCtr &C = *P.ctr;
    const uint8_t *M = C.res_par ? P.M1 : P.M0;
    const uint32_t *row = reinterpret_cast<const uint32_t *>(M + static_cast<size_t>(C.s) * P.R);
    uint32_t *ms = reinterpret_cast<uint32_t *>(P.MS);
    __shared__ uint32_t s_sum;
    if (threadIdx.x == 0) s_sum = 0;
    __syncthreads();
    uint32_t part = 0;
    for (int i = threadIdx.x; i < P.R / 4; i += blockDim.x) {
        const uint32_t x = vmax4(ms[i], row[i]);
        ms[i] = x;
        part = __dp4a(x, 0x01010101u, part);
    }
    atomicAdd(&s_sum, part);
    __syncthreads();
    if (threadIdx.x == 0) P.ctr->gms = s_sum;  // sum_j M_S'[j] after the merge
}

// Merge of the registers of k seeds and their byte sum (Eq. 3 then the sum behind Eq. 2).
__global__ void k_estimate(const DevProb *__restrict__ prob, const int32_t *__restrict__ seeds, int k,
                           unsigned long long *gsum_out) {
    const DevProb &P = *prob;
    const uint8_t *M = P.ctr->res_par ? P.M1 : P.M0;
    __shared__ unsigned long long s_sum;
    if (threadIdx.x == 0) s_sum = 0;
    __syncthreads();
    unsigned long long part = 0;
    for (int i = threadIdx.x; i < P.R / 4; i += blockDim.x) {
        uint32_t mx = 0;
        for (int a = 0; a < k; ++a)
            mx = vmax4(mx, reinterpret_cast<const uint32_t *>(M + static_cast<size_t>(seeds[a]) * P.R)[i]);
        part += __dp4a(mx, 0x01010101u, 0u);
    }
    atomicAdd(&s_sum, part);
    __syncthreads();
    if (threadIdx.x == 0) *gsum_out = s_sum;
}

// Live-simulation masks (Eq. 4-5 evaluated once per edge and simulation): bit j of live[e] is set iff edge e is
// sampled in simulation j; with them each edge's class, npairs[e] (live in at most dense_min simulations: its pair
// count) or ndense[e] = 1.  A thread per edge, in chunks of kLiveChunk consecutive edges a block (each edge's row
// found by a binary search among the chunk's rows).  The test (h XOR X_j) <= T can only pass where the top byte
// of h XOR X_j is at most T's top byte tb, so the block groups the simulations by the top byte of X_j, and an edge
// visits only the groups whose top byte is (h's top byte) XOR t, t = 0 .. tb: for t < tb every simulation of the
// group passes (its h XOR X_j is below tb * 2^24 <= T), for t = tb each is compared in full.  An edge with tb >= 128
// (p >= 1/2) tests every simulation.  A warp forms its 32 edges' masks in shared memory and writes them as one
// contiguous block.
constexpr int kLiveChunk = 2048;

template <int R>
__global__ void __launch_bounds__(kBlock) k_live_masks(const DevProb P, int32_t *npairs, int32_t *ndense) {
    constexpr int W = R / 32;
    constexpr int SW = W + 1;  // words a staged row (odd, so the lanes' rows start in different banks)
    __shared__ uint32_t sX[R];
    __shared__ uint16_t sSim[R];     // simulations grouped by the top byte of X_j
    __shared__ uint32_t sOfs[257];   // group g: sSim[sOfs[g] .. sOfs[g + 1])
    __shared__ uint32_t sCur[256];
    __shared__ uint32_t sM[kWarpsPerBlock][32 * SW];
    __shared__ int64_t s_u0, s_u1;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    for (int k = threadIdx.x; k < 257; k += blockDim.x) sOfs[k] = 0;
    __syncthreads();
    for (int j = threadIdx.x; j < R; j += blockDim.x) {
        const uint32_t x = __ldg(&P.X[j]);
        sX[j] = x;
        atomicAdd(&sOfs[(x >> 24) + 1], 1u);
    }
    __syncthreads();
    if (wib == 0) {  // inclusive scan of the 256 group sizes: sOfs[g + 1] = end of group g
        uint32_t c[8], sum = 0;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            c[i] = sOfs[1 + 8 * lane + i];
            sum += c[i];
        }
        uint32_t incl = sum;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t y = __shfl_up_sync(kFull, incl, off);
            if (lane >= off) incl += y;
        }
        uint32_t run = incl - sum;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            sCur[8 * lane + i] = run;
            run += c[i];
            sOfs[1 + 8 * lane + i] = run;
        }
    }
    __syncthreads();
    for (int j = threadIdx.x; j < R; j += blockDim.x) sSim[atomicAdd(&sCur[sX[j] >> 24], 1u)] = static_cast<uint16_t>(j);
    __syncthreads();
    const int64_t m = P.m, n = P.n;
    const uint64_t chunks = (static_cast<uint64_t>(m) + kLiveChunk - 1) / kLiveChunk;
    uint32_t *row = &sM[wib][lane * SW];
    for (uint64_t c = blockIdx.x; c < chunks; c += gridDim.x) {
        const int64_t e0 = static_cast<int64_t>(c) * kLiveChunk;
        const int64_t e1 = e0 + kLiveChunk < m ? e0 + kLiveChunk : m;
        if (threadIdx.x == 0) {  // the rows holding edges e0 and e1 - 1 (the last u with xadj[u] <= e)
            int64_t lo = 0, hi = n - 1;
            while (lo < hi) {
                const int64_t mid = (lo + hi + 1) >> 1;
                if (__ldg(&P.xadj[mid]) <= e0) lo = mid; else hi = mid - 1;
            }
            s_u0 = lo;
            hi = n - 1;
            while (lo < hi) {
                const int64_t mid = (lo + hi + 1) >> 1;
                if (__ldg(&P.xadj[mid]) <= e1 - 1) lo = mid; else hi = mid - 1;
            }
            s_u1 = lo;
        }
        __syncthreads();
        const int64_t u0 = s_u0, u1 = s_u1;
        for (int64_t eb = e0 + 32 * wib; eb < e1; eb += kBlock) {  // this warp's 32 edges
#pragma unroll
            for (int k = 0; k < W; ++k) row[k] = 0u;
            const int64_t e = eb + lane;
            uint32_t cnt = 0;
            if (e < e1) {
                int64_t lo = u0, hi = u1;
                while (lo < hi) {
                    const int64_t mid = (lo + hi + 1) >> 1;
                    if (__ldg(&P.xadj[mid]) <= e) lo = mid; else hi = mid - 1;
                }
                const int32_t v = __ldg(&P.adj[e]);
                uint32_t T = 0;
                bool ok = false;
                edge_threshold(P, e, v, T, ok);
                if (ok) {
                    const uint32_t h = edge_hash(static_cast<uint64_t>(lo), static_cast<uint64_t>(v),
                                                 static_cast<uint64_t>(n), P.undirected != 0);
                    const uint32_t tb = T >> 24;
                    if (tb >= 128) {
                        for (int k = 0; k < W; ++k) {
                            uint32_t w = 0;
#pragma unroll 8
                            for (int b = 0; b < 32; ++b) w |= ((h ^ sX[32 * k + b]) <= T ? 1u : 0u) << b;
                            row[k] = w;
                            cnt += __popc(w);
                        }
                    } else {
                        const uint32_t ht = h >> 24;
                        for (uint32_t t = 0; t <= tb; ++t) {
                            const uint32_t grp = ht ^ t;
                            const uint32_t i1 = sOfs[grp + 1];
                            for (uint32_t i = sOfs[grp]; i < i1; ++i) {
                                const uint32_t j = sSim[i];
                                if (t < tb || (h ^ sX[j]) <= T) {
                                    row[j >> 5] |= 1u << (j & 31);
                                    ++cnt;
                                }
                            }
                        }
                    }
                }
                const bool dense = cnt > static_cast<uint32_t>(P.dense_min);
                npairs[e] = dense ? 0 : static_cast<int32_t>(cnt);
                ndense[e] = dense ? 1 : 0;
            }
            __syncwarp();
            const int ne = e1 - eb < 32 ? static_cast<int>(e1 - eb) : 32;
            uint32_t *out = P.live + static_cast<size_t>(eb) * W;
            for (int q = lane; q < ne * W; q += 32) out[q] = sM[wib][(q / W) * SW + q % W];
            __syncwarp();
        }
        __syncthreads();  // the chunk's rows are read before the next chunk's replace them
    }
}

// The same classification per in-edge k (edge ein[k]), gathered from the out-edges' counts.
__global__ void __launch_bounds__(kBlock) k_inpair_counts(const DevProb P, const int32_t *__restrict__ np_out,
                                                          const int32_t *__restrict__ nd_out, int32_t *npairs,
                                                          int32_t *ndense) {
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t k = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; k < P.m; k += stride) {
        const int64_t e = __ldg(&P.ein[k]);
        npairs[k] = __ldg(&np_out[e]);
        ndense[k] = __ldg(&nd_out[e]);
    }
}

// The pairs and dense in-edges in in-CSR order: in-edge k (out-CSR edge e = ein[k], source u) gets e's out-pairs
// at ipofs[k] as (u, simulation, out-pair index) with its target v in iv, or one dense entry (u, e).  A warp takes
// kInEdgeChunk consecutive in-edges, 32 at a time: lane t loads in-edge t's source, out-CSR pair offset and row
// (a short forward walk from the previous group's row), so the dependent loads ein -> pofs of 32 in-edges are in
// flight together; then the warp writes the group's pairs 32 at a time, lane i pair i, finding the in-edge that holds
// it by a binary search over the lanes' pair offsets (shuffles), so every store is coalesced.  The dense in-edges
// follow, a thread per in-edge.
constexpr int kInEdgeChunk = 1024;

__global__ void __launch_bounds__(kBlock) k_inpair_fill(const DevProb P, int32_t *iu, uint16_t *ij, uint32_t *iop,
                                                        int32_t *iv, int32_t *idu, uint32_t *ide) {
    const int lane = threadIdx.x & 31;
    const uint64_t worker = (static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nworkers = (static_cast<uint64_t>(gridDim.x) * blockDim.x) >> 5;
    const int64_t m = P.m, n = P.n;
    const uint64_t chunks = (static_cast<uint64_t>(m) + kInEdgeChunk - 1) / kInEdgeChunk;
    for (uint64_t c = worker; c < chunks; c += nworkers) {
        const int64_t k0 = static_cast<int64_t>(c) * kInEdgeChunk;
        const int64_t k1 = k0 + kInEdgeChunk < m ? k0 + kInEdgeChunk : m;
        int32_t vb = 0;  // the in-CSR row holding in-edge k0 (the last v with xadj_in[v] <= k0)
        {
            int64_t lo = 0, hi = n - 1;
            while (lo < hi) {
                const int64_t mid = (lo + hi + 1) >> 1;
                if (__ldg(&P.xadj_in[mid]) <= k0) lo = mid; else hi = mid - 1;
            }
            vb = static_cast<int32_t>(lo);
        }
        for (int64_t kb = k0; kb < k1; kb += 32) {
            const int64_t k = kb + lane;
            const int64_t kend = kb + 32 < k1 ? kb + 32 : k1;
            const int64_t Q0 = __ldg(&P.ipofs[kb]);
            const uint32_t np = static_cast<uint32_t>(__ldg(&P.ipofs[kend]) - Q0);  // the group's pairs
            int32_t v = vb, u = 0;
            uint32_t a = 0xFFFFFFFFu;  // this in-edge's first pair, from Q0 (past the group: after every pair)
            int64_t pp0 = 0;
            if (k < kend) {
                while (__ldg(&P.xadj_in[v + 1]) <= k) ++v;
                const int64_t e = __ldg(&P.ein[k]);
                a = static_cast<uint32_t>(__ldg(&P.ipofs[k]) - Q0);
                u = __ldg(&P.adj_in[k]);
                pp0 = __ldg(&P.pofs[e]);
            }
            vb = __shfl_sync(kFull, v, 31);  // the last lane's row (a later group starts at or after it)
            for (uint32_t r = 0; r < np; r += 32) {
                const uint32_t qo = r + lane;
                // the in-edge holding pair qo: the last lane t with a_t <= qo (a is non-decreasing over the lanes)
                int t = 0;
#pragma unroll
                for (int step = 16; step > 0; step >>= 1) {
                    const uint32_t at = __shfl_sync(kFull, a, t + step);
                    if (at <= qo) t += step;
                }
                const uint32_t at = __shfl_sync(kFull, a, t);
                const int64_t pt = __shfl_sync(kFull, pp0, t);
                const int32_t ut = __shfl_sync(kFull, u, t);
                const int32_t vt = __shfl_sync(kFull, v, t);
                if (qo < np) {
                    const int64_t q = Q0 + qo;
                    const int64_t pp = pt + (qo - at);
                    iu[q] = ut;
                    // the slot map inverts itself
                    ij[q] = static_cast<uint16_t>(sw_slot(__ldg(&P.pq[pp]) & 0x3FFu, 0));
                    iv[q] = vt;
                    if (iop) iop[q] = static_cast<uint32_t>(pp);  // the same pair in out-CSR order
                }
            }
        }
    }
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t k = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; k < m; k += stride) {
        const int64_t dd = __ldg(&P.idofs[k]);
        if (__ldg(&P.idofs[k + 1]) != dd) {
            idu[dd] = __ldg(&P.adj_in[k]);
            ide[dd] = __ldg(&P.ein[k]);
        }
    }
}

// Residual blocking in the pair words of a rebuild: every in-pair (u, v, j) whose (v, j) S reached since the last
// rebuild (set in vis, not yet in vis_done) gets rank 0 in the problem's copy of the out-pair words, so the first
// sweep needs no test.  rnew (set by k_init) marks the vertices with such bits.  A thread takes 8 consecutive
// in-pairs (targets and simulations loaded as 16-byte vectors, a warp reading 1 KB of targets at once) and tests
// the blocked bits only of pairs whose target is marked; consecutive in-pairs mostly share their target (in-CSR
// order), so those tests hit the same cached words.
__global__ void __launch_bounds__(kBlock) k_block_pairs(const DevProb *__restrict__ probs,
                                                        const int32_t *__restrict__ act, int nact) {
    const uint64_t tid = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    const uint64_t nthreads = static_cast<uint64_t>(gridDim.x) * blockDim.x;
    uint64_t base = 0;
    for (int q = 0; q < nact; ++q) {
        const DevProb &P = probs[act[q]];
        if (!P.pqb || P.ctr->lvl == 0) continue;
        const uint64_t npairs = static_cast<uint64_t>(P.ipofs[P.m]);
        const uint64_t cnt = (npairs + 7) / 8;  // octets of in-pairs
        const uint64_t first = first_owned(tid, nthreads, base);
        base += cnt;
        // vector loads need 16-byte aligned octets (the device allocator aligns far more; checked, not assumed)
        const bool vec = ((reinterpret_cast<uintptr_t>(P.iv) | reinterpret_cast<uintptr_t>(P.ij)) & 15u) == 0;
        for (uint64_t o = first; o < cnt; o += nthreads) {
            const uint64_t q0 = o * 8;
            int32_t v[8];
            uint32_t j[8];
            if (vec && q0 + 8 <= npairs) {
                const int4 a = __ldg(reinterpret_cast<const int4 *>(P.iv + q0));
                const int4 b = __ldg(reinterpret_cast<const int4 *>(P.iv + q0) + 1);
                const uint4 c = __ldg(reinterpret_cast<const uint4 *>(P.ij + q0));
                v[0] = a.x, v[1] = a.y, v[2] = a.z, v[3] = a.w, v[4] = b.x, v[5] = b.y, v[6] = b.z, v[7] = b.w;
                const uint32_t cw[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    j[2 * i] = cw[i] & 0xFFFFu;
                    j[2 * i + 1] = cw[i] >> 16;
                }
            } else {
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    v[i] = q0 + i < npairs ? __ldg(&P.iv[q0 + i]) : -1;
                    j[i] = q0 + i < npairs ? __ldg(&P.ij[q0 + i]) : 0u;
                }
            }
            uint32_t marked = 0;
#pragma unroll
            for (int i = 0; i < 8; ++i)
                if (v[i] >= 0 && test_bit(P.rnew, v[i])) marked |= 1u << i;
            if (!marked) continue;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                if ((marked >> i) & 1u) {
                    const size_t w = static_cast<size_t>(v[i]) * P.W + (j[i] >> 5);
                    if (((P.vis[w] & ~P.vis_done[w]) >> (j[i] & 31)) & 1u)
                        P.pqb[__ldg(&P.iop[q0 + i])] = static_cast<uint16_t>(sw_slot(j[i], 0));  // rank 0
                }
            }
        }
    }
}

// After k_block_pairs: the newly blocked (v, j) (set in vis, not yet in vis_done) become 0 in the problem's initial
// registers Mi (residual blocking), and vis_done takes vis for the rows with new bits.  A warp per 32 vertices
// (most words of rnew are zero), a lane per 32-simulation word of a marked row.
__global__ void __launch_bounds__(kBlock) k_block_done(const DevProb *__restrict__ probs,
                                                       const int32_t *__restrict__ act, int nact) {
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const uint64_t worker = static_cast<uint64_t>(blockIdx.x) * kWarpsPerBlock + wib;
    const uint64_t nworkers = static_cast<uint64_t>(gridDim.x) * kWarpsPerBlock;
    uint64_t base = 0;
    for (int q = 0; q < nact; ++q) {
        const DevProb &P = probs[act[q]];
        if (!P.vis_done || P.ctr->lvl == 0) continue;
        const uint64_t cnt = (static_cast<uint64_t>(P.n) + 31) / 32;
        const uint64_t first = first_owned(worker, nworkers, base);
        base += cnt;
        for (uint64_t l = first; l < cnt; l += nworkers)
            for (uint32_t m = P.rnew[l]; m; m &= m - 1u) {
                const uint64_t v = l * 32 + (__ffs(m) - 1);
                const size_t row = v * static_cast<size_t>(P.W);
                for (int k = lane; k < P.W; k += 32) {
                    const uint32_t x = P.vis[row + k];
                    for (uint32_t nb = x & ~P.vis_done[row + k]; nb; nb &= nb - 1u)
                        P.Mi[v * P.R + 32u * k + (__ffs(nb) - 1)] = 0;
                    P.vis_done[row + k] = x;
                }
            }
    }
}

// Push-unit descriptor of every vertex (its in-pairs and dense in-edges).
__global__ void __launch_bounds__(kBlock) k_vertex_desc(const DevProb P, UnitD *vdesc) {
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t v = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; v < P.n; v += stride) {
        const int64_t k0 = P.xadj_in[v], k1 = P.xadj_in[v + 1];
        UnitD d;
        d.p0 = P.ipofs[k0];
        d.d0 = P.idofs[k0];
        d.np = static_cast<uint32_t>(P.ipofs[k1] - d.p0);
        d.nd = static_cast<uint32_t>(P.idofs[k1] - d.d0);
        d.u = static_cast<int32_t>(v);
        d.hu = 0;
        vdesc[v] = d;
    }
}

// Sweep-unit descriptors of every row (its whole edge range) and every task (its task_edges(deg)-edge slice).
__global__ void __launch_bounds__(kBlock) k_unit_desc(const DevProb P, UnitD *rdesc, UnitD *tdesc) {
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < P.n + P.n_tasks; i += stride) {
        int64_t u, e0, e1;
        if (i < P.n) {
            u = i;
            e0 = P.xadj[u];
            e1 = P.xadj[u + 1];
        } else {
            const int64_t task = i - P.n;
            u = P.task_row[task];
            const int64_t te = task_edges(P.xadj[u + 1] - P.xadj[u]);
            e0 = P.xadj[u] + (task - P.task_off[u]) * te;
            e1 = min(e0 + te, P.xadj[u + 1]);
        }
        UnitD d;
        d.p0 = P.pofs[e0];
        d.d0 = P.dofs[e0];
        d.np = static_cast<uint32_t>(P.pofs[e1] - d.p0);
        d.nd = static_cast<uint32_t>(P.dofs[e1] - d.d0);
        d.u = static_cast<int32_t>(u);
        d.hu = vertex_hash(static_cast<uint32_t>(u));
        // a split row's own descriptor is only read by the first sweep, which leaves the row to its tasks
        if (i < P.n && e1 - e0 > kHeavyDeg) d.u = -1;
        (i < P.n ? rdesc[i] : tdesc[i - P.n]) = d;
    }
}

// The initial registers of every (v, j): Mi[v][j] = clz(vertex_hash(v) XOR Y_j) (Algorithm 1's initialisation, no
// seed set yet).  A thread per 16-register chunk, Y staged in shared memory.
template <int R>
__global__ void __launch_bounds__(kBlock) k_init_table(const DevProb P) {
    constexpr int CH = R / 16;
    __shared__ __align__(16) uint32_t sY[R];
    for (int j = threadIdx.x; j < R; j += blockDim.x) sY[j] = __ldg(&P.Y[j]);
    __syncthreads();
    const uint64_t items = static_cast<uint64_t>(P.n) * CH;
    for (uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < items;
         i += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
        const uint32_t v = static_cast<uint32_t>(i / CH);
        const int ch = static_cast<int>(i % CH);
        reinterpret_cast<uint4 *>(P.Mi)[i] = init_chunk(sY, vertex_hash(v), ch, 0u);
    }
}

// Writes the pairs of every sparse edge at pofs[e] (simulations in increasing order) and the dense edge ids: the
// first sweep's word of every pair, and its target and simulation when pv is given (pulling sweeps after the first,
// or a rebuild that tests each pair's target).  A warp takes 32 consecutive edges, a lane each (its live mask loaded
// with 16-byte loads, Y staged in shared memory): the lanes write their pair words into a per-warp stage in shared
// memory at their offsets within the 32 edges' pairs, which are contiguous, and the warp then copies the stage out
// with coalesced stores (edges with more pairs than the stage holds write directly).
constexpr int kPairStage = 2048;  // pair words a warp stages (32 edges of at most 64 pairs each)

template <int R>
__global__ void __launch_bounds__(kBlock) k_pair_fill(const DevProb P, int32_t *pv, uint16_t *pj, uint16_t *pq,
                                                      uint32_t *dlist) {
    constexpr int W = R / 32;
    constexpr int VW = W < 4 ? W : 4;
    __shared__ uint32_t sY[R];
    __shared__ uint16_t sP[kWarpsPerBlock][kPairStage];
    for (int j = threadIdx.x; j < R; j += blockDim.x) sY[j] = __ldg(&P.Y[j]);
    __syncthreads();
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const uint64_t worker = (static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nworkers = (static_cast<uint64_t>(gridDim.x) * blockDim.x) >> 5;
    const int64_t m = P.m;
    uint16_t *stage = sP[wib];
    for (uint64_t it = worker; it < (static_cast<uint64_t>(m) + 31) / 32; it += nworkers) {
        const int64_t e0 = static_cast<int64_t>(it) * 32;
        const int64_t e1 = e0 + 32 < m ? e0 + 32 : m;
        const int64_t pb = __ldg(&P.pofs[e0]), pe = __ldg(&P.pofs[e1]);
        const bool staged = pe - pb <= kPairStage;
        const int64_t e = e0 + lane;
        if (e < e1) {
            const int64_t d0 = __ldg(&P.dofs[e]);
            if (__ldg(&P.dofs[e + 1]) != d0) {
                dlist[d0] = static_cast<uint32_t>(e);
            } else {
                const int64_t p0 = __ldg(&P.pofs[e]);
                if (__ldg(&P.pofs[e + 1]) != p0) {
                    uint32_t w[W];
#pragma unroll
                    for (int c = 0; c < W; c += VW) ldg_words<VW>(P.live + static_cast<size_t>(e) * W + c, w + c);
                    const int32_t v = __ldg(&P.adj[e]);
                    const uint32_t hv = vertex_hash(static_cast<uint32_t>(v));
                    int64_t at = p0;
#pragma unroll
                    for (int k = 0; k < W; ++k) {
                        for (uint32_t b = w[k]; b; b &= b - 1u) {
                            const uint32_t j = 32u * k + __ffs(b) - 1u;
                            if (pv) {
                                pv[at] = v;
                                pj[at] = static_cast<uint16_t>(j);
                            }
                            // the first sweep's word: accumulator slot and the initial rank of (v, j)
                            const uint16_t word = static_cast<uint16_t>(
                                sw_slot(j, 0) | (static_cast<uint32_t>(__clz(hv ^ sY[j])) << 10));
                            if (staged)
                                stage[at - pb] = word;
                            else
                                pq[at] = word;
                            ++at;
                        }
                    }
                }
            }
        }
        if (!staged) continue;  // the same for the whole warp
        __syncwarp();
        for (int64_t i = lane; i < pe - pb; i += 32) pq[pb + i] = stage[i];
        __syncwarp();
    }
}

// ------------------------------------------------------------------------------------------------------------
// Graph preparation: simulation words, in-degree / in-CSR, weighted-cascade thresholds, heavy-row tasks.

// splitmix64 output i from `seed`: the state after i+1 Weyl steps through the variant-13 mixer.
__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t i) {
    uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Simulation words (reading of Section 3.1: X_r, Y_r are the high halves of splitmix64 outputs 2r and 2r+1).
__global__ void k_words(uint64_t seed, int R, uint32_t *X, uint32_t *Y) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    const uint32_t x = static_cast<uint32_t>(splitmix64_at(seed, 2ull * r) >> 32);
    X[r] = x;
    Y[r] = static_cast<uint32_t>(splitmix64_at(seed, 2ull * r + 1) >> 32);
}

// ------------------------------------------------------------------------------------------------------------
// Influence scoring by plain sample-then-diffuse Monte Carlo (the separate influence oracle of Section 4, which
// draws with mt19937).  Sample s draws edge e's value as output (e mod kMcChunk) of its own mt19937 stream for the
// chunk of kMcChunk edges holding e (out-CSR order), seeded by init_genrand with the high half of splitmix64
// output s * nchunks + floor(e / kMcChunk) of the run seed; the edge is live iff the draw is <= its threshold.

// MT19937 (Matsumoto & Nishimura, ACM TOMACS 8(1), 1998): 624-word state seeded by init_genrand, regenerated 624
// words at a time by the twist, tempered on output.  The state lives in the thread's local memory.
struct Mt19937 {
    uint32_t mt[624];
    int i;
    __device__ __forceinline__ void seed(uint32_t s) {
        mt[0] = s;
        for (int k = 1; k < 624; ++k) mt[k] = 1812433253u * (mt[k - 1] ^ (mt[k - 1] >> 30)) + static_cast<uint32_t>(k);
        i = 624;
    }
    __device__ __forceinline__ static uint32_t twist_word(uint32_t a, uint32_t b, uint32_t far) {
        const uint32_t x = (a & 0x80000000u) | (b & 0x7FFFFFFFu);
        return far ^ (x >> 1) ^ ((x & 1u) ? 0x9908B0DFu : 0u);
    }
    // in place, in index order: words below 227 combine with old words 397 on, later ones with new words 227 back
    __device__ __forceinline__ void twist() {
        for (int k = 0; k < 227; ++k) mt[k] = twist_word(mt[k], mt[k + 1], mt[k + 397]);
        for (int k = 227; k < 623; ++k) mt[k] = twist_word(mt[k], mt[k + 1], mt[k - 227]);
        mt[623] = twist_word(mt[623], mt[0], mt[396]);
        i = 0;
    }
    __device__ __forceinline__ uint32_t next() {
        if (i >= 624) twist();
        uint32_t y = mt[i++];
        y ^= y >> 11;
        y ^= (y << 7) & 0x9D2C5680u;
        y ^= (y << 15) & 0xEFC60000u;
        y ^= y >> 18;
        return y;
    }
};

// Live masks of samples s0 .. s0 + 32 W - 1 (bit s - s0 of word (s - s0) / 32 of edge e's row): a warp takes 32
// consecutive samples over one edge chunk, a lane per sample's stream, and forms each edge's word by ballot.
// Lanes at or past nvalid (samples beyond the requested count) leave their bit 0.
template <int W>
__global__ void __launch_bounds__(kBlock) k_mc_live(const DevProb *__restrict__ prob, uint64_t seed, int64_t s0,
                                                    int64_t nvalid, int64_t nchunks) {
    const DevProb &P = *prob;
    const int lane = threadIdx.x & 31;
    const uint64_t warp = (static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = (static_cast<uint64_t>(gridDim.x) * blockDim.x) >> 5;
    Mt19937 g;
    for (uint64_t unit = warp; unit < static_cast<uint64_t>(W) * nchunks; unit += nwarps) {
        const int k = static_cast<int>(unit % W);
        const int64_t c = static_cast<int64_t>(unit / W);
        const int64_t s = static_cast<int64_t>(k) * 32 + lane;
        const bool valid = s < nvalid;
        g.seed(static_cast<uint32_t>(splitmix64_at(seed, static_cast<uint64_t>(s0 + s) * nchunks + c) >> 32));
        const int64_t e0 = c * kMcChunk;
        const int64_t e1 = e0 + kMcChunk < P.m ? e0 + kMcChunk : P.m;
        for (int64_t e = e0; e < e1; ++e) {
            const uint32_t x = g.next();
            uint32_t T;
            bool ok;
            edge_threshold(P, e, __ldg(&P.adj[e]), T, ok);
            const unsigned b = __ballot_sync(kFull, valid && ok && x <= T);
            if (lane == 0) P.live[static_cast<size_t>(e) * W + k] = b;
        }
    }
}

// Per-sample reach counts: counts[j] += |{v : bit j of vis[v]}|.  A block of 32 W threads, one per sample,
// strides over the vertices.
__global__ void k_sample_counts(const DevProb *__restrict__ prob, unsigned long long *counts) {
    const DevProb &P = *prob;
    const int j = threadIdx.x;
    unsigned long long c = 0;
    for (int64_t v = blockIdx.x; v < P.n; v += gridDim.x)
        c += (__ldcg(&P.vis[static_cast<size_t>(v) * P.W + (j >> 5)]) >> (j & 31)) & 1u;
    if (c) atomicAdd(&counts[j], c);
}

__global__ void k_indeg(const int32_t *__restrict__ adj, int64_t m, int32_t *__restrict__ indeg) {
    for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < m;
         e += static_cast<int64_t>(gridDim.x) * blockDim.x)
        atomicAdd(&indeg[adj[e]], 1);
}

__global__ void k_wc_thresholds(const int32_t *__restrict__ indeg, int64_t n, uint32_t *__restrict__ T) {
    for (int64_t v = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; v < n;
         v += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int32_t d = indeg[v];
        T[v] = d > 0 ? 0xFFFFFFFFu / static_cast<uint32_t>(d) : 0u;
    }
}

// In-CSR fill: every edge e = (u, v) takes the next free place among v's in-edges.  A block takes kTrChunk
// consecutive edges and first counts them per target in a shared-memory hash table, so a target that many of them
// share (a hub) costs one returned global atomic per block instead of one per edge; the edges then take their
// places from the block's reservation.  (The order of a vertex's in-edges is free: nothing depends on it.)
constexpr int kTrChunk = 1024;
constexpr int kTrSlots = 2048;  // hash slots (twice the edges of a chunk)
__global__ void __launch_bounds__(kBlock) k_transpose_fill(const int64_t *__restrict__ xadj,
                                                           const int32_t *__restrict__ adj, int64_t n, int64_t m,
                                                           unsigned long long *__restrict__ cursor,
                                                           int32_t *__restrict__ adj_in, uint32_t *__restrict__ ein) {
    __shared__ int32_t s_key[kTrSlots];
    __shared__ uint32_t s_cnt[kTrSlots];
    __shared__ unsigned long long s_base[kTrSlots];
    __shared__ int64_t s_u0, s_u1;
    constexpr int PER = kTrChunk / kBlock;  // edges a thread
    const uint64_t chunks = (static_cast<uint64_t>(m) + kTrChunk - 1) / kTrChunk;
    for (uint64_t c = blockIdx.x; c < chunks; c += gridDim.x) {
        const int64_t e0 = static_cast<int64_t>(c) * kTrChunk;
        const int64_t e1 = e0 + kTrChunk < m ? e0 + kTrChunk : m;
        for (int k = threadIdx.x; k < kTrSlots; k += blockDim.x) {
            s_key[k] = -1;
            s_cnt[k] = 0;
        }
        if (threadIdx.x == 0) {  // the rows holding edges e0 and e1 - 1 (the last u with xadj[u] <= e)
            int64_t lo = 0, hi = n - 1;
            while (lo < hi) {
                const int64_t mid = (lo + hi + 1) >> 1;
                if (xadj[mid] <= e0) lo = mid; else hi = mid - 1;
            }
            s_u0 = lo;
            hi = n - 1;
            while (lo < hi) {
                const int64_t mid = (lo + hi + 1) >> 1;
                if (xadj[mid] <= e1 - 1) lo = mid; else hi = mid - 1;
            }
            s_u1 = lo;
        }
        __syncthreads();
        int32_t slot[PER];
        uint32_t rank[PER];
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            const int64_t e = e0 + threadIdx.x + static_cast<int64_t>(i) * kBlock;
            slot[i] = -1;
            rank[i] = 0;
            if (e < e1) {
                const int32_t v = adj[e];
                uint32_t h = (static_cast<uint32_t>(v) * 0x9E3779B1u) >> 21;  // 11 bits: kTrSlots
                for (;;) {  // linear probing; the table has twice the chunk's edges, so a free slot exists
                    const int32_t k = atomicCAS(&s_key[h], -1, v);
                    if (k == -1 || k == v) break;
                    h = (h + 1) & (kTrSlots - 1);
                }
                slot[i] = static_cast<int32_t>(h);
                rank[i] = atomicAdd(&s_cnt[h], 1u);
            }
        }
        __syncthreads();
        for (int k = threadIdx.x; k < kTrSlots; k += blockDim.x)
            if (s_cnt[k]) s_base[k] = atomicAdd(&cursor[s_key[k]], static_cast<unsigned long long>(s_cnt[k]));
        __syncthreads();
        const int64_t u0 = s_u0, u1 = s_u1;
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            if (slot[i] < 0) continue;
            const int64_t e = e0 + threadIdx.x + static_cast<int64_t>(i) * kBlock;
            int64_t lo = u0, hi = u1;  // the row of e among the chunk's rows
            while (lo < hi) {
                const int64_t mid = (lo + hi + 1) >> 1;
                if (__ldg(&xadj[mid]) <= e) lo = mid; else hi = mid - 1;
            }
            const unsigned long long at = s_base[slot[i]] + rank[i];
            adj_in[at] = static_cast<int32_t>(lo);
            ein[at] = static_cast<uint32_t>(e);
        }
        __syncthreads();  // the table is reset for the next chunk
    }
}

__global__ void k_row_tasks(const int64_t *__restrict__ xadj, int64_t n, int32_t *__restrict__ ntask,
                            uint32_t *__restrict__ heavy) {
    for (int64_t u = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; u < n;
         u += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t d = xadj[u + 1] - xadj[u];
        const bool h = d > kHeavyDeg;
        const int64_t te = task_edges(d);
        ntask[u] = h ? static_cast<int32_t>((d + te - 1) / te) : 0;
        if (h) set_bit(heavy, u);
    }
}

// Row classes of a graph: light rows with out-edges, split rows with few / many tasks (block-compacted lists), and
// the row of every task.
__global__ void __launch_bounds__(kBlock) k_classes(const int64_t *__restrict__ xadj,
                                                    const int64_t *__restrict__ task_off, int64_t n,
                                                    int32_t *__restrict__ task_row, int32_t *light, unsigned int *nl,
                                                    int32_t *hsmall, unsigned int *nhs, int32_t *hbig,
                                                    unsigned int *nhb) {
    const int64_t words = (n + 31) >> 5;
    const uint64_t chunks = (words + kBlock - 1) / kBlock;
    for (uint64_t ch = blockIdx.x; ch < chunks; ch += gridDim.x) {
        const int64_t i = static_cast<int64_t>(ch) * kBlock + threadIdx.x;
        uint32_t wl = 0, ws = 0, wb = 0;
        if (i < words) {
            for (int b = 0; b < 32; ++b) {
                const int64_t u = i * 32 + b;
                if (u >= n) break;
                const int64_t d = xadj[u + 1] - xadj[u];
                if (d >= 1 && d <= kHeavyDeg) {
                    wl |= 1u << b;
                } else if (d > kHeavyDeg) {
                    const int64_t t0 = task_off[u], t1 = task_off[u + 1];
                    if (t1 - t0 > kBigTasks) wb |= 1u << b; else ws |= 1u << b;
                    for (int64_t k = t0; k < t1; ++k) task_row[k] = static_cast<int32_t>(u);
                }
            }
        }
        block_append_bits(wl, i, light, nl);
        block_append_bits(ws, i, hsmall, nhs);
        block_append_bits(wb, i, hbig, nhb);
    }
}

// Exclusive prefix sum of n int32 counts into n+1 int64 offsets: per-block scans, a scan of the block totals, and
// the add-back.
constexpr int kScanItems = 8;

__global__ void k_scan_blocks(const int32_t *__restrict__ in, int64_t n, int64_t *__restrict__ out,
                              int64_t *__restrict__ block_sums) {
    __shared__ int64_t s_warp[kWarpsPerBlock];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t start = (static_cast<int64_t>(blockIdx.x) * kBlock + threadIdx.x) * kScanItems;
    int64_t v[kScanItems];
    int64_t sum = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        v[i] = (start + i < n) ? in[start + i] : 0;
        sum += v[i];
    }
    int64_t incl = sum;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int64_t y = __shfl_up_sync(kFull, incl, off);
        if (lane >= off) incl += y;
    }
    if (lane == 31) s_warp[wib] = incl;
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t run = 0;
        for (int i = 0; i < kWarpsPerBlock; ++i) {
            const int64_t x = s_warp[i];
            s_warp[i] = run;
            run += x;
        }
        block_sums[blockIdx.x] = run;
    }
    __syncthreads();
    int64_t run = s_warp[wib] + incl - sum;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        if (start + i < n) out[start + i] = run;
        run += v[i];
    }
}

// Exclusive scan of the block sums in one block of kSumThreads threads: each takes a contiguous slice, the slice
// totals are scanned across the block, and each thread rewrites its slice.
constexpr int kSumThreads = 1024;
__global__ void __launch_bounds__(kSumThreads) k_scan_sums(int64_t *__restrict__ block_sums, int64_t nb,
                                                          int64_t *__restrict__ total_out) {
    __shared__ int64_t s_warp[kSumThreads / 32];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t per = (nb + kSumThreads - 1) / kSumThreads;
    const int64_t b0 = threadIdx.x * per, b1 = b0 + per < nb ? b0 + per : nb;
    int64_t sum = 0;
    for (int64_t b = b0; b < b1; ++b) sum += block_sums[b];
    int64_t incl = sum;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int64_t y = __shfl_up_sync(kFull, incl, off);
        if (lane >= off) incl += y;
    }
    if (lane == 31) s_warp[wib] = incl;
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t run = 0;
        for (int i = 0; i < kSumThreads / 32; ++i) {
            const int64_t x = s_warp[i];
            s_warp[i] = run;
            run += x;
        }
        *total_out = run;
    }
    __syncthreads();
    int64_t run = s_warp[wib] + incl - sum;
    for (int64_t b = b0; b < b1; ++b) {
        const int64_t x = block_sums[b];
        block_sums[b] = run;
        run += x;
    }
}

__global__ void k_scan_add(int64_t *__restrict__ out, int64_t n, const int64_t *__restrict__ block_sums) {
    const int64_t per = static_cast<int64_t>(kBlock) * kScanItems;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        out[i] += block_sums[i / per];
}

// Argument checks on device-resident CSR arrays: flag 0 bad ends, 1 decreasing offsets, 2 target out of range.
__global__ void k_validate(const int64_t *__restrict__ xadj, const int32_t *__restrict__ adj, int64_t n, int64_t m,
                           unsigned int *flags) {
    const int64_t tid = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t nth = static_cast<int64_t>(gridDim.x) * blockDim.x;
    if (tid == 0 && (xadj[0] != 0 || xadj[n] != m)) flags[0] = 1;
    for (int64_t u = tid; u < n; u += nth)
        if (xadj[u + 1] < xadj[u]) flags[1] = 1;
    for (int64_t e = tid; e < m; e += nth) {
        const int32_t v = adj[e];
        if (v < 0 || v >= n) flags[2] = 1;
    }
}

// Order-free 64-bit fingerprint of a graph for exported sketches: the wrapping sum over edges of a splitmix64-style
// mix of (edge index, source, target, per-edge threshold).  A warp per row.
__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
__global__ void k_graph_hash(const int64_t *__restrict__ xadj, const int32_t *__restrict__ adj, int64_t n,
                             const uint32_t *__restrict__ T_edge, unsigned long long *out) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
    unsigned long long acc = 0;
    for (int64_t u = warp; u < n; u += nwarps)
        for (int64_t e = xadj[u] + lane; e < xadj[u + 1]; e += 32) {
            const unsigned long long t = T_edge ? T_edge[e] : 0u;
            acc += mix64(static_cast<unsigned long long>(e) * 0x9E3779B97F4A7C15ull ^
                         (static_cast<unsigned long long>(u) << 32) ^ static_cast<uint32_t>(adj[e]) ^ (t << 17));
        }
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(kFull, acc, off);
    if (lane == 0 && acc) atomicAdd(out, acc);
}

// Order-free checksum of a byte array (8-byte words; bytes a multiple of 8): the wrapping sum of mix64(index, word).
__global__ void k_checksum(const unsigned long long *__restrict__ x, uint64_t words, unsigned long long *out) {
    unsigned long long acc = 0;
    for (uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < words;
         i += static_cast<uint64_t>(gridDim.x) * blockDim.x)
        acc += mix64(i * 0x9E3779B97F4A7C15ull ^ __ldg(&x[i]));
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(kFull, acc, off);
    if ((threadIdx.x & 31) == 0 && acc) atomicAdd(out, acc);
}

// Checks of an undirected input: every row strictly increasing (flag 4) and every (u, v) matched by (v, u) (flag 5,
// found by binary search in the sorted row of v).  A warp per row.
__global__ void k_validate_undirected(const int64_t *__restrict__ xadj, const int32_t *__restrict__ adj, int64_t n,
                                      unsigned int *flags) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
    for (int64_t u = warp; u < n; u += nwarps) {
        const int64_t e0 = xadj[u], e1 = xadj[u + 1];
        for (int64_t e = e0 + lane; e < e1; e += 32) {
            const int32_t v = adj[e];
            if (e > e0 && adj[e - 1] >= v) flags[4] = 1;
            int64_t lo = xadj[v], hi = xadj[v + 1];
            while (lo < hi) {
                const int64_t mid = (lo + hi) >> 1;
                if (adj[mid] < u) lo = mid + 1; else hi = mid;
            }
            if (lo >= xadj[v + 1] || adj[lo] != u) flags[5] = 1;
        }
    }
}

// Per-edge thresholds of Eq. 5: T = ceil(p * 2^32) - 1 in double (exact for float p), never live for p <= 0.
__global__ void k_edge_thresholds(const float *__restrict__ p, int64_t m, uint32_t *__restrict__ T,
                                  uint8_t *__restrict__ ok, unsigned int *flags) {
    for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < m;
         e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const double q = static_cast<double>(p[e]);
        if (!(q >= 0.0 && q <= 1.0)) flags[3] = 1;
        const bool live = q > 0.0;
        ok[e] = live ? 1 : 0;
        T[e] = live ? static_cast<uint32_t>(ceil(q * 4294967296.0) - 1.0) : 0u;
    }
}

// ------------------------------------------------------------------------------------------------------------
// Host-side launchers

static int g_sms = 0;
static int g_device = 0;
static int g_variant = 0;     // default register budget of the first-sweep kernel (IM_PROP_VARIANT)
static int g_grid_warp = 0;   // blocks for warp-striped kernels
static int g_grid_block = 0;  // blocks for block-striped kernels

cudaError_t configure(int device) {
    cudaDeviceProp prop;
    cudaError_t e = cudaGetDeviceProperties(&prop, device);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_init, kBlock, 0);
    if (e != cudaSuccess) return e;
    if (occ < 1) occ = 1;
    g_sms = prop.multiProcessorCount;
    g_device = device;
    g_grid_warp = prop.multiProcessorCount * occ;  // grid-stride kernels: one wave of 256-thread blocks
    g_grid_block = prop.multiProcessorCount * 4;
    if (const char *v = getenv("IM_PROP_VARIANT")) g_variant = atoi(v);
    return cudaSuccess;
}

template <int R, int MINB, bool FIRST>
static void launch_gather(const DevProb *probs, const int32_t *act, int nact, cudaStream_t s) {
    static int grid = 0;
    const int smem = kWarpsPerBlock * GSlots<R>::kPropBytesPerWarp;
    auto kern = FIRST ? k_first<R, MINB> : k_propg<R, MINB>;
    if (grid == 0) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        int occ = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kBlock, smem);
        grid = g_sms * (occ > 0 ? occ : 1);
    }
    kern<<<grid, kBlock, smem, s>>>(probs, act, nact);
}

template <int R, int MINB>
static void launch_push(const DevProb *probs, const int32_t *act, int nact, bool skip_full, cudaStream_t s) {
    static int grid = 0;
    if (grid == 0) {
        int occ = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_push<R, MINB>, kBlock, 0);
        grid = g_sms * (occ > 0 ? occ : 1);
    }
    k_push<R, MINB><<<grid, kBlock, 0, s>>>(probs, act, nact, skip_full ? 1 : 0);
}

template <int R>
static void launch_combines(const DevProb *probs, const int32_t *act, int nact, cudaStream_t s) {
    static int grid_s = 0, grid_b = 0;
    const int smem = kWarpsPerBlock * GSlots<R>::kBytesPerWarp;
    if (grid_s == 0) {
        cudaFuncSetAttribute(k_combine<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        cudaFuncSetAttribute(k_combine_big<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        int occ = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_combine<R>, kBlock, smem);
        grid_s = g_sms * (occ > 0 ? occ : 1);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_combine_big<R>, kBlock, smem);
        grid_b = g_sms * (occ > 0 ? occ : 1);
    }
    k_combine<R><<<grid_s, kBlock, smem, s>>>(probs, act, nact);
    k_combine_big<R><<<grid_b, kBlock, smem, s>>>(probs, act, nact);
}

#define IMK_R_SWITCH(R, CALL)                                \
    switch (R) {                                             \
        case 64: { constexpr int RR = 64; CALL; } break;     \
        case 128: { constexpr int RR = 128; CALL; } break;   \
        case 256: { constexpr int RR = 256; CALL; } break;   \
        case 512: { constexpr int RR = 512; CALL; } break;   \
        case 1024: { constexpr int RR = 1024; CALL; } break; \
        default: break;                                      \
    }

// The first sweep of the listed problems that start a diffusion.  variant: resident blocks per SM the kernel's
// register budget targets (3, 4 or 6; 0: the default, 4, or IM_PROP_VARIANT); every variant gives the same
// registers.  Then one sweep of the others (launch_prop): in k_push, or in k_propg when later sweeps pull too
// (pull_more); pulls says that launch_first ran for this sweep.  Each returns the launches.
int launch_first(int R, const DevProb *probs, const int32_t *act, int nact, int variant, cudaStream_t s) {
    switch (variant > 0 ? variant : g_variant) {
        case 3: IMK_R_SWITCH(R, (launch_gather<RR, 3, true>(probs, act, nact, s))); break;
        case 6: IMK_R_SWITCH(R, (launch_gather<RR, 6, true>(probs, act, nact, s))); break;
        default: IMK_R_SWITCH(R, (launch_gather<RR, 4, true>(probs, act, nact, s))); break;
    }
    return 1;
}
int launch_prop(int R, const DevProb *probs, const int32_t *act, int nact, bool pulls, bool pull_more,
                cudaStream_t s) {
    if (!pulls) {
        IMK_R_SWITCH(R, (launch_push<RR, kPushMinBlocks>(probs, act, nact, false, s)));
        return 1;
    }
    if (pull_more) {
        IMK_R_SWITCH(R, (launch_gather<RR, 4, false>(probs, act, nact, s)));
    } else {
        IMK_R_SWITCH(R, (launch_push<RR, kPushMinBlocks>(probs, act, nact, true, s)));
    }
    return 1;
}
void launch_combine(int R, const DevProb *probs, const int32_t *act, int nact, cudaStream_t s) {
    IMK_R_SWITCH(R, (launch_combines<RR>(probs, act, nact, s)));
}
// The frontier kernel runs one wave (its last block is found by one atomic per block).
void launch_frontier(const DevProb *probs, const int32_t *act, int nact, GridBar *gb, cudaStream_t s) {
    k_frontier<<<g_sms * 3, kBlock, 0, s>>>(probs, act, nact, gb);  // 3 blocks an SM at its register count
}
int launch_init(const DevProb *probs, const int32_t *act, int nact, cudaStream_t s) {
    k_init<<<g_grid_warp, kBlock, 0, s>>>(probs, act, nact);
    k_block_pairs<<<g_grid_warp, kBlock, 0, s>>>(probs, act, nact);
    k_block_done<<<g_grid_warp, kBlock, 0, s>>>(probs, act, nact);
    return 3;
}
template <int R>
static void launch_scan_r(const DevProb *probs, const int32_t *act, int nact, cudaStream_t s) {
    static int grid = 0;  // one wave of this R's scan kernel (its register count sets the blocks per SM)
    if (grid == 0) {
        int occ = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_scan<R>, kBlock, 0);
        grid = g_sms * (occ > 0 ? occ : 1);
    }
    k_scan<R><<<grid, kBlock, 0, s>>>(probs, act, nact);
}
void launch_scan(int R, const DevProb *probs, const int32_t *act, int nact, cudaStream_t s) {
    IMK_R_SWITCH(R, (launch_scan_r<RR>(probs, act, nact, s)));
}
int launch_celf(int R, const DevProb *probs, const int32_t *act, int nact, cudaStream_t s) {
    k_celf_max<<<g_grid_warp, kBlock, 0, s>>>(probs, act, nact);
    k_celf_tau<<<nact, 128, 0, s>>>(probs, act, nact);
    IMK_R_SWITCH(R, (k_celf_eval<RR><<<g_grid_warp, kBlock, 0, s>>>(probs, act, nact)));
    return 3;
}
void launch_choose(const DevProb *probs, const int32_t *act, int nact, int32_t step, cudaStream_t s) {
    k_choose<<<nact, kBlock, 0, s>>>(probs, act, nact, step);
}
void launch_seed_set(const DevProb *prob, const int32_t *seeds, int k, int W, cudaStream_t s) {
    k_seed_set<<<(k * W + 255) / 256, 256, 0, s>>>(prob, seeds, k);
}
template <int R>
static void launch_bfs_level_r(const DevProb *probs, const int32_t *act, int nact, GridBar *gb, cudaStream_t s) {
    static int grid = 0;  // one wave: the SM count times the blocks that fit
    if (grid == 0) {
        int occ = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_bfs_level<R>, kBlock, 0);
        grid = g_sms * (occ > 0 ? occ : 1);
    }
    k_bfs_level<R><<<grid, kBlock, 0, s>>>(probs, act, nact, gb);
}
void launch_bfs_level(int R, const DevProb *probs, const int32_t *act, int nact, GridBar *gb, cudaStream_t s) {
    IMK_R_SWITCH(R, (launch_bfs_level_r<RR>(probs, act, nact, gb, s)));
}
template <int R>
static bool launch_bfs_run_r(const DevProb *probs, const int32_t *act, int nact, GridBar *gb, uint32_t limit,
                             cudaStream_t s) {
    static int grid = -1;
    if (grid < 0) {
        int coop = 0, occ = 0;
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, g_device);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_bfs_run<R>, kRunBlock, 0);
        grid = (coop && occ > 0) ? g_sms * std::min(occ, 2) : 0;
    }
    if (grid == 0) return false;
    void *args[] = {const_cast<DevProb **>(&probs), const_cast<int32_t **>(&act), &nact, &gb, &limit};
    if (cudaMemsetAsync(gb, 0, sizeof(GridBar), s) != cudaSuccess) return false;
    if (cudaLaunchCooperativeKernel(reinterpret_cast<const void *>(k_bfs_run<R>), dim3(grid), dim3(kRunBlock), args,
                                    0, s) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return true;
}
bool launch_bfs_run(int R, const DevProb *probs, const int32_t *act, int nact, GridBar *gb, uint32_t barrier_limit,
                    cudaStream_t s) {
    bool ok = false;
    IMK_R_SWITCH(R, (ok = launch_bfs_run_r<RR>(probs, act, nact, gb, barrier_limit, s)));
    return ok;
}
void launch_merge(const DevProb *probs, const int32_t *act, int nact, cudaStream_t s) {
    k_merge<<<nact, 128, 0, s>>>(probs, act, nact);
}
void launch_estimate(const DevProb *prob, const int32_t *seeds, int k, unsigned long long *gsum, cudaStream_t s) {
    k_estimate<<<1, 256, 0, s>>>(prob, seeds, k, gsum);
}
void launch_validate(const int64_t *xadj, const int32_t *adj, int64_t n, int64_t m, unsigned int *flags,
                     cudaStream_t s) {
    k_validate<<<g_grid_block, kBlock, 0, s>>>(xadj, adj, n, m, flags);
}
void launch_checksum(const void *x, uint64_t bytes, unsigned long long *out, cudaStream_t s) {
    k_checksum<<<g_grid_block, kBlock, 0, s>>>(static_cast<const unsigned long long *>(x), bytes / 8, out);
}
void launch_graph_hash(const int64_t *xadj, const int32_t *adj, int64_t n, const uint32_t *T_edge,
                       unsigned long long *out, cudaStream_t s) {
    k_graph_hash<<<g_grid_warp, kBlock, 0, s>>>(xadj, adj, n, T_edge, out);
}
void launch_validate_undirected(const int64_t *xadj, const int32_t *adj, int64_t n, unsigned int *flags,
                                cudaStream_t s) {
    k_validate_undirected<<<g_grid_warp, kBlock, 0, s>>>(xadj, adj, n, flags);
}
void launch_edge_thresholds(const float *p, int64_t m, uint32_t *T, uint8_t *ok, unsigned int *flags,
                            cudaStream_t s) {
    if (m > 0) k_edge_thresholds<<<g_grid_block, kBlock, 0, s>>>(p, m, T, ok, flags);
}
template <int R>
static void launch_live_masks_r(const DevProb &P, int32_t *npairs, int32_t *ndense, cudaStream_t s) {
    static int grid = 0;
    if (grid == 0) {
        int occ = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_live_masks<R>, kBlock, 0);
        grid = g_sms * (occ > 0 ? occ : 1);
    }
    k_live_masks<R><<<grid, kBlock, 0, s>>>(P, npairs, ndense);
}
void launch_live_masks(const DevProb &P, int32_t *npairs, int32_t *ndense, cudaStream_t s) {
    IMK_R_SWITCH(P.R, (launch_live_masks_r<RR>(P, npairs, ndense, s)));
}
void launch_init_table(const DevProb &P, cudaStream_t s) {
    IMK_R_SWITCH(P.R, (k_init_table<RR><<<g_grid_block, kBlock, 0, s>>>(P)));
}
void launch_pair_fill(const DevProb &P, int32_t *pv, uint16_t *pj, uint16_t *pq, uint32_t *dlist, cudaStream_t s) {
    IMK_R_SWITCH(P.R, (k_pair_fill<RR><<<g_grid_warp, kBlock, 0, s>>>(P, pv, pj, pq, dlist)));
}
void launch_inpair_counts(const DevProb &P, const int32_t *np_out, const int32_t *nd_out, int32_t *npairs,
                          int32_t *ndense, cudaStream_t s) {
    k_inpair_counts<<<g_grid_block, kBlock, 0, s>>>(P, np_out, nd_out, npairs, ndense);
}
void launch_inpair_fill(const DevProb &P, int32_t *iu, uint16_t *ij, uint32_t *iop, int32_t *iv, int32_t *idu,
                        uint32_t *ide, cudaStream_t s) {
    k_inpair_fill<<<g_grid_warp, kBlock, 0, s>>>(P, iu, ij, iop, iv, idu, ide);
}
void launch_vertex_desc(const DevProb &P, UnitD *vdesc, cudaStream_t s) {
    k_vertex_desc<<<g_grid_block, kBlock, 0, s>>>(P, vdesc);
}
void launch_unit_desc(const DevProb &P, UnitD *rdesc, UnitD *tdesc, cudaStream_t s) {
    k_unit_desc<<<g_grid_block, kBlock, 0, s>>>(P, rdesc, tdesc);
}
void launch_mc_live(int R, const DevProb *prob, uint64_t seed, int64_t s0, int64_t nvalid, int64_t nchunks,
                    cudaStream_t s) {
    const int64_t warps = static_cast<int64_t>(R / 32) * nchunks;
    const int64_t cap = static_cast<int64_t>(g_sms) * 8 * kWarpsPerBlock;  // 8 blocks an SM at most
    const int blocks = static_cast<int>((std::min(warps, cap) + kWarpsPerBlock - 1) / kWarpsPerBlock);
    if (blocks > 0) IMK_R_SWITCH(R, (k_mc_live<RR / 32><<<blocks, kBlock, 0, s>>>(prob, seed, s0, nvalid, nchunks)));
}
void launch_sample_counts(int R, const DevProb *prob, unsigned long long *counts, cudaStream_t s) {
    k_sample_counts<<<g_sms * 2, R, 0, s>>>(prob, counts);
}
void launch_words(uint64_t seed, int R, uint32_t *X, uint32_t *Y, cudaStream_t s) {
    k_words<<<(R + 255) / 256, 256, 0, s>>>(seed, R, X, Y);
}
void launch_indeg(const int32_t *adj, int64_t m, int32_t *indeg, cudaStream_t s) {
    if (m > 0) k_indeg<<<g_grid_block, kBlock, 0, s>>>(adj, m, indeg);
}
void launch_wc_thresholds(const int32_t *indeg, int64_t n, uint32_t *T, cudaStream_t s) {
    k_wc_thresholds<<<g_grid_block, kBlock, 0, s>>>(indeg, n, T);
}
void launch_transpose_fill(const int64_t *xadj, const int32_t *adj, int64_t n, int64_t m, unsigned long long *cursor,
                           int32_t *adj_in, uint32_t *ein, cudaStream_t s) {
    if (m > 0) k_transpose_fill<<<g_sms * 4, kBlock, 0, s>>>(xadj, adj, n, m, cursor, adj_in, ein);
}
void launch_row_tasks(const int64_t *xadj, int64_t n, int32_t *ntask, uint32_t *heavy, cudaStream_t s) {
    k_row_tasks<<<g_grid_block, kBlock, 0, s>>>(xadj, n, ntask, heavy);
}
void launch_classes(const int64_t *xadj, const int64_t *task_off, int64_t n, int32_t *task_row, int32_t *light,
                    unsigned int *counts, int32_t *hsmall, int32_t *hbig, cudaStream_t s) {
    k_classes<<<g_grid_block, kBlock, 0, s>>>(xadj, task_off, n, task_row, light, counts, hsmall, counts + 1, hbig,
                                              counts + 2);
}
int64_t scan_block_count(int64_t n) {
    const int64_t per = static_cast<int64_t>(kBlock) * kScanItems;
    return (n + per - 1) / per;
}
int launch_exclusive_scan(const int32_t *in, int64_t n, int64_t *out, int64_t *block_sums, cudaStream_t s) {
    const int64_t nb = scan_block_count(n);
    if (nb > 0) k_scan_blocks<<<static_cast<unsigned>(nb), kBlock, 0, s>>>(in, n, out, block_sums);
    k_scan_sums<<<1, kSumThreads, 0, s>>>(block_sums, nb, out + n);
    if (nb > 1) k_scan_add<<<g_grid_block, kBlock, 0, s>>>(out, n, block_sums);
    return 1 + (nb > 0 ? 1 : 0) + (nb > 1 ? 1 : 0);
}

}  // namespace imk
