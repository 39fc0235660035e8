/*
 * Single-threaded CPU oracle for HyperFuseR (Goktürk & Kaya, arXiv 2105.04023).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or load this file; it exists so that the
 * tests, the smoke check and the benchmark's CPU baseline can compare the CUDA library against a plain, slow,
 * obviously correct restatement of the paper.  It shares no code with the CUDA library.
 *
 * What it computes, in the paper's order and notation:
 *   - FM sketch registers M_v[j], one uint8 per vertex v and Monte-Carlo simulation j (Section 2.2, Eq. 1-3),
 *     initialised as clz(hash(v) XOR hash(j)) (Algorithm 1, initialisation loop);
 *   - the hash-based fused sampling test of Section 3.1 (Eq. 4 and Eq. 5): edge (u,v) exists in simulation r iff
 *     (h(u,v) XOR X_r) / h_max < w_uv, with h_max = 2^32;
 *   - Simulate (Algorithm 2): pull-based diffusion of register maxima over sampled edges until the live set L is
 *     empty (or |L'| <= eps_c |V|), run as Jacobi sweeps (every read in a sweep sees the previous sweep's registers);
 *   - the greedy loop with error-adaptive rebuilding (Algorithm 1 and Section 3.2.1).
 *
 * Readings of the paper taken here (the CUDA library takes the same ones):
 *   R1 direction: u pulls from its out-neighbour v, M_u[j] = max(M_u[j], M_v[j]) (Algorithm 2 and Fig. 5).
 *   R2 edge hash: key = u*n + v as a 64-bit integer, h = fmix32(lo32(key) XOR fmix32(hi32(key))), where fmix32 is
 *      the MurmurHash3 finaliser (Eq. 4 names Murmur3); h_max = 2^32.
 *   R3 per-simulation words: the splitmix64 sequence (Steele, Lea & Flood 2014) seeded with the run seed; X_r is the
 *      high half of output 2r, Y_r (the "hash(j)" of the initialisation) the high half of output 2r+1.
 *   R4 live test: T = ceil(p * 2^32) - 1 and the edge is live iff (h XOR X_r) <= T, which is Eq. 5's comparison
 *      of the draw with the edge weight, P < w, with P = (h XOR X_r) / 2^32; p <= 0 never samples the edge.
 *      Weighted cascade uses p = 1/indeg(v) exactly: T = floor((2^32 - 1) / indeg(v)).
 *   R5 initial rank: rank(v, j) = clz32(fmix32(v XOR 0x9E3779B9) XOR Y_j), clz32(0) = 32.
 *   R6 blocked registers: on a rebuild every (v, j) with v in R_{G_j}(S) is set to 0 and never updated, so the
 *      rebuilt sketch is the sketch of the residual sample (Section 3.2.1: the rebuild covers only the vertices
 *      S has not reached).
 *   R7 eps_c: the diffusion stops after the first sweep with |L'| <= eps_c * |V| (Section 3.2).
 *   R8 thresholds: eps_g and eps_l are separate; a step keeps the sketch iff err_l < eps_l or err_g < eps_g;
 *      delta = 0 gives err_l = +infinity.
 *   R9 argmax: over v not in S, ties to the smallest vertex id.
 *   R10 e, sigma and the errors are computed in double from integer register sums and reach counts.
 *   R11 sigma is the mean reach of S over the same R hash-sampled graphs.
 *   R12 the rebuild decided after the K-th seed is recorded but its diffusion is not run (its sketch is never read).
 *   R15 influence scoring (the separate sample-then-diffuse oracle of the experiments, Section 4, which draws with
 *      mt19937): sample s draws edge e's value as output (e mod C) of its own mt19937 stream for the chunk of
 *      C = 8192 edges holding e (out-CSR order), seeded by init_genrand with the high half of splitmix64 output
 *      s * nchunks + floor(e / C) of the run seed; the edge is live iff the draw is <= T (R4's threshold).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_EINVAL 1
#define OR_ENOMEM 2

#define OR_IC 0
#define OR_WC 1
#define OR_PER_EDGE 2

/* FM correction factor of Eq. 2. */
static const double OR_PHI = 0.77351;

/* MurmurHash3's 32-bit finaliser (Appleby, public domain): xor-shift / multiply avalanche. */
uint32_t or_fmix32(uint32_t x)
{
    x ^= x >> 16;
    x *= 0x85EBCA6Bu;
    x ^= x >> 13;
    x *= 0xC2B2AE35u;
    x ^= x >> 16;
    return x;
}

/* The i-th output (0-based) of splitmix64 started from `seed`: the state after i+1 steps of the Weyl increment,
 * passed through the variant-13 mixer. */
uint64_t or_splitmix64(uint64_t seed, uint64_t i)
{
    uint64_t z = seed + (i + 1u) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* Reading R3: X_r and Y_r for r < R. */
void or_sim_words(uint64_t seed, int32_t R, uint32_t *X, uint32_t *Y)
{
    for (int32_t r = 0; r < R; ++r) {
        X[r] = (uint32_t)(or_splitmix64(seed, 2u * (uint64_t)r) >> 32);
        Y[r] = (uint32_t)(or_splitmix64(seed, 2u * (uint64_t)r + 1u) >> 32);
    }
}

/* Eq. 4 under reading R2. */
uint32_t or_edge_hash(int64_t u, int64_t v, int64_t n)
{
    uint64_t key = (uint64_t)u * (uint64_t)n + (uint64_t)v;
    return or_fmix32((uint32_t)key ^ or_fmix32((uint32_t)(key >> 32)));
}

/*
 * Reading R16 (undirected inputs, Section 4's undirected graphs stored with both directions): the two directions of
 * an undirected edge are one edge of the influence graph, so both take the hash of the ordered key (min, max) and
 * are live in the same simulations; a sampled undirected graph then reaches exactly the connected component.
 */
uint32_t or_edge_hash_dir(int64_t u, int64_t v, int64_t n, int32_t undirected)
{
    if (undirected && v < u) return or_edge_hash(v, u, n);
    return or_edge_hash(u, v, n);
}

int32_t or_clz32(uint32_t x)
{
    int32_t c = 0;
    if (x == 0) return 32;
    while (!(x & 0x80000000u)) {
        x <<= 1;
        ++c;
    }
    return c;
}

/* Reading R5: the FM rank of vertex v in simulation j (Algorithm 1's initialisation, Eq. 1 with one item). */
int32_t or_init_rank(int64_t v, uint32_t Yj)
{
    return or_clz32(or_fmix32((uint32_t)v ^ 0x9E3779B9u) ^ Yj);
}

/* Reading R4 for a probability p: sets *T and returns 1 if the edge can be sampled, 0 if never. */
int32_t or_threshold_from_p(double p, uint32_t *T)
{
    if (!(p > 0.0)) {
        *T = 0;
        return 0;
    }
    double c = ceil(p * 4294967296.0);
    *T = (uint32_t)(c - 1.0);
    return 1;
}

/* Eq. 5 under reading R4. */
int32_t or_is_live(uint32_t h, uint32_t Xr, uint32_t T, int32_t possible)
{
    return possible && ((h ^ Xr) <= T);
}

/* Per-edge thresholds for the three models (Section 2.1): IC constant p, WC 1/indeg(v), or one p per edge. */
int32_t or_edge_thresholds(int64_t n, int64_t m, const int64_t *xadj, const int32_t *adj, int32_t model, double p,
                           const float *p_edge, uint32_t *T, uint8_t *possible)
{
    (void)xadj;
    if (model == OR_IC) {
        uint32_t t;
        int32_t ok = or_threshold_from_p(p, &t);
        for (int64_t e = 0; e < m; ++e) {
            T[e] = t;
            possible[e] = (uint8_t)ok;
        }
        return OR_OK;
    }
    if (model == OR_WC) {
        int64_t *indeg = (int64_t *)calloc((size_t)(n > 0 ? n : 1), sizeof(int64_t));
        if (!indeg) return OR_ENOMEM;
        for (int64_t e = 0; e < m; ++e) indeg[adj[e]]++;
        for (int64_t e = 0; e < m; ++e) {
            T[e] = (uint32_t)(0xFFFFFFFFull / (uint64_t)indeg[adj[e]]);
            possible[e] = 1;
        }
        free(indeg);
        return OR_OK;
    }
    if (model == OR_PER_EDGE) {
        for (int64_t e = 0; e < m; ++e) possible[e] = (uint8_t)or_threshold_from_p((double)p_edge[e], &T[e]);
        return OR_OK;
    }
    return OR_EINVAL;
}

/* Algorithm 1, initialisation loop: M_v[j] = clz(hash(v) XOR hash(j)); blocked (v, j) get 0 (reading R6). */
void or_init_registers(int64_t n, int32_t R, const uint32_t *Y, const uint8_t *blocked, uint8_t *M)
{
    for (int64_t v = 0; v < n; ++v)
        for (int32_t j = 0; j < R; ++j) {
            size_t at = (size_t)v * (size_t)R + (size_t)j;
            M[at] = (blocked && blocked[at]) ? 0 : (uint8_t)or_init_rank(v, Y[j]);
        }
}

/*
 * Algorithm 2 (Simulate) as Jacobi sweeps.  L starts as V.  In a sweep every u with an out-neighbour v in L merges,
 * for every simulation j where (u, v) is sampled and u is not blocked, the previous sweep's M_v[j] into M_u[j]; u
 * joins L' if any of its registers grew.  The loop stops after a sweep with |L'| <= eps_c |V| (or max_sweeps > 0
 * sweeps).  Work count: every (u, v) with v in L counts R edge-simulation visits.
 * frontier_log[s] receives |L| at the start of sweep s for s < log_cap.
 */
int32_t or_simulate(int64_t n, const int64_t *xadj, const int32_t *adj, const uint32_t *T, const uint8_t *possible,
                    int32_t R, const uint32_t *X, const uint8_t *blocked, uint8_t *M, double eps_c, int64_t max_sweeps,
                    int64_t *sweeps_out, uint64_t *visits_out, int64_t *frontier_log, int64_t log_cap,
                    int32_t undirected)
{
    int64_t sweeps = 0;
    uint64_t visits = 0;
    if (n <= 0) {
        *sweeps_out = 0;
        *visits_out = 0;
        return OR_OK;
    }
    size_t bytes = (size_t)n * (size_t)R;
    uint8_t *inL = (uint8_t *)malloc((size_t)n);
    uint8_t *inL2 = (uint8_t *)malloc((size_t)n);
    uint8_t *Mold = (uint8_t *)malloc(bytes);
    if (!inL || !inL2 || !Mold) {
        free(inL);
        free(inL2);
        free(Mold);
        return OR_ENOMEM;
    }
    memset(inL, 1, (size_t)n);
    int64_t sizeL = n;
    for (;;) {
        if (sweeps < log_cap) frontier_log[sweeps] = sizeL;
        memcpy(Mold, M, bytes);
        memset(inL2, 0, (size_t)n);
        int64_t sizeL2 = 0;
        for (int64_t u = 0; u < n; ++u) {
            int changed = 0;
            for (int64_t e = xadj[u]; e < xadj[u + 1]; ++e) {
                int64_t v = adj[e];
                if (!inL[v]) continue;
                visits += (uint64_t)R;
                uint32_t h = or_edge_hash_dir(u, v, n, undirected);
                for (int32_t j = 0; j < R; ++j) {
                    size_t at = (size_t)u * (size_t)R + (size_t)j;
                    if (!or_is_live(h, X[j], T[e], possible[e])) continue;
                    if (blocked && blocked[at]) continue;
                    uint8_t mv = Mold[(size_t)v * (size_t)R + (size_t)j];
                    if (mv > M[at]) {
                        M[at] = mv;
                        changed = 1;
                    }
                }
            }
            if (changed) {
                inL2[u] = 1;
                ++sizeL2;
            }
        }
        ++sweeps;
        uint8_t *t = inL;
        inL = inL2;
        inL2 = t;
        sizeL = sizeL2;
        if ((double)sizeL <= (double)n * eps_c) break;
        if (max_sweeps > 0 && sweeps >= max_sweeps) break;
    }
    free(inL);
    free(inL2);
    free(Mold);
    *sweeps_out = sweeps;
    *visits_out = visits;
    return OR_OK;
}

/*
 * Adds seed s to the reach sets (Algorithm 1: the set S reaches, in every simulation): for every simulation
 * j a breadth-first search from s over the edges sampled in j, not entering vertices already in R_{G_j}(S).
 * `reached` holds one byte per (v, j).  Returns how many (v, j) pairs were newly reached.
 */
int64_t or_reach_add(int64_t n, const int64_t *xadj, const int32_t *adj, const uint32_t *T, const uint8_t *possible,
                     int32_t R, const uint32_t *X, int64_t s, uint8_t *reached, int32_t undirected)
{
    int64_t added = 0;
    int64_t *queue = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    if (!queue) return -1;
    for (int32_t j = 0; j < R; ++j) {
        if (reached[(size_t)s * (size_t)R + (size_t)j]) continue;
        int64_t head = 0, tail = 0;
        reached[(size_t)s * (size_t)R + (size_t)j] = 1;
        queue[tail++] = s;
        ++added;
        while (head < tail) {
            int64_t u = queue[head++];
            for (int64_t e = xadj[u]; e < xadj[u + 1]; ++e) {
                int64_t v = adj[e];
                size_t at = (size_t)v * (size_t)R + (size_t)j;
                if (reached[at]) continue;
                if (!or_is_live(or_edge_hash_dir(u, v, n, undirected), X[j], T[e], possible[e])) continue;
                reached[at] = 1;
                queue[tail++] = v;
                ++added;
            }
        }
    }
    free(queue);
    return added;
}

/* Eq. 2 on the integer register sum g of an R-register sketch. */
double or_estimate_from_sum(uint64_t g, int32_t R)
{
    return exp2((double)g / (double)R) / OR_PHI;
}

/* Registers after a fresh build: initialisation then Simulate with no blocked set. */
int32_t or_build(int64_t n, int64_t m, const int64_t *xadj, const int32_t *adj, int32_t model, double p,
                 const float *p_edge, int32_t R, uint64_t seed, double eps_c, uint8_t *M, int64_t *sweeps_out,
                 uint64_t *visits_out, int64_t *frontier_log, int64_t log_cap, int32_t undirected)
{
    uint32_t *X = (uint32_t *)malloc((size_t)R * 4), *Y = (uint32_t *)malloc((size_t)R * 4);
    uint32_t *T = (uint32_t *)malloc((size_t)(m > 0 ? m : 1) * 4);
    uint8_t *possible = (uint8_t *)malloc((size_t)(m > 0 ? m : 1));
    int32_t rc = OR_ENOMEM;
    if (X && Y && T && possible) {
        or_sim_words(seed, R, X, Y);
        rc = or_edge_thresholds(n, m, xadj, adj, model, p, p_edge, T, possible);
        if (rc == OR_OK) {
            or_init_registers(n, R, Y, NULL, M);
            rc = or_simulate(n, xadj, adj, T, possible, R, X, NULL, M, eps_c, 0, sweeps_out, visits_out, frontier_log,
                             log_cap, undirected);
        }
    }
    free(X);
    free(Y);
    free(T);
    free(possible);
    return rc;
}

/*
 * Algorithm 1 with the error-adaptive rebuild of Section 3.2.1.  Per step k the outputs are the seed, sigma (mean
 * reach of S over the R samples), e (the sketch estimate of the gain since the last rebuild), the integer register
 * sum behind e, and whether the error check asked for a rebuild.  Totals: edge-simulation visits and sweeps over all
 * diffusions, and the number of diffusions run.
 * literal: the rebuild as Algorithms 1 and 2 print it (reading R17): every register is re-initialised to its rank
 * and Simulate only leaves the blocked (u, j) un-updated, so a blocked vertex keeps its rank and still passes it to
 * unblocked in-neighbours; otherwise (reading R6) blocked registers are 0.  undirected: reading R16.
 */
int32_t or_select_seeds(int64_t n, int64_t m, const int64_t *xadj, const int32_t *adj, int32_t model, double p,
                        const float *p_edge, int32_t R, int32_t K, double eps_g, double eps_l, double eps_c,
                        uint64_t seed, int32_t *seeds, double *sigma_out, double *est_out, uint64_t *gsum_out,
                        uint8_t *rebuilt_out, uint64_t *visits_total, int64_t *sweeps_total, int32_t *builds_out,
                        int32_t literal, int32_t undirected)
{
    if (n <= 0 || K < 1 || K > n || R < 1) return OR_EINVAL;
    size_t bytes = (size_t)n * (size_t)R;
    uint32_t *X = (uint32_t *)malloc((size_t)R * 4), *Y = (uint32_t *)malloc((size_t)R * 4);
    uint32_t *T = (uint32_t *)malloc((size_t)(m > 0 ? m : 1) * 4);
    uint8_t *possible = (uint8_t *)malloc((size_t)(m > 0 ? m : 1));
    uint8_t *M = (uint8_t *)malloc(bytes);
    uint8_t *reached = (uint8_t *)calloc(bytes, 1);
    uint8_t *inS = (uint8_t *)calloc((size_t)n, 1);
    uint8_t *MS = (uint8_t *)calloc((size_t)R, 1);
    int32_t rc = OR_ENOMEM;
    uint64_t visits = 0;
    int64_t sweeps = 0;
    int32_t builds = 0;
    if (!X || !Y || !T || !possible || !M || !reached || !inS || !MS) goto done;
    or_sim_words(seed, R, X, Y);
    rc = or_edge_thresholds(n, m, xadj, adj, model, p, p_edge, T, possible);
    if (rc != OR_OK) goto done;

    /* S <- {}; initial registers; M <- Simulate(G, M, J, {}); M_S' <- 0; varsigma <- 0 */
    or_init_registers(n, R, Y, NULL, M);
    {
        int64_t sw;
        uint64_t vi;
        rc = or_simulate(n, xadj, adj, T, possible, R, X, NULL, M, eps_c, 0, &sw, &vi, NULL, 0, undirected);
        if (rc != OR_OK) goto done;
        sweeps += sw;
        visits += vi;
        ++builds;
    }
    double varsigma = 0.0;
    int64_t reach_count = 0;
    for (int32_t k = 0; k < K; ++k) {
        /* s <- argmax_{v not in S} Estimate(Merge(M_S', M_v)); the estimate is increasing in the register sum */
        int64_t best = -1;
        uint64_t best_g = 0;
        for (int64_t v = 0; v < n; ++v) {
            if (inS[v]) continue;
            uint64_t g = 0;
            const uint8_t *row = M + (size_t)v * (size_t)R;
            for (int32_t j = 0; j < R; ++j) g += (uint64_t)(row[j] > MS[j] ? row[j] : MS[j]);
            if (best < 0 || g > best_g) {
                best = v;
                best_g = g;
            }
        }
        int64_t s = best;
        inS[s] = 1;
        seeds[k] = (int32_t)s;
        /* e <- Estimate(Merge(M_S', M_s)) */
        double e = or_estimate_from_sum(best_g, R);
        /* R_G(S) and the Monte-Carlo influence sigma over the same R samples */
        int64_t added = or_reach_add(n, xadj, adj, T, possible, R, X, s, reached, undirected);
        if (added < 0) {
            rc = OR_ENOMEM;
            goto done;
        }
        reach_count += added;
        double sigma = (double)reach_count / (double)R;
        double delta = sigma - varsigma;
        double err_l = (delta == 0.0) ? INFINITY : fabs((e - delta) / delta);
        double err_g = fabs((e - delta) / sigma);
        sigma_out[k] = sigma;
        est_out[k] = e;
        gsum_out[k] = best_g;
        if (err_l < eps_l || err_g < eps_g) {
            /* M_S' <- Merge(M_S', M_s) */
            const uint8_t *row = M + (size_t)s * (size_t)R;
            for (int32_t j = 0; j < R; ++j)
                if (row[j] > MS[j]) MS[j] = row[j];
            rebuilt_out[k] = 0;
        } else {
            rebuilt_out[k] = 1;
            if (k + 1 < K) {
                /* re-initialise with R_G(S) blocked, M <- Simulate(G, M, J, R_G(S)) */
                int64_t sw;
                uint64_t vi;
                or_init_registers(n, R, Y, literal ? NULL : reached, M);
                rc = or_simulate(n, xadj, adj, T, possible, R, X, reached, M, eps_c, 0, &sw, &vi, NULL, 0, undirected);
                if (rc != OR_OK) goto done;
                sweeps += sw;
                visits += vi;
                ++builds;
            }
            memset(MS, 0, (size_t)R);
            varsigma = sigma;
        }
    }
    rc = OR_OK;
done:
    if (visits_total) *visits_total = visits;
    if (sweeps_total) *sweeps_total = sweeps;
    if (builds_out) *builds_out = builds;
    free(X);
    free(Y);
    free(T);
    free(possible);
    free(M);
    free(reached);
    free(inS);
    free(MS);
    return rc;
}

/* Estimate of a seed set on a built sketch (Eq. 3 merge of the seeds' registers, then Eq. 2). */
double or_estimate_set(int64_t n, int32_t R, const uint8_t *M, const int32_t *S, int32_t k, uint64_t *gsum_out)
{
    (void)n;
    uint64_t g = 0;
    for (int32_t j = 0; j < R; ++j) {
        uint8_t mx = 0;
        for (int32_t i = 0; i < k; ++i) {
            uint8_t x = M[(size_t)S[i] * (size_t)R + (size_t)j];
            if (x > mx) mx = x;
        }
        g += mx;
    }
    if (gsum_out) *gsum_out = g;
    return or_estimate_from_sum(g, R);
}

/*
 * One register by its definition (Section 2.2 with Algorithm 2's fixpoint): M_v[j] is the largest initial rank over
 * the vertices that v reaches in sample j.  Breadth-first search over the edges sampled in j.  `seen` is caller
 * scratch of n bytes, all zero on entry and returned all zero; `queue` holds n entries.
 */
int32_t or_register_at(int64_t n, const int64_t *xadj, const int32_t *adj, const uint32_t *T, const uint8_t *possible,
                       const uint32_t *X, const uint32_t *Y, int64_t v, int32_t j, uint8_t *seen, int64_t *queue,
                       int32_t undirected)
{
    int64_t head = 0, tail = 0;
    int32_t best = 0;
    seen[v] = 1;
    queue[tail++] = v;
    while (head < tail) {
        int64_t u = queue[head++];
        int32_t r = or_init_rank(u, Y[j]);
        if (r > best) best = r;
        for (int64_t e = xadj[u]; e < xadj[u + 1]; ++e) {
            int64_t w = adj[e];
            if (seen[w]) continue;
            if (!or_is_live(or_edge_hash_dir(u, w, n, undirected), X[j], T[e], possible[e])) continue;
            seen[w] = 1;
            queue[tail++] = w;
        }
    }
    for (int64_t i = 0; i < tail; ++i) seen[queue[i]] = 0;
    return best;
}

/*
 * MT19937 (Matsumoto & Nishimura, "Mersenne Twister: a 623-dimensionally equidistributed uniform pseudo-random
 * number generator", ACM TOMACS 8(1), 1998): a 624-word state seeded by init_genrand, regenerated 624 words at a
 * time by the twist (lower 31 bits of the next word joined to the top bit of this one, shifted, XORed with the
 * matrix row 0x9908B0DF when odd, and with the word 397 places on), and tempered on output.
 */
typedef struct {
    uint32_t mt[624];
    int32_t i;
} or_mt19937;

void or_mt_seed(or_mt19937 *g, uint32_t s)
{
    g->mt[0] = s;
    for (int32_t i = 1; i < 624; ++i) g->mt[i] = 1812433253u * (g->mt[i - 1] ^ (g->mt[i - 1] >> 30)) + (uint32_t)i;
    g->i = 624;
}

static void or_mt_twist(or_mt19937 *g)
{
    for (int32_t i = 0; i < 624; ++i) {
        uint32_t x = (g->mt[i] & 0x80000000u) | (g->mt[(i + 1) % 624] & 0x7FFFFFFFu);
        uint32_t xa = x >> 1;
        if (x & 1u) xa ^= 0x9908B0DFu;
        g->mt[i] = g->mt[(i + 397) % 624] ^ xa;
    }
    g->i = 0;
}

uint32_t or_mt_next(or_mt19937 *g)
{
    if (g->i >= 624) or_mt_twist(g);
    uint32_t y = g->mt[g->i++];
    y ^= y >> 11;
    y ^= (y << 7) & 0x9D2C5680u;
    y ^= (y << 15) & 0xEFC60000u;
    y ^= y >> 18;
    return y;
}

/* The first `count` outputs of the generator seeded with s (for the pins). */
void or_mt_outputs(uint32_t s, int64_t count, uint32_t *out)
{
    or_mt19937 g;
    or_mt_seed(&g, s);
    for (int64_t i = 0; i < count; ++i) out[i] = or_mt_next(&g);
}

#define OR_MC_CHUNK 8192

/* Reading R15: the seed of sample s's stream for edge chunk c. */
uint32_t or_mc_stream_seed(uint64_t seed, int64_t s, int64_t c, int64_t nchunks)
{
    return (uint32_t)(or_splitmix64(seed, (uint64_t)s * (uint64_t)nchunks + (uint64_t)c) >> 32);
}

/* Reading R15: live[e] = 1 iff edge e is live in sample s. */
int32_t or_mc_live(int64_t m, const uint32_t *T, const uint8_t *possible, uint64_t seed, int64_t s, uint8_t *live)
{
    const int64_t nchunks = (m + OR_MC_CHUNK - 1) / OR_MC_CHUNK;
    or_mt19937 g;
    for (int64_t c = 0; c < nchunks; ++c) {
        or_mt_seed(&g, or_mc_stream_seed(seed, s, c, nchunks));
        const int64_t e1 = (c + 1) * OR_MC_CHUNK < m ? (c + 1) * OR_MC_CHUNK : m;
        for (int64_t e = c * OR_MC_CHUNK; e < e1; ++e) {
            const uint32_t x = or_mt_next(&g);
            live[e] = (uint8_t)(possible[e] && x <= T[e]);
        }
    }
    return OR_OK;
}

/*
 * Influence of a seed set by plain sample-then-diffuse Monte Carlo (the influence oracle of Section 4): in each of
 * the N samples s0 .. s0 + N - 1 every edge is drawn live or not (reading R15), and a breadth-first search from S
 * over the live edges counts the vertices reached.  reach[i] gets sample s0 + i's count (nullable); returns the
 * total over the samples, or a negative value on error.
 */
int64_t or_influence_mc(int64_t n, int64_t m, const int64_t *xadj, const int32_t *adj, int32_t model, double p,
                        const float *p_edge, const int32_t *S, int32_t k, int64_t s0, int64_t N, uint64_t seed,
                        int64_t *reach)
{
    uint32_t *T = (uint32_t *)malloc((size_t)(m > 0 ? m : 1) * sizeof(uint32_t));
    uint8_t *possible = (uint8_t *)malloc((size_t)(m > 0 ? m : 1));
    uint8_t *live = (uint8_t *)malloc((size_t)(m > 0 ? m : 1));
    uint8_t *seen = (uint8_t *)calloc((size_t)(n > 0 ? n : 1), 1);
    int64_t *queue = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    int64_t total = 0;
    if (!T || !possible || !live || !seen || !queue) {
        total = -OR_ENOMEM;
        goto done;
    }
    if (or_edge_thresholds(n, m, xadj, adj, model, p, p_edge, T, possible) != OR_OK) {
        total = -OR_EINVAL;
        goto done;
    }
    for (int64_t s = s0; s < s0 + N; ++s) {
        or_mc_live(m, T, possible, seed, s, live);
        int64_t head = 0, tail = 0;
        for (int32_t i = 0; i < k; ++i) {
            if (seen[S[i]]) continue;
            seen[S[i]] = 1;
            queue[tail++] = S[i];
        }
        while (head < tail) {
            const int64_t u = queue[head++];
            for (int64_t e = xadj[u]; e < xadj[u + 1]; ++e) {
                const int64_t v = adj[e];
                if (seen[v] || !live[e]) continue;
                seen[v] = 1;
                queue[tail++] = v;
            }
        }
        if (reach) reach[s - s0] = tail;
        total += tail;
        for (int64_t i = 0; i < tail; ++i) seen[queue[i]] = 0;
    }
done:
    free(T);
    free(possible);
    free(live);
    free(seen);
    free(queue);
    return total;
}
