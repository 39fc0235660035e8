"""Planted mistakes: each case compiles the oracle with one plausible mistake and requires a pin of
``test_oracle_pins.py`` to fail on it, so the pins are shown to bite (a dropped term, a wrong sign, index or
operand, a wrong constant).  CPU only; the mistakes are planted in a temporary copy of the oracle, never in the
CUDA path."""
from __future__ import annotations

import os
import subprocess
import sys

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.c")

MUTATIONS = {
    # Eq. 5 under reading R4: the live test's compare off by one
    "live_compare": ("return possible && ((h ^ Xr) <= T);", "return possible && ((h ^ Xr) < T);"),
    # Algorithm 2 as Jacobi sweeps: reading the registers being written (Gauss-Seidel)
    "gauss_seidel": ("uint8_t mv = Mold[(size_t)v * (size_t)R + (size_t)j];",
                     "uint8_t mv = M[(size_t)v * (size_t)R + (size_t)j];"),
    # reading R6: the blocked-register test dropped
    "blocked_dropped": ("if (blocked && blocked[at]) continue;", "if (0) continue;"),
    # reading R5: a wrong vertex hash
    "vertex_hash": ("or_fmix32((uint32_t)v ^ 0x9E3779B9u)", "or_fmix32((uint32_t)v ^ 0x9E3779B8u)"),
    # reading R9: ties to the largest id
    "tie_break": ("if (best < 0 || g > best_g)", "if (best < 0 || g >= best_g)"),
    # Section 3.2.1: err_g divided by delta instead of sigma
    "err_g_denominator": ("double err_g = fabs((e - delta) / sigma);", "double err_g = fabs((e - delta) / delta);"),
    # MT19937: a tempering mask bit (bit 12; the low 7 bits of y << 7 are zero, so a change there is no mistake),
    # the twist's far offset, the seeding multiplier
    "mt_temper": ("y ^= (y << 7) & 0x9D2C5680u;", "y ^= (y << 7) & 0x9D2C4680u;"),
    "mt_twist_offset": ("g->mt[(i + 397) % 624]", "g->mt[(i + 396) % 624]"),
    "mt_seeding": ("1812433253u", "1812433255u"),
    # reading R15: sample and chunk swapped in the stream index
    "mc_stream_index": ("(uint64_t)s * (uint64_t)nchunks + (uint64_t)c", "(uint64_t)c * (uint64_t)nchunks + (uint64_t)s"),
    # reading R15: a draw equal to the threshold read as dead
    "mc_live_compare": ("live[e] = (uint8_t)(possible[e] && x <= T[e]);", "live[e] = (uint8_t)(possible[e] && x < T[e]);"),
    # the scorer counting a repeated seed twice
    "mc_seed_repeat": ("if (seen[S[i]]) continue;", "if (0) continue;"),
    # reading R3: X and Y drawn from the same splitmix64 outputs
    "sim_words_index": ("Y[r] = (uint32_t)(or_splitmix64(seed, 2u * (uint64_t)r + 1u) >> 32);",
                        "Y[r] = (uint32_t)(or_splitmix64(seed, 2u * (uint64_t)r) >> 32);"),
    # reading R2: the edge key's halves combined the other way round
    "edge_hash_halves": ("return or_fmix32((uint32_t)key ^ or_fmix32((uint32_t)(key >> 32)));",
                         "return or_fmix32((uint32_t)(key >> 32) ^ or_fmix32((uint32_t)key));"),
    # reading R4 for weighted cascade: a threshold one too large
    "wc_threshold": ("T[e] = (uint32_t)(0xFFFFFFFFull / (uint64_t)indeg[adj[e]]);",
                     "T[e] = (uint32_t)(0xFFFFFFFFull / (uint64_t)indeg[adj[e]]) + 1u;"),
    # reading R14: the visits of a sweep miscounted
    "visits": ("visits += (uint64_t)R;", "visits += (uint64_t)R + 1u;"),
    # reading R7: the eps_c stop one frontier vertex early (a change that never stops would hang the pins instead)
    "eps_c_stop": ("if ((double)sizeL <= (double)n * eps_c) break;",
                   "if ((double)sizeL <= (double)n * eps_c + 1.0) break;"),
    # Algorithm 1's reach: an edge's liveness taken from the next simulation's word (a search that re-entered reached
    # vertices would overrun its queue instead)
    "reach_wrong_simulation": ("if (!or_is_live(or_edge_hash_dir(u, v, n, undirected), X[j], T[e], possible[e])) continue;",
                               "if (!or_is_live(or_edge_hash_dir(u, v, n, undirected), X[(j + 1) % R], T[e], possible[e])) "
                               "continue;"),
    # Eq. 2: the FM correction factor
    "phi": ("static const double OR_PHI = 0.77351;", "static const double OR_PHI = 0.7735;"),
    # Eq. 3: M_S' merged with a min instead of a max
    "merge_min": ("if (row[j] > MS[j]) MS[j] = row[j];", "if (row[j] < MS[j]) MS[j] = row[j];"),
    # Section 3.2.1: the rebuild without the reached registers blocked
    "rebuild_unblocked": ("or_init_registers(n, R, Y, literal ? NULL : reached, M);",
                          "or_init_registers(n, R, Y, NULL, M);"),
    # reading R17: the literal rebuild zeroing the blocked registers as the residual one does
    "literal_zeroes": ("or_init_registers(n, R, Y, literal ? NULL : reached, M);",
                       "or_init_registers(n, R, Y, reached, M);"),
    # reading R16: an undirected edge hashed by its direction
    "undirected_key": ("if (undirected && v < u) return or_edge_hash(v, u, n);", "if (0) return or_edge_hash(v, u, n);"),
    # reading R8: the sketch kept only when both errors are small
    "keep_rule_and": ("if (err_l < eps_l || err_g < eps_g) {", "if (err_l < eps_l && err_g < eps_g) {"),
    # reading R9: seeds already in S scanned again
    "argmax_includes_S": ("if (inS[v]) continue;", "if (0) continue;"),
    # reading R8: delta = 0 read as no local error
    "err_l_delta_zero": ("double err_l = (delta == 0.0) ? INFINITY : fabs((e - delta) / delta);",
                         "double err_l = (delta == 0.0) ? 0.0 : fabs((e - delta) / delta);"),
    # reading R12: the rebuild after the K-th seed run anyway
    "last_rebuild_run": ("if (k + 1 < K) {", "if (k < K) {"),
    # the sweep limit one sweep late, the empty-graph guard, the K <= n check (found by an operator sweep)
    "sweep_limit": ("if (max_sweeps > 0 && sweeps >= max_sweeps) break;",
                    "if (max_sweeps > 0 && sweeps > max_sweeps) break;"),
    "empty_graph_guard": ("    if (n <= 0) {\n        *sweeps_out = 0;", "    if (n < 0) {\n        *sweeps_out = 0;"),
    "k_zero_accepted": ("if (n <= 0 || K < 1 || K > n || R < 1) return OR_EINVAL;",
                        "if (n <= 0 || K < 0 || K > n || R < 1) return OR_EINVAL;"),
    # Algorithm 2's L: every out-neighbour pulled from, not only those that changed
    "frontier_ignored": ("if (!inL[v]) continue;", "if (0) continue;"),
    # reading R4: the threshold rounded down instead of up
    "threshold_rounding": ("double c = ceil(p * 4294967296.0);", "double c = floor(p * 4294967296.0);"),
    # reading R3: X drawn from the next splitmix64 output
    "sim_words_shift": ("X[r] = (uint32_t)(or_splitmix64(seed, 2u * (uint64_t)r) >> 32);",
                        "X[r] = (uint32_t)(or_splitmix64(seed, 2u * (uint64_t)r + 2u) >> 32);"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_a_pin_catches_the_planted_mistake(name, tmp_path):
    old, new = MUTATIONS[name]
    text = open(SRC).read()
    assert text.count(old) == 1, f"mutation site of {name} not found exactly once"
    src = tmp_path / "oracle_mutant.c"
    src.write_text(text.replace(old, new))
    lib = oracle.compile_source(str(src), str(tmp_path / "liboracle_mutant.so"))
    env = dict(os.environ, ORACLE_LIBRARY=lib)
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", "test_oracle_pins.py"), "-x",
                        "-q", "-p", "no:cacheprovider"], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode != 0, f"no pin failed with the planted mistake {name}:\n{r.stdout[-2000:]}"
    assert "failed" in r.stdout, r.stdout[-2000:]
