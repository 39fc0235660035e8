"""GB300-native (sm_103a) sketch-based influence maximisation after HyperFuseR (arXiv 2105.04023).

Python front end of the C ABI in ``include/im.h``.  The functions keep the C names (``im_build_sketches``,
``im_estimate``, ``im_select_seeds`` ...) and only marshal arguments: every step runs in the library's CUDA kernels.
Graphs are given as numpy arrays (copied by the library, ``IM_MEM_HOST``) or as CUDA torch tensors
(``IM_MEM_DEVICE``: used in place).
"""
from __future__ import annotations

import ctypes
import weakref
from dataclasses import dataclass

import numpy as np

from . import _lib
from ._lib import IM_BLOCK_LITERAL, IM_BLOCK_RESIDUAL, IM_IC_CONST, IM_PER_EDGE, IM_WC  # noqa: F401


class ImError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_lib.STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


def _addr(a) -> int | None:
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return int(a.data_ptr())


@dataclass
class Graph:
    """An out-neighbour CSR graph plus its diffusion model, ready to hand to the library."""

    n: int
    xadj: object  # int64[n+1]: numpy (host) or torch CUDA tensor (device)
    adj: object  # int32[m]
    model: int = IM_IC_CONST
    p: float = 0.0
    p_edge: object = None  # float32[m] for IM_PER_EDGE
    undirected: bool = False  # both directions of every edge stored, rows sorted

    def c(self) -> _lib.im_graph:
        dev = not isinstance(self.xadj, np.ndarray)
        for a in (self.xadj, self.adj, self.p_edge):
            if a is None:
                continue
            if dev and getattr(a, "is_cuda", False) is False:
                raise TypeError("mixing host and device arrays in one graph")
            if isinstance(a, np.ndarray) and not a.flags.c_contiguous:
                raise TypeError("host arrays must be C-contiguous")
        if isinstance(self.xadj, np.ndarray):
            assert self.xadj.dtype == np.int64 and self.adj.dtype == np.int32
        else:
            import torch

            assert self.xadj.dtype == torch.int64 and self.adj.dtype == torch.int32
            assert self.xadj.is_contiguous() and self.adj.is_contiguous()
        m = int(self.adj.shape[0])
        return _lib.im_graph(n=self.n, m=m, xadj=_addr(self.xadj), adj=_addr(self.adj), model=self.model, p=self.p,
                             p_edge=_addr(self.p_edge), memory=_lib.IM_MEM_DEVICE if dev else _lib.IM_MEM_HOST,
                             undirected=1 if self.undirected else 0)

    @staticmethod
    def from_synth(g, model: int, p: float = 0.0, p_edge=None, device: str | None = None,
                   undirected: bool = False) -> "Graph":
        """Wraps a ``synth.graphs.Graph``; with ``device='cuda'`` the arrays are uploaded as torch tensors."""
        if device is None:
            pe = None if p_edge is None else np.ascontiguousarray(p_edge, dtype=np.float32)
            return Graph(g.n, np.ascontiguousarray(g.xadj, np.int64), np.ascontiguousarray(g.adj, np.int32), model, p,
                         pe, undirected)
        import torch

        pe = None if p_edge is None else torch.as_tensor(np.asarray(p_edge, np.float32), device=device)
        return Graph(g.n, torch.as_tensor(g.xadj, device=device), torch.as_tensor(g.adj, device=device), model, p,
                     pe, undirected)


def params(R: int, K: int = 1, eps_g: float = 0.01, eps_l: float = 0.3, eps_c: float = 0.0, seed: int = 1,
           max_sweeps: int = 0, blocking: int = IM_BLOCK_RESIDUAL) -> _lib.im_params:
    return _lib.im_params(R=R, K=K, eps_g=eps_g, eps_l=eps_l, eps_c=eps_c, seed=seed, max_sweeps=max_sweeps,
                          blocking=blocking)


def _sync_torch():
    try:
        import torch

        if torch.cuda.is_available() and torch.cuda.is_initialized():
            torch.cuda.synchronize()
    except ImportError:
        pass


class Context:
    """An im_ctx on one CUDA device (work runs on a stream the context owns)."""

    def __init__(self, device: int = 0):
        self._L = _lib.load()
        h = ctypes.c_void_p()
        st = self._L.im_ctx_create(device, None, ctypes.byref(h))
        if st != 0:
            raise ImError(st, f"cannot create a context on CUDA device {device}")
        self.h = h
        self._children = weakref.WeakSet()  # servers and sketches, destroyed before the context

    def close(self):
        if self.h:
            for c in list(self._children):
                c.close()
            self._L.im_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st: int):
        if st != 0:
            raise ImError(st, self._L.im_last_error(self.h).decode())

    def set_timing(self, on: bool):
        self._check(self._L.im_ctx_set_timing(self.h, 1 if on else 0))

    def stats(self) -> dict:
        s = _lib.im_stats()
        self._check(self._L.im_ctx_stats(self.h, ctypes.byref(s)))
        return {k: getattr(s, k) for k, _ in _lib.im_stats._fields_}

    def im_autotune(self, graph: Graph, prm: _lib.im_params) -> dict:
        """Times the candidate launch shapes on the graph's first diffusion and keeps the fastest for its class."""
        _sync_torch()
        g = graph.c()
        t = _lib.im_tuning()
        self._check(self._L.im_autotune(self.h, ctypes.byref(g), ctypes.byref(prm), ctypes.byref(t)))
        return {k: getattr(t, k) for k, _ in _lib.im_tuning._fields_}

    # --- the C calls, same names --------------------------------------------------------------------------------
    def im_build_sketches(self, graph: Graph, prm: _lib.im_params) -> "Sketch":
        _sync_torch()
        g = graph.c()
        out = ctypes.c_void_p()
        self._check(self._L.im_build_sketches(self.h, ctypes.byref(g), ctypes.byref(prm), ctypes.byref(out)))
        return Sketch(self, out, graph.n, prm.R)

    def _select_out(self, K: int, trace: bool):
        seeds = np.zeros(K, np.int32)
        arrs = {}
        tr = None
        if trace:
            arrs = dict(seeds=np.zeros(K, np.int32), sigma=np.zeros(K, np.float64), estimate=np.zeros(K, np.float64),
                        gsum=np.zeros(K, np.uint64), rebuilt=np.zeros(K, np.uint8))
            tr = _lib.im_trace(**{k: v.ctypes.data for k, v in arrs.items()})
        return seeds, arrs, tr

    def im_select_seeds_from(self, sketch: "Sketch", prm: _lib.im_params, trace: bool = True) -> dict:
        """im_select_seeds starting from a built or imported sketch (same R, seed, eps_c and max_sweeps)."""
        _sync_torch()
        seeds, arrs, tr = self._select_out(prm.K, trace)
        sigma = ctypes.c_double()
        reb = ctypes.c_int32()
        self._check(self._L.im_select_seeds_from(self.h, sketch.h, ctypes.byref(prm), seeds.ctypes.data,
                                                 ctypes.addressof(sigma), ctypes.addressof(reb),
                                                 ctypes.byref(tr) if tr is not None else None))
        out = dict(seeds=seeds, sigma_final=sigma.value, rebuilds=reb.value)
        out.update(arrs)
        return out

    def im_sketch_import(self, graph: Graph, data: bytes) -> "Sketch":
        """A sketch recreated from im_sketch_export's bytes on the graph it was built on."""
        _sync_torch()
        g = graph.c()
        buf = np.frombuffer(data, dtype=np.uint8)
        h = ctypes.c_void_p()
        self._check(self._L.im_sketch_import(self.h, ctypes.byref(g), buf.ctypes.data, int(buf.size), ctypes.byref(h)))
        R = int(np.frombuffer(data[24:28], dtype=np.int32)[0])
        return Sketch(self, h, graph.n, R)

    def im_select_seeds(self, graph: Graph, prm: _lib.im_params, trace: bool = True) -> dict:
        _sync_torch()
        g = graph.c()
        K = prm.K
        seeds = np.zeros(K, np.int32)
        sigma = ctypes.c_double()
        reb = ctypes.c_int32()
        tr = None
        arrs = {}
        if trace:
            arrs = dict(seeds=np.zeros(K, np.int32), sigma=np.zeros(K, np.float64), estimate=np.zeros(K, np.float64),
                        gsum=np.zeros(K, np.uint64), rebuilt=np.zeros(K, np.uint8))
            tr = _lib.im_trace(**{k: v.ctypes.data for k, v in arrs.items()})
        self._check(self._L.im_select_seeds(self.h, ctypes.byref(g), ctypes.byref(prm), seeds.ctypes.data,
                                            ctypes.addressof(sigma), ctypes.addressof(reb),
                                            ctypes.byref(tr) if tr is not None else None))
        out = dict(seeds=seeds, sigma_final=sigma.value, rebuilds=reb.value)
        out.update(arrs)
        return out

    def im_select_seeds_batch(self, graphs: list[Graph], prms: list[_lib.im_params]) -> list[dict]:
        _sync_torch()
        nq = len(graphs)
        gs = (_lib.im_graph * nq)(*[g.c() for g in graphs])
        ps = (_lib.im_params * nq)(*prms)
        seeds = [np.zeros(p.K, np.int32) for p in prms]
        ptrs = (ctypes.c_void_p * nq)(*[s.ctypes.data for s in seeds])
        sig = np.zeros(nq, np.float64)
        reb = np.zeros(nq, np.int32)
        self._check(self._L.im_select_seeds_batch(self.h, nq, ctypes.addressof(gs), ctypes.addressof(ps),
                                                  ctypes.addressof(ptrs), sig.ctypes.data, reb.ctypes.data))
        return [dict(seeds=seeds[i], sigma_final=float(sig[i]), rebuilds=int(reb[i])) for i in range(nq)]

    def im_influence_mc(self, graph: Graph, seeds, nsamples: int, seed: int) -> tuple[float, np.ndarray]:
        """Sample-then-diffuse influence of a seed set over `nsamples` mt19937-sampled graphs (the scoring of
        Section 4); returns (mean reach, reach of each sample)."""
        _sync_torch()
        g = graph.c()
        S = np.ascontiguousarray(seeds, dtype=np.int32)
        reach = np.zeros(max(int(nsamples), 1), np.uint64)
        sigma = ctypes.c_double()
        self._check(self._L.im_influence_mc(self.h, ctypes.byref(g), S.ctypes.data, int(S.shape[0]), int(nsamples),
                                            int(seed) & 0xFFFFFFFFFFFFFFFF, ctypes.addressof(sigma),
                                            reach.ctypes.data))
        return sigma.value, reach[: int(nsamples)]

    def im_estimate_static(self, registers, seeds) -> tuple[float, int]:
        """Estimate of a seed set from a register matrix and seed ids already on the device (CUDA torch tensors:
        uint8 [n, R] and int32 [k]); the library allocates nothing for this call."""
        import torch

        assert registers.is_cuda and registers.dtype == torch.uint8 and registers.dim() == 2
        assert seeds.is_cuda and seeds.dtype == torch.int32 and seeds.dim() == 1
        registers = registers.contiguous()
        seeds = seeds.contiguous()
        _sync_torch()
        est = ctypes.c_double()
        g = ctypes.c_uint64()
        self._check(self._L.im_estimate_static(self.h, registers.data_ptr(), int(registers.shape[0]),
                                               int(registers.shape[1]), seeds.data_ptr(), int(seeds.shape[0]),
                                               ctypes.addressof(est), ctypes.addressof(g)))
        return est.value, g.value


class Server:
    """An im_server: resident graphs, an HBM-budgeted query queue and continuous batching on one context."""

    def __init__(self, ctx: Context, hbm_budget_bytes: int, max_active: int = 256):
        self.ctx = ctx
        h = ctypes.c_void_p()
        ctx._check(ctx._L.im_server_create(ctx.h, int(hbm_budget_bytes), int(max_active), ctypes.byref(h)))
        self.h = h
        ctx._children.add(self)
        self._keep = []
        self._K = {}

    def close(self):
        if self.h:
            self.ctx._L.im_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def im_server_add_graph(self, graph: Graph) -> int:
        _sync_torch()
        g = graph.c()
        gid = ctypes.c_int32()
        self.ctx._check(self.ctx._L.im_server_add_graph(self.h, ctypes.byref(g), ctypes.addressof(gid)))
        self._keep.append(graph)
        return gid.value

    def im_server_submit(self, graph_id: int, prm: _lib.im_params) -> int:
        t = ctypes.c_uint64()
        self.ctx._check(self.ctx._L.im_server_submit(self.h, int(graph_id), ctypes.byref(prm), ctypes.addressof(t)))
        self._K[t.value] = prm.K
        return t.value

    def im_server_footprint(self, graph_id: int, prm: _lib.im_params) -> int:
        b = ctypes.c_uint64()
        self.ctx._check(self.ctx._L.im_server_footprint(self.h, int(graph_id), ctypes.byref(prm),
                                                        ctypes.addressof(b)))
        return b.value

    def im_server_step(self) -> tuple[int, int]:
        a = ctypes.c_int32()
        q = ctypes.c_int32()
        self.ctx._check(self.ctx._L.im_server_step(self.h, ctypes.addressof(a), ctypes.addressof(q)))
        return a.value, q.value

    def im_server_poll(self, ticket: int):
        """None while queued or running, else dict(seeds, sigma_final, rebuilds); raises for failed queries."""
        K = self._K[ticket]
        seeds = np.zeros(K, np.int32)
        sig = ctypes.c_double()
        reb = ctypes.c_int32()
        st = self.ctx._L.im_server_poll(self.h, ctypes.c_uint64(ticket), seeds.ctypes.data, ctypes.addressof(sig),
                                        ctypes.addressof(reb))
        if st == _lib.IM_ENOTREADY:
            return None
        del self._K[ticket]
        self.ctx._check(st)
        return dict(seeds=seeds, sigma_final=sig.value, rebuilds=reb.value)

    def im_server_cancel(self, ticket: int):
        self.ctx._check(self.ctx._L.im_server_cancel(self.h, ctypes.c_uint64(ticket)))

    def im_server_info(self) -> dict:
        used = ctypes.c_uint64()
        kept = ctypes.c_int32()
        hits = ctypes.c_uint64()
        self.ctx._check(self.ctx._L.im_server_info(self.h, ctypes.addressof(used), ctypes.addressof(kept),
                                                   ctypes.addressof(hits)))
        return dict(used_bytes=used.value, kept_builds=kept.value, build_hits=hits.value)


class Sketch:
    """An im_sketch: registers of a built sketch, kept on the device."""

    def __init__(self, ctx: Context, h: ctypes.c_void_p, n: int, R: int):
        self.ctx, self.h, self.n, self.R = ctx, h, n, R
        ctx._children.add(self)

    def close(self):
        if self.h:
            self.ctx._L.im_sketch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def im_sketch_export(self) -> bytes:
        """The sketch as bytes: an im_sketch_header, the X and Y words, then the n*R registers."""
        size = ctypes.c_uint64()
        self.ctx._check(self.ctx._L.im_sketch_export(self.ctx.h, self.h, None, 0, ctypes.addressof(size)))
        buf = np.zeros(size.value, np.uint8)
        self.ctx._check(self.ctx._L.im_sketch_export(self.ctx.h, self.h, buf.ctypes.data, size.value,
                                                     ctypes.addressof(size)))
        return buf.tobytes()

    def im_sketch_registers(self) -> np.ndarray:
        M = np.zeros((self.n, self.R), np.uint8)
        self.ctx._check(self.ctx._L.im_sketch_registers(self.ctx.h, self.h, M.ctypes.data))
        return M

    def im_sketch_info(self, log_cap: int = 4096) -> tuple[int, int, np.ndarray]:
        sw = ctypes.c_int64()
        vi = ctypes.c_uint64()
        log = np.zeros(log_cap, np.int64)
        self.ctx._check(self.ctx._L.im_sketch_info(self.ctx.h, self.h, ctypes.addressof(sw), ctypes.addressof(vi),
                                                   log.ctypes.data, log_cap))
        return sw.value, vi.value, log[: min(sw.value, log_cap)]

    def im_estimate(self, seeds, exact: bool = False) -> tuple[float, float | None]:
        s = np.ascontiguousarray(seeds, dtype=np.int32)
        est = ctypes.c_double()
        sig = ctypes.c_double()
        self.ctx._check(self.ctx._L.im_estimate(self.ctx.h, self.h, s.ctypes.data, int(s.shape[0]),
                                                ctypes.addressof(est), ctypes.addressof(sig) if exact else None))
        return est.value, (sig.value if exact else None)
