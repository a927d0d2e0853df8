"""Oracle runs in worker processes for the full-size GPU tests (test infrastructure).

The pool is started with the "spawn" method: the test process has already initialised CUDA,
and a forked child of such a process can hang.  Workers import only the oracle and the input
generators, never the CUDA library.
"""
from __future__ import annotations

import concurrent.futures as cf
import multiprocessing as mp
import os

import numpy as np


def pool(workers: int | None = None) -> cf.ProcessPoolExecutor:
    n = workers or max(1, min(16, (os.cpu_count() or 2) - 1))
    return cf.ProcessPoolExecutor(max_workers=n, mp_context=mp.get_context("spawn"))


def batch_chunk(sub, ratio: int, mode: str):
    """Every graph of `sub` coarsened alone by the oracle; per graph its composed lift, final
    super-node count, final coarse CSR and the carried mass of its last level."""
    from oracle import oracle as O
    out = []
    for levels, total in O.coarsen_batch(sub, ratio, mode):
        last = levels[-1]
        cg = last.coarse.graph
        out.append((total, last.n_c, cg.rowptr, cg.col, cg.w, getattr(last, "mass", None)))
    return out


def chunks(B: int, parts: int):
    edges = np.linspace(0, B, parts + 1).astype(int)
    return [np.arange(edges[i], edges[i + 1]) for i in range(parts) if edges[i + 1] > edges[i]]


def coarsen_config(name: str, one_level: bool = False):
    """The oracle's coarsening of a named workload, generated in the worker: its levels and
    composed lift, or (one_level) a single level straight to n / ratio."""
    from oracle import oracle as O
    from paper_2204_11757_gb300 import inputs as I
    g, cfg = I.config_graph(name)
    if one_level:
        lv = O.coarsen_level(g, max(1, g.n // cfg["ratio"]))
        return [lv], lv.lift
    return O.coarsen(g, cfg["ratio"], cfg["mode"])


def coarsen_config_reordered(name: str):
    """The oracle's coarsening of a named workload under the adjacency-reordering option: the
    levels of the renumbered graph, the composed lift in the caller's numbering, and perm."""
    from oracle import oracle as O
    from paper_2204_11757_gb300 import inputs as I
    g, cfg = I.config_graph(name)
    return O.coarsen_reordered(g, cfg["ratio"], cfg["mode"])
