"""PyTorch-facing API of the GB300 coarsener.

PyTorch provides device memory (the library's workspace comes from PyTorch's caching allocator
through the C ABI's allocator callbacks), streams, and autograd.  Every step of the method runs
in libspcoarsen.so; this module only marshals tensors to the C ABI and copies retained results
into tensors.
"""
from __future__ import annotations

import ctypes
import dataclasses
from typing import List, Optional

import numpy as np
import torch

from . import native as N

_DT = {torch.int32: N.SPC_I32, torch.float32: N.SPC_F32, torch.float64: N.SPC_F64}
_TD = {N.SPC_I32: torch.int32, N.SPC_F32: torch.float32, N.SPC_F64: torch.float64}


@dataclasses.dataclass
class CSR:
    """Symmetric CSR on one device (cuda for the normal path, cpu for the host-buffer path)."""
    rowptr: torch.Tensor  # int64[n+1]
    col: torch.Tensor     # int32[nnz]
    w: torch.Tensor       # int32 / float32 / float64 [nnz]

    @property
    def n(self) -> int:
        return int(self.rowptr.shape[0] - 1)

    @property
    def nnz(self) -> int:
        return int(self.col.shape[0])

    @staticmethod
    def from_numpy(rowptr, col, w, device="cuda", pin=False) -> "CSR":
        def conv(a):
            t = torch.from_numpy(np.ascontiguousarray(a))
            if device == "cpu":
                return t.pin_memory() if pin else t
            return t.to(device)
        return CSR(conv(rowptr), conv(col), conv(w))

    @staticmethod
    def from_graph(g, device="cuda", pin=False) -> "CSR":
        return CSR.from_numpy(g.rowptr, g.col, g.w, device=device, pin=pin)


@dataclasses.dataclass
class Level:
    """One level's results, copied out of the context into tensors."""
    n: int
    m: int
    n_c: int
    m_c: int
    m_inter: int
    status: int
    ms: float
    score: torch.Tensor
    lift: torch.Tensor
    emap: torch.Tensor
    self_mass: torch.Tensor
    a_und: torch.Tensor
    rowptr_c: torch.Tensor
    col_c: torch.Tensor
    w_c: torch.Tensor
    perm: torch.Tensor
    seg: torch.Tensor
    graph_ptr_c: Optional[torch.Tensor] = None
    # accumulated internal weight of every super-node (the self-mass reading), else None
    mass: Optional[torch.Tensor] = None

    def coarse_csr(self) -> CSR:
        return CSR(self.rowptr_c, self.col_c, self.w_c)


def _ptr(t: Optional[torch.Tensor]):
    if t is None:
        return None
    if not t.is_contiguous():
        raise ValueError("tensors passed to the C ABI must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


class Context:
    """An spc_context bound to one CUDA device and stream."""

    def __init__(self, device=None, stream: Optional[torch.cuda.Stream] = None,
                 torch_allocator: bool = True, alloc_hook=None):
        """alloc_hook (optional, with torch_allocator): called with the byte count before every
        workspace allocation; returning False makes that allocation fail (the library then
        returns SPC_ERR_OOM), which lets a caller exercise the out-of-memory path."""
        if not torch.cuda.is_available():
            raise RuntimeError("the coarsener needs a CUDA device (there is no CPU path)")
        self.lib = N.lib()
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None
                                   else torch.device(device).index or 0)
        with torch.cuda.device(self.device):
            self.stream = stream or torch.cuda.current_stream(self.device)
            self._handle = ctypes.c_void_p()
            self._alloc_struct = None
            if torch_allocator:
                dev = self.device.index
                st = self.stream

                def _alloc(_ctx, nbytes):
                    if alloc_hook is not None and not alloc_hook(int(nbytes)):
                        return None
                    try:
                        return torch.cuda.caching_allocator_alloc(int(nbytes), dev, st)
                    except Exception:  # out of memory -> NULL -> SPC_ERR_OOM
                        return None

                def _free(_ctx, p):
                    torch.cuda.caching_allocator_delete(p)

                self._cb = (N.ALLOC_FN(_alloc), N.FREE_FN(_free))
                self._alloc_struct = N.spc_allocator(self._cb[0], self._cb[1], None)
            N.check(self.lib.spc_context_create(
                ctypes.byref(self._handle),
                ctypes.byref(self._alloc_struct) if self._alloc_struct is not None else None,
                ctypes.c_void_p(self.stream.cuda_stream)), "spc_context_create")

    # ---- lifetime -------------------------------------------------------------------------
    def close(self):
        if getattr(self, "_handle", None) is not None and self._handle.value:
            with torch.cuda.device(self.device):
                self.lib.spc_context_destroy(self._handle)
            self._handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_wait_limit(self, iterations: int):
        """Bound every device-side wait of later calls (0: the default); a wait that reaches
        the bound makes the call raise SpcError(SPC_ERR_TIMEOUT)."""
        N.check(self.lib.spc_context_set_wait_limit(self._handle, int(iterations)),
                "spc_context_set_wait_limit")

    # ---- helpers --------------------------------------------------------------------------
    def _csr(self, g: CSR) -> N.spc_csr:
        if g.rowptr.dtype != torch.int64 or g.col.dtype != torch.int32:
            raise TypeError("rowptr must be int64 and col int32")
        if g.w.dtype not in _DT:
            raise TypeError(f"unsupported weight dtype {g.w.dtype}")
        return N.spc_csr(g.n, g.nnz, _ptr(g.rowptr), _ptr(g.col), _ptr(g.w), _DT[g.w.dtype])

    def _copy_from(self, ptr, count: int, dtype, device=None) -> torch.Tensor:
        t = torch.empty(max(count, 0), dtype=dtype, device=device or self.device)
        if count > 0:
            nbytes = count * t.element_size()
            N.check(self.lib.spc_copy(self._handle, _ptr(t), ctypes.c_void_p(ptr), nbytes),
                    "spc_copy")
        return t

    @staticmethod
    def _score_dtype(w: torch.Tensor):
        return torch.float32 if w.dtype == torch.float32 else torch.float64

    # ---- single steps -----------------------------------------------------------------------
    def score(self, g: CSR) -> torch.Tensor:
        """S0-S3: the score of every undirected edge in eid order."""
        c = self._csr(g)
        out = torch.empty(g.nnz // 2, dtype=self._score_dtype(g.w), device=g.col.device)
        m = ctypes.c_int64(0)
        N.check(self.lib.spc_score(self._handle, ctypes.byref(c), _ptr(out), ctypes.byref(m)),
                "spc_score")
        return out

    def sort_fitness(self, f: torch.Tensor) -> torch.Tensor:
        """S4: edge ids sorted by (f, eid)."""
        order = torch.empty(f.shape[0], dtype=torch.int32, device=f.device)
        dt = N.SPC_F32 if f.dtype == torch.float32 else N.SPC_F64
        N.check(self.lib.spc_sort_fitness(self._handle, f.shape[0], _ptr(f), dt, _ptr(order)),
                "spc_sort_fitness")
        return order

    def select_merges(self, g: CSR, f: torch.Tensor, n_c: int):
        """S5-S6: the merge partition for scores f; returns (lift, merged, n_c, status)."""
        c = self._csr(g)
        lift = torch.empty(g.n, dtype=torch.int32, device=g.col.device)
        merged = torch.empty(g.nnz // 2, dtype=torch.uint8, device=g.col.device)
        nca = ctypes.c_int64(0)
        st = N.check(self.lib.spc_select_merges(self._handle, ctypes.byref(c), _ptr(f), int(n_c),
                                                _ptr(lift), _ptr(merged), ctypes.byref(nca)),
                     "spc_select_merges")
        return lift, merged, int(nca.value), st

    def contract(self, g: CSR, lift: torch.Tensor, n_c: int) -> Level:
        """S7: contraction by a given lift; returns the level's results."""
        c = self._csr(g)
        mc = ctypes.c_int64(0)
        N.check(self.lib.spc_contract(self._handle, ctypes.byref(c), _ptr(lift), int(n_c),
                                      ctypes.byref(mc)), "spc_contract")
        return self.level(0)

    # ---- the method ----------------------------------------------------------------------
    def coarsen(self, g: CSR, n_c: int, levels: int = 1, validate: bool = True,
                schedule: int = 0, lift_out: Optional[torch.Tensor] = None,
                use_graph: bool = True, self_mass: bool = True, reorder: bool = False):
        """Coarsen to n_c super-nodes in `levels` levels; returns (lift, n_c_actual, status).
        With use_graph, a call that repeats the previous one on unchanged input replays the
        recorded schedule as one CUDA graph.  self_mass selects the multilevel reading: every
        level after the first scores its input with each super-node's accumulated internal
        weight on the diagonal (the merged node of the proof of Theorem 2); False scores the
        coarse graph without it.  reorder first renumbers the graph by (8-hop min label,
        2-hop min label, id) (see reorder_perm); the lift stays in the caller's numbering."""
        c = self._csr(g)
        opts = N.spc_options(int(levels), int(bool(validate)), int(bool(use_graph)), int(schedule),
                             int(bool(self_mass)), int(bool(reorder)))
        lift = lift_out if lift_out is not None else torch.empty(g.n, dtype=torch.int32,
                                                                 device=g.col.device)
        nca = ctypes.c_int64(0)
        st = N.check(self.lib.spc_coarsen(self._handle, ctypes.byref(c), int(n_c),
                                          ctypes.byref(opts), _ptr(lift), ctypes.byref(nca)),
                     "spc_coarsen")
        return lift, int(nca.value), st

    def coarsen_batched(self, g: CSR, graph_ptr: torch.Tensor, ratio: int, levels: int,
                        validate: bool = True, schedule: int = 0, use_graph: bool = True,
                        self_mass: bool = True):
        """Coarsen every graph of a block-diagonal batch to floor(n_b / ratio) super-nodes
        (self_mass as in coarsen)."""
        c = self._csr(g)
        B = int(graph_ptr.shape[0] - 1)
        opts = N.spc_options(int(levels), int(bool(validate)), int(bool(use_graph)), int(schedule),
                             int(bool(self_mass)), 0)
        lift = torch.empty(g.n, dtype=torch.int32, device=g.col.device)
        gpc = torch.empty(B + 1, dtype=torch.int64, device=g.col.device)
        st = N.check(self.lib.spc_coarsen_batched(self._handle, ctypes.byref(c), _ptr(graph_ptr),
                                                  B, int(ratio), ctypes.byref(opts), _ptr(lift),
                                                  _ptr(gpc)), "spc_coarsen_batched")
        return lift, gpc, st

    def reorder_perm(self, n: int) -> torch.Tensor:
        """perm[x] = the id of node x in the renumbered graph of the last coarsening made with
        reorder=True."""
        out = torch.empty(n, dtype=torch.int32, device=self.device)
        N.check(self.lib.spc_get_reorder(self._handle, _ptr(out)), "spc_get_reorder")
        return out

    def take_result(self) -> "Result":
        """The last coarsening's result in buffers the caller owns (they outlive later calls
        on this context); see Result."""
        r = N.spc_result()
        N.check(self.lib.spc_take_result(self._handle, ctypes.byref(r)), "spc_take_result")
        return Result(self, r)

    # ---- retained results ------------------------------------------------------------------
    def level_count(self) -> int:
        return int(self.lib.spc_level_count(self._handle))

    def level_info(self, l: int) -> N.spc_level:
        info = N.spc_level()
        N.check(self.lib.spc_get_level(self._handle, l, ctypes.byref(info)), "spc_get_level")
        return info

    def level(self, l: int, batched_B: Optional[int] = None) -> Level:
        i = self.level_info(l)
        wt = _TD[i.wtype]
        st = _TD[i.scoretype]
        acc = torch.int64 if i.wtype == N.SPC_I32 else wt
        cp = self._copy_from
        return Level(
            n=i.n, m=i.m, n_c=i.n_c, m_c=i.m_c, m_inter=i.m_inter, status=i.status, ms=i.ms,
            score=cp(i.score, i.m, st), lift=cp(i.lift, i.n, torch.int32),
            emap=cp(i.emap, i.m, torch.int32), self_mass=cp(i.self_mass, i.n_c, acc),
            a_und=cp(i.a_und, i.m_c, wt), rowptr_c=cp(i.rowptr_c, i.n_c + 1, torch.int64),
            col_c=cp(i.col_c, 2 * i.m_c, torch.int32), w_c=cp(i.w_c, 2 * i.m_c, wt),
            perm=cp(i.perm, i.m_inter, torch.int32), seg=cp(i.seg, i.m_c + 1, torch.int32),
            graph_ptr_c=(cp(i.graph_ptr_c, batched_B + 1, torch.int64)
                         if batched_B is not None else None),
            mass=cp(i.mass, i.n_c, acc) if i.mass else None)

    def levels(self, batched_B: Optional[int] = None) -> List[Level]:
        return [self.level(l, batched_B) for l in range(self.level_count())]

    def compose_emap(self) -> torch.Tensor:
        m = self.level_info(0).m
        out = torch.empty(m, dtype=torch.int32, device=self.device)
        N.check(self.lib.spc_compose_emap(self._handle, _ptr(out)), "spc_compose_emap")
        return out

    # ---- differentiable contraction ------------------------------------------------------------
    def contract_forward(self, perm, seg, m_c: int, w_und: torch.Tensor) -> torch.Tensor:
        out = torch.empty(m_c, dtype=w_und.dtype, device=w_und.device)
        N.check(self.lib.spc_contract_forward(self._handle, _ptr(perm), _ptr(seg), int(m_c),
                                              _ptr(w_und), _DT[w_und.dtype], _ptr(out)),
                "spc_contract_forward")
        return out

    def contract_backward(self, emap: torch.Tensor, grad_a: torch.Tensor) -> torch.Tensor:
        out = torch.empty(emap.shape[0], dtype=grad_a.dtype, device=grad_a.device)
        N.check(self.lib.spc_contract_backward(self._handle, _ptr(emap), emap.shape[0],
                                               _ptr(grad_a), _ptr(out), _DT[grad_a.dtype]),
                "spc_contract_backward")
        return out

    def pool_features(self, lift: torch.Tensor, n_c: int, x: torch.Tensor) -> torch.Tensor:
        """Mean of every super-node's member features (x: n-by-F, float32 or float64)."""
        x = x.contiguous()
        lift = lift.to(torch.int32).contiguous()
        F = x.shape[1]
        out = torch.empty((n_c, F), dtype=x.dtype, device=x.device)
        N.check(self.lib.spc_pool_features(self._handle, lift.shape[0], _ptr(lift), n_c, F,
                                           _DT[x.dtype], _ptr(x), _ptr(out)),
                "spc_pool_features")
        return out

    def pool_features_backward(self, lift: torch.Tensor, n_c: int,
                               grad_xc: torch.Tensor) -> torch.Tensor:
        grad_xc = grad_xc.contiguous()
        lift = lift.to(torch.int32).contiguous()
        F = grad_xc.shape[1]
        out = torch.empty((lift.shape[0], F), dtype=grad_xc.dtype, device=grad_xc.device)
        N.check(self.lib.spc_pool_features_backward(self._handle, lift.shape[0], _ptr(lift), n_c,
                                                    F, _DT[grad_xc.dtype], _ptr(grad_xc),
                                                    _ptr(out)),
                "spc_pool_features_backward")
        return out

    # ---- timing / accounting --------------------------------------------------------------------
    def time_kernel(self, substr: Optional[str]):
        N.check(self.lib.spc_time_kernel(self._handle, substr.encode() if substr else None),
                "spc_time_kernel")

    def kernel_time(self):
        n = ctypes.c_int64(0)
        ms = ctypes.c_double(0.0)
        N.check(self.lib.spc_kernel_time(self._handle, ctypes.byref(n), ctypes.byref(ms)),
                "spc_kernel_time")
        return int(n.value), float(ms.value)

    def kernel_profile(self):
        """{kernel name: (launches, total ms, algorithmic bytes, fp ops)} for the launches
        timed since time_kernel(); bytes are the summed per-launch algorithmic DRAM bytes of
        the launches that carry a byte model (0 for the others), fp ops the score kernels'
        required additions and subtractions (0 for the others)."""
        buf = ctypes.create_string_buffer(1 << 16)
        N.check(self.lib.spc_kernel_profile(self._handle, buf, len(buf)), "spc_kernel_profile")
        out = {}
        for line in buf.value.decode().splitlines():
            name, cnt, ms, nbytes, ops = line.split("\t")
            out[name] = (int(cnt), float(ms), float(nbytes), float(ops))
        return out

    @property
    def launch_count(self) -> int:
        return int(self.lib.spc_launch_count(self._handle))

    @property
    def last_call_replayed(self) -> bool:
        """Whether the last coarsening call replayed the previous identical call's graph."""
        return bool(self.lib.spc_last_call_replayed(self._handle))


class Result:
    """A coarsening result owned by the caller (spc_take_result): the lift, the composed edge
    map, the coarse graph and the carried mass, in device buffers that stay valid until free()
    (or garbage collection) whatever the context computes meanwhile."""

    def __init__(self, context: Context, r):
        self.context, self._r = context, r
        self.n, self.m, self.n_c, self.m_c = int(r.n), int(r.m), int(r.n_c), int(r.m_c)
        self.wtype = _TD[r.wtype]

    def tensors(self) -> dict:
        """Copies of every buffer as tensors on the context's device."""
        r, cp = self._r, self.context._copy_from
        acc = torch.int64 if self.wtype == torch.int32 else self.wtype
        out = {"lift": cp(r.lift, self.n, torch.int32), "emap": cp(r.emap, self.m, torch.int32),
               "rowptr_c": cp(r.rowptr_c, self.n_c + 1, torch.int64),
               "col_c": cp(r.col_c, 2 * self.m_c, torch.int32),
               "w_c": cp(r.w_c, 2 * self.m_c, self.wtype)}
        out["mass"] = cp(r.mass, self.n_c, acc) if r.mass else None
        return out

    def free(self):
        if self._r is not None and getattr(self.context, "_handle", None) is not None \
                and self.context._handle.value:
            self.context.lib.spc_result_free(self.context._handle, ctypes.byref(self._r))
        self._r = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


@dataclasses.dataclass
class ContractionPlan:
    """The assignment of a (multilevel) coarsening, held fixed for differentiation."""
    context: Context
    perms: List[torch.Tensor]
    segs: List[torch.Tensor]
    emaps: List[torch.Tensor]
    m_cs: List[int]

    @staticmethod
    def from_levels(ctx: Context, levels: List[Level]) -> "ContractionPlan":
        return ContractionPlan(ctx, [lv.perm for lv in levels], [lv.seg for lv in levels],
                               [lv.emap for lv in levels], [lv.m_c for lv in levels])


class ContractWeights(torch.autograd.Function):
    """a = S_L ... S_1 w: fine undirected edge weights -> coarse undirected edge weights
    (Definition 1, level by level, sums in ascending fine edge id).  Backward gathers every
    coarse gradient back to its fine edges, 0 for edges inside a super-node (the assignment
    is held fixed)."""

    @staticmethod
    def forward(ctx, w_und: torch.Tensor, plan: ContractionPlan):
        a = w_und.contiguous()
        for perm, seg, m_c in zip(plan.perms, plan.segs, plan.m_cs):
            a = plan.context.contract_forward(perm, seg, m_c, a)
        ctx.plan = plan
        return a

    @staticmethod
    def backward(ctx, grad_a: torch.Tensor):
        plan = ctx.plan
        g = grad_a.contiguous()
        for emap in reversed(plan.emaps):
            g = plan.context.contract_backward(emap, g)
        return g, None


def contract_weights(w_und: torch.Tensor, plan: ContractionPlan) -> torch.Tensor:
    return ContractWeights.apply(w_und, plan)


class PoolFeatures(torch.autograd.Function):
    """xc = mean of each super-node's member features (the node counterpart of Definition 2's
    averaging over super-node sizes); backward divides every coarse gradient by the member
    count and hands it to the members (the lift is held fixed)."""

    @staticmethod
    def forward(ctx, x: torch.Tensor, lift: torch.Tensor, n_c: int, context: Context):
        ctx.lift, ctx.n_c, ctx.context = lift, n_c, context
        return context.pool_features(lift, n_c, x)

    @staticmethod
    def backward(ctx, grad_xc: torch.Tensor):
        return ctx.context.pool_features_backward(ctx.lift, ctx.n_c, grad_xc), None, None, None


def pool_features(x: torch.Tensor, lift: torch.Tensor, n_c: int, context: Context) -> torch.Tensor:
    return PoolFeatures.apply(x, lift, n_c, context)
