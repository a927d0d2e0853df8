"""Full-size workloads in the configuration bench.py times, against the CPU oracle (needs a GPU).

Every configuration is compared with the oracle bit for bit, at every level:
* the 2048x2048 FP64 mesh (6 halving levels) and the 129^3 tetrahedral mesh (7 levels);
* the 2^23-point random geometric graph, 8 halving levels, one level straight to n/256, and 8
  levels under the adjacency-reordering option;
* the 10,000-mesh batch (3 levels): every graph of the batch against the oracle run on that
  graph alone (graphs of a batch are independent).
Scores, lifts, edge maps, coarse CSRs, coarse weights, self-mass and the carried mass of the
self-mass reading are compared as bit patterns.

The oracle's runs start with the module in spawned worker processes (they take minutes on the
largest graph) and the GPU runs in this process meanwhile.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2204_11757_gb300 import inputs as I

import oracle_workers as W

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

SINGLE = ["c2_tri2048_f64", "c3_tet129_f64", "c4_rgg8m_f32"]


@pytest.fixture(scope="module")
def oracle_runs():
    """Futures of every oracle run of this module: the longest first, then the batch chunks."""
    from oracle import oracle as O
    O.build()  # compiled once here, not by every worker at the same time
    pool = W.pool()
    fut = {"c4_rgg8m_f32": pool.submit(W.coarsen_config, "c4_rgg8m_f32"),
           "c4_reordered": pool.submit(W.coarsen_config_reordered, "c4_rgg8m_f32"),
           "c4_one": pool.submit(W.coarsen_config, "c4_rgg8m_f32", True),
           "c3_tet129_f64": pool.submit(W.coarsen_config, "c3_tet129_f64"),
           "c2_tri2048_f64": pool.submit(W.coarsen_config, "c2_tri2048_f64")}
    batch, bcfg = I.config_graph("c5_batch10k_f32")
    parts = W.chunks(batch.B, 40)
    fut["c5"] = [(idx, pool.submit(W.batch_chunk, I.subsample_batch(batch, idx), bcfg["ratio"],
                                   bcfg["mode"])) for idx in parts]
    yield fut, (batch, bcfg)
    pool.shutdown(wait=False, cancel_futures=True)


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__ as ge
    ge.build()
    from paper_2204_11757_gb300 import api
    c = api.Context()
    yield c
    c.close()


def _bits(a):
    a = np.ascontiguousarray(a)
    if a.dtype.kind != "f":
        return a
    return a.view(np.uint64) if a.dtype.itemsize == 8 else a.view(np.uint32)


def _same(got, want):
    got = got.cpu().numpy() if hasattr(got, "cpu") else got
    assert got.dtype == want.dtype and got.shape == want.shape
    assert np.array_equal(_bits(got), _bits(want))


def _same_level(lv, ref):
    co = ref.coarse
    assert lv.n_c == ref.n_c and lv.m_c == co.m_c
    _same(lv.score, ref.f)
    _same(lv.lift, ref.lift)
    _same(lv.emap, co.emap)
    _same(lv.rowptr_c, co.graph.rowptr)
    _same(lv.col_c, co.graph.col)
    _same(lv.w_c, co.graph.w)
    _same(lv.a_und, co.a_und)
    _same(lv.self_mass, co.self_mass)
    if getattr(ref, "mass", None) is not None:
        _same(lv.mass, ref.mass)


@pytest.mark.parametrize("name", SINGLE)
def test_multilevel_bitexact(ctx, oracle_runs, name):
    from paper_2204_11757_gb300 import api
    g, cfg = I.config_graph(name)
    L = int(round(np.log2(cfg["ratio"])))
    lift, nc, st = ctx.coarsen(api.CSR.from_graph(g), g.n // cfg["ratio"], levels=L)
    got = ctx.levels()
    del g
    levels, total = oracle_runs[0][name].result()
    assert len(got) == len(levels) == L
    assert nc == levels[-1].n_c
    _same(lift, total)
    for lv, ref in zip(got, levels):
        _same_level(lv, ref)


def test_rgg_one_level_bitexact(ctx, oracle_runs):
    """One pass of Algorithm 1 straight to n/256: most merges chain into one super-node whose
    self-mass is a left-to-right binary32 sum of tens of millions of terms."""
    from paper_2204_11757_gb300 import api
    g, cfg = I.config_graph("c4_rgg8m_f32_one")
    lift, nc, st = ctx.coarsen(api.CSR.from_graph(g), g.n // cfg["ratio"], levels=1)
    got = ctx.levels()
    del g
    levels, total = oracle_runs[0]["c4_one"].result()
    assert nc == levels[0].n_c
    _same(lift, total)
    _same_level(got[0], levels[0])


def test_rgg_reordered_bitexact(ctx, oracle_runs):
    """The adjacency-reordering option on the 2^23-point RGG, 8 levels: the renumbering, the
    composed lift in the caller's numbering and every level of the renumbered graph."""
    from paper_2204_11757_gb300 import api
    g, cfg = I.config_graph("c4_rgg8m_f32")
    L = int(round(np.log2(cfg["ratio"])))
    lift, nc, st = ctx.coarsen(api.CSR.from_graph(g), g.n // cfg["ratio"], levels=L,
                               reorder=True)
    perm = ctx.reorder_perm(g.n)
    got = ctx.levels()
    del g
    levels, total, perm_ref = oracle_runs[0]["c4_reordered"].result()
    _same(perm, perm_ref)
    assert len(got) == len(levels) == L
    assert nc == levels[-1].n_c
    _same(lift, total)
    for lv, ref in zip(got, levels):
        _same_level(lv, ref)


def test_batch10k_every_graph(ctx, oracle_runs):
    from paper_2204_11757_gb300 import api
    fut, (b, cfg) = oracle_runs
    lift, gpc, st = ctx.coarsen_batched(api.CSR.from_graph(b.graph),
                                        torch.from_numpy(b.graph_ptr).cuda(), cfg["ratio"],
                                        levels=3)
    lift = lift.cpu().numpy(); gpc = gpc.cpu().numpy()
    last = ctx.level(2, batched_B=b.B)
    rp = last.rowptr_c.cpu().numpy(); cc = last.col_c.cpu().numpy(); wc = last.w_c.cpu().numpy()
    mass = last.mass.cpu().numpy()
    checked = 0
    for idx, f in fut["c5"]:
        for bi, (total, n_c, crp, ccol, cw, cmass) in zip(idx, f.result()):
            n0, n1 = b.graph_ptr[bi], b.graph_ptr[bi + 1]
            s0, s1 = gpc[bi], gpc[bi + 1]
            assert s1 - s0 == n_c
            assert np.array_equal(lift[n0:n1] - s0, total)
            assert np.array_equal(rp[s0:s1 + 1] - rp[s0], crp)
            assert np.array_equal(cc[rp[s0]:rp[s1]] - s0, ccol)
            assert np.array_equal(_bits(wc[rp[s0]:rp[s1]]), _bits(cw))
            assert np.array_equal(_bits(mass[s0:s1]), _bits(cmass))
            checked += 1
    assert checked == b.B
