"""Full-size workloads in the configuration bench.py times, against the CPU oracle (needs a GPU).

* 2048x2048 FP64 mesh, 6 halving levels, and the 129^3 tetrahedral mesh, 7 levels: every level
  bit-exact with the oracle (the oracle runs each in about a minute).
* 2^23-point random geometric graph, 8 levels: level 0 bit-exact with the oracle's level to
  n/2; the deeper levels checked through properties that hold at any size.
* 10,000-mesh batch, 3 levels: the whole batch on the GPU, 40 sampled graphs through the oracle
  (graphs of a batch are independent, so each sampled graph's result is exactly checkable).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O
from paper_2204_11757_gb300 import inputs as I

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


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
    return a.view(np.uint64) if a.dtype.itemsize == 8 else a.view(np.uint32)


def _same_level(lv, ref):
    co = ref.coarse
    assert lv.n_c == ref.n_c and lv.m_c == co.m_c
    assert np.array_equal(_bits(lv.score.cpu().numpy()), _bits(ref.f))
    assert np.array_equal(lv.lift.cpu().numpy(), ref.lift)
    assert np.array_equal(lv.emap.cpu().numpy(), co.emap)
    assert np.array_equal(lv.rowptr_c.cpu().numpy(), co.graph.rowptr)
    assert np.array_equal(lv.col_c.cpu().numpy(), co.graph.col)
    assert np.array_equal(_bits(lv.w_c.cpu().numpy()), _bits(co.graph.w))
    assert np.array_equal(_bits(lv.self_mass.cpu().numpy()), _bits(co.self_mass))


@pytest.mark.parametrize("name", ["c2_tri2048_f64", "c3_tet129_f64"])
def test_mesh_multilevel_bitexact(ctx, name):
    from paper_2204_11757_gb300 import api
    g, cfg = I.config_graph(name)
    L = int(round(np.log2(cfg["ratio"])))
    lift, nc, st = ctx.coarsen(api.CSR.from_graph(g), g.n // cfg["ratio"], levels=L)
    got = ctx.levels()
    levels, total = O.coarsen(g, cfg["ratio"], cfg["mode"])
    assert nc == levels[-1].n_c
    assert np.array_equal(lift.cpu().numpy(), total)
    for lv, ref in zip(got, levels):
        _same_level(lv, ref)


def _valid_level(fine_n, fine_eu, fine_ev, fine_w, lv, target):
    lift = lv.lift.cpu().numpy()
    assert lv.n_c == target
    assert lift.min() == 0 and lift.max() == lv.n_c - 1
    # ids by smallest member: first occurrences appear in increasing order
    order = np.unique(lift, return_index=True)[1]
    assert np.all(np.diff(order) > 0)
    em = lv.emap.cpu().numpy()
    U, V = lift[fine_eu], lift[fine_ev]
    assert np.all((em >= 0) == (U != V))
    rp = lv.rowptr_c.cpu().numpy(); cc = lv.col_c.cpu().numpy(); wc = lv.w_c.cpu().numpy()
    rows = np.repeat(np.arange(lv.n_c), np.diff(rp))
    assert not np.any(cc == rows)
    # symmetric pattern with bit-identical mirrored weights
    key = rows.astype(np.int64) * lv.n_c + cc
    tkey = cc.astype(np.int64) * lv.n_c + rows
    o1, o2 = np.argsort(key), np.argsort(tkey)
    assert np.array_equal(key[o1], tkey[o2])
    assert np.array_equal(_bits(wc[o1]), _bits(wc[o2]))
    # every coarse weight and self-mass is a left-to-right binary32 sum of its fine weights:
    # within (len - 1) u sum|w| of the exact sum (u = 2^-24)
    u = 2.0 ** -24 if wc.dtype == np.float32 else 2.0 ** -53
    fw = fine_w.astype(np.float64)
    a = lv.a_und.cpu().numpy().astype(np.float64)
    sel = em >= 0
    exact = np.bincount(em[sel], weights=fw[sel], minlength=lv.m_c)
    cnt = np.bincount(em[sel], minlength=lv.m_c)
    assert np.all(np.abs(a - exact) <= np.maximum(cnt - 1, 0) * u * exact + 1e-300)
    sm = lv.self_mass.cpu().numpy().astype(np.float64)
    intra = ~sel
    exact_s = np.bincount(U[intra], weights=fw[intra], minlength=lv.n_c)
    cnt_s = np.bincount(U[intra], minlength=lv.n_c)
    assert np.all(np.abs(sm - exact_s) <= np.maximum(cnt_s - 1, 0) * u * exact_s + 1e-300)


def test_rgg_level0_bitexact_and_deep_levels_valid(ctx):
    from paper_2204_11757_gb300 import api
    g, cfg = I.config_graph("c4_rgg8m_f32")
    lift, nc, st = ctx.coarsen(api.CSR.from_graph(g), g.n // cfg["ratio"], levels=8)
    got = ctx.levels()
    ref0 = O.coarsen_level(g, g.n // 2)
    _same_level(got[0], ref0)
    targets = O.level_targets(g.n, cfg["ratio"], cfg["mode"])
    cur_eu, cur_ev, cur_w, cur_n = g.eu, g.ev, g.w_und, g.n
    for lv, t in zip(got, targets):
        _valid_level(cur_n, cur_eu, cur_ev, cur_w, lv, t)
        rp = lv.rowptr_c.cpu().numpy(); cc = lv.col_c.cpu().numpy()
        cur_eu, cur_ev, cur_w = I.upper_edges(rp, cc, lv.w_c.cpu().numpy())
        cur_n = lv.n_c


def test_batch10k_sampled_graphs(ctx):
    from paper_2204_11757_gb300 import api
    b, cfg = I.config_graph("c5_batch10k_f32")
    lift, gpc, st = ctx.coarsen_batched(api.CSR.from_graph(b.graph),
                                        torch.from_numpy(b.graph_ptr).cuda(), cfg["ratio"],
                                        levels=3)
    lift = lift.cpu().numpy(); gpc = gpc.cpu().numpy()
    last = ctx.level(2, batched_B=b.B)
    rp = last.rowptr_c.cpu().numpy(); cc = last.col_c.cpu().numpy(); wc = last.w_c.cpu().numpy()
    rng = np.random.default_rng(5)
    sample = np.sort(rng.choice(b.B, size=40, replace=False))
    sub = I.subsample_batch(b, sample)
    res = O.coarsen_batch(sub, cfg["ratio"], cfg["mode"])
    for k, bi in enumerate(sample):
        levels_ref, total_ref = res[k]
        n0, n1 = b.graph_ptr[bi], b.graph_ptr[bi + 1]
        assert gpc[bi + 1] - gpc[bi] == levels_ref[-1].n_c
        assert np.array_equal(lift[n0:n1] - gpc[bi], total_ref)
        cg = levels_ref[-1].coarse.graph
        s0, s1 = gpc[bi], gpc[bi + 1]
        assert np.array_equal(rp[s0:s1 + 1] - rp[s0], cg.rowptr)
        assert np.array_equal(cc[rp[s0]:rp[s1]] - s0, cg.col)
        assert np.array_equal(_bits(wc[rp[s0]:rp[s1]]), _bits(cg.w))
