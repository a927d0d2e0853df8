"""GPU path vs the CPU oracle, element by element, through the C ABI (needs a GB300).

Integer, index and topology results must be bit-exact; scores are compared as bit patterns
(the paper's order of operations is fixed, see the oracle); coarse weights are compared bit
for bit too, because both sides sum in ascending fine edge id.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O
from paper_2204_11757_gb300 import inputs as I

import golden_io

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__ as ge
    ge.build()
    from paper_2204_11757_gb300 import api
    c = api.Context()
    yield c
    c.close()


def _api():
    from paper_2204_11757_gb300 import api
    return api


def _bits(a):
    a = np.ascontiguousarray(a)
    return a.view(np.uint64) if a.dtype.itemsize == 8 else a.view(np.uint32)


def _small_graphs():
    gs = [I.path_graph(2), I.path_graph(7), I.cycle_graph(9), I.complete_graph(6)]
    for seed in range(6):
        wt = ["unit", "int", "float"][seed % 3]
        dt = np.float64 if wt == "float" else np.int32
        gs.append(I.random_graph(40 + 10 * seed, 0.1, seed, weight=wt, dtype=dt,
                                 connected=seed % 2 == 0))
    gs.append(I.random_graph(50, 0.2, 99, weight="float", dtype=np.float32, connected=True))
    rows, _ = I.config_graph("c1_tri64_unit")
    gs.append(rows)
    return gs


SMALL = _small_graphs()
MID = ["s2_tri256_f64", "s3_tet33_f64", "s4_rgg64k_f32"]


def _graph(name):
    g, _ = I.config_graph(name)
    return g


# ---- S0-S3 -------------------------------------------------------------------------------------

@pytest.mark.parametrize("gi", range(len(SMALL)))
@pytest.mark.parametrize("schedule", [1, 2, 3])
def test_score_small_bitexact(ctx, gi, schedule):
    g = SMALL[gi]
    api = _api()
    ref = O.score(g)
    csr = api.CSR.from_graph(g)
    if schedule == 1:
        f = ctx.score(csr).cpu().numpy()
    else:
        ctx.coarsen(csr, g.n, levels=1, schedule=schedule)
        f = ctx.level(0).score.cpu().numpy()
    assert f.dtype == ref.dtype
    assert np.array_equal(_bits(f), _bits(ref))


@pytest.mark.parametrize("name", MID)
@pytest.mark.parametrize("schedule", [1, 3])
def test_score_mid_bitexact(ctx, name, schedule):
    g = _graph(name)
    api = _api()
    ref = O.score(g)
    csr = api.CSR.from_graph(g)
    if schedule == 1:
        f = ctx.score(csr).cpu().numpy()
    else:
        ctx.coarsen(csr, g.n, levels=1, schedule=schedule)
        f = ctx.level(0).score.cpu().numpy()
    assert np.array_equal(_bits(f), _bits(ref))


@pytest.mark.parametrize("weight,dt", [("float", np.float32), ("float", np.float64),
                                       ("int", np.int32)])
def test_staged_schedule_on_mixed_row_lengths(ctx, weight, dt):
    """The staged schedule with every kind of row -- binary64 and int: rows b of up to 32
    entries staged, longer ones (up to 256) walked in place; binary32 (packed (column, p)
    pairs): rows b staged while the warp's area has room, the rest walked in place -- tiles
    whose rows a exceed the stage walked in place, and hub rows left to the hub kernels, on a
    heavy-tailed graph, then on its multilevel coarsening, every score bit-exact with the
    oracle."""
    api = _api()
    g = I.powerlaw_graph(4039, 22, 7, weight, dt)
    deg = np.diff(g.rowptr)
    assert deg.max() > 256 and np.any((deg > 32) & (deg <= 256)) and np.any(deg <= 32)
    csr = api.CSR.from_graph(g)
    ctx.coarsen(csr, g.n, levels=1, schedule=3)
    assert np.array_equal(_bits(ctx.level(0).score.cpu().numpy()), _bits(O.score(g)))
    levels_ref, total_ref = O.coarsen(g, 8, "halving")
    lift, nca, st = ctx.coarsen(csr, levels_ref[-1].target, levels=len(levels_ref), schedule=3)
    assert np.array_equal(lift.cpu().numpy(), total_ref)
    for lv, ref in zip(ctx.levels(), levels_ref):
        assert np.array_equal(_bits(lv.score.cpu().numpy()), _bits(ref.f))


# ---- S4 ------------------------------------------------------------------------------------------

@pytest.mark.parametrize("name", ["c1_tri64_unit", "s2_tri256_f64", "s4_rgg64k_f32"])
def test_sort_fitness(ctx, name):
    g = _graph(name)
    f = O.score(g)
    ref = O.sort_fitness(f)
    order = ctx.sort_fitness(torch.from_numpy(f).cuda()).cpu().numpy()
    assert np.array_equal(order, ref)


def test_sort_fitness_ties_and_ragged(ctx):
    rng = np.random.default_rng(3)
    for m in (1, 2, 4095, 4096, 4097, 20000):
        f = rng.integers(0, 7, size=m).astype(np.float64) / 4.0  # many exact ties
        ref = O.sort_fitness(f)
        assert np.array_equal(ctx.sort_fitness(torch.from_numpy(f).cuda()).cpu().numpy(), ref)
        f32 = f.astype(np.float32)
        ref32 = O.sort_fitness(f32)
        assert np.array_equal(ctx.sort_fitness(torch.from_numpy(f32).cuda()).cpu().numpy(), ref32)


# ---- S5-S6 ---------------------------------------------------------------------------------------

def _ref_select(g, n_c):
    f = O.score(g)
    order = O.sort_fitness(f)
    rep, merged, s, rc = O.greedy_merge(g, order, n_c)
    lift, nc = O.relabel(rep)
    return f, lift, merged, nc, rc


@pytest.mark.parametrize("gi", range(len(SMALL)))
def test_select_small(ctx, gi):
    g = SMALL[gi]
    api = _api()
    csr = api.CSR.from_graph(g)
    for n_c in sorted({1, 2, max(1, g.n // 3), max(1, g.n // 2), g.n - 1 if g.n > 1 else 1,
                       g.n, g.n + 5}):
        f, lift_ref, merged_ref, nc_ref, rc = _ref_select(g, n_c)
        lift, merged, nc, st = ctx.select_merges(csr, torch.from_numpy(f).cuda(), n_c)
        assert nc == nc_ref
        assert np.array_equal(lift.cpu().numpy(), lift_ref)
        assert np.array_equal(merged.cpu().numpy().astype(bool), merged_ref)
        assert st == rc


@pytest.mark.parametrize("name", MID)
def test_select_mid(ctx, name):
    g = _graph(name)
    api = _api()
    f, lift_ref, merged_ref, nc_ref, rc = _ref_select(g, g.n // 2)
    lift, merged, nc, st = ctx.select_merges(api.CSR.from_graph(g), torch.from_numpy(f).cuda(),
                                             g.n // 2)
    assert nc == nc_ref and st == rc
    assert np.array_equal(lift.cpu().numpy(), lift_ref)
    assert np.array_equal(merged.cpu().numpy().astype(bool), merged_ref)


def test_select_disconnected_and_isolated(ctx):
    api = _api()
    # three components plus two isolated nodes
    eu = np.array([0, 1, 3, 4, 5, 8]); ev = np.array([1, 2, 4, 5, 6, 9])
    g = I.csr_from_edges(12, eu, ev, np.ones(6, np.int32))
    csr = api.CSR.from_graph(g)
    for n_c in (1, 3, 5, 6, 7, 12):
        f, lift_ref, merged_ref, nc_ref, rc = _ref_select(g, n_c)
        lift, merged, nc, st = ctx.select_merges(csr, torch.from_numpy(f).cuda(), n_c)
        assert np.array_equal(lift.cpu().numpy(), lift_ref)
        assert nc == nc_ref and st == rc
    assert nc_ref == 12


# ---- S7 --------------------------------------------------------------------------------------------

def _check_level(lv, ref_level, exact_weights=True):
    co = ref_level.coarse
    assert lv.n_c == ref_level.n_c
    assert lv.m_c == co.m_c
    assert np.array_equal(lv.lift.cpu().numpy(), ref_level.lift)
    assert np.array_equal(lv.emap.cpu().numpy(), co.emap)
    assert np.array_equal(lv.rowptr_c.cpu().numpy(), co.graph.rowptr)
    assert np.array_equal(lv.col_c.cpu().numpy(), co.graph.col)
    for got, want in ((lv.w_c, co.graph.w), (lv.a_und, co.a_und), (lv.self_mass, co.self_mass)):
        got = got.cpu().numpy()
        assert got.dtype == want.dtype
        assert np.array_equal(_bits(got) if got.dtype.kind == "f" else got,
                              _bits(want) if want.dtype.kind == "f" else want)
    # the accumulated internal weight of the self-mass reading
    if getattr(ref_level, "mass", None) is not None:
        assert lv.mass is not None
        got, want = lv.mass.cpu().numpy(), ref_level.mass
        assert got.dtype == want.dtype
        assert np.array_equal(_bits(got) if got.dtype.kind == "f" else got,
                              _bits(want) if want.dtype.kind == "f" else want)
    # perm/seg describe each coarse edge's fine edges in ascending eid order
    perm = lv.perm.cpu().numpy(); seg = lv.seg.cpu().numpy()
    assert seg[0] == 0 and seg[-1] == lv.m_inter
    em = co.emap
    for k in np.linspace(0, max(lv.m_c - 1, 0), num=min(lv.m_c, 50)).astype(int):
        es = perm[seg[k]:seg[k + 1]]
        assert np.all(np.diff(es) > 0)
        assert np.all(em[es] == k)


@pytest.mark.parametrize("gi", range(len(SMALL)))
def test_contract_small(ctx, gi):
    g = SMALL[gi]
    api = _api()
    for n_c in sorted({1, max(1, g.n // 4), max(1, g.n // 2), g.n}):
        ref = O.coarsen_level(g, n_c)
        lv = ctx.contract(api.CSR.from_graph(g), torch.from_numpy(ref.lift).cuda(), ref.n_c)
        _check_level(lv, ref)


@pytest.mark.parametrize("name", golden_io.FILES)
def test_hand_examples_through_single_steps(ctx, name):
    """The hand-worked examples (tests/golden) through the ABI's single steps, against the values
    worked on paper rather than the oracle: score bits, each target's lift and contraction."""
    rows, ncs = golden_io.parse(name)
    n, eu, ev, w = golden_io.edges(rows)
    api = _api()
    csr = api.CSR.from_graph(I.csr_from_edges(n, eu, ev, w))
    f = ctx.score(csr)
    assert [int(x) for x in _bits(f.cpu().numpy())] == golden_io.ints(rows, "score_f64_bits")
    for nc, (lift, emap, sm, rp, cc, wc) in ncs.items():
        if nc >= n:
            continue
        got, _, nca, _ = ctx.select_merges(csr, f, nc)
        assert nca == nc
        assert got.cpu().numpy().tolist() == lift, nc
        lv = ctx.contract(csr, got, nc)
        assert lv.n_c == nc
        assert lv.emap.cpu().numpy().tolist() == emap, nc
        assert lv.self_mass.cpu().numpy().tolist() == sm, nc
        assert lv.rowptr_c.cpu().numpy().tolist() == rp, nc
        assert lv.col_c.cpu().numpy().tolist() == cc, nc
        assert lv.w_c.cpu().numpy().tolist() == wc, nc


def test_contract_int_overflow_reported(ctx):
    api = _api()
    from paper_2204_11757_gb300 import native as N
    g = I.csr_from_edges(3, np.array([0, 0]), np.array([1, 2]),
                         np.array([2 ** 31 - 1, 2 ** 31 - 1], dtype=np.int32))
    with pytest.raises(N.SpcError) as ei:
        ctx.contract(api.CSR.from_graph(g), torch.tensor([0, 1, 1], dtype=torch.int32).cuda(), 2)
    assert ei.value.status == -8


def _bucket_graph(k_clique, kb, n_cycle, dtype, seed):
    """A clique on k_clique nodes lifted to super-node 0 (one long self-mass sum), a complete
    bipartite K_{kb,kb} between super-nodes 1 and 2 (one coarse edge of kb^2 fine edges, all in
    bucket 1), and a cycle of n_cycle nodes lifted in pairs (many buckets of one item)."""
    rng = np.random.default_rng(seed)
    iu, iv = np.triu_indices(k_clique, 1)
    A = k_clique + np.arange(kb)
    B = k_clique + kb + np.arange(kb)
    C = k_clique + 2 * kb + np.arange(n_cycle)
    bu, bv = np.meshgrid(A, B, indexing="ij")
    eu = np.concatenate([iu, bu.ravel(), C, [0, A[0]]])
    ev = np.concatenate([iv, bv.ravel(), np.roll(C, -1), [A[0], C[0]]])
    n = k_clique + 2 * kb + n_cycle
    if np.dtype(dtype).kind == "f":
        w = rng.uniform(0.25, 4.0, eu.size).astype(dtype)
    else:
        w = rng.integers(1, 1000, eu.size).astype(dtype)
    g = I.csr_from_edges(n, eu, ev, w)
    lift = np.concatenate([np.zeros(k_clique), np.ones(kb), np.full(kb, 2),
                           3 + np.arange(n_cycle) // 2]).astype(np.int32)
    return g, lift, 3 + n_cycle // 2


@pytest.mark.parametrize("dt", [np.float64, np.float32, np.int32])
@pytest.mark.parametrize("kb,bucket_path", [(5, True), (17, True), (33, True), (91, False)])
def test_contract_bucket_and_radix_paths(ctx, dt, kb, bucket_path):
    """The contraction groups edges by buckets (ranked per item when short, sorted by one CTA
    when long) while no bucket exceeds 8192 items, by radix sorts otherwise (K_{91,91} puts 8281
    edges in one bucket).  Both give the oracle's coarse graph bit for bit, including segments
    longer than one thread's share (the clique's 300 intra edges, the bipartite coarse edge)."""
    api = _api()
    g, lift, n_c = _bucket_graph(25, kb, 4000, dt, kb)
    ref = O.contract(g, lift, n_c)
    ctx.time_kernel("*")
    try:
        lv = ctx.contract(api.CSR.from_graph(g), torch.from_numpy(lift).cuda(), n_c)
        prof = ctx.kernel_profile()
    finally:
        ctx.time_kernel(None)
    ranked = any("k_bucket_rank_inter" in k for k in prof)
    radix = any("k_classify" in k for k in prof)  # the radix path's compaction
    assert ranked == bucket_path and radix != bucket_path, sorted(prof)
    _check_level(lv, O.Level(n_c=n_c, lift=lift, coarse=ref))


@pytest.mark.parametrize("dt", [np.float64, np.int32])
def test_contract_many_giant_buckets(ctx, dt):
    """Nine disjoint K_{91,91} blocks, each a pair of super-nodes: nine buckets above 8192 items
    (the radix path), chained: the oracle's coarse graph bit for bit."""
    api = _api()
    rng = np.random.default_rng(11)
    kb, blocks = 91, 9
    eu, ev, lift = [], [], []
    for q in range(blocks):
        A = 2 * kb * q + np.arange(kb)
        B = A + kb
        bu, bv = np.meshgrid(A, B, indexing="ij")
        eu.append(bu.ravel())
        ev.append(bv.ravel())
        lift += [2 * q] * kb + [2 * q + 1] * kb
    eu.append(np.arange(0, 2 * kb * (blocks - 1), 2 * kb))  # chain the blocks
    ev.append(np.arange(2 * kb, 2 * kb * blocks, 2 * kb))
    eu = np.concatenate(eu)
    ev = np.concatenate(ev)
    n = 2 * kb * blocks
    w = (rng.uniform(0.5, 2.0, eu.size) if dt == np.float64
         else rng.integers(1, 100, eu.size)).astype(dt)
    g = I.csr_from_edges(n, eu, ev, w)
    lift = np.array(lift, dtype=np.int32)
    ref = O.contract(g, lift, 2 * blocks)
    ctx.time_kernel("*")
    try:
        lv = ctx.contract(api.CSR.from_graph(g), torch.from_numpy(lift).cuda(), 2 * blocks)
        prof = ctx.kernel_profile()
    finally:
        ctx.time_kernel(None)
    assert any("k_classify" in k for k in prof), sorted(prof)
    _check_level(lv, O.Level(n_c=2 * blocks, lift=lift, coarse=ref))


@pytest.mark.parametrize("dt", [np.float64, np.int32])
@pytest.mark.parametrize("center_last", [False, True])
def test_contract_star_rows_paths(ctx, dt, center_last):
    """A star of 2000 leaves, each node its own super-node after a relabelling.  With the
    centre numbered last, its coarse row has 2000 lower entries (ascending U'), which the
    lower-row buckets refuse (radix path); numbered first, its 2000 coarse edges share one
    inter bucket instead (sorted by one CTA) while every lower row holds one entry."""
    api = _api()
    rng = np.random.default_rng(7)
    leaves = 2000
    n = leaves + 1
    center = n - 1 if center_last else 0
    others = np.array([x for x in range(n) if x != center])
    w = (rng.uniform(0.5, 2.0, leaves) if dt == np.float64
         else rng.integers(1, 100, leaves)).astype(dt)
    # a few leaf-leaf chords so that coarse rows differ in length
    cu = others[:-1:7]
    cv = others[1::7][:cu.size]
    wc = np.ones(cu.size, dtype=dt)
    g = I.csr_from_edges(n, np.concatenate([np.full(leaves, center), cu]),
                         np.concatenate([others, cv]), np.concatenate([w, wc]))
    lift = np.empty(n, dtype=np.int32)
    lift[center] = n - 1 if center_last else 0
    lift[others] = rng.permutation(n - 1) + (0 if center_last else 1)
    ref = O.contract(g, lift, n)
    ctx.time_kernel("*")
    try:
        lv = ctx.contract(api.CSR.from_graph(g), torch.from_numpy(lift).cuda(), n)
        prof = ctx.kernel_profile()
    finally:
        ctx.time_kernel(None)
    lower_ranked = any("k_lower_scatter" in k for k in prof)
    long_sorted = any("k_bucket_sort_long" in k for k in prof)
    assert lower_ranked == (not center_last), sorted(prof)
    assert long_sorted == (not center_last), sorted(prof)
    assert any("k_bucket_rank_inter" in k for k in prof), sorted(prof)
    _check_level(lv, O.Level(n_c=n, lift=lift, coarse=ref))


@pytest.mark.parametrize("dt", [np.float64, np.float32])
def test_contract_long_lower_row_on_bucket_path(ctx, dt):
    """A star of 100 leaves beside a 100 x 100 grid, every node its own super-node with the
    star's centre numbered last: its coarse row has 100 lower entries, past one thread's share
    (32), while the grid's many short rows keep the lower rows on the bucket path; the long row
    is filled by a warp.  The coarse graph equals the oracle's."""
    api = _api()
    rng = np.random.default_rng(11)
    side, leaves = 100, 100
    ng = side * side
    n = ng + leaves + 1
    gu, gv = [], []
    for r in range(side):
        for c in range(side):
            x = r * side + c
            if c + 1 < side:
                gu.append(x); gv.append(x + 1)
            if r + 1 < side:
                gu.append(x); gv.append(x + side)
    center = n - 1
    su = np.full(leaves, center)
    sv = np.arange(ng, ng + leaves)
    eu = np.concatenate([np.array(gu), su]); ev = np.concatenate([np.array(gv), sv])
    w = rng.uniform(0.5, 2.0, eu.size).astype(dt)
    g = I.csr_from_edges(n, eu, ev, w)
    lift = np.empty(n, dtype=np.int32)
    lift[:n - 1] = rng.permutation(n - 1)
    lift[center] = n - 1
    ref = O.contract(g, lift, n)
    ctx.time_kernel("*")
    try:
        lv = ctx.contract(api.CSR.from_graph(g), torch.from_numpy(lift).cuda(), n)
        prof = ctx.kernel_profile()
    finally:
        ctx.time_kernel(None)
    assert any("k_fill_lower_rows" in k for k in prof), sorted(prof)
    assert any("k_fill_lower_long" in k for k in prof), sorted(prof)
    _check_level(lv, O.Level(n_c=n, lift=lift, coarse=ref))


def test_repeated_coarsening_replays_with_giant_super_nodes(ctx):
    """Three disjoint cliques K_150 (11,175 edges each) joined by two edges, coarsened to 3:
    three giant super-nodes.  Every value the host reads while coarsening must be the same on
    a repeated call (no order set by atomics), or the replay's check of its logged values
    fails and every call runs host-driven; the third call must be a replay."""
    api = _api()
    k, cl = 150, 3
    eu, ev = [], []
    for q in range(cl):
        iu, iv = np.triu_indices(k, 1)
        eu.append(iu + q * k)
        ev.append(iv + q * k)
    eu.append(np.arange(cl - 1) * k)
    ev.append(np.arange(1, cl) * k + 1)
    eu = np.concatenate(eu)
    ev = np.concatenate(ev)
    w = np.random.default_rng(3).uniform(0.5, 2.0, eu.size)
    g = I.csr_from_edges(k * cl, eu, ev, w)
    ref = O.coarsen_level(g, cl)
    csr = api.CSR.from_graph(g)
    for _ in range(3):
        lift, n_c, st = ctx.coarsen(csr, cl, levels=1)
    assert ctx.last_call_replayed
    assert n_c == ref.n_c
    _check_level(ctx.level(0), ref)


# ---- full method ------------------------------------------------------------------------------------

@pytest.mark.parametrize("name", ["c1_tri64_unit", "s2_tri256_f64", "s3_tet33_f64",
                                  "s4_rgg64k_f32", "s4_rgg64k_f32_one"])
def test_coarsen_levels_match_oracle(ctx, name):
    g, cfg = I.config_graph(name)
    api = _api()
    levels_ref, total_ref = O.coarsen(g, cfg["ratio"], cfg["mode"])
    L = len(levels_ref)
    n_c = levels_ref[-1].target
    lift, nca, st = ctx.coarsen(api.CSR.from_graph(g), n_c, levels=L)
    assert nca == levels_ref[-1].n_c
    assert np.array_equal(lift.cpu().numpy(), total_ref)
    got = ctx.levels()
    assert len(got) == L
    for lv, ref in zip(got, levels_ref):
        assert np.array_equal(_bits(lv.score.cpu().numpy()), _bits(ref.f))
        _check_level(lv, ref)
    em = ctx.compose_emap().cpu().numpy()
    assert np.array_equal(em, O.compose_emaps(levels_ref))


POWERLAW = [("f64", "float", np.float64), ("f32", "float", np.float32),
            ("int", "int", np.int32), ("unit", "unit", np.int32)]


@pytest.mark.parametrize("name,weight,dt", POWERLAW, ids=[p[0] for p in POWERLAW])
def test_powerlaw_multilevel_bitexact(ctx, name, weight, dt):
    """Heavy-tailed degrees shaped like a social network (n = 4039, mean degree 44, 46 rows
    longer than 256 entries, hubs adjacent to hubs): every level of a coarsening to n/8 in three
    halving levels, scores included, bit-exact with the oracle."""
    g = I.powerlaw_graph(4039, 22, 7, weight, dt)
    assert int(np.max(np.diff(g.rowptr))) > 256
    api = _api()
    levels_ref, total_ref = O.coarsen(g, 8, "halving")
    L = len(levels_ref)
    lift, nca, st = ctx.coarsen(api.CSR.from_graph(g), levels_ref[-1].target, levels=L)
    assert nca == levels_ref[-1].n_c
    assert np.array_equal(lift.cpu().numpy(), total_ref)
    for lv, ref in zip(ctx.levels(), levels_ref):
        assert np.array_equal(_bits(lv.score.cpu().numpy()), _bits(ref.f))
        _check_level(lv, ref)


@pytest.mark.parametrize("name", ["s2_tri256_f64", "s4_rgg64k_f32", "powerlaw_int"])
def test_coarsen_without_self_mass_matches_oracle(ctx, name):
    """The other multilevel reading (each level scores the coarse graph without its internal
    weight): every level bit-exact with the oracle's self_mass_degree=False, and no carried
    mass reported."""
    api = _api()
    if name == "powerlaw_int":
        g, ratio, mode = I.powerlaw_graph(4039, 22, 7, "int", np.int32), 8, "halving"
    else:
        g, cfg = I.config_graph(name)
        ratio, mode = cfg["ratio"], cfg["mode"]
    levels_ref, total_ref = O.coarsen(g, ratio, mode, self_mass_degree=False)
    L = len(levels_ref)
    lift, nca, st = ctx.coarsen(api.CSR.from_graph(g), levels_ref[-1].target, levels=L,
                                self_mass=False)
    assert nca == levels_ref[-1].n_c
    assert np.array_equal(lift.cpu().numpy(), total_ref)
    for lv, ref in zip(ctx.levels(), levels_ref):
        assert lv.mass is None
        assert np.array_equal(_bits(lv.score.cpu().numpy()), _bits(ref.f))
        _check_level(lv, ref)


def test_self_mass_reading_differs_and_carries_the_internal_weight(ctx):
    """The two readings agree on the first level and part from the second on; under the
    self-mass reading every level's carried mass of an integer-weight graph is exactly the
    total weight of the original edges inside each super-node."""
    api = _api()
    g = I.random_graph(3000, 0.003, 21, weight="int", dtype=np.int32, connected=True)
    csr = api.CSR.from_graph(g)
    lift_a, _, _ = ctx.coarsen(csr, g.n // 16, levels=4)
    lv_a = ctx.levels()
    lift_b, _, _ = ctx.coarsen(csr, g.n // 16, levels=4, self_mass=False)
    lv_b = ctx.levels()
    assert torch.equal(lv_a[0].lift, lv_b[0].lift)
    assert not all(torch.equal(x.lift, y.lift) for x, y in zip(lv_a, lv_b))
    comp = np.arange(g.n)
    for lv in lv_a:
        comp = lv.lift.cpu().numpy()[comp]
        inside = comp[g.eu] == comp[g.ev]
        want = np.bincount(comp[g.eu][inside], weights=g.w_und[inside].astype(np.float64),
                           minlength=lv.n_c).astype(np.int64)
        assert np.array_equal(lv.mass.cpu().numpy(), want)
    assert np.array_equal(comp, lift_a.cpu().numpy())


def test_coarsen_host_buffers_match_device(ctx):
    api = _api()
    g, cfg = I.config_graph("s2_tri256_f64")
    dev_lift, nc1, _ = ctx.coarsen(api.CSR.from_graph(g), g.n // 64, levels=6)
    host = api.CSR.from_graph(g, device="cpu", pin=True)
    lift_h = torch.empty(g.n, dtype=torch.int32).pin_memory()
    lift, nc2, _ = ctx.coarsen(host, g.n // 64, levels=6, lift_out=lift_h)
    assert nc1 == nc2
    assert np.array_equal(lift.numpy(), dev_lift.cpu().numpy())


def test_coarsen_batched_matches_per_graph_oracle(ctx):
    api = _api()
    b, cfg = I.config_graph("s5_batch40_f32")
    res = O.coarsen_batch(b, cfg["ratio"], cfg["mode"])
    csr = api.CSR.from_graph(b.graph)
    gp = torch.from_numpy(b.graph_ptr).cuda()
    lift, gpc, st = ctx.coarsen_batched(csr, gp, cfg["ratio"], levels=3)
    lift = lift.cpu().numpy(); gpc = gpc.cpu().numpy()
    for bi, (levels_ref, total_ref) in enumerate(res):
        n0, n1 = b.graph_ptr[bi], b.graph_ptr[bi + 1]
        assert gpc[bi + 1] - gpc[bi] == levels_ref[-1].n_c
        assert np.array_equal(lift[n0:n1] - gpc[bi], total_ref)
    # the final coarse graphs, graph by graph
    last = ctx.level(2, batched_B=b.B)
    rp = last.rowptr_c.cpu().numpy(); cc = last.col_c.cpu().numpy(); wc = last.w_c.cpu().numpy()
    for bi, (levels_ref, _) in enumerate(res):
        cg = levels_ref[-1].coarse.graph
        s0, s1 = gpc[bi], gpc[bi + 1]
        seg_rp = rp[s0:s1 + 1] - rp[s0]
        assert np.array_equal(seg_rp, cg.rowptr)
        assert np.array_equal(cc[rp[s0]:rp[s1]] - s0, cg.col)
        assert np.array_equal(_bits(wc[rp[s0]:rp[s1]]), _bits(cg.w))


@pytest.mark.parametrize("dt", [np.float32, np.float64])
def test_batched_per_graph_prefixes(ctx, dt):
    """A batch of random geometric graphs (their first level needs about 1.7 times n - n_c of
    the lightest scores, so their first per-graph slab of 1.5 times falls short and is
    extended), meshes, a disconnected graph and graphs too small to keep a super-node of eight:
    every graph's lift and final coarse graph equal the oracle's coarsening of that graph
    (binary32 and binary64 weights: 32- and 64-bit score keys)."""
    api = _api()
    graphs = [I.rgg_3d(4096, 12.0, 31, dtype=dt),
              I.tri_mesh_2d(40, 30, 5, jitter=0.3, weight="inv_len", dtype=dt),
              I.rgg_3d(20000, 12.0, 32, dtype=dt), I.path_graph(5, dt),
              I.random_graph(3000, 0.0012, 17, weight="float", dtype=dt, connected=False),
              I.rgg_3d(1500, 8.0, 33, dtype=dt),
              I.tet_mesh_3d(12, 6, jitter=0.25, weight="inv_len", dtype=dt)]
    b = I.batch_of(graphs)
    assert b.graph.m > 65536  # large enough for the per-graph prefixes
    res = O.coarsen_batch(b, 8, "halving")
    csr = api.CSR.from_graph(b.graph)
    gp = torch.from_numpy(b.graph_ptr).cuda()
    ctx.time_kernel("*")
    try:
        lift, gpc, st = ctx.coarsen_batched(csr, gp, 8, levels=3)
        prof = ctx.kernel_profile()
    finally:
        ctx.time_kernel(None)
    # level 0 (the levels below 65,536 edges take no prefix): the first slabs, the extension
    # of the graphs that fell short, the final check
    assert prof.get("k_graph_prefix<KT>", (0,))[0] >= 3, sorted(prof)
    lift = lift.cpu().numpy(); gpc = gpc.cpu().numpy()
    last = ctx.level(2, batched_B=b.B)
    rp = last.rowptr_c.cpu().numpy(); cc = last.col_c.cpu().numpy(); wc = last.w_c.cpu().numpy()
    for bi, (levels_ref, total_ref) in enumerate(res):
        n0, n1 = b.graph_ptr[bi], b.graph_ptr[bi + 1]
        assert gpc[bi + 1] - gpc[bi] == levels_ref[-1].n_c
        assert np.array_equal(lift[n0:n1] - gpc[bi], total_ref)
        cg = levels_ref[-1].coarse.graph
        s0, s1 = gpc[bi], gpc[bi + 1]
        assert np.array_equal(rp[s0:s1 + 1] - rp[s0], cg.rowptr)
        assert np.array_equal(cc[rp[s0]:rp[s1]] - s0, cg.col)
        assert np.array_equal(_bits(wc[rp[s0]:rp[s1]]), _bits(cg.w))


# ---- S9 and the autograd Function ---------------------------------------------------------------------

def test_backward_and_autograd(ctx):
    api = _api()
    g, cfg = I.config_graph("s4_rgg64k_f32")
    levels_ref, _ = O.coarsen(g, cfg["ratio"], cfg["mode"])
    L = len(levels_ref)
    ctx.coarsen(api.CSR.from_graph(g), levels_ref[-1].target, levels=L)
    levels = ctx.levels()
    plan = api.ContractionPlan.from_levels(ctx, levels)
    w = torch.from_numpy(g.w_und).cuda().requires_grad_(True)
    a = api.contract_weights(w, plan)
    assert np.array_equal(_bits(a.detach().cpu().numpy()), _bits(levels_ref[-1].coarse.a_und))
    gvec = torch.randn(a.shape[0], dtype=torch.float32, device="cuda",
                       generator=torch.Generator("cuda").manual_seed(0))
    (a * gvec).sum().backward()
    em = O.compose_emaps(levels_ref)
    ref = O.contract_backward(em, gvec.cpu().numpy())
    assert np.array_equal(w.grad.cpu().numpy(), ref)


def test_rgg64k_contraction_finite_differences(ctx):
    """The 2^16-point RGG coarsened to n/256 in 8 levels, its contraction differentiated with
    the assignment held fixed: central differences of L(w) = <a(w), g> along random directions
    match <grad, direction> from the backward kernel -- in binary64 (the same plan applied to
    binary64 weights) to 1e-9, and in the configured binary32 to the rounding of the sums."""
    api = _api()
    g, cfg = I.config_graph("s4_rgg64k_f32")
    levels_ref, _ = O.coarsen(g, cfg["ratio"], cfg["mode"])
    ctx.coarsen(api.CSR.from_graph(g), levels_ref[-1].target, levels=len(levels_ref))
    plan = api.ContractionPlan.from_levels(ctx, ctx.levels())
    gen = torch.Generator("cuda").manual_seed(3)
    for dt, h, rtol in ((torch.float64, 1e-3, 1e-9), (torch.float32, 5e-2, 1e-3)):
        w = torch.from_numpy(g.w_und.astype(np.float64)).to("cuda", dt).requires_grad_(True)
        a = api.contract_weights(w, plan)
        gvec = torch.randn(a.shape[0], dtype=dt, device="cuda", generator=gen)
        (a * gvec).sum().backward()
        for _ in range(3):
            d = torch.randint(0, 2, w.shape, device="cuda", generator=gen).to(dt) * 2 - 1
            lp = (api.contract_weights(w.detach() + h * d, plan).double() * gvec.double()).sum()
            lm = (api.contract_weights(w.detach() - h * d, plan).double() * gvec.double()).sum()
            fd = ((lp - lm) / (2 * h)).item()
            dot = (w.grad.double() * d.double()).sum().item()
            assert abs(fd - dot) <= rtol * max(1.0, abs(dot)), (dt, fd, dot)


def test_autograd_gradcheck_and_fd_float64(ctx):
    api = _api()
    g = I.random_graph(60, 0.1, 5, weight="float", dtype=np.float64, connected=True)
    ctx.coarsen(api.CSR.from_graph(g), 9, levels=2)
    plan = api.ContractionPlan.from_levels(ctx, ctx.levels())
    w = torch.from_numpy(g.w_und).cuda().requires_grad_(True)
    assert torch.autograd.gradcheck(lambda x: api.contract_weights(x, plan), (w,), eps=1e-6,
                                    atol=1e-8)
    # central finite differences of L(w) = <a(w), gvec>
    a = api.contract_weights(w, plan)
    gvec = torch.linspace(-2, 3, a.shape[0], dtype=torch.float64, device="cuda")
    (a * gvec).sum().backward()
    h = 1e-4
    for e in (0, 7, 33, g.m - 1):
        wp = w.detach().clone(); wp[e] += h
        wm = w.detach().clone(); wm[e] -= h
        fd = ((api.contract_weights(wp, plan) * gvec).sum()
              - (api.contract_weights(wm, plan) * gvec).sum()) / (2 * h)
        assert abs(fd.item() - w.grad[e].item()) < 1e-8


# ---- error paths -----------------------------------------------------------------------------------

def _bad(kind, dtype=np.float64):
    g = I.random_graph(30, 0.2, 1, weight="float", dtype=dtype, connected=True)
    rowptr, col, w = g.rowptr.copy(), g.col.copy(), g.w.copy()
    if kind == "unsorted":
        r = np.argmax(np.diff(rowptr) >= 3)
        a = rowptr[r]
        col[a], col[a + 1] = col[a + 1], col[a]
    elif kind == "asym":
        w[5] = w[5] * 1.5
    elif kind == "asym_ulp":  # one unit in the last place, one entry
        w[5] = np.nextafter(w[5], w.dtype.type(np.inf))
    elif kind == "weight":
        w[3] = -1.0
        # keep it symmetric so only the weight check can fire
        r = np.searchsorted(rowptr, 3, side="right") - 1
        y = col[3]
        j = rowptr[y] + np.searchsorted(col[rowptr[y]:rowptr[y + 1]], r)
        w[j] = -1.0
    elif kind == "range":
        col[-1] = 10 ** 6
    return rowptr, col, w


@pytest.mark.parametrize("dt", [np.float64, np.float32])
@pytest.mark.parametrize("kind,code", [("unsorted", -4), ("asym", -2), ("asym_ulp", -2),
                                       ("weight", -9), ("range", -4)])
def test_invalid_input_reported(ctx, kind, code, dt):
    """Every input check, on binary64 (symmetry by the score walks) and binary32 (symmetry by
    the fingerprint of the flat normalise kernel) graphs."""
    api = _api()
    from paper_2204_11757_gb300 import native as N
    rowptr, col, w = _bad(kind, dt)
    csr = api.CSR.from_numpy(rowptr, col, w)
    with pytest.raises(N.SpcError) as ei:
        ctx.coarsen(csr, 5, levels=1)
    assert ei.value.status == code
    # the context stays usable
    g = I.path_graph(5)
    lift, nc, st = ctx.coarsen(api.CSR.from_graph(g), 2)
    assert nc == 2


def _balanced_asymmetric(dtype=np.float64):
    """Symmetric graph with a long row (node 599, 400 neighbours), then two defects that keep
    the entry count even and every row sorted: an upper entry (450, 599) whose mirror the long
    row lacks, and an upper entry (x, y) between short rows removed while its mirror (y, x)
    stays."""
    n = 600
    rng = np.random.default_rng(21)
    edges = {(int(a), 599) for a in range(400)}
    while len(edges) < 1400:
        a, b = sorted(rng.integers(0, 599, size=2))
        if a != b:
            edges.add((int(a), int(b)))
    eu = np.array([e[0] for e in sorted(edges)]); ev = np.array([e[1] for e in sorted(edges)])
    g = I.csr_from_edges(n, eu, ev, rng.uniform(0.5, 1.5, size=eu.shape[0]))
    rows = [list(zip(g.col[g.rowptr[x]:g.rowptr[x + 1]], g.w[g.rowptr[x]:g.rowptr[x + 1]]))
            for x in range(n)]
    assert all(c != 599 for c, _ in rows[450])
    rows[450].append((599, 1.0))
    x = next(x for x in range(420, 598) if any(c > x and c != 599 for c, _ in rows[x]))
    drop = next(c for c, _ in rows[x] if c > x and c != 599)
    rows[x] = [(c, wv) for c, wv in rows[x] if c != drop]
    rowptr = np.zeros(n + 1, dtype=np.int64)
    rowptr[1:] = np.cumsum([len(r) for r in rows])
    col = np.array([c for r in rows for c, _ in r], dtype=np.int32)
    w = np.array([wv for r in rows for _, wv in r], dtype=dtype)
    assert rowptr[-1] == g.nnz
    return rowptr, col, w


@pytest.mark.parametrize("dt", [np.float64, np.float32])
def test_asymmetry_hidden_by_balanced_counts_is_reported(ctx, dt):
    """Equal numbers of entries above and below the diagonal, yet not symmetric: the missing
    mirror of an entry pointing into a long row must be found (binary64: by the score kernels'
    lookup in the long row; binary32: by the symmetry fingerprint), with and without graph
    replay."""
    api = _api()
    from paper_2204_11757_gb300 import native as N
    rowptr, col, w = _balanced_asymmetric(dt)
    csr = api.CSR.from_numpy(rowptr, col, w)
    for _ in range(3):
        with pytest.raises(N.SpcError) as ei:
            ctx.coarsen(csr, 50, levels=1)
        assert ei.value.status == -2
    with pytest.raises(N.SpcError) as ei:
        ctx.score(csr)
    assert ei.value.status == -2


def test_long_row_weight_asymmetry_reported_binary32(ctx):
    """A binary32 hub whose row holds one weight a unit in the last place off its mirror: the
    fingerprint covers the entries of long rows too."""
    api = _api()
    from paper_2204_11757_gb300 import native as N
    g = I.powerlaw_graph(4039, 22, 7, "float", np.float32)
    deg = np.diff(g.rowptr)
    h = int(np.argmax(deg))
    assert deg[h] > 256
    w = g.w.copy()
    j = int(g.rowptr[h]) + 3
    w[j] = np.nextafter(w[j], np.float32(np.inf))
    csr = api.CSR.from_numpy(g.rowptr, g.col, w)
    with pytest.raises(N.SpcError) as ei:
        ctx.coarsen(csr, g.n // 2, levels=1)
    assert ei.value.status == -2
    # unchanged weights pass
    ctx.coarsen(api.CSR.from_graph(g), g.n // 2, levels=1)


def test_invalid_arguments(ctx):
    api = _api()
    from paper_2204_11757_gb300 import native as N
    g = I.path_graph(5)
    with pytest.raises(N.SpcError) as ei:
        ctx.coarsen(api.CSR.from_graph(g), 0)
    assert ei.value.status == -1


def test_self_loop_reported(ctx):
    api = _api()
    from paper_2204_11757_gb300 import native as N
    rowptr = np.array([0, 2, 3], dtype=np.int64)
    col = np.array([0, 1, 0], dtype=np.int32)
    w = np.ones(3, dtype=np.float64)
    with pytest.raises(N.SpcError) as ei:
        ctx.score(api.CSR.from_numpy(rowptr, col, w))
    assert ei.value.status in (-3, -2)


def test_contract_rejects_out_of_range_lift(ctx):
    api = _api()
    from paper_2204_11757_gb300 import native as N
    g = I.path_graph(6)
    bad = torch.tensor([0, 1, 2, 3, 4, 9], dtype=torch.int32, device="cuda")
    with pytest.raises(N.SpcError) as ei:
        ctx.contract(api.CSR.from_graph(g), bad, 5)
    assert ei.value.status == -1


# ---- long rows and hubs (exact parallel evaluation of the sequential sums) -----------------------

HUBS = [
    ("star64", lambda: I.star_ties(12, np.float64)),
    ("star32", lambda: I.star_ties(12, np.float32)),
    ("star64_chords", lambda: I.star_ties(11, np.float64, chords=3000, seed=1)),
    ("star32_chords", lambda: I.star_ties(11, np.float32, chords=3000, seed=2)),
    ("hubs_f64", lambda: I.hub_graph(6000, [5000, 3000, 700, 300, 257], 3, "float", np.float64)),
    ("hubs_f32", lambda: I.hub_graph(6000, [5000, 3000, 700, 300], 4, "float", np.float32)),
    ("hubs_int", lambda: I.hub_graph(6000, [4000, 2500, 600], 5, "int", np.int32)),
    ("hubs_unit", lambda: I.hub_graph(5000, [4999, 4000, 256, 257, 258], 6, "unit", np.int32)),
]


@pytest.mark.parametrize("name,make", HUBS, ids=[h[0] for h in HUBS])
def test_hub_scores_and_level_bitexact(ctx, name, make):
    g = make()
    api = _api()
    ref_f = O.score(g)
    csr = api.CSR.from_graph(g)
    f = ctx.score(csr).cpu().numpy()
    bad = np.nonzero(_bits(f) != _bits(ref_f))[0]
    assert bad.size == 0, (bad[:10], f[bad[:5]], ref_f[bad[:5]])
    for n_c in (max(1, g.n // 2), max(1, g.n // 7)):
        ref = O.coarsen_level(g, n_c)
        lift, nc, st = ctx.coarsen(csr, n_c, levels=1)
        assert nc == ref.n_c
        _check_level(ctx.level(0), ref)


def test_prefix_filter_retry_on_cliques(ctx):
    """Merging to n/4 on disjoint K4s needs all 3n/4 clique merges; the score prefix that the
    spanning-forest rounds start from cannot hold them (its edges close cycles), so the rounds
    are rerun on all edges -- the result must still be the oracle's."""
    api = _api()
    for dt in (np.float64, np.float32):
        g = I.clique_ring(20000, 4, 8, dt)
        for n_c in (g.n // 4, g.n // 2, g.n // 3):
            ref = O.coarsen_level(g, n_c)
            lift, nc, st = ctx.coarsen(api.CSR.from_graph(g), n_c, levels=1)
            assert nc == ref.n_c
            _check_level(ctx.level(0), ref)


@pytest.mark.parametrize("seed", [0, 1])
def test_scores_with_extreme_weight_ranges(ctx, seed):
    """Weights spanning 1e-300 .. 1e300: normalised weights reach the subnormal range, which the
    per-row reciprocal division must hand to the IEEE division."""
    api = _api()
    g0 = I.random_graph(300, 0.05, 40 + seed, weight="float", dtype=np.float64, connected=True)
    rng = np.random.default_rng(seed)
    w = 10.0 ** rng.uniform(-300, 300, size=g0.m)
    g = I.csr_from_edges(g0.n, g0.eu, g0.ev, w)
    ref = O.score(g)
    f = ctx.score(api.CSR.from_graph(g)).cpu().numpy()
    assert np.array_equal(_bits(f), _bits(ref))
    p_ref = O.normalise(g, O.degree(g))
    assert (p_ref[p_ref > 0] < 2.0 ** -1000).any()  # the fallback range is exercised


# ---- the recorded schedule replayed as a CUDA graph ---------------------------------------------

def _levels_equal(a, b):
    for x, y in zip(a, b):
        for f in ("lift", "emap", "rowptr_c", "col_c", "w_c", "a_und", "self_mass", "score",
                  "perm", "seg"):
            assert torch.equal(getattr(x, f), getattr(y, f)), f


def test_graph_replay_matches_host_driven(ctx):
    """Call 1 runs host-driven and records, call 2 captures and replays, call 3 replays; all
    three must equal the oracle.  Then the weights change in place: the checksum sends the
    call back to the host-driven path, which must give the new oracle result."""
    api = _api()
    g, cfg = I.config_graph("s2_tri256_f64")
    levels_ref, total_ref = O.coarsen(g, cfg["ratio"], cfg["mode"])
    csr = api.CSR.from_graph(g)
    n0 = ctx.launch_count
    runs = []
    for call in range(3):
        lift, nc, st = ctx.coarsen(csr, g.n // 64, levels=6)
        assert np.array_equal(lift.cpu().numpy(), total_ref)
        got = ctx.levels()
        for lv, ref in zip(got, levels_ref):
            _check_level(lv, ref)
        runs.append(got)
    _levels_equal(runs[0], runs[1])
    _levels_equal(runs[0], runs[2])
    assert ctx.launch_count > n0
    # new weights in the same buffers (scaled unevenly: a different coarsening)
    rng = np.random.default_rng(3)
    w_und = g.w_und * rng.uniform(0.5, 2.0, size=g.m)
    g2 = I.csr_from_edges(g.n, g.eu, g.ev, w_und)
    csr.w.copy_(torch.from_numpy(g2.w).cuda())
    levels2, total2 = O.coarsen(g2, cfg["ratio"], cfg["mode"])
    for call in range(2):
        lift, nc, st = ctx.coarsen(csr, g.n // 64, levels=6)
        assert np.array_equal(lift.cpu().numpy(), total2)
        for lv, ref in zip(ctx.levels(), levels2):
            _check_level(lv, ref)


def test_graph_replay_batched(ctx):
    api = _api()
    b, cfg = I.config_graph("s5_batch40_f32")
    csr = api.CSR.from_graph(b.graph)
    gp = torch.from_numpy(b.graph_ptr).cuda()
    outs = [ctx.coarsen_batched(csr, gp, cfg["ratio"], levels=3) for _ in range(3)]
    for lift, gpc, st in outs[1:]:
        assert torch.equal(lift, outs[0][0]) and torch.equal(gpc, outs[0][1])
    res = O.coarsen_batch(b, cfg["ratio"], cfg["mode"])
    lift = outs[2][0].cpu().numpy(); gpc = outs[2][1].cpu().numpy()
    for bi, (levels_ref, total_ref) in enumerate(res):
        n0, n1 = b.graph_ptr[bi], b.graph_ptr[bi + 1]
        assert np.array_equal(lift[n0:n1] - gpc[bi], total_ref)


def test_results_owned_by_the_caller_outlive_later_calls(ctx):
    """spc_take_result hands over the coarse graph, the composed edge map, the lift and the
    carried mass in buffers the caller owns: two coarsenings (and a third call in between) are
    held at once and each still equals its oracle result."""
    api = _api()
    cases = [("s2_tri256_f64", 16), ("s4_rgg64k_f32", 8)]
    held = []
    for name, ratio in cases:
        g, cfg = I.config_graph(name)
        L = int(round(np.log2(ratio)))
        ctx.coarsen(api.CSR.from_graph(g), g.n // ratio, levels=L)
        held.append((g, ratio, ctx.take_result()))
    ctx.coarsen(api.CSR.from_graph(I.cycle_graph(50)), 5, levels=2)  # overwrites the retained levels
    for g, ratio, res in held:
        levels_ref, total_ref = O.coarsen(g, ratio, "halving")
        t = res.tensors()
        last = levels_ref[-1]
        assert (res.n, res.m, res.n_c, res.m_c) == (g.n, g.m, last.n_c, last.coarse.m_c)
        assert np.array_equal(t["lift"].cpu().numpy(), total_ref)
        assert np.array_equal(t["emap"].cpu().numpy(), O.compose_emaps(levels_ref))
        assert np.array_equal(t["rowptr_c"].cpu().numpy(), last.coarse.graph.rowptr)
        assert np.array_equal(t["col_c"].cpu().numpy(), last.coarse.graph.col)
        assert np.array_equal(_bits(t["w_c"].cpu().numpy()), _bits(last.coarse.graph.w))
        assert np.array_equal(_bits(t["mass"].cpu().numpy()), _bits(last.mass))
        res.free()
    from paper_2204_11757_gb300 import native as N
    ctx.contract(api.CSR.from_graph(I.cycle_graph(8)),
                 torch.zeros(8, dtype=torch.int32, device="cuda"), 1)
    with pytest.raises(N.SpcError) as e:  # a single step leaves no coarsening result
        ctx.take_result()
    assert e.value.status == -1


def _reorder_case(name):
    if name == "powerlaw":
        return I.powerlaw_graph(4039, 22, 7, "float", np.float32), 8
    if name == "disconnected":
        g = I.random_graph(3000, 0.0012, 17, weight="int", dtype=np.int32, connected=False)
        return g, 4
    g, cfg = I.config_graph(name)
    return g, cfg["ratio"]


@pytest.mark.parametrize("name", ["s4_rgg64k_f32", "s2_tri256_f64", "powerlaw", "disconnected"])
def test_reordered_coarsening_matches_oracle(ctx, name):
    """The adjacency-reordering option: the renumbering equals the oracle's (8-hop min label,
    2-hop min label, id), the lift equals the oracle's
    coarsening of the renumbered graph read back in the caller's numbering, and every retained
    level equals the oracle's level of the renumbered graph, bit for bit.  A second call replays
    the captured graph with the same result."""
    api = _api()
    g, ratio = _reorder_case(name)
    L = int(round(np.log2(ratio)))
    levels_ref, total_ref, perm_ref = O.coarsen_reordered(g, ratio, "halving")
    csr = api.CSR.from_graph(g)
    for call in range(2):
        lift, nca, st = ctx.coarsen(csr, levels_ref[-1].target, levels=L, reorder=True)
        assert np.array_equal(ctx.reorder_perm(g.n).cpu().numpy(), perm_ref)
        assert nca == levels_ref[-1].n_c
        assert np.array_equal(lift.cpu().numpy(), total_ref)
        for lv, ref in zip(ctx.levels(), levels_ref):
            assert np.array_equal(_bits(lv.score.cpu().numpy()), _bits(ref.f))
            _check_level(lv, ref)
    assert ctx.last_call_replayed
    ctx.coarsen(csr, levels_ref[-1].target, levels=L)
    from paper_2204_11757_gb300 import native as N
    with pytest.raises(N.SpcError):
        ctx.reorder_perm(g.n)  # the last call did not reorder
