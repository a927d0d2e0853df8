"""Failure paths through the C ABI (needs a GPU): workspace allocations that fail, and device
waits that give up.  Nothing here faults, traps or hangs the GPU.  The allocation failures are
made on the host (the allocator callback returns NULL); the waits are loops bounded by the
context's wait limit, which the tests lower so that a wait gives up after one iteration, and
every index stays in range when one does."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O
from paper_2204_11757_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    import __graft_entry__ as ge
    ge.build()
    from paper_2204_11757_gb300 import api as A
    return A


def _graph():
    return I.tri_mesh_2d(48, 40, 3, jitter=0.3, weight="inv_len", dtype=np.float64)


def test_allocation_failure_reports_oom_and_the_context_recovers(api):
    """A workspace allocation that fails -- the first, one in the middle, the last of a call --
    makes the call return SPC_ERR_OOM; the same context, given memory again, coarsens exactly as
    the oracle does."""
    from paper_2204_11757_gb300 import native as N
    g = _graph()
    levels_ref, total_ref = O.coarsen(g, 16, "halving")
    count = []
    with api.Context(alloc_hook=lambda nb: count.append(nb) or True) as c:
        c.coarsen(api.CSR.from_graph(g), levels_ref[-1].target, levels=4)
    A = len(count)
    assert A > 10
    for fail_at in sorted({1, 2, A // 3, A // 2, A}):
        seen = [0]
        allow = [False]

        def hook(nb):
            seen[0] += 1
            return allow[0] or seen[0] < fail_at

        with api.Context(alloc_hook=hook) as c:
            csr = api.CSR.from_graph(g)
            with pytest.raises(N.SpcError) as e:
                c.coarsen(csr, levels_ref[-1].target, levels=4)
            assert e.value.status == -5, fail_at  # SPC_ERR_OOM
            allow[0] = True
            lift, nc, st = c.coarsen(csr, levels_ref[-1].target, levels=4)
            assert nc == levels_ref[-1].n_c
            assert np.array_equal(lift.cpu().numpy(), total_ref)


def test_union_find_wait_gives_up_with_timeout(api):
    """With the wait limit at one iteration, every union-find walk that meets a non-root gives
    up: the merge selection returns SPC_ERR_TIMEOUT instead of waiting.  With the default limit
    the same context selects exactly the oracle's partition.  (The graph is small enough that
    the scans of the call run in one block, with no look-back.)"""
    from paper_2204_11757_gb300 import native as N
    g = I.random_graph(3000, 0.002, 8, weight="float", dtype=np.float64, connected=True)
    assert g.n <= 16384 and g.m <= 16384
    n_c = 30
    ref = O.coarsen_level(g, n_c)
    with api.Context() as c:
        csr = api.CSR.from_graph(g)
        f = c.score(csr)
        c.set_wait_limit(1)
        with pytest.raises(N.SpcError) as e:
            c.select_merges(csr, f, n_c)
        assert e.value.status == -7  # SPC_ERR_TIMEOUT
        c.set_wait_limit(0)
        lift, merged, nca, st = c.select_merges(csr, f, n_c)
        assert nca == ref.n_c
        assert np.array_equal(lift.cpu().numpy(), ref.lift)


def test_look_back_wait_gives_up_with_timeout(api):
    """The radix sort's look-back waits for the tiles before it.  With the wait limit at one
    iteration a tile that finds its predecessor unpublished gives up (its writes stay inside
    the output), and the call returns SPC_ERR_TIMEOUT; the default limit sorts exactly."""
    from paper_2204_11757_gb300 import native as N
    rng = np.random.default_rng(4)
    f = rng.random(1 << 22)
    ft = torch.from_numpy(f).cuda()
    with api.Context() as c:
        c.set_wait_limit(1)
        codes = []
        for _ in range(5):
            try:
                c.sort_fitness(ft)
                codes.append(0)
            except N.SpcError as e:
                codes.append(e.status)
        assert -7 in codes, codes
        assert set(codes) <= {0, -7}
        c.set_wait_limit(0)
        order = c.sort_fitness(ft).cpu().numpy()
        assert np.array_equal(order, np.lexsort((np.arange(f.shape[0]), f)).astype(np.int32))
