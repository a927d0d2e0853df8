"""Node-feature pooling on the GPU vs the CPU oracle, element by element (needs a GB300).

The pooled features are the mean of each super-node's members, summed in ascending member id
and divided once by the member count, so the GPU result must equal the oracle's bit for bit;
so must the gradient (one division per element).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O
from paper_2204_11757_gb300 import inputs as I

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


def _same_bits(got, want):
    got = np.ascontiguousarray(got)
    want = np.ascontiguousarray(want)
    assert got.dtype == want.dtype and got.shape == want.shape
    u = np.uint64 if got.dtype.itemsize == 8 else np.uint32
    bad = np.nonzero(got.view(u).ravel() != want.view(u).ravel())[0]
    assert bad.size == 0, (bad[:8], got.ravel()[bad[:4]], want.ravel()[bad[:4]])


def _check(ctx, lift, n_c, x, g):
    lt = torch.from_numpy(lift).cuda()
    xc = ctx.pool_features(lt, n_c, torch.from_numpy(x).cuda()).cpu().numpy()
    _same_bits(xc, O.pool_features(lift, n_c, x))
    gx = ctx.pool_features_backward(lt, n_c, torch.from_numpy(g).cuda()).cpu().numpy()
    _same_bits(gx, O.pool_backward(lift, n_c, g))


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("F", [1, 3, 32, 65])
def test_pool_random_lifts(ctx, dtype, F):
    """Random assignments (some super-nodes empty), member counts from 0 to a few hundred,
    features of mixed sign and magnitude."""
    rng = np.random.default_rng(F)
    n, n_c = 20000, 700
    lift = (rng.pareto(1.2, size=n) * 40).astype(np.int64) % n_c
    lift = lift.astype(np.int32)
    x = (rng.standard_normal((n, F)) * 10.0 ** rng.integers(-3, 4, size=(n, 1))).astype(dtype)
    g = rng.standard_normal((n_c, F)).astype(dtype)
    _check(ctx, lift, n_c, x, g)


@pytest.mark.parametrize("name,F", [("c1_tri64_unit", 8), ("s2_tri256_f64", 16),
                                    ("s4_rgg64k_f32", 5)])
def test_pool_on_coarsening_lifts(ctx, name, F):
    """The composed lift of a multilevel coarsening: super-nodes of every size up to the hub
    super-node of the deep levels."""
    api = _api()
    g, cfg = I.config_graph(name)
    levels = 1 if cfg["mode"] == "one" else int(round(np.log2(cfg["ratio"])))
    lift, n_c, _ = ctx.coarsen(api.CSR.from_graph(g), g.n // cfg["ratio"], levels=levels)
    lift = lift.cpu().numpy()
    rng = np.random.default_rng(3)
    for dtype in (np.float32, np.float64):
        x = rng.standard_normal((g.n, F)).astype(dtype)
        gr = rng.standard_normal((n_c, F)).astype(dtype)
        _check(ctx, lift, n_c, x, gr)
    if name != "c1_tri64_unit":
        assert np.bincount(lift).max() > 256  # super-nodes of several chunks are covered


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_pool_extreme_magnitudes(ctx, dtype):
    """Features and gradients from the subnormal range to near overflow, so that the
    divisions take both the reciprocal path and the IEEE division."""
    rng = np.random.default_rng(9)
    n, n_c, F = 6000, 333, 7
    lift = rng.integers(0, n_c, size=n).astype(np.int32)
    info = np.finfo(dtype)
    lo, hi = np.log2(float(info.tiny)) - 10, np.log2(float(info.max)) - 12
    def vals(shape):
        e = rng.uniform(lo, hi, size=shape)
        return (rng.choice([-1.0, 1.0], size=shape) * np.exp2(e)).astype(dtype)
    _check(ctx, lift, n_c, vals((n, F)), vals((n_c, F)))


def test_pool_autograd(ctx):
    api = _api()
    rng = np.random.default_rng(4)
    n, n_c, F = 300, 17, 4
    lift = torch.from_numpy(rng.integers(0, n_c, size=n).astype(np.int32)).cuda()
    x = torch.randn(n, F, dtype=torch.float64, device="cuda").requires_grad_(True)
    assert torch.autograd.gradcheck(lambda t: api.pool_features(t, lift, n_c, ctx), (x,),
                                    eps=1e-6, atol=1e-9)


def test_pool_invalid_lift_and_edge_sizes(ctx):
    from paper_2204_11757_gb300 import native as N
    lift = torch.tensor([0, 1, 5], dtype=torch.int32, device="cuda")
    x = torch.ones(3, 2, dtype=torch.float32, device="cuda")
    with pytest.raises(N.SpcError) as e:
        ctx.pool_features(lift, 3, x)
    assert e.value.status == -1
    # the context stays usable; one node per super-node gives x back exactly
    lift = torch.arange(3, dtype=torch.int32, device="cuda")
    x = torch.randn(3, 2, dtype=torch.float32, device="cuda")
    assert torch.equal(ctx.pool_features(lift, 3, x), x)
