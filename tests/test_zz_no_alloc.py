"""The allocation-free fitness sort, spc_sort_fitness_static, against spc_sort_fitness.

spc_sort_fitness_static serves callers that must not allocate GPU memory (it keeps its
temporaries in a fixed device array of the library).  Called through the C ABI twice in a row
on different inputs, it must give the same order as the context-based entry point.  This file
is collected last, so a run that stops at its first failure has run every other test before it.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import __graft_entry__ as ge
    ge.build()
    from paper_2204_11757_gb300 import api, native
    ctx = api.Context()
    yield api, native, ctx
    ctx.close()


def _static_sort(native, f: torch.Tensor) -> torch.Tensor:
    order = torch.full((f.shape[0],), -1, dtype=torch.int32, device=f.device)
    dt = native.SPC_F32 if f.dtype == torch.float32 else native.SPC_F64
    stream = torch.cuda.current_stream(f.device).cuda_stream
    rc = native.lib().spc_sort_fitness_static(f.shape[0], ctypes.c_void_p(f.data_ptr()), dt,
                                              ctypes.c_void_p(order.data_ptr()),
                                              ctypes.c_void_p(stream))
    assert rc == 0, native.STATUS_NAMES.get(rc, rc)
    torch.cuda.synchronize()
    return order


def test_static_sort_matches_context_sort_twice(env):
    api, native, ctx = env
    rng = np.random.default_rng(11)
    # first call: binary64 scores with many exact ties, ragged size
    f1 = torch.from_numpy(rng.integers(0, 9, size=300_001).astype(np.float64) / 8.0).cuda()
    # second call right after: binary32 scores of another size, overwriting the shared array
    f2 = torch.from_numpy(rng.random(1_000_000).astype(np.float32) * 2.0).cuda()
    got1 = _static_sort(native, f1)
    got2 = _static_sort(native, f2)
    assert torch.equal(got1, ctx.sort_fitness(f1))
    assert torch.equal(got2, ctx.sort_fitness(f2))
    # and the first input again, after the array held the second one
    assert torch.equal(_static_sort(native, f1), ctx.sort_fitness(f1))


def test_static_sort_rejects_what_it_cannot_do_without_memory(env):
    api, native, ctx = env
    L = native.lib()
    big = torch.zeros((1 << 20) + 1, dtype=torch.float64, device="cuda")
    out = torch.empty(big.shape[0], dtype=torch.int32, device="cuda")
    rc = L.spc_sort_fitness_static(big.shape[0], ctypes.c_void_p(big.data_ptr()), native.SPC_F64,
                                   ctypes.c_void_p(out.data_ptr()), None)
    assert rc == -10  # SPC_ERR_TOO_LARGE, nothing launched
    host = torch.zeros(8, dtype=torch.float64)
    hout = torch.empty(8, dtype=torch.int32)
    rc = L.spc_sort_fitness_static(8, ctypes.c_void_p(host.data_ptr()), native.SPC_F64,
                                   ctypes.c_void_p(hout.data_ptr()), None)
    assert rc == -1  # host memory would need staging, which needs memory
    one = torch.ones(1, dtype=torch.float32, device="cuda")
    assert torch.equal(_static_sort(native, one), torch.zeros(1, dtype=torch.int32, device="cuda"))
