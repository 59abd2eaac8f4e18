"""The no-allocation entry point (ttq_integrate_noalloc) gives the same result
as the plan entry points (ttq_plan_create + ttq_plan_run with a caller-owned
workspace) on two calls in a row.

It exists for callers that must not call cudaMalloc (a framework's memory pool
or a fixed memory budget owns the device memory); it works in a fixed 16 MiB
scratch array inside the library.  This file is collected last so that a run
stopping at the first failure has already run every other test."""
import ctypes

import pytest

from paper_1903_11554_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1903_11554_gb300 import build
    build.build()


def noalloc(p):
    from paper_1903_11554_gb300 import binding
    lib = binding.load()
    arrays = binding._Arrays(p)
    st = binding.make_struct(p, arrays)
    res = binding.TTQResult()
    stream = torch.cuda.current_stream().cuda_stream
    rc = lib.ttq_integrate_noalloc(ctypes.byref(st), ctypes.c_void_p(stream), ctypes.byref(res))
    return rc, res


@pytest.mark.parametrize("make", [lambda: inputs.config_c4(),
                                  lambda: inputs.make_problem("E", "cube", 6, 33, rank_cap=20, precision="dd")])
def test_noalloc_matches_plan_entry_point(make):
    from paper_1903_11554_gb300 import binding
    p = make()
    ref = binding.integrate(p)
    for _ in range(2):                       # the scratch keeps the last call's contents
        rc, res = noalloc(p)
        assert rc == 0, binding.load().ttq_last_error()
        assert abs(res.value - ref["value"]) <= 1e-12 * abs(ref["value"])
        assert abs(res.value_lo - ref["value_lo"]) <= 1e-12 * abs(ref["value"])
        assert (res.sweeps, res.max_rank, res.status, res.n_eval) == \
            (ref["sweeps"], ref["max_rank"], ref["status"], ref["n_eval"])


def test_noalloc_rejects_problems_beyond_its_scratch():
    from paper_1903_11554_gb300 import binding
    p = inputs.config_d12()                  # needs ~129 MB of workspace
    assert binding.workspace_bytes(p) > 16 << 20
    rc, _ = noalloc(p)
    assert rc == -4                          # TTQ_ERR_WORKSPACE
    assert b"16 MiB" in binding.load().ttq_last_error()
