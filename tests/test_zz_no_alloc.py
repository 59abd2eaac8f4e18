"""The no-allocation entry point (ttq_integrate_noalloc) gives the same result
as the plan entry points (ttq_plan_create + ttq_plan_run with a caller-owned
workspace) on two calls in a row.

It exists for callers that must not call cudaMalloc (a framework's memory pool
or a fixed memory budget owns the device memory); it works in a fixed 16 MiB
scratch array inside the library.  This file is collected last so that a run
stopping at the first failure has already run every other test."""
import ctypes
from fractions import Fraction

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
    ref_sum = Fraction(ref["value"]) + Fraction(ref["value_lo"])
    free = []
    for _ in range(2):                       # the scratch keeps the last call's contents
        rc, res = noalloc(p)
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
        assert rc == 0, binding.load().ttq_last_error()
        assert abs(res.value - ref["value"]) <= 1e-12 * abs(ref["value"])
        # the double-double value (hi + lo) against the plan path's, at the
        # double-double tolerance (value_lo is 0 for both in FP64 mode)
        got_sum = Fraction(res.value) + Fraction(res.value_lo)
        assert abs(got_sum - ref_sum) <= Fraction(1e-15) * abs(ref_sum)
        assert (res.sweeps, res.max_rank, res.status, res.n_eval) == \
            (ref["sweeps"], ref["max_rank"], ref["status"], ref["n_eval"])
    # the second call found everything it needs in place: device memory did not move
    assert free[1] == free[0], free


def test_noalloc_rejects_problems_beyond_its_scratch():
    from paper_1903_11554_gb300 import binding
    p = inputs.config_d12()                  # needs ~129 MB of workspace
    assert binding.workspace_bytes(p) > 16 << 20
    rc, _ = noalloc(p)
    assert rc == -4                          # TTQ_ERR_WORKSPACE
    assert b"16 MiB" in binding.load().ttq_last_error()


def test_noalloc_refuses_a_capturing_stream():
    """Called while its stream is being captured into a CUDA graph, the entry
    point returns TTQ_ERR_INVALID_ARG before any CUDA work, and the capture
    the caller started still completes."""
    from paper_1903_11554_gb300 import binding
    p = inputs.config_c4()
    noalloc(p)                               # first call on the device: scratch address looked up
    x = torch.zeros(16, device="cuda")
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        g.capture_begin()
        x.add_(1.0)
        rc, _ = noalloc(p)
        g.capture_end()
    assert rc == -1
    assert b"capturing" in binding.load().ttq_last_error()
    g.replay()
    torch.cuda.synchronize()
    assert float(x[0]) == 1.0
