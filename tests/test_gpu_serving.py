"""Serving with continuous batching: requests arrive while others are on the
GPU, are admitted at sweep boundaries as slots and pool memory free up, and
each result is the same as alone (needs a GB300)."""
import pytest

from oracle import ttcross
from paper_1903_11554_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1903_11554_gb300 import build
    build.build()


def requests():
    return [
        inputs.make_problem("C", "rn", 4, 41, L=10.0, rank_cap=12, seed=21),
        inputs.make_problem("E", "cube", 6, 33, rank_cap=20, tol=1e-10, seed=22),
        inputs.make_problem("D", "cube", 7, 17, rank_cap=8, seed=23),
        inputs.make_problem("D", "rn", 5, 33, L=8.0, rank_cap=10, seed=24),
        inputs.make_problem("E", "cube", 5, 48, rank_cap=16, precision="dd", seed=25),
        inputs.make_problem("C", "cube", 9, 65, rank_cap=24, tol=1e-9, seed=26),
        inputs.make_problem("TEST", "cube", 3, 33, d=5, rank_cap=8, seed=27),
        inputs.make_problem("C", "cube", 5, 33, rank_cap=16, seed=28),
        inputs.make_problem("D", "rn", 6, 49, L=12.0, rank_cap=16, seed=29),
        inputs.make_problem("E", "cube", 8, 33, rank_cap=24, seed=30),
    ]


def serve(reqs, pool_bytes, max_slots=64, per_step=3, batched=False):
    from paper_1903_11554_gb300 import binding
    srv = binding.Server(pool_bytes, max_slots=max_slots)
    srv.set_mode(batched)
    ids, out, peak_queue, peak_flight = [], {}, 0, 0
    pending = list(reqs)
    for _ in range(10000):
        for _ in range(per_step):                # arrivals between sweeps
            if pending:
                ids.append(srv.submit(pending.pop(0)))
        flight, queued, _ = srv.step(1)
        peak_queue = max(peak_queue, queued)
        peak_flight = max(peak_flight, flight)
        out.update(srv.drain())
        if not pending and len(out) == len(reqs):
            break
    srv.close()
    return [out[i] for i in ids], peak_queue, peak_flight


@pytest.mark.parametrize("batched", [False, True])
def test_served_results_equal_alone(batched):
    from paper_1903_11554_gb300 import binding
    reqs = requests()
    alone = [binding.integrate(p) for p in reqs]
    served, _, flight = serve(reqs, 1 << 30, per_step=2, batched=batched)
    assert flight > 1                            # requests overlapped on the device
    for a, b in zip(served, alone):
        assert a == b
    for p, r in zip(reqs[:4], served[:4]):
        ref = ttcross.integrate(p)["value"]
        assert abs(r["value"] - ref) <= 1e-12 * abs(ref)


@pytest.mark.parametrize("batched", [False, True])
def test_admission_by_memory_queues_and_completes(batched):
    from paper_1903_11554_gb300 import binding
    reqs = requests()
    alone = [binding.integrate(p) for p in reqs]
    need = max(binding.workspace_bytes(p) for p in reqs)
    served, peak_queue, flight = serve(reqs, need + (1 << 18) + 4096, per_step=5, batched=batched)
    assert peak_queue > 0                        # requests waited for memory
    for a, b in zip(served, alone):
        assert a == b


def test_admission_rejects_oversized_and_poll_states():
    from paper_1903_11554_gb300 import binding
    srv = binding.Server(8 << 20, max_slots=4)
    big = inputs.config_d12()
    with pytest.raises(binding.TTQError):
        srv.submit(big)
    rid = srv.submit(inputs.make_problem("C", "cube", 4, 17, rank_cap=6))
    assert srv.poll(rid) is None                 # pending
    for _ in range(100):
        srv.step(1)
        if srv.stats()["retired"] and srv.stats()["in_flight"] == 0:
            break
    srv.step(1)
    assert srv.poll(rid) is not None
    with pytest.raises(binding.TTQError):
        srv.poll(rid)                            # already returned
    srv.close()
