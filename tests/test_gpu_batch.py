"""Batched CS decompositions (csd_batch_*): many real FP64 CSDs of sizes
n ~ U{16..256} in one autotuned, graph-captured launch.  Angles against the
CPU oracle on sampled instances (1e-12 n), backward error and orthogonality
<= 50 n u for every instance, and the graph replay reproduces the first
run bit for bit."""
import numpy as np
import pytest

from oracle import csd as O
from oracle import metrics as M
from paper_1804_09002_gb300 import inputs as I
from tests.gpu_util import U, to_dev, to_host

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1804_09002_gb300 import binding
    return binding


def _instances(count, seed):
    rng = np.random.default_rng(seed)
    sizes = [int(v) for v in rng.integers(16, 257, count)]
    data = [I.haar_csd(n, seed=seed * 10000 + i) for i, n in enumerate(sizes)]
    return sizes, data


def test_batch_matches_oracle_and_bars(B):
    count = 96
    sizes, data = _instances(count, 5)
    ctx = B.Context(0)
    try:
        plan = B.Batch(ctx, sizes)
        plan.load([to_dev(d[0]) for d in data], [to_dev(d[1]) for d in data])
        status = plan.run()
        assert np.all(status == 0)
        first = plan.theta.clone()
        worst_be = worst_orth = worst_th = 0.0
        for i, (n, (A1, A2, th)) in enumerate(zip(sizes, data)):
            R = plan.result(i)
            U1, U2, V1, t = (to_host(R[k]) for k in ("U1", "U2", "V1", "theta"))
            assert np.all(np.diff(t) >= 0)
            assert np.max(np.abs(t - th)) <= 1e-12 * n
            be = M.backward_error_fro(A1, A2, U1, U2, t, V1)
            orth = max(M.orthogonality(X) for X in (U1, U2, V1))
            assert be <= 50 * n * U and orth <= 50 * n * U, (i, n, be / U, orth / U)
            worst_be, worst_orth = max(worst_be, be / (n * U)), max(worst_orth, orth / (n * U))
            if i % 12 == 0:  # sampled instances against the oracle
                ref = O.csd(A1, A2)
                worst_th = max(worst_th, np.max(np.abs(t - ref["theta"])) / n)
                assert np.max(np.abs(t - ref["theta"])) <= 1e-12 * n
        # the captured graph replays the same arithmetic
        plan.run()
        assert torch.equal(plan.theta, first)
        st = plan.stats()
        assert st["granularity"] in (16, 32, 64) and st["buckets"] >= 1
        print(f"batch of {count}: worst backward {worst_be:.2f} n u, orthogonality {worst_orth:.2f} n u, "
              f"theta vs oracle {worst_th:.2e} n; autotuner {st}")
        plan.close()
    finally:
        ctx.close()


def test_batch_new_inputs_same_plan(B):
    """New data in the same packed buffers: the graph reads it (no re-capture)."""
    sizes, data = _instances(8, 7)
    _, data2 = _instances(8, 8)
    ctx = B.Context(0)
    try:
        plan = B.Batch(ctx, sizes)
        plan.load([to_dev(d[0]) for d in data], [to_dev(d[1]) for d in data])
        plan.run()
        # same sizes, other matrices (regenerate at the plan's sizes)
        data2 = [I.haar_csd(n, seed=900 + i) for i, n in enumerate(sizes)]
        plan.load([to_dev(d[0]) for d in data2], [to_dev(d[1]) for d in data2])
        plan.run()
        for i, (n, (A1, A2, th)) in enumerate(zip(sizes, data2)):
            t = to_host(plan.result(i)["theta"])
            assert np.max(np.abs(t - th)) <= 1e-12 * n
        plan.close()
    finally:
        ctx.close()


def test_batch_large_bucket_every_instance_every_replay(B):
    """One bucket of 320 instances (n ~ U{129..192}, about 30k Jacobi pairs
    per round): every instance meets the bars, and three graph replays give
    bit-identical results (a data race in a batched kernel shows up as
    run-to-run differences at this load)."""
    rng = np.random.default_rng(11)
    sizes = [int(v) for v in rng.integers(129, 193, 320)]
    data = [I.haar_csd(n, seed=110000 + i) for i, n in enumerate(sizes)]
    ctx = B.Context(0)
    try:
        plan = B.Batch(ctx, sizes)
        plan.load([to_dev(d[0]) for d in data], [to_dev(d[1]) for d in data])
        status = plan.run()
        assert np.all(status == 0), np.nonzero(status)[0][:10]
        ref = [plan.V1.clone(), plan.theta.clone()]
        dev = plan.V1.device
        for i, (n, (A1, A2, th)) in enumerate(zip(sizes, data)):
            R = plan.result(i)
            eye = torch.eye(n, dtype=torch.float64, device=dev)
            c, s = torch.cos(R["theta"]), torch.sin(R["theta"])
            a1, a2 = to_dev(A1), to_dev(A2)
            be = torch.sqrt(torch.linalg.norm(a1 - (R["U1"] * c) @ R["V1"].T) ** 2 +
                            torch.linalg.norm(a2 - (R["U2"] * s) @ R["V1"].T) ** 2) / np.sqrt(n)
            orth = max(float(torch.linalg.norm(X.T @ X - eye)) for X in (R["U1"], R["U2"], R["V1"]))
            assert float(be) <= 50 * n * U and orth <= 50 * n * U, (i, n, float(be) / U, orth / U)
            assert np.max(np.abs(to_host(R["theta"]) - th)) <= 1e-12 * n
        for _ in range(3):
            plan.run()
            assert torch.equal(plan.V1, ref[0]) and torch.equal(plan.theta, ref[1])
        plan.close()
    finally:
        ctx.close()
