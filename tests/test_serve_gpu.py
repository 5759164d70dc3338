"""Continuous-batching server: admission by HBM footprint, requests joining a
running batch, and each result equal to the same job run alone (FP32 within
1e-5 of the field scale, FP64 within 1e-12)."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1710_09534_gb300 import build
    build.build()
    import paper_1710_09534_gb300 as T
    return T


def test_served_results_equal_runs_alone(T):
    from paper_1710_09534_gb300.serve import Request, Server
    jobs = W.served_requests(10, seed=7, lo=64, hi=192, steps_lo=40, steps_hi=300)
    reqs = []
    for i, (w, steps) in enumerate(jobs):
        reqs.append(Request(i, w, steps, ("fp32", "fp16", "fp32", "fp64", "bf16")[i % 5], arrival=0.02 * i))
    lib = T.load_library()
    sizes = sorted(int(lib.tlb_workspace_bytes(w.nx, w.ny, T.PRECISIONS[r.precision])) for r, (w, _) in zip(reqs, jobs))
    budget = sizes[-1] + sizes[-2] + sizes[-3]  # at most a few resident at once
    srv = Server(budget, max_lattices=8, chunk=64)
    stats = srv.run(reqs)
    srv.close()
    s = stats.summary()
    assert s["requests"] == 10 and s["peak_resident_bytes"] <= budget
    assert 1 <= s["peak_resident_lattices"] < 10  # the budget forced queueing
    assert s["p99_s"] >= s["p50_s"] > 0
    for r in reqs:
        assert r.done is not None and r.admitted >= r.arrival - 1e-9
        L = T.lattice_from_workload(r.workload, r.precision)
        L.step(r.steps)
        ref = L.fields()
        tol = 1e-12 if r.precision == "fp64" else 1e-5
        for k in ("c1", "c2", "ux", "uy", "p"):
            scale = max(float(np.abs(ref[k]).max()), 1e-6)
            assert np.abs(r.fields[k] - ref[k]).max() <= tol * scale, (r.rid, k)


def test_request_larger_than_budget_is_rejected(T):
    from paper_1710_09534_gb300.serve import Request, Server
    (w, steps), = W.served_requests(1, seed=1, lo=128, hi=128, steps_lo=10, steps_hi=10)
    srv = Server(1024, max_lattices=2)
    with pytest.raises(ValueError):
        srv.run([Request(0, w, steps)])
    srv.close()
