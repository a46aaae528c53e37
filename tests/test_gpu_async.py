"""Asynchronous solves (kron_regress_async / kron_ridge_async): the Alg. 2 solve enqueued on
the stream without waiting, its report written in device memory; when the stream is being
captured, the whole solve (tables, sketch, tiles, the Richardson loop as conditional WHILE
nodes, the final FP64 check) goes into the caller's CUDA graph.

Bar: bit-identical to the synchronous solve (which is itself oracle-pinned in
test_gpu_parity.py) at lambda = 0, including the BF16 first phase with its FP32 refinement
and the (1+eps)-aware rule; at lambda > 0 the asynchronous solve applies the preconditioner in
FP64 (the host's choice for badly conditioned factors), so x agrees to the FP32 bar."""
import numpy as np
import pytest
import torch

import paper_2209_04876_gb300 as kr
from _parity import assert_elementwise
from workloads import kron_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    kr.lib()


def dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


def problem(I, R, dist, seed):
    prob = kron_problem(I, R, dist=dist, seed=seed, noise_rel=0.05)
    return [dev(A) for A in prob["As"]], dev(prob["b"])


CASES = [
    ([64, 48, 40], [4, 3, 5], "lognormal_rows", 0, 0),
    ([96, 128, 64], [4, 32, 16], "outliers", 1, 1),
    ([96, 128, 64], [4, 32, 16], "outliers", 2, 0),
    ([200, 150], [8, 6], "gauss", 0, 1),
]


def same_report(r, rep):
    for k in ("iters", "iters_reduced", "precision_used", "s", "distinct", "converged", "stop"):
        assert r[k] == rep[k], (k, r[k], rep[k])
    assert r["rel_update"] == rep["rel_update"]


@pytest.mark.parametrize("I,R,dist,prec,stop", CASES)
def test_async_solve_matches_sync(I, R, dist, prec, stop):
    As, b = problem(I, R, dist, seed=5)
    kw = dict(eps=0.1, seed=3, call_id=7, tol=1e-7, max_iter=300, precision=prec, stop_rule=stop)
    x, rep = kr.kron_regress(As, b, **kw)
    g0 = kr.graph_count()
    xa, rd = kr.kron_regress_async(As, b, **kw)
    r = kr.read_dev_report(rd)
    print("I=%s R=%s prec %d stop %d: %d iterations (%d reduced), status %s" % (I, R, prec, stop, r["iters"],
                                                                             r["iters_reduced"], r["status"]))
    assert r["status"] == "KR_OK"
    assert torch.equal(xa, x)
    same_report(r, rep)
    assert r["obj_sampled"] == rep["obj_sampled"]
    # one loop graph, and one more for the refinement of a reduced-precision solve
    assert kr.graph_count() - g0 == 1 + (1 if rep["precision_used"] else 0)


def test_async_ridge_matches_sync_to_fp32():
    As, b = problem([80, 60, 50], [5, 4, 6], "gauss", seed=8)
    lam = 1e-3
    kw = dict(eps=0.1, seed=4, call_id=2, tol=1e-7, max_iter=300)
    x, rep = kr.kron_ridge(As, b, lam, **kw)
    xa, rd = kr.kron_ridge_async(As, b, lam, **kw)
    r = kr.read_dev_report(rd)
    assert r["status"] == "KR_OK" and r["converged"]
    assert r["s"] == rep["s"] and r["distinct"] == rep["distinct"]
    assert_elementwise(xa.cpu().numpy(), x.cpu().numpy().astype(np.float64), 1e-5, "ridge x, asynchronous vs synchronous")
    # both x are within the FP32 bar of one minimiser: their objectives agree to first order in
    # the difference
    assert abs(r["obj_sampled"] - rep["obj_sampled"]) <= 1e-7 * rep["obj_sampled"]


@pytest.mark.parametrize("prec", [0, 1])
def test_async_solve_captured_into_caller_graph(prec):
    """Captured with torch.cuda.graph: the library launches nothing during the capture; each
    replay re-runs the whole solve on the current contents of b."""
    I, R = [96, 128, 64], [4, 32, 16]
    As, b = problem(I, R, "outliers", seed=11)
    kw = dict(eps=0.1, seed=9, call_id=1, tol=1e-7, max_iter=300, precision=prec, stop_rule=1)
    x_ref, rep = kr.kron_regress(As, b, **kw)  # sizes every buffer of the context
    x = torch.empty_like(x_ref)
    rd = torch.zeros(64, dtype=torch.uint8, device="cuda")
    graph = torch.cuda.CUDAGraph()
    n0, l0 = kr.graph_count(), kr.launch_count()
    with torch.cuda.graph(graph, capture_error_mode="relaxed"):
        kr.kron_regress_async(As, b, x=x, report=rd, **kw)
    assert kr.graph_count() == n0
    torch.cuda.synchronize()
    x.zero_()
    graph.replay()
    torch.cuda.synchronize()
    r = kr.read_dev_report(rd)
    assert r["status"] == "KR_OK"
    assert torch.equal(x, x_ref)
    same_report(r, rep)
    # a new right-hand side in the same buffer: the replay solves it
    _, b2 = problem(I, R, "outliers", seed=12)
    b.copy_(b2)
    graph.replay()
    torch.cuda.synchronize()
    x2, rep2 = kr.kron_regress(As, b2, **kw)
    assert torch.equal(x, x2)
    same_report(kr.read_dev_report(rd), rep2)
    print("prec %d: %d kernels captured, %d iterations" % (prec, kr.launch_count() - l0, r["iters"]))


def test_async_rank_deficient_factor_reports_on_device():
    """A rank-deficient factor: the synchronous solve stops with KR_ERANK before sampling; the
    asynchronous one cannot read the check back, runs on (its sampler stays inside its tables)
    and reports KR_ERANK in the device report."""
    As, b = problem([64, 48, 40], [4, 3, 5], "gauss", seed=2)
    A0 = As[0].clone()
    A0[:, 1] = A0[:, 0]
    As[0] = A0
    kw = dict(eps=0.1, seed=1, call_id=1, tol=1e-7, max_iter=50)
    with pytest.raises(kr.KronError) as e:
        kr.kron_regress(As, b, **kw)
    assert e.value.name == "KR_ERANK"
    _, rd = kr.kron_regress_async(As, b, **kw)
    assert kr.read_dev_report(rd)["status"] == "KR_ERANK"
    # the context is still usable
    As2, b2 = problem([64, 48, 40], [4, 3, 5], "gauss", seed=3)
    _, rep = kr.kron_regress(As2, b2, **kw)
    assert rep["converged"]


def test_async_argument_errors():
    As, b = problem([30, 20], [3, 2], "gauss", seed=1)
    with pytest.raises(kr.KronError) as e:
        kr.kron_ridge_async(As, b, 0.0)
    assert e.value.name == "KR_EINVAL"
    with pytest.raises(ValueError):
        kr.kron_regress_async(As, b, report=torch.zeros(8, dtype=torch.uint8, device="cuda"))
    with pytest.raises(ValueError):
        kr.kron_regress_async([A.t() for A in As], b)
