"""Reduced-precision sampled products with FP32 refinement (kr_opts.precision 1: BF16,
2: FP8 e4m3 with per-row scales), against the oracle's FP64 minimiser of the same sampled
problem (Alg. 2, Thm 4.5).

The first phase of the Richardson loop runs its slab passes with BF16 or e4m3 tensor-core
products (FP32 accumulation, FP32 residuals); the loop then continues with FP32-accurate
passes until the stopping rule holds, so the fixed point is the FP32 path's. Bars: the
relative gap of the sampled objective, (f~(x) - f~(x*)) / f~(x*), at most 1e-6; x element-wise
within the FP32 path's bar; and, with the (1+eps)-aware rule, f(x) <= (1 + eps) OPT. Shapes
with R_{N-1} a multiple of 32 run e4m3; a multiple of 16 only, BF16 (e4m3 falls back);
N = 2 covers the one-prefix-mode form."""
import numpy as np
import pytest
import torch

import paper_2209_04876_gb300 as kr
from _parity import assert_elementwise, solution_bar, worst_component
from oracle import kron as ko
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


def host(t):
    return t.detach().cpu().numpy()


def f32(As):
    return [np.asarray(A, dtype=np.float32).astype(np.float64) for A in As]


def same_sample(As, b, rep, seed, cid, lam, eps):
    t = kr.kron_leverage([dev(A) for A in As])
    cdfs, probs = [host(c) for c in t["cdf"]], [host(p) for p in t["prob"]]
    smp = ko.draw_sample(As, rep["s"], seed, cid, cdfs=cdfs, probs=probs)
    assert smp.keys.shape[0] == rep["distinct"]
    xs, _ = ko.richardson(As, b[smp.keys], smp, lam, eps, tol=1e-13, max_iter=5000)
    return xs, smp


CASES = [
    # I, R, dist, precision asked, precision run
    ([64, 96, 80], [4, 32, 16], "lognormal_rows", 2, 2),
    ([64, 96, 80], [4, 32, 16], "lognormal_rows", 1, 1),
    ([48, 128, 96], [3, 64, 32], "gauss", 2, 2),
    ([100, 64, 50], [6, 16, 8], "outliers", 2, 1),
    ([100, 64, 50], [6, 16, 8], "outliers", 1, 1),
    ([512, 300], [32, 24], "gauss", 1, 1),
    ([30, 40, 50], [5, 6, 7], "gauss", 1, 0),
]


@pytest.mark.parametrize("I,R,dist,prec,ran", CASES)
@pytest.mark.parametrize("lam", [0.0, 1e-3])
def test_reduced_precision_refined_matches_oracle(I, R, dist, prec, ran, lam):
    prob = kron_problem(I, R, dist=dist, seed=41, noise_rel=0.05)
    As = f32(prob["As"])
    b = prob["b"].astype(np.float32).astype(np.float64)
    eps, seed, cid = 0.1, 7, 3
    solve = (lambda **kw: kr.kron_ridge([dev(A) for A in As], dev(b), lam, **kw)) if lam > 0 else \
        (lambda **kw: kr.kron_regress([dev(A) for A in As], dev(b), **kw))
    x, rep = solve(eps=eps, seed=seed, call_id=cid, tol=1e-7, max_iter=500, precision=prec)
    assert rep["converged"]
    assert rep["precision_used"] == ran
    if ran:
        assert 0 < rep["iters_reduced"] < rep["iters"], rep
    xs, smp = same_sample(As, b, rep, seed, cid, lam, eps)
    f_x = ko.sampled_objective(As, b[smp.keys], smp, host(x).astype(np.float64), lam)
    f_s = ko.sampled_objective(As, b[smp.keys], smp, xs, lam)
    gap = (f_x - f_s) / f_s
    err = worst_component(host(x), xs)[0]
    print("I=%s R=%s prec %d (ran %d) lam %g: %d + %d steps, objective gap %.2e, x error %.2e of max|x*|" % (
        I, R, prec, ran, lam, rep["iters_reduced"], rep["iters"] - rep["iters_reduced"], gap, err))
    assert gap <= 1e-6
    assert_elementwise(host(x), xs, solution_bar(As), "x after refinement")


@pytest.mark.parametrize("prec", [1, 2])
def test_reduced_precision_eps_rule_certifies(prec):
    """With the (1+eps)-aware rule the refinement ends once FP32 passes certify the step;
    the returned x is a (1+eps)-approximate least-squares solution."""
    I, R = [96, 128, 64], [4, 32, 16]
    prob = kron_problem(I, R, dist="outliers", seed=43, noise_rel=0.05)
    As = f32(prob["As"])
    b = prob["b"].astype(np.float32).astype(np.float64)
    eps = 0.1
    x, rep = kr.kron_regress([dev(A) for A in As], dev(b), eps=eps, seed=9, call_id=1, max_iter=200,
                             stop_rule=kr.STOP_EPS, precision=prec)
    assert rep["stop"] in (1, 2, 3) and rep["precision_used"] == prec
    assert rep["iters"] > rep["iters_reduced"] >= 1
    opt = ko.objective(As, b, ko.closed_form_ls(As, b), 0.0)
    ratio = ko.objective(As, b, host(x).astype(np.float64), 0.0) / opt
    print("prec %d: %d + %d steps, f(x)/OPT = %.6f" % (prec, rep["iters_reduced"], rep["iters"] - rep["iters_reduced"],
                                                       ratio))
    assert ratio <= 1 + eps
