"""GPU parity of Alg. 3 (FastFactorMatrixUpdate) and TuckerALS through the C ABI.

The factor step is compared row by row with the oracle's Alg. 3 on the identical
sketches (same Philox streams, the GPU's own sampling tables), iterated by the oracle
to 1e-13: the FP32 fixed point sits within 1e-5 relative of the FP64 one. Whole sweeps
are compared with exact ALS (the quality guarantee), since the sampled trajectory is
not unique across precisions.
"""
import numpy as np
import pytest
import torch

import paper_2209_04876_gb300 as kr
from _parity import assert_elementwise
from oracle import kron as ko
from oracle import tucker as tk
from workloads import tucker_init, tucker_tensor

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
    return t.detach().cpu().numpy().astype(np.float64)


def _state(I, R, seed, noise=0.01):
    data = tucker_tensor(I, R, seed=seed, noise_rel=noise)
    X = data["X"].astype(np.float32).astype(np.float64)
    As = [np.asarray(A, np.float32).astype(np.float64) for A in tucker_init(I, R, seed=seed + 1)]
    G = tk.initial_core(X, As).astype(np.float32).astype(np.float64)
    return X, As, G


@pytest.mark.parametrize("I,R,lam", [
    ([24, 20, 18], [3, 3, 2], 1e-3),
    ([17, 33, 12], [4, 2, 3], 0.05),
    ([40, 36], [5, 5], 1e-3),
    ([12, 10, 9, 8], [2, 3, 2, 2], 1e-3),
])
def test_factor_update_matches_oracle_rows(I, R, lam):
    X, As, G = _state(I, R, seed=3)
    eps, seed, cid = 0.1, 17, 40
    N = len(I)
    for n in range(N):
        A_gpu = [dev(A) for A in As]
        rep = kr.tucker_factor_update(dev(X), A_gpu, dev(G), n, lam, eps=eps, seed=seed, call_id=cid + n, tol=1e-7,
                                      max_iter=500)
        assert rep["converged"]
        others = [m for m in range(N) if m != n]
        tab = kr.kron_leverage([A_gpu[m] for m in others])
        cdfs = [c.cpu().numpy() for c in tab["cdf"]]
        probs = [p.cpu().numpy() for p in tab["prob"]]
        A_ref, _ = tk.fast_factor_matrix_update(X, As, G, n, lam, eps, seed, cid + n, tol=1e-13, max_iter=5000,
                                                cdfs=cdfs, probs=probs)
        got = host(A_gpu[n])
        err = np.linalg.norm(got - A_ref, axis=1) / np.linalg.norm(A_ref, axis=1)
        # z = G_(n)^T y is held in FP32: its rounding (~eps32) reaches a = (G+)^T z amplified by
        # up to cond(G_(n)) (Lemma 5.1 substitution); otherwise the FP32-path bar of 1e-5
        bar = max(1e-5, 4 * np.finfo(np.float32).eps * np.linalg.cond(tk.unfold(G, n)))
        assert err.max() <= bar, (n, err.max(), bar)
        assert_elementwise(got, A_ref, bar, "A[%d] (bar %.2e)" % (n, bar))
        for m in others:  # only A[n] changes
            np.testing.assert_array_equal(host(A_gpu[m]), np.asarray(As[m], np.float32))


@pytest.mark.parametrize("n", [0, 1])
def test_factor_update_eps_rule_matches_oracle(n):
    """kr_opts.stop_rule 1 in the factor step (slab path, two other modes): the rows' (1+eps)-aware
    rule on the device (q = g^T M+ g from the row kernel, the row objective from its slab's
    tile partials plus the penalty terms) ends the loop once every row's rule holds, which is
    where the oracle's row rule has stopped its slowest row, within one iteration; every row is
    then a (1+eps)-approximate ridge solution on its sample, the guarantee the rule certifies."""
    I, R, lam = [24, 20, 18], [3, 3, 2], 1e-3
    X, As, G = _state(I, R, seed=3)
    eps, seed, cid = 0.1, 17, 40
    N = len(I)
    A_gpu = [dev(A) for A in As]
    rep = kr.tucker_factor_update(dev(X), A_gpu, dev(G), n, lam, eps=eps, seed=seed, call_id=cid, tol=1e-7,
                                  max_iter=500, stop_rule=kr.STOP_EPS)
    assert rep["stop"] == 3, rep
    others = [m for m in range(N) if m != n]
    tab = kr.kron_leverage([A_gpu[m] for m in others])
    cdfs = [c.cpu().numpy() for c in tab["cdf"]]
    probs = [p.cpu().numpy() for p in tab["prob"]]
    As_o = [As[m] for m in others]
    Gn = tk.unfold(G, n)
    w = tk.penalty_weight(As_o, eps)
    P = tk.WoodburyPreconditioner(As_o, Gn, lam, w)
    Xn = tk.unfold(X, n)
    s = rep["s"]
    got = host(A_gpu[n])
    its = []
    worst = 0.0
    for i in range(I[n]):
        smp = tk.row_sample(As_o, s, seed, cid, i, cdfs=cdfs, probs=probs)
        b_s = Xn[i][smp.keys]
        _, _, it = tk.row_richardson(As_o, Gn, b_s, smp, lam, eps, w, P=P, max_iter=500, stop="eps")
        its.append(it)
        rows = ko.sampled_rows(As_o, smp.keys)
        Y = rows @ Gn.T
        y = tk.row_ridge_on_sample(As_o, Gn, b_s, smp, lam)

        def f(v):
            r = Y @ v - b_s
            return float(np.sum(smp.omega * r * r) + lam * v @ v)

        ratio = f(got[i]) / f(y)
        worst = max(worst, ratio)
        assert ratio <= 1 + eps, (i, ratio)
    print("mode %d: device stopped at %d, oracle rows at %d..%d; worst f(a)/f(y*) %.6f" % (
        n, rep["iters"], min(its), max(its), worst))
    assert abs(rep["iters"] - max(its)) <= 1


def test_tucker_sweeps_reach_exact_als_quality():
    I, R = [32, 28, 24], [3, 3, 3]
    X, As, G = _state(I, R, seed=7)
    lam, eps = 1e-3, 0.1
    A_gpu = [dev(A) for A in As]
    G_gpu = dev(G)
    rep = kr.tucker_als_sweep(dev(X), A_gpu, G_gpu, lam, eps=eps, sweeps=4, seed=5, call_id=0, tol=1e-7,
                              max_iter=300)
    assert rep["iters"] > 0
    rre_gpu = tk.rre(X, host(G_gpu).reshape(R), [host(A) for A in A_gpu])
    he = []
    tk.tucker_als(X, As, G, lam, 4, sampled=False, history=he)
    assert rre_gpu <= (1 + 2 * eps) * he[-1]
    assert rre_gpu < 2e-4  # 1% relative noise -> ~1e-4 floor


GRAPH_CASES = [
    ([32, 28, 24], [3, 3, 3], 0.0, 0, 0),
    ([32, 28, 24], [3, 3, 3], 1e-3, 0, 0),
    ([40, 48, 36], [4, 16, 8], 0.0, 1, 0),
    ([40, 48, 36], [4, 16, 8], 0.0, 0, 1),
    ([20, 18, 16, 14], [2, 3, 2, 3], 0.0, 0, 0),
    ([40, 36], [5, 5], 0.0, 0, 0),
]


@pytest.mark.parametrize("I,R,lam,prec,stop", GRAPH_CASES)
def test_sampled_sweeps_as_one_graph(I, R, lam, prec, stop):
    """Sweeps after the first are captured into ONE CUDA graph: every factor step's and core
    step's Richardson loop is a conditional WHILE node (the BF16 core steps' FP32 refinement
    a second one, entered on the device), the rank and capacitance checks and the penalty w
    device words. Against host-driven sweeps (OPT_DEVICE_LOOP 0): bit for bit where the
    host sweeps are themselves reproducible and the same arithmetic runs (lambda = 0);
    with lambda > 0 the graph applies the core steps' preconditioner in FP64, so factors,
    core and RRE agree to FP32 rounding. Exactly one graph more than a one-sweep call."""
    X, As, G = _state(I, R, seed=13)
    eps = 0.1

    def run(loop, sweeps):
        kr.set_option(kr.OPT_DEVICE_LOOP, loop)
        A_gpu = [dev(A) for A in As]
        G_gpu = dev(G)
        g0 = kr.graph_count()
        rep = kr.tucker_als_sweep(dev(X), A_gpu, G_gpu, lam, eps=eps, sweeps=sweeps, seed=5, call_id=0, tol=1e-7,
                                  max_iter=300, precision=prec, stop_rule=stop)
        return [host(A) for A in A_gpu] + [host(G_gpu)], rep, kr.graph_count() - g0

    try:
        h1, hrep, hg = run(0, 4)
        h2, _, _ = run(0, 4)
        _, _, g_one = run(1, 1)
        gr, grep_, gg = run(1, 4)
    finally:
        kr.set_option(kr.OPT_DEVICE_LOOP, 1)
    assert hg == 0
    assert gg == g_one + 1, (gg, g_one)
    reproducible = all(np.array_equal(a, b) for a, b in zip(h1, h2))
    rre_h = tk.rre(X, h1[-1].reshape(R), h1[:-1])
    rre_g = tk.rre(X, gr[-1].reshape(R), gr[:-1])
    dev_max = max(np.abs(a - b).max() / np.abs(a).max() for a, b in zip(h1, gr))
    print("I=%s R=%s lam %g prec %d stop %d: host reproducible %s, graph vs host max rel diff %.2e, RRE %.6e / %.6e, "
          "iters %d / %d" % (I, R, lam, prec, stop, reproducible, dev_max, rre_h, rre_g, hrep["iters"], grep_["iters"]))
    assert grep_["precision_used"] == hrep["precision_used"]
    if prec:
        assert grep_["precision_used"] == prec and grep_["iters_reduced"] > 0
    if reproducible and lam == 0.0:
        for a, b in zip(h1, gr):
            np.testing.assert_array_equal(a, b)
        assert grep_["iters"] == hrep["iters"]
        assert grep_["iters_reduced"] == hrep["iters_reduced"]
        assert grep_["distinct"] == hrep["distinct"] and grep_["s"] == hrep["s"]
        assert grep_["obj_sampled"] == hrep["obj_sampled"]
    else:
        assert dev_max <= 1e-3
        assert abs(rre_g - rre_h) <= 1e-4 * rre_h
    he = []
    tk.tucker_als(X, As, G, lam, 4, sampled=False, history=he)
    assert rre_g <= (1 + 2 * eps) * he[-1]


def test_tucker_core_step_is_alg2_on_vec_x():
    """The core step of a sweep equals kron_ridge on vec(X) with the updated factors."""
    I, R = [20, 18, 16], [2, 3, 2]
    X, As, G = _state(I, R, seed=9)
    lam, eps = 1e-3, 0.1
    A_gpu = [dev(A) for A in As]
    G_gpu = dev(G)
    kr.tucker_als_sweep(dev(X), A_gpu, G_gpu, lam, eps=eps, sweeps=1, seed=3, call_id=100, tol=1e-7, max_iter=300)
    x, _ = kr.kron_ridge([A.clone() for A in A_gpu], dev(X.reshape(-1)), lam, eps=eps, seed=3, call_id=100 + 3,
                         tol=1e-7, max_iter=300)
    torch.testing.assert_close(G_gpu.reshape(-1), x, rtol=0, atol=0)


def test_tucker_argument_errors():
    X, As, G = _state([10, 9, 8], [2, 2, 2], seed=1)
    A_gpu = [dev(A) for A in As]
    with pytest.raises(kr.KronError) as e:
        kr.tucker_factor_update(dev(X), A_gpu, dev(G), 3, 1e-3)
    assert e.value.name == "KR_EINVAL"
    with pytest.raises(kr.KronError) as e:
        kr.tucker_als_sweep(dev(X), A_gpu, dev(G), -1.0)
    assert e.value.name == "KR_EINVAL"


def test_inplace_arguments_must_be_contiguous():
    X, As, G = _state([10, 9, 8], [2, 2, 2], seed=1)
    A_gpu = [dev(A) for A in As]
    Gnc = dev(G).permute(2, 1, 0)  # non-contiguous view
    with pytest.raises(ValueError):
        kr.tucker_factor_update(dev(X), A_gpu, Gnc, 0, 1e-3)
