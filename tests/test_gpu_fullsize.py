"""Parity at the full sizes of the paper-shaped workloads, in the bench's launch
configuration, against the CPU oracle (FP64) on the same sample:

* the whole sketch, bit-exact (every draw regrouped by the oracle's sampler, in a pool of
  spawned processes);
* x element by element against the oracle's FP64 Richardson solve of the same sampled
  problem (run with step 1 to its minimiser; the minimiser does not depend on the step),
  and for the (1+eps)-aware rule the oracle's iteration count and iterate;
* Thm 4.5's f(x) <= (1 + eps) OPT with OPT from the oracle's closed form.

Workloads: N=3 512x32 log-normal rows (eps 0.1 and 0.05), N=3 1024x64 with 10 % outlier
rows and a Tucker right-hand side (eps 0.05, 261,654,300 draws), 8 problems of the 64-problem
batched ridge, N=2 256x16 (dense QR), and the Tucker 256^3 workload."""
import math

import numpy as np
import pytest
import torch

import paper_2209_04876_gb300 as kr
from _parity import assert_elementwise, oracle_multiset, solution_bar
from oracle import kron as ko
from oracle import tucker as tk
from workloads import CONFIGS, batched_shapes, kron_problem, kron_problem_device, tucker_init, tucker_tensor

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    kr.lib()


def dev(a, dtype=torch.float32):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def check_sketch(As_d, b_d, b32, s, seed, cid, I, chunk=4_000_000):
    """The library's sketch of (seed, cid) against the oracle's grouping of all s draws
    (keys, multiplicities, gathered b bit-exact; weights to FP32 rounding). Returns the
    oracle's Sample."""
    tab = kr.kron_leverage(As_d)
    sk = kr.kron_sketch(As_d, tab["cdf"], tab["prob"], b_d, s, seed, cid)
    keys, counts, omega, bt = (v.cpu().numpy() for v in sk.export())
    sk.free()
    cdfs = [c.cpu().numpy() for c in tab["cdf"]]
    probs = [p.cpu().numpy() for p in tab["prob"]]
    rk, rc = oracle_multiset(cdfs, s, seed, cid, I, chunk=chunk)
    np.testing.assert_array_equal(keys, rk)
    np.testing.assert_array_equal(counts, rc)
    np.testing.assert_array_equal(bt, b32[rk])
    om = ko.sample_weights(rk, rc, probs, I, s)
    np.testing.assert_allclose(omega, om, rtol=1e-6)
    return ko.Sample(rk, rc, om, s)


def check_solution(As64, b_s, smp, lam, eps, x, what, tol=1e-9):
    """x (the library's tol = 1e-7 solve) against the oracle's sampled minimiser."""
    xs, it = ko.richardson(As64, b_s, smp, lam, eps, step=1.0, tol=tol, max_iter=400)
    xg = x.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(xg - xs) <= 1e-5 * np.linalg.norm(xs), what
    assert_elementwise(xg, xs, solution_bar(As64), what)
    return xs


@pytest.mark.parametrize("eps", [0.1, 0.05])
def test_512cubed_lognormal_full_size(eps):
    """N=3, 512x32 log-normal rows, b of length 512^3 with 5 % noise: the whole sketch
    bit-exact; x against the oracle's sampled minimiser; (1+eps) against the closed form."""
    w = CONFIGS["kron_n3_512x32_lognormal"]
    prob = kron_problem(w["I"], w["R"], dist=w["dist"], seed=2209, noise_rel=w["noise_rel"])
    As32 = [np.ascontiguousarray(A, dtype=np.float32) for A in prob["As"]]
    b32 = np.ascontiguousarray(prob["b"], dtype=np.float32)
    del prob
    As_d = [dev(A) for A in As32]
    b_d = dev(b32)
    seed, cid = 1, 0
    x, rep = kr.kron_regress(As_d, b_d, eps=eps, seed=seed, call_id=cid, tol=1e-7, max_iter=200)
    assert rep["converged"] and rep["s"] == ko.sample_count(32 ** 3, eps)
    smp = check_sketch(As_d, b_d, b32, rep["s"], seed, cid, w["I"])
    assert smp.keys.shape[0] == rep["distinct"]
    As64 = [A.astype(np.float64) for A in As32]
    b64 = b32.astype(np.float64)
    check_solution(As64, b64[smp.keys], smp, 0.0, eps, x, "x (512^3, eps %g)" % eps)
    f_s = ko.sampled_objective(As64, b64[smp.keys], smp, x.cpu().numpy().astype(np.float64), 0.0)
    assert abs(rep["obj_sampled"] - f_s) <= 1e-5 * f_s
    opt = ko.objective(As64, b64, ko.closed_form_ls(As64, b64), 0.0)
    assert ko.objective(As64, b64, x.cpu().numpy().astype(np.float64), 0.0) <= (1 + eps) * opt


def test_large_1024cubed_r64_outliers():
    """The largest workload, as the bench runs it: N=3, A(n) 1024x64 Gaussian with 10 % of
    the rows scaled x20, b a rank-(64,64,64) Tucker tensor + 1 % noise (1024^3 FP32, 4 GB,
    the bench's seeded device generator), eps = 0.05, s = 261,654,300 draws.
    (a) the whole sketch bit-exact; (b) the (1+eps)-aware rule stops at the oracle's
    iteration with the oracle's iterate; (c) the tol = 1e-7 solve against the oracle's
    sampled minimiser, element by element; (d) Thm 4.5 against the oracle's closed form."""
    w = CONFIGS["kron_n3_1024x64_outliers"]
    p = kron_problem_device(w["I"], w["R"], dist=w["dist"], seed=2210, noise_rel=w["noise_rel"], b_kind=w["b_kind"],
                            tucker_rank=w["tucker_rank"])
    As_d, b_d = p["As"], p["b"]
    del p
    eps, seed, cid = w["eps"], 1, 3
    xe, re_ = kr.kron_regress(As_d, b_d, eps=eps, seed=seed, call_id=cid, stop_rule=kr.STOP_EPS, max_iter=200)
    x, rep = kr.kron_regress(As_d, b_d, eps=eps, seed=seed, call_id=cid, tol=1e-7, max_iter=200)
    s = rep["s"]
    assert rep["converged"] and re_["stop"] == 3 and s == ko.sample_count(64 ** 3, eps) == 261654300
    b32 = b_d.cpu().numpy()
    smp = check_sketch(As_d, b_d, b32, s, seed, cid, w["I"])
    assert smp.keys.shape[0] == rep["distinct"] == re_["distinct"]
    del b_d
    torch.cuda.empty_cache()
    As64 = [A.cpu().double().numpy() for A in As_d]
    b_s = b32[smp.keys].astype(np.float64)
    # (b) the eps-aware rule: same stopping iteration, same iterate
    xo, it_o = ko.richardson(As64, b_s, smp, 0.0, eps, stop="eps", tol=1e-13, max_iter=400)
    assert it_o == re_["iters"], (it_o, re_["iters"])
    assert_elementwise(xe.cpu().numpy().astype(np.float64), xo, solution_bar(As64), "x after the eps rule (1024^3)")
    # (c) the converged solve
    check_solution(As64, b_s, smp, 0.0, eps, x, "x (1024^3)")
    del b_s, smp
    # (d) Thm 4.5 with f and OPT in FP64 from the oracle
    b64 = b32.astype(np.float64)
    del b32
    opt = ko.objective(As64, b64, ko.closed_form_ls(As64, b64), 0.0)
    assert ko.objective(As64, b64, xe.cpu().numpy().astype(np.float64), 0.0) <= (1 + eps) * opt
    assert ko.objective(As64, b64, x.cpu().numpy().astype(np.float64), 0.0) <= (1 + eps) * opt


# 8 problems of the 64-problem batch, from 2M to 98M entries of b and R up to 20,150
BATCH_CHECKED = [51, 45, 25, 37, 31, 5, 60, 13]


def test_batched_ridge_64_problems_full_size():
    """The batched-ridge workload at its full size: 64 problems, N = 3, I_n ~ U{64..1024},
    R_n ~ U{4..32}, lambda = 1e-3, Gaussian factors, b = Kronecker signal + 1 % noise
    (about 36 GB of right-hand sides, generated on the device). Every problem meets
    f(x) <= (1 + eps) OPT against the exact ridge solution; the results on 1 and 4 worker
    contexts are bit-identical; 8 problems of the batch match the oracle's solve of the
    same sampled problem element by element, and their OPT the oracle's FP64 closed form."""
    shapes = batched_shapes()
    lam, eps, seed, cid = 1e-3, 0.1, 5, 900
    probs = [kron_problem_device(I, R, dist="gauss", seed=3000 + k, noise_rel=0.01) for k, (I, R) in enumerate(shapes)]
    batch = [(p["As"], p["b"]) for p in probs]
    out = {}
    try:
        for workers in (4, 1):
            kr.set_option(kr.OPT_BATCH_WORKERS, workers)
            out[workers] = kr.kron_ridge_batched(batch, lam, eps=eps, seed=seed, call_id=cid, tol=1e-7, max_iter=300)
    finally:
        kr.set_option(kr.OPT_BATCH_WORKERS, 4)
    (xs4, reps4), (xs1, reps1) = out[4], out[1]
    for p, (As_d, b_d) in enumerate(batch):
        assert reps4[p]["converged"]
        assert torch.equal(xs4[p], xs1[p]) and reps4[p]["iters"] == reps1[p]["iters"]
        KtB = kr.kron_matmul(As_d, b_d, trans=[1] * 3)
        xstar = kr.kron_precond(As_d, KtB, lam)
        opt = kr.kron_objective(As_d, b_d, xstar, lam)
        f = kr.kron_objective(As_d, b_d, xs4[p], lam)
        assert f <= (1.0 + eps) * opt, (p, shapes[p], f / opt)
    for p in BATCH_CHECKED:
        As_d, b_d = batch[p]
        As64 = [A.cpu().double().numpy() for A in As_d]
        b64 = b_d.cpu().double().numpy()
        tab = kr.kron_leverage(As_d)
        smp = ko.draw_sample(As64, reps4[p]["s"], seed, cid + p, cdfs=[c.cpu().numpy() for c in tab["cdf"]],
                             probs=[q.cpu().numpy() for q in tab["prob"]])
        assert smp.keys.shape[0] == reps4[p]["distinct"], p
        check_solution(As64, b64[smp.keys], smp, lam, eps, xs4[p], "x of batch problem %d %s" % (p, shapes[p]))
        opt_cf = ko.objective(As64, b64, ko.closed_form_ridge(As64, b64, lam), lam)
        assert ko.objective(As64, b64, xs4[p].cpu().numpy().astype(np.float64), lam) <= (1 + eps) * opt_cf


def test_n2_256x16_exact_sampled_solution():
    """N=2, A(n) 256x16 Gaussian, b = K x_true + 0.01 N(0,1): x against the dense QR
    solution of the same sampled system."""
    w = CONFIGS["kron_n2_256x16"]
    prob = kron_problem(w["I"], w["R"], dist="gauss", seed=1, noise_abs=w["noise_abs"])
    As = [np.asarray(A, np.float32).astype(np.float64) for A in prob["As"]]
    b = prob["b"].astype(np.float32).astype(np.float64)
    x, rep = kr.kron_regress([dev(A) for A in As], dev(b), eps=w["eps"], seed=3, call_id=4, tol=1e-7,
                             max_iter=300)
    tab = kr.kron_leverage([dev(A) for A in As])
    smp = ko.draw_sample(As, rep["s"], 3, 4, cdfs=[c.cpu().numpy() for c in tab["cdf"]],
                         probs=[p.cpu().numpy() for p in tab["prob"]])
    assert smp.keys.shape[0] == rep["distinct"]
    xs = ko.sampled_exact_solve(As, b[smp.keys], smp, 0.0)
    xg = x.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(xg - xs) <= 1e-5 * np.linalg.norm(xs)
    assert_elementwise(xg, xs, solution_bar(As), "x (256x16, dense QR)")
    opt = ko.objective(As, b, ko.closed_form_ls(As, b), 0.0)
    assert ko.objective(As, b, xg, 0.0) <= (1 + w["eps"]) * opt


def test_tucker_256cubed_rank16():
    """Tucker workload: 256^3 tensor of multilinear rank (16,16,16) + 1% noise, lambda =
    1e-3, eps = 0.1. (a) Alg. 3 rows at full size against the oracle's Alg. 3 on the same
    per-row sketches (a sample of rows); (b) 10 sampled sweeps reach exact-ALS quality."""
    I, R = [256, 256, 256], [16, 16, 16]
    data = tucker_tensor(I, R, seed=11, noise_rel=0.01)
    X = np.ascontiguousarray(data["X"], dtype=np.float32)
    X64 = X.astype(np.float64)
    As = [np.asarray(A, np.float32).astype(np.float64) for A in tucker_init(I, R, seed=12)]
    G = tk.initial_core(X64, As).astype(np.float32).astype(np.float64)
    lam, eps, seed = 1e-3, 0.1, 5
    # (a) one factor step of mode 1
    n = 1
    A_gpu = [dev(A) for A in As]
    rep = kr.tucker_factor_update(dev(X), A_gpu, dev(G), n, lam, eps=eps, seed=seed, call_id=7, tol=1e-7,
                                  max_iter=300)
    assert rep["converged"]
    others = [m for m in range(3) if m != n]
    tab = kr.kron_leverage([A_gpu[m] for m in others])
    cdfs = [c.cpu().numpy() for c in tab["cdf"]]
    probs = [p.cpu().numpy() for p in tab["prob"]]
    rows = [0, 1, 77, 128, 255]
    A_ref, _ = tk.fast_factor_matrix_update(X64, As, G, n, lam, eps, seed, 7, tol=1e-12, max_iter=3000, rows=rows,
                                            cdfs=cdfs, probs=probs)
    got = A_gpu[n].cpu().numpy().astype(np.float64)
    bar = max(1e-5, 4 * np.finfo(np.float32).eps * np.linalg.cond(tk.unfold(G, n)))
    for i in rows:
        assert np.linalg.norm(got[i] - A_ref[i]) <= bar * np.linalg.norm(A_ref[i])
    assert_elementwise(got[rows], A_ref[rows], bar, "Alg. 3 rows (bar %.2e)" % bar)
    # (b) 10 sweeps
    A_gpu = [dev(A) for A in As]
    G_gpu = dev(G)
    kr.tucker_als_sweep(dev(X), A_gpu, G_gpu, lam, eps=eps, sweeps=10, seed=seed, call_id=100, tol=1e-7,
                        max_iter=300)
    rre_gpu = tk.rre(X64, G_gpu.cpu().numpy().astype(np.float64).reshape(R),
                     [A.cpu().numpy().astype(np.float64) for A in A_gpu])
    he = []
    tk.tucker_als(X64, As, G, lam, 10, sampled=False, history=he)
    assert rre_gpu <= (1 + 2 * eps) * he[-1]
    assert rre_gpu < 2e-4
