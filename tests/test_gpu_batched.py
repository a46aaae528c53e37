"""The batched ridge (many independent Kronecker ridge problems of uneven shapes, each
an Alg. 2 solve with its own sketch): solved concurrently on worker contexts, every
problem's result is bit-identical to solving it alone, whatever the number of workers;
a hard error in one problem is reported for the batch."""
import numpy as np
import pytest
import torch

import paper_2209_04876_gb300 as kr
from _parity import assert_elementwise, solution_bar
from oracle import kron as ko
from workloads import kron_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    kr.lib()


@pytest.fixture(autouse=True)
def _default_workers():
    yield
    kr.set_option(kr.OPT_BATCH_WORKERS, 4)


def dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


def _problems():
    # uneven shapes drawn once from a seeded generator: N = 2 and 3, I_n in [16, 96],
    # R_n in [2, 8], a mix of factor distributions (the batched-ridge workload in miniature)
    rng = np.random.default_rng(2209)
    out = []
    for k in range(9):
        N = 3 if k % 3 else 2
        I = [int(v) for v in rng.integers(16, 97, size=N)]
        R = [int(min(v, i)) for v, i in zip(rng.integers(2, 9, size=N), I)]
        prob = kron_problem(I, R, dist=["gauss", "lognormal_rows", "outliers"][k % 3], seed=100 + k, noise_rel=0.01)
        out.append(([A.astype(np.float32) for A in prob["As"]], prob["b"].astype(np.float32)))
    return out


@pytest.mark.parametrize("workers", [1, 3, 4, 9])
def test_batched_matches_individual_solves(workers):
    probs = _problems()
    lam, eps, seed, cid = 1e-3, 0.1, 11, 40
    kr.set_option(kr.OPT_BATCH_WORKERS, workers)
    xs, reps = kr.kron_ridge_batched([([dev(A) for A in As], dev(b)) for As, b in probs], lam, eps=eps, seed=seed,
                                     call_id=cid, tol=1e-7, max_iter=300)
    for p, (As, b) in enumerate(probs):
        x1, r1 = kr.kron_ridge([dev(A) for A in As], dev(b), lam, eps=eps, seed=seed, call_id=cid + p, tol=1e-7,
                               max_iter=300)
        assert torch.equal(xs[p], x1)
        assert reps[p]["iters"] == r1["iters"] and reps[p]["distinct"] == r1["distinct"]
        assert reps[p]["obj_sampled"] == r1["obj_sampled"]


def test_batched_against_oracle():
    """Every problem of the batch against the oracle's solve on the same sample."""
    probs = _problems()
    lam, eps, seed, cid = 1e-3, 0.1, 12, 70
    xs, reps = kr.kron_ridge_batched([([dev(A) for A in As], dev(b)) for As, b in probs], lam, eps=eps, seed=seed,
                                     call_id=cid, tol=1e-7, max_iter=300)
    for p in range(len(probs)):
        As = [A.astype(np.float64) for A in probs[p][0]]
        b = probs[p][1].astype(np.float64)
        t = kr.kron_leverage([dev(A) for A in probs[p][0]])
        smp = ko.draw_sample(As, reps[p]["s"], seed, cid + p, cdfs=[c.cpu().numpy() for c in t["cdf"]],
                             probs=[q.cpu().numpy() for q in t["prob"]])
        assert smp.keys.shape[0] == reps[p]["distinct"]
        xs_ref, _ = ko.richardson(As, b[smp.keys], smp, lam, eps, tol=1e-13, max_iter=5000)
        got = xs[p].cpu().numpy().astype(np.float64)
        assert np.linalg.norm(got - xs_ref) <= 1e-5 * np.linalg.norm(xs_ref), p
        assert_elementwise(got, xs_ref, solution_bar(As), "x of problem %d" % p)


def test_batched_reports_first_hard_error():
    probs = _problems()[:4]
    bad = ([np.ones((3, 4), np.float32), probs[1][0][1]], np.ones(3 * probs[1][0][1].shape[0], np.float32))  # R > I
    batch = [([dev(A) for A in As], dev(b)) for As, b in probs[:2]] + [([dev(A) for A in bad[0]], dev(bad[1]))]
    with pytest.raises(kr.KronError) as e:
        kr.kron_ridge_batched(batch, 1e-3, eps=0.1, seed=1, call_id=0)
    assert e.value.name == "KR_EINVAL"


@pytest.fixture
def _fused_modes():
    yield
    kr.set_option(kr.OPT_BATCH_MODE, 0)
    kr.set_option(kr.OPT_AUTOTUNE, 0)
    kr.set_option(kr.OPT_SLAB_TILE_ENTRIES, 16384)


def _batch_shapes(count, seed):
    # the batched-ridge recipe: N = 3, I_n uniform in [64, 256], R_n uniform in [4, 16]
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        I = [int(v) for v in rng.integers(64, 257, size=3)]
        R = [int(v) for v in rng.integers(4, 17, size=3)]
        prob = kron_problem(I, R, dist="gauss", seed=300 + k, noise_rel=0.01)
        out.append(([A.astype(np.float32) for A in prob["As"]], prob["b"].astype(np.float32)))
    return out


def test_fused_batch_bit_identical(_fused_modes):
    """One context per problem, every Richardson loop a node of one CUDA graph: each x and
    report equals the problem's single solve bit for bit (and the worker-context mode's)."""
    probs = _batch_shapes(12, 77)
    lam, eps, seed, cid = 1e-3, 0.1, 5, 10
    args = [([dev(A) for A in As], dev(b)) for As, b in probs]
    kr.set_option(kr.OPT_BATCH_MODE, 1)
    xs_f, reps_f = kr.kron_ridge_batched(args, lam, eps=eps, seed=seed, call_id=cid, tol=1e-7, max_iter=300)
    kr.set_option(kr.OPT_BATCH_MODE, 0)
    xs_w, _ = kr.kron_ridge_batched(args, lam, eps=eps, seed=seed, call_id=cid, tol=1e-7, max_iter=300)
    for p, (As, b) in enumerate(args):
        x1, r1 = kr.kron_ridge(As, b, lam, eps=eps, seed=seed, call_id=cid + p, tol=1e-7, max_iter=300)
        assert torch.equal(xs_f[p], x1), p
        assert torch.equal(xs_w[p], x1), p
        assert reps_f[p]["iters"] == r1["iters"] and reps_f[p]["distinct"] == r1["distinct"]
        assert reps_f[p]["obj_sampled"] == r1["obj_sampled"]


def test_fused_batch_eps_rule_and_precision(_fused_modes):
    """Problems that stop after different numbers of steps, with a second loop round for the
    FP32 refinement of reduced-precision steps: still bit-identical to single solves."""
    probs = _batch_shapes(6, 78)
    lam, eps, seed, cid = 1e-3, 0.1, 6, 30
    args = [([dev(A) for A in As], dev(b)) for As, b in probs]
    kr.set_option(kr.OPT_BATCH_MODE, 1)
    kw = dict(eps=eps, seed=seed, tol=1e-7, max_iter=300, stop_rule=kr.STOP_EPS, precision=1)
    xs_f, reps_f = kr.kron_ridge_batched(args, lam, call_id=cid, **kw)
    for p, (As, b) in enumerate(args):
        x1, r1 = kr.kron_ridge(As, b, lam, call_id=cid + p, **kw)
        assert torch.equal(xs_f[p], x1), p
        assert reps_f[p]["iters"] == r1["iters"] and reps_f[p]["iters_reduced"] == r1["iters_reduced"]


def test_autotune_records_choices_and_reproduces(_fused_modes):
    """The autotuner times one slab pass per candidate tile budget for each new shape class,
    keeps the fastest, and a solve with that budget set by hand reproduces the tuned solve."""
    probs = _batch_shapes(4, 79)
    lam, eps, seed, cid = 1e-3, 0.1, 7, 50
    args = [([dev(A) for A in As], dev(b)) for As, b in probs]
    kr.set_option(kr.OPT_AUTOTUNE, 1)
    kr.set_option(kr.OPT_BATCH_MODE, 1)
    xs, reps = kr.kron_ridge_batched(args, lam, eps=eps, seed=seed, call_id=cid, tol=1e-7, max_iter=300)
    table = {e["key"]: e for e in kr.autotune_report()}
    kr.set_option(kr.OPT_AUTOTUNE, 0)
    kr.set_option(kr.OPT_BATCH_MODE, 0)
    for p, (As, b) in enumerate(args):
        I = [A.shape[0] for A in As]
        R = [A.shape[1] for A in As]
        key = (3, I[1], R[1], I[2], R[2], int(reps[p]["s"]).bit_length() - 1)
        assert key in table, (key, list(table))
        e = table[key]
        assert e["budget"] in (2048, 4096, 8192, 16384, 32768)
        assert e["ms"][e["budget"]] == min(e["ms"].values())
        kr.set_option(kr.OPT_SLAB_TILE_ENTRIES, e["budget"])
        x1, _ = kr.kron_ridge(As, b, lam, eps=eps, seed=seed, call_id=cid + p, tol=1e-7, max_iter=300)
        assert torch.equal(xs[p], x1), p
