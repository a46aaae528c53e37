"""GPU parity: every step of the hot path, through the C ABI, against the CPU oracle.

Bars: bit-exact for integer work (sampled indices, grouping, multiplicities, gathers);
FP64 steps (leverage, CDF) to 1e-9 relative; FP32 products to 1e-5 relative (a few ulps
times the reduction length); solutions of the FP32 path within 1e-5 relative of the
oracle's exact minimiser of the same sampled problem. Every floating-point comparison is
made twice: norm-wise, and element by element (each component within the bar times the
reference's largest component; the worst component is reported).
"""
import math

import numpy as np
import pytest
import torch

import paper_2209_04876_gb300 as kr
from _parity import assert_elementwise, precond_bar, solution_bar, worst_component
from oracle import kron as ko
from workloads import kron_problem

pytestmark = pytest.mark.gpu

SHAPES = [
    ([65], [5]),
    ([17, 33], [3, 7]),
    ([256, 256], [16, 16]),
    ([64, 48, 40], [4, 3, 5]),
    ([9, 11, 7, 13], [2, 3, 2, 4]),
    ([130, 70, 33], [33, 9, 17]),
]


def dev(a, dtype=torch.float32):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def host(t):
    return t.detach().cpu().numpy()


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def f32_factors(As):
    """The FP32 values the GPU sees, promoted exactly to float64 for the oracle."""
    return [np.asarray(A, dtype=np.float32).astype(np.float64) for A in As]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    kr.lib()


def tables(As):
    t = kr.kron_leverage([dev(A) for A in As])
    return [host(c) for c in t["cdf"]], [host(p) for p in t["prob"]], t


# ------------------------------------------------------------------ a1 + a2

@pytest.mark.parametrize("I,R", SHAPES)
def test_leverage_cdf_prob(I, R):
    prob = kron_problem(I, R, dist="lognormal_rows", seed=1)
    As = f32_factors(prob["As"])
    cdfs, probs, t = tables(As)
    for n, A in enumerate(As):
        lev_o = ko.leverage_scores(A)
        lev_g = host(t["lev"][n])
        assert rel(lev_g, lev_o) < 1e-9
        assert_elementwise(lev_g, lev_o, 1e-9, "leverage scores")
        assert abs(lev_g.sum() - R[n]) < 1e-9 * R[n]
        # same CDF convention as the oracle, bit for bit, given the same scores
        np.testing.assert_array_equal(cdfs[n], ko.cdf_table(lev_g))
        np.testing.assert_allclose(probs[n], lev_g / lev_g.sum(), rtol=1e-15)
        assert t["rank"][n] == R[n]


def test_leverage_rank_deficient_reports_erank():
    rng = np.random.default_rng(2)
    A = rng.standard_normal((40, 3))
    A = np.concatenate([A, A[:, :1] * 2.0], axis=1)  # rank 3 of 4
    B = rng.standard_normal((30, 2))
    with pytest.raises(kr.KronError) as e:
        kr.kron_leverage([dev(A), dev(B)])
    assert e.value.name == "KR_ERANK"


# ------------------------------------------------------------------ a3

@pytest.mark.parametrize("I,R", SHAPES)
@pytest.mark.parametrize("s,seed,cid,row", [(1, 0, 0, 0), (4099, 7, 3, 0), (100003, 2 ** 40 + 5, 2 ** 31 + 9, 77)])
def test_sampler_bit_exact(I, R, s, seed, cid, row):
    As = f32_factors(kron_problem(I, R, dist="lognormal_rows", seed=4)["As"])
    cdfs, probs, t = tables(As)
    idx, w = kr.kron_sample(t["cdf"], t["prob"], s, seed, cid, row=row)
    ref = ko.sample_draws(cdfs, s, seed, cid, row=row)
    np.testing.assert_array_equal(host(idx), ref)
    p = np.ones(s)
    for n in range(len(I)):
        p *= probs[n][ref[:, n]]
    np.testing.assert_allclose(host(w), 1.0 / np.sqrt(s * p), rtol=2e-7)


def test_sampler_edge_tables():
    """Zero-mass rows (leading, inner, trailing), a single row, and a point mass."""
    levs = [np.array([0.0, 0.0, 0.3, 0.0, 0.7, 0.0]), np.array([1.0]), np.array([0.0, 5.0, 0.0]),
            np.array([1e-300, 1.0, 1e-17, 3.0])]
    cdfs = [ko.cdf_table(l) for l in levs]
    probs = [ko.probabilities(l) for l in levs]
    s = 200000
    idx, _ = kr.kron_sample([dev(c, torch.float64) for c in cdfs], [dev(p, torch.float64) for p in probs], s, 5, 1,
                            want_w=False)
    ref = ko.sample_draws(cdfs, s, 5, 1)
    got = host(idx)
    np.testing.assert_array_equal(got, ref)
    for n, l in enumerate(levs):
        assert np.all(l[got[:, n]] > 0)
    assert np.all(got[:, 2] == 1)


# ------------------------------------------------------------------ a4 + a5

@pytest.fixture(params=[1, 2, 3], ids=["radix", "rank", "dense"])
def grouping(request):
    """The groupings of the draws: radix sort + runs; ranks in a bitmap of the key space with
    the counts added per draw; ranks with dense per-key counters set by the draws."""
    kr.set_option(kr.OPT_GROUPING, request.param)
    yield request.param
    kr.set_option(kr.OPT_GROUPING, 0)


@pytest.mark.parametrize("I,R", SHAPES)
@pytest.mark.parametrize("s", [1, 997, 60000])
def test_sketch_grouping_weights_gather(I, R, s, grouping):
    prob = kron_problem(I, R, dist="lognormal_rows", seed=5, noise_rel=0.1)
    As = f32_factors(prob["As"])
    b = prob["b"].astype(np.float32)
    cdfs, probs, t = tables(As)
    sk = kr.kron_sketch([dev(A) for A in As], t["cdf"], t["prob"], dev(b), s, 13, 2)
    keys, counts, omega, bt = (host(v) for v in sk.export())
    idx = ko.sample_draws(cdfs, s, 13, 2)
    rk, rc = ko.group_samples(idx, I)
    np.testing.assert_array_equal(keys, rk)
    np.testing.assert_array_equal(counts, rc)
    assert counts.sum() == s
    np.testing.assert_array_equal(bt, b[rk])
    np.testing.assert_allclose(omega, ko.sample_weights(rk, rc, probs, I, s), rtol=1e-6)
    sk.free()


def test_sketch_long_runs_split_into_entries(grouping):
    """A row drawn more than 65535 times is stored as several entries of the same row (the
    multiplicity field is 16 bits): per row, the entries' counts add up to the oracle's
    multiplicity, the dominant row takes ceil(count / 65535) entries, and b~ and the weights
    are those of the row."""
    As = f32_factors([np.array([[100.0], [1.0], [1.0]]), np.array([[1.0], [50.0]]),
                      np.array([[80.0], [1.0], [2.0], [1.0]])])
    I = [3, 2, 4]
    b = np.arange(24, dtype=np.float32) + 1.0
    s = 400000
    cdfs, probs, t = tables(As)
    sk = kr.kron_sketch([dev(A) for A in As], t["cdf"], t["prob"], dev(b), s, 21, 3)
    keys, counts, omega, bt = (host(v) for v in sk.export())
    sk.free()
    rk, rc = ko.group_samples(ko.sample_draws(cdfs, s, 21, 3), I)
    uk, inv = np.unique(keys, return_inverse=True)
    np.testing.assert_array_equal(uk, rk)
    np.testing.assert_array_equal(np.bincount(inv, weights=counts).astype(np.int64), rc)
    assert int(counts.sum()) == s and counts.max() <= 65535
    top = int(np.argmax(rc))
    assert rc[top] > 2 * 65535
    assert int(np.sum(keys == rk[top])) == -(-int(rc[top]) // 65535)
    np.testing.assert_array_equal(bt, b[keys])
    np.testing.assert_allclose(omega, ko.sample_weights(keys, counts, probs, I, s), rtol=1e-6)


def test_sketch_dense_key_space(grouping):
    """1.5 M draws on a key space of 122,880 rows: about 40 % of all rows are drawn, so a
    tile of 65,536 keys of the rank grouping holds 20-28 thousand distinct keys (more than
    its shared-memory staging takes)."""
    I, R = [40, 48, 64], [3, 4, 5]
    prob = kron_problem(I, R, dist="lognormal_rows", seed=5, noise_rel=0.1)
    As = f32_factors(prob["As"])
    b = prob["b"].astype(np.float32)
    cdfs, probs, t = tables(As)
    s = 1500000
    sk = kr.kron_sketch([dev(A) for A in As], t["cdf"], t["prob"], dev(b), s, 13, 2)
    keys, counts, omega, bt = (host(v) for v in sk.export())
    sk.free()
    rk, rc = ko.group_samples(ko.sample_draws(cdfs, s, 13, 2), I)
    assert len(rk) > 40000
    np.testing.assert_array_equal(keys, rk)
    np.testing.assert_array_equal(counts, rc)
    np.testing.assert_array_equal(bt, b[rk])
    np.testing.assert_allclose(omega, ko.sample_weights(rk, rc, probs, I, s), rtol=1e-6)


# ------------------------------------------------------------------ KronMatMul, preconditioner

@pytest.mark.parametrize("I,R", SHAPES)
def test_kron_matmul(I, R):
    As = f32_factors(kron_problem(I, R, seed=6)["As"])
    rng = np.random.default_rng(7)
    x = rng.standard_normal(int(np.prod(R))).astype(np.float32)
    y = kr.kron_matmul([dev(A) for A in As], dev(x))
    assert rel(host(y), ko.kron_matvec(As, x)) < 1e-5
    assert_elementwise(host(y), ko.kron_matvec(As, x), 1e-5, "KronMatMul")
    z = rng.standard_normal(int(np.prod(I))).astype(np.float32)
    g = kr.kron_matmul([dev(A) for A in As], dev(z), trans=[1] * len(As))
    assert rel(host(g), ko.kron_rmatvec(As, z)) < 1e-5
    assert_elementwise(host(g), ko.kron_rmatvec(As, z), 1e-5, "transposed KronMatMul")


@pytest.mark.parametrize("I,R", SHAPES)
@pytest.mark.parametrize("lam", [0.0, 0.37])
def test_preconditioner(I, R, lam):
    As = f32_factors(kron_problem(I, R, dist="lognormal_rows", seed=8)["As"])
    g = np.random.default_rng(9).standard_normal(int(np.prod(R))).astype(np.float32)
    d = kr.kron_precond([dev(A) for A in As], dev(g), lam)
    P = ko.KronPreconditioner(As, lam)
    ref = P.apply(g)
    kappa = float(P.D.max() / P.D.min())
    err = rel(host(d), ref)
    print("precond I=%s R=%s lam=%g: rel %.3e, elementwise %.3e, kappa(M) %.3e" % (
        I, R, lam, err, worst_component(host(d), ref)[0], kappa))
    bar = precond_bar(As, lam)
    assert err < bar, (err, bar)
    assert_elementwise(host(d), ref, bar, "M+ g (bar %.2e)" % bar)


# ------------------------------------------------------------------ a7 + a8

@pytest.mark.parametrize("I,R", SHAPES)
def test_sampled_residual_products(I, R):
    prob = kron_problem(I, R, dist="lognormal_rows", seed=10, noise_rel=0.2)
    As = f32_factors(prob["As"])
    b = prob["b"].astype(np.float32)
    cdfs, probs, t = tables(As)
    s = 3 * int(np.prod(R)) + 101
    sk = kr.kron_sketch([dev(A) for A in As], t["cdf"], t["prob"], dev(b), s, 21, 4)
    keys, counts, _, _ = (host(v) for v in sk.export())
    x = np.random.default_rng(11).standard_normal(int(np.prod(R))).astype(np.float32)
    g, obj = sk.residual(dev(x))
    om = ko.sample_weights(keys, counts, probs, I, s)
    u = ko.sampled_forward(As, keys, x)
    r = om * (b[keys] - u)
    g_ref = ko.sampled_transpose(As, keys, r)
    assert rel(host(g), g_ref) < 1e-5
    assert_elementwise(host(g), g_ref, 1e-5, "K~^T Omega (b~ - K~ x)")
    assert abs(obj - np.sum(om * (b[keys] - u) ** 2)) <= 1e-5 * np.sum(om * (b[keys] - u) ** 2)
    sk.free()


# ------------------------------------------------------------------ full solves

def _oracle_same_sample(As, b, rep, seed, cid, cdfs, probs, lam, eps):
    smp = ko.draw_sample(As, rep["s"], seed, cid, cdfs=cdfs, probs=probs)
    assert smp.keys.shape[0] == rep["distinct"]
    xs, _ = ko.richardson(As, b[smp.keys], smp, lam, eps, tol=1e-13, max_iter=5000)
    return xs, smp


@pytest.mark.parametrize("I,R,dist", [
    ([256, 256], [16, 16], "gauss"),
    ([64, 48, 40], [4, 3, 5], "lognormal_rows"),
    ([65], [5], "gauss"),
    ([9, 11, 7, 13], [2, 3, 2, 4], "outliers"),
    ([130, 70, 33], [33, 9, 17], "gauss"),
    ([1, 60, 45], [1, 6, 5], "gauss"),         # a mode with a single row: one slab of cells
    ([50, 1, 40], [5, 1, 4], "lognormal_rows"),  # single-row middle mode: cells = slabs
    ([40, 30, 1], [4, 3, 1], "gauss"),         # single-row last mode: one sampled row per cell
])
def test_regress_matches_oracle_on_same_sample(I, R, dist):
    prob = kron_problem(I, R, dist=dist, seed=12, noise_rel=0.05)
    As = f32_factors(prob["As"])
    b = prob["b"].astype(np.float32).astype(np.float64)
    eps, seed, cid = 0.1, 99, 5
    x, rep = kr.kron_regress([dev(A) for A in As], dev(b), eps=eps, seed=seed, call_id=cid, tol=1e-7, max_iter=500)
    assert rep["converged"]
    cdfs, probs, _ = tables(As)
    xs, smp = _oracle_same_sample(As, b, rep, seed, cid, cdfs, probs, 0.0, eps)
    assert rel(host(x), xs) <= 1e-5
    assert_elementwise(host(x), xs, solution_bar(As), "x")
    f_s = ko.sampled_objective(As, b[smp.keys], smp, host(x).astype(np.float64), 0.0)
    assert abs(rep["obj_sampled"] - f_s) <= 1e-5 * f_s
    # the (1 + eps) guarantee of Thm 4.5 for this seed
    opt = ko.objective(As, b, ko.closed_form_ls(As, b), 0.0)
    assert ko.objective(As, b, host(x), 0.0) <= (1 + eps) * opt


@pytest.mark.parametrize("I,R", [([256, 256], [16, 16]), ([64, 48, 40], [4, 3, 5]), ([33, 20], [8, 6])])
@pytest.mark.parametrize("lam", [1e-3, 2.0])
def test_ridge_matches_oracle_on_same_sample(I, R, lam):
    prob = kron_problem(I, R, dist="gauss", seed=13, noise_rel=0.01)
    As = f32_factors(prob["As"])
    b = prob["b"].astype(np.float32).astype(np.float64)
    eps, seed, cid = 0.1, 5, 6
    x, rep = kr.kron_ridge([dev(A) for A in As], dev(b), lam, eps=eps, seed=seed, call_id=cid, tol=1e-7,
                           max_iter=500)
    cdfs, probs, _ = tables(As)
    xs, smp = _oracle_same_sample(As, b, rep, seed, cid, cdfs, probs, lam, eps)
    assert rel(host(x), xs) <= 1e-5
    assert_elementwise(host(x), xs, solution_bar(As), "x")
    opt = ko.objective(As, b, ko.closed_form_ridge(As, b, lam), lam)
    assert ko.objective(As, b, host(x), lam) <= (1 + eps) * opt


def test_objective_full():
    prob = kron_problem([64, 48, 40], [4, 3, 5], seed=14, noise_rel=0.3)
    As = f32_factors(prob["As"])
    b = prob["b"].astype(np.float32)
    x = np.random.default_rng(1).standard_normal(60).astype(np.float32)
    f = kr.kron_objective([dev(A) for A in As], dev(b), dev(x), 0.25)
    ref = ko.objective(As, b.astype(np.float64), x, 0.25)
    assert abs(f - ref) <= 1e-6 * ref


@pytest.mark.parametrize("I,R", [([64, 48, 40], [4, 3, 5]),
                                 ([256, 256, 256], [16, 16, 16])])  # b's copy outlasts the draws and sort
@pytest.mark.parametrize("gather,pinned", [(1, True), (0, True), (1, False)],
                         ids=["in-place", "copied", "pageable"])
def test_host_io_matches_device_path(I, R, gather, pinned):
    """Host buffers: a page-locked b is read in place at the sampled rows (OPT_HOST_GATHER 1),
    or copied on the context's copy stream while the solve stream builds the tables, draws
    and groups (OPT_HOST_GATHER 0, and any pageable b); the result is the device path's,
    bit for bit."""
    prob = kron_problem(I, R, seed=15, noise_rel=0.05)
    As = [np.asarray(A, dtype=np.float32) for A in prob["As"]]
    b = prob["b"].astype(np.float32)
    xd, rd = kr.kron_regress([dev(A) for A in As], dev(b), eps=0.1, seed=3, call_id=1)
    bh = torch.tensor(b)
    if pinned:
        bh = bh.pin_memory()
    try:
        kr.set_option(kr.OPT_HOST_GATHER, gather)
        xh, rh = kr.kron_regress([torch.tensor(A) for A in As], bh, eps=0.1, seed=3, call_id=1, host_io=True)
    finally:
        kr.set_option(kr.OPT_HOST_GATHER, 1)
    np.testing.assert_array_equal(host(xd), xh.numpy())
    assert rd["iters"] == rh["iters"] and rd["distinct"] == rh["distinct"]


def test_deterministic_reruns():
    prob = kron_problem([64, 48, 40], [4, 3, 5], dist="lognormal_rows", seed=16, noise_rel=0.05)
    As = [dev(A) for A in prob["As"]]
    b = dev(prob["b"])
    x1, _ = kr.kron_regress(As, b, eps=0.1, seed=1, call_id=2)
    x2, _ = kr.kron_regress(As, b, eps=0.1, seed=1, call_id=2)
    assert torch.equal(x1, x2)


# ------------------------------------------------------------------ error paths (host-side, no device faults)

def test_invalid_arguments():
    As = [dev(np.ones((8, 2)) + np.eye(8, 2)), dev(np.eye(5, 3) + 0.1)]
    b = dev(np.ones(40))
    with pytest.raises(kr.KronError) as e:
        kr.kron_regress(As, b, eps=0.0)
    assert e.value.name == "KR_EINVAL"
    with pytest.raises(kr.KronError) as e:
        kr.kron_regress(As, b, eps=1.5)
    assert e.value.name == "KR_EINVAL"
    with pytest.raises(kr.KronError) as e:
        kr.kron_ridge(As, b, lam=0.0)
    assert e.value.name == "KR_EINVAL"
    with pytest.raises(kr.KronError) as e:  # R > I
        kr.kron_regress([dev(np.ones((2, 3))), As[1]], dev(np.ones(10)), eps=0.1)
    assert e.value.name == "KR_EINVAL"
    for p in (-1, 3):  # 0 FP32, 1 BF16, 2 FP8 e4m3
        with pytest.raises(kr.KronError) as e:
            kr.kron_regress(As, b, eps=0.1, precision=p)
        assert e.value.name == "KR_EINVAL"


def test_nonfinite_rhs_reports_enonfinite():
    prob = kron_problem([32, 16], [4, 3], seed=17, noise_rel=0.1)
    b = prob["b"].copy()
    b[:] = np.nan
    with pytest.raises(kr.KronError) as e:
        kr.kron_regress([dev(A) for A in prob["As"]], dev(b), eps=0.1)
    assert e.value.name == "KR_ENONFINITE"


def test_max_iter_reports_enotconv():
    prob = kron_problem([64, 48], [8, 6], seed=18, noise_rel=0.1)
    with pytest.raises(kr.KronError) as e:
        kr.kron_regress([dev(A) for A in prob["As"]], dev(prob["b"]), eps=0.1, max_iter=2, tol=1e-12)
    assert e.value.name == "KR_ENOTCONV"
