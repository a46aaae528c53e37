"""GPU parity of the fused slab pass (the sampled products of Alg. 2's Richardson step,
Thm 4.4 with T = the last mode, evaluated slab by slab) against the oracle.

Every variant of the kernel is run: R_N padded to 4, 8, 16 and 64 lanes' worth of
columns, R_{N-1} = 64, the tensor-core form of the tile products (R_{N-1} a multiple of
16), A(N) in shared memory and read through L1, N = 2 (one slab),
3 and 4 (prefix mode products), slabs without sampled rows, and a small tile budget that
splits cells across lane groups and slabs across tiles. The per-cell formulation is run
on the same inputs as a cross-check of the two evaluation orders.
"""
import numpy as np
import pytest
import torch

import paper_2209_04876_gb300 as kr
from _parity import assert_elementwise, solution_bar
from oracle import kron as ko
from workloads import kron_problem, tucker_init, tucker_tensor

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    kr.lib()


@pytest.fixture(autouse=True)
def _default_options():
    yield
    kr.set_option(kr.OPT_SLAB_PASS, 1)
    kr.set_option(kr.OPT_SLAB_TILE_ENTRIES, 16384)
    kr.set_option(kr.OPT_DEVICE_LOOP, 1)
    kr.timing_enable(False)


def dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


def host(t):
    return t.detach().cpu().numpy().astype(np.float64)


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300)


def _problem(I, R, dist, seed, zero_rows=0):
    prob = kron_problem(I, R, dist=dist, seed=seed, noise_rel=0.05)
    As = [np.asarray(A, np.float32).astype(np.float64) for A in prob["As"]]
    if zero_rows:
        As[0][:zero_rows] = 0.0  # zero leverage: these slabs are never sampled
    b = prob["b"].astype(np.float32).astype(np.float64)
    return As, b


def _solve(As, b, lam, slab, budget=16384, seed=7, cid=3):
    kr.set_option(kr.OPT_SLAB_PASS, int(slab))
    kr.set_option(kr.OPT_SLAB_TILE_ENTRIES, budget)
    kr.timing_enable(True)
    kr.timing_reset()
    if lam > 0:
        x, rep = kr.kron_ridge([dev(A) for A in As], dev(b), lam, eps=0.1, seed=seed, call_id=cid, tol=1e-7,
                               max_iter=500)
    else:
        x, rep = kr.kron_regress([dev(A) for A in As], dev(b), eps=0.1, seed=seed, call_id=cid, tol=1e-7,
                                 max_iter=500)
    launches = kr.timing_read()
    kr.timing_enable(False)
    return x, rep, launches


def _oracle(As, b, rep, lam, seed=7, cid=3):
    t = kr.kron_leverage([dev(A) for A in As])
    cdfs = [c.cpu().numpy() for c in t["cdf"]]
    probs = [p.cpu().numpy() for p in t["prob"]]
    smp = ko.draw_sample(As, rep["s"], seed, cid, cdfs=cdfs, probs=probs)
    assert smp.keys.shape[0] == rep["distinct"]
    xs, _ = ko.richardson(As, b[smp.keys], smp, lam, 0.1, tol=1e-13, max_iter=5000)
    return xs, smp


SHAPES = [
    ([256, 256], [16, 16], "gauss", 0),            # N = 2: one slab, 16 columns per lane
    ([300, 200], [16, 7], "lognormal_rows", 0),    # N = 2, R_N = 7 padded to 8
    ([64, 48, 40], [4, 3, 5], "lognormal_rows", 0),
    ([9, 11, 7, 13], [2, 3, 2, 4], "outliers", 0),  # N = 4: two prefix modes
    ([130, 70, 40], [2, 3, 33], "gauss", 0),       # R_N = 33 padded to 64 (4 lanes per row)
    ([20, 100, 30], [1, 64, 3], "gauss", 0),       # R_{N-1} = 64
    ([20, 30, 100], [1, 3, 64], "lognormal_rows", 0),  # R_N = 64, A(N) in shared memory
    ([3, 4, 2000], [1, 2, 64], "gauss", 0),        # R_N = 64, A(N) too large for shared memory
    ([40, 30, 50], [3, 4, 5], "gauss", 25),        # 25 of 40 slabs never sampled
    # R_{N-1} a multiple of 16: Y and Z on the TF32 tensor path (three products per term)
    ([40, 50, 60], [3, 16, 8], "lognormal_rows", 0),  # one n tile
    ([24, 64, 48], [2, 32, 24], "gauss", 0),          # R_N = 24 padded to 32 (padding columns dropped)
    ([16, 40, 80], [2, 16, 64], "outliers", 0),       # R_N = 64, A(N) in shared memory
    ([6, 70, 40], [2, 32, 32], "lognormal_rows", 4),  # bench ranks, slabs without sampled rows
]


@pytest.mark.parametrize("budget", [16384, 256])
@pytest.mark.parametrize("I,R,dist,zero", SHAPES)
def test_slab_pass_matches_oracle(I, R, dist, zero, budget):
    As, b = _problem(I, R, dist, seed=21, zero_rows=zero)
    x, rep, launches = _solve(As, b, 0.0, slab=True, budget=budget)
    assert launches["slab"][1] > 0 and launches["resid"][1] == 0
    assert rep["converged"]
    xs, smp = _oracle(As, b, rep, 0.0)
    assert rel(host(x), xs) <= 1e-5
    assert_elementwise(host(x), xs, solution_bar(As), "x")
    f_s = ko.sampled_objective(As, b[smp.keys], smp, host(x), 0.0)
    assert abs(rep["obj_sampled"] - f_s) <= 1e-5 * f_s


@pytest.mark.parametrize("I,R", [([64, 48, 40], [4, 3, 5]), ([256, 256], [16, 16])])
def test_slab_pass_ridge_matches_oracle(I, R):
    As, b = _problem(I, R, "gauss", seed=22)
    lam = 0.5
    x, rep, launches = _solve(As, b, lam, slab=True, budget=512)
    assert launches["slab"][1] > 0
    xs, _ = _oracle(As, b, rep, lam)
    assert rel(host(x), xs) <= 1e-5
    assert_elementwise(host(x), xs, solution_bar(As), "x")


@pytest.mark.parametrize("I,R,dist,zero", [SHAPES[2], SHAPES[4], SHAPES[8]])
def test_slab_and_per_cell_forms_agree(I, R, dist, zero):
    As, b = _problem(I, R, dist, seed=23, zero_rows=zero)
    xa, ra, la = _solve(As, b, 0.0, slab=True)
    xb, rb, lb = _solve(As, b, 0.0, slab=False)
    assert la["slab"][1] > 0 and lb["slab"][1] == 0 and lb["resid"][1] > 0
    assert ra["distinct"] == rb["distinct"]
    assert rel(host(xa), host(xb)) <= 2e-5
    assert_elementwise(host(xa), host(xb), 2e-5, "slab vs per-cell x")
    assert abs(ra["obj_sampled"] - rb["obj_sampled"]) <= 1e-5 * rb["obj_sampled"]


@pytest.mark.parametrize("budget", [16384, 256])
def test_slab_pass_is_deterministic(budget):
    """Fixed-order sums everywhere (segments, partials, multi-tile slabs): reruns match
    bit for bit although tiles go to teams in a different order each time."""
    As, b = _problem([64, 48, 40], [4, 3, 5], "lognormal_rows", seed=24)
    x1, r1, _ = _solve(As, b, 0.0, slab=True, budget=budget)
    x2, r2, _ = _solve(As, b, 0.0, slab=True, budget=budget)
    assert torch.equal(x1, x2)
    assert r1["obj_sampled"] == r2["obj_sampled"] and r1["iters"] == r2["iters"]


@pytest.mark.parametrize("I,R,lam", [([64, 48, 40], [4, 3, 5], 0.0), ([40, 30, 50], [3, 4, 5], 0.3),
                                     ([256, 256], [16, 16], 0.0)])
def test_device_loop_matches_host_loop(I, R, lam):
    """Richardson steps as one CUDA graph (device-side stopping rule) give the same iterate,
    bit for bit, and the same iteration count as returning to the host after every step."""
    As, b = _problem(I, R, "lognormal_rows", seed=25)
    out = []
    for loop in (1, 0):
        kr.set_option(kr.OPT_DEVICE_LOOP, loop)
        l0 = kr.launch_count()
        if lam > 0:
            x, rep = kr.kron_ridge([dev(A) for A in As], dev(b), lam, eps=0.1, seed=4, call_id=2, tol=1e-7,
                                   max_iter=500)
        else:
            x, rep = kr.kron_regress([dev(A) for A in As], dev(b), eps=0.1, seed=4, call_id=2, tol=1e-7,
                                     max_iter=500)
        out.append((x, rep, kr.launch_count() - l0))
    (xg, rg, lg), (xh, rh, lh) = out
    assert torch.equal(xg, xh)
    assert rg["iters"] == rh["iters"] and rg["converged"] == rh["converged"]
    assert rg["obj_sampled"] == rh["obj_sampled"]
    assert lg == lh  # launches inside the graph are counted per step


def test_device_loop_stops_at_max_iter():
    As, b = _problem([64, 48, 40], [4, 3, 5], "gauss", seed=26)
    with pytest.raises(kr.KronError) as e:
        kr.kron_regress([dev(A) for A in As], dev(b), eps=0.1, seed=4, call_id=2, tol=1e-14, max_iter=5)
    assert e.value.name == "KR_ENOTCONV"
    x, rep = kr.kron_regress([dev(A) for A in As], dev(b), eps=0.1, seed=4, call_id=2, tol=1e-14, max_iter=5,
                             raise_notconv=False)
    assert rep["iters"] == 5


def test_set_option_rejects_bad_values():
    for key, val in [(kr.OPT_SLAB_PASS, 2), (kr.OPT_SLAB_TILE_ENTRIES, 100), (kr.OPT_SLAB_TILE_ENTRIES, (1 << 22) + 1),
                     (kr.OPT_DEVICE_LOOP, 7), (kr.OPT_BATCH_WORKERS, 0), (kr.OPT_BATCH_WORKERS, 33),
                     (kr.OPT_GROUPING, -1), (kr.OPT_GROUPING, 4), (kr.OPT_HOST_GATHER, 2), (99, 1)]:
        with pytest.raises(kr.KronError) as e:
            kr.set_option(key, val)
        assert e.value.name == "KR_EINVAL"


@pytest.mark.parametrize("I,R,dist,lam", [
    ([256, 256], [16, 16], "gauss", 0.0),
    ([64, 48, 40], [4, 3, 5], "lognormal_rows", 0.0),
    ([9, 11, 7, 13], [2, 3, 2, 4], "outliers", 1e-3),
    ([6, 70, 40], [2, 32, 32], "lognormal_rows", 0.0),
])
def test_groupings_give_identical_solves(I, R, dist, lam):
    """Radix sort + runs, ranks in a key bitmap with per-draw counts, and ranks with dense
    per-key counters build the same sketch, so whole solves agree bit for bit (same merged
    rows, iterations and iterate); repeated dense-counter builds leave the counters clean."""
    As, b = _problem(I, R, dist, seed=23)
    out = []
    try:
        for g in (1, 2, 3, 3):
            kr.set_option(kr.OPT_GROUPING, g)
            x, rep, launches = _solve(As, b, lam, slab=True)
            out.append((host(x), rep))
    finally:
        kr.set_option(kr.OPT_GROUPING, 0)
    (x1, r1) = out[0]
    for x2, r2 in out[1:]:
        assert r1["distinct"] == r2["distinct"] and r1["iters"] == r2["iters"]
        np.testing.assert_array_equal(x1, x2)


def test_groupings_give_identical_tucker_factor_steps():
    """The batched-row sketch of an Alg. 3 factor step (one draw batch per row of X_(n))
    through both groupings."""
    I, R = [24, 20, 18], [3, 3, 2]
    X = tucker_tensor(I, R, seed=3, noise_rel=0.01)["X"].astype(np.float32)
    As = [np.asarray(A, np.float32) for A in tucker_init(I, R, seed=4)]
    G = np.random.default_rng(5).standard_normal(R).astype(np.float32)
    got = []
    try:
        for g in (1, 2, 3):
            kr.set_option(kr.OPT_GROUPING, g)
            A_gpu = [dev(A) for A in As]
            kr.tucker_factor_update(dev(X), A_gpu, dev(G), 1, 1e-3, eps=0.1, seed=9, call_id=2, tol=1e-7, max_iter=500)
            got.append(host(A_gpu[1]))
    finally:
        kr.set_option(kr.OPT_GROUPING, 0)
    np.testing.assert_array_equal(got[0], got[1])
    np.testing.assert_array_equal(got[0], got[2])
