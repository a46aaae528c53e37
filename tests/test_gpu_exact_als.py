"""Exact TuckerALS on the GPU (KronMatMul factor and core updates, App. C) and the RRE
entry point, against the oracle's exact ALS (factor_update_exact, core_update_exact) and its
RRE. Bars: the FP32 projections of X with FP64 normal equations reach the oracle's factors
and core within 1e-4 of the largest entry (element by element) after one sweep; the RRE
trajectory within 1e-4 relative."""
import numpy as np
import pytest
import torch

import paper_2209_04876_gb300 as kr
from _parity import assert_elementwise
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


def _state(I, R, seed, noise=0.05, rank_mult=2):
    Rt = [min(rank_mult * r, i) for r, i in zip(R, I)]
    X = tucker_tensor(I, Rt, seed=seed, noise_rel=noise)["X"].astype(np.float32).astype(np.float64)
    As = [np.asarray(A, np.float32).astype(np.float64) for A in tucker_init(I, R, seed=seed + 1)]
    G = tk.initial_core(X, As).astype(np.float32).astype(np.float64)
    return X, As, G


@pytest.mark.parametrize("I,R,lam", [
    ([24, 20, 18], [3, 3, 2], 0.0),
    ([30, 26, 22], [4, 5, 3], 1e-3),
    ([12, 10, 9, 8], [2, 3, 2, 2], 1e-3),
    ([40, 36], [4, 4], 0.0),
])
def test_exact_sweep_matches_oracle(I, R, lam):
    X, As, G = _state(I, R, seed=7)
    A_gpu = [dev(A) for A in As]
    G_gpu = dev(G)
    rre = kr.tucker_als_exact_sweep(dev(X), A_gpu, G_gpu, lam, sweeps=1)
    hist = []
    As_o, G_o = tk.tucker_als(X, As, G, lam, 1, sampled=False, history=hist)
    for n in range(len(I)):
        assert_elementwise(A_gpu[n].cpu().numpy(), As_o[n], 1e-4, "A[%d] after one exact sweep" % n)
    assert_elementwise(G_gpu.cpu().numpy().reshape(-1), G_o.reshape(-1), 1e-4, "G after one exact sweep")
    assert abs(rre[0] - hist[0]) <= 1e-4 * hist[0], (rre[0], hist[0])


def test_rre_entry_point():
    X, As, G = _state([20, 18, 16], [4, 3, 5], seed=3)
    got = kr.tucker_rre(dev(X), [dev(A) for A in As], dev(G))
    ref = tk.rre(X, G, As)
    assert abs(got - ref) <= 1e-6 * ref + 1e-12, (got, ref)


def test_exact_als_256cubed_trajectory():
    """The Tucker workload (256^3, multilinear rank (16,16,16) + 1 % noise, lambda = 1e-3):
    five exact sweeps, RRE per sweep against the oracle's exact ALS."""
    I, R = [256, 256, 256], [16, 16, 16]
    data = tucker_tensor(I, R, seed=11, noise_rel=0.01)
    X = np.asarray(data["X"], np.float32).astype(np.float64)
    As = [np.asarray(A, np.float32).astype(np.float64) for A in tucker_init(I, R, seed=12)]
    G = tk.initial_core(X, As).astype(np.float32).astype(np.float64)
    lam = 1e-3
    A_gpu = [dev(A) for A in As]
    rre = kr.tucker_als_exact_sweep(dev(X), A_gpu, dev(G), lam, sweeps=5)
    hist = []
    tk.tucker_als(X, As, G, lam, 5, sampled=False, history=hist)
    for k in range(5):
        assert abs(rre[k] - hist[k]) <= 1e-3 * hist[k] + 1e-7, (k, rre[k], hist[k])


def test_exact_sweep_rejects_singular_factor_systems():
    """lambda = 0 with R_n > prod_{m != n} R_m: G_(n) (K^T K) G_(n)^T is singular."""
    X, As, G = _state([40, 36], [5, 4], seed=7)
    with pytest.raises(kr.KronError) as e:
        kr.tucker_als_exact_sweep(dev(X), [dev(A) for A in As], dev(G), 0.0, sweeps=1)
    assert e.value.name == "KR_EINVAL"


@pytest.mark.parametrize("lam", [0.0, 1e-3])
def test_exact_sweeps_as_one_graph_match_host_sweeps(lam):
    """Sweeps after the first are captured into one CUDA graph (N factor updates, the core
    update and the RRE terms of each): factors, core and RRE equal the host-driven sweeps bit
    for bit, and exactly one graph ran for the call."""
    X, As, G = _state([40, 36, 30], [5, 4, 6], seed=21)
    out = {}
    for loop in (0, 1):
        kr.set_option(kr.OPT_DEVICE_LOOP, loop)
        A_gpu = [dev(A) for A in As]
        G_gpu = dev(G)
        g0 = kr.graph_count()
        rre = kr.tucker_als_exact_sweep(dev(X), A_gpu, G_gpu, lam, sweeps=4)
        out[loop] = ([A.cpu() for A in A_gpu], G_gpu.cpu(), rre, kr.graph_count() - g0)
    kr.set_option(kr.OPT_DEVICE_LOOP, 1)
    assert out[0][3] == 0 and out[1][3] == 1
    for a, b in zip(out[0][0], out[1][0]):
        assert torch.equal(a, b)
    assert torch.equal(out[0][1], out[1][1])
    assert out[0][2] == out[1][2]
