"""JL-approximate leverage scores on the GPU (KR_OPT_JL_K) against the oracle's
jl_leverage_scores (the same Philox sign matrices), and solves sampled by them against the
oracle on the same sample."""
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


@pytest.fixture
def jl():
    def set_jl(k, seed):
        kr.set_option(kr.OPT_JL_K, k)
        kr.set_option(kr.OPT_JL_SEED, seed)
    yield set_jl
    kr.set_option(kr.OPT_JL_K, 0)
    kr.set_option(kr.OPT_JL_SEED, 0)


def dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


@pytest.mark.parametrize("I,R,k", [([300, 200], [12, 30], 16), ([64, 48, 40], [4, 3, 5], 1), ([1000, 513], [64, 7], 64)])
def test_jl_scores_match_oracle(I, R, k, jl):
    As = [np.asarray(A, np.float32).astype(np.float64) for A in kron_problem(I, R, dist="lognormal_rows", seed=4)["As"]]
    jl(k, 2 ** 33 + 17)
    t = kr.kron_leverage([dev(A) for A in As])
    for n, A in enumerate(As):
        ref = ko.jl_leverage_scores(A, k, 2 ** 33 + 17, n)
        got = t["lev"][n].cpu().numpy()
        np.testing.assert_allclose(got, ref, rtol=1e-9, atol=0)
        # sum_i l~_i = ||Q Pi||_F^2 / k = ||Pi||_F^2 / k = rank, for any sign matrix
        assert np.all(got >= 0) and abs(got.sum() - A.shape[1]) <= 1e-9 * A.shape[1]


def test_solve_with_jl_scores(jl):
    """Alg. 2 sampled by JL scores (k = 32): x against the oracle's solve of the same sample
    (drawn from the GPU's JL tables), and (1+eps) against the closed form."""
    prob = kron_problem([64, 48, 40], [4, 3, 5], dist="lognormal_rows", seed=12, noise_rel=0.05)
    As = [np.asarray(A, np.float32).astype(np.float64) for A in prob["As"]]
    b = prob["b"].astype(np.float32).astype(np.float64)
    eps, seed, cid = 0.1, 9, 3
    jl(32, 5)
    x, rep = kr.kron_regress([dev(A) for A in As], dev(b), eps=eps, seed=seed, call_id=cid, tol=1e-7, max_iter=300)
    t = kr.kron_leverage([dev(A) for A in As])
    for n, A in enumerate(As):
        np.testing.assert_allclose(t["lev"][n].cpu().numpy(), ko.jl_leverage_scores(A, 32, 5, n), rtol=1e-9)
    smp = ko.draw_sample(As, rep["s"], seed, cid, cdfs=[c.cpu().numpy() for c in t["cdf"]],
                         probs=[p.cpu().numpy() for p in t["prob"]])
    assert smp.keys.shape[0] == rep["distinct"]
    xs, _ = ko.richardson(As, b[smp.keys], smp, 0.0, eps, step=1.0, tol=1e-11, max_iter=2000)
    assert_elementwise(x.cpu().numpy().astype(np.float64), xs, solution_bar(As), "x (JL scores)")
    opt = ko.objective(As, b, ko.closed_form_ls(As, b), 0.0)
    assert ko.objective(As, b, x.cpu().numpy().astype(np.float64), 0.0) <= (1 + eps) * opt


def test_jl_option_range():
    for v in (-1, 65):
        with pytest.raises(kr.KronError):
            kr.set_option(kr.OPT_JL_K, v)
