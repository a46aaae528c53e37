"""Randomised TuckerALS at the paper's image-tensor shapes (App. D), against exact ALS.

The datasets (cardiac MRI 256x256x14x20, hyperspectral 1024x1344x33, COIL-100
7200x120x120x3) are not used: synthetic tensors of those shapes stand in, built as Tucker
tensors of twice the decomposition rank (capped by the mode size) with a core spectrum that
decays as exp(-1.2 r_n / R_n) and 10 % relative noise, so a rank-R decomposition leaves a
tail, as on images. Both algorithms start from the same factors (QR of Gaussians) and core
(X x_m A(m)^T) and run 5 sweeps (the paper's count), lambda = 1e-3, eps = 0.1; the sampled
sweep uses Alg. 3 factor steps and Alg. 2 core steps (the core steps stop by the
(1+eps)-aware rule: on these tensors the FP32 core solve floors near a 1e-5 relative step, above
a 1e-7 tolerance), the exact one the KronMatMul updates.
Every step of the sampled sweep is a (1+eps)-approximate minimiser of its subproblem, so
its RRE may trail the exact one by more than (1+eps) in the first sweep from a random start
(the N+1 steps' slack compounds); from the second sweep on it must stay within (1 + eps),
and after the last within (1 + eps/4) (the paper reports 0.356 vs 0.351 on the cardiac
tensor). The exact RRE never rises."""
import time

import pytest
import torch

import paper_2209_04876_gb300 as kr
from workloads import IMAGE_SHAPES, tucker_tensor_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    kr.lib()


def _init(X, I, R, seed):
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    As = [torch.linalg.qr(torch.randn(i, r, generator=g, device="cuda"))[0].contiguous() for i, r in zip(I, R)]
    G = kr.kron_matmul(As, X.reshape(-1), trans=[1] * len(As))
    return As, G


@pytest.mark.parametrize("name", sorted(IMAGE_SHAPES))
def test_sampled_tucker_tracks_exact_als(name):
    I, R = IMAGE_SHAPES[name]["I"], IMAGE_SHAPES[name]["R"]
    Rt = [min(2 * r, i) for r, i in zip(R, I)]
    X = tucker_tensor_device(I, Rt, seed=31, noise_rel=0.1, decay_rank=R)
    lam, eps, sweeps = 1e-3, 0.1, 5
    out = {}
    for kind in ("exact", "sampled"):
        As, G = _init(X, I, R, seed=32)
        rre = []
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if kind == "exact":
            rre = kr.tucker_als_exact_sweep(X, As, G, lam, sweeps=sweeps)
        else:
            for k in range(sweeps):
                kr.tucker_als_sweep(X, As, G, lam, eps=eps, sweeps=1, seed=5, call_id=100 + k * (len(I) + 1),
                                    tol=1e-7, max_iter=300, stop_rule=kr.STOP_EPS)
                rre.append(kr.tucker_rre(X, As, G))
        torch.cuda.synchronize()
        out[kind] = (rre, (time.perf_counter() - t0) / sweeps)
    (re, te), (rs, ts) = out["exact"], out["sampled"]
    print("%s: exact RRE %s (%.1f ms/sweep), sampled RRE %s (%.1f ms/sweep)" % (
        name, ["%.4f" % v for v in re], 1e3 * te, ["%.4f" % v for v in rs], 1e3 * ts))
    assert all(b <= a * (1 + 1e-4) for a, b in zip(re, re[1:]))
    for k in range(1, sweeps):
        assert rs[k] <= (1 + eps) * re[k], (k, rs[k], re[k])
    assert rs[-1] <= (1 + eps / 4) * re[-1], (rs[-1], re[-1])
    assert 0.0 < re[-1] < 1.0
