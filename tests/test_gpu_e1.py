"""The paper's synthetic experiment E1 (§6 and App. D) run through the library.

A(1), A(2) in R^{n x d} with entries N(1, 0.001) (0.001 read as the standard deviation: the
reading under which the closed-form optimum reproduces the printed OPT values), b = 1,
lambda = 1e-3, eps = 0.1, delta = 0.01, and the theory sample count of Alg. 2,
1680 R ln(40 R) ln(1/delta) / eps, scaled by the experiments' alpha = 1e-5. The printed
losses (Table 4 for d = 8..64, Table 2 for d = 64 up to n = 16,384; golden files in
tests/golden/) are context from the paper's machine and its random draws, so the checks are
loose: the optimum within 20 % of the printed OPT (mean over 3 seeds), and the library's
loss ratio f(x) / OPT at least 1 and at most the printed Alg. 2 ratio plus 0.05.

The factors are nearly rank one (cond(A(n)^T A(n)) near 1e8), so the FP32 gradient's rounding
leaves Richardson on a floor far above a 1e-7 relative step; the solves use the
(1+eps)-aware stopping rule, which is what the experiment measures. Where the oracle finishes
quickly (n <= 1024), the oracle's solve of the same sampled problem with the same rule is the
reference: the library's loss within 0.1 eps OPT of the oracle's."""
import math
import os

import numpy as np
import pytest
import torch

import paper_2209_04876_gb300 as kr
from oracle import kron as ko

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def _golden(name):
    rows = []
    with open(os.path.join(HERE, "golden", name)) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                d, n, opt, alg2 = line.split()
                rows.append((int(d), int(n), float(opt), float(alg2)))
    return rows


# At d = 64, n = 16,384 the minimiser is large along the factors' weak directions
# (||K|| ||x|| / ||Kx|| near 740) while the residuals are about 1.7e-4 of b: the FP32 sampled
# products round u_j = (Kx)_j by about as much as the residual itself, and the FP32 path does
# not converge (the FP64 oracle does, on the same sample). Kept as a strict expected failure.
FP32_OUT_OF_RANGE = {(64, 16384)}
ROWS = [pytest.param(*r, marks=pytest.mark.xfail(strict=True, raises=kr.KronError,
                                                  reason="FP32 sampled products lose the residual to cancellation"))
        if (r[0], r[1]) in FP32_OUT_OF_RANGE else r
        for r in _golden("e1_table4.txt") + _golden("e1_table2.txt")]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    kr.lib()


def e1_samples(d, eps=0.1, delta=0.01, alpha=1e-5):
    R = d * d
    return int(math.ceil(alpha * math.ceil(1680 * R * math.log(40 * R) * math.log(1 / delta) / eps)))


@pytest.mark.parametrize("d,n,opt_paper,alg2_paper", ROWS)
def test_e1_losses_through_the_library(d, n, opt_paper, alg2_paper):
    lam, eps = 1e-3, 0.1
    s = e1_samples(d)
    opts, ratios = [], []
    for seed in range(3):
        rng = np.random.default_rng(seed)
        As = [rng.normal(1.0, 1e-3, size=(n, d)).astype(np.float32).astype(np.float64) for _ in range(2)]
        As_d = [torch.tensor(A, dtype=torch.float32, device="cuda") for A in As]
        b_d = torch.ones(n * n, dtype=torch.float32, device="cuda")
        x, rep = kr.kron_ridge(As_d, b_d, lam, eps=eps, seed=seed, call_id=1, num_samples=s,
                               stop_rule=kr.STOP_EPS, max_iter=300)
        assert rep["s"] == s and rep["stop"] in (1, 3), rep
        loss = kr.kron_objective(As_d, b_d, x, lam)
        b64 = np.ones(n * n)
        opt = ko.objective(As, b64, ko.closed_form_ridge(As, b64, lam), lam)
        opts.append(opt)
        ratios.append(loss / opt)
        if n <= 1024:
            tab = kr.kron_leverage(As_d)
            smp = ko.draw_sample(As, s, seed, 1, cdfs=[c.cpu().numpy() for c in tab["cdf"]],
                                 probs=[p.cpu().numpy() for p in tab["prob"]])
            assert smp.keys.shape[0] == rep["distinct"]
            xo, _ = ko.richardson(As, b64[smp.keys], smp, lam, eps, stop="eps", tol=1e-13, max_iter=2000)
            loss_o = ko.objective(As, b64, xo, lam)
            assert abs(loss - loss_o) <= 0.1 * eps * opt, (d, n, seed, loss / opt, loss_o / opt)
        del b_d
    print("E1 d=%d n=%d: OPT %.4g (paper %.4g), loss/OPT %.4f (paper %.4f)" % (
        d, n, np.mean(opts), opt_paper, np.mean(ratios), alg2_paper / opt_paper))
    assert abs(np.mean(opts) / opt_paper - 1) < 0.2
    assert 1.0 - 1e-9 <= min(ratios) and np.mean(ratios) <= alg2_paper / opt_paper + 0.05
