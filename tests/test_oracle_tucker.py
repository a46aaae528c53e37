"""Pins for the Alg. 3 / TuckerALS oracle (CPU only)."""
import math

import numpy as np
import pytest

from oracle import kron as ko
from oracle import tucker as tk
from workloads import tucker_init, tucker_tensor


def _setup(seed=0, I=(7, 6, 5), R=(3, 2, 2)):
    rng = np.random.default_rng(seed)
    As = [rng.standard_normal((i, r)) for i, r in zip(I, R)]
    G = rng.standard_normal(R)
    return As, G


def test_unfolding_identity():
    """X_(n) = A(n) G_(n) K^T with K = (x)_{m != n} A(m) in C-order (reading of §2)."""
    As, G = _setup(1)
    X = tk.reconstruct(G, As)
    for n in range(3):
        K = ko.kron_dense([As[m] for m in range(3) if m != n])
        np.testing.assert_allclose(tk.unfold(X, n), As[n] @ tk.unfold(G, n) @ K.T, rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(tk.fold(tk.unfold(X, n), n, X.shape), X)


def test_reconstruct_brute_force_and_kron():
    """X = G x_1 A(1) x_2 A(2) x_3 A(3), entry by entry as the quadruple sum, and as
    (A(1) (x) A(2) (x) A(3)) vec G with np.kron (C-order vec)."""
    As, G = _setup(2, I=(4, 3, 5), R=(2, 3, 2))
    X = tk.reconstruct(G, As)
    for i in range(4):
        for j in range(3):
            for k in range(5):
                v = sum(G[a, b, c] * As[0][i, a] * As[1][j, b] * As[2][k, c]
                        for a in range(2) for b in range(3) for c in range(2))
                assert abs(X[i, j, k] - v) <= 1e-12 * (1 + abs(v))
    K = np.kron(np.kron(As[0], As[1]), As[2])
    np.testing.assert_allclose(X.reshape(-1), K @ G.reshape(-1), rtol=1e-12, atol=1e-12)


def test_rre_and_tucker_loss_closed_forms():
    """RRE = ||X^ - X||^2 / ||X||^2 and the regularised loss ||X^ - X||^2 + lam (||G||^2 +
    sum ||A(n)||^2), on cases whose values are known: an exact decomposition (RRE 0), X twice
    the reconstruction (RRE 1/4), a zero core (RRE 1), and a rank-one 2 x 2 example by hand."""
    As, G = _setup(3)
    Xh = tk.reconstruct(G, As)
    assert tk.rre(Xh, G, As) == pytest.approx(0.0, abs=1e-28)
    assert tk.rre(2.0 * Xh, G, As) == pytest.approx(0.25, rel=1e-12)
    assert tk.rre(Xh, np.zeros_like(G), As) == pytest.approx(1.0, rel=1e-12)
    # X = [[1, 2], [3, 4]], G = [[2]], a = [1, 1], b = [1, 2]: X^ = 2 a b^T = [[2, 4], [2, 4]],
    # X^ - X = [[1, 2], [-1, 0]]: ||.||^2 = 6, ||X||^2 = 30; ||G||^2 + ||a||^2 + ||b||^2 = 4 + 2 + 5
    X = np.array([[1.0, 2.0], [3.0, 4.0]])
    G1 = np.array([[2.0]])
    A1 = [np.array([[1.0], [1.0]]), np.array([[1.0], [2.0]])]
    assert tk.rre(X, G1, A1) == pytest.approx(6.0 / 30.0, rel=1e-14)
    assert tk.tucker_loss(X, G1, A1, 0.5) == pytest.approx(6.0 + 0.5 * 11.0, rel=1e-14)


@pytest.mark.parametrize("lam", [0.0, 0.05])
def test_woodbury_matches_dense_inverse(lam):
    """The Woodbury form with the standard minus sign equals inv(M) (App. C)."""
    As, G = _setup(2)
    for n in range(3):
        others = [As[m] for m in range(3) if m != n]
        Gn = tk.unfold(G, n)
        w = tk.penalty_weight(others, 0.1)
        M = tk.dense_penalised_matrix(others, Gn, lam, w)
        P = tk.WoodburyPreconditioner(others, Gn, lam, w)
        v = np.random.default_rng(3).standard_normal(M.shape[0])
        np.testing.assert_allclose(P.apply(v), np.linalg.solve(M, v), rtol=1e-8, atol=1e-10)
        # the paper's printed '+' sign does not give the inverse
        a = P.base.apply(v)
        plus = a + P.AinvU @ (P.Cinv @ (P.V @ a))
        assert np.linalg.norm(plus - np.linalg.solve(M, v)) > 1e-3 * np.linalg.norm(a)


def test_penalty_weight_bound():
    """w >= (1 + 12/eps) ||[K; sqrt(lam)(G^T)^+] N||_2^2 (Lemma 5.2 via Alg. 3)."""
    As, G = _setup(4)
    lam, eps = 0.3, 0.1
    for n in range(3):
        others = [As[m] for m in range(3) if m != n]
        Gn = tk.unfold(G, n)
        K = ko.kron_dense(others)
        Gp = np.linalg.pinv(Gn)
        Nm = np.eye(Gp.shape[0]) - Gp @ Gn
        big = np.vstack([K, math.sqrt(lam) * Gp.T]) @ Nm
        assert tk.penalty_weight(others, eps) >= (1 + 12 / eps) * np.linalg.norm(big, 2) ** 2 * (1 - 1e-12)
        np.testing.assert_allclose(Gp.T @ Nm, 0, atol=1e-10)


def test_factor_row_richardson_converges_to_dense_solve_and_near_ridge():
    """Alg. 3's loop converges to the penalised sketched minimiser, whose y is a
    (1+eps) solution of the y-space ridge on the same sample (Lemmas 5.1, 5.2)."""
    As, G = _setup(5, I=(9, 8, 7), R=(3, 3, 2))
    X = tk.reconstruct(G, As) + 0.05 * np.random.default_rng(6).standard_normal((9, 8, 7))
    lam, eps = 0.01, 0.1
    n = 1
    others = [As[m] for m in range(3) if m != n]
    Gn = tk.unfold(G, n)
    w = tk.penalty_weight(others, eps)
    Xn = tk.unfold(X, n)
    for i in range(3):
        smp = tk.row_sample(others, 400, seed=7, call_id=9, row=i)
        b_s = Xn[i][smp.keys]
        z, a, it = tk.row_richardson(others, Gn, b_s, smp, lam, eps, w, tol=1e-14)
        zd, ad = tk.row_dense_solve(others, Gn, b_s, smp, lam, w)
        np.testing.assert_allclose(a, ad, rtol=1e-8, atol=1e-10)
        y = tk.row_ridge_on_sample(others, Gn, b_s, smp, lam)
        rows = ko.sampled_rows(others, smp.keys) @ Gn.T

        def f(v):
            r = rows @ v - b_s
            return float(np.sum(smp.omega * r * r) + lam * v @ v)

        assert f(y) <= f(ad) <= (1 + eps) * f(y)


def test_exact_factor_update_matches_per_row_lstsq():
    As, G = _setup(8)
    X = tk.reconstruct(G, As) + 0.1 * np.random.default_rng(9).standard_normal((7, 6, 5))
    lam = 0.02
    for n in range(3):
        K = ko.kron_dense([As[m] for m in range(3) if m != n])
        KG = K @ tk.unfold(G, n).T
        Xn = tk.unfold(X, n)
        A_new = tk.factor_update_exact(X, As, G, n, lam)
        for i in range(X.shape[n]):
            ref = np.linalg.lstsq(np.vstack([KG, math.sqrt(lam) * np.eye(KG.shape[1])]),
                                  np.concatenate([Xn[i], np.zeros(KG.shape[1])]), rcond=None)[0]
            np.testing.assert_allclose(A_new[i], ref, rtol=1e-9, atol=1e-11)


def test_exact_als_monotone_and_reaches_noise_floor():
    """Exact ALS never increases the regularised loss; on a Tucker tensor with 1%
    relative noise the RRE settles at about the noise energy (1e-4)."""
    data = tucker_tensor([20, 18, 16], [3, 3, 2], seed=10, noise_rel=0.01)
    X = data["X"]
    As = tucker_init([20, 18, 16], [3, 3, 2], seed=11)
    G = tk.initial_core(X, As)
    lam = 1e-6
    prev = tk.tucker_loss(X, G, As, lam)
    for k in range(8):
        for n in range(3):
            As[n] = tk.factor_update_exact(X, As, G, n, lam)
            cur = tk.tucker_loss(X, G, As, lam)
            assert cur <= prev * (1 + 1e-10)
            prev = cur
        G = tk.core_update_exact(X, As, lam)
        cur = tk.tucker_loss(X, G, As, lam)
        assert cur <= prev * (1 + 1e-10)
        prev = cur
    r = tk.rre(X, G, As)
    assert 0.5e-4 < r < 1.5e-4


def test_sampled_factor_step_is_one_plus_eps_per_row():
    """Thm 5.3: each sampled factor-row update is a (1+eps) solution of that row's
    ridge problem (same state for both), on at least 90% of rows."""
    data = tucker_tensor([16, 14, 12], [2, 2, 2], seed=12, noise_rel=0.01)
    X = data["X"]
    As = tucker_init([16, 14, 12], [2, 2, 2], seed=13)
    G = tk.initial_core(X, As)
    lam, eps = 1e-3, 0.1
    for n in range(3):
        Aex = tk.factor_update_exact(X, As, G, n, lam)
        Asm, _ = tk.fast_factor_matrix_update(X, As, G, n, lam, eps, 5, n, tol=1e-12)
        K = ko.kron_dense([As[m] for m in range(3) if m != n])
        KG = K @ tk.unfold(G, n).T
        Xn = tk.unfold(X, n)

        def f(v, i):
            r = KG @ v - Xn[i]
            return r @ r + lam * v @ v

        ok = sum(f(Asm[i], i) <= (1 + eps) * f(Aex[i], i) for i in range(X.shape[n]))
        assert ok >= 0.9 * X.shape[n]


def test_sampled_als_reaches_exact_als_quality():
    data = tucker_tensor([16, 14, 12], [2, 2, 2], seed=12, noise_rel=0.01)
    X = data["X"]
    As0 = tucker_init([16, 14, 12], [2, 2, 2], seed=13)
    G0 = tk.initial_core(X, As0)
    he, hs = [], []
    tk.tucker_als(X, As0, G0, 1e-3, 4, sampled=False, history=he)
    tk.tucker_als(X, As0, G0, 1e-3, 4, sampled=True, eps=0.1, seed=5, history=hs, tol=1e-12)
    # every sweep takes a (1+eps) factor step and a (1+eps) core step, so the sampled
    # fixed point is within about (1+eps)^2 of the exact one in reconstruction error
    assert hs[-1] <= (1 + 2 * 0.1) * he[-1]
    assert hs[-1] < 2e-4  # at the 1e-4 noise floor


def test_factor_row_richardson_rate_with_large_penalty_needs_exact_eigenvectors():
    """With factors far from orthonormal the penalty w = (1 + 12/eps) prod sigma_max^2 reaches
    ~1e10 and dwarfs the smallest eigenvalues of K^T K (~1). With the exact (FP64)
    eigen-decomposition in the Woodbury base, Alg. 3's Richardson still contracts at the
    Lemma 4.2 rate (about 24 iterations to 1e-10). An orthogonality error of 1e-5 in the
    eigenvectors perturbs K^T K by about w * 1e-5 and costs more than five times as many
    iterations: the reason the GPU factor step keeps its Woodbury chain in FP64."""
    rng = np.random.default_rng(21)
    I, R = (24, 20, 18), (4, 4, 3)
    As = []
    for i, r in zip(I, R):
        Q, _ = np.linalg.qr(rng.standard_normal((i, r)))
        As.append(Q @ np.diag(np.geomspace(100.0, 1.0, r)))
    G = rng.standard_normal(R)
    X = tk.reconstruct(G, As) + 0.01 * rng.standard_normal(I)
    lam, eps, n = 1e-3, 0.1, 0
    others = [As[m] for m in range(3) if m != n]
    Gn = tk.unfold(G, n)
    w = tk.penalty_weight(others, eps)
    assert w > 1e10
    s = ko.sample_count(int(np.prod([A.shape[1] for A in others])), eps)
    smp = tk.row_sample(others, s, seed=3, call_id=5, row=0)
    b_s = tk.unfold(X, n)[0][smp.keys]
    _, a, it_exact = tk.row_richardson(others, Gn, b_s, smp, lam, eps, w, tol=1e-10, max_iter=200)
    assert it_exact <= 30
    _, ad = tk.row_dense_solve(others, Gn, b_s, smp, lam, w)
    np.testing.assert_allclose(a, ad, rtol=1e-6, atol=1e-9)

    P = tk.WoodburyPreconditioner(others, Gn, lam, w)
    r2 = np.random.default_rng(0)
    P.base.V = [V + 1e-5 * r2.standard_normal(V.shape) for V in P.base.V]
    # rebuild the pieces that depend on the base inverse
    P.AinvU = np.stack([P.base.apply(P.U[:, k]) for k in range(P.U.shape[1])], axis=1)
    P.C = np.eye(Gn.shape[0]) + P.V @ P.AinvU
    P.Cinv = np.linalg.inv(P.C)
    with np.errstate(over="ignore", invalid="ignore"):
        _, _, it_pert = tk.row_richardson(others, Gn, b_s, smp, lam, eps, w, P=P, tol=1e-10, max_iter=200)
    assert it_pert > 5 * it_exact


@pytest.mark.parametrize("I,R,n", [((9, 8, 7), (3, 3, 2), 1), ((7, 6, 5, 4), (2, 2, 2, 2), 0)])
def test_factor_row_eps_stopping_rule(I, R, n):
    """The eps-aware rule on Alg. 3's penalised system: the sample's M^-1 M~ spectrum lies in
    [1 - sqrt(eps), 1 + sqrt(eps)], the excess bound holds after every step, and the rule
    stops after a handful of steps with a row that is still a (1+eps) solution of the
    y-space ridge on the same sample (Lemma 5.2); with two and with three other modes."""
    As, G = _setup(5, I=I, R=R)
    X = tk.reconstruct(G, As) + 0.05 * np.random.default_rng(6).standard_normal(I)
    lam, eps = 0.01, 0.1
    N = len(I)
    others = [As[m] for m in range(N) if m != n]
    Gn = tk.unfold(G, n)
    Gp = np.linalg.pinv(Gn)
    w = tk.penalty_weight(others, eps)
    Xn = tk.unfold(X, n)
    M = tk.dense_penalised_matrix(others, Gn, lam, w)
    P = tk.WoodburyPreconditioner(others, Gn, lam, w)
    rho2, c1 = ko.eps_stop_bound(eps)
    for i in range(3):
        smp = tk.row_sample(others, ko.sample_count(int(np.prod([A.shape[1] for A in others])), eps), seed=7,
                            call_id=9, row=i)
        b_s = Xn[i][smp.keys]
        rows = ko.sampled_rows(others, smp.keys)
        Mt = M - ko.kron_dense(others).T @ ko.kron_dense(others) + rows.T @ (smp.omega[:, None] * rows)
        ev = np.linalg.eigvals(np.linalg.solve(M, Mt)).real
        assert 1 - math.sqrt(eps) <= ev.min() and ev.max() <= 1 + math.sqrt(eps)
        zs, _ = tk.row_dense_solve(others, Gn, b_s, smp, lam, w)
        fstar = tk.row_objective(others, Gn, Gp, b_s, smp, zs, lam, w)
        z = np.zeros(Gn.shape[1])
        for _ in range(8):
            g = tk.row_gradient(others, Gn, Gp, b_s, smp, z, lam, w)
            q = float(g @ P.apply(g))
            z_next = z - (1 - math.sqrt(eps)) * P.apply(g)
            # the gradient is that of half the objective: excess(z) = (z - z*)^T M~ (z - z*)
            assert tk.row_objective(others, Gn, Gp, b_s, smp, z_next, lam, w) - fstar <= rho2 * q / c1 * (1 + 1e-9)
            z = z_next
        _, a, it = tk.row_richardson(others, Gn, b_s, smp, lam, eps, w, stop="eps")
        _, _, it_full = tk.row_richardson(others, Gn, b_s, smp, lam, eps, w, tol=1e-14)
        assert it <= 12 and it < it_full
        y = tk.row_ridge_on_sample(others, Gn, b_s, smp, lam)
        Y = rows @ Gn.T

        def f(v):
            r = Y @ v - b_s
            return float(np.sum(smp.omega * r * r) + lam * v @ v)

        assert f(a) <= (1 + eps) * f(y)
