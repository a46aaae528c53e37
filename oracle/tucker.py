"""FP64 CPU oracle for FastFactorMatrixUpdate (Alg. 3) and TuckerALS (Alg. 1).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Conventions (C-order, as in oracle.kron): the mode-n unfolding X_(n) has rows
indexed by i_n and columns by the remaining indices in C-order (last fastest), so
that X ~ G x_1 A(1) ... x_N A(N) gives X_(n) = A(n) G_(n) K^T with
K = (x)_{m != n} A(m) in increasing m. Row i of a factor update solves
min_y ||K G_(n)^T y - b_i||^2 + lam ||y||^2 (Alg. 1, factor-row step).

Alg. 3 (App. C) substitutes z = G_(n)^T y (Lemma 5.1) and enforces the subspace
constraint with a penalty block sqrt(w) N, N = I - G_(n)^T (G_(n)^T)^+ (Lemma 5.2):
the sketched problem's normal matrix is
  M~ = K~^T K~ + lam G+ (G+)^T + w N,       G = G_(n), G+ = pinv(G)
and Richardson is preconditioned by the unsketched M = K^T K + lam G+(G+)^T + w N,
applied with the Woodbury identity
  M^-1 = A^-1 - A^-1 U (I + V A^-1 U)^-1 V A^-1,  A = K^T K + w I, U = G+,
  V = lam (G+)^T - w G.
The paper prints a '+' before the correction term of this identity; the standard
identity (and the dense inverse of M, checked by a test) has '-'.

Readings: samples are drawn only over the modes m != n (K excludes mode n), with a
fresh sketch per factor row (counter row = i); w = (1 + 12/eps) * prod_{m!=n}
sigma_max(A(m))^2, an upper bound of the paper's ||[K; sqrt(lam)(G^T)^+] N^+||^2
because N^+ = N is an orthogonal projector and (G^T)^+ N = 0. "Until convergence": the
relative step test, or (stop="eps") the eps-aware rule of oracle.kron.richardson on the
penalised objective (row_objective).
"""
import math

import numpy as np

from . import kron as ko


def unfold(X, n):
    """Mode-n unfolding, columns in C-order over the remaining modes."""
    X = np.asarray(X, dtype=np.float64)
    return np.moveaxis(X, n, 0).reshape(X.shape[n], -1)


def fold(M, n, shape):
    shape = list(shape)
    rest = shape[:n] + shape[n + 1:]
    return np.moveaxis(np.asarray(M).reshape([shape[n]] + rest), 0, n)


def reconstruct(G, As):
    X = np.asarray(G, dtype=np.float64)
    for n, A in enumerate(As):
        X = ko.mode_product(X, A, n)
    return X


def rre(X, G, As):
    """Relative reconstruction error ||X^ - X||_F^2 / ||X||_F^2 (App. D)."""
    X = np.asarray(X, dtype=np.float64)
    d = reconstruct(G, As) - X
    return float(np.sum(d * d) / np.sum(X * X))


def tucker_loss(X, G, As, lam):
    """Regularised Tucker loss of §2."""
    X = np.asarray(X, dtype=np.float64)
    d = reconstruct(G, As) - X
    reg = np.sum(np.asarray(G) ** 2) + sum(np.sum(np.asarray(A) ** 2) for A in As)
    return float(np.sum(d * d) + lam * reg)


def penalty_weight(As_other, eps):
    s2 = 1.0
    for A in As_other:
        s2 *= float(np.linalg.norm(np.asarray(A, dtype=np.float64), 2)) ** 2
    return (1.0 + 12.0 / eps) * s2


class WoodburyPreconditioner:
    """M^-1 for M = K^T K + lam G+ (G+)^T + w (I - G+ G), by the Woodbury identity."""

    def __init__(self, As_other, Gn, lam, w):
        self.base = ko.KronPreconditioner(As_other, w)  # (K^T K + w I)^-1
        self.Gn = np.asarray(Gn, dtype=np.float64)
        self.Gp = np.linalg.pinv(self.Gn)  # R_{!=n} x R_n
        self.U = self.Gp
        self.V = lam * self.Gp.T - w * self.Gn  # R_n x R_{!=n}
        AinvU = np.stack([self.base.apply(self.U[:, k]) for k in range(self.U.shape[1])], axis=1)
        self.AinvU = AinvU
        self.C = np.eye(self.Gn.shape[0]) + self.V @ AinvU  # capacitance, R_n x R_n
        self.Cinv = np.linalg.inv(self.C)

    def apply(self, g):
        a = self.base.apply(g)
        return a - self.AinvU @ (self.Cinv @ (self.V @ a))


def dense_penalised_matrix(As_other, Gn, lam, w):
    """M = K^T K + lam G+(G+)^T + w N with N = I - G+ G (tiny sizes)."""
    K = ko.kron_dense(As_other)
    Gp = np.linalg.pinv(np.asarray(Gn, dtype=np.float64))
    Nm = np.eye(Gp.shape[0]) - Gp @ np.asarray(Gn, dtype=np.float64)
    return K.T @ K + lam * Gp @ Gp.T + w * Nm.T @ Nm


def row_sample(As_other, s, seed, call_id, row, cdfs=None, probs=None):
    return ko.draw_sample(As_other, s, seed, call_id, cdfs=cdfs, probs=probs, row=row)


def row_gradient(As_other, Gn, Gp, b_s, sample, z, lam, w):
    """(K~^T K~ + w I) z + lam G+ (G^T)^+ z - w G+ G z - K~^T b~ (Alg. 3 Richardson step)."""
    z = np.asarray(z, dtype=np.float64)
    u = ko.sampled_forward(As_other, sample.keys, z)
    r = sample.omega * (u - b_s)
    g = ko.sampled_transpose(As_other, sample.keys, r)
    g = g + w * z + lam * (Gp @ (Gp.T @ z)) - w * (Gp @ (Gn @ z))
    return g


def row_objective(As_other, Gn, Gp, b_s, sample, z, lam, w):
    """The penalised sketched objective Alg. 3's loop minimises:
    ||S(K z - b)||^2 + lam ||(G^T)^+ z||^2 + w ||N z||^2, N = I - G+ G."""
    z = np.asarray(z, dtype=np.float64)
    r = ko.sampled_forward(As_other, sample.keys, z) - b_s
    Nz = z - Gp @ (Gn @ z)
    return float(np.sum(sample.omega * r * r) + lam * np.sum((Gp.T @ z) ** 2) + w * np.dot(Nz, Nz))


def row_richardson(As_other, Gn, b_s, sample, lam, eps, w, P=None, tol=1e-13, max_iter=2000,
                   step=None, stop="step", theta=0.01):
    """Alg. 3's loop for one row. stop="step": until ||step|| <= tol ||z||. stop="eps": the
    rule of kron.richardson on the penalised objective (its sampled matrix obeys the same
    bounds (1 - sqrt(eps)) M <= M~ <= (1 + sqrt(eps)) M, since M~ - M = K~^T K~ - K^T K and the
    penalty terms of M are positive semidefinite)."""
    Gn = np.asarray(Gn, dtype=np.float64)
    Gp = np.linalg.pinv(Gn)
    if P is None:
        P = WoodburyPreconditioner(As_other, Gn, lam, w)
    alpha = (1.0 - math.sqrt(eps)) if step is None else step
    rho2, c1 = ko.eps_stop_bound(eps)
    z = np.zeros(Gn.shape[1])
    it = 0
    for it in range(1, max_iter + 1):
        g = row_gradient(As_other, Gn, Gp, b_s, sample, z, lam, w)
        pg = P.apply(g)
        if stop == "eps":
            q = float(np.dot(g, pg))
            floor = row_objective(As_other, Gn, Gp, b_s, sample, z, lam, w) - q / c1
        d = alpha * pg
        z = z - d
        if stop == "eps" and rho2 * q / c1 <= theta * eps * max(floor, 0.0):
            break
        if np.linalg.norm(d) <= tol * max(np.linalg.norm(z), 1e-300):
            break
    return z, Gp.T @ z, it  # z, a_i (= (G^T)^+ z = z^T G+), iterations


def row_dense_solve(As_other, Gn, b_s, sample, lam, w):
    """The minimiser of the penalised sketched problem (what Alg. 3's loop converges to)."""
    Gn = np.asarray(Gn, dtype=np.float64)
    Gp = np.linalg.pinv(Gn)
    rows = ko.sampled_rows(As_other, sample.keys)
    Kt = rows * sample.omega[:, None]
    Mt = rows.T @ Kt + lam * Gp @ Gp.T + w * (np.eye(Gp.shape[0]) - Gp @ Gn)
    rhs = Kt.T @ np.asarray(b_s, dtype=np.float64)
    z = np.linalg.solve(Mt, rhs)
    return z, Gp.T @ z


def row_ridge_on_sample(As_other, Gn, b_s, sample, lam):
    """argmin_y ||S(K G^T y - b)||^2 + lam ||y||^2 (y-space, no penalty)."""
    rows = ko.sampled_rows(As_other, sample.keys) @ np.asarray(Gn, dtype=np.float64).T
    w = np.sqrt(sample.omega)
    return ko.qr_solve(rows * w[:, None], w * np.asarray(b_s, dtype=np.float64), lam)


def factor_update_exact(X, As, G, n, lam):
    """Exact factor update of Alg. 1 for all rows at once, by KronMatMul (App. C):
    (G_(n) (K^T K) G_(n)^T + lam I) Y^T = G_(n) K^T X_(n)^T."""
    N = len(As)
    Gn = unfold(G, n)
    others = [As[m] for m in range(N) if m != n]
    grams = [np.asarray(A, dtype=np.float64).T @ np.asarray(A, dtype=np.float64) for A in others]
    KtK = ko.kron_dense(grams)
    H = Gn @ KtK @ Gn.T + lam * np.eye(Gn.shape[0])
    Z = np.asarray(X, dtype=np.float64)
    for m in range(N):
        if m != n:
            Z = ko.mode_product(Z, np.asarray(As[m], dtype=np.float64).T, m)
    Zn = unfold(Z, n)  # I_n x R_{!=n}:  row i = K^T b_i
    rhs = Gn @ Zn.T
    return np.linalg.solve(H, rhs).T


def core_update_exact(X, As, lam):
    """Exact core update of Alg. 1 (closed-form ridge)."""
    R = [A.shape[1] for A in As]
    return ko.closed_form_ridge(As, np.asarray(X, dtype=np.float64).reshape(-1), lam).reshape(R)


def call_id_for(base, sweep, step, N):
    """Sketch call id for sweep k and step n (0..N-1 factor steps, N = core step)."""
    return int(base) + sweep * (N + 1) + step


def fast_factor_matrix_update(X, As, G, n, lam, eps, seed, call_id, c=4.0, s=None, tol=1e-13,
                              max_iter=2000, rows=None, cdfs=None, probs=None):
    """Alg. 3 for mode n. Returns the new A(n) (rows not in ``rows`` are left as is)."""
    N = len(As)
    others = [As[m] for m in range(N) if m != n]
    Rn = [A.shape[1] for A in others]
    Rne = int(np.prod(Rn))
    if s is None:
        s = ko.sample_count(Rne, eps, c)
    Gn = unfold(G, n)
    w = penalty_weight(others, eps)
    P = WoodburyPreconditioner(others, Gn, lam, w)
    if cdfs is None or probs is None:
        levs = [ko.leverage_scores(A) for A in others]
        cdfs = [ko.cdf_table(l) for l in levs]
        probs = [ko.probabilities(l) for l in levs]
    Xn = unfold(X, n)
    Anew = np.array(As[n], dtype=np.float64, copy=True)
    rows = range(Xn.shape[0]) if rows is None else rows
    iters = []
    for i in rows:
        smp = row_sample(others, s, seed, call_id, i, cdfs=cdfs, probs=probs)
        b_s = Xn[i][smp.keys]
        _, a, it = row_richardson(others, Gn, b_s, smp, lam, eps, w, P=P, tol=tol, max_iter=max_iter)
        Anew[i] = a
        iters.append(it)
    return Anew, iters


def tucker_als(X, As0, G0, lam, sweeps, sampled=False, eps=0.1, seed=0, call_id_base=0, c=4.0,
               tol=1e-13, max_iter=2000, history=None):
    """Alg. 1: N factor updates then one core update per sweep (exact or sampled)."""
    As = [np.array(A, dtype=np.float64, copy=True) for A in As0]
    G = np.array(G0, dtype=np.float64, copy=True)
    N = len(As)
    for k in range(sweeps):
        for n in range(N):
            if sampled:
                As[n], _ = fast_factor_matrix_update(
                    X, As, G, n, lam, eps, seed, call_id_for(call_id_base, k, n, N), c=c,
                    tol=tol, max_iter=max_iter)
            else:
                As[n] = factor_update_exact(X, As, G, n, lam)
        if sampled:
            x, _, _ = ko.fast_kronecker_regression(
                As, np.asarray(X).reshape(-1), lam, eps, seed=seed,
                call_id=call_id_for(call_id_base, k, N, N), c=c, tol=tol, max_iter=max_iter)
            G = x.reshape([A.shape[1] for A in As])
        else:
            G = core_update_exact(X, As, lam)
        if history is not None:
            history.append(rre(X, G, As))
    return As, G


def initial_core(X, As):
    """G = X x_1 A(1)^T ... x_N A(N)^T (exact core for orthonormal factors)."""
    G = np.asarray(X, dtype=np.float64)
    for n, A in enumerate(As):
        G = ko.mode_product(G, np.asarray(A, dtype=np.float64).T, n)
    return G
