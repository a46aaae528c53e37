"""FP64 CPU oracle for FastKroneckerRegression (Alg. 2) and its building blocks.

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import this module; the library never does.

Everything is plain NumPy in float64, written from the paper's definitions:

* vec / linearisation order: C-order (last index fastest). Row (i1..iN) of
  K = A(1) (x) ... (x) A(N) is b[((i1*I2 + i2)*I3 + ...)]; the unknown x is indexed
  the same way over (r1..rN). This is the only order under which K = A(1)(x)...(x)A(N)
  pairs with vec(X) in Alg. 1 (core update), and it is ``np.kron``'s convention.
* Leverage scores: eq. (ridge leverage via SVD) in §3, with lambda = 0 for the
  sampling distribution (Alg. 2 samples by statistical scores; the ridge scores of K
  do not factor, Lemma 4.1).
* Product distribution and SampleRows: Def. of leverage score sampling (§3),
  Lemma 4.1, proof of Thm 4.5 (one CDF per factor, coordinates drawn independently).
* Richardson: Lemma 4.2 and Alg. 2 (step 1 - sqrt(eps), preconditioner
  M+ = (V1 (x)...(x) VN) D (V1 (x)...(x) VN)^T with D = (S1^2 (x)...(x) SN^2 + lambda I)^+).

Readings where the paper is silent (all mirrored by the CUDA path):
* CDF: cdf[i] = fl(prefix_i / total) with a left-to-right float64 prefix sum; every
  entry from the last positive-mass row on is set to exactly 1.0; a uniform u selects
  the smallest i with u < cdf[i] (zero-mass rows are never chosen).
* Sample count s = ceil(c * R * ln(R) / eps) (the experiments' scaled form of Alg. 2's
  s), at least 1.
* Duplicated draws are merged: a row drawn c times gets weight omega = c / (s p), which
  gives the same sketched objective as c separate rows of weight 1/(s p).
* Convergence: stop when ||step|| <= tol * ||x||; or (stop="eps") once the Lemma 4.2 bound
  on the sampled objective's remaining excess falls below theta * eps of its minimum
  (eps_stop_bound; the O(log 1/eps) iterations of the proof of Thm 4.5).
"""
import math

import numpy as np

from .philox import draw_uniforms

# ----------------------------------------------------------------------------
# Kronecker products and mode products (§2 n-mode product, Lemma 4.3 KronMatMul)
# ----------------------------------------------------------------------------


def kron_dense(As):
    """Materialise K = A(1) (x) ... (x) A(N) (tiny sizes only)."""
    K = np.ones((1, 1))
    for A in As:
        K = np.kron(K, np.asarray(A, dtype=np.float64))
    return K


def mode_product(X, A, n):
    """n-mode product X x_n A: multiplies every mode-n fiber of X by A (A is J x I_n)."""
    Y = np.tensordot(np.asarray(A, dtype=np.float64), X, axes=([1], [n]))  # J, rest...
    return np.moveaxis(Y, 0, n)


def kron_matvec(As, x):
    """(A(1) (x) ... (x) A(N)) x via N mode products (KronMatMul, Lemma 4.3)."""
    R = [A.shape[1] for A in As]
    X = np.asarray(x, dtype=np.float64).reshape(R)
    for n, A in enumerate(As):
        X = mode_product(X, A, n)
    return X.reshape(-1)


def kron_rmatvec(As, y):
    """(A(1) (x) ... (x) A(N))^T y via N mode products with the transposed factors."""
    I = [A.shape[0] for A in As]
    Y = np.asarray(y, dtype=np.float64).reshape(I)
    for n, A in enumerate(As):
        Y = mode_product(Y, np.asarray(A, dtype=np.float64).T, n)
    return Y.reshape(-1)


# ----------------------------------------------------------------------------
# Leverage scores (§3, Lemma 4.1)
# ----------------------------------------------------------------------------


def numerical_rank(svals, shape):
    """Rank with the usual tolerance max(m, n) * eps64 * sigma_max."""
    if svals.size == 0:
        return 0
    tol = max(shape) * np.finfo(np.float64).eps * svals[0]
    return int(np.sum(svals > tol))


def leverage_scores(A, lam=0.0):
    """lambda-ridge leverage scores sum_k s_k^2/(s_k^2+lam) u_ik^2 from the thin SVD.

    With lam = 0 these are the statistical leverage scores, ||U_i||^2 over the
    rank-r left singular vectors.
    """
    A = np.asarray(A, dtype=np.float64)
    U, S, _ = np.linalg.svd(A, full_matrices=False)
    r = numerical_rank(S, A.shape)
    U, S = U[:, :r], S[:r]
    if lam == 0.0:
        return np.sum(U * U, axis=1)
    f = S * S / (S * S + lam)
    return (U * U) @ f


def jl_signs(R, k, seed, mode):
    """The R x k Rademacher matrix of the JL-approximate scores of factor `mode`: entry (r, j)
    is +1 or -1 by the low bit of word w0 of Philox4x32-10 under key (seed lo, seed hi) at
    counter (r * k + j, 0, mode, 0) (0 -> +1, 1 -> -1)."""
    from .philox import philox4x32_10

    t = np.arange(R * k, dtype=np.uint64)
    w0, _, _, _ = philox4x32_10(t, np.zeros_like(t), np.full_like(t, int(mode)), np.zeros_like(t),
                                int(seed) & 0xFFFFFFFF, (int(seed) >> 32) & 0xFFFFFFFF)
    return np.where((w0 & 1) == 0, 1.0, -1.0).reshape(R, k)


def jl_leverage_scores(A, k, seed, mode):
    """JL-approximate statistical leverage scores (the approximate scores of Alg. 2's first
    steps, App. B's Johnson-Lindenstrauss lemma): l~_i = ||e_i^T A R^-1 Pi||^2 / k with R the
    triangular factor of A (QR with a positive diagonal, i.e. the Cholesky factor of A^T A
    transposed) and Pi = jl_signs(R, k, seed, mode). E[l~_i] = l_i; each is within (1 +- delta)
    of l_i with high probability for k = O(log(I) / delta^2)."""
    A = np.asarray(A, dtype=np.float64)
    Q, Rq = np.linalg.qr(A)
    sgn = np.where(np.diag(Rq) < 0, -1.0, 1.0)
    Q = Q * sgn[None, :]  # the QR with a positive diagonal: A R^-1 = Q
    P = jl_signs(A.shape[1], k, seed, mode)
    Y = Q @ P
    return np.sum(Y * Y, axis=1) / float(k)


def factor_rank(A):
    A = np.asarray(A, dtype=np.float64)
    return numerical_rank(np.linalg.svd(A, compute_uv=False), A.shape)


# ----------------------------------------------------------------------------
# Product distribution and SampleRows (§3 Def., Lemma 4.1, proof of Thm 4.5)
# ----------------------------------------------------------------------------


def cdf_table(lev):
    """Normalised CDF of one factor's leverage distribution (left-to-right prefix)."""
    lev = np.asarray(lev, dtype=np.float64)
    n = lev.shape[0]
    cdf = np.empty(n, dtype=np.float64)
    total = 0.0
    for i in range(n):  # explicit left-to-right accumulation
        total += float(lev[i])
        cdf[i] = total
    T = total
    for i in range(n):
        cdf[i] = cdf[i] / T
    pos = np.nonzero(lev > 0.0)[0]
    if pos.size:
        cdf[pos[-1]:] = 1.0
    return cdf


def probabilities(lev):
    """p_n(i) = l_i / sum_j l_j."""
    lev = np.asarray(lev, dtype=np.float64)
    return lev / np.sum(lev)


def inverse_cdf(cdf, u):
    """Smallest i with u < cdf[i] for each uniform u."""
    return np.searchsorted(np.asarray(cdf, dtype=np.float64), np.asarray(u), side="right")


def sample_draws(cdfs, s, seed, call_id, row=0, t0=0):
    """s i.i.d. draws of a multi-index from the product distribution (SampleRows on K).

    Returns idx of shape (s, L) with L = len(cdfs); coordinate m of draw t uses the
    m-th uniform of draw t (see oracle.philox).
    """
    L = len(cdfs)
    t = np.arange(t0, t0 + s, dtype=np.uint64)
    u = draw_uniforms(seed, call_id, t, L, row=row)
    idx = np.empty((s, L), dtype=np.int64)
    for m in range(L):
        idx[:, m] = inverse_cdf(cdfs[m], u[m])
    return idx


def sample_count(R, eps, c=4.0):
    """s = ceil(c R ln R / eps), at least 1."""
    if R <= 1:
        return 1
    return max(1, int(math.ceil(c * R * math.log(R) / eps)))


def linear_index(idx, I):
    """C-order linear row index of multi-indices idx (s x N)."""
    key = np.zeros(idx.shape[0], dtype=np.int64)
    for n in range(idx.shape[1]):
        key = key * int(I[n]) + idx[:, n]
    return key


def group_samples(idx, I):
    """Distinct sampled rows (sorted by linear index) and their multiplicities."""
    keys = linear_index(idx, I)
    uniq, counts = np.unique(keys, return_counts=True)
    return uniq, counts


def unravel(keys, I):
    return np.stack(np.unravel_index(np.asarray(keys, dtype=np.int64), tuple(int(v) for v in I)), axis=1)


def sample_weights(keys, counts, probs, I, s):
    """omega_j = c_j / (s * prod_n p_n(i_n)): squared SampleRows entries, merged."""
    sub = unravel(keys, I)
    p = np.ones(keys.shape[0], dtype=np.float64)
    for n in range(len(I)):
        p = p * probs[n][sub[:, n]]
    return counts.astype(np.float64) / (float(s) * p)


def sampled_rows(As, keys):
    """Rows of K at the given linear indices: row (i1..iN) = A1[i1] (x) ... (x) AN[iN]."""
    I = [A.shape[0] for A in As]
    sub = unravel(keys, I)
    rows = np.ones((keys.shape[0], 1))
    for n, A in enumerate(As):
        a = np.asarray(A, dtype=np.float64)[sub[:, n]]
        rows = (rows[:, :, None] * a[:, None, :]).reshape(keys.shape[0], -1)
    return rows


# ----------------------------------------------------------------------------
# Sampled products (Thm 4.4): (SK)x and (SK)^T r without materialising K
# ----------------------------------------------------------------------------


def sampled_forward(As, keys, x, chunk=1 << 20):
    """u_j = (Kx)[key_j]. Cells are the first N-1 coordinates, T = {N} (last mode):
    Y = X x_1 A1 ... x_{N-1} A_{N-1} over all cells, then u_j = <A_N[i_N], Y[cell_j]>."""
    N = len(As)
    I = [A.shape[0] for A in As]
    R = [A.shape[1] for A in As]
    X = np.asarray(x, dtype=np.float64).reshape(R)
    for n in range(N - 1):
        X = mode_product(X, As[n], n)
    Y = X.reshape(-1, R[-1])  # cells x R_N
    AT = np.asarray(As[-1], dtype=np.float64)
    keys = np.asarray(keys, dtype=np.int64)
    u = np.empty(keys.shape[0], dtype=np.float64)
    for a in range(0, keys.shape[0], chunk):
        k = keys[a:a + chunk]
        cell, it = np.divmod(k, I[-1])
        u[a:a + chunk] = np.einsum("jr,jr->j", Y[cell], AT[it])
    return u


def sampled_transpose(As, keys, r):
    """K^T restricted to the sampled rows applied to r: sum_j r_j K[key_j, :].

    With the rows split as in Thm 4.4 (cells = the first N-1 coordinates, T = {N}):
    W[cell, :] = sum_{j in cell} r_j A_N[i_N(j), :], i.e. W = S A_N for the sparse
    cells x I_N matrix S holding r_j at (cell_j, i_N(j)) (a library sparse-dense
    product), then W x_1 A_1^T ... x_{N-1} A_{N-1}^T."""
    import scipy.sparse as sp

    N = len(As)
    I = [A.shape[0] for A in As]
    R = [A.shape[1] for A in As]
    ncell = int(np.prod(I[:-1])) if N > 1 else 1
    AT = np.asarray(As[-1], dtype=np.float64)
    keys = np.asarray(keys, dtype=np.int64)
    r = np.asarray(r, dtype=np.float64)
    cell, it = np.divmod(keys, I[-1])
    S = sp.csr_matrix((r, (cell, it)), shape=(ncell, I[-1]))
    W = np.asarray(S @ AT)
    G = W.reshape(list(I[:-1]) + [R[-1]])
    for n in range(N - 1):
        G = mode_product(G, np.asarray(As[n], dtype=np.float64).T, n)
    return G.reshape(-1)


# ----------------------------------------------------------------------------
# Preconditioner (Alg. 2, lines building D and M+; square KronMatMul theorem, App. B)
# ----------------------------------------------------------------------------


class KronPreconditioner:
    """M+ = (V1 (x) ... (x) VN) D (V1 (x) ... (x) VN)^T, D = (S1^2 (x)...(x) SN^2 + lam I)^+,
    from the eigen-decompositions of the factor Gram matrices A(n)^T A(n) = Vn Sn^2 Vn^T."""

    def __init__(self, As, lam):
        self.V = []
        self.sig2 = []
        for A in As:
            A = np.asarray(A, dtype=np.float64)
            w, V = np.linalg.eigh(A.T @ A)
            self.V.append(V)
            self.sig2.append(np.maximum(w, 0.0))
        d = np.ones(1)
        for s2 in self.sig2:
            d = np.kron(d, s2)
        d = d + lam
        with np.errstate(divide="ignore"):
            self.D = np.where(d > 0, 1.0 / np.where(d > 0, d, 1.0), 0.0)
        self.R = [A.shape[1] for A in As]

    def apply(self, g):
        X = np.asarray(g, dtype=np.float64).reshape(self.R)
        for n, V in enumerate(self.V):
            X = mode_product(X, V.T, n)
        X = X * self.D.reshape(self.R)
        for n, V in enumerate(self.V):
            X = mode_product(X, V, n)
        return X.reshape(-1)

    def dense(self):
        V = kron_dense(self.V)
        return V @ np.diag(self.D) @ V.T


# ----------------------------------------------------------------------------
# Alg. 2 FastKroneckerRegression, restated step by step
# ----------------------------------------------------------------------------


class Sample:
    """The sketch S of Alg. 2: distinct sampled rows, multiplicities, weights."""

    def __init__(self, keys, counts, omega, s):
        self.keys = keys
        self.counts = counts
        self.omega = omega
        self.s = s


def draw_sample(As, s, seed, call_id, cdfs=None, probs=None, row=0):
    """Leverage scores -> CDFs -> s draws -> grouped sample with weights."""
    I = [A.shape[0] for A in As]
    if cdfs is None or probs is None:
        levs = [leverage_scores(A) for A in As]
        cdfs = [cdf_table(l) for l in levs]
        probs = [probabilities(l) for l in levs]
    idx = sample_draws(cdfs, s, seed, call_id, row=row)
    keys, counts = group_samples(idx, I)
    omega = sample_weights(keys, counts, probs, I, s)
    return Sample(keys, counts, omega, s)


def sampled_gradient(As, b_s, sample, x, lam):
    """K~^T K~ x + lam x - K~^T b~ = sum_j omega_j (u_j - b~_j) K[key_j,:] + lam x."""
    u = sampled_forward(As, sample.keys, x)
    r = sample.omega * (u - b_s)
    return sampled_transpose(As, sample.keys, r) + lam * np.asarray(x, dtype=np.float64)


def sampled_objective(As, b_s, sample, x, lam):
    """||S(Kx - b)||^2 + lam ||x||^2 on the (merged) sample."""
    u = sampled_forward(As, sample.keys, x)
    x = np.asarray(x, dtype=np.float64)
    return float(np.sum(sample.omega * (u - b_s) ** 2) + lam * np.dot(x, x))


def eps_stop_bound(eps):
    """Constants of the eps-aware stopping rule of `richardson` (reading of "until convergence").

    The proof of Thm 4.5 gives (1 - sqrt(eps)) M <= H <= (1 + sqrt(eps)) M for the sampled
    normal matrix H = K~^T K~ + lam I and the preconditioner's M = K^T K + lam I (exact Gram,
    beta = 1). With the step alpha = 1 - sqrt(eps), the eigenvalues of I - alpha M+ H lie in
    [eps, 2 sqrt(eps) - eps], so the excess e(x) = f~(x) - min f~ contracts by
    rho^2 = (2 sqrt(eps) - eps)^2 per step (Lemma 4.2), and the gradient g at x bounds it:
    g^T M+ g >= (1 - sqrt(eps)) e(x). Returns (rho^2, 1 - sqrt(eps))."""
    se = math.sqrt(eps)
    return (2.0 * se - eps) ** 2, 1.0 - se


def richardson(As, b_s, sample, lam, eps, tol=1e-13, max_iter=2000, step=None, x0=None,
               history=None, stop="step", theta=0.01):
    """Alg. 2 Richardson loop: x <- x - (1 - sqrt(eps)) M+ (K~^T K~ x + lam x - K~^T b~).

    stop="step": until ||step|| <= tol ||x||. stop="eps": until the bound on the sampled
    objective's excess after the step, rho^2 g^T M+ g / (1 - sqrt(eps)) (eps_stop_bound), is at
    most theta * eps times the lower bound f~(x) - g^T M+ g / (1 - sqrt(eps)) of its minimum; the
    relative-step test stays in force there too, so a problem whose sampled minimum is zero
    (where that lower bound never turns positive) still stops."""
    R = int(np.prod([A.shape[1] for A in As]))
    P = KronPreconditioner(As, lam)
    alpha = (1.0 - math.sqrt(eps)) if step is None else step
    rho2, c1 = eps_stop_bound(eps)
    x = np.zeros(R) if x0 is None else np.array(x0, dtype=np.float64)
    it = 0
    for it in range(1, max_iter + 1):
        g = sampled_gradient(As, b_s, sample, x, lam)
        pg = P.apply(g)
        if stop == "eps":
            q = float(np.dot(g, pg))
            floor = sampled_objective(As, b_s, sample, x, lam) - q / c1
        d = alpha * pg
        x = x - d
        if history is not None:
            history.append(x.copy())
        if stop == "eps" and rho2 * q / c1 <= theta * eps * max(floor, 0.0):
            break
        if np.linalg.norm(d) <= tol * max(np.linalg.norm(x), 1e-300):
            break
    return x, it


def fast_kronecker_regression(As, b, lam, eps, s=None, seed=0, call_id=0, c=4.0,
                              tol=1e-13, max_iter=2000, cdfs=None, probs=None):
    """Alg. 2 end to end (exact Gram and exact leverage scores, i.e. beta = 1)."""
    R = int(np.prod([A.shape[1] for A in As]))
    if s is None:
        s = sample_count(R, eps, c)
    sample = draw_sample(As, s, seed, call_id, cdfs=cdfs, probs=probs)
    b_s = np.asarray(b, dtype=np.float64)[sample.keys]
    x, it = richardson(As, b_s, sample, lam, eps, tol=tol, max_iter=max_iter)
    return x, sample, it


# ----------------------------------------------------------------------------
# Exact references: closed forms and dense QR (tiny sizes)
# ----------------------------------------------------------------------------


def objective(As, b, x, lam):
    """f(x) = ||Kx - b||^2 + lam ||x||^2 (full, unsampled)."""
    r = kron_matvec(As, x) - np.asarray(b, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    return float(np.dot(r, r) + lam * np.dot(x, x))


def closed_form_ls(As, b):
    """x* = (A(1)^+ (x) ... (x) A(N)^+) b (lambda = 0, full column rank)."""
    return kron_matvec([np.linalg.pinv(np.asarray(A, dtype=np.float64)) for A in As], b)


def closed_form_ridge(As, b, lam):
    """x*_lam = (V1(x)..VN) (S^2 + lam I)^-1 (S1(x)..SN) (U1(x)..UN)^T b from thin SVDs
    (the factorisation used in the proof of Lemma 4.1)."""
    if lam == 0.0:
        return closed_form_ls(As, b)
    Us, Ss, Vs = [], [], []
    for A in As:
        U, S, Vt = np.linalg.svd(np.asarray(A, dtype=np.float64), full_matrices=False)
        Us.append(U)
        Ss.append(S)
        Vs.append(Vt.T)
    c = kron_rmatvec(Us, b)  # (U1 (x) ... (x) UN)^T b
    sig = np.ones(1)
    for S in Ss:
        sig = np.kron(sig, S)
    c = c * sig / (sig * sig + lam)
    return kron_matvec(Vs, c)


def qr_solve(M, y, lam=0.0):
    """argmin ||Mx - y||^2 + lam ||x||^2 by Householder QR of [M; sqrt(lam) I]."""
    M = np.asarray(M, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    if lam > 0:
        M = np.vstack([M, math.sqrt(lam) * np.eye(M.shape[1])])
        y = np.concatenate([y, np.zeros(M.shape[1])])
    Q, Rm = np.linalg.qr(M)
    return np.linalg.solve(Rm, Q.T @ y)


def sampled_exact_solve(As, b_s, sample, lam):
    """x~* = argmin ||S(Kx - b)||^2 + lam ||x||^2 by dense QR of [sqrt(omega) K_S; sqrt(lam) I]."""
    rows = sampled_rows(As, sample.keys)
    w = np.sqrt(sample.omega)
    return qr_solve(rows * w[:, None], w * np.asarray(b_s, dtype=np.float64), lam)
