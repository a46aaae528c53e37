"""The oracle's pins catch plausible mistakes (CPU only): each test plants one mistake in a
copy of an oracle step (a swapped factor order, a transposed operand, a shifted prefix, a
dropped factor of the weight, a wrong split of the row key, row norms for leverage scores)
and checks that the independent reference its pin uses (np.kron, a QR factorisation, a
brute-force enumeration, the dense rows of K) rejects the copy while it accepts the oracle."""
import numpy as np

from oracle import kron as ko


def _factors(seed, I=(4, 3, 5), R=(2, 3, 2)):
    rng = np.random.default_rng(seed)
    return [rng.standard_normal((i, r)) for i, r in zip(I, R)]


def _far(a, b, tol=1e-8):
    return np.max(np.abs(np.asarray(a) - np.asarray(b))) > tol * (1.0 + np.max(np.abs(b)))


def test_kron_matvec_factor_order_mistake_is_caught():
    As = _factors(1)
    x = np.random.default_rng(2).standard_normal(2 * 3 * 2)
    ref = ko.kron_dense(As) @ x
    assert not _far(ko.kron_matvec(As, x), ref)

    def reversed_modes(As, x):  # the modes applied in the opposite order
        R = [A.shape[1] for A in As]
        X = np.asarray(x).reshape(R[::-1])
        for n, A in enumerate(As[::-1]):
            X = ko.mode_product(X, A, n)
        return X.reshape(-1)

    y = reversed_modes(As, x)
    assert y.shape != ref.shape or _far(y, ref)


def test_kron_rmatvec_untransposed_factor_is_caught():
    rng = np.random.default_rng(3)
    As = [rng.standard_normal((3, 3)), rng.standard_normal((4, 4))]  # square: the mistake runs
    y = rng.standard_normal(12)
    ref = ko.kron_dense(As).T @ y
    assert not _far(ko.kron_rmatvec(As, y), ref)

    def untransposed(As, y):
        Y = np.asarray(y).reshape([A.shape[0] for A in As])
        for n, A in enumerate(As):
            Y = ko.mode_product(Y, A, n)
        return Y.reshape(-1)

    assert _far(untransposed(As, y), ref)


def test_leverage_from_row_norms_is_caught():
    rng = np.random.default_rng(4)
    A = rng.standard_normal((20, 3)) * np.exp(rng.standard_normal((20, 1)))
    Q, _ = np.linalg.qr(A)
    ref = np.sum(Q * Q, axis=1)
    assert not _far(ko.leverage_scores(A), ref)
    norms = np.sum(A * A, axis=1)
    mutant = norms / norms.sum() * 3  # sums to the rank, like the real scores
    assert abs(mutant.sum() - 3) < 1e-12 and _far(mutant, ref)


def test_shifted_cdf_prefix_is_caught():
    rng = np.random.default_rng(5)
    lev = rng.random(9)
    lev[[2, 6]] = 0.0
    p = lev / lev.sum()
    u = rng.random(4000)

    def brute(cdf_unused, u):  # the definition: i with sum_{k<i} p_k <= u < sum_{k<=i} p_k
        out = np.empty(u.shape[0], dtype=np.int64)
        for j, v in enumerate(u):
            acc = 0.0
            for i, pi in enumerate(p):
                acc += pi
                if v < acc:
                    out[j] = i
                    break
            else:
                out[j] = len(p) - 1
        return out

    ref = brute(None, u)
    good = ko.inverse_cdf(ko.cdf_table(lev), u)
    assert np.mean(good != ref) < 1e-3  # rounding at the boundaries only
    shifted = np.concatenate([[0.0], ko.cdf_table(lev)[:-1]])  # exclusive prefix
    bad = np.minimum(ko.inverse_cdf(shifted, u), len(p) - 1)
    assert np.mean(bad != ref) > 0.3


def test_weights_without_sample_count_are_caught():
    I = [3, 2]
    probs = [np.array([0.5, 0.3, 0.2]), np.array([0.6, 0.4])]
    keys = np.array([0, 3, 5])  # (0,0), (1,1), (2,1)
    counts = np.array([2, 1, 4])
    s = 7
    hand = np.array([2 / (7 * 0.5 * 0.6), 1 / (7 * 0.3 * 0.4), 4 / (7 * 0.2 * 0.4)])
    assert not _far(ko.sample_weights(keys, counts, probs, I, s), hand, 1e-14)
    dropped = ko.sample_weights(keys, counts, probs, I, 1)  # the 1/s factor dropped
    assert _far(dropped, hand, 1e-14)


def test_wrong_key_split_in_sampled_forward_is_caught():
    As = _factors(6, I=(4, 3, 5), R=(2, 2, 3))
    rng = np.random.default_rng(7)
    keys = rng.choice(4 * 3 * 5, size=25, replace=False)
    x = rng.standard_normal(2 * 2 * 3)
    ref = ko.sampled_rows(As, keys) @ x
    assert not _far(ko.sampled_forward(As, keys, x), ref)
    # the row key split by the first mode's size instead of the last one's
    X = np.asarray(x).reshape(2, 2, 3)
    for n in range(2):
        X = ko.mode_product(X, As[n], n)
    Y = X.reshape(-1, 3)
    cell, it = np.divmod(keys, 4)
    ok = (cell < Y.shape[0]) & (it < 5)
    bad = np.einsum("jr,jr->j", Y[np.minimum(cell, Y.shape[0] - 1)], As[2][np.minimum(it, 4)])
    assert _far(bad[ok], ref[ok])
