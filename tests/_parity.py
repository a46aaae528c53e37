"""Comparison helpers of the GPU parity tests (test infrastructure)."""
import multiprocessing
import os

import numpy as np


def worst_component(got, ref):
    """(max_i |got_i - ref_i| / ||ref||_inf, argmax i) in float64."""
    a = np.asarray(got, dtype=np.float64).reshape(-1)
    b = np.asarray(ref, dtype=np.float64).reshape(-1)
    scale = max(float(np.max(np.abs(b))) if b.size else 0.0, 1e-300)
    d = np.abs(a - b)
    i = int(np.argmax(d)) if d.size else 0
    return (float(d[i]) / scale if d.size else 0.0), i


def assert_elementwise(got, ref, tol, what="result"):
    """Every component within tol * ||ref||_inf of the reference; the message names the
    worst component, its value and the reference's."""
    a = np.asarray(got, dtype=np.float64).reshape(-1)
    b = np.asarray(ref, dtype=np.float64).reshape(-1)
    assert a.shape == b.shape, (what, a.shape, b.shape)
    err, i = worst_component(a, b)
    assert err <= tol, "%s: worst component %d: %.9g vs %.9g (%.3e of max|ref|, bar %.1e)" % (
        what, i, a[i], b[i], err, tol)
    return err


def _chunk_multiset(cdfs, t0, n, seed, call_id, I):
    from oracle import kron as ko

    idx = ko.sample_draws(cdfs, n, seed, call_id, t0=t0)
    return ko.group_samples(idx, I)


def oracle_multiset(cdfs, s, seed, call_id, I, chunk=4_000_000, procs=None):
    """The oracle's grouped sample (distinct linear keys, multiplicities) of all s draws,
    drawn in chunks of consecutive draw indices by a pool of spawned processes (the
    multiset does not depend on how the draws are split)."""
    tasks = [(cdfs, t0, min(chunk, s - t0), seed, call_id, I) for t0 in range(0, s, chunk)]
    ctx = multiprocessing.get_context("spawn")
    with ctx.Pool(procs or max(1, min(len(tasks), os.cpu_count() or 1))) as pool:
        parts = pool.starmap(_chunk_multiset, tasks)
    keys = np.concatenate([k for k, _ in parts])
    counts = np.concatenate([c for _, c in parts])
    del parts
    uk, inv = np.unique(keys, return_inverse=True)
    return uk, np.bincount(inv, weights=counts, minlength=uk.shape[0]).astype(np.int64)


U32 = 2.0 ** -24  # unit roundoff of FP32


def solution_bar(As):
    """Element-wise bar of an FP32-path solution against the oracle's sampled minimiser:
    max(1e-5, 4 u32 sqrt(cond(K))) with cond(K) = prod_n cond(A(n)). At the FP32 fixed
    point of the explicit-residual iteration, the rounding of each sampled residual
    (about u32 |b~_j|, independent across rows) reaches x through the sampled system's
    pseudo-inverse; summed with random signs its size relative to x grows like
    sqrt(cond(K)). The bar is 1e-5 for every well-conditioned shape."""
    c = float(np.prod([np.linalg.cond(np.asarray(A, dtype=np.float64)) for A in As]))
    return max(1e-5, 4.0 * U32 * np.sqrt(c))


def precond_bar(As, lam):
    """Bar of the FP32 preconditioner M+ g against the exact one: 1e-5 for lambda = 0
    (FP64 Cholesky inverses rounded to FP32); for lambda > 0 max(1e-5, 2 u32 max_n
    cond(G_n)): the FP32 Jacobi eigenpairs of G_n = A(n)^T A(n) carry absolute errors of
    about u32 ||G_n||, i.e. a relative error u32 cond(G_n) in the smallest eigenvalues, whose
    inverses M+ applies. The preconditioner only has to be a spectral approximation of the
    normal matrix (Lemma 4.2): this rounding changes the rate, not the fixed point."""
    if lam == 0:
        return 1e-5
    c = max(np.linalg.cond(np.asarray(A, dtype=np.float64).T @ np.asarray(A, dtype=np.float64)) for A in As)
    return max(1e-5, 2.0 * U32 * c)
