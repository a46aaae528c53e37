"""Comparison helpers of the GPU parity tests (test infrastructure)."""
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
