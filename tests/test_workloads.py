"""The seeded input recipes (CPU): shapes, structure and noise levels as stated."""
import numpy as np
import pytest

from oracle import kron as ko
from workloads import batched_shapes, kron_problem, kron_problem_device


def test_kron_problem_noise_is_relative():
    prob = kron_problem([12, 10, 9], [3, 2, 2], dist="lognormal_rows", seed=5, noise_rel=0.05)
    sig = ko.kron_matvec(prob["As"], prob["x_true"])
    assert abs(np.linalg.norm(prob["b"] - sig) / np.linalg.norm(sig) - 0.05) < 1e-12


@pytest.mark.parametrize("dist", ["gauss", "lognormal_rows", "outliers"])
def test_kron_problem_device_recipe_on_cpu(dist):
    """The device-side generator (run here on torch's CPU device): factor shapes, seeded
    reproducibility, b = K x_true + noise with ||noise|| = 0.01 ||K x_true||, and the
    outlier rows scaled by 20."""
    torch = pytest.importorskip("torch")
    I, R = [9, 8, 7], [3, 2, 2]
    p1 = kron_problem_device(I, R, dist=dist, seed=11, noise_rel=0.01, device="cpu")
    p2 = kron_problem_device(I, R, dist=dist, seed=11, noise_rel=0.01, device="cpu")
    assert [tuple(A.shape) for A in p1["As"]] == [(9, 3), (8, 2), (7, 2)]
    assert torch.equal(p1["b"], p2["b"])
    As = [A.double().numpy() for A in p1["As"]]
    sig = ko.kron_matvec(As, p1["x_true"].double().numpy())
    rel = np.linalg.norm(p1["b"].double().numpy() - sig) / np.linalg.norm(sig)
    assert abs(rel - 0.01) < 1e-4  # float32 generation
    if dist == "outliers":
        norms = np.linalg.norm(As[0], axis=1)
        assert norms.max() > 5 * np.median(norms)


def test_batched_shapes_ranges():
    sh = batched_shapes()
    assert len(sh) == 64
    for I, R in sh:
        assert len(I) == 3 and all(64 <= v <= 1024 for v in I) and all(4 <= v <= 32 for v in R)
