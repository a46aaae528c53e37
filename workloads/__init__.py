"""Seeded synthetic inputs shared by the tests, the bench and the oracle runs.

This module only builds inputs (factor matrices, right-hand sides, tensors); it
holds none of the regression method's arithmetic (no leverage scores, sampling,
sampled products, preconditioning or iteration). Random numbers the method itself
draws are not made here: both implementations derive them from (seed, call id).

Recipes (all float64 generation with numpy's PCG64 ``default_rng(seed)``, cast to
float32 for the device):

* ``kron_problem``: N factors I_n x R_n. ``dist='gauss'``: i.i.d. N(0,1);
  ``'lognormal_rows'``: each row scaled by exp(z), z ~ N(0, sigma^2) (skewed leverage);
  ``'outliers'``: Gaussian with a seeded 10% of rows scaled by 20 (high-leverage rows);
  ``'paper_e1'``: entries N(1, 0.001) read as mean 1, standard deviation 0.001 (the reading
  under which the closed-form optimum reproduces the paper's printed OPT values).
  Right-hand side: ``b = K x_true + noise`` with x_true ~ N(0,1)^R, noise Gaussian,
  either absolute (``noise_abs``) or scaled to ``noise_rel * ||K x_true||``; or a
  rank-(r,...,r) Tucker tensor plus relative noise (``b_kind='tucker'``); or all ones.
* ``tucker_tensor``: X = G x_1 Q1 ... x_N QN + noise, G ~ N(0,1)^{R}, Qn orthonormal
  (QR of a Gaussian), noise scaled to ``noise_rel * ||signal||``.
* ``tucker_tensor_device``: the ``tucker_tensor`` recipe generated in float32 on a CUDA device.
* ``IMAGE_SHAPES``: synthetic stand-ins for the paper's image tensors (App. D): the shapes and
  decomposition ranks of the cardiac MRI, hyperspectral and COIL-100 tensors, filled with a
  Tucker tensor of twice the decomposition rank (capped by the mode size) whose core decays
  as exp(-1.2 r_n / R_n) along every mode, plus 10 % noise.
* ``batched_shapes``: per-problem I_n ~ U{lo..hi}, R_n ~ U{rlo..rhi}.
* ``kron_problem_device``: the ``kron_problem`` recipe (b_kind 'kron' or 'tucker', relative
  noise) generated in float32 on a CUDA device with torch's seeded generator, for batches and
  workloads whose right-hand sides (up to 4 GB each) are too slow to build on the host. Same
  recipe, not the same numbers as the numpy generator.
"""
import numpy as np


def _signal_from_core(core, factors):
    """Multiply a dense core by one matrix per mode (builds a structured signal)."""
    T = core
    for n, F in enumerate(factors):
        T = np.moveaxis(np.tensordot(F, T, axes=([1], [n])), 0, n)
    return T


def make_factors(I, R, dist="gauss", seed=0, sigma=1.0, outlier_frac=0.1, outlier_scale=20.0):
    rng = np.random.default_rng(seed)
    As = []
    for In, Rn in zip(I, R):
        if dist == "paper_e1":
            A = rng.normal(1.0, 1e-3, size=(In, Rn))
        else:
            A = rng.standard_normal((In, Rn))
        if dist == "lognormal_rows":
            A = A * np.exp(sigma * rng.standard_normal(In))[:, None]
        elif dist == "outliers":
            k = max(1, int(round(outlier_frac * In)))
            rows = rng.choice(In, size=k, replace=False)
            A[rows] *= outlier_scale
        As.append(A)
    return As


def kron_problem(I, R, dist="gauss", seed=0, noise_abs=None, noise_rel=None, b_kind="kron",
                 tucker_rank=None, sigma=1.0):
    """Returns dict(As=[float64 I_n x R_n], b=float64 (prod I), x_true or None)."""
    I = [int(v) for v in I]
    R = [int(v) for v in R]
    As = make_factors(I, R, dist=dist, seed=seed, sigma=sigma)
    rng = np.random.default_rng(seed + 1000003)
    x_true = None
    if b_kind == "ones":
        b = np.ones(int(np.prod(I)))
    else:
        if b_kind == "kron":
            x_true = rng.standard_normal(int(np.prod(R)))
            sig = _signal_from_core(x_true.reshape(R), As)
        elif b_kind == "tucker":
            r = tucker_rank or R
            core = rng.standard_normal(tuple(r))
            facs = [rng.standard_normal((In, rn)) for In, rn in zip(I, r)]
            sig = _signal_from_core(core, facs)
        else:
            raise ValueError(b_kind)
        sig = sig.reshape(-1)
        noise = rng.standard_normal(sig.shape[0])
        if noise_abs is not None:
            noise *= noise_abs
        elif noise_rel is not None:
            noise *= noise_rel * np.linalg.norm(sig) / np.linalg.norm(noise)
        else:
            noise[:] = 0.0
        b = sig + noise
    return dict(As=As, b=b, x_true=x_true, I=I, R=R)


def kron_problem_device(I, R, dist="gauss", seed=0, noise_rel=0.01, sigma=1.0, device="cuda", b_kind="kron",
                        tucker_rank=None):
    """Returns dict(As=[float32 I_n x R_n on device], b=float32 (prod I) on device, x_true, I, R).
    b_kind 'kron': b = K x_true + noise; 'tucker': b = a rank-(r,...,r) Tucker tensor (Gaussian
    core and factors, independent of the A(n)) + noise, x_true None."""
    import torch

    I = [int(v) for v in I]
    R = [int(v) for v in R]
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    As = []
    for In, Rn in zip(I, R):
        A = torch.randn(In, Rn, generator=g, device=device)
        if dist == "lognormal_rows":
            A *= torch.exp(sigma * torch.randn(In, 1, generator=g, device=device))
        elif dist == "outliers":
            rows = torch.randperm(In, generator=g, device=device)[:max(1, int(round(0.1 * In)))]
            A[rows] *= 20.0
        elif dist != "gauss":
            raise ValueError(dist)
        As.append(A.contiguous())
    if b_kind == "kron":
        x_true = torch.randn(int(np.prod(R)), generator=g, device=device)
        T = x_true.reshape(R)
        facs = As
    elif b_kind == "tucker":
        r = [int(v) for v in (tucker_rank or R)]
        x_true = None
        T = torch.randn(*r, generator=g, device=device)
        facs = [torch.randn(In, rn, generator=g, device=device) for In, rn in zip(I, r)]
    else:
        raise ValueError(b_kind)
    for n, A in enumerate(facs):
        T = torch.movedim(torch.tensordot(A, T, dims=([1], [n])), 0, n)
    b = T.reshape(-1).contiguous()
    del T
    noise = torch.randn(b.numel(), generator=g, device=device)
    noise *= noise_rel * torch.linalg.vector_norm(b) / torch.linalg.vector_norm(noise)
    b += noise
    return dict(As=As, b=b, x_true=x_true, I=I, R=R)


def tucker_tensor(I, R, seed=0, noise_rel=0.01):
    """Synthetic Tucker tensor: Gaussian core, orthonormal factors, relative noise."""
    rng = np.random.default_rng(seed)
    core = rng.standard_normal(tuple(R))
    Qs = []
    for In, Rn in zip(I, R):
        Q, _ = np.linalg.qr(rng.standard_normal((In, Rn)))
        Qs.append(Q)
    X = _signal_from_core(core, Qs)
    noise = rng.standard_normal(X.shape)
    noise *= noise_rel * np.linalg.norm(X) / np.linalg.norm(noise)
    return dict(X=X + noise, core=core, Qs=Qs)


def tucker_tensor_device(I, R, seed=0, noise_rel=0.01, device="cuda", decay_rank=None, decay=1.2):
    """The ``tucker_tensor`` recipe in float32 on a CUDA device with torch's seeded generator
    (Gaussian core, orthonormal factors from the QR of Gaussians, relative noise): for
    tensors of hundreds of millions of entries. Same recipe, not the same numbers. With
    decay_rank, core index r_n is scaled by exp(-decay r_n / decay_rank[n]) (a decaying
    multilinear spectrum, as in images: a rank-decay_rank decomposition leaves a tail)."""
    import torch

    I = [int(v) for v in I]
    R = [int(v) for v in R]
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    T = torch.randn(*R, generator=g, device=device)
    if decay_rank is not None:
        for n, (Rn, Dn) in enumerate(zip(R, decay_rank)):
            w = torch.exp(-decay * torch.arange(Rn, device=device, dtype=torch.float32) / float(Dn))
            shape = [1] * len(R)
            shape[n] = Rn
            T = T * w.reshape(shape)
    for n, (In, Rn) in enumerate(zip(I, R)):
        Q, _ = torch.linalg.qr(torch.randn(In, Rn, generator=g, device=device))
        T = torch.movedim(torch.tensordot(Q, T, dims=([1], [n])), 0, n)
    X = T.contiguous()
    del T
    noise = torch.randn(X.shape, generator=g, device=device)
    noise *= noise_rel * torch.linalg.vector_norm(X) / torch.linalg.vector_norm(noise)
    X += noise
    return X


def tucker_init(I, R, seed=0):
    """Initial factors: Q factor of a seeded Gaussian I_n x R_n per mode."""
    rng = np.random.default_rng(seed)
    return [np.linalg.qr(rng.standard_normal((In, Rn)))[0] for In, Rn in zip(I, R)]


def batched_shapes(nprob=64, N=3, ilo=64, ihi=1024, rlo=4, rhi=32, seed=2209):
    rng = np.random.default_rng(seed)
    I = rng.integers(ilo, ihi + 1, size=(nprob, N))
    R = rng.integers(rlo, rhi + 1, size=(nprob, N))
    return [(list(map(int, i)), list(map(int, r))) for i, r in zip(I, R)]


# Named workloads (sizes of the paper-shaped synthetic configurations).
CONFIGS = {
    "kron_n2_256x16": dict(I=[256, 256], R=[16, 16], dist="gauss", noise_abs=0.01, eps=0.1, lam=0.0),
    "kron_n3_512x32_lognormal": dict(I=[512, 512, 512], R=[32, 32, 32], dist="lognormal_rows",
                                     noise_rel=0.05, eps=0.1, lam=0.0),
    "kron_n3_1024x64_outliers": dict(I=[1024, 1024, 1024], R=[64, 64, 64], dist="outliers",
                                     noise_rel=0.01, eps=0.05, lam=0.0, b_kind="tucker",
                                     tucker_rank=[64, 64, 64]),
}


# Shapes and decomposition ranks of the paper's image tensors (App. D; the datasets are not
# used: synthetic Tucker tensors of these shapes stand in for them).
IMAGE_SHAPES = {
    "cardiac_mri_256x256x14x20": dict(I=[256, 256, 14, 20], R=[8, 8, 4, 4]),
    "hyperspectral_1024x1344x33_r8": dict(I=[1024, 1344, 33], R=[8, 8, 8]),
    "hyperspectral_1024x1344x33_r16": dict(I=[1024, 1344, 33], R=[16, 16, 4]),
    "coil100_7200x120x120x3": dict(I=[7200, 120, 120, 3], R=[16, 4, 4, 2]),
}
