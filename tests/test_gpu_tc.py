"""KronMatMul (Lemma 4.3) with its contiguous-index mode product on the tcgen05 tensor
cores (3xTF32: TF32 hi/lo operand splits, FP32 accumulation in tensor memory), against the
oracle's FP64 KronMatMul and against the CUDA-core path.

Bar: every component within 1e-5 of the reference's largest component (the FP32 path's bar);
the 3xTF32 product keeps about 21 bits per operand, so its error is a few FP32 units times
the reduction length's square root, like the CUDA-core kernel's. Shapes cover ragged row
counts (not a multiple of the 128-row tile), reduction lengths that are not a multiple of
the 32-float stage, outputs from 1 to 256 columns (one to eight 32-column accumulator
chunks, two to six pipeline stages) and both storage orders of the factor."""
import numpy as np
import pytest
import torch

import paper_2209_04876_gb300 as kr
from _parity import assert_elementwise, worst_component
from oracle import kron as ko

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    kr.lib()
    yield
    kr.set_option(kr.OPT_TENSOR_CORES, 1)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def host(t):
    return t.cpu().numpy()


# (I, R): K^T z with A(n) of I_n x R_n; the last mode's product (I_N -> R_N over rows of
# I_N contiguous floats) qualifies for the tensor cores when prod(I[:-1]) >= 1024
CASES = [
    ([2048, 1024], [32, 64]),
    ([3001, 100], [7, 17]),
    ([1100, 36], [5, 1]),
    ([64, 64, 256], [8, 8, 200]),
    ([32, 64, 512], [4, 4, 256]),
    ([16, 80, 96], [3, 5, 33]),
    ([256, 256, 256], [16, 16, 16]),
]


@pytest.mark.parametrize("I,R", CASES)
def test_kron_rmatvec_tensor_cores(I, R):
    rng = np.random.default_rng(sum(I) + sum(R))
    As = [rng.standard_normal((i, r)).astype(np.float32) for i, r in zip(I, R)]
    z = rng.standard_normal(int(np.prod(I))).astype(np.float32)
    ref = ko.kron_rmatvec([A.astype(np.float64) for A in As], z.astype(np.float64))
    Ad = [dev(A) for A in As]
    zd = dev(z)
    kr.set_option(kr.OPT_TENSOR_CORES, 1)
    n0 = kr.tc_launch_count()
    g_tc = host(kr.kron_matmul(Ad, zd, trans=[1] * len(I)))
    assert kr.tc_launch_count() == n0 + 1, "the tensor-core product did not run"
    kr.set_option(kr.OPT_TENSOR_CORES, 0)
    g_cc = host(kr.kron_matmul(Ad, zd, trans=[1] * len(I)))
    assert kr.tc_launch_count() == n0 + 1
    kr.set_option(kr.OPT_TENSOR_CORES, 1)
    e_tc, e_cc = worst_component(g_tc, ref)[0], worst_component(g_cc, ref)[0]
    print("I=%s R=%s: tensor cores %.3e, CUDA cores %.3e of max|ref|" % (I, R, e_tc, e_cc))
    assert_elementwise(g_tc, ref, 1e-5, "K^T z on tensor cores")
    assert_elementwise(g_cc, ref, 1e-5, "K^T z on CUDA cores")


def test_kron_matmul_untransposed_factor():
    """B(n) stored J_n x I_n (trans 0): the factor's split reads it row by row."""
    rng = np.random.default_rng(5)
    I, J = [1500, 200], [9, 40]
    Bs = [rng.standard_normal((j, i)).astype(np.float32) for i, j in zip(I, J)]
    z = rng.standard_normal(int(np.prod(I))).astype(np.float32)
    ref = ko.kron_matvec([B.astype(np.float64) for B in Bs], z.astype(np.float64))
    n0 = kr.tc_launch_count()
    y = host(kr.kron_matmul([dev(B) for B in Bs], dev(z)))
    assert kr.tc_launch_count() == n0 + 1
    assert_elementwise(y, ref, 1e-5, "K z on tensor cores")


def test_tensor_core_product_extreme_values():
    """Operands spanning many binades, with exact zeros and a row of zeros: each output is
    within 1e-5 of its own sum of absolute terms (the FP32 dot-product bound), so the
    split keeps FP32 accuracy at every scale."""
    rng = np.random.default_rng(6)
    I, R = [2000, 64], [3, 32]
    A0 = rng.standard_normal((I[0], R[0])).astype(np.float32)
    A1 = (rng.standard_normal((I[1], R[1])) * np.exp2(rng.integers(-20, 20, size=(I[1], R[1])))).astype(np.float32)
    A1[5] = 0.0
    A1[7, 3] = 0.0
    z = (rng.standard_normal(int(np.prod(I))) * np.exp2(rng.integers(-10, 10, size=int(np.prod(I))))).astype(
        np.float32)
    A64 = [A0.astype(np.float64), A1.astype(np.float64)]
    ref = ko.kron_rmatvec(A64, z.astype(np.float64))
    mag = ko.kron_rmatvec([np.abs(A) for A in A64], np.abs(z.astype(np.float64)))
    n0 = kr.tc_launch_count()
    g = host(kr.kron_matmul([dev(A0), dev(A1)], dev(z), trans=[1, 1])).astype(np.float64)
    assert kr.tc_launch_count() == n0 + 1
    err = np.abs(g - ref) / np.maximum(mag, 1e-300)
    i = int(np.argmax(err))
    print("worst error over the sum of |terms|: %.3e (output %d)" % (err[i], i))
    assert err[i] <= 1e-5, (i, g[i], ref[i], mag[i])
