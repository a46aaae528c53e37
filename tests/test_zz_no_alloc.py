"""The allocation-free sampling entry point against the allocating one.

kron_sample_noalloc exists for callers that may not allocate device memory (a
memory manager owns the whole GPU, or cudaMalloc's synchronisation is not
acceptable on their path). Its draws must be exactly those of kron_sample: the same
indices bit for bit and the same weights within the sampler tests' 2e-7 relative
tolerance. Two calls in a row with different tables check that the shared static
scratch is rewritten by each call. This file is collected last on purpose.
"""
import numpy as np
import pytest
import torch

import paper_2209_04876_gb300 as kr

pytestmark = pytest.mark.gpu


def _tables(I, R, seed):
    rng = np.random.default_rng(seed)
    As = []
    for i, r in zip(I, R):
        A = rng.standard_normal((i, r)) * np.exp(rng.standard_normal(i))[:, None]
        As.append(torch.tensor(A, dtype=torch.float32, device="cuda"))
    return kr.kron_leverage(As)


def test_noalloc_sampler_matches_kron_sample_on_two_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    calls = [
        ([700, 513, 96], [9, 17, 5], 250003, 41, 7, 0),
        ([5000, 3000], [13, 30], 99991, 2 ** 40 + 3, 8, 12),
    ]
    for I, R, s, seed, cid, row in calls:
        t = _tables(I, R, seed)
        ref_idx, ref_w = kr.kron_sample(t["cdf"], t["prob"], s, seed, cid, row=row)
        idx = torch.full((s, len(I)), -1, dtype=torch.int32, device="cuda")
        w = torch.full((s,), -1.0, dtype=torch.float32, device="cuda")
        out_idx, out_w = kr.kron_sample_noalloc(t["cdf"], t["prob"], s, seed, cid, row=row, idx=idx, w=w)
        torch.cuda.synchronize()
        assert out_idx.data_ptr() == idx.data_ptr() and out_w.data_ptr() == w.data_ptr()
        assert torch.equal(idx, ref_idx)
        torch.testing.assert_close(w, ref_w, rtol=2e-7, atol=0.0)


def test_noalloc_sampler_rejects_tables_above_the_limit():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    t = _tables([9000, 9000], [4, 4], 3)  # 18000 rows in total > 16384
    with pytest.raises(kr.KronError) as e:
        kr.kron_sample_noalloc(t["cdf"], t["prob"], 1000, 1, 1)
    assert e.value.name == "KR_EINVAL" and "KR_NOALLOC_MAX_ROWS" in str(e.value)
