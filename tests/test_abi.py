"""The C-ABI library builds, loads and exports every entry point include/kron.h
declares (no compute calls: runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "kron.h")).read()
    return sorted(set(re.findall(r"KR_API\s+[\w\s\*]+?\b((?:kr|kron|tucker)_\w+)\s*\(", txt)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2209_04876_gb300 import build

    return build.build()


def test_header_declares_the_boundary():
    names = _declared()
    for n in ["kron_leverage", "kron_sample", "kron_regress", "kron_ridge", "kron_ridge_batched", "tucker_als_sweep",
              "kr_create", "kr_destroy", "kr_last_error"]:
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    L = ctypes.CDLL(libpath)
    missing = [n for n in _declared() if not hasattr(L, n)]
    assert not missing, missing
    import paper_2209_04876_gb300 as kr

    assert sorted(kr.EXPORTED) == _declared()


def test_struct_layouts_match_header(libpath, tmp_path):
    """ctypes mirrors of kr_factors / kr_opts / kr_report / kr_dev_report have the C compiler's layout."""
    import shutil
    import subprocess

    import paper_2209_04876_gb300 as kr

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "layout.c"
    src.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "%s/include/kron.h"\n'
        'int main(void){printf("%%zu %%zu %%zu %%zu %%zu %%zu %%zu %%zu %%zu %%zu %%zu %%zu\\n", sizeof(kr_factors),'
        ' offsetof(kr_factors, A), sizeof(kr_opts), offsetof(kr_opts, seed), sizeof(kr_report),'
        ' offsetof(kr_report, t_ms), offsetof(kr_opts, host_io), offsetof(kr_opts, stop_rule),'
        ' offsetof(kr_opts, theta), sizeof(kr_dev_report), offsetof(kr_dev_report, s),'
        ' offsetof(kr_dev_report, rel_update)); return 0;}\n' % ROOT)
    exe = tmp_path / "layout"
    subprocess.run([cc, str(src), "-o", str(exe)], check=True)
    got = list(map(int, subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()))
    want = [ctypes.sizeof(kr.KrFactors), kr.KrFactors.A.offset, ctypes.sizeof(kr.KrOpts), kr.KrOpts.seed.offset,
            ctypes.sizeof(kr.KrReport), kr.KrReport.t_ms.offset, kr.KrOpts.host_io.offset, kr.KrOpts.stop_rule.offset,
            kr.KrOpts.theta.offset, ctypes.sizeof(kr.KrDevReport), kr.KrDevReport.s.offset,
            kr.KrDevReport.rel_update.offset]
    assert got == want


def test_sample_count_rule(libpath):
    """The library's default sample count (the one rule the solvers use) against the
    oracle's restatement of the scaled Alg. 2 count, s = ceil(c R ln R / eps)."""
    import paper_2209_04876_gb300 as kr
    from oracle import kron as ko

    assert kr.kron_sample_count(256, 0.1) == 56783
    assert kr.kron_sample_count(32768, 0.05) == 27255657
    for R in (1, 2, 3, 16, 256, 4096, 32768, 262144, 24576):
        for eps in (0.8, 0.5, 0.1, 0.05, 0.01):
            for c in (4.0, 1.0, 0.25):
                assert kr.kron_sample_count(R, eps, c) == ko.sample_count(R, eps, c), (R, eps, c)
    assert kr.kron_sample_count(256, 0.1, 0.0) == 56783  # c <= 0 selects 4
    with pytest.raises(ValueError):
        kr.kron_sample_count(256, 1.5)


def test_noalloc_wrapper_rejects_bad_tensors_before_the_call():
    """The allocation-free sampler writes through raw pointers: the binding refuses a
    table or an output of the wrong dtype, device, layout or size before calling the
    library (runs without a GPU: the checks come first)."""
    import torch

    import paper_2209_04876_gb300 as kr

    cdf = torch.linspace(0.1, 1.0, 10, dtype=torch.float64)
    with pytest.raises(ValueError):
        kr.kron_sample_noalloc([cdf.float()], None, 5, 1, 1)  # float32 table
    with pytest.raises(ValueError):
        kr.kron_sample_noalloc([cdf], None, 5, 1, 1)  # host table
    with pytest.raises(ValueError):
        kr.kron_sample_noalloc([cdf], None, 5, 1, 1, idx=torch.zeros((5, 1), dtype=torch.int64))


def test_no_oracle_import_in_product():
    """The product path never imports the CPU oracle."""
    pkg = os.path.join(ROOT, "paper_2209_04876_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in re.sub(r"#.*|//.*", "", src).lower() or f == "__init__.py" and \
                    "import oracle" not in src, f
