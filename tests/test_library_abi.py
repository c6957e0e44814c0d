"""The C-ABI library loads on a machine without a GPU and exports every function that
include/hp.h declares; host-only logic (FFT stage code) is checked against numpy."""

import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "hp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hp_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    import paper_2203_15684_gb300 as P
    if not os.path.exists(P.LIB_PATH):
        from paper_2203_15684_gb300 import build as B
        B.build()
    return P.lib()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "hp_setup" in names and "hp_response" in names and "hp_hubbard" in names
    for n in names:
        assert hasattr(lib, n), n


@pytest.mark.parametrize("n", [2, 3, 4, 5, 12, 20, 24, 36, 45, 72, 90])
def test_fft_stage_logic_on_host(lib, n):
    import paper_2203_15684_gb300 as P
    rng = np.random.default_rng(n)
    x = rng.standard_normal((9, n)) + 1j * rng.standard_normal((9, n))
    assert np.allclose(P.selftest_fft_host(x, -1), np.fft.fft(x, axis=1), atol=1e-11)
    assert np.allclose(P.selftest_fft_host(x, +1), np.fft.ifft(x, axis=1) * n, atol=1e-11)


def test_setup_without_gpu_reports_error(lib):
    import paper_2203_15684_gb300 as P
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import workloads as W
    with pytest.raises(P.HPError) as e:
        P.Context.from_workload(W.tiny())
    assert e.value.code == 6  # HP_ECUDA, no fallback
