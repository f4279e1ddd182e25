"""CPU checks of the C-ABI library: it builds for sm_103a, loads without a
GPU, exports every function that include/wave2d.h declares, and fails
loudly (no CPU fallback) when no device is present."""
import ctypes
import os
import re

import pytest

from conftest import ROOT

HEADER = os.path.join(ROOT, "include", "wave2d.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(wave2d_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libw():
    from paper_1904_04048_gb300 import build
    build.build()
    from paper_1904_04048_gb300 import wave2d
    return wave2d


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("wave2d_create", "wave2d_first_step", "wave2d_step_n", "wave2d_error_vs_exact",
                     "wave2d_get_state", "wave2d_set_state", "wave2d_destroy", "wave2d_last_error"):
        assert required in names


def test_every_declared_symbol_is_exported(libw):
    L = ctypes.CDLL(libw.LIB_PATH)
    for name in declared_functions():
        assert hasattr(L, name), name
    assert set(declared_functions()) == set(libw.SIGNATURES), "binding and header disagree"


def test_pure_host_entry_points(libw):
    assert abs(libw.lambda_max(5) - 2 ** -0.5) < 1e-15
    assert abs(libw.lambda_max(9) - ((3 - 3 ** 0.5) / 2) ** 0.5) < 1e-15
    assert abs(libw.lambda_max(9, conventional=True) - 3 ** 0.5 / 2) < 1e-15
    assert libw.lambda_max(13) == libw.lambda_max(5)
    assert libw.launch_count() >= 0


def test_argument_errors_need_no_gpu(libw):
    with pytest.raises(libw.Wave2DError) as e:
        libw.Wave2D(8, 8, 0.1, 0.05, scheme=7)
    assert e.value.code == libw.ERR_ARG
    with pytest.raises(libw.Wave2DError) as e:
        libw.Wave2D(0, 8, 0.1, 0.05)
    assert e.value.code == libw.ERR_ARG
    with pytest.raises(libw.Wave2DError) as e:
        libw.Wave2D(8, 8, 0.1, 0.09, scheme=5)  # lambda 0.9 > 1/sqrt2
    assert e.value.code == libw.ERR_UNSTABLE
    with pytest.raises(libw.Wave2DError) as e:
        libw.Wave2D(8, 8, -0.1, 0.05)
    assert e.value.code == libw.ERR_ARG


def test_no_cpu_fallback_without_device(libw):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(libw.Wave2DError) as e:
        libw.Wave2D(8, 8, 0.1, 0.05)
    assert e.value.code == libw.ERR_CUDA


def test_binding_refuses_missing_library(monkeypatch, tmp_path):
    from paper_1904_04048_gb300 import wave2d
    monkeypatch.setattr(wave2d, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(wave2d, "_lib", None)
    with pytest.raises(ImportError):
        wave2d.lib()
