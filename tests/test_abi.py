"""The C-ABI library builds for sm_103a, loads, and exports every function include/csc.h declares.
Argument checks that fail before any CUDA call are exercised here without a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1709_09479_gb300 import build
    if not os.path.exists(build.LIB):
        build.build()
    return ctypes.CDLL(build.LIB)


def declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"\b(csc_\w+)\s*\(", text)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert {"csc_init", "csc_code", "csc_learn", "csc_objective", "csc_destroy"} <= set(names)
    for n in names:
        assert hasattr(lib, n), n


def test_version_and_argument_errors_without_gpu(lib):
    from paper_1709_09479_gb300 import csc
    assert "sm_103a" in csc.csc_version()
    with pytest.raises(csc.CscError) as e:
        csc.csc_init(J=4, K=2, fs=(3, 3), dims=(16, 16), n_images=1, beta=1.0, rho=1.0)
    assert e.value.status == 2 and "J" in str(e.value)
    with pytest.raises(csc.CscError) as e:
        csc.csc_init(J=1, K=2, fs=(4, 3), dims=(16, 16), n_images=1, beta=1.0, rho=1.0)
    assert e.value.status == 2
    with pytest.raises(csc.CscError) as e:
        csc.csc_init(J=1, K=2, fs=(3, 3), dims=(16, 15), n_images=1, beta=1.0, rho=1.0)
    assert e.value.status == 2
    with pytest.raises(csc.CscError) as e:
        csc.csc_init(J=1, K=2, fs=(3, 3), dims=(22, 16), n_images=1, beta=1.0, rho=1.0)   # 11 | H
    assert e.value.status == 2
    with pytest.raises(csc.CscError) as e:
        csc.csc_init(J=1, K=2, fs=(3, 3), dims=(16, 16), n_images=1, beta=-1.0, rho=1.0)
    assert e.value.status == 1
    assert lib.csc_code(None, None, None, None, None, 1) == 1



def test_uneven_size_checks_without_gpu(lib):
    """csc_init_uneven accepts any side in [8, 1024] with the filter inside (odd and prime sides
    included: the host plans their Bluestein tables before any CUDA call) and rejects the rest with
    CSC_ERR_SHAPE naming the size; without a GPU an accepted batch then fails with CSC_ERR_CUDA."""
    from paper_1709_09479_gb300 import csc
    for bad in [(2000, 64), (64, 6), (9, 4), (1025, 1025)]:
        with pytest.raises(csc.CscError) as e:
            csc.csc_init_uneven(1, 2, (5, 5), [(64, 64), bad], 1.0, 1.0)
        assert e.value.status == 2 and f"{bad[0]}x{bad[1]}" in str(e.value)
    if not _has_gpu():
        with pytest.raises(csc.CscError) as e:
            csc.csc_init_uneven(1, 2, (5, 5), [(67, 131), (64, 64), (509, 1024), (8, 9)], 1.0, 1.0)
        assert e.value.status == 4


def _has_gpu():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def test_binding_constants_match_the_header():
    """The Python binding's flag, precision and status constants are the values include/csc.h
    defines (the binding passes them through the C ABI as plain integers)."""
    from paper_1709_09479_gb300 import csc
    text = open(os.path.join(ROOT, "include", "csc.h")).read()
    defines = {m.group(1): int(m.group(2)) for m in re.finditer(r"#define\s+(CSC_FLAG_\w+)\s+(\d+)", text)}
    assert defines, "no CSC_FLAG_* defines found"
    for name, value in defines.items():
        assert getattr(csc, name) == value, name
    enums = {m.group(1): int(m.group(2)) for m in re.finditer(r"\b(CSC_(?:FP32|MIXED_\w+))\s*=\s*(\d+)", text)}
    for name, value in enums.items():
        assert getattr(csc, name) == value, name


def test_uneven_spatial_refusals_without_gpu():
    """CSC_FLAG_SPATIAL on an uneven batch is checked on the host before any CUDA call: colour
    images, reduced precision, supports above 11 x 11 and filter sets beyond one CTA's shared memory
    give CSC_ERR_UNSUPPORTED; an accepted batch then needs the device (CSC_ERR_CUDA without one)."""
    from paper_1709_09479_gb300 import csc
    dims = [(64, 64), (67, 131)]
    for J, K, fs, prec in [(3, 4, (3, 3), csc.CSC_FP32), (1, 4, (13, 13), csc.CSC_FP32),
                           (1, 4, (5, 5), csc.CSC_MIXED_BF16), (1, 416, (5, 5), csc.CSC_FP32)]:
        with pytest.raises(csc.CscError) as e:
            csc.csc_init_uneven(J, K, fs, dims, 1.0, 1.0, precision=prec, flags=csc.CSC_FLAG_SPATIAL)
        assert e.value.status == 8, (J, K, fs, prec)
    if not _has_gpu():
        with pytest.raises(csc.CscError) as e:
            csc.csc_init_uneven(1, 415, (11, 11), dims, 1.0, 1.0, flags=csc.CSC_FLAG_SPATIAL)
        assert e.value.status == 4
