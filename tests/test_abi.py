"""The C-ABI library builds, loads and exports every entry point include/*.h declares (no GPU),
and the host-side argument checks that need no device behave as documented."""
import ctypes
import glob
import os
import re

import pytest

from paper_2211_05009_gb300 import binding as B
from paper_2211_05009_gb300.build import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(lbm_[a-z_0-9]+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    path = build()
    return ctypes.CDLL(path)


def test_header_declares_the_planned_abi():
    names = declared_symbols()
    for n in ("lbm_create", "lbm_step", "lbm_moments", "lbm_residual", "lbm_stream_function",
              "lbm_mass", "lbm_probe", "lbm_run_to_residual", "lbm_save", "lbm_load", "lbm_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    assert set(declared_symbols()) <= set(B.EXPORTED) | {"lbm_info"}


def test_invalid_arguments_rejected_without_device(lib):
    B.library()
    out = ctypes.c_void_p()
    L = B.library()
    assert L.lbm_create_ex(2, 10, 0.8, 0.1, 2, 0, ctypes.byref(out)) == B.LBM_EINVAL
    assert "nx, ny >= 3" in B.lbm_last_error(None)
    assert L.lbm_create_ex(10, 10, 0.5, 0.1, 2, 0, ctypes.byref(out)) == B.LBM_EINVAL
    assert L.lbm_create_ex(10, 10, 0.8, 0.1, 9, 0, ctypes.byref(out)) == B.LBM_EINVAL
    assert L.lbm_create(10, 10, -5.0, 0.1, 2, ctypes.byref(out)) == B.LBM_EINVAL
    assert L.lbm_create_flags(10, 10, 0.0, 0.1, 2, 1, ctypes.byref(out)) == B.LBM_EINVAL
    assert "Re" in B.lbm_last_error(None)
    assert L.lbm_create_flags(10, 10, 100.0, 0.1, 2, 2, ctypes.byref(out)) == B.LBM_EINVAL
    assert "flags" in B.lbm_last_error(None)
    assert out.value is None


def test_python_package_does_no_method_arithmetic():
    """Re -> nu -> tau (Eq. 5) happens in the library only: no Python module of the package
    spells the relation between Re, nu and tau."""
    pkg = os.path.join(ROOT, "paper_2211_05009_gb300")
    for path in glob.glob(os.path.join(pkg, "*.py")):
        code = "\n".join(l.split("#")[0] for l in open(path).read().splitlines())
        assert not re.search(r"\b(tau|nu)\s*=[^=].*\b(Re|re)\b", code), path
        assert not re.search(r"\b3(\.0)?\s*\*[^\n]*\+\s*0\.5\b", code), path  # tau = 3 nu + 1/2
        assert not re.search(r"\(\s*tau\s*-\s*0\.5\s*\)", code), path  # nu = (tau - 1/2)/3


def test_create_without_gpu_fails_loudly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    out = ctypes.c_void_p()
    rc = B.library().lbm_create(16, 16, 100.0, 0.1, 2, ctypes.byref(out))
    assert rc == B.LBM_ECUDA and out.value is None
    assert "no CUDA device" in B.lbm_last_error(None)


def test_binding_constants_match_the_header():
    """Every integer #define of include/*.h that the binding mirrors has the header's value."""
    seen = 0
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        for name, expr in re.findall(r"#define\s+(LBM_[A-Z0-9_]+)\s+\(?([0-9]+(?:\s*<<\s*[0-9]+)?)\)?", open(h).read()):
            if hasattr(B, name):
                assert getattr(B, name) == eval(expr), name
                seen += 1
    assert seen >= 5
