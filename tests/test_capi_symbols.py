"""The CUDA library builds for sm_103a, loads without a GPU, and exports every
entry point that include/*.h declares (no compute call is made here)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"\b(aapdhg_\w+)\s*\(", src):
            if not m.group(1).endswith("_fn"):
                names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2508_08062_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("aapdhg_create", "aapdhg_iterate", "aapdhg_get_iterate", "aapdhg_get_kkt",
              "aapdhg_set_method", "aapdhg_set_steps", "aapdhg_destroy"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    from paper_2508_08062_gb300 import binding
    assert set(binding.EXPORTS) == _declared()


def test_library_is_built_for_sm103a():
    from paper_2508_08062_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)


def test_no_cpu_fallback_without_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    import lpgen
    from paper_2508_08062_gb300 import Solver
    with pytest.raises(RuntimeError):
        Solver(lpgen.toy_feasibility())
