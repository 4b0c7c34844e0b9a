"""The C-ABI library builds for sm_103a, loads, and exports every declared symbol."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "aim.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int|void|const char\*)\s+(aim_\w+)\s*\(", src, re.M)))


def test_header_declares_api():
    names = declared_symbols()
    for n in ("aim_setup", "aim_march", "aim_matvec", "aim_rhs", "aim_destroy"):
        assert n in names


def test_library_loads_and_exports():
    from paper_1408_7060_gb300 import abi

    lib = abi.load()
    for n in declared_symbols():
        assert hasattr(lib, n), n
    assert set(abi.EXPORTS) == set(declared_symbols())


def test_setup_without_gpu_fails_cleanly():
    """Without a device aim_setup returns an error code (never a crash)."""
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1408_7060_gb300 import abi
    from paper_1408_7060_gb300.inputs import make_workload

    w = make_workload("sphere480")
    with pytest.raises(abi.AimError):
        abi.aim_setup(*w.mesh, w.grid_n, w.origin, w.h, w.near_radius, w.dt, w.f_c)


def test_kernel_classes_match_header():
    """The binding's kernel-class count is the header's enum, and every class has a name
    (aim_kernel_name needs no context and no device)."""
    from paper_1408_7060_gb300 import abi

    src = open(os.path.join(ROOT, "include", "aim.h")).read()
    body = re.search(r"enum\s*{\s*(AIM_K_ANTERP_XFFT[^}]*)}", src).group(1)
    names = [n for n in re.findall(r"^\s*(AIM_K_\w+)", body, re.M) if n != "AIM_K_COUNT"]
    assert len(names) == abi.AIM_K_COUNT
    lib = abi.load()
    got = [lib.aim_kernel_name(i).decode() for i in range(abi.AIM_K_COUNT + 1)]
    assert "?" not in got[:-1] and len(set(got[:-1])) == abi.AIM_K_COUNT
    assert got[-1] == "?"
