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


def test_struct_layouts_match_header():
    """The binding's ctypes structs list the header's fields in order (a field added to
    one side only would shift every later field)."""
    from paper_1408_7060_gb300 import abi

    src = open(os.path.join(ROOT, "include", "aim.h")).read()
    for name, cls in (("aim_opts", abi.aim_opts), ("aim_stats", abi.aim_stats), ("aim_info", abi.aim_info)):
        end = src.index("} " + name + ";")
        body = src[src.rindex("typedef struct {", 0, end) + len("typedef struct {"):end]
        body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
        fields = []
        for decl in body.split(";"):
            decl = decl.strip()
            if not decl:
                continue
            names = decl.split(None, 1)[1] if not decl.startswith("const ") else decl.split(None, 2)[2]
            for n in names.split(","):
                fields.append(re.sub(r"[\s*]|\[\d+\]", "", n))
        assert [f for f, _ in cls._fields_] == fields, name


def test_z_lengths_agree():
    """The z transform lengths the library chooses from (api.cu), dispatches
    (operator_impl.cuh) and the bench's memory plan assumes are the same list."""
    import bench

    api = open(os.path.join(ROOT, "paper_1408_7060_gb300", "csrc", "api.cu")).read()
    impl = open(os.path.join(ROOT, "paper_1408_7060_gb300", "csrc", "operator_impl.cuh")).read()
    chosen = [int(x) for x in re.search(r"for \(int lz : \{([\d, ]+)\}\)", api).group(1).split(",")]
    body = re.search(r"inline void with_zlen\(int lz, F&& f\) \{(.*?)default:", impl, re.S).group(1)
    dispatched = [int(x) for x in re.findall(r"case (\d+):", body)]
    assert chosen == dispatched == list(bench.Z_LENGTHS)
