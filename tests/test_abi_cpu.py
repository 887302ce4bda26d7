"""C ABI checks that need no GPU: the library loads, exports every function
include/pf.h declares, its ctypes structures match the C layout, and host-side
validation rejects malformed systems before any CUDA call."""
import ctypes
import os
import re
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pf.h")


@pytest.fixture(scope="session")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2011_11880_gb300 import _lib
    return _lib.load()


def header_functions():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"^PF_API\s+[\w\s\*]*?\b(pf_\w+)\s*\(", src, re.M)))


def test_header_declares_expected_api():
    names = header_functions()
    for required in ("pf_build", "pf_residual", "pf_jacobian", "pf_residual_jacobian", "pf_vjp",
                     "pf_build_batch", "pf_pattern", "pf_incidence", "pf_contributions", "pf_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", lib._name], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (pf_\w+)", out))
    declared = set(header_functions())
    assert declared <= exported, declared - exported
    for n in declared:
        assert getattr(lib, n) is not None


def test_binding_covers_header(lib):
    from paper_2011_11880_gb300 import _lib
    assert set(_lib.SIGNATURES) == set(header_functions())


def test_struct_layout_matches_c(tmp_path):
    from paper_2011_11880_gb300 import _lib
    structs = {"pf_system": _lib.PfSystem, "pf_instance": _lib.PfInstance, "pf_dims": _lib.PfDims,
               "pf_overrides": _lib.PfOverrides, "pf_grads": _lib.PfGrads, "pf_tuning": _lib.PfTuning}
    lines = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{HEADER}"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("return 0; }")
    c = tmp_path / "layout.c"
    c.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-o", str(exe), str(c)], check=True)
    got = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    for ln in got:
        if not ln:
            continue
        cname, field, val = ln.split()
        py = structs[cname]
        want = ctypes.sizeof(py) if field == "size" else getattr(py, field).offset
        assert int(val) == want, (cname, field, val, want)


def test_error_strings(lib):
    for code in range(8):
        assert lib.pf_error_string(code) and lib.pf_error_string(code) != b"unknown error code"
    assert lib.pf_error_string(99) == b"unknown error code"


def _build(lib, sys, formulation=0):
    from paper_2011_11880_gb300.context import _SystemArrays
    arr = _SystemArrays(sys)
    h = ctypes.c_void_p()
    rc = lib.pf_build(ctypes.byref(arr.struct), formulation, None, ctypes.byref(h))
    return rc, (lib.pf_last_error() or b"").decode(), h


def base_system():
    import gridgen
    return gridgen.PowerSystem.build(
        3, branches=[(0, 1, 0.01, 0.1, 0.02), (1, 2, 0.01, 0.1, 0.0)], loads=[(1, 0.5, 0.1)],
        pvs=[(2, 0.3, 1.01)], slack=(0, 1.0, 0.0), shunts=[(1, 0.0, 0.1)])


@pytest.mark.parametrize("mutate,expect", [
    (lambda s: s.br_to.__setitem__(0, 7), "out of range"),
    (lambda s: s.br_to.__setitem__(0, 0), "from == to"),
    (lambda s: (s.br_r.__setitem__(1, 0.0), s.br_x.__setitem__(1, 0.0)), "r^2 + x^2 > 0"),
    (lambda s: s.br_tap.__setitem__(0, -1.0), "tap"),
    (lambda s: s.br_x.__setitem__(0, np.nan), "finite"),
    (lambda s: setattr(s, "slack_bus", 5), "slack bus out of range"),
    (lambda s: s.pv_bus.__setitem__(0, 0), "slack bus"),
    (lambda s: s.load_bus.__setitem__(0, -1), "out of range"),
    (lambda s: s.sh_bus.__setitem__(0, 3), "out of range"),
    (lambda s: setattr(s, "n_bus", 1), "n_bus"),
])
def test_host_validation_rejects(lib, mutate, expect):
    s = base_system()
    mutate(s)
    rc, msg, h = _build(lib, s)
    assert rc == 1 and expect in msg, (rc, msg)
    assert not h.value


def test_extended_rejects_two_pv_on_one_bus(lib):
    import gridgen
    s = gridgen.PowerSystem.build(3, branches=[(0, 1, 0.01, 0.1, 0), (1, 2, 0.01, 0.1, 0)],
                                  pvs=[(2, 0.3, 1.01), (2, 0.1, 1.01)], slack=(0, 1.0, 0.0))
    rc, msg, _ = _build(lib, s, formulation=1)
    assert rc == 1 and "two PV units" in msg


def test_bad_formulation(lib):
    rc, msg, _ = _build(lib, base_system(), formulation=7)
    assert rc == 1 and "formulation" in msg


def test_null_arguments(lib):
    h = ctypes.c_void_p()
    assert lib.pf_build(None, 0, None, ctypes.byref(h)) == 1
    assert lib.pf_residual(None, None, None, None) == 1
    assert lib.pf_get_dims(None, None) == 1
    lib.pf_destroy(None)


def _build_batch(lib, systems, instances, formulation=0):
    from paper_2011_11880_gb300._lib import PfInstance, PfSystem
    from paper_2011_11880_gb300.context import _SystemArrays
    arrs = [_SystemArrays(x) for x in systems]
    grids = (PfSystem * len(arrs))(*[a.struct for a in arrs])
    inst = (PfInstance * max(len(instances), 1))(*[PfInstance(g, o) for g, o in instances])
    h = ctypes.c_void_p()
    rc = lib.pf_build_batch(grids, len(arrs), inst if instances else None, len(instances), formulation, None,
                            ctypes.byref(h))
    return rc, (lib.pf_last_error() or b"").decode(), h


@pytest.mark.parametrize("instances,expect", [
    ([], "no instances"),
    ([(0, -1), (1, -1)], "grid index out of range"),
    ([(0, 2)], "outage branch out of range"),
    ([(0, -2)], "outage branch out of range"),
])
def test_batch_validation_rejects(lib, instances, expect):
    rc, msg, h = _build_batch(lib, [base_system()], instances)
    assert rc == 1 and expect in msg, (rc, msg)
    assert not h.value


def test_package_refuses_to_load_without_the_library(tmp_path):
    """No CPU fallback: a copy of the package without libpf.so fails to import."""
    import shutil
    src = os.path.join(ROOT, "paper_2011_11880_gb300")
    dst = tmp_path / "paper_2011_11880_gb300"
    dst.mkdir()
    for f in os.listdir(src):
        if f.endswith(".py"):
            shutil.copy(os.path.join(src, f), dst / f)
    r = subprocess.run([sys.executable, "-c", "import paper_2011_11880_gb300"], cwd=tmp_path,
                       capture_output=True, text=True)
    assert r.returncode != 0
    assert "ImportError" in r.stderr and "libpf.so not found" in r.stderr
