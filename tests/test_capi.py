"""The C ABI without a GPU: the library builds for sm_103a, loads, exports
every entry point that include/hweno.h declares, and the binding declares
them all; argument checks that precede any CUDA call return HWENO_EINVAL."""
import ctypes
import os
import subprocess

import pytest
import torch

from _util import header_functions

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def hw():
    from paper_2207_05258_gb300 import build
    build.build()
    from paper_2207_05258_gb300 import hweno
    return hweno


def test_library_exports_every_declared_function(hw):
    names = header_functions()
    assert len(names) >= 15
    lib = ctypes.CDLL(hw.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", hw.LIB_PATH], capture_output=True,
                         text=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if " T " in l}
    assert set(names) <= exported
    assert set(hw.SIGNATURES) == set(names)


def test_binding_constants_match_the_header(hw):
    text = open(os.path.join(ROOT, "include", "hweno.h")).read()
    defines = dict(l.split()[1:3] for l in text.splitlines()
                   if l.startswith("#define HWENO_") and len(l.split()) >= 3)
    value = lambda name: int(defines["HWENO_" + name].strip("()"))
    assert value("TILE_VARIANTS") == hw.TILE_VARIANTS
    assert value("CLUSTER_MAX_POINTS") == hw.CLUSTER_MAX_POINTS
    assert value("MAX_SIZE_CLASSES") == hw.MAX_SIZE_CLASSES
    for name in ("OK", "EINVAL", "ENOMEM", "ECUDA", "ENONFINITE", "ETIMEOUT", "ENOTSUP",
                 "BURGERS", "EULER", "BUCKLEY"):
        assert value(name) == getattr(hw, name), name


def test_default_options_are_the_papers(hw):
    o = hw.default_options()
    assert list(o.lin_w) == [0.98, 0.01, 0.01] and list(o.lim_d) == [0.98, 0.01, 0.01]
    assert o.eps == 1e-6 and o.cfl == 0.6 and o.limiter == 1 and o.eig_avg == 0


def _create(hw, eq=0, dim=1, nx=16, ny=16, batch=1, nxs=None, prec=0, bc=(0, 0, 0, 0),
            gamma=1.4, y1=1.0):
    arr = (ctypes.c_int * len(nxs))(*nxs) if nxs else None
    g = hw.Grid(dim, nx, ny, 0.0, 1.0, 0.0, y1, batch,
                ctypes.cast(arr, ctypes.POINTER(ctypes.c_int)) if arr else None, prec)
    b = hw.Bc(*bc)
    h = ctypes.c_void_p()
    rc = hw.lib.hweno_create(ctypes.byref(h), eq, ctypes.byref(g), gamma, ctypes.byref(b))
    if rc == 0:
        hw.lib.hweno_destroy(h)
    return rc, h


@pytest.mark.parametrize("kw", [
    dict(nx=3), dict(nx=0), dict(batch=0), dict(batch=2, nxs=[16, 2]), dict(eq=3), dict(dim=3),
    dict(eq=2, dim=2), dict(eq=2, bc=(2, 2, 0, 0)),
    dict(prec=5), dict(bc=(0, 1, 0, 0)), dict(bc=(4, 1, 0, 0)), dict(bc=(9, 9, 0, 0)),
    dict(eq=1, gamma=1.0), dict(dim=2, batch=2), dict(dim=2, ny=3), dict(dim=2, y1=0.0),
    dict(dim=2, bc=(1, 1, 5, 4)), dict(dim=2, eq=0, bc=(1, 1, 4, 5)),
])
def test_create_rejects_invalid_problems(hw, kw):
    rc, h = _create(hw, **kw)
    assert rc == hw.EINVAL and not h.value


def test_null_arguments(hw):
    assert hw.lib.hweno_create(None, 0, None, 1.4, None) == hw.EINVAL
    assert hw.lib.hweno_measure_fp64_peak(None, None) == hw.EINVAL
    assert hw.lib.hweno_destroy(None) == 0
    assert hw.lib.hweno_last_error(None) == b"null context"
    assert hw.lib.hweno_step(None, None, None, None, None, 1.0, None, None) == hw.EINVAL
    assert hw.lib.hweno_num_points(None) == -1


@pytest.mark.skipif(torch.cuda.is_available(), reason="checks the no-GPU failure path")
def test_valid_create_without_gpu_fails_cleanly(hw):
    rc, h = _create(hw, nx=64)
    assert rc in (hw.ECUDA, hw.ENOMEM) and not h.value


def test_binding_refuses_cpu_tensors(hw):
    with pytest.raises(ValueError):
        hw._ptr(torch.zeros(4))


@pytest.mark.parametrize("field,value", [("eps", 0.0), ("eps", 1e-30), ("eps", 1e7),
                                         ("lin_w", (1 - 2e-7, 1e-7, 1e-7)),
                                         ("lim_d", (0.5, 0.5 - 1e-9, 1e-9)),
                                         ("lin_w", (0.5, 0.3, 0.3))])
def test_out_of_range_options_are_rejected_before_any_cuda_call(hw, field, value):
    """The allocation-free step checks its options before it touches a device
    pointer: eps outside [1e-20, 1e6], a linear weight below 1e-6 or weights
    that do not sum to 1 are HWENO_EINVAL (host buffers stand in for the
    device ones, which are never read)."""
    import numpy as np
    o = hw.default_options()
    if field == "eps":
        o.eps = value
    else:
        for i, x in enumerate(value):
            getattr(o, field)[i] = x
    n = 32
    U = np.zeros(3 * n); V = np.zeros(3 * n); t = np.zeros(1)
    bc = hw.Bc(1, 1, 0, 0)
    ptr = lambda a: ctypes.c_void_p(a.ctypes.data)
    rc = hw.lib.hweno_step_1d_noalloc(hw.EULER, n, 0.0, 1.0, 1.4, ctypes.byref(bc),
                                      ctypes.byref(o), ptr(U), ptr(V), ptr(t), 1.0, None, None)
    assert rc == hw.EINVAL


def test_binding_structs_match_the_header_layout(hw, tmp_path):
    """The ctypes mirrors of hweno_grid, hweno_bc and hweno_options have the
    C structs' size and field offsets (a C program compiled against the
    header prints them)."""
    structs = {"hweno_grid": hw.Grid, "hweno_bc": hw.Bc, "hweno_options": hw.Options}
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "hweno.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append('  printf("%s size %%zu\\n", sizeof(%s));' % (cname, cname))
        for f, _ in py._fields_:
            lines.append('  printf("%s %s %%zu\\n", offsetof(%s, %s));' % (cname, f, cname, f))
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                    str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], capture_output=True, text=True,
                               check=True).stdout.splitlines():
        a, b, v = line.split()
        got[(a, b)] = int(v)
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)
