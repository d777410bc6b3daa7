"""The C-ABI library builds, loads and exports every entry point include/bte.h declares; its
host-side validation rejects bad inputs before any CUDA call (runs without a GPU)."""
import ctypes as ct
import os
import re

import numpy as np
import pytest

from paper_2306_14181_gb300 import bte, build, inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return bte.load()


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "bte.h")).read()
    return sorted(set(re.findall(r"^(?:bte_status|void|const char \*)\s*\**\s*(bte_\w+)\s*\(", text, re.M)))


def test_header_declares_the_binding_exports():
    assert declared_symbols() == sorted(bte.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name
    out = os.popen("nm -D --defined-only %s" % bte.LIB_PATH).read()
    for name in declared_symbols():
        assert re.search(r"\bT %s\b" % name, out), name


def _create(**over):
    cfg = inputs.hotspot_2d(nx=8, ny=6, nb=2, ntheta=1, nphi=1)
    args = dict(dim=cfg["dim"], n=cfg["n"], h=cfg["h"], C=cfg["C"], vabs=cfg["v"], tau=cfg["tau"], quad=cfg["quad"],
                bc=cfg["bc"], T_wall=cfg["Tw"], dt=cfg["dt"], stream=0)
    args.update(over)
    return bte.bte_create(**args)


@pytest.mark.parametrize("over,frag", [
    (dict(dim=4), "dim"),
    (dict(n=(1, 6, 1)), "extent"),
    (dict(n=(8, 6, 3)), "inactive"),
    (dict(dt=0.0), "dt"),
    (dict(dt=float("nan")), "dt"),
    (dict(tau=np.array([1e-12, -1.0])), "band 1"),
    (dict(C=np.array([1.0, 0.0])), "band 1"),
    (dict(bc=[3, 1, 0, 1, 3, 3]), "periodic"),
    (dict(bc=[9, 1, 0, 1, 3, 3]), "bad type"),
    (dict(quad=("octant", 0, 2)), "OCTANT"),
    (dict(quad=("gl1d", 1)), "GL1D"),
    (dict(storage=7), "storage"),
    (dict(limiter=5), "limiter"),
    (dict(quad=("explicit", np.array([[1.0, 0, 0], [0.0, 1, 0]]), np.array([1.0, 1.0])), bc=[2, 2, 0, 0, 3, 3]),
     "mirror"),
    (dict(dT_jump=(0.5, 0.0, 0.0)), "dT_jump needs a periodic pair"),        # x walls are diffuse
    (dict(bc=[3, 3, 0, 1, 3, 3], dT_jump=(0.5, 0.0, 0.2)), "inactive axis 2"),
    (dict(bc=[3, 3, 0, 1, 3, 3], dT_jump=(float("inf"), 0.0, 0.0)), "non-finite dT_jump"),
    (dict(bc=[4, 4, 0, 1, 3, 3]), "at most one interface wall"),
    (dict(bc=[0, 1, 0, 1, 4, 3]), "interface on an inactive axis"),
])
def test_host_validation_rejects_bad_input(lib, over, frag):
    with pytest.raises(bte.BteError) as ei:
        _create(**over)
    assert ei.value.status == bte.BTE_EINVAL
    assert frag in str(ei.value)


def test_interface_walls_need_fp32_storage(lib):
    with pytest.raises(bte.BteError) as ei:
        _create(bc=[0, 4, 0, 1, 3, 3], storage=bte.BTE_STORE_F16)
    assert ei.value.status == bte.BTE_EUNSUPPORTED


def test_null_arguments_are_rejected_by_the_newer_calls(lib):
    assert lib.bte_interface(None, 1, None, 0, None, None) == bte.BTE_EINVAL
    assert lib.bte_step_pair(None, None, 1) == bte.BTE_EINVAL
    assert lib.bte_sis_iterate(None, 1) == bte.BTE_EINVAL
    assert lib.bte_run_steady_implicit(None, 10, 1, 1e-6, 1e-6, None, None, None) == bte.BTE_EINVAL
    assert lib.bte_set_steady_scheme(None, 0) == bte.BTE_EINVAL
    assert lib.bte_set_wait_limit(None, 0, 0) == bte.BTE_EINVAL


def test_null_arguments_are_rejected(lib):
    out = ct.c_void_p()
    assert lib.bte_create(None, None, None, None, None, ct.byref(out)) == bte.BTE_EINVAL
    assert lib.bte_create(None, None, None, None, None, None) == bte.BTE_EINVAL
    assert lib.bte_step(None, 1) == bte.BTE_EINVAL
    lib.bte_destroy(None)   # ignored
    assert b"NULL" in lib.bte_last_error(None)


def test_binding_declares_argument_types_of_every_export(lib):
    """Every entry point the binding calls has its argument types declared (a pointer passed
    without them would be truncated to a C int)."""
    for name in bte.EXPORTS:
        f = getattr(lib, name)
        assert f.argtypes is not None, name
