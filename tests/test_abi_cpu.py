"""Host-side checks of the C ABI that need no GPU: the library builds for
sm_103a, loads, and exports every entry point the public header declares;
the Python binding wraps each of them."""
import ctypes
import os
import re
import subprocess

import pytest

from conftest import ROOT
from paper_2208_09267_gb300 import build, lbm

HEADER = os.path.join(ROOT, "include", "lbm_vanse.h")


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^LBM_API[^;(]*?\b(lbm_vanse_\w+)\s*\(", text, flags=re.M)))


def test_header_declares_the_abi():
    names = declared_functions()
    for required in ("lbm_vanse_create", "lbm_vanse_set_epsilon", "lbm_vanse_set_force",
                     "lbm_vanse_step", "lbm_vanse_moments", "lbm_vanse_destroy"):
        assert required in names


def test_library_builds_and_exports_every_declared_symbol():
    path = build.build()
    assert os.path.exists(path)
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT (lbm_vanse_\w+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing


def test_library_loads_and_binding_covers_the_header():
    L = lbm.lib()
    for name in declared_functions():
        assert hasattr(L, name)
        assert name in lbm._SIGS, f"binding lacks {name}"
    assert set(lbm._SIGS) == set(declared_functions())
    assert "sm_103a" in lbm.version()


def test_struct_layouts_match_the_header():
    """The binding's ctypes structs have the header's field order and size."""
    text = open(HEADER).read()
    body = text[text.index("typedef struct {", text.index("LBM_AXIS_X")):text.index("} lbm_vanse_params;")]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = re.findall(r"\b(\w+)(?:\s*,\s*(\w+))?(?:\s*,\s*(\w+))?\s*;", body)
    flat = [f for group in fields for f in group if f]
    assert [f[0] for f in lbm.Params._fields_] == flat
    assert ctypes.sizeof(lbm.Params) == 136


def test_params_default_and_device_bytes_need_no_gpu():
    p = lbm.Params()
    assert lbm.lib().lbm_vanse_params_default(ctypes.byref(p)) == 0
    assert (p.lattice, p.storage, p.nx, p.tau) == (1, 1, 32, 0.6)
    b32 = lbm.device_bytes("D3Q19", (256, 256, 256), "fp32")
    b16 = lbm.device_bytes("D3Q19", (256, 256, 256), "fp16")
    n = 256 ** 3
    assert 19 * n * 4 < b32 < 19 * n * 4 + 3 * n * 4 + (1 << 24)
    assert 19 * n * 2 < b16 < b32
    assert lbm.device_bytes("D2Q9", (4, 4, 2)) == 0  # invalid: D2Q9 needs nz = 1
    # d_t phi is double-buffered like phi_ref (a refresh fills the spare pair):
    # two pitched FP32 fields, rows of 45 cells stored at a pitch of 48
    stored = 48 * 20 * 12
    with_deps = lbm.device_bytes("D3Q19", (45, 20, 12), "fp32", with_deps=True)
    assert with_deps - lbm.device_bytes("D3Q19", (45, 20, 12), "fp32") == 2 * stored * 4
    with_deps64 = lbm.device_bytes("D3Q19", (45, 20, 12), "fp64", with_deps=True)
    assert with_deps64 - lbm.device_bytes("D3Q19", (45, 20, 12), "fp64") == 2 * stored * 8


def test_noalloc_limits_match_the_header():
    """The binding's staging-array limits are the header's."""
    text = open(os.path.join(ROOT, "include", "lbm_vanse.h")).read()
    m = re.search(r"#define LBM_NOALLOC_SCRATCH_BYTES \(\(size_t\)(\d+) << (\d+)\)", text)
    assert m, "LBM_NOALLOC_SCRATCH_BYTES not found"
    scratch = int(m.group(1)) << int(m.group(2))
    assert re.search(r"#define LBM_NOALLOC_MAX_CELLS \(\(long long\)\(LBM_NOALLOC_SCRATCH_BYTES / 20\)\)", text)
    assert lbm.NOALLOC_SCRATCH_BYTES == scratch
    assert lbm.NOALLOC_MAX_CELLS == scratch // 20


def _params(**kw):
    p = lbm.Params()
    assert lbm.lib().lbm_vanse_params_default(ctypes.byref(p)) == 0
    for k, v in kw.items():
        setattr(p, k, v)
    return p


@pytest.mark.parametrize("kw,word", [
    (dict(tau=0.5), "tau"), (dict(tau=float("nan")), "tau"), (dict(lattice=4), "lattice"),
    (dict(lattice=3, ny=2, nz=1), "D1Q3"), (dict(drag_model=1, drag_d=0.0), "drag"),
    (dict(les_cs=-0.1), "les_cs"), (dict(les_cs=0.2, kernel=2), "one-cell"),
    (dict(quad_auto=2), "quad_auto"),
    (dict(storage=7), "storage"), (dict(nx=0), "nx"), (dict(lattice=0, nz=2), "D2Q9"),
    (dict(quad_dim=4), "quad_dim"), (dict(rho0=0.0), "rho0"),
    (dict(lattice=0, nz=1, walls=4), "walls"), (dict(quad_axes=8), "quad_axes")])
def test_create_rejects_bad_parameters_on_the_host(kw, word):
    """Parameter checks run before any device work: LBM_EINVAL, no handle,
    and a message naming the parameter."""
    p = _params(**kw)
    h = ctypes.c_void_p()
    assert lbm.lib().lbm_vanse_create(ctypes.byref(p), ctypes.byref(h)) == -1
    assert h.value is None
    assert word in lbm.last_error(None)


def test_create_over_budget_fails_with_enomem_on_the_host():
    """Admission by HBM budget (the serving path's failure mode), injected
    with a budget far below the lattice's device bytes."""
    p = _params(nx=64, ny=64, nz=64, hbm_budget_bytes=1 << 20)
    h = ctypes.c_void_p()
    assert lbm.lib().lbm_vanse_create(ctypes.byref(p), ctypes.byref(h)) == -2
    assert h.value is None
    assert "budget" in lbm.last_error(None)


def test_null_handles_are_rejected_on_the_host():
    L = lbm.lib()
    assert L.lbm_vanse_set_epsilon(None, None, None, 0, 0) == -1
    assert L.lbm_vanse_stage_epsilon(None, None, None, 0, 0) == -1
    assert L.lbm_vanse_commit_epsilon(None) == -1
    assert L.lbm_vanse_set_force(None, None, None, None, 0, 0) == -1
    assert L.lbm_vanse_init_equilibrium(None, None, None, 0, 0) == -1
    assert L.lbm_vanse_step(None, 1, 0.0, 0, None) == -1
    assert L.lbm_vanse_moments(None, None, None, None, 0) == -1
    assert L.lbm_vanse_get_populations(None, None) == -1
    assert L.lbm_vanse_steps_done(None) == -1
    assert L.lbm_vanse_batch_step(None, 1, 0) == -1
    assert "NULL" in lbm.last_error(None)
    L.lbm_vanse_destroy(None)  # accepted
