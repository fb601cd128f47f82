"""The C-ABI library builds, loads and exports every entry point that
include/mc.h declares; host-side argument validation runs before any device
work (no compute call needs a GPU here)."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mc.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(mc_[a-z_0-9]+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def built():
    from paper_2410_10503_gb300 import build as B
    path = B.build()
    assert os.path.exists(path)
    return path


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["mc_create", "mc_forward", "mc_adjoint", "mc_spdhg_run", "mc_pdhg_run",
                     "mc_set_data", "mc_norms", "mc_destroy", "mc_last_error"]:
        assert required in names


def test_library_exports_every_declared_symbol(built):
    out = subprocess.run(["nm", "-D", "--defined-only", built], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT (mc_[a-z_0-9]+)$", out, flags=re.M))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing


def test_binding_covers_every_declared_symbol(built):
    from paper_2410_10503_gb300 import _native as N
    assert sorted(N.SIGNATURES) == declared_functions()
    L = N.load()
    for name in declared_functions():
        assert getattr(L, name) is not None
    assert b"sm_103a" in L.mc_version()


def _create(geom, n_gates, motion):
    from paper_2410_10503_gb300 import _native as N
    L = N.load()
    out = ctypes.c_void_p()
    st = L.mc_create(ctypes.byref(geom) if geom is not None else None, n_gates,
                     ctypes.byref(motion) if motion is not None else None, None, ctypes.byref(out))
    return st, L.mc_last_error(None).decode(), out.value


def test_create_rejects_bad_arguments_on_the_host(built):
    from paper_2410_10503_gb300 import _native as N
    rigid = np.zeros((2, 3))
    m = N.mc_motion(N.MC_MOTION_RIGID, rigid.ctypes.data, None)
    for geom, ng, msg in [(N.mc_geometry(1, 10, 10), 2, "n=1"),
                          (N.mc_geometry(4096, 10, 10), 2, "n=4096"),
                          (N.mc_geometry(16, 0, 10), 2, "n_angles=0"),
                          (N.mc_geometry(16, 10, 0), 2, "n_bins=0"),
                          (N.mc_geometry(16, 10, 10), 0, "n_gates=0")]:
        st, err, h = _create(geom, ng, m)
        assert st == N.MC_EINVAL and msg in err and not h
    st, err, h = _create(None, 2, m)
    assert st == N.MC_EINVAL
    bad = N.mc_motion(7, rigid.ctypes.data, None)
    st, err, _ = _create(N.mc_geometry(16, 10, 10), 2, bad)
    assert st == N.MC_EINVAL and "kind" in err
    nofield = N.mc_motion(N.MC_MOTION_FIELD, None, None)
    st, err, _ = _create(N.mc_geometry(16, 10, 10), 2, nofield)
    assert st == N.MC_EINVAL and "field" in err


def test_null_context_calls_fail_cleanly(built):
    from paper_2410_10503_gb300 import _native as N
    L = N.load()
    assert L.mc_reset(None) == N.MC_EINVAL
    assert L.mc_forward(None, 0, None, None) == N.MC_EINVAL
    assert L.mc_spdhg_run(None, 1, None, None, None) == N.MC_EINVAL
    assert L.mc_set_field(None, 0, None) == N.MC_EINVAL
    assert L.mc_set_subsets(None, 2) == N.MC_EINVAL
    assert L.mc_autotune(None, 1, None) == N.MC_EINVAL
    assert L.mc_batch_spdhg_run(None, 0, 1, None, None) == N.MC_EINVAL
    assert L.mc_vjp(None, 0, None, None, None, None) == N.MC_EINVAL
    assert L.mc_get_shapes(None, None) == N.MC_EINVAL
    L.mc_destroy(None)


def test_no_gpu_means_loud_failure(built):
    """Without an sm_103a device the library refuses instead of falling back."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2410_10503_gb300 import Context, MCError
    with pytest.raises(MCError) as ei:
        Context(16, 10, 23, 2, rigid=np.zeros((2, 3)))
    assert "MC_EDEVICE" in str(ei.value)
