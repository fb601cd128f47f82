"""mc_forward_static, the allocation-free forward operator, against the
context path (mc_forward / mc_project) through the C ABI.

Some callers cannot allocate device memory (an allocator hook, a plugin with
a fixed memory budget, a host whose GPU memory already belongs to its own
pool); this entry point keeps all of its scratch in a fixed array built into
the library.  Two calls in a row (different geometry and motion) must both
match the existing entry points, which checks that the shared scratch is
reset between calls; sizes beyond the fixed array are refused on the host.
The entry point is also checked on its own against the FP64 oracle of A D
(Sec. II-A), and its companion mc_forward_static_status must report a
device-side wait that ran out.  This file is collected last on purpose.
"""
import ctypes
import os

import numpy as np
import pytest

import mc_synth as S

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = 1e-5


@pytest.fixture(scope="module")
def mc():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2410_10503_gb300 as M
    from paper_2410_10503_gb300 import build
    build.build()
    return M


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def call_static(mc, n, na, nb, rigid, x):
    """One mc_forward_static call on torch's current stream."""
    from paper_2410_10503_gb300 import _native as N
    L = mc.lib()
    geom = N.mc_geometry(n, na, nb)
    out = torch.empty((na, nb), dtype=torch.float32, device="cuda")
    err = ctypes.create_string_buffer(512)
    rig = None if rigid is None else np.ascontiguousarray(rigid, dtype=np.float64)
    st = L.mc_forward_static(ctypes.byref(geom), None if rig is None else rig.ctypes.data,
                             x.data_ptr(), out.data_ptr(), torch.cuda.current_stream().cuda_stream,
                             err, len(err))
    return st, err.value.decode(), out


def test_static_forward_matches_context_path_twice(mc):
    cases = [(128, 180, 183, 4, 101), (96, 90, 101, 3, 202)]
    for n, na, nb, N, seed in cases:                      # two calls in a row
        rig = S.rigid_motion(N, 6.0, 3.0, seed)
        ctx = mc.Context(n, na, nb, N, rigid=rig)
        x = torch.as_tensor(S.random_image(n, seed + 1), dtype=torch.float32, device="cuda")
        ref = ctx.forward(N - 1, x).cpu().numpy()
        st, msg, out = call_static(mc, n, na, nb, rig[N - 1], x)
        assert st == 0, msg
        assert rel_l2(out.cpu().numpy(), ref) <= TOL
        ctx.close()


def test_static_forward_without_motion_matches_project(mc):
    n, na, nb = 64, 60, 64
    ctx = mc.Context(n, na, nb, 1, rigid=np.zeros((1, 3)))
    x = torch.as_tensor(S.phantom(n, 6, 5, 3.0, 16.0), dtype=torch.float32, device="cuda")
    for _ in range(2):
        st, msg, out = call_static(mc, n, na, nb, None, x)
        assert st == 0, msg
        assert rel_l2(out.cpu().numpy(), ctx.project(x).cpu().numpy()) <= TOL
    ctx.close()


def test_static_forward_refuses_oversize_and_host_arrays(mc):
    x = torch.zeros((2048, 2048), dtype=torch.float32, device="cuda")
    st, msg, _ = call_static(mc, 2048, 4096, 4096, None, x)
    assert st == -1 and "scratch" in msg
    from paper_2410_10503_gb300 import _native as N
    geom = N.mc_geometry(16, 8, 23)
    xh = np.zeros((16, 16), np.float32)
    out = torch.empty((8, 23), dtype=torch.float32, device="cuda")
    err = ctypes.create_string_buffer(256)
    st = mc.lib().mc_forward_static(ctypes.byref(geom), None, xh.ctypes.data, out.data_ptr(), None,
                                    err, len(err))
    assert st == -1 and "device memory" in err.value.decode()


def status(mc):
    from paper_2410_10503_gb300 import _native as N  # noqa: F401
    err = ctypes.create_string_buffer(256)
    st = mc.lib().mc_forward_static_status(torch.cuda.current_stream().cuda_stream, err, len(err))
    return st, err.value.decode()


def test_static_forward_matches_oracle(mc):
    """A D x of the FP64 oracle (rigid motion and none), independent of the
    context path; <= 1e-5 relative L2 as for every float32 operator."""
    import oracle as O
    n, na, nb = 48, 60, 53
    g = O.Geometry(n, na, nb)
    rig = S.rigid_motion(3, 7.0, 4.0, 31)
    xh = S.random_image(n, 32)
    x = torch.as_tensor(xh, dtype=torch.float32, device="cuda")
    for rigid in (rig[2], None):
        st, msg, out = call_static(mc, n, na, nb, rigid, x)
        assert st == 0, msg
        x64 = x.cpu().numpy().astype(np.float64)
        ref = O.A(x64, g) if rigid is None else O.Ai(x64, O.Problem(g, O.Motion(rigid=rig), None, 1.0), 2)
        assert rel_l2(out.cpu().numpy(), ref) <= TOL
        assert status(mc) == (0, "")


def test_static_status_reports_a_wait_that_ran_out(mc):
    """With the test hook the projection's waits run out: the call itself
    returns MC_OK (the failure happens on the device), the status call
    reports MC_ETIMEOUT, and the next call without the hook is correct
    again."""
    n, na, nb = 64, 60, 64
    ctx = mc.Context(n, na, nb, 1, rigid=np.zeros((1, 3)))
    x = torch.as_tensor(S.phantom(n, 6, 5, 3.0, 16.0), dtype=torch.float32, device="cuda")
    os.environ["MC_STATIC_TEST_STALL"] = "1"
    try:
        st, msg, _ = call_static(mc, n, na, nb, None, x)
        assert st == 0, msg
        st, msg = status(mc)
        assert st == -4 and "ran out" in msg
    finally:
        del os.environ["MC_STATIC_TEST_STALL"]
    st, msg, out = call_static(mc, n, na, nb, None, x)
    assert st == 0, msg
    assert status(mc) == (0, "")
    assert rel_l2(out.cpu().numpy(), ctx.project(x).cpu().numpy()) <= TOL
    ctx.close()
