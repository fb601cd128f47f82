"""mc_forward_static, the allocation-free forward operator, against the
context path (mc_forward / mc_project) through the C ABI.

Some callers cannot allocate device memory (an allocator hook, a plugin with
a fixed memory budget, a host whose GPU memory already belongs to its own
pool); this entry point keeps all of its scratch in a fixed array built into
the library.  Two calls in a row (different geometry and motion) must both
match the existing entry points, which checks that the shared scratch is
reset between calls; sizes beyond the fixed array are refused on the host.
This file is collected last on purpose.
"""
import ctypes

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
