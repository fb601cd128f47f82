"""GPU parity of every operator kernel against the FP64 oracle, called
through the C ABI.  Tolerance: 1e-5 relative L2 per float32 operator
application; the transpose pair passes the float32 dot test to ~1e-6;
integer work (gate draw) is bit-exact."""
import math

import numpy as np
import pytest

import mc_synth as S
import oracle as O

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = 1e-5


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def cuda(a):
    return torch.as_tensor(np.asarray(a, dtype=np.float32)).cuda().contiguous()


def host(t):
    return t.detach().cpu().numpy().astype(np.float64)


@pytest.fixture(scope="module")
def mc():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2410_10503_gb300 as M
    from paper_2410_10503_gb300 import build
    build.build()
    return M


GEOMS = [
    (2, 1, 1), (3, 2, 4), (9, 4, 13), (16, 8, 23), (37, 41, 53), (64, 60, 64),
    (100, 36, 141), (128, 180, 183),
]


def _rigid(N, seed, rot=5.0, shift=3.0):
    return S.rigid_motion(N, rot, shift, seed)


@pytest.mark.parametrize("n,na,nb", GEOMS)
def test_project_matches_oracle(mc, n, na, nb):
    g = O.Geometry(n, na, nb)
    ctx = mc.Context(n, na, nb, 1, rigid=np.zeros((1, 3)))
    for x in (S.phantom(n, 6, 1, n / 16 + 0.5, n / 4 + 1), S.random_image(n, 2) - 0.5):
        y = host(ctx.project(cuda(x)))
        assert rel_l2(y, O.A(x, g)) <= TOL


@pytest.mark.parametrize("n,na,nb", GEOMS)
def test_backproject_matches_oracle(mc, n, na, nb):
    g = O.Geometry(n, na, nb)
    ctx = mc.Context(n, na, nb, 1, rigid=np.zeros((1, 3)))
    y = S.random_sinogram(na, nb, 3)
    x = host(ctx.backproject(cuda(y)))
    assert rel_l2(x, O.At(y, g)) <= TOL


# the limits of mc_create (n <= 2048, n_angles and n_bins <= 8192), each with
# the other sizes small enough for the oracle: the largest image with a wide
# ragged detector, the most angles, the most bins
LIMIT_GEOMS = [(2048, 5, 2900), (16, 8192, 23), (64, 7, 8192)]


@pytest.mark.parametrize("n,na,nb", LIMIT_GEOMS)
def test_operators_at_size_limits(mc, n, na, nb):
    g = O.Geometry(n, na, nb)
    rig = _rigid(2, 31, rot=8.0, shift=6.0)
    ctx = mc.Context(n, na, nb, 2, rigid=rig)
    P = O.Problem(g, O.Motion(rigid=rig), np.zeros((2, na, nb)), 1.0)
    x = S.phantom(n, 6, 32, n / 16 + 0.5, n / 4 + 1)
    y = S.random_sinogram(na, nb, 33)
    assert rel_l2(host(ctx.project(cuda(x))), O.A(x, g)) <= TOL
    assert rel_l2(host(ctx.backproject(cuda(y))), O.At(y, g)) <= TOL
    assert rel_l2(host(ctx.forward(1, cuda(x))), O.Ai(x, P, 1)) <= TOL
    assert rel_l2(host(ctx.adjoint(1, cuda(y))), O.Ait(y, P, 1)) <= TOL


@pytest.mark.parametrize("kind", ["rigid", "field"])
@pytest.mark.parametrize("n", [16, 37, 128])
def test_warp_and_transpose_match_oracle(mc, kind, n):
    N = 3
    if kind == "rigid":
        rig = _rigid(N, 5, rot=8.0, shift=6.0)
        m = O.Motion(rigid=rig)
        ctx = mc.Context(n, 4, n + 3, N, rigid=rig)
    else:
        f = S.rbf_fields(n, N, seed=6, width=max(2.0, n / 8), max_disp=max(1.5, n / 16))
        m = O.Motion(fields=f)
        ctx = mc.Context(n, 4, n + 3, N, fields=cuda(f))
    x = S.random_image(n, 7)
    v = S.random_image(n, 8) - 0.5
    for i in range(N):
        assert rel_l2(host(ctx.warp(i, cuda(x))), O.D(x, m, i, n)) <= TOL
        assert rel_l2(host(ctx.warp_adjoint(i, cuda(v))), O.Dt(v, m, i, n)) <= TOL


def test_zero_motion_warp_is_exact_identity(mc):
    n = 40
    ctx = mc.Context(n, 4, 43, 2, rigid=np.zeros((2, 3)))
    x = cuda(S.random_image(n, 9))
    assert torch.equal(ctx.warp(1, x), x)
    assert torch.equal(ctx.warp_adjoint(1, x), x)


@pytest.mark.parametrize("kind", ["rigid", "field"])
def test_gated_forward_adjoint_match_oracle(mc, kind):
    n, na, nb, N = 128, 180, 183, 4
    g = O.Geometry(n, na, nb)
    if kind == "rigid":
        rig = _rigid(N, 10)
        m = O.Motion(rigid=rig)
        ctx = mc.Context(n, na, nb, N, rigid=rig)
    else:
        f = S.rbf_fields(n, N, seed=11, width=20.0, max_disp=4.0)
        m = O.Motion(fields=f)
        ctx = mc.Context(n, na, nb, N, fields=f)
    P = O.Problem(g, m, np.zeros((N, na, nb)), 1.0)
    x = S.phantom(n, 10, 12, 5, 40)
    xr = S.random_image(n, 13) - 0.5
    y = S.random_sinogram(na, nb, 14)
    for i in range(N):
        assert rel_l2(host(ctx.forward(i, cuda(x))), O.Ai(x, P, i)) <= TOL
        assert rel_l2(host(ctx.forward(i, cuda(xr))), O.Ai(xr, P, i)) <= TOL
        assert rel_l2(host(ctx.adjoint(i, cuda(y))), O.Ait(y, P, i)) <= TOL


def test_float32_dot_test(mc):
    """<A_i x, y> = <x, A_i^* y> with both sides from the GPU kernels."""
    n, na, nb, N = 128, 180, 183, 3
    rig = _rigid(N, 15)
    ctx = mc.Context(n, na, nb, N, rigid=rig)
    x = S.random_image(n, 16)
    y = S.random_sinogram(na, nb, 17)
    for i in range(N):
        ax = host(ctx.forward(i, cuda(x)))
        aty = host(ctx.adjoint(i, cuda(y)))
        lhs, rhs = float(np.sum(ax * y)), float(np.sum(x * aty))
        assert abs(lhs - rhs) <= 2e-6 * math.sqrt(np.sum(ax ** 2) * np.sum(y ** 2))


def test_headline_size_operators(mc):
    """512^2 image, 720 angles x 729 bins, N = 10 rigid gates (the benchmark
    workload), full outputs against the oracle."""
    n, na, nb, N = 512, 720, 729, 10
    g = O.Geometry(n, na, nb)
    rig = S.rigid_motion(N, 8.0, 6.0, seed=2002)
    ctx = mc.Context(n, na, nb, N, rigid=rig)
    P = O.Problem(g, O.Motion(rigid=rig), np.zeros((N, na, nb)), 1.0)
    x = S.phantom(n, 40, 1002)
    y = S.random_sinogram(na, nb, 18)
    i = 7
    assert rel_l2(host(ctx.forward(i, cuda(x))), O.Ai(x, P, i)) <= TOL
    assert rel_l2(host(ctx.adjoint(i, cuda(y))), O.Ait(y, P, i)) <= TOL


def test_host_and_device_pointers_agree(mc):
    n, na, nb = 64, 60, 64
    rig = _rigid(2, 19)
    ctx = mc.Context(n, na, nb, 2, rigid=rig)
    x = S.random_image(n, 20).astype(np.float32)
    y = S.random_sinogram(na, nb, 21).astype(np.float32)
    np.testing.assert_array_equal(ctx.forward(1, x), host(ctx.forward(1, cuda(x))).astype(np.float32))
    np.testing.assert_array_equal(ctx.adjoint(1, y), host(ctx.adjoint(1, cuda(y))).astype(np.float32))


def test_operators_are_deterministic(mc):
    n, na, nb = 96, 90, 101
    rig = _rigid(2, 22)
    ctx = mc.Context(n, na, nb, 2, rigid=rig)
    x, y = cuda(S.random_image(n, 23)), cuda(S.random_sinogram(na, nb, 24))
    assert torch.equal(ctx.forward(1, x), ctx.forward(1, x))
    assert torch.equal(ctx.adjoint(1, y), ctx.adjoint(1, y))


def test_gate_draw_bit_exact(mc):
    ctx = mc.Context(8, 4, 9, 10, rigid=np.zeros((10, 3)))
    for seed, stream, k0 in [(4002, 0, 0), (12345678901, 3, 2**32 - 5), (7, 1, 10**9)]:
        got = ctx.draw_gates(seed, stream, k0, 5000)
        np.testing.assert_array_equal(got, O.draw_gates(seed, stream, k0, 5000, 10))


def test_invalid_gate_and_state_errors(mc):
    ctx = mc.Context(16, 8, 23, 2, rigid=np.zeros((2, 3)))
    with pytest.raises(mc.MCError) as e:
        ctx.forward(2, cuda(np.zeros((16, 16))))
    assert "MC_EINVAL" in str(e.value)
    with pytest.raises(mc.MCError) as e:
        ctx.spdhg_run(1, seed=1)
    assert "MC_ESTATE" in str(e.value)
    with pytest.raises(mc.MCError):
        ctx.set_data(np.zeros(2 * 8 * 23, np.float32), alpha=-1.0)


def test_autotune_keeps_parity(mc):
    """mc_autotune picks launch shapes from its candidate sets; the tuned
    operators still meet the FP64 oracle, and an item split alone changes no
    bit of the forward."""
    n, na, nb, N = 128, 180, 183, 3
    rig = _rigid(N, 21)
    ctx = mc.Context(n, na, nb, N, rigid=rig)
    P = O.Problem(O.Geometry(n, na, nb), O.Motion(rigid=rig), np.zeros((N, na, nb)), 1.0)
    x = S.phantom(n, 10, 22, 5, 40)
    y = S.random_sinogram(na, nb, 23)
    t = ctx.autotune(reps=2)
    assert t["lines_per_chunk"] in (2, 4, 8, 16) and t["rows_per_thread"] in (4, 8, 14, 16, 28)
    assert ctx.shapes()["lines_per_chunk"] == t["lines_per_chunk"]
    assert ctx.shapes()["rows_per_thread"] == t["rows_per_thread"]
    assert t["group_slots"] in (2, 4, 8) and t["items_per_block"] >= 1
    for i in range(N):
        assert rel_l2(host(ctx.forward(i, cuda(x))), O.Ai(x, P, i)) <= TOL
        assert rel_l2(host(ctx.adjoint(i, cuda(y))), O.Ait(y, P, i)) <= TOL
    fresh = mc.Context(n, na, nb, N, rigid=rig)
    if t["lines_per_chunk"] == 16:     # the creation-time chunk at 128^2 (wide guard, 3-stage ring)
        np.testing.assert_array_equal(host(ctx.forward(1, cuda(x))), host(fresh.forward(1, cuda(x))))


def test_shared_load_peak_is_plausible(mc):
    """mc_measure_shared_load_peak: conflict-free 64-bit shared loads deliver
    at most the data path's 128 B per clock per SM, and a healthy GPU gets
    close to it; the clock it reports matches bytes/s over bytes/clk."""
    r = mc.shared_load_peak(reps=20)
    assert r is not None
    assert 96.0 <= r["bytes_per_clk_per_sm"] <= 130.0, r
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    ghz = r["bytes_per_s"] / (r["bytes_per_clk_per_sm"] * sms) / 1e9
    assert abs(ghz - r["sm_ghz"]) <= 0.05 * r["sm_ghz"], r


# forward chunk sizes (MC_OPT_FORWARD_LINES), each against the oracle: small
# images get layouts with the wide guard and whole 16-line chunks (384^2: a
# 3-stage ring, 96^2 and 256^2); 512^2 keeps the narrow guard, where a 16-line
# chunk is sampled in two clamped 8-line parts
@pytest.mark.parametrize("n,na,nb", [(512, 20, 517), (384, 24, 401), (256, 45, 300), (96, 30, 101)])
@pytest.mark.parametrize("lc", [2, 4, 8, 16])
def test_forward_chunk_sizes_match_oracle(mc, n, na, nb, lc):
    from paper_2410_10503_gb300 import _native as N
    g = O.Geometry(n, na, nb)
    rig = _rigid(2, 41, rot=8.0, shift=6.0)
    ctx = mc.Context(n, na, nb, 2, rigid=rig)
    ctx.set_option(N.MC_OPT_FORWARD_LINES, lc)
    sh = ctx.shapes()
    two_parts = lc == 16 and sh["guard"] == 17
    assert sh["lines_per_chunk"] == lc and sh["lines_per_part"] == (8 if two_parts else lc)
    assert sh["consumer_warps"] == (15 if two_parts else 23)
    P = O.Problem(g, O.Motion(rigid=rig), np.zeros((2, na, nb)), 1.0)
    x = S.phantom(n, 6, 42, n / 16 + 0.5, n / 4 + 1)
    y = S.random_sinogram(na, nb, 43)
    assert rel_l2(host(ctx.project(cuda(x))), O.A(x, g)) <= TOL
    assert rel_l2(host(ctx.forward(1, cuda(x))), O.Ai(x, P, 1)) <= TOL
    assert rel_l2(host(ctx.adjoint(1, cuda(y))), O.Ait(y, P, 1)) <= TOL
    ctx.close()


@pytest.mark.parametrize("n,na,nb", [(16, 8, 23), (96, 30, 101), (384, 24, 401), (512, 20, 517),
                                     (520, 8, 537), (768, 12, 785), (1024, 6, 1041), (2048, 5, 2900)])
def test_context_shapes_match_plan(mc, n, na, nb):
    """A new context uses the shapes mc_plan_shapes computes on the host for
    its geometry and this GPU's SM count, and they drive its launches: the
    projection at those shapes matches the oracle."""
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    ctx = mc.Context(n, na, nb, 1, rigid=np.zeros((1, 3)))
    assert ctx.shapes() == mc.plan_shapes(n, na, nb, sms)
    x = S.phantom(n, 6, 44, n / 16 + 0.5, n / 4 + 1)
    assert rel_l2(host(ctx.project(cuda(x))), O.A(x, O.Geometry(n, na, nb))) <= TOL
    ctx.close()


def test_forward_chunk_size_refusals(mc):
    from paper_2410_10503_gb300 import _native as N
    ctx = mc.Context(520, 8, 40, 1, rigid=np.zeros((1, 3)))   # 520 lines: not whole 16-line chunks
    for bad in (16, 3, 32):
        with pytest.raises(mc.MCError):
            ctx.set_option(N.MC_OPT_FORWARD_LINES, bad)
    ctx.set_option(N.MC_OPT_FORWARD_LINES, 8)
    ctx.close()


# backprojection tile heights (MC_OPT_BACKPROJECT_ROWS), each against the
# oracle: 28-row tiles run two blocks per SM with more registers per thread
@pytest.mark.parametrize("n,na,nb", [(512, 20, 517), (96, 30, 101)])
@pytest.mark.parametrize("rows", [4, 8, 14, 16, 28])
def test_backprojection_tile_heights_match_oracle(mc, n, na, nb, rows):
    from paper_2410_10503_gb300 import _native as N
    g = O.Geometry(n, na, nb)
    rig = _rigid(2, 51, rot=8.0, shift=6.0)
    ctx = mc.Context(n, na, nb, 2, rigid=rig)
    ctx.set_option(N.MC_OPT_BACKPROJECT_ROWS, rows)
    assert ctx.shapes()["rows_per_thread"] == rows
    P = O.Problem(g, O.Motion(rigid=rig), np.zeros((2, na, nb)), 1.0)
    y = S.random_sinogram(na, nb, 52)
    assert rel_l2(host(ctx.backproject(cuda(y))), O.At(y, g)) <= TOL
    assert rel_l2(host(ctx.adjoint(1, cuda(y))), O.Ait(y, P, 1)) <= TOL
    for bad in (0, 12, 32):
        with pytest.raises(mc.MCError):
            ctx.set_option(N.MC_OPT_BACKPROJECT_ROWS, bad)
    ctx.close()
