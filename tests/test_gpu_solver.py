"""GPU SPDHG / PDHG against the FP64 oracle, through the C ABI.

Same data, same squared norms (so the same step sizes), same Philox gate
sequence: after 50 epochs the float32 iterate matches the oracle's to
<= 1e-4 relative L2.  Plus norms, objective, trace, determinism, graph replay
and resume."""
import numpy as np
import pytest

import mc_synth as S
import oracle as O

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def mc():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2410_10503_gb300 as M
    from paper_2410_10503_gb300 import build
    build.build()
    return M


def problem(W, kind="rigid"):
    sd = S.seeds(W.cid)
    g = O.Geometry(W.n, W.n_angles, W.n_bins)
    if kind == "rigid":
        m = O.Motion(rigid=S.rigid_motion(W.n_gates, W.max_rot_deg, W.max_shift, sd["motion"]))
    else:
        m = O.Motion(fields=S.rbf_fields(W.n, W.n_gates, sd["motion"], W.rbf_count,
                                         W.rbf_width, W.rbf_max_disp))
    xt = S.phantom(W.n, W.n_ellipses, sd["phantom"], W.axis_lo, W.axis_hi)
    eps = S.noise(W.n_gates, W.n_angles, W.n_bins, sd["noise"])
    return O.make_problem(g, m, xt, eps, W.alpha, W.noise_level), sd


def context(mc, P):
    g, m = P.geom, P.motion
    if m.rigid is not None:
        ctx = mc.Context(g.n, g.na, g.nb, P.N, rigid=m.rigid)
    else:
        ctx = mc.Context(g.n, g.na, g.nb, P.N, fields=m.fields)
    ctx.set_data(P.d.astype(np.float32), P.alpha)
    return ctx


@pytest.fixture(scope="module")
def rigid128(mc):
    """128^2, 180 x 183, N = 4 rigid gates (+-5 deg, +-3 px), alpha = 1e-2."""
    P, sd = problem(S.WORKLOADS["rigid128"])
    norms = O.gate_norms2(P, iters=30, tol=1e-13)
    return P, sd, norms


def test_norms_match_oracle(mc, rigid128):
    P, _, norms = rigid128
    ctx = context(mc, P)
    got = ctx.norms(max_iter=60, tol=1e-9)
    np.testing.assert_allclose(got, norms, rtol=1e-5)


def test_step_sizes_match_oracle(mc, rigid128):
    P, _, norms = rigid128
    ctx = context(mc, P)
    ctx.set_norms(norms)
    N = P.N
    for pd, st in [(False, O.step_sizes(norms[:N].max(), P.alpha, N, N)),
                   (True, O.step_sizes(norms[N], P.alpha, N, 1))]:
        s = ctx.steps(pdhg=pd)
        for key, ref in [("sigma", st.sigma[0]), ("tau", st.tau), ("theta", st.theta),
                         ("kappa", st.kappa)]:
            assert abs(s[key] - ref) <= 1e-12 * abs(ref)


def test_objective_matches_oracle(mc, rigid128):
    P, _, _ = rigid128
    ctx = context(mc, P)
    x = S.phantom(P.geom.n, 10, 5, 5, 40)
    assert abs(ctx.objective(x.astype(np.float32)) - O.objective(x, P)) <= 1e-5 * O.objective(x, P)


@pytest.fixture(scope="module")
def spdhg50(mc, rigid128):
    P, sd, norms = rigid128
    st = O.step_sizes(norms[:P.N].max(), P.alpha, P.N, P.N)
    return O.spdhg(P, 50, st, seed=sd["gates"], stream=0)


def test_spdhg_50_epochs_matches_oracle(mc, rigid128, spdhg50):
    P, sd, norms = rigid128
    ctx = context(mc, P)
    ctx.set_norms(norms)
    x, _ = ctx.spdhg_run(50, seed=sd["gates"])
    assert rel_l2(x, spdhg50.x) <= 1e-4
    assert ctx.iteration() == 50 * P.N


def test_pdhg_50_epochs_matches_oracle(mc, rigid128):
    P, _, norms = rigid128
    ctx = context(mc, P)
    ctx.set_norms(norms)
    x, _ = ctx.pdhg_run(50)
    ro = O.pdhg(P, 50, O.step_sizes(norms[P.N], P.alpha, P.N, 1))
    assert rel_l2(x, ro.x) <= 1e-4


def test_spdhg_field_motion_matches_oracle(mc):
    """Non-rigid gates (Gaussian-bump fields) at 64^2, 20 epochs."""
    W = S.WORKLOADS["rbf256"].scaled(n=64, n_angles=90, n_bins=93, n_gates=5, rbf_width=10.0,
                                     rbf_max_disp=3.0, n_ellipses=8, axis_lo=3.0, axis_hi=12.0,
                                     alpha=1e-2)
    P, sd = problem(W, kind="rbf")
    norms = O.gate_norms2(P, iters=30, tol=1e-13)
    ctx = context(mc, P)
    ctx.set_norms(norms)
    x, _ = ctx.spdhg_run(20, seed=sd["gates"])
    ro = O.spdhg(P, 20, O.step_sizes(norms[:P.N].max(), P.alpha, P.N, P.N), seed=sd["gates"])
    assert rel_l2(x, ro.x) <= 1e-4


def test_trace_matches_oracle_paper_regime(mc):
    """32^2 problem with kappa = ||A||^2/alpha = 70 (the paper's regime):
    relative error and saddle distance per epoch against the oracle's."""
    n, N = 32, 4
    W = S.WORKLOADS["rigid128"].scaled(n=n, n_angles=48, n_bins=47, n_gates=N, n_ellipses=5,
                                       axis_lo=3.0, axis_hi=10.0)
    P, sd = problem(W)
    nA = O.power_norm2(lambda v: O.At(O.A(v, P.geom), P.geom), (n, n))
    P.alpha = nA / 70.0
    xs = O.solve_xstar(P, tol=1e-13)
    ys = O.ystar(P, xs)
    norms = O.gate_norms2(P, iters=40, tol=1e-13)
    ctx = context(mc, P)
    ctx.set_norms(norms)
    ctx.set_reference(xs.astype(np.float32))
    E = 12
    x, tr = ctx.spdhg_run(E, seed=sd["gates"], trace=True)
    ro = O.spdhg(P, E, O.step_sizes(norms[:N].max(), P.alpha, N, N), seed=sd["gates"],
                 x_star=xs, y_star=ys)
    ref = np.array(ro.trace[1:])
    np.testing.assert_allclose(tr[:, 0], ref[:, 0], rtol=2e-3)
    np.testing.assert_allclose(tr[:, 1], ref[:, 1], rtol=5e-3)
    assert np.all(np.isnan(tr[:, 2]))
    # objective in the trace when asked for
    ctx.set_option(3, 1)
    _, tr2 = ctx.spdhg_run(1, seed=sd["gates"], trace=True)
    assert np.isfinite(tr2[0, 2])


def test_runs_are_deterministic_graph_or_not_and_resume(mc, rigid128):
    P, sd, norms = rigid128
    outs = []
    for graph in (1, 0):
        ctx = context(mc, P)
        ctx.set_norms(norms)
        ctx.set_option(1, graph)
        outs.append(ctx.spdhg_run(6, seed=sd["gates"])[0])
    np.testing.assert_array_equal(outs[0], outs[1])
    ctx = context(mc, P)
    ctx.set_norms(norms)
    ctx.spdhg_run(3, seed=sd["gates"], x_out=False)
    x_resumed, _ = ctx.spdhg_run(3, seed=sd["gates"])
    np.testing.assert_array_equal(x_resumed, outs[0])
    ctx.reset()
    np.testing.assert_array_equal(ctx.spdhg_run(6, seed=sd["gates"])[0], outs[0])
    # PDHG graph replay == plain launches
    pd = []
    for graph in (1, 0):
        ctx = context(mc, P)
        ctx.set_norms(norms)
        ctx.set_option(1, graph)
        pd.append(ctx.pdhg_run(3)[0])
    np.testing.assert_array_equal(pd[0], pd[1])


def test_device_and_host_outputs_agree(mc, rigid128):
    P, sd, norms = rigid128
    ctx = context(mc, P)
    ctx.set_norms(norms)
    xd = torch.empty((P.geom.n, P.geom.n), dtype=torch.float32, device="cuda")
    ctx.spdhg_run(2, seed=sd["gates"], x_out=xd)
    ctx.reset()
    xh, _ = ctx.spdhg_run(2, seed=sd["gates"])
    np.testing.assert_array_equal(xd.cpu().numpy(), xh)


def test_solve_normal_matches_oracle_xstar(mc):
    """GPU conjugate gradients (float32 operators, float64 inner products)
    reach the oracle's x* on a 48^2 problem in the paper's regime (kappa = 70)."""
    n, N = 48, 4
    W = S.WORKLOADS["rigid128"].scaled(n=n, n_angles=72, n_bins=71, n_gates=N, n_ellipses=6,
                                       axis_lo=3.0, axis_hi=14.0)
    P, sd = problem(W)
    nA = O.power_norm2(lambda v: O.At(O.A(v, P.geom), P.geom), (n, n))
    P.alpha = nA / 70.0
    xs = O.solve_xstar(P, tol=1e-13)
    ctx = context(mc, P)
    x, iters, rel = ctx.solve_normal(max_iter=400, tol=1e-6)
    assert rel <= 1e-6 and iters < 400
    assert rel_l2(x, xs) <= 1e-5


def test_motion_compensation_beats_no_mc(mc):
    """Sec. III: reconstructing gated data without motion compensation
    (D_i = identity for every gate) is blurred; the motion-compensated
    solution is closer to the true image.  Paper regime (kappa = 70), 64^2,
    N = 5 rigid gates of up to 8 degrees and 4 px."""
    n, N = 64, 5
    W = S.WORKLOADS["rigid128"].scaled(n=n, n_angles=90, n_bins=93, n_gates=N, n_ellipses=8,
                                       axis_lo=3.0, axis_hi=16.0, max_rot_deg=8.0, max_shift=4.0)
    P, sd = problem(W)
    xt = S.phantom(W.n, W.n_ellipses, sd["phantom"], W.axis_lo, W.axis_hi)
    nA = O.power_norm2(lambda v: O.At(O.A(v, P.geom), P.geom), (n, n))
    alpha = nA / 70.0
    errs = {}
    for label, rig in [("mc", P.motion.rigid), ("no_mc", np.zeros_like(P.motion.rigid))]:
        ctx = mc.Context(n, P.geom.na, P.geom.nb, N, rigid=rig)
        ctx.set_data(P.d.astype(np.float32), alpha)
        x, iters, rel = ctx.solve_normal(max_iter=300, tol=1e-6)
        errs[label] = rel_l2(x, xt)
        ctx.close()
    assert errs["mc"] < 0.8 * errs["no_mc"], errs
