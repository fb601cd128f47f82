"""Sampling over gates x angle subsets on the GPU (mc_set_subsets) against
the oracle: block norms, the Philox block draw (bit-exact), and block-sampled
SPDHG iterates, for rigid and dense-field motion and for subset counts that
do and do not divide the number of angles."""
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


def problem(W, kind):
    sd = S.seeds(W.cid)
    g = O.Geometry(W.n, W.n_angles, W.n_bins)
    if kind == "rigid":
        m = O.Motion(rigid=S.rigid_motion(W.n_gates, W.max_rot_deg, W.max_shift, sd["motion"]))
    else:
        m = O.Motion(fields=S.rbf_fields(W.n, W.n_gates, sd["motion"], W.rbf_count, W.rbf_width,
                                         W.rbf_max_disp))
    xt = S.phantom(W.n, W.n_ellipses, sd["phantom"], W.axis_lo, W.axis_hi)
    eps = S.noise(W.n_gates, W.n_angles, W.n_bins, sd["noise"])
    return O.make_problem(g, m, xt, eps, W.alpha, W.noise_level), sd


def context(mc, P):
    g, m = P.geom, P.motion
    kw = dict(rigid=m.rigid) if m.rigid is not None else dict(fields=m.fields)
    ctx = mc.Context(g.n, g.na, g.nb, P.N, **kw)
    ctx.set_data(P.d.astype(np.float32), P.alpha)
    return ctx


CASES = {
    # 128^2, 180 x 183, N = 4 rigid, S = 4 (divides 180)
    "rigid128_S4": ("rigid128", "rigid", 4, dict()),
    # 64^2 dense fields, 90 angles, S = 7 (ragged: subsets of 13 and 12 angles)
    "rbf64_S7": ("rbf256", "rbf", 7, dict(n=64, n_angles=90, n_bins=93, n_gates=3, rbf_width=10.0,
                                          rbf_max_disp=3.0, n_ellipses=8, axis_lo=3.0,
                                          axis_hi=12.0, alpha=1e-2)),
    # 96^2, 160 x 137, N = 3 rigid, S = 16: eight line bands per subset launch
    # (the banded forward's group counters at their largest band count)
    "rigid96_S16": ("rigid128", "rigid", 16, dict(n=96, n_angles=160, n_bins=137, n_gates=3, n_ellipses=8,
                                                   axis_lo=4.0, axis_hi=24.0)),
}


@pytest.fixture(scope="module", params=list(CASES))
def case(request, mc):
    name, kind, Ssub, kw = CASES[request.param]
    W = S.WORKLOADS[name].scaled(**kw) if kw else S.WORKLOADS[name]
    P, sd = problem(W, kind)
    nb2 = O.block_norms2(P, Ssub, iters=40, tol=1e-13)
    return P, sd, Ssub, nb2


def test_block_norms_match_oracle(mc, case):
    P, _, Ssub, nb2 = case
    ctx = context(mc, P)
    ctx.set_subsets(Ssub)
    got = ctx.norms(max_iter=60, tol=1e-9)
    assert got.shape == (P.N * Ssub + 1,)
    np.testing.assert_allclose(got, nb2, rtol=1e-5)
    st = ctx.steps()
    ref = O.step_sizes(got[:-1].max(), P.alpha, P.N, P.N * Ssub)
    assert abs(st["kappa"] - ref.kappa) <= 1e-12 * ref.kappa
    assert abs(st["omega"] - ref.omega) <= 1e-12


def test_block_draw_is_bit_exact(mc, case):
    P, sd, Ssub, _ = case
    ctx = context(mc, P)
    ctx.set_subsets(Ssub)
    got = ctx.draw_gates(sd["gates"], 3, 1000, 4096)
    np.testing.assert_array_equal(got, O.draw_gates(sd["gates"], 3, 1000, 4096, P.N * Ssub))


def test_block_spdhg_matches_oracle(mc, case):
    """20 epochs (20 N S iterations) against the oracle's block SPDHG with the
    same norms and Philox stream; graph replay and plain launches agree."""
    P, sd, Ssub, nb2 = case
    E = 20
    ref = O.spdhg(P, E, O.step_sizes(nb2[:-1].max(), P.alpha, P.N, P.N * Ssub), seed=sd["gates"],
                  subsets=Ssub)
    outs = []
    for graph in (1, 0):
        ctx = context(mc, P)
        ctx.set_subsets(Ssub)
        with pytest.raises(mc.MCError, match="norms"):
            ctx.spdhg_run(1, seed=sd["gates"])
        ctx.set_norms(nb2)
        ctx.set_option(1, graph)
        x, _ = ctx.spdhg_run(E, seed=sd["gates"])
        assert ctx.iteration() == E * P.N * Ssub
        outs.append(x)
    assert rel_l2(outs[0], ref.x) <= 1e-4
    np.testing.assert_array_equal(outs[0], outs[1])


def test_subsets_one_restores_gate_sampling_and_errors(mc):
    W = S.WORKLOADS["rigid128"].scaled(n=48, n_angles=72, n_bins=71, n_ellipses=6, axis_lo=3.0,
                                       axis_hi=14.0)
    P, sd = problem(W, "rigid")
    norms = O.gate_norms2(P, iters=30, tol=1e-13)
    a = context(mc, P)
    a.set_subsets(5)
    a.set_subsets(1)
    a.set_norms(norms)
    b = context(mc, P)
    b.set_norms(norms)
    np.testing.assert_array_equal(a.spdhg_run(4, seed=sd["gates"])[0],
                                  b.spdhg_run(4, seed=sd["gates"])[0])
    for bad in (0, W.n_angles + 1):
        with pytest.raises(mc.MCError, match="subsets"):
            a.set_subsets(bad)
    # the full operators are untouched by the split
    a.set_subsets(6)
    x = S.random_image(W.n, 2).astype(np.float32)
    np.testing.assert_array_equal(a.forward(1, x), b.forward(1, x))


def test_subset_launch_shapes_and_autotune(mc, case):
    """The subset launches' band count and backprojection tile height
    (MC_OPT_SUBSET_BANDS / MC_OPT_SUBSET_ROWS) change results only within
    float32 rounding; mc_autotune with subsets picks the band count and keeps
    the norms, step sizes and iterates; bad values are refused."""
    from paper_2410_10503_gb300 import _native as N
    P, sd, Ssub, nb2 = case
    E = 10
    ref = O.spdhg(P, E, O.step_sizes(nb2[:-1].max(), P.alpha, P.N, P.N * Ssub), seed=sd["gates"],
                  subsets=Ssub)
    for bands, rows in ((1, 0), (3, 8), (8, 16), (2, 28)):
        ctx = context(mc, P)
        ctx.set_subsets(Ssub)
        ctx.set_norms(nb2)
        ctx.set_option(N.MC_OPT_SUBSET_BANDS, bands)      # tables rebuilt, norms kept
        ctx.set_option(N.MC_OPT_SUBSET_ROWS, rows)
        x, _ = ctx.spdhg_run(E, seed=sd["gates"])
        assert rel_l2(x, ref.x) <= 1e-4, (bands, rows)
        ctx.close()
    ctx = context(mc, P)
    ctx.set_subsets(Ssub)
    ctx.set_norms(nb2)
    x1, _ = ctx.spdhg_run(E // 2, seed=sd["gates"])
    steps = ctx.steps()
    ctx.autotune(reps=1)
    assert ctx.steps() == steps
    x, _ = ctx.spdhg_run(E - E // 2, seed=sd["gates"])      # continues from the kept iterates
    assert ctx.iteration() == E * P.N * Ssub
    assert rel_l2(x, ref.x) <= 1e-4
    for opt, bad in ((N.MC_OPT_SUBSET_BANDS, 9), (N.MC_OPT_SUBSET_BANDS, -1), (N.MC_OPT_SUBSET_ROWS, 5)):
        with pytest.raises(mc.MCError):
            ctx.set_option(opt, bad)
    ctx.close()


def test_two_part_chunks_in_subset_launches(mc):
    """At 512^2 the layouts keep the narrow guard and the forward streams
    16-line chunks sampled in two 8-line parts with 15 consumer warps; the
    subset launches run its banded instance.  64 angles x 529 bins, N = 2
    rigid gates, S = 4 subsets of 16 angles, 4 epochs against the oracle's
    block SPDHG, at 1 and 4 line bands."""
    import ctypes
    from paper_2410_10503_gb300 import _native as N
    W = S.WORKLOADS["rigid512"].scaled(n=512, n_angles=64, n_bins=529, n_gates=2)
    out = (ctypes.c_int32 * 10)()
    assert N.load().mc_plan_shapes(ctypes.byref(N.mc_geometry(W.n, W.n_angles, W.n_bins)), 152, out) == 0
    assert (out[0], out[3], out[4], out[9]) == (17, 16, 8, 15)       # guard, chunk, part, warps
    P, sd = problem(W, "rigid")
    Ssub, E = 4, 4
    nb2 = O.block_norms2(P, Ssub, iters=8)      # only sets the step sizes, which both sides share
    ref = O.spdhg(P, E, O.step_sizes(nb2[:-1].max(), P.alpha, P.N, P.N * Ssub), seed=sd["gates"],
                  subsets=Ssub)
    for bands in (1, 4):
        ctx = context(mc, P)
        ctx.set_subsets(Ssub)
        ctx.set_norms(nb2)
        ctx.set_option(N.MC_OPT_SUBSET_BANDS, bands)
        x, _ = ctx.spdhg_run(E, seed=sd["gates"])
        assert rel_l2(x, ref.x) <= 1e-4, bands
        ctx.close()
