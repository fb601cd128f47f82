"""Many independent slices in one batched run (mc_batch_spdhg_run): every
slice equals its own mc_spdhg_run bit for bit, one slice is checked against
the oracle, and a slice without step sizes is reported by index."""
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


def slice_problem(W):
    sd = S.seeds(W.cid)
    g = O.Geometry(W.n, W.n_angles, W.n_bins)
    if W.motion == "rigid":
        m = O.Motion(rigid=S.rigid_motion(W.n_gates, W.max_rot_deg, W.max_shift, sd["motion"]))
    else:
        m = O.Motion(fields=S.rbf_fields(W.n, W.n_gates, sd["motion"], W.rbf_count, W.rbf_width,
                                         W.rbf_max_disp))
    xt = S.phantom(W.n, W.n_ellipses, sd["phantom"], W.axis_lo, W.axis_hi)
    eps = S.noise(W.n_gates, W.n_angles, W.n_bins, sd["noise"])
    return O.make_problem(g, m, xt, eps, 1e-2, W.noise_level), sd


def make_ctx(mc, P, norms, subsets=1):
    m = P.motion
    kw = dict(rigid=m.rigid) if m.rigid is not None else dict(fields=m.fields)
    ctx = mc.Context(P.geom.n, P.geom.na, P.geom.nb, P.N, **kw)
    ctx.set_data(P.d.astype(np.float32), P.alpha)
    if subsets > 1:
        ctx.set_subsets(subsets)
    ctx.set_norms(norms)
    return ctx


@pytest.fixture(scope="module")
def slices():
    """Three slices of different sizes, gate counts and motion kinds (the
    mixed-size batch recipe at small sides), one with angle subsets."""
    ws = S.slice_batch(3, seed=6100, sides=(48, 64, 40))
    out = []
    for j, W in enumerate(ws):
        W = W.scaled(n_gates=3 + j)
        P, sd = slice_problem(W)
        sub = 3 if j == 2 else 1
        nrm = O.block_norms2(P, sub, iters=30, tol=1e-12) if sub > 1 else O.gate_norms2(P, 30, 1e-12)
        out.append((W, P, sd, nrm, sub))
    return out


def test_batch_equals_separate_runs_and_oracle(mc, slices):
    E = 6
    batch = [make_ctx(mc, P, nrm, sub) for _, P, _, nrm, sub in slices]
    mc.batch_spdhg_run(batch, E, seeds=[sd["gates"] for _, _, sd, _, _ in slices])
    xs = []
    for (W, P, sd, nrm, sub), ctx in zip(slices, batch):
        assert ctx.iteration() == E * P.N * sub
        own = make_ctx(mc, P, nrm, sub)
        x_own, _ = own.spdhg_run(E, seed=sd["gates"])
        x_b, _ = ctx.spdhg_run(0, seed=sd["gates"])           # read x^K without running
        np.testing.assert_array_equal(x_b, x_own)
        xs.append(x_b)
    W, P, sd, nrm, sub = slices[1]
    ref = O.spdhg(P, E, O.step_sizes(nrm[:P.N].max(), P.alpha, P.N, P.N), seed=sd["gates"])
    assert rel_l2(xs[1], ref.x) <= 1e-4


def test_batch_reports_the_failing_slice(mc, slices):
    W, P, sd, nrm, _ = slices[0]
    good = make_ctx(mc, P, nrm)
    bad = mc.Context(P.geom.n, P.geom.na, P.geom.nb, P.N, rigid=P.motion.rigid)
    bad.set_data(P.d.astype(np.float32), P.alpha)            # no norms: no step sizes
    with pytest.raises(mc.MCError, match="norms"):
        mc.batch_spdhg_run([good, bad], 1, seeds=[1, 2])


# ---- mc_batch: one launch per stage over all slices --------------------------
@pytest.fixture(scope="module")
def merged_slices():
    """Four slices of different sizes, gate counts and motion kinds (gate
    sampling only), plus a larger slice whose forward and backprojection take
    other launch shapes (4 lines per chunk; its own rows per thread)."""
    ws = S.slice_batch(4, seed=6200, sides=(48, 64, 40, 56))
    out = []
    for j, W in enumerate(ws):
        W = W.scaled(n_gates=3 + j)
        P, sd = slice_problem(W)
        out.append((W, P, sd, O.gate_norms2(P, 30, 1e-12)))
    return out


def big_slice(mc):
    """n = 560 (4 lines per chunk), 60 angles, rigid, 3 gates: compared with
    its own run only (no oracle at this size)."""
    W = S.WORKLOADS["rigid128"].scaled(n=560, n_angles=60, n_bins=577, n_gates=3, n_ellipses=12,
                                       axis_lo=10.0, axis_hi=60.0)
    sd = S.seeds(W.cid)
    rig = S.rigid_motion(3, 4.0, 3.0, sd["motion"])
    ctx = mc.Context(W.n, W.n_angles, W.n_bins, 3, rigid=rig)
    xt = torch.as_tensor(S.phantom(W.n, 12, sd["phantom"], 10.0, 60.0), dtype=torch.float32, device="cuda")
    d = torch.stack([ctx.forward(i, xt) for i in range(3)])
    ctx.set_data(d, 1e-2)
    ctx.set_norms(np.array([2.0e4, 2.0e4, 2.0e4, 6.0e4]))
    return ctx, d, rig




def test_merged_batch_equals_separate_runs_and_oracle(mc, merged_slices):
    E = 4
    ctxs = [make_ctx(mc, P, nrm) for _, P, _, nrm in merged_slices]
    big, d_big, rig_big = big_slice(mc)
    ctxs.append(big)
    seeds = [sd["gates"] for _, _, sd, _ in merged_slices] + [777]
    n3 = merged_slices[3][1].N                        # slice 3 samples its gates non-uniformly
    ps = [None, None, None, np.linspace(1.0, 2.0, n3) / np.linspace(1.0, 2.0, n3).sum(), None]
    with mc.Batch(ctxs) as b:
        b.run(2, seeds, ps=ps)            # two runs in a row continue the state
        b.run(E - 2, seeds, ps=ps)
    for j, ((W, P, sd, nrm), ctx) in enumerate(zip(merged_slices, ctxs)):
        assert ctx.iteration() == E * P.N
        own = make_ctx(mc, P, nrm)
        x_own, _ = own.spdhg_run(E, seed=sd["gates"], p=ps[j])
        x_b, _ = ctx.spdhg_run(0, seed=sd["gates"], p=ps[j])
        np.testing.assert_array_equal(x_b, x_own)
        own.close()
    own = mc.Context(560, 60, 577, 3, rigid=rig_big)
    own.set_data(d_big, 1e-2)
    own.set_norms(np.array([2.0e4, 2.0e4, 2.0e4, 6.0e4]))
    x_own, _ = own.spdhg_run(E, seed=777)
    x_b, _ = big.spdhg_run(0, seed=777)
    np.testing.assert_array_equal(x_b, x_own)
    # one slice against the FP64 oracle
    W, P, sd, nrm = merged_slices[1]
    ref = O.spdhg(P, E, O.step_sizes(nrm[:P.N].max(), P.alpha, P.N, P.N), seed=sd["gates"])
    x1, _ = ctxs[1].spdhg_run(0, seed=sd["gates"])
    assert rel_l2(x1, ref.x) <= 1e-4
    for c in ctxs:
        c.close()


def test_merged_batch_reports_the_failing_slice(mc, merged_slices):
    W, P, sd, nrm = merged_slices[0]
    good = make_ctx(mc, P, nrm)
    bad = mc.Context(P.geom.n, P.geom.na, P.geom.nb, P.N, rigid=P.motion.rigid
                     if P.motion.rigid is not None else np.zeros((P.N, 3)))
    bad.set_data(P.d.astype(np.float32), P.alpha)            # no norms: no step sizes
    with mc.Batch([good, bad]) as b:
        with pytest.raises(mc.MCError, match="slice 1"):
            b.run(1, seeds=[1, 2])
    sub = make_ctx(mc, P, O.block_norms2(P, 2, iters=10, tol=1e-8), subsets=2)
    with pytest.raises(mc.MCError):
        mc.Batch([good, sub])


def test_merged_batch_refuses_changed_launch_shapes(mc, merged_slices):
    W, P, sd, nrm = merged_slices[1]
    a = make_ctx(mc, P, nrm)
    W2, P2, sd2, nrm2 = merged_slices[2]
    c = make_ctx(mc, P2, nrm2)
    from paper_2410_10503_gb300 import _native as N
    with mc.Batch([a, c]) as b:
        b.run(1, seeds=[1, 2])
        # new forward tables after the batch was made (a chunk size other than
        # the current one, so that the change does not depend on timings)
        lc = 8 if a.shapes()["lines_per_chunk"] != 8 else 16
        a.set_option(N.MC_OPT_FORWARD_LINES, lc)
        with pytest.raises(mc.MCError, match="launch shapes"):
            b.run(1, seeds=[1, 2])
    with mc.Batch([a, c]) as b:             # a new batch takes them
        b.run(1, seeds=[1, 2])
        rows = 8 if c.shapes()["rows_per_thread"] != 8 else 14
        c.set_option(N.MC_OPT_BACKPROJECT_ROWS, rows)      # so does a shape option
        with pytest.raises(mc.MCError, match="launch shapes"):
            b.run(1, seeds=[1, 2])
    a.close()
    c.close()


def test_one_slice_batch_follows_new_step_sizes(mc, merged_slices):
    """A batch of one slice runs the one-slice kernels on its arguments by
    value (16-iteration graphs): a run after new step sizes must use them, and
    every run equals the slice's own runs."""
    W, P, sd, nrm = merged_slices[0]
    ctx = make_ctx(mc, P, nrm)
    own = make_ctx(mc, P, nrm)
    E = 40 // P.N + 1                                   # more than 16 iterations: the graphs replay
    with mc.Batch([ctx]) as b:
        b.run(E, [sd["gates"]])
        own.spdhg_run(E, seed=sd["gates"])
        for c in (ctx, own):
            c.set_norms(np.asarray(nrm) * 1.7)          # new sigma, tau (theta stays 1)
        b.run(E, [sd["gates"]])
        x_own, _ = own.spdhg_run(E, seed=sd["gates"])
    x_b, _ = ctx.spdhg_run(0, seed=sd["gates"])
    assert ctx.iteration() == 2 * E * P.N
    np.testing.assert_array_equal(x_b, x_own)
    ctx.close()
    own.close()


def test_merged_batch_with_tall_tiles_and_two_part_chunks(mc):
    """A 512^2 slice (16-line chunks in two 8-line parts, 28-row backprojection
    tiles) merged with a 96^2 slice (whole 16-line chunks, short tiles): each
    stage runs one launch per shape class between a fork and a join; each
    slice equals its own runs bit for bit."""
    def make(n, na, nb, N, seed, norms=None):
        rig = S.rigid_motion(N, 6.0, 4.0, seed)
        ctx = mc.Context(n, na, nb, N, rigid=rig)
        xt = torch.as_tensor(S.phantom(n, 8, seed + 1, n / 16 + 0.5, n / 4 + 1), dtype=torch.float32,
                             device="cuda")
        d = torch.stack([ctx.forward(i, xt) for i in range(N)])
        ctx.set_data(d, 1e-2)
        norms = ctx.norms(max_iter=10, tol=1e-4) * 1.05 if norms is None else norms
        ctx.set_norms(norms)
        return ctx, norms
    shapes = {512: (24, 529, 3, 7100, 11), 96: (30, 101, 4, 7200, 12)}
    made = {n: make(n, *v[:4]) for n, v in shapes.items()}
    with mc.Batch([made[512][0], made[96][0]]) as b:
        b.run(3, seeds=[shapes[512][4], shapes[96][4]])
    for n, (ctx, norms) in made.items():
        na, nb, N, seed, gseed = shapes[n]
        own, _ = make(n, na, nb, N, seed, norms)
        x_own, _ = own.spdhg_run(3, seed=gseed)
        x_b, _ = ctx.spdhg_run(0, seed=gseed)
        np.testing.assert_array_equal(x_b, x_own)
        own.close()
        ctx.close()
