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
