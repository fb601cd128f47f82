"""Staged upload of the next data set (mc_stage_data / mc_commit_data): the
upload overlaps a run on the current data without disturbing it, and a
commit makes the context run exactly as after mc_set_data with that data."""
import numpy as np
import pytest

import mc_synth as S
import oracle as O

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def mc():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2410_10503_gb300 as M
    from paper_2410_10503_gb300 import build
    build.build()
    return M


@pytest.fixture(scope="module")
def prob():
    W = S.WORKLOADS["rigid128"].scaled(n=64, n_angles=90, n_bins=93, n_gates=4, n_ellipses=8,
                                       axis_lo=3.0, axis_hi=16.0)
    sd = S.seeds(W.cid)
    g = O.Geometry(W.n, W.n_angles, W.n_bins)
    m = O.Motion(rigid=S.rigid_motion(W.n_gates, W.max_rot_deg, W.max_shift, sd["motion"]))
    xt = S.phantom(W.n, W.n_ellipses, sd["phantom"], W.axis_lo, W.axis_hi)
    P = O.make_problem(g, m, xt, S.noise(W.n_gates, W.n_angles, W.n_bins, sd["noise"]), W.alpha,
                       W.noise_level)
    d1 = P.d.astype(np.float32)
    d2 = (0.9 * P.d + 0.01).astype(np.float32)
    return W, P, d1, d2, O.gate_norms2(P, iters=30, tol=1e-12)


def make(mc, W, P, d, norms, store="f32"):
    ctx = mc.Context(W.n, W.n_angles, W.n_bins, W.n_gates, rigid=P.motion.rigid)
    ctx.set_data(d, P.alpha)
    ctx.set_storage(store)
    ctx.set_norms(norms)
    return ctx


@pytest.mark.parametrize("store", ["f32", "f16"])
def test_staged_upload_overlaps_a_run_and_commits_like_set_data(mc, prob, store):
    W, P, d1, d2, norms = prob
    x_ref1, _ = make(mc, W, P, d1, norms, store).spdhg_run(2, seed=11)
    ref2 = make(mc, W, P, d1, norms, store)
    ref2.set_data(d2, P.alpha)
    x_ref2, _ = ref2.spdhg_run(3, seed=12)
    ctx = make(mc, W, P, d1, norms, store)
    ctx.stage_data(torch.from_numpy(d2).pin_memory())    # lands while the next run works on d1
    x1, _ = ctx.spdhg_run(2, seed=11)
    np.testing.assert_array_equal(x1, x_ref1)
    ctx.commit_data(P.alpha)
    assert ctx.iteration() == 0
    x2, _ = ctx.spdhg_run(3, seed=12)
    np.testing.assert_array_equal(x2, x_ref2)


def test_commit_needs_a_stage_and_takes_the_last_one(mc, prob):
    W, P, d1, d2, norms = prob
    ref = make(mc, W, P, d2, norms)
    x_ref, _ = ref.spdhg_run(3, seed=12)
    ctx = make(mc, W, P, d1, norms)
    with pytest.raises(mc.MCError) as e:
        ctx.commit_data(P.alpha)
    assert "MC_ESTATE" in str(e.value)
    ctx.stage_data(torch.zeros(d1.shape).pin_memory())
    ctx.stage_data(torch.from_numpy(d2).pin_memory())
    with pytest.raises(mc.MCError) as e:                  # refused: stays staged
        ctx.commit_data(-1.0)
    assert "MC_EINVAL" in str(e.value)
    ctx.commit_data(P.alpha)
    x, _ = ctx.spdhg_run(3, seed=12)
    np.testing.assert_array_equal(x, x_ref)
    with pytest.raises(mc.MCError):                       # consumed
        ctx.commit_data(P.alpha)


def test_stage_refuses_device_memory(mc, prob):
    W, P, d1, d2, norms = prob
    ctx = make(mc, W, P, d1, norms)
    dev = torch.zeros(d1.size, dtype=torch.float32, device="cuda")
    with pytest.raises(TypeError):
        ctx.stage_data(dev)
    assert mc.lib().mc_stage_data(ctx._h, dev.data_ptr()) == -1      # MC_EINVAL at the ABI
    assert mc.lib().mc_stage_data(ctx._h, None) == -1
