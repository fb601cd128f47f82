"""Checkpoint / resume of the solver state and host-simulated allocation
failure (the failure handling the method itself does not have)."""
import os
import time

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
    return W, P, sd, O.gate_norms2(P, iters=30, tol=1e-12)


def make(mc, W, P, norms, store="f32", subsets=1):
    ctx = mc.Context(W.n, W.n_angles, W.n_bins, W.n_gates, rigid=P.motion.rigid)
    ctx.set_data(P.d.astype(np.float32), P.alpha)
    ctx.set_storage(store)
    if subsets > 1:
        ctx.set_subsets(subsets)
        norms = O.block_norms2(P, subsets, iters=30, tol=1e-12)
    ctx.set_norms(norms)
    return ctx


@pytest.mark.parametrize("store,subsets", [("f32", 1), ("f16", 1), ("f32", 3)])
def test_interrupt_at_25_resumes_bit_identically(mc, prob, store, subsets):
    """Save at epoch 25, load into a fresh context, run 25 more: identical to
    50 uninterrupted epochs (iterate, trace of the resumed part, counter)."""
    W, P, sd, norms = prob
    full = make(mc, W, P, norms, store, subsets)
    x50, _ = full.spdhg_run(50, seed=sd["gates"])
    a = make(mc, W, P, norms, store, subsets)
    a.spdhg_run(25, seed=sd["gates"], x_out=False)
    state = a.save_state()
    x25, _ = a.spdhg_run(0, seed=sd["gates"])
    b = make(mc, W, P, norms, store, subsets)
    b.load_state(state)
    np.testing.assert_array_equal(b.spdhg_run(0, seed=sd["gates"])[0], x25)
    assert b.iteration() == 25 * W.n_gates * subsets
    x_resumed, _ = b.spdhg_run(25, seed=sd["gates"])
    np.testing.assert_array_equal(x_resumed, x50)
    # graph replay off after the load gives the same iterates too
    c = make(mc, W, P, norms, store, subsets)
    c.set_option(1, 0)
    c.load_state(state)
    np.testing.assert_array_equal(c.spdhg_run(25, seed=sd["gates"])[0], x50)


def test_load_state_rejects_mismatches(mc, prob):
    W, P, sd, norms = prob
    a = make(mc, W, P, norms)
    state = a.save_state()
    with pytest.raises(mc.MCError, match="storage"):
        make(mc, W, P, norms, store="bf16").load_state(state)
    with pytest.raises(mc.MCError, match="truncated"):
        a.load_state(state[:-8])
    with pytest.raises(mc.MCError, match="not a saved"):
        a.load_state(bytes(len(state)))
    other = mc.Context(W.n + 2, W.n_angles, W.n_bins, W.n_gates, rigid=P.motion.rigid)
    with pytest.raises(mc.MCError, match="geometry"):
        other.load_state(state)


def test_simulated_allocation_failure_is_reported_and_leaves_nothing(mc, prob):
    """Every device allocation of mc_create fails once in turn (MC_ENOMEM, a
    message, nothing left allocated); with exactly the creation's count the
    context is made and its next allocation fails instead."""
    W, P, sd, norms = prob
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    ctx = None
    try:
        for k in range(400):
            os.environ["MC_FAIL_ALLOC_AFTER"] = str(k)
            try:
                ctx = mc.Context(W.n, W.n_angles, W.n_bins, W.n_gates, rigid=P.motion.rigid)
                break
            except mc.MCError as e:
                assert e.status == -2 and "simulated allocation failure" in str(e), str(e)
        assert ctx is not None and k > 10
        with pytest.raises(mc.MCError, match="simulated allocation failure"):
            ctx.set_storage("f16")
        ctx.close()
    finally:
        del os.environ["MC_FAIL_ALLOC_AFTER"]
    torch.cuda.synchronize()
    assert abs(torch.cuda.mem_get_info()[0] - free0) <= 8 << 20
    ok = mc.Context(W.n, W.n_angles, W.n_bins, W.n_gates, rigid=P.motion.rigid)
    ok.set_storage("f16")
    ok.close()


@pytest.mark.parametrize("subsets", [1, 4])
def test_bounded_wait_running_out_is_reported_and_the_context_recovers(mc, prob, subsets):
    """The failure path of the device-side waits, without a fault: with
    MC_OPT_TEST_STALL the next forward's producer issues no copies, so its
    consumers' bounded ring waits run out; the run reports MC_ETIMEOUT, and
    afterwards the same context (reset) reproduces an undisturbed run bit for
    bit.  subsets=4 takes the banded forward."""
    from paper_2410_10503_gb300 import _native as N
    W, P, sd, norms = prob
    ref_ctx = make(mc, W, P, norms, subsets=subsets)
    ref, _ = ref_ctx.spdhg_run(3, seed=sd["gates"])
    ctx = make(mc, W, P, norms, subsets=subsets)
    ctx.set_option(N.MC_OPT_TEST_STALL, 1)
    t0 = time.perf_counter()
    with pytest.raises(mc.MCError) as e:
        ctx.spdhg_run(1, seed=sd["gates"])
    print(f"stalled epoch returned after {time.perf_counter() - t0:.3f} s")
    assert "MC_ETIMEOUT" in str(e.value)
    ctx.reset()
    x, _ = ctx.spdhg_run(3, seed=sd["gates"])
    np.testing.assert_array_equal(x, ref)


def test_wait_running_out_in_a_run_that_did_not_wait_is_reported_later(mc, prob):
    """A run with device (or no) outputs returns without waiting; a bounded
    wait that ran out in it is reported by mc_sync (and only once), and the
    reset context reproduces an undisturbed run."""
    from paper_2410_10503_gb300 import _native as N
    W, P, sd, norms = prob
    ref_ctx = make(mc, W, P, norms)
    ref, _ = ref_ctx.spdhg_run(2, seed=sd["gates"])
    ctx = make(mc, W, P, norms)
    ctx.set_option(N.MC_OPT_TEST_STALL, 1)
    x_dev = torch.empty((W.n, W.n), dtype=torch.float32, device="cuda")
    ctx.spdhg_run(1, seed=sd["gates"], x_out=x_dev)          # returns without waiting
    with pytest.raises(mc.MCError) as e:
        ctx.sync()
    assert "MC_ETIMEOUT" in str(e.value)
    ctx.sync()                                               # reported once
    ctx.reset()
    ctx.spdhg_run(2, seed=sd["gates"], x_out=x_dev)
    ctx.sync()
    np.testing.assert_array_equal(x_dev.cpu().numpy(), ref)
