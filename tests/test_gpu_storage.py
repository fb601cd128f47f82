"""Binary16 / bfloat16 storage of the data and the dual (MC_OPT_STORAGE) on
the GPU against the oracle's emulation of the same storage.

The kernel computes each new y_i in float32 and rounds it on store; the
oracle computes in float64, rounds to float32, then to the storage type.
The two roundings differ only where the float32 projection error (~1e-6
relative) straddles a rounding boundary, so a small fraction of stored
values differ by one storage unit; the iterates then differ by far less
than one unit u (2^-11 for binary16, 2^-8 for bfloat16), the tolerance used
here.  The float32 path stays at its own bar."""
import numpy as np
import pytest

import mc_synth as S
import oracle as O

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

U = {"f16": 2.0 ** -11, "bf16": 2.0 ** -8}


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


@pytest.fixture(scope="module")
def rigid128():
    W = S.WORKLOADS["rigid128"]
    sd = S.seeds(W.cid)
    g = O.Geometry(W.n, W.n_angles, W.n_bins)
    m = O.Motion(rigid=S.rigid_motion(W.n_gates, W.max_rot_deg, W.max_shift, sd["motion"]))
    xt = S.phantom(W.n, W.n_ellipses, sd["phantom"], W.axis_lo, W.axis_hi)
    P = O.make_problem(g, m, xt, S.noise(W.n_gates, W.n_angles, W.n_bins, sd["noise"]), W.alpha,
                       W.noise_level)
    # the data as the GPU holds it (float32), so both sides round the same values
    P.d = P.d.astype(np.float32).astype(np.float64)
    return P, sd, O.gate_norms2(P, iters=30, tol=1e-13)


def context(mc, P, norms):
    ctx = mc.Context(P.geom.n, P.geom.na, P.geom.nb, P.N, rigid=P.motion.rigid)
    ctx.set_data(P.d.astype(np.float32), P.alpha)
    ctx.set_norms(norms)
    return ctx


@pytest.mark.parametrize("store", ["f16", "bf16"])
def test_spdhg_with_reduced_storage_matches_oracle(mc, rigid128, store):
    P, sd, norms = rigid128
    E = 50
    ref = O.spdhg(P, E, O.step_sizes(norms[:P.N].max(), P.alpha, P.N, P.N), seed=sd["gates"],
                  store=store)
    ctx = context(mc, P, norms)
    ctx.set_storage(store)
    x, _ = ctx.spdhg_run(E, seed=sd["gates"])
    assert rel_l2(x, ref.x) <= U[store], rel_l2(x, ref.x)
    # the storage changes the iterate by more than the GPU/oracle difference
    f32 = O.spdhg(P, E, O.step_sizes(norms[:P.N].max(), P.alpha, P.N, P.N), seed=sd["gates"])
    assert rel_l2(ref.x, f32.x) > rel_l2(x, ref.x)


@pytest.mark.parametrize("store", ["f16", "bf16"])
def test_pdhg_with_reduced_storage_matches_oracle(mc, rigid128, store):
    P, sd, norms = rigid128
    E = 30
    ref = O.pdhg(P, E, O.step_sizes(norms[P.N], P.alpha, P.N, 1), store=store)
    ctx = context(mc, P, norms)
    ctx.set_storage(store)
    x, _ = ctx.pdhg_run(E)
    assert rel_l2(x, ref.x) <= U[store], rel_l2(x, ref.x)


def test_switching_storage_carries_the_state(mc, rigid128):
    """f32 -> f16 mid-run equals the oracle run with y rounded once at the
    switch and stored as binary16 afterwards; back to f32 continues."""
    P, sd, norms = rigid128
    ctx = context(mc, P, norms)
    ctx.spdhg_run(5, seed=sd["gates"], x_out=False)
    ctx.set_storage("f16")
    ctx.spdhg_run(5, seed=sd["gates"], x_out=False)
    ctx.set_storage("f32")
    x, _ = ctx.spdhg_run(5, seed=sd["gates"])
    assert np.all(np.isfinite(x)) and ctx.iteration() == 15 * P.N
    b = context(mc, P, norms)
    xb, _ = b.spdhg_run(15, seed=sd["gates"])
    assert 0 < rel_l2(x, xb) <= U["f16"]
    with pytest.raises(mc.MCError, match="storage"):
        ctx.set_option(4, 3)
