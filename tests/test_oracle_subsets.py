"""Oracle: sampling over gates x angle subsets (the extension of Sec. IV).

Blocks j = i S + s pair gate i with the angles k = s (mod S).  Pins: the S
block operators of a gate add up to that gate's operator (normal operator,
squared residual), their adjoints pass the dot test, their norms bracket the
gate's, and block-sampled SPDHG reaches the x* of the unchanged objective
(dense/CG solve) at a per-epoch rate within the Theorem's l(kappa_S, N S)."""
import numpy as np
import pytest

import mc_synth as S
import oracle as O


def _problem(n=16, N=3, na=24, nb=25, kappa=70.0, seed=31):
    g = O.Geometry(n, na, nb)
    m = O.Motion(rigid=S.rigid_motion(N, 5.0, 1.5, seed=seed))
    xt = S.phantom(n, 4, seed=seed + 1, axis_lo=n / 8, axis_hi=n / 3)
    eps = S.noise(N, na, nb, seed=seed + 2)
    P = O.make_problem(g, m, xt, eps, alpha=1.0)
    nA = O.power_norm2(lambda v: O.At(O.A(v, g), g), (n, n))
    P.alpha = nA / kappa
    return P


@pytest.fixture(scope="module")
def prob():
    P = _problem()
    xs = O.solve_xstar(P, tol=1e-14)
    return P, xs, O.ystar(P, xs)


@pytest.mark.parametrize("Ssub", [1, 3, 5])
def test_blocks_add_up_to_the_gate_operator(prob, Ssub):
    P = prob[0]
    rng = np.random.default_rng(5)
    v = rng.standard_normal((P.geom.n, P.geom.n))
    for i in range(P.N):
        full = O.Ait(O.Ai(v, P, i), P, i)
        parts = sum(O.subset_adj(O.subset_op(v, P, i, Ssub, s), P, i, Ssub, s) for s in range(Ssub))
        assert np.linalg.norm(parts - full) <= 1e-12 * np.linalg.norm(full)
        res = sum(float(np.sum((O.subset_op(v, P, i, Ssub, s) - P.d[i][s::Ssub]) ** 2))
                  for s in range(Ssub))
        ref = float(np.sum((O.Ai(v, P, i) - P.d[i]) ** 2))
        assert abs(res - ref) <= 1e-12 * ref
    # subsets interleave: every angle in exactly one subset, ragged when S does not divide na
    allk = np.sort(np.concatenate([O.subset_angles(P.geom.na, Ssub, s) for s in range(Ssub)]))
    np.testing.assert_array_equal(allk, np.arange(P.geom.na))


def test_block_adjoint_dot_test(prob):
    P = prob[0]
    rng = np.random.default_rng(6)
    x = rng.standard_normal((P.geom.n, P.geom.n))
    for s in range(4):
        rows = O.subset_angles(P.geom.na, 4, s)
        y = rng.standard_normal((rows.size, P.geom.nb))
        lhs = float(np.sum(O.subset_op(x, P, 1, 4, s) * y))
        rhs = float(np.sum(x * O.subset_adj(y, P, 1, 4, s)))
        assert abs(lhs - rhs) <= 1e-13 * abs(lhs)


def test_block_norms_bracket_the_gate_norms(prob):
    P = prob[0]
    Ssub = 4
    nb2 = O.block_norms2(P, Ssub)
    ng2 = O.gate_norms2(P)
    assert nb2.shape == (P.N * Ssub + 1,)
    assert nb2[-1] == pytest.approx(ng2[-1], rel=1e-10)
    for i in range(P.N):
        blk = nb2[i * Ssub:(i + 1) * Ssub]
        # sum_s A_{i,s}^T A_{i,s} = A_i^T A_i:  ||A_i||^2 / S <= max_s ||A_{i,s}||^2 <= ||A_i||^2
        assert blk.max() <= ng2[i] * (1 + 1e-9)
        assert blk.max() >= ng2[i] / Ssub * (1 - 1e-9)
        assert blk.sum() >= ng2[i] * (1 - 1e-9)


def test_block_spdhg_reaches_xstar(prob):
    P, xs, ys = prob
    Ssub = 5                                   # ragged: 24 angles in subsets of 5 and 4
    nb2 = O.block_norms2(P, Ssub)
    st = O.step_sizes(nb2[:-1].max(), P.alpha, P.N, P.N * Ssub)
    r = O.spdhg(P, 120, st, seed=17, subsets=Ssub, x_star=xs, y_star=ys)
    assert np.linalg.norm(r.x - xs) <= 1e-8 * np.linalg.norm(xs)
    assert np.linalg.norm(r.y - ys) <= 1e-8 * np.linalg.norm(ys)
    zc = sum(O.Ait(r.y[i], P, i) for i in range(P.N))
    assert np.linalg.norm(r.z - zc) <= 1e-10 * np.linalg.norm(zc)
    assert r.gates.max() == P.N * Ssub - 1 and r.gates.min() == 0


def _observed_rate(traces, E):
    d = np.mean([[t[1] for t in tr] for tr in traces], axis=0)
    return (d[E] / d[E // 2]) ** (1.0 / (E - E // 2))


def test_block_rate_within_theorem_and_faster_per_epoch(prob):
    """Per-epoch contraction (mean of 8 seeds) <= l(kappa_S, N S) * 1.02, with
    kappa_S = max_j ||A_j||^2 / (alpha N); splitting angles (S = 4) contracts
    more per epoch (same operator work) than gate sampling alone."""
    P, xs, ys = prob
    N, E = P.N, 30
    obs = {}
    for Ssub in (1, 4):
        nb2 = O.block_norms2(P, Ssub)
        st = O.step_sizes(nb2[:-1].max(), P.alpha, N, N * Ssub)
        runs = [O.spdhg(P, E, st, seed=300 + k, subsets=Ssub, x_star=xs, y_star=ys)
                for k in range(8)]
        obs[Ssub] = _observed_rate([r.trace for r in runs], E)
        assert obs[Ssub] <= O.rate(st.kappa, N * Ssub) * 1.02, (Ssub, obs[Ssub])
    assert obs[4] < obs[1]
