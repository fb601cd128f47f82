"""Pins of the oracle's solver side against closed forms and direct solves.

prox maps -- scalar golden-section minimisation of the defining problems and
the Moreau identity (using the primal f_i as printed in Sec. II-A, not the
derived conjugate).  x* -- dense Cholesky of the normal equations on 32x32
images.  Algorithm 1 / PDHG -- convergence to that x*, observed per-epoch
rates against the Theorem's l(kappa, n) (Sec. II-B), SPDHG faster than PDHG.
Rate function -- closed values and the kappa >= 10 claim of Sec. II-B.
"""
import math

import numpy as np
import pytest
import scipy.linalg as sla

import mc_synth as S
import oracle as O


def golden_min(fun, lo, hi, tol=1e-12):
    gr = (math.sqrt(5.0) - 1.0) / 2.0
    a, b = lo, hi
    c, d = b - gr * (b - a), a + gr * (b - a)
    while abs(b - a) > tol * (1.0 + abs(a) + abs(b)):
        if fun(c) < fun(d):
            b = d
        else:
            a = c
        c, d = b - gr * (b - a), a + gr * (b - a)
    return 0.5 * (a + b)


@pytest.mark.parametrize("v,tau,alpha", [(1.3, 0.7, 0.2), (-2.0, 5.0, 1e-3), (0.4, 1e-2, 30.0)])
def test_prox_g_is_the_minimiser(v, tau, alpha):
    """prox_{tau g}(v) = argmin_u alpha u^2 + (u - v)^2 / (2 tau)."""
    u = golden_min(lambda u: alpha * u * u + (u - v) ** 2 / (2 * tau), -10, 10)
    assert abs(O.prox_g(np.array(v), tau, alpha) - u) < 1e-7 * (1 + abs(u))


@pytest.mark.parametrize("v,sigma,d,N", [(0.8, 0.3, 1.1, 4), (-1.5, 2.0, -0.4, 10), (3.0, 1e-3, 2.0, 20)])
def test_prox_fstar_by_moreau_identity(v, sigma, d, N):
    """prox_{sigma f*}(v) = v - sigma prox_{f/sigma}(v/sigma) with the primal
    f(w) = N^-1 (w - d)^2 as printed; prox_{f/sigma}(u) minimised numerically."""
    u = v / sigma
    w = golden_min(lambda w: (w - d) ** 2 / N + 0.5 * sigma * (w - u) ** 2, -1e4, 1e4)
    assert abs(O.prox_fstar(np.array(v), sigma, d, N) - (v - sigma * w)) < 1e-7 * (1 + abs(v))


def _small_problem(n=16, N=4, na=24, nb=25, kappa=70.0, seed=21):
    g = O.Geometry(n, na, nb)
    m = O.Motion(rigid=S.rigid_motion(N, 5.0, 1.5, seed=seed))
    xt = S.phantom(n, 4, seed=seed + 1, axis_lo=n / 8, axis_hi=n / 3)
    eps = S.noise(N, na, nb, seed=seed + 2)
    P = O.make_problem(g, m, xt, eps, alpha=1.0)
    nA = O.power_norm2(lambda v: O.At(O.A(v, g), g), (n, n))
    P.alpha = nA / kappa            # the paper's regime: kappa = ||A||^2/alpha
    return P


@pytest.fixture(scope="module")
def small70():
    P = _small_problem()
    xs = O.solve_xstar(P, tol=1e-14)
    return P, xs, O.ystar(P, xs), O.gate_norms2(P)


def test_xstar_matches_dense_cholesky():
    """CG on the normal equations equals a dense Cholesky solve of
    (alpha I + N^-1 sum A_i^T A_i) x = N^-1 sum A_i^T d_i on 32x32 images."""
    P = _small_problem(n=32, na=40, nb=47, kappa=500.0, seed=31)
    n, N = P.geom.n, P.N
    Am = [O.dense_matrix(lambda e, i=i: O.Ai(e, P, i), n * n, (n, n)) for i in range(N)]
    M = P.alpha * np.eye(n * n) + sum(a.T @ a for a in Am) / N
    rhs = sum(a.T @ P.d[i].reshape(-1) for i, a in enumerate(Am)) / N
    xd = sla.cho_solve(sla.cho_factor(M), rhs)
    xs = O.solve_xstar(P, tol=1e-14).reshape(-1)
    assert np.linalg.norm(xs - xd) <= 1e-10 * np.linalg.norm(xd)


def test_xstar_optimality_and_ystar(small70):
    """0 = 2 alpha x* + sum_i A_i^* y_i* with y_i* = grad f_i(A_i x*), and the
    objective's central-difference gradient equals 2 (M x - b)."""
    P, xs, ys, _ = small70
    res = 2 * P.alpha * xs + sum(O.Ait(ys[i], P, i) for i in range(P.N))
    assert np.linalg.norm(res) <= 1e-10 * np.linalg.norm(2 * P.alpha * xs)
    rng = np.random.default_rng(5)
    x = rng.uniform(size=xs.shape)
    v = rng.standard_normal(xs.shape)
    h = 1e-4
    fd = (O.objective(x + h * v, P) - O.objective(x - h * v, P)) / (2 * h)
    an = float(np.sum(2 * (O.normal_apply(x, P) - O.normal_rhs(P)) * v))
    assert abs(fd - an) <= 1e-7 * abs(an)


def test_power_iteration_matches_dense_eigenvalue(small70):
    P, _, _, nrm = small70
    n, N = P.geom.n, P.N
    Am = [O.dense_matrix(lambda e, i=i: O.Ai(e, P, i), n * n, (n, n)) for i in range(N)]
    for i in range(N):
        lam = np.linalg.eigvalsh(Am[i].T @ Am[i])[-1]
        assert abs(nrm[i] - lam) <= 1e-8 * lam
    K = np.concatenate(Am, axis=0)
    lam = np.linalg.eigvalsh(K.T @ K)[-1]
    assert abs(nrm[N] - lam) <= 1e-8 * lam


def test_step_sizes_balance_the_rate():
    """omega tau sigma ||A||^2 = 1/n and omega^n = l(kappa, n)."""
    for N, n in [(4, 4), (10, 1), (20, 20)]:
        st = O.step_sizes(1234.5, 1e-2, N, n)
        assert abs(st.omega * st.tau * st.sigma[0] * 1234.5 - 1.0 / n) < 1e-12
        assert abs(st.omega ** n - O.rate(st.kappa, n)) < 1e-12
        assert abs(st.kappa - 1234.5 / (1e-2 * N)) < 1e-9 * st.kappa


def test_spdhg_and_pdhg_reach_xstar(small70):
    P, xs, ys, nrm = small70
    N = P.N
    stS = O.step_sizes(nrm[:N].max(), P.alpha, N, N)
    stP = O.step_sizes(nrm[N], P.alpha, N, 1)
    rs = O.spdhg(P, 140, stS, seed=7, x_star=xs, y_star=ys)
    rp = O.pdhg(P, 200, stP, x_star=xs, y_star=ys)
    assert rs.trace[-1][0] < 1e-10
    assert rp.trace[-1][0] < 1e-10
    # dual iterates converge to y* too, and z = sum_i A_i^* y_i is kept exact
    assert np.linalg.norm(rs.y - ys) <= 1e-8 * np.linalg.norm(ys)
    zc = sum(O.Ait(rs.y[i], P, i) for i in range(N))
    assert np.linalg.norm(rs.z - zc) <= 1e-10 * np.linalg.norm(zc)


def _observed_rate(traces, E):
    d = np.mean([[t[1] for t in tr] for tr in traces], axis=0)
    return (d[E] / d[E // 2]) ** (1.0 / (E - E // 2))


@pytest.mark.parametrize("kappa", [70.0, 1000.0])
def test_observed_rates_within_theorem(kappa):
    """Per-epoch contraction of the saddle distance <= l(kappa^S, N) for SPDHG
    (mean over 8 seeds, the bound holds in expectation) and <= l(kappa^P, 1)
    for PDHG, with kappa from power-iteration norms; SPDHG is faster."""
    P = _small_problem(kappa=kappa)
    N = P.N
    xs = O.solve_xstar(P, tol=1e-14)
    ys = O.ystar(P, xs)
    nrm = O.gate_norms2(P)
    kS, kP = O.theorem_kappas(nrm, P.alpha, N)
    E = 40
    rp = O.pdhg(P, E, O.step_sizes(nrm[N], P.alpha, N, 1), x_star=xs, y_star=ys)
    stS = O.step_sizes(nrm[:N].max(), P.alpha, N, N)
    rs = [O.spdhg(P, E, stS, seed=100 + s, x_star=xs, y_star=ys) for s in range(8)]
    obsP = _observed_rate([rp.trace], E)
    obsS = _observed_rate([r.trace for r in rs], E)
    assert obsP <= O.rate(kP, 1) * 1.02
    assert obsS <= O.rate(kS, N) * 1.02
    assert obsS < obsP


def test_literal_algorithm_text_is_slower(small70):
    """The text as printed (step (i) with z^k, zbar accumulated on zbar^k)
    converges more slowly than the standard reading: kept as a negative test."""
    P, xs, ys, nrm = small70
    st = O.step_sizes(nrm[:P.N].max(), P.alpha, P.N, P.N)
    E = 30
    std = O.spdhg(P, E, st, seed=3, x_star=xs, y_star=ys)
    lit = O.spdhg(P, E, st, seed=3, x_star=xs, y_star=ys, literal=True)
    assert lit.trace[-1][1] > 10 * std.trace[-1][1]


def test_rate_function_closed_values():
    assert O.rate(0.0, 1) == 0.0
    assert abs(O.rate(3.0, 1) - 1.0 / 3.0) < 1e-15
    assert abs(O.rate(8.0, 1) - 0.5) < 1e-15
    assert abs(O.rate(8.0, 2) - 0.5625) < 1e-15          # (1 - 1/4)^2
    # n -> infinity: exp(-2 / (1 + sqrt(1 + kappa)))
    assert abs(O.rate(24.0, 1e7) - math.exp(-2.0 / 6.0)) < 1e-7


def test_kappa_ge_10_claim_brute_force():
    """Sec. II-B: for kappa >= 10, l(kappa/N, N) < l(kappa, 1) for all N >= 2;
    below that the claim can fail (e.g. kappa = 5, N = 2)."""
    for kappa in np.geomspace(10.0, 1e6, 400):
        for N in range(2, 201):
            assert O.rate(kappa / N, N) < O.rate(kappa, 1)
    assert O.rate(5.0 / 2, 2) > O.rate(5.0, 1)


def test_theorem_kappas():
    nrm = np.array([2.0, 3.0, 2.5, 10.0])
    kS, kP = O.theorem_kappas(nrm, 0.5, 3)
    assert kS == 3.0 / 1.5 and kP == 10.0 / 1.5


def test_spdhg_nonuniform_sampling_reaches_xstar(small70):
    """Serial sampling with P(i) = p_i (Algorithm 1 step (ii)): the increment
    weighted by theta/p_i and steps of the uniform rule with n = 1/min p_i
    (omega tau sigma ||A_i||^2 = min p <= p_i) still reach x* and y*; the
    draw follows p."""
    P, xs, ys, nrm = small70
    N = P.N
    p = np.array([0.4, 0.3, 0.2, 0.1])
    st = O.step_sizes(nrm[:N].max(), P.alpha, N, 1.0 / p.min())
    assert abs(st.omega * st.tau * st.sigma[0] * nrm[:N].max() - p.min()) < 1e-12
    r = O.spdhg(P, 260, st, seed=11, p=p, x_star=xs, y_star=ys)
    assert r.trace[-1][0] < 1e-9
    assert np.linalg.norm(r.y - ys) <= 1e-7 * np.linalg.norm(ys)
    freq = np.bincount(r.gates, minlength=N) / len(r.gates)
    np.testing.assert_allclose(freq, p, atol=0.04)


def test_make_problem_noise_scale():
    """d_i - A_i x_true = eps_i with eps_i ~ N(0, sigma^2 / N) i.i.d. per bin
    and sigma = 1% of the largest clean value over ALL gates and bins
    (Sec. II-A; the variance sigma^2/N of the configurations).  Each gate's
    empirical variance must match sigma^2/N within a 5-sigma chi^2 bound; the
    gates' own maxima differ by far more than that bound, so a per-gate
    maximum, or sigma in place of sigma/sqrt(N), fails."""
    n, na, nb, N = 32, 60, 47, 4
    g = O.Geometry(n, na, nb)
    rig = np.array([[0.0, 0.0, 0.0], [0.1, 9.0, 0.0], [-0.2, -10.0, 6.0], [0.05, 0.0, -11.0]])
    m = O.Motion(rigid=rig)
    xt = np.zeros((n, n))
    xt[4:12, 20:28] = 1.0          # bright block near one edge: shifts cut it differently
    xt[16:30, 4:18] = 0.3
    eps = S.noise(N, na, nb, seed=77)
    P = O.make_problem(g, m, xt, eps, alpha=1.0, noise_level=0.01)
    clean = np.stack([O.A(O.D(xt, m, i, n), g) for i in range(N)])
    sigma = 0.01 * clean.max()
    var_expected = sigma ** 2 / N
    M = na * nb
    bound = 5.0 * math.sqrt(2.0 / M)
    per_gate_max = clean.reshape(N, -1).max(axis=1)
    # the pin discriminates: per-gate maxima differ from the global one
    assert per_gate_max.min() < (1.0 - 4 * bound) * per_gate_max.max()
    for i in range(N):
        r = (P.d[i] - clean[i]).ravel()
        v = float(np.mean(r * r))
        assert abs(v / var_expected - 1.0) <= bound, (i, v / var_expected)
