"""Oracle: reduced-precision storage of the data d and the dual y.

Pins: bfloat16 rounding against a brute-force nearest-value search with the
ties-to-even rule, binary16 at its boundary values; the data-quantisation
floor against its closed-form bound ||x*(d_h) - x*(d)|| <= ||d_h - d|| /
(2 sqrt(alpha N)) (from H^-1 A^T/N with H = alpha I + A^T A / N, whose
singular values are s / (N^(1/2) (alpha + s^2/N)) <= 1 / (2 sqrt(alpha N))),
and SPDHG with stored y reaching x*(d_h) to within a few rounding units."""
import copy

import numpy as np
import pytest

import mc_synth as S
import oracle as O


def _bf16_brute(v32):
    """Nearest bfloat16 by trying the two bracketing candidates."""
    out = np.empty_like(v32)
    for k, v in enumerate(v32):
        u = int(np.float32(v).view(np.uint32))
        lo = u & 0xFFFF0000
        hi = lo + 0x10000
        fl = float(np.uint32(lo).view(np.float32))
        fh = float(np.uint32(hi).view(np.float32))
        dl, dh = abs(float(v) - fl), abs(fh - float(v))
        if dl < dh or (dl == dh and ((lo >> 16) & 1) == 0):
            out[k] = fl
        else:
            out[k] = fh
    return out


def test_bf16_rounding_matches_brute_force_and_ties_to_even():
    rng = np.random.default_rng(1)
    v = np.concatenate([rng.standard_normal(3000) * 10.0 ** rng.integers(-8, 8, 3000),
                        np.array([1 + 2 ** -8, 1 + 3 * 2 ** -8, 1 + 2 ** -8 + 2 ** -20, -(1 + 2 ** -8),
                                  2.0 ** -126, 3.0e38])]).astype(np.float32)
    got = O.round_storage(v, "bf16")
    np.testing.assert_array_equal(got, _bf16_brute(v).astype(np.float64))
    assert list(got[-6:-2]) == [1.0, 1.015625, 1.0078125, -1.0]
    # results are bfloat16 values: the low 16 bits of their binary32 are zero
    assert np.all(got.astype(np.float32).view(np.uint32) & 0xFFFF == 0)
    normal = np.abs(v) >= 2.0 ** -126
    assert np.all(np.abs(got - v)[normal] <= 2.0 ** -8 * np.abs(v.astype(np.float64))[normal])


def test_f16_boundary_values():
    r = O.round_storage(np.array([1 + 2 ** -11, 1 + 3 * 2 ** -11, 65504.0, 2.0 ** -24, 2.0 ** -26]), "f16")
    assert list(r) == [1.0, 1 + 2 ** -9, 65504.0, 2.0 ** -24, 0.0]
    assert O.round_storage(np.array([0.1]), "f32")[0] == float(np.float32(0.1))


def _problem():
    n, N, na, nb = 16, 4, 24, 25
    g = O.Geometry(n, na, nb)
    m = O.Motion(rigid=S.rigid_motion(N, 5.0, 1.5, seed=31))
    xt = S.phantom(n, 4, seed=32, axis_lo=n / 8, axis_hi=n / 3)
    P = O.make_problem(g, m, xt, S.noise(N, na, nb, seed=33), alpha=1.0)
    P.alpha = O.power_norm2(lambda v: O.At(O.A(v, g), g), (n, n)) / 70.0
    return P


@pytest.fixture(scope="module")
def prob():
    P = _problem()
    return P, O.solve_xstar(P, tol=1e-14), O.gate_norms2(P)


@pytest.mark.parametrize("store,u", [("f16", 2.0 ** -11), ("bf16", 2.0 ** -8)])
def test_storage_floor_within_bound(prob, store, u):
    P, xs, nrm = prob
    Ph = copy.copy(P)
    Ph.d = O.round_storage(P.d, store)
    e = np.linalg.norm(Ph.d - P.d)
    assert e <= u * np.linalg.norm(P.d) + 2.0 ** -25 * np.sqrt(P.d.size)
    xh = O.solve_xstar(Ph, tol=1e-14)
    floor = np.linalg.norm(xh - xs)
    assert floor <= e / (2.0 * np.sqrt(P.alpha * P.N))
    assert floor > 0
    # SPDHG with stored d and y settles within a few rounding units of x*(d_h)
    st = O.step_sizes(nrm[:P.N].max(), P.alpha, P.N, P.N)
    r = O.spdhg(P, 100, st, seed=5, store=store, x_star=xs)
    assert np.linalg.norm(r.x - xh) <= 4 * u * np.linalg.norm(xs)
    zc = sum(O.Ait(r.y[i], P, i) for i in range(P.N))
    assert np.linalg.norm(r.z - zc) <= 1e-10 * np.linalg.norm(zc)
    # the stored dual holds representable values only
    np.testing.assert_array_equal(O.round_storage(r.y, store), r.y)


def test_f32_storage_is_a_plain_rounding(prob):
    P, xs, nrm = prob
    st = O.step_sizes(nrm[:P.N].max(), P.alpha, P.N, P.N)
    a = O.spdhg(P, 40, st, seed=5)
    b = O.spdhg(P, 40, st, seed=5, store="f32")
    assert np.linalg.norm(a.x - b.x) <= 1e-6 * np.linalg.norm(a.x)
