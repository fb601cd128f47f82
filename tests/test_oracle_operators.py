"""Pins of the FP64 oracle's operators against facts fixed by geometry and
mathematics (not against the oracle itself).

A (Joseph ray transform) -- analytic chord of a disc, exact column/row sums at
0 and 90 degrees, the 90-degree rotation symmetry of the parallel-beam
transform.  A^T, D^T -- the dot-product (adjoint) identity.  D -- identity,
exact integer shifts and the exact 90-degree permutation.  Philox4x32-10 --
published known-answer vectors.
"""
import math
import os

import numpy as np
import pytest

import mc_synth as S
import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- Joseph A
@pytest.mark.parametrize("n,R", [(64, 20.0), (128, 40.0)])
def test_chord_of_disc(n, R):
    """(A x)(k, b) ~ 2 sqrt(R^2 - s_b^2) for a centred disc of radius R."""
    g = O.Geometry(n, 30, n + 9)
    y = O.A(S.disc_area_image(n, R), g)
    s = np.arange(g.nb) - 0.5 * (g.nb - 1)
    m = np.abs(s) < R - 2
    ref = 2.0 * np.sqrt(R * R - s[m] ** 2)
    rel = np.abs(y[:, m] - ref) / (2 * R)
    assert rel.max() < 1e-2
    assert np.sqrt(np.mean(rel ** 2)) < 3e-3


def test_chord_error_shrinks_with_resolution():
    """Doubling the resolution (disc scaled with it) halves the RMS error."""
    errs = []
    for n, R in [(64, 20.0), (128, 40.0), (256, 80.0)]:
        g = O.Geometry(n, 12, n + 9)
        y = O.A(S.disc_area_image(n, R), g)
        s = np.arange(g.nb) - 0.5 * (g.nb - 1)
        m = np.abs(s) < R - 2
        ref = 2.0 * np.sqrt(R * R - s[m] ** 2)
        errs.append(np.sqrt(np.mean(((y[:, m] - ref) / (2 * R)) ** 2)))
    assert errs[1] < 0.75 * errs[0] and errs[2] < 0.75 * errs[1]


def _half_sums(v, nb, n):
    """0.5 (v[c0] + v[c0+1]) with c0 = b - hb + h - 1/2 and zeros outside."""
    h, hb = 0.5 * (n - 1), 0.5 * (nb - 1)
    out = np.zeros(nb)
    for b in range(nb):
        c0 = int(round(b - hb + h - 0.5))
        for c in (c0, c0 + 1):
            if 0 <= c < n:
                out[b] += 0.5 * v[c]
    return out


@pytest.mark.parametrize("n,nb", [(16, 21), (32, 33), (10, 15)])
def test_zero_degrees_is_half_column_sums(n, nb):
    """phi = 0 with n even and nb odd: every ray lies midway between two
    columns, so the projection is the mean of two neighbouring column sums."""
    x = S.random_image(n, 1)
    y = O.A(x, O.Geometry(n, 8, nb))
    np.testing.assert_allclose(y[0], _half_sums(x.sum(axis=0), nb, n), rtol=0, atol=1e-12)


@pytest.mark.parametrize("n,nb", [(16, 21), (32, 33)])
def test_ninety_degrees_is_half_row_sums(n, nb):
    """phi = pi/2: rays are horizontal, midway between two rows."""
    x = S.random_image(n, 2)
    y = O.A(x, O.Geometry(n, 8, nb))
    np.testing.assert_allclose(y[4], _half_sums(x.sum(axis=1), nb, n), rtol=0, atol=1e-10)


@pytest.mark.parametrize("n,na,nb", [(16, 30, 23), (15, 18, 22)])
def test_rotation_by_90_degrees(n, na, nb):
    """Rotating the image by +90 degrees shifts the angle index by na/2; angles
    that wrap past pi also flip the detector (s -> -s).  na/4 is not an
    integer here, so no angle sits on the 45-degree driving-axis tie."""
    g = O.Geometry(n, na, nb)
    x = S.random_image(n, 3)
    y, yr = O.A(x, g), O.A(np.rot90(x), g)
    half = na // 2
    np.testing.assert_allclose(yr[:half], y[half:], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(yr[half:], y[:half, ::-1], rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("n,na,nb", [(16, 12, 23), (15, 20, 22), (32, 45, 40), (9, 4, 13)])
def test_ray_transform_adjoint_dot(n, na, nb):
    """<A x, y> = <x, A^T y>; A^T is a separate scatter implementation."""
    g = O.Geometry(n, na, nb)
    x = S.random_image(n, 4)
    y = S.random_sinogram(na, nb, 5)
    lhs = float(np.sum(O.A(x, g) * y))
    rhs = float(np.sum(x * O.At(y, g)))
    assert abs(lhs - rhs) <= 1e-13 * max(abs(lhs), 1.0) * 10


def test_ray_transform_adjoint_matches_dense_transpose():
    """Column j of A^T equals row j of A, built from unit vectors."""
    n, g = 8, O.Geometry(8, 6, 11)
    Am = O.dense_matrix(lambda e: O.A(e, g), n * n, (n, n))
    Atm = O.dense_matrix(lambda e: O.At(e, g), g.na * g.nb, (g.na, g.nb))
    np.testing.assert_allclose(Atm, Am.T, rtol=0, atol=1e-14)


def test_ray_outside_image_is_zero():
    """Bins far outside the image see nothing.  At 0 and 90 degrees the bins
    sample each line at unit spacing, so every pixel's hat weights sum to one
    and the mass per angle is exactly sum(x); elsewhere only approximately."""
    n = 16
    g = O.Geometry(n, 10, 41)
    x = S.random_image(n, 6)
    y = O.A(x, g)
    assert np.all(y[:, :3] == 0) and np.all(y[:, -3:] == 0)
    np.testing.assert_allclose(y[[0, 5]].sum(axis=1), x.sum(), rtol=1e-12)
    np.testing.assert_allclose(y.sum(axis=1), x.sum(), rtol=2e-2)


# ---------------------------------------------------------------- warp D
def test_warp_zero_motion_is_identity():
    n = 24
    x = S.random_image(n, 7)
    rig = O.Motion(rigid=np.zeros((1, 3)))
    fld = O.Motion(fields=np.zeros((1, 2, n, n), dtype=np.float32))
    np.testing.assert_array_equal(O.D(x, rig, 0, n), x)
    np.testing.assert_array_equal(O.D(x, fld, 0, n), x)
    np.testing.assert_array_equal(O.Dt(x, rig, 0, n), x)


def test_warp_integer_shift_is_exact_shift_with_zero_fill():
    """q = p + (tx, ty): (D x)[r, c] = x[r + ty, c + tx], zero outside."""
    n, tx, ty = 20, 2, -3
    x = S.random_image(n, 8)
    w = O.D(x, O.Motion(rigid=np.array([[0.0, tx, ty]])), 0, n)
    ref = np.zeros_like(x)
    for r in range(n):
        for c in range(n):
            if 0 <= r + ty < n and 0 <= c + tx < n:
                ref[r, c] = x[r + ty, c + tx]
    np.testing.assert_array_equal(w, ref)
    f = np.zeros((1, 2, n, n), dtype=np.float32)
    f[0, 0], f[0, 1] = tx, ty
    np.testing.assert_array_equal(O.D(x, O.Motion(fields=f), 0, n), ref)


def test_warp_quarter_turn_is_permutation():
    """phi = pi/2 about the centre (n even) maps pixel centres onto pixel
    centres: (D x)[r, c] = x[c, n-1-r], i.e. numpy rot90."""
    n = 16
    x = S.random_image(n, 9)
    w = O.D(x, O.Motion(rigid=np.array([[math.pi / 2, 0.0, 0.0]])), 0, n)
    np.testing.assert_allclose(w, np.rot90(x), rtol=0, atol=1e-12)


def test_warp_bilinear_half_pixel_shift():
    """A half-pixel shift averages neighbours: closed form of bilinear weights."""
    n = 12
    x = S.random_image(n, 10)
    w = O.D(x, O.Motion(rigid=np.array([[0.0, 0.5, 0.0]])), 0, n)
    ref = np.zeros_like(x)
    ref[:, :-1] = 0.5 * (x[:, :-1] + x[:, 1:])
    ref[:, -1] = 0.5 * x[:, -1]
    np.testing.assert_allclose(w, ref, rtol=0, atol=1e-15)


@pytest.mark.parametrize("kind", ["rigid", "field"])
def test_warp_adjoint_dot(kind):
    n = 32
    if kind == "rigid":
        m = O.Motion(rigid=np.array([[0.13, 1.7, -2.2]]))
    else:
        m = O.Motion(fields=S.rbf_fields(n, 2, seed=11, width=8.0, max_disp=3.0)[1:])
    x, v = S.random_image(n, 12), S.random_image(n, 13) - 0.5
    lhs = float(np.sum(O.D(x, m, 0, n) * v))
    rhs = float(np.sum(x * O.Dt(v, m, 0, n)))
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)


def test_gated_operator_adjoint_dot():
    """<A_i x, y> = <x, A_i^* y> for the composed per-gate operator."""
    n = 24
    g = O.Geometry(n, 20, 35)
    m = O.Motion(rigid=S.rigid_motion(3, 5.0, 3.0, seed=14))
    P = O.Problem(g, m, np.zeros((3, g.na, g.nb)), 1e-2)
    x, y = S.random_image(n, 15), S.random_sinogram(g.na, g.nb, 16)
    for i in range(3):
        lhs = float(np.sum(O.Ai(x, P, i) * y))
        rhs = float(np.sum(x * O.Ait(y, P, i)))
        assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


# ---------------------------------------------------------------- Philox
def _kat():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            v = [int(t, 16) for t in line.split()]
            rows.append((tuple(v[0:4]), tuple(v[4:6]), tuple(v[6:10])))
    return rows


@pytest.mark.parametrize("ctr,key,out", _kat())
def test_philox_known_answers(ctr, key, out):
    assert O.philox4x32_10(ctr, key) == out


def test_gate_draw_uniform():
    """Serial uniform sampling: all gates in range, frequencies ~ 1/N."""
    N, K = 10, 200000
    g = O.draw_gates(1234, 0, 0, K, N)
    assert g.min() >= 0 and g.max() < N
    cnt = np.bincount(g, minlength=N)
    chi2 = float(np.sum((cnt - K / N) ** 2 / (K / N)))
    assert chi2 < 33.7          # 99.99% quantile of chi^2 with 9 dof
    # counters are independent of how the sequence is split
    np.testing.assert_array_equal(O.draw_gates(1234, 0, 500, 100, N), g[500:600])


def test_gate_draw_nonuniform():
    p = np.array([0.5, 0.25, 0.125, 0.125])
    K = 200000
    g = O.draw_gates(99, 3, 0, K, 4, p=p)
    freq = np.bincount(g, minlength=4) / K
    np.testing.assert_allclose(freq, p, atol=5e-3)


# ---------------------------------------------------------------- field derivative
H = 2.0 ** -10          # finite-difference step (~1e-3), exact in float32


def _field_away_from_grid(n, seed, amp=2.0):
    """Dense field on a 2^-12 grid whose sample positions stay >= 0.05 px from
    grid lines, so that f +- H is exact in float32 and stays in one bilinear
    cell (where the central difference is exact)."""
    rng = np.random.default_rng(seed)
    f = rng.uniform(-amp, amp, size=(2, n, n))
    frac = f - np.floor(f)
    f = np.where(frac < 0.05, f + 0.05, f)
    f = np.where(frac > 0.95, f - 0.05, f)
    return (np.round(f * 4096.0) / 4096.0).astype(np.float32)


def test_field_vjp_matches_central_differences():
    """<g, d(D_u x)/du . e> against central differences of <g, D_u x>."""
    n = 12
    x = S.random_image(n, 31)
    g = S.random_image(n, 32) - 0.5
    f = _field_away_from_grid(n, 33)
    vjp = O.warp_field_vjp(x, g, f, n)
    rng = np.random.default_rng(34)
    for _ in range(16):
        ch, r, c = rng.integers(0, 2), rng.integers(0, n), rng.integers(0, n)
        fp, fm = f.copy(), f.copy()
        fp[ch, r, c] += H
        fm[ch, r, c] -= H
        lp = float(np.sum(g * O.D(x, O.Motion(fields=fp[None]), 0, n)))
        lm = float(np.sum(g * O.D(x, O.Motion(fields=fm[None]), 0, n)))
        assert abs((lp - lm) / (2 * H) - vjp[ch, r, c]) <= 1e-9 * (1 + abs(vjp[ch, r, c]))


def test_loss_field_gradient_directional_derivatives():
    """Gradient of N^-1 ||A D_u x - d||^2 w.r.t. u along random directions,
    against central differences (step 1e-3) of the oracle's loss."""
    n, N = 16, 2
    g = O.Geometry(n, 20, 23)
    f = np.stack([np.zeros((2, n, n), np.float32), _field_away_from_grid(n, 35, amp=1.5)])
    P = O.Problem(g, O.Motion(fields=f), S.random_sinogram(20, 23, 36)[None].repeat(N, 0), 1.0)
    x = S.random_image(n, 37)
    grad = O.loss_field_grad(x, P, 1)
    rng = np.random.default_rng(38)
    def loss(fi):
        Pq = O.Problem(g, O.Motion(fields=np.stack([f[0], fi])), P.d, 1.0)
        r = O.Ai(x, Pq, 1) - P.d[1]
        return float(np.sum(r * r)) / N
    for _ in range(6):
        # sign directions on a sparse support: f +- H e is exact in float32 and
        # stays in every cell; moving one component per pixel keeps the warped
        # image linear and the loss quadratic in H, so the central difference
        # equals the directional derivative
        e = rng.choice([-1.0, 1.0], size=(2, n, n)) * (rng.uniform(size=(2, n, n)) < 0.3)
        e[1][e[0] != 0] = 0.0      # one component per pixel: no bilinear cross term
        fd = (loss((f[1] + H * e).astype(np.float32)) - loss((f[1] - H * e).astype(np.float32))) / (2 * H)
        an = float(np.sum(grad * e))
        assert abs(fd - an) <= 1e-7 * (abs(an) + 1.0)
