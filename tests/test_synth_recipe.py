"""The seeded synthetic inputs (mc_synth) have the recipe the design states:
the workloads' sizes and motion ranges, the seed scheme, the batched-slices
mix, and the generators' ranges and determinism.  These stand in for the
paper's walnut and chest slices (Sec. III), which are not available."""
import numpy as np
import pytest

import mc_synth as S


def test_workload_table():
    W = S.WORKLOADS
    want = {
        "rigid128": (128, 180, 183, 4, "rigid", 10, 1e-2),
        "rigid512": (512, 720, 729, 10, "rigid", 40, 1e-3),
        "rbf512": (512, 720, 729, 20, "rbf", 40, 1e-3),
        "rbf256": (256, 360, 365, 8, "rbf", 20, 1e-3),
    }
    for name, (n, na, nb, N, kind, ell, alpha) in want.items():
        w = W[name]
        assert (w.n, w.n_angles, w.n_bins, w.n_gates, w.motion, w.n_ellipses, w.alpha) == \
            (n, na, nb, N, kind, ell, alpha), name
    assert (W["rigid128"].max_rot_deg, W["rigid128"].max_shift) == (5.0, 3.0)
    assert (W["rigid512"].max_rot_deg, W["rigid512"].max_shift) == (8.0, 6.0)
    for name in ("rbf512", "rbf256"):
        assert (W[name].rbf_count, W[name].rbf_max_disp) == (16, 8.0)
    assert len({w.cid for w in W.values()}) == len(W)          # distinct seeds per workload


def test_seed_scheme():
    assert S.seeds(2) == {"phantom": 1002, "motion": 2002, "noise": 3002, "gates": 4002}
    assert S.seeds(2, run=3)["gates"] == 4005


def test_rigid_motion_ranges_and_rest_gate():
    m = S.rigid_motion(200, 8.0, 6.0, seed=2002)
    assert m.shape == (200, 3) and m.dtype == np.float64
    assert np.all(m[0] == 0.0)                                   # gate 0 at rest
    assert np.abs(m[1:, 0]).max() <= np.deg2rad(8.0)
    assert np.abs(m[1:, 1:]).max() <= 6.0
    # uniform draws: the extremes come close to the bounds, the mean near 0
    assert np.abs(m[1:, 0]).max() > 0.9 * np.deg2rad(8.0)
    assert abs(m[1:, 1:].mean()) < 0.6
    assert np.array_equal(m, S.rigid_motion(200, 8.0, 6.0, seed=2002))
    assert not np.array_equal(m, S.rigid_motion(200, 8.0, 6.0, seed=2003))
    assert np.all(S.rigid_motion(1, 8.0, 6.0, seed=1) == 0.0)


def test_rbf_fields_peak_displacement():
    n, N = 48, 4
    f = S.rbf_fields(n, N, seed=7, count=16, width=n / 12.8, max_disp=8.0)
    assert f.shape == (N, 2, n, n) and f.dtype == np.float32
    assert np.all(f[0] == 0.0)
    for g in range(1, N):
        mag = np.sqrt(f[g, 0].astype(np.float64) ** 2 + f[g, 1].astype(np.float64) ** 2)
        assert mag.max() == pytest.approx(8.0, rel=1e-6)        # scaled to the stated maximum
    assert np.array_equal(f, S.rbf_fields(n, N, seed=7, count=16, width=n / 12.8, max_disp=8.0))


def test_phantom_support_and_values():
    n = 128
    x = S.phantom(n, 10, seed=1001, axis_lo=5.0, axis_hi=40.0)
    assert x.shape == (n, n) and x.dtype == np.float64
    assert x.min() >= 0.0 and x.max() > 0.0
    # every centre lies within 0.35 n of the image centre and every semi-axis
    # is at most axis_hi, so nothing lies beyond 0.35 n + 40 px
    h = 0.5 * (n - 1)
    c = np.arange(n) - h
    X, Y = np.meshgrid(c, c)
    assert np.all(x[np.hypot(X, Y) > 0.35 * n + 40.0] == 0.0)
    # additive ellipses of intensity U[0, 1]: at most 10 overlap
    assert x.max() <= 10.0
    assert np.array_equal(x, S.phantom(n, 10, seed=1001, axis_lo=5.0, axis_hi=40.0))


def test_disc_area_image_integral():
    # covered fraction per pixel: the sum is the disc's area within the
    # supersampling's resolution
    a = S.disc_area_image(64, 20.0, supersample=16)
    assert a.min() >= 0.0 and a.max() <= 1.0
    assert a.sum() == pytest.approx(np.pi * 20.0 ** 2, rel=2e-3)


def test_noise_and_test_arrays():
    e = S.noise(3, 40, 50, seed=3002)
    assert e.shape == (3, 40, 50)
    assert abs(e.mean()) < 0.05 and abs(e.var() - 1.0) < 0.05     # standard normals, 6000 draws
    x = S.random_image(32, 1)
    assert x.shape == (32, 32) and x.min() >= 0.0 and x.max() < 1.0
    assert S.random_sinogram(7, 9, 2).shape == (7, 9)


def test_slice_batch_mix():
    sl = S.slice_batch(64)
    sides = [w.n for w in sl]
    assert [sides.count(s) for s in S.SLICE_SIDES] == [13, 13, 13, 13, 12]
    assert all(w.n_angles == round(1.4 * w.n) and w.n_bins == w.n + 17 for w in sl)
    assert all(4 <= w.n_gates <= 32 for w in sl)
    assert sum(w.n_gates for w in sl) == 1221
    assert [w.motion for w in sl[:4]] == ["rigid", "rbf", "rigid", "rbf"]
    assert all(w.alpha == 1e-3 for w in sl)
    assert all(w.n_ellipses == max(10, w.n // 25) for w in sl)
    assert all(w.rbf_width == w.n / 12.8 and w.axis_hi == w.n / 12.8 for w in sl)
    assert len({w.cid for w in sl}) == 64
