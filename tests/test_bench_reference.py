"""The reference arm of bench.py (the FP64 oracle on the host): its bounded
per-step sample keeps every s-th angle of the workload, which is exactly the
workload's rays at those angles, and the arm prints one JSON line."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import mc_synth as S
import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


@pytest.mark.parametrize("stride", [2, 3, 4])
def test_strided_geometry_holds_every_sth_angle(stride):
    """Angle k' of the n_a/s-angle geometry is angle k' s of the full one
    (phi = k' pi/(n_a/s) = k' s pi/n_a, and the column/row rule agrees), so
    its A_i x is every s-th row of the full A_i x and its A_i^* y is the full
    A_i^* of y placed in those rows (angles rounded separately: up to an ulp
    of phi apart)."""
    n, na, nb, N = 24, 36, 31, 2
    rig = S.rigid_motion(N, 8.0, 3.0, 7)
    full = O.Problem(O.Geometry(n, na, nb), O.Motion(rigid=rig), np.zeros((N, na, nb)), 1.0)
    part = O.Problem(O.Geometry(n, na // stride, nb), O.Motion(rigid=rig),
                     np.zeros((N, na // stride, nb)), 1.0)
    x = S.phantom(n, 5, 8, 2, 8)
    ys = S.random_sinogram(na // stride, nb, 9)
    y = np.zeros((na, nb))
    y[::stride] = ys
    for i in range(N):
        a_full, a_part = O.Ai(x, full, i), O.Ai(x, part, i)
        np.testing.assert_allclose(a_part, a_full[::stride], rtol=0, atol=1e-12 * np.abs(a_full).max())
        b_full, b_part = O.Ait(y, full, i), O.Ait(ys, part, i)
        np.testing.assert_allclose(b_part, b_full, rtol=0, atol=1e-12 * np.abs(b_full).max())


def test_reference_stride_fits_the_budget():
    assert bench.reference_stride(720, 25) == 1
    assert bench.reference_stride(720, 205) == 3
    for steps in (1, 50, 205, 1000, 10000):
        s = bench.reference_stride(720, steps, budget_s=60.0)
        assert 720 % s == 0
        assert steps * 1.3 / s <= 60.0 or s == 720
        smaller = [d for d in range(1, s) if 720 % d == 0]
        assert all(steps * 1.3 / d > 60.0 for d in smaller)


def test_reference_arm_prints_one_json_line():
    """A short run whose budget forces a stride above 1 (the whole workload
    pair would not fit)."""
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "2", "--warmup", "1", "--reference-budget-s", "1.0"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    out = json.loads(lines[0])
    assert out["impl"] == "reference" and out["unit"] == bench.UNIT and out["steps"] == 2
    assert out["value"] > 0 and out["e2e"]["value"] == out["value"]
    assert out["cpu_baseline"]["kind"] == "oracle" and "k = 0, 4, 8, ..." in out["cpu_baseline"]["sample"]


@pytest.mark.parametrize("n,na,nb", [(16, 12, 23), (15, 20, 22), (9, 4, 13), (12, 16, 12)])
def test_algorithmic_units_match_a_brute_force_count(n, na, nb):
    """S (the roofline's unit: Joseph samples with a non-zero in-image
    weight) against the oracle: an image that is 1 on one driving line (a
    column for column-driven angles, a row otherwise) projects to a non-zero
    value on ray (k, b) exactly when that ray's sample on the line has a
    non-zero weight, since the ray's other samples lie on other lines."""
    from types import SimpleNamespace
    g = O.Geometry(n, na, nb)
    cols = np.zeros(na, dtype=np.int64)
    rows = np.zeros(na, dtype=np.int64)
    for l in range(n):
        e = np.zeros((n, n))
        e[:, l] = 1.0
        cols += np.count_nonzero(O.A(e, g), axis=1)
        e = np.zeros((n, n))
        e[l, :] = 1.0
        rows += np.count_nonzero(O.A(e, g), axis=1)
    xd = np.array([na <= 4 * k <= 3 * na for k in range(na)])
    brute = int(np.sum(np.where(xd, cols, rows)))
    assert bench.algorithmic_units(SimpleNamespace(n=n, n_angles=na, n_bins=nb)) == brute


def test_cpu_baseline_more_legs_report_without_failing():
    """The extra oracle timings on a small workload: two spawned processes,
    a few pairs and a short solver run; every leg reports a value."""
    out = bench.cpu_baseline_more(S.WORKLOADS["rigid128"], cores=2, small_pairs=2, epochs=2,
                                  timeout_s=120.0)
    assert out["all_cores"]["cores"] == 2 and out["all_cores"]["value"] > 0, out
    assert out["pairs_rigid128"]["value"] > 0, out
    s = out["solvers_rigid128"]
    assert s["epochs"] == 2 and s["spdhg_s"] > 0 and s["pdhg_s"] > 0, out
