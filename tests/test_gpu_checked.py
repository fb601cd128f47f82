"""The bounds-checked build (MC_CHECKED=1: every shared-memory gather index
checked against its line or window, a failed check sets the device error
word, which every call turns into MC_EDEVICE) on tiny and ragged cases:
operators and runs must match the oracle with a clean error word.  Runs in
a child process, because a process loads one flavour of the library."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

CASES = [(8, 6, 9), (9, 4, 13), (16, 8, 23), (32, 36, 41), (37, 41, 53)]


def _child():
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import mc_synth as S
    import oracle as O
    import paper_2410_10503_gb300 as M
    from paper_2410_10503_gb300 import _native, build
    build.build(checked=True)
    assert _native.lib_path().endswith(os.path.join("checked", "libmc.so"))

    def rel(a, b):
        a = np.asarray(a, np.float64).ravel(); b = np.asarray(b, np.float64).ravel()
        return float(np.linalg.norm(a - b) / np.linalg.norm(b))

    worst = 0.0
    for n, na, nb in CASES:
        g = O.Geometry(n, na, nb)
        for kind in ("rigid", "field"):
            N = 3
            if kind == "rigid":
                rig = S.rigid_motion(N, 8.0, 2.0, n)
                m = O.Motion(rigid=rig)
                ctx = M.Context(n, na, nb, N, rigid=rig)
            else:
                f = S.rbf_fields(n, N, n, 4, max(2.0, n / 6), 1.5)
                m = O.Motion(fields=f)
                ctx = M.Context(n, na, nb, N, fields=f)
            P = O.Problem(g, m, np.zeros((N, na, nb)), 1.0)
            x = S.random_image(n, 1) - 0.3
            y = S.random_sinogram(na, nb, 2)
            for i in range(N):
                worst = max(worst, rel(ctx.forward(i, x.astype(np.float32)), O.Ai(x, P, i)))
                worst = max(worst, rel(ctx.adjoint(i, y.astype(np.float32)), O.Ait(y, P, i)))
            # a short run, with angle subsets where the angles allow
            xt = S.phantom(n, 3, 5, n / 8 + 0.5, n / 3 + 1)
            Pd = O.make_problem(g, m, xt, S.noise(N, na, nb, 6), 1e-1)
            ctx.set_data(Pd.d.astype(np.float32), Pd.alpha)
            sub = 2 if na >= 4 else 1
            if sub > 1:
                ctx.set_subsets(sub)
            nrm = O.block_norms2(Pd, sub, 30, 1e-12) if sub > 1 else O.gate_norms2(Pd, 30, 1e-12)
            ctx.set_norms(nrm)
            xr, _ = ctx.spdhg_run(4, seed=9)
            ref = O.spdhg(Pd, 4, O.step_sizes(nrm[:-1].max(), Pd.alpha, N, N * sub), seed=9, subsets=sub)
            worst = max(worst, rel(xr, ref.x))
            ctx.close()
    print(json.dumps({"worst_rel_l2": worst}))


def test_checked_build_is_clean_on_tiny_and_ragged_cases():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    env = dict(os.environ, MC_CHECKED="1")
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--child"], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    assert out["worst_rel_l2"] <= 1e-4, out


if __name__ == "__main__" and "--child" in sys.argv:
    _child()
