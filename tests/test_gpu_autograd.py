"""Differentiation of A_i = A D_{u_i} (Sec. II-A) on the GPU: mc_vjp and
mc_set_field through the C ABI, and the torch.autograd face.

Pins: the FP64 oracle's vector-Jacobian products (themselves pinned by exact
central differences on the CPU), and central differences of the float32 GPU
loss along 64 random directions of the 256^2, 360 x 365, N = 8 non-rigid
workload, with the loss  sum_i N^-1 ||A_i x - d_i||^2."""
import numpy as np
import pytest

import mc_synth as S
import oracle as O

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


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


def field_problem(W):
    sd = S.seeds(W.cid)
    g = O.Geometry(W.n, W.n_angles, W.n_bins)
    m = O.Motion(fields=S.rbf_fields(W.n, W.n_gates, sd["motion"], W.rbf_count, W.rbf_width,
                                     W.rbf_max_disp))
    xt = S.phantom(W.n, W.n_ellipses, sd["phantom"], W.axis_lo, W.axis_hi)
    eps = S.noise(W.n_gates, W.n_angles, W.n_bins, sd["noise"])
    return O.make_problem(g, m, xt, eps, W.alpha, W.noise_level), sd


SMALL = dict(n=64, n_angles=90, n_bins=93, n_gates=3, rbf_width=10.0, rbf_max_disp=3.0,
             n_ellipses=8, axis_lo=3.0, axis_hi=12.0)


def test_vjp_matches_oracle(mc):
    """mc_vjp at 64^2 (several tiles, ragged tail of the 256-thread grid):
    grad_x = A_i^* r and grad_field against the oracle, host and device arrays."""
    W = S.WORKLOADS["rbf256"].scaled(**SMALL)
    P, _ = field_problem(W)
    n = W.n
    ctx = mc.Context(n, W.n_angles, W.n_bins, W.n_gates, fields=P.motion.fields)
    x = S.random_image(n, 11).astype(np.float32)
    r = S.random_sinogram(W.n_angles, W.n_bins, 12).astype(np.float32)
    for gate in range(W.n_gates):
        gx, gf = ctx.vjp(gate, x, r)
        b = O.At(r.astype(np.float64), P.geom)
        assert rel_l2(gx, O.Ait(r.astype(np.float64), P, gate)) <= 1e-5
        ref = O.warp_field_vjp(x, b, P.motion.fields[gate], n)
        assert rel_l2(gf, ref) <= 1e-5
        gxd, gfd = ctx.vjp(gate, torch.as_tensor(x, device="cuda"), torch.as_tensor(r, device="cuda"))
        np.testing.assert_array_equal(gxd.cpu().numpy(), gx)
        np.testing.assert_array_equal(gfd.cpu().numpy(), gf)
    # one output alone, and the rigid-context refusal
    gx1, gf1 = ctx.vjp(0, x, r, grad_field=False)
    assert gf1 is None and rel_l2(gx1, ctx.adjoint(0, r)) == 0.0
    rig = mc.Context(n, W.n_angles, W.n_bins, 2, rigid=np.zeros((2, 3)))
    with pytest.raises(mc.MCError, match="dense-field"):
        rig.vjp(0, x, r)
    with pytest.raises(mc.MCError, match="dense-field"):
        rig.set_field(0, np.zeros((2, n, n), np.float32))


def test_set_field_equals_fresh_context(mc):
    """After mc_set_field the operators and a graph-replayed SPDHG run are
    bit-identical to a context created with the new field."""
    W = S.WORKLOADS["rbf256"].scaled(**SMALL)
    P, sd = field_problem(W)
    n, N = W.n, W.n_gates
    F1 = S.rbf_fields(n, N, 777, W.rbf_count, W.rbf_width, W.rbf_max_disp)
    F_mix = P.motion.fields.copy()
    F_mix[1] = F1[1]
    fresh = mc.Context(n, W.n_angles, W.n_bins, N, fields=F_mix)
    ctx = mc.Context(n, W.n_angles, W.n_bins, N, fields=P.motion.fields)
    d = P.d.astype(np.float32)
    norms = np.full(N + 1, 1.0)
    for c in (fresh, ctx):
        c.set_data(d, 1e-2)
    ctx.set_norms(norms * 50.0)
    ctx.spdhg_run(2, seed=sd["gates"], x_out=False)     # captures graphs on the old field
    ctx.set_field(1, F1[1])
    with pytest.raises(mc.MCError, match="norms"):
        ctx.spdhg_run(1, seed=sd["gates"])
    x = S.random_image(n, 5).astype(np.float32)
    y = S.random_sinogram(W.n_angles, W.n_bins, 6).astype(np.float32)
    for g in range(N):
        np.testing.assert_array_equal(ctx.forward(g, x), fresh.forward(g, x))
        np.testing.assert_array_equal(ctx.adjoint(g, y), fresh.adjoint(g, y))
        np.testing.assert_array_equal(ctx.warp_adjoint(g, x), fresh.warp_adjoint(g, x))
    for c in (fresh, ctx):
        c.set_norms(norms * 60.0)
        c.reset()
    a = ctx.spdhg_run(3, seed=sd["gates"])[0]
    b = fresh.spdhg_run(3, seed=sd["gates"])[0]
    np.testing.assert_array_equal(a, b)
    bad = F1[1].copy()
    bad[0, 3, 4] = np.nan
    with pytest.raises(mc.MCError, match="not finite"):
        ctx.set_field(1, bad)


@pytest.fixture(scope="module")
def rbf256(mc):
    """The 256^2, 360 x 365, N = 8 non-rigid workload; x is a different
    phantom so that every residual is large."""
    W = S.WORKLOADS["rbf256"]
    P, sd = field_problem(W)
    x = S.phantom(W.n, 12, 99, 4.0, 40.0)
    return W, P, x


def torch_loss(mc, ctx, x, fields, d):
    N = fields.shape[0]
    loss = 0.0
    for i in range(N):
        y = mc.project_gate(ctx, i, x, fields[i])
        loss = loss + ((y.double() - d[i].double()) ** 2).sum() / N
    return loss


def test_autograd_gradients_match_oracle(mc, rbf256):
    W, P, x = rbf256
    N = W.n_gates
    ctx = mc.Context(W.n, W.n_angles, W.n_bins, N, fields=P.motion.fields)
    xt = torch.tensor(x, dtype=torch.float32, device="cuda", requires_grad=True)
    ft = torch.tensor(P.motion.fields, dtype=torch.float32, device="cuda", requires_grad=True)
    d = torch.tensor(P.d, dtype=torch.float32, device="cuda")
    loss = torch_loss(mc, ctx, xt, ft, d)
    loss.backward()
    x32 = x.astype(np.float32).astype(np.float64)
    # oracle: loss and gradients of sum_i N^-1 ||A_i x - d_i||^2 at the same float32 inputs
    Pd = O.Problem(P.geom, P.motion, P.d.astype(np.float32).astype(np.float64), P.alpha)
    res = [O.Ai(x32, Pd, i) - Pd.d[i] for i in range(N)]
    ref_loss = sum(float((r ** 2).sum()) for r in res) / N
    assert abs(loss.item() - ref_loss) <= 1e-5 * ref_loss
    gx_ref = sum(O.Ait((2.0 / N) * res[i], Pd, i) for i in range(N))
    assert rel_l2(xt.grad.cpu().numpy(), gx_ref) <= 1e-4
    for i in range(N):
        gf_ref = O.loss_field_grad(x32, Pd, i)
        assert rel_l2(ft.grad[i].cpu().numpy(), gf_ref) <= 1e-4, i


def kink_free_direction(field, h, rng):
    """Random direction (2, n, n) that is zero wherever a step of size h would
    carry the sample position across a grid line (the bilinear kinks)."""
    v = rng.standard_normal(field.shape)
    u = field.astype(np.float64)
    frac = u - np.floor(u)
    near = np.minimum(frac, 1.0 - frac) <= 2.0 * h * np.abs(v) + 1e-6
    v[near] = 0.0
    return v


def test_autograd_central_differences_64_directions(mc, rbf256):
    """Central differences (step 1e-3) of the float32 GPU loss along 64 random
    directions, against <grad, applied step>.  Field directions avoid the
    kinks at grid lines; the loss is quadratic in x, so image differences
    are exact up to rounding."""
    W, P, x = rbf256
    N = W.n_gates
    ctx = mc.Context(W.n, W.n_angles, W.n_bins, N, fields=P.motion.fields)
    F = P.motion.fields.astype(np.float32)
    xt = torch.tensor(x, dtype=torch.float32, device="cuda", requires_grad=True)
    ft = torch.tensor(F, device="cuda", requires_grad=True)
    d = torch.tensor(P.d, dtype=torch.float32, device="cuda")
    loss = torch_loss(mc, ctx, xt, ft, d)
    loss.backward()
    gx = xt.grad.double().cpu().numpy()
    gf = ft.grad.double().cpu().numpy()
    h = 1e-3
    rng = np.random.default_rng(64)
    x32 = x.astype(np.float32)

    def L(xa, fa):
        with torch.no_grad():
            return torch_loss(mc, ctx, torch.as_tensor(xa, device="cuda"),
                              torch.as_tensor(fa, device="cuda"), d).item()

    dfd, dlin = np.zeros(64), np.zeros(64)
    for k in range(64):
        if k % 2 == 0:                      # field direction, all gates
            v = np.stack([kink_free_direction(F[i], h, rng) for i in range(N)])
            fp = (F + h * v).astype(np.float32)
            fm = (F - h * v).astype(np.float32)
            dlin[k] = float((gf * (fp.astype(np.float64) - fm.astype(np.float64))).sum())
            dfd[k] = L(x32, fp) - L(x32, fm)
        else:                               # image direction
            v = rng.standard_normal(x.shape) * np.abs(x).max()
            xp = (x32 + h * v).astype(np.float32)
            xm = (x32 - h * v).astype(np.float32)
            dlin[k] = float((gx * (xp.astype(np.float64) - xm.astype(np.float64))).sum())
            dfd[k] = L(xp, F) - L(xm, F)
    # The float32 loss carries rounding noise of about 1e-6 of the projections
    # times the residuals, independent of the direction; so the check is the
    # relative L2 error over the 32 directions of each kind, and each
    # direction's error against the RMS directional derivative.
    for kind, sl in (("field", slice(0, None, 2)), ("image", slice(1, None, 2))):
        a, b = dfd[sl], dlin[sl]
        rms = np.sqrt(np.mean(b ** 2))
        rel = np.linalg.norm(a - b) / np.linalg.norm(b)
        worst = np.abs(a - b).max() / rms
        print(f"{kind}: rel_l2 {rel:.3e}  worst/rms {worst:.3e}  rms {rms:.4e}  "
              f"loss {loss.item():.6e}")
        assert rel <= 5e-3, (kind, rel)
        assert worst <= 1e-2, (kind, worst)


def test_backward_restores_the_forward_field(mc):
    """Two graphs built on different fields of the same gate each get the
    gradient of their own operator."""
    W = S.WORKLOADS["rbf256"].scaled(**SMALL)
    P, _ = field_problem(W)
    n = W.n
    ctx = mc.Context(n, W.n_angles, W.n_bins, W.n_gates, fields=P.motion.fields)
    F1 = S.rbf_fields(n, W.n_gates, 4242, W.rbf_count, W.rbf_width, W.rbf_max_disp)
    x = torch.tensor(S.random_image(n, 3), dtype=torch.float32, device="cuda")
    grads = []
    for F in (P.motion.fields[0], F1[0]):
        f = torch.tensor(F, device="cuda", requires_grad=True)
        y = mc.project_gate(ctx, 0, x, f)
        grads.append((f, (y ** 2).sum()))
    for f, l in reversed(grads):       # backward of the first graph after the field changed
        l.backward()
    for (f, _), F in zip(grads, (P.motion.fields[0], F1[0])):
        r = 2.0 * O.Ai(x.cpu().numpy().astype(np.float64),
                       O.Problem(P.geom, O.Motion(fields=F[None]), np.zeros(1), 1.0), 0)
        ref = O.warp_field_vjp(x.cpu().numpy(), O.At(r, P.geom), F, n)
        assert rel_l2(f.grad.cpu().numpy(), ref) <= 1e-4


def test_backward_through_an_older_field_leaves_the_newest_in_place(mc):
    """Backward of a graph whose field has since been replaced uses that
    graph's field for its gradient, then puts the newest field back: a later
    forward of the gate outside autograd applies the field set last."""
    W = S.WORKLOADS["rbf256"].scaled(**SMALL)
    P, _ = field_problem(W)
    n = W.n
    ctx = mc.Context(n, W.n_angles, W.n_bins, W.n_gates, fields=P.motion.fields)
    F1 = S.rbf_fields(n, W.n_gates, 4343, W.rbf_count, W.rbf_width, W.rbf_max_disp)
    x = torch.tensor(S.random_image(n, 5), dtype=torch.float32, device="cuda")
    f0 = torch.tensor(P.motion.fields[0], device="cuda", requires_grad=True)
    l0 = (mc.project_gate(ctx, 0, x, f0) ** 2).sum()          # graph on the first field
    ctx.set_field(0, torch.tensor(F1[0], device="cuda"))       # replaced outside autograd
    l0.backward()
    x64 = x.cpu().numpy().astype(np.float64)
    r = 2.0 * O.Ai(x64, O.Problem(P.geom, O.Motion(fields=P.motion.fields[:1]), np.zeros(1), 1.0), 0)
    ref = O.warp_field_vjp(x.cpu().numpy(), O.At(r, P.geom), P.motion.fields[0], n)
    assert rel_l2(f0.grad.cpu().numpy(), ref) <= 1e-4
    y_now = ctx.forward(0, x).cpu().numpy()
    y_ref = O.Ai(x64, O.Problem(P.geom, O.Motion(fields=F1[:1]), np.zeros(1), 1.0), 0)
    assert rel_l2(y_now, y_ref) <= 1e-5
    ctx.close()
