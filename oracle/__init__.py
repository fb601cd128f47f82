"""FP64 CPU oracle for motion-compensated SPDHG -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg (``--impl reference`` and the ``cpu_baseline`` object) may import this
package.  The product path (``paper_2410_10503_gb300``) never does, and it
shares no code with it: the operators live in ``mc_oracle.c`` (plain loops,
double precision), the algorithm below in plain numpy.

What each function follows (arXiv 2410.10503):
  * ``A``/``At``            ray transform and adjoint, Sec. II-A and Sec. III
                             ("2D parallel geometry"); Joseph sampling.
  * ``D``/``Dt``             displacement operator D_i: X -> X, Sec. II-A
                             (bilinear pull-back), and its transpose.
  * ``Ai``/``Ait``           A_i = A D_i and A_i^* = D_i^T A^T, Sec. II-A.
  * ``objective``            O(x) = g(x) + sum_i f_i(A_i x), Sec. II-A.
  * ``prox_g``/``prox_fstar`` the proximal maps of Algorithm 1 for
                             g = alpha||x||^2 and f_i = N^-1||. - d_i||^2.
  * ``spdhg``/``pdhg``       Algorithm 1; PDHG is p_i = 1 with all gates.
  * ``rate``                 l(kappa, n) of Sec. II-B.
  * ``theorem_kappas``       condition numbers of the Theorem, Sec. II-B.
  * ``step_sizes``           admissible steps for the strongly convex case.
  * ``draw_gates``           serial uniform sampling P(i in S) = p_i
                             (Algorithm 1 step (ii)) with Philox4x32-10.

Readings where the paper is silent or garbled (the same ones the CUDA path
takes): Algorithm 1 is read as standard SPDHG -- step (i) uses z-bar^k and
z-bar^{k+1} = z^{k+1} + (theta/p_i) A_i^*(y_i^{k+1} - y_i^k); step sizes are
sigma_i = 1/(mu_f (s-1)), tau = (1-w)/(2 mu_g w), theta = w with
mu_g = 2 alpha, mu_f = N/2, s = sqrt(1+kappa), w = 1 - 2/(n(1+s)), n = N for
SPDHG and 1 for PDHG, which make the per-epoch rate exactly l(kappa, n).
"""
from __future__ import annotations

import ctypes
import math
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

from .build import build_oracle

_lib = None


def _L():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build_oracle())
        dp = ctypes.POINTER(ctypes.c_double)
        fp = ctypes.POINTER(ctypes.c_float)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        lib.or_ray_transform.argtypes = [ctypes.c_int] * 3 + [dp, dp]
        lib.or_ray_transform_adj.argtypes = [ctypes.c_int] * 3 + [dp, dp]
        lib.or_warp.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                ctypes.c_double, fp, dp, dp]
        lib.or_warp_adj.argtypes = lib.or_warp.argtypes
        lib.or_philox4x32_10.argtypes = [u32p, u32p, u32p]
        lib.or_warp_field_vjp.argtypes = [ctypes.c_int, fp, dp, dp, dp]
        lib.or_warp_field_vjp.restype = None
        lib.or_draw_gates.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64,
                                      ctypes.c_int, ctypes.c_int,
                                      ctypes.POINTER(ctypes.c_uint64),
                                      ctypes.POINTER(ctypes.c_int32)]
        for f in (lib.or_ray_transform, lib.or_ray_transform_adj, lib.or_warp,
                  lib.or_warp_adj, lib.or_philox4x32_10, lib.or_draw_gates):
            f.restype = None
        _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


# ---------------------------------------------------------------- operators
@dataclass
class Geometry:
    n: int          # image side
    na: int         # number of angles over [0, pi)
    nb: int         # number of detector bins


def A(x: np.ndarray, g: Geometry) -> np.ndarray:
    """Ray transform A x (Sec. II-A; 2D parallel beam, Sec. III)."""
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(g.n, g.n)
    y = np.empty((g.na, g.nb))
    _L().or_ray_transform(g.n, g.na, g.nb, _dp(x), _dp(y))
    return y


def At(y: np.ndarray, g: Geometry) -> np.ndarray:
    """Adjoint A^T y (backprojection), ray-driven scatter."""
    y = np.ascontiguousarray(y, dtype=np.float64).reshape(g.na, g.nb)
    x = np.empty((g.n, g.n))
    _L().or_ray_transform_adj(g.n, g.na, g.nb, _dp(y), _dp(x))
    return x


@dataclass
class Motion:
    """Motion states of the N gates: rigid (N,3)=[phi,tx,ty] or fields (N,2,n,n) f32."""
    rigid: Optional[np.ndarray] = None
    fields: Optional[np.ndarray] = None

    @property
    def n_gates(self) -> int:
        return len(self.rigid) if self.rigid is not None else len(self.fields)


def _warp_call(fn, v: np.ndarray, m: Motion, i: int, n: int) -> np.ndarray:
    v = np.ascontiguousarray(v, dtype=np.float64).reshape(n, n)
    out = np.empty((n, n))
    if m.fields is not None:
        f = np.ascontiguousarray(m.fields[i], dtype=np.float32)
        fn(n, 0.0, 0.0, 0.0, f.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), _dp(v), _dp(out))
    else:
        phi, tx, ty = (float(t) for t in m.rigid[i])
        fn(n, phi, tx, ty, None, _dp(v), _dp(out))
    return out


def D(x: np.ndarray, m: Motion, i: int, n: int) -> np.ndarray:
    """Displacement operator D_i x: bilinear pull-back warp (Sec. II-A)."""
    return _warp_call(_L().or_warp, x, m, i, n)


def Dt(v: np.ndarray, m: Motion, i: int, n: int) -> np.ndarray:
    """Transpose D_i^T v: scatter of the bilinear taps of D_i."""
    return _warp_call(_L().or_warp_adj, v, m, i, n)


@dataclass
class Problem:
    """Gated data model d_i = A D_i x + eps_i and the weight alpha (Sec. II-A)."""
    geom: Geometry
    motion: Motion
    d: np.ndarray          # (N, na, nb) float64
    alpha: float

    @property
    def N(self) -> int:
        return self.motion.n_gates


def warp_field_vjp(x, g, field_i, n: int) -> np.ndarray:
    """(2, n, n): g(p) times the derivative of the pull-back warp (D_u x)(p)
    with respect to u_x(p) and u_y(p) (dense field of one gate, float32)."""
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(n, n)
    g = np.ascontiguousarray(g, dtype=np.float64).reshape(n, n)
    f = np.ascontiguousarray(field_i, dtype=np.float32).reshape(2, n, n)
    out = np.empty((2, n, n))
    _L().or_warp_field_vjp(n, f.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), _dp(x), _dp(g), _dp(out))
    return out


def loss_field_grad(x, P: Problem, i: int) -> np.ndarray:
    """Gradient of N^-1 ||A D_{u_i} x - d_i||^2 with respect to the field u_i
    (the differentiated data term of Sec. II-A)."""
    r = (2.0 / P.N) * (Ai(x, P, i) - P.d[i])
    return warp_field_vjp(x, At(r, P.geom), P.motion.fields[i], P.geom.n)


def Ai(x, P: Problem, i: int) -> np.ndarray:
    """A_i x = A D_i x."""
    return A(D(x, P.motion, i, P.geom.n), P.geom)


def Ait(y, P: Problem, i: int) -> np.ndarray:
    """A_i^* y = D_i^T A^T y."""
    return Dt(At(y, P.geom), P.motion, i, P.geom.n)


def make_problem(geom: Geometry, motion: Motion, x_true: np.ndarray, eps: np.ndarray,
                 alpha: float, noise_level: float = 0.01) -> Problem:
    """d_i = A_i x_true + eps_i with eps_i ~ N(0, sigma^2 / N) (Sec. II-A);
    sigma = noise_level * max over gates and bins of the clean data."""
    N = motion.n_gates
    clean = np.stack([A(D(x_true, motion, i, geom.n), geom) for i in range(N)])
    sigma = noise_level * clean.max()
    d = clean + (sigma / math.sqrt(N)) * np.asarray(eps, dtype=np.float64)
    return Problem(geom, motion, d, alpha)


# ------------------------------------------------------------ model pieces
def objective(x, P: Problem) -> float:
    """O(x) = alpha ||x||^2 + sum_i N^-1 ||A_i x - d_i||^2 (Sec. II-A)."""
    val = P.alpha * float(np.sum(x * x))
    for i in range(P.N):
        r = Ai(x, P, i) - P.d[i]
        val += float(np.sum(r * r)) / P.N
    return val


def prox_g(v, tau: float, alpha: float):
    """prox_{tau g}(v), g = alpha ||x||^2: argmin alpha||u||^2 + ||u-v||^2/(2 tau)."""
    return v / (1.0 + 2.0 * tau * alpha)


def prox_fstar(v, sigma: float, d, N: int):
    """prox_{sigma f_i^*}(v) for f_i(w) = N^-1 ||w - d_i||^2, whose conjugate is
    f_i^*(y) = <y, d_i> + (N/4)||y||^2."""
    return (v - sigma * d) / (1.0 + sigma * N / 2.0)


# ------------------------------------------------------------ gate sampling
def philox4x32_10(ctr, key) -> tuple:
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (ctypes.c_uint32 * 4)()
    _L().or_philox4x32_10(c, k, o)
    return tuple(int(v) for v in o)


def gate_thresholds(p) -> np.ndarray:
    """uint64 thresholds floor(2^32 * cumsum(p)), last one forced to 2^32."""
    p = np.asarray(p, dtype=np.float64)
    cum = np.cumsum(p / p.sum())
    th = np.floor(cum * 4294967296.0).astype(np.uint64)
    th[-1] = np.uint64(4294967296)
    return th


def draw_gates(seed: int, stream: int, k0: int, count: int, n_gates: int,
               p=None) -> np.ndarray:
    """Gate index per iteration k0..k0+count-1 (Algorithm 1 step (ii))."""
    out = np.empty(count, dtype=np.int32)
    th = None
    if p is not None:
        thr = gate_thresholds(p)
        th = thr.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))
    _L().or_draw_gates(ctypes.c_uint64(seed), ctypes.c_uint32(stream), ctypes.c_uint64(k0),
                       count, n_gates, th, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    return out


# ------------------------------------------------------------ rates, steps
def rate(kappa: float, n: float) -> float:
    """l(kappa, n) = (1 - 2 n^-1 (1 + sqrt(1 + kappa))^-1)^n (Sec. II-B)."""
    return (1.0 - 2.0 / (n * (1.0 + math.sqrt(1.0 + kappa)))) ** n


def power_norm2(apply_normal, shape, iters: int = 200, tol: float = 1e-12,
                seed: int = 7) -> float:
    """Largest eigenvalue of a symmetric PSD operator by power iteration
    (Rayleigh quotient); used for ||A_i||^2 and ||(A_1..A_N)||^2."""
    v = np.random.default_rng(seed).uniform(0.5, 1.0, size=shape)
    v /= np.linalg.norm(v)
    lam = 0.0
    for _ in range(iters):
        w = apply_normal(v)
        lam_new = float(np.vdot(v, w))
        v = w / np.linalg.norm(w)
        if lam > 0 and abs(lam_new - lam) <= tol * lam_new:
            lam = lam_new
            break
        lam = lam_new
    return lam


def gate_norms2(P: Problem, iters: int = 200, tol: float = 1e-12) -> np.ndarray:
    """[||A_1||^2, ..., ||A_N||^2, ||(A_1; ...; A_N)||^2] (Theorem, Sec. II-B)."""
    n = P.geom.n
    out = [power_norm2(lambda v, i=i: Ait(Ai(v, P, i), P, i), (n, n), iters, tol)
           for i in range(P.N)]
    out.append(power_norm2(lambda v: sum(Ait(Ai(v, P, i), P, i) for i in range(P.N)),
                           (n, n), iters, tol))
    return np.array(out)


def theorem_kappas(norms2, alpha: float, N: int) -> tuple:
    """kappa^SPDHG = max_i ||A_i||^2/(alpha N), kappa^PDHG = ||(A_i)||^2/(alpha N)."""
    norms2 = np.asarray(norms2, dtype=np.float64)
    return float(norms2[:N].max()) / (alpha * N), float(norms2[N]) / (alpha * N)


@dataclass
class Steps:
    sigma: np.ndarray     # per gate
    tau: float
    theta: float
    kappa: float
    omega: float          # per-iteration contraction; per epoch omega^n = l(kappa, n)


def step_sizes(norm2: float, alpha: float, N: int, n: int) -> Steps:
    """Step sizes for the strongly convex case (moduli mu_g = 2 alpha of g and
    mu_f = N/2 of f_i^*), chosen so that omega tau sigma ||A||^2 = 1/n and the
    per-epoch contraction is l(kappa, n) with kappa = ||A||^2/(alpha N).
    n = N and norm2 = max_i ||A_i||^2 for SPDHG; n = 1 and the stacked norm
    for PDHG."""
    mu_g, mu_f = 2.0 * alpha, N / 2.0
    kappa = norm2 / (mu_g * mu_f)
    s = math.sqrt(1.0 + kappa)
    omega = 1.0 - 2.0 / (n * (1.0 + s))
    sigma = 1.0 / (mu_f * (s - 1.0))
    tau = (1.0 - omega) / (2.0 * mu_g * omega)
    return Steps(np.full(N, sigma), tau, omega, kappa, omega)


# ------------------------------------------------------------ solvers
@dataclass
class RunResult:
    x: np.ndarray                    # x^K of Algorithm 1
    y: np.ndarray                    # (N, na, nb)
    z: np.ndarray
    gates: np.ndarray                # drawn gate per iteration
    trace: list = field(default_factory=list)   # per epoch: (rel_err_x, saddle_dist2)


def _trace_entry(x, y, x_star, y_star):
    if x_star is None:
        return (math.nan, math.nan)
    dx = x - x_star
    rel = float(np.linalg.norm(dx) / np.linalg.norm(x_star))
    d2 = float(np.sum(dx * dx))
    if y_star is not None:
        d2 += float(np.sum((y - y_star) ** 2))
    return (rel, d2)


def spdhg(P: Problem, epochs: int, st: Steps, seed: int, stream: int = 0, p=None,
          x_star=None, y_star=None, literal: bool = False, subsets: int = 1,
          store: Optional[str] = None) -> RunResult:
    """Algorithm 1 (SPDHG) with serial sampling of one block per iteration.

    Standard reading (default):
      (i)   x^{k+1} = prox_{tau g}(x^k - tau zbar^k)
      (ii)  draw i; y_i^{k+1} = prox_{sigma_i f_i^*}(y_i^k + sigma_i A_i x^{k+1})
      (iii) z^{k+1} = z^k + A_i^*(y_i^{k+1} - y_i^k)
            zbar^{k+1} = z^{k+1} + (theta/p_i) A_i^*(y_i^{k+1} - y_i^k)
    ``literal=True`` runs the text as printed (step (i) with z^k, zbar
    accumulated on zbar^k); it is kept only as a negative test.

    ``subsets = S > 1`` samples gates and angle subsets together (the
    extension of Sec. IV): the blocks are j = 0 .. N S - 1 with gate j // S
    and angle subset j % S, operator A_{i,s} (subset_op) and data term
    N^-1 ||A_{i,s} x - d_{i,s}||^2, so the objective is unchanged; the draw
    is uniform over the N S blocks (p_j = 1/(N S)) and an epoch is N S
    iterations.  ``st`` then comes from step_sizes(max_j ||A_j||^2, alpha,
    N, N S).  ``gates`` holds the drawn block indices.

    ``store`` ('f32', 'f16', 'bf16') keeps the data d and the dual y in that
    storage type (round_storage): d is rounded once, each new y_i is rounded
    when stored, and the increment applied to z is the difference of the
    stored values, so z = sum_i A_i^* y_i holds for the stored y.
    """
    g, N, S = P.geom, P.N, int(subsets)
    nblk = N * S
    if S > 1 and p is not None:
        raise ValueError("non-uniform sampling is defined over gates only")
    probs = np.full(nblk, 1.0 / nblk) if p is None else np.asarray(p, dtype=np.float64) / np.sum(p)
    K = epochs * nblk
    blocks = draw_gates(seed, stream, 0, K, nblk, p)
    d = round_storage(P.d, store)
    x = np.zeros((g.n, g.n)); z = np.zeros_like(x); zbar = np.zeros_like(x)
    y = np.zeros((N, g.na, g.nb))
    res = RunResult(x, y, z, blocks)
    res.trace.append(_trace_entry(x, y, x_star, y_star))
    for k in range(K):
        x = prox_g(x - st.tau * (z if literal else zbar), st.tau, P.alpha)      # (i)
        j = int(blocks[k])                                                       # (ii)
        i, s = divmod(j, S)
        rows = subset_angles(g.na, S, s)
        y_new = round_storage(prox_fstar(y[i][rows] + st.sigma[i] * subset_op(x, P, i, S, s),
                                         st.sigma[i], d[i][rows], N), store)
        dz = subset_adj(y_new - y[i][rows], P, i, S, s)
        y[i][rows] = y_new
        z = z + dz                                                               # (iii)
        zbar = (zbar + (1.0 + st.theta / probs[j]) * dz) if literal \
            else (z + (st.theta / probs[j]) * dz)
        if (k + 1) % nblk == 0:
            res.trace.append(_trace_entry(x, y, x_star, y_star))
    res.x, res.y, res.z = x, y, z
    return res


# ------------------------------------------------------------ storage types
def round_storage(v, kind: Optional[str]):
    """v as stored in `kind`, returned as float64: None keeps v; 'f32' is
    IEEE binary32, 'f16' binary16, 'bf16' bfloat16 (the upper 16 bits of a
    binary32: 8 exponent bits, 7 stored significand bits).  Each rounds to
    nearest, ties to even, through binary32 first (the kernels compute in
    float32 and convert on store)."""
    if kind is None:
        return v
    v32 = np.asarray(v, dtype=np.float32)
    if kind == "f32":
        return v32.astype(np.float64)
    if kind == "f16":
        return v32.astype(np.float16).astype(np.float64)
    if kind == "bf16":
        u = v32.view(np.uint32).astype(np.uint64)
        u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
        return u.astype(np.uint32).view(np.float32).astype(np.float64)
    raise ValueError(f"unknown storage type {kind!r}")


# ------------------------------------------------------------ angle subsets
def subset_angles(na: int, S: int, s: int) -> np.ndarray:
    """Angle indices of subset s of S: k = s, s + S, s + 2S, ... (< na)."""
    return np.arange(s, na, S)


def subset_op(x, P: Problem, i: int, S: int, s: int) -> np.ndarray:
    """A_{i,s} x: the rows of A_i x at the angles of subset s."""
    return Ai(x, P, i)[subset_angles(P.geom.na, S, s)]


def subset_adj(ys, P: Problem, i: int, S: int, s: int) -> np.ndarray:
    """A_{i,s}^* ys = A_i^* (ys in the subset's rows, zero elsewhere)."""
    full = np.zeros((P.geom.na, P.geom.nb))
    full[subset_angles(P.geom.na, S, s)] = ys
    return Ait(full, P, i)


def block_norms2(P: Problem, S: int, iters: int = 200, tol: float = 1e-12) -> np.ndarray:
    """[||A_{0,0}||^2, ||A_{0,1}||^2, ..., ||A_{N-1,S-1}||^2, ||(A_1; ...; A_N)||^2]:
    block j = i S + s, then the stacked norm (unchanged by the split)."""
    n = P.geom.n
    out = [power_norm2(lambda v, i=i, s=s: subset_adj(subset_op(v, P, i, S, s), P, i, S, s),
                       (n, n), iters, tol)
           for i in range(P.N) for s in range(S)]
    out.append(power_norm2(lambda v: sum(Ait(Ai(v, P, i), P, i) for i in range(P.N)),
                           (n, n), iters, tol))
    return np.array(out)


def pdhg(P: Problem, epochs: int, st: Steps, x_star=None, y_star=None,
         store: Optional[str] = None) -> RunResult:
    """PDHG: Algorithm 1 with p_i = 1 and S = all gates (Sec. II-A); ``store``
    as for spdhg."""
    g, N = P.geom, P.N
    d = round_storage(P.d, store)
    x = np.zeros((g.n, g.n)); z = np.zeros_like(x); zbar = np.zeros_like(x)
    y = np.zeros((N, g.na, g.nb))
    res = RunResult(x, y, z, np.arange(N, dtype=np.int32))
    res.trace.append(_trace_entry(x, y, x_star, y_star))
    for _ in range(epochs):
        x = prox_g(x - st.tau * zbar, st.tau, P.alpha)
        dz = np.zeros_like(x)
        for i in range(N):
            y_new = round_storage(prox_fstar(y[i] + st.sigma[i] * Ai(x, P, i), st.sigma[i], d[i], N),
                                  store)
            dz += Ait(y_new - y[i], P, i)
            y[i] = y_new
        z = z + dz
        zbar = z + st.theta * dz
        res.trace.append(_trace_entry(x, y, x_star, y_star))
    res.x, res.y, res.z = x, y, z
    return res


# ------------------------------------------------------------ saddle point
def normal_rhs(P: Problem) -> np.ndarray:
    return sum(Ait(P.d[i], P, i) for i in range(P.N)) / P.N


def normal_apply(v, P: Problem) -> np.ndarray:
    """(alpha I + N^-1 sum_i A_i^T A_i) v, the Hessian of O divided by 2."""
    return P.alpha * v + sum(Ait(Ai(v, P, i), P, i) for i in range(P.N)) / P.N


def solve_xstar(P: Problem, tol: float = 1e-12, max_iter: int = 20000) -> np.ndarray:
    """x* from grad O = 0: (alpha I + N^-1 sum A_i^T A_i) x = N^-1 sum A_i^T d_i,
    by conjugate gradients to relative residual ``tol``."""
    b = normal_rhs(P)
    x = np.zeros_like(b)
    r = b.copy(); p = r.copy()
    rr = float(np.sum(r * r)); bb = rr
    for _ in range(max_iter):
        if rr <= tol * tol * bb:
            break
        q = normal_apply(p, P)
        a = rr / float(np.sum(p * q))
        x += a * p
        r -= a * q
        rr_new = float(np.sum(r * r))
        p = r + (rr_new / rr) * p
        rr = rr_new
    return x


def ystar(P: Problem, x_star) -> np.ndarray:
    """y_i* = grad f_i(A_i x*) = (2/N)(A_i x* - d_i)."""
    return np.stack([(2.0 / P.N) * (Ai(x_star, P, i) - P.d[i]) for i in range(P.N)])


def dense_matrix(apply, n_in: int, shape_in) -> np.ndarray:
    """Columns apply(e_j) for j < n_in (small problems only)."""
    cols = []
    for j in range(n_in):
        e = np.zeros(n_in); e[j] = 1.0
        cols.append(np.asarray(apply(e.reshape(shape_in))).reshape(-1))
    return np.stack(cols, axis=1)
