"""GB300-native motion-compensated SPDHG (arXiv 2410.10503).

Python face of libmc (include/mc.h): the same entry points, argument
marshalling only.  Arrays may be torch tensors (CUDA or CPU) or numpy arrays;
CUDA tensors are passed as device pointers, everything else as host pointers
(the library stages those through its own device buffers).  Results come back
as CUDA tensors when the input was one, else as numpy arrays.

Streams: the library orders its work on the context's stream.  Calls that
take CUDA tensors are ordered after the caller's current torch stream (the
context stream waits on it) and the current stream waits for the context
stream afterwards, so results behave as if computed on the current stream.

Every computation runs in the library's CUDA kernels; when libmc is not
built, or no sm_103a GPU is present, the calls raise instead of falling back.
"""
from __future__ import annotations

import ctypes
from typing import Optional

import numpy as np

from . import _native as N

__all__ = ["Context", "Batch", "MCError", "lib", "version", "project_gate", "batch_spdhg_run", "shared_load_peak",
           "plan_shapes"]

try:  # torch is plumbing here (device memory, streams); optional for host arrays
    import torch
except Exception:  # pragma: no cover
    torch = None


class MCError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{N.STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def lib():
    return N.load()


def version() -> str:
    return lib().mc_version().decode()


SHAPE_KEYS = ("guard", "pitch", "layout_lines", "lines_per_chunk", "lines_per_part", "ring_stages",
              "rows_per_thread", "dual_guard", "dual_pitch", "consumer_warps")


def plan_shapes(n: int, n_angles: int, n_bins: int, sms: int) -> dict:
    """The launch shapes and layouts a context of this geometry gets on a GPU
    with `sms` SMs (mc_plan_shapes; host only, no device needed)."""
    out = np.zeros(len(SHAPE_KEYS), np.int32)
    st = lib().mc_plan_shapes(ctypes.byref(N.mc_geometry(int(n), int(n_angles), int(n_bins))), int(sms),
                              out.ctypes.data)
    if st != 0:
        raise MCError(st, f"no shapes for n={n}, n_angles={n_angles}, n_bins={n_bins}, sms={sms}")
    return dict(zip(SHAPE_KEYS, out.tolist()))


def _is_tensor(a) -> bool:
    return torch is not None and isinstance(a, torch.Tensor)


def _arg(a, dtype, count: int, name: str):
    """(pointer, keepalive) of a contiguous array with `count` elements."""
    if _is_tensor(a):
        tdt = {np.float32: torch.float32, np.float64: torch.float64, np.int32: torch.int32}[dtype]
        if a.dtype != tdt:
            raise TypeError(f"{name}: expected {tdt}, got {a.dtype}")
        if not a.is_contiguous():
            raise ValueError(f"{name}: tensor must be contiguous")
        if a.numel() != count:
            raise ValueError(f"{name}: expected {count} elements, got {a.numel()}")
        return a.data_ptr(), a
    arr = np.ascontiguousarray(a, dtype=dtype)
    if arr.size != count:
        raise ValueError(f"{name}: expected {count} elements, got {arr.size}")
    return arr.ctypes.data, arr


def _empty_like_kind(ref, shape, dtype=np.float32):
    if _is_tensor(ref) and ref.is_cuda:
        tdt = {np.float32: torch.float32, np.float64: torch.float64, np.int32: torch.int32}[dtype]
        return torch.empty(shape, dtype=tdt, device=ref.device)
    return np.empty(shape, dtype=dtype)


class Context:
    """One reconstruction problem on the current CUDA device (mc_create)."""

    def __init__(self, n: int, n_angles: int, n_bins: int, n_gates: int,
                 rigid=None, fields=None, stream: Optional[int] = None):
        L = lib()
        self._L = L
        self.n, self.n_angles, self.n_bins, self.n_gates = n, n_angles, n_bins, n_gates
        g = N.mc_geometry(n, n_angles, n_bins)
        keep = []
        if (rigid is None) == (fields is None):
            raise ValueError("give exactly one of rigid (N x 3) or fields (N x 2 x n x n)")
        if rigid is not None:
            p, k = _arg(rigid, np.float64, n_gates * 3, "rigid")
            m = N.mc_motion(N.MC_MOTION_RIGID, p, None)
        else:
            p, k = _arg(fields, np.float32, n_gates * 2 * n * n, "fields")
            m = N.mc_motion(N.MC_MOTION_FIELD, None, p)
        keep.append(k)
        self._stream = None
        if torch is not None and torch.cuda.is_available():
            self._stream = (torch.cuda.ExternalStream(stream) if stream
                            else torch.cuda.Stream())
            stream = self._stream.cuda_stream
        if keep and _is_tensor(keep[0]) and keep[0].is_cuda:
            self._stream.wait_stream(torch.cuda.current_stream())
        out = ctypes.c_void_p()
        st = L.mc_create(ctypes.byref(g), n_gates, ctypes.byref(m),
                         ctypes.c_void_p(stream) if stream else None, ctypes.byref(out))
        if st != 0:
            raise MCError(st, L.mc_last_error(None).decode())
        self._h = out.value
        self.kind = "rigid" if rigid is not None else "field"
        self._field_version = {}
        # the field each gate currently uses (copies), so that autograd can put
        # a field back after differentiating through an older one
        self._fields_now = {}
        self._fields_init = None
        if fields is not None:
            self._fields_init = (fields.detach().clone() if _is_tensor(fields)
                                 else np.array(fields, dtype=np.float32, copy=True))
        self.subsets = 1

    # -- plumbing --------------------------------------------------------------
    def _check(self, st: int):
        if st != 0:
            raise MCError(st, self._L.mc_last_error(self._h).decode())

    @property
    def stream(self):
        """The torch stream the context orders its work on (None without CUDA)."""
        return self._stream

    def _call(self, fn, *args, cuda_args=()):
        """Run one C call ordered after the current torch stream when any of
        `cuda_args` is a CUDA tensor, and make the current stream wait for it."""
        handoff = self._stream is not None and any(
            _is_tensor(a) and a.is_cuda for a in cuda_args)
        if handoff:
            cur = torch.cuda.current_stream()
            if cur != self._stream:
                self._stream.wait_stream(cur)
        st = fn(self._h, *args)
        if handoff:
            cur = torch.cuda.current_stream()
            if cur != self._stream:
                cur.wait_stream(self._stream)
        self._check(st)

    def close(self):
        if getattr(self, "_h", None):
            self._L.mc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def img_count(self):
        return self.n * self.n

    @property
    def sino_count(self):
        return self.n_angles * self.n_bins

    # -- operators ----------------------------------------------------------------
    def _op(self, fn, args, x, n_in, out, out_shape):
        px, kx = _arg(x, np.float32, n_in, "input")
        if out is None:
            out = _empty_like_kind(x, out_shape)
        po, ko = _arg(out, np.float32, int(np.prod(out_shape)), "out")
        self._call(fn, *args, px, po, cuda_args=(x, out))
        return out

    def forward(self, gate: int, x, out=None):
        """A_i x = A D_i x."""
        return self._op(self._L.mc_forward, (gate,), x, self.img_count, out,
                        (self.n_angles, self.n_bins))

    def adjoint(self, gate: int, y, out=None):
        """A_i^* y = D_i^T A^T y."""
        return self._op(self._L.mc_adjoint, (gate,), y, self.sino_count, out, (self.n, self.n))

    def project(self, x, out=None):
        """A x (no motion)."""
        return self._op(self._L.mc_project, (), x, self.img_count, out, (self.n_angles, self.n_bins))

    def backproject(self, y, out=None):
        """A^T y."""
        return self._op(self._L.mc_backproject, (), y, self.sino_count, out, (self.n, self.n))

    def warp(self, gate: int, x, out=None):
        """D_i x."""
        return self._op(self._L.mc_warp, (gate,), x, self.img_count, out, (self.n, self.n))

    def warp_adjoint(self, gate: int, v, out=None):
        """D_i^T v."""
        return self._op(self._L.mc_warp_adjoint, (gate,), v, self.img_count, out, (self.n, self.n))

    # -- differentiation -------------------------------------------------------
    def set_field(self, gate: int, field):
        """Replace gate `gate`'s dense displacement field (2 x n x n); drops
        the norms, step sizes and reference (mc_set_field)."""
        p, k = _arg(field, np.float32, 2 * self.img_count, "field")
        self._call(self._L.mc_set_field, gate, p, cuda_args=(field,))
        self._field_version[gate] = self._field_version.get(gate, 0) + 1
        self._fields_now[gate] = (field.detach().clone() if _is_tensor(field)
                                  else np.array(field, dtype=np.float32, copy=True))

    def field_version(self, gate: int) -> int:
        """How many times set_field replaced this gate's field."""
        return self._field_version.get(gate, 0)

    def current_field(self, gate: int):
        """A copy of the field gate `gate` uses now (2 x n x n): the last one
        given to set_field, else the one given at construction."""
        if self.kind != "field":
            raise ValueError("rigid-motion context has no displacement field")
        if gate in self._fields_now:
            return self._fields_now[gate]
        f = self._fields_init
        return f.reshape(self.n_gates, 2, self.n, self.n)[gate]

    def vjp(self, gate: int, x, r, grad_x=True, grad_field=True):
        """(A_i^* r, b * grad of the warp sample w.r.t. u_i) with b = A^T r
        (mc_vjp); either part may be skipped (None is returned for it)."""
        pr, kr = _arg(r, np.float32, self.sino_count, "r")
        px = None
        if grad_field:
            px, kx = _arg(x, np.float32, self.img_count, "x")
        gx = _empty_like_kind(r, (self.n, self.n)) if grad_x else None
        gf = _empty_like_kind(r, (2, self.n, self.n)) if grad_field else None
        pgx = _arg(gx, np.float32, self.img_count, "grad_x")[0] if grad_x else None
        pgf = _arg(gf, np.float32, 2 * self.img_count, "grad_field")[0] if grad_field else None
        self._call(self._L.mc_vjp, gate, px, pr, pgx, pgf, cuda_args=(x, r, gx, gf))
        return gx, gf

    # -- problem ------------------------------------------------------------------
    def set_data(self, d, alpha: float):
        p, k = _arg(d, np.float32, self.n_gates * self.sino_count, "d")
        self._call(self._L.mc_set_data, p, float(alpha), cuda_args=(d,))

    def stage_data(self, d):
        """Start uploading the next data set (host array; pinned memory for an
        asynchronous copy) while the context keeps working (mc_stage_data);
        commit_data makes it current.  The arrays are kept alive until then."""
        if _is_tensor(d) and d.is_cuda:
            raise TypeError("stage_data takes host data; use set_data for CUDA tensors")
        p, k = _arg(d, np.float32, self.n_gates * self.sino_count, "d")
        self._check(self._L.mc_stage_data(self._h, p))
        # every array staged since the last commit may still be in flight
        self._staged = (getattr(self, "_staged", None) or []) + [k]

    def commit_data(self, alpha: float):
        """Make the staged data current, as set_data would (mc_commit_data).
        The staged arrays are released once the commit has succeeded (a
        refused commit leaves the upload staged)."""
        self._check(self._L.mc_commit_data(self._h, float(alpha)))
        self._staged = None

    @property
    def n_blocks(self) -> int:
        """Sampled blocks: gates, or gates x angle subsets after set_subsets."""
        return self.n_gates * self.subsets

    def set_subsets(self, subsets: int):
        """Sample gates x `subsets` interleaved angle subsets (mc_set_subsets);
        drops the norms and step sizes."""
        self._check(self._L.mc_set_subsets(self._h, int(subsets)))
        self.subsets = int(subsets)

    def norms(self, max_iter: int = 200, tol: float = 1e-6) -> np.ndarray:
        """[||A_j||^2 per block, stacked ||(A_1; ...; A_N)||^2] (mc_norms)."""
        out = np.empty(self.n_blocks + 1)
        self._check(self._L.mc_norms(self._h, max_iter, tol, out.ctypes.data))
        return out

    def set_norms(self, norms2):
        p, k = _arg(norms2, np.float64, self.n_blocks + 1, "norms2")
        self._check(self._L.mc_set_norms(self._h, p))

    def steps(self, pdhg: bool = False) -> dict:
        out = np.empty(5)
        self._check(self._L.mc_get_steps(self._h, 1 if pdhg else 0, out.ctypes.data))
        return dict(zip(("sigma", "tau", "theta", "kappa", "omega"), out.tolist()))

    def set_reference(self, x_star):
        if x_star is None:
            self._check(self._L.mc_set_reference(self._h, None))
            return
        p, k = _arg(x_star, np.float32, self.img_count, "x_star")
        self._call(self._L.mc_set_reference, p, cuda_args=(x_star,))

    def reset(self):
        self._check(self._L.mc_reset(self._h))

    def solve_normal(self, max_iter: int = 500, tol: float = 1e-6, x_out=None, like=None):
        """x* of (alpha I + N^-1 sum A_i^T A_i) x = N^-1 sum A_i^T d_i by CG;
        returns (x, iterations, relative residual)."""
        if x_out is None:
            x_out = _empty_like_kind(like, (self.n, self.n)) if like is not None else \
                np.empty((self.n, self.n), np.float32)
        px = _arg(x_out, np.float32, self.img_count, "x_out")[0]
        info = np.zeros(2)
        self._call(self._L.mc_solve_normal, int(max_iter), float(tol), px, info.ctypes.data,
                   cuda_args=(x_out,))
        return x_out, int(info[0]), float(info[1])

    def _sampling(self, seed, stream, p):
        """mc_sampling for a run or draw; p (N probabilities) is kept alive
        on the struct while the call runs."""
        s = N.mc_sampling(int(seed), int(stream), None)
        if p is not None:
            arr = np.ascontiguousarray(p, dtype=np.float64)
            if arr.size != self.n_gates:
                raise ValueError(f"p: expected {self.n_gates} probabilities, got {arr.size}")
            s.p = arr.ctypes.data
            s._keep = arr
        return s

    def _run(self, which, epochs, seed, stream, x_out, trace, like, p=None):
        if x_out is None:
            x_out = _empty_like_kind(like, (self.n, self.n)) if like is not None else \
                np.empty((self.n, self.n), np.float32)
        elif x_out is False:
            x_out = None
        px = _arg(x_out, np.float32, self.img_count, "x_out")[0] if x_out is not None else None
        tr = np.full((max(epochs, 0), 3), np.nan) if trace else None
        pt = tr.ctypes.data if tr is not None else None
        if which == 0:
            s = self._sampling(seed, stream, p)
            self._call(self._L.mc_spdhg_run, epochs, ctypes.byref(s), px, pt, cuda_args=(x_out,))
        else:
            self._call(self._L.mc_pdhg_run, epochs, px, pt, cuda_args=(x_out,))
        return x_out, tr

    def spdhg_run(self, epochs: int, seed: int, stream: int = 0, x_out=None, trace=False, like=None,
                  p=None):
        """Algorithm 1 for `epochs` epochs; returns (x^K, trace or None).
        x_out=False skips the copy of x (fully asynchronous with device arrays).
        p: None (uniform) or N sampling probabilities P(i) = p_i."""
        return self._run(0, epochs, seed, stream, x_out, trace, like, p)

    def pdhg_run(self, epochs: int, x_out=None, trace=False, like=None):
        return self._run(1, epochs, 0, 0, x_out, trace, like)

    def sync(self):
        """Wait for the context's work; raises for a device-side failure of a
        run that returned without waiting (device or no outputs)."""
        self._check(self._L.mc_sync(self._h))

    def draw_gates(self, seed: int, stream: int, k0: int, count: int, out=None, p=None):
        if out is None:
            out = np.empty(count, np.int32)
        po = _arg(out, np.int32, count, "out")[0]
        s = self._sampling(seed, stream, p)
        self._call(self._L.mc_draw_gates, ctypes.byref(s), k0, count, po, cuda_args=(out,))
        return out

    def objective(self, x) -> float:
        p, k = _arg(x, np.float32, self.img_count, "x")
        out = ctypes.c_double()
        self._call(self._L.mc_objective, p, ctypes.addressof(out), cuda_args=(x,))
        return out.value

    def set_option(self, option: int, value: int):
        self._check(self._L.mc_set_option(self._h, option, int(value)))

    def shapes(self) -> dict:
        """The launch shapes and layouts this context uses now (mc_get_shapes),
        keyed as plan_shapes."""
        out = np.zeros(len(SHAPE_KEYS), np.int32)
        self._check(self._L.mc_get_shapes(self._h, out.ctypes.data))
        return dict(zip(SHAPE_KEYS, out.tolist()))

    def autotune(self, reps: int = 5) -> dict:
        """Time the projectors' launch shapes on this geometry and keep the
        fastest (mc_autotune)."""
        out = np.zeros(4, np.int32)
        self._check(self._L.mc_autotune(self._h, int(reps), out.ctypes.data))
        return dict(zip(("lines_per_chunk", "items_per_block", "group_slots", "rows_per_thread"),
                        out.tolist()))

    def set_storage(self, kind: str):
        """Storage type of d and y in the iterations: 'f32', 'f16' or 'bf16'
        (MC_OPT_STORAGE)."""
        code = {"f32": N.MC_STORE_F32, "f16": N.MC_STORE_F16, "bf16": N.MC_STORE_BF16}[kind]
        self.set_option(N.MC_OPT_STORAGE, code)

    def profile(self) -> dict:
        cap = 16
        names = (ctypes.c_char_p * cap)()
        counts = (ctypes.c_int64 * cap)()
        ms = (ctypes.c_double * cap)()
        n_out = ctypes.c_int32()
        self._check(self._L.mc_profile_read(self._h, cap, ctypes.addressof(names),
                                            ctypes.addressof(counts), ctypes.addressof(ms),
                                            ctypes.addressof(n_out)))
        return {names[i].decode(): (int(counts[i]), float(ms[i])) for i in range(n_out.value)}

    def profile_reset(self):
        self._check(self._L.mc_profile_reset(self._h))

    def save_state(self) -> bytes:
        """Checkpoint of the solver state (mc_save_state) as bytes."""
        size = ctypes.c_uint64()
        self._check(self._L.mc_state_size(self._h, ctypes.byref(size)))
        buf = (ctypes.c_char * size.value)()
        self._check(self._L.mc_save_state(self._h, buf, size.value))
        return bytes(buf)

    def load_state(self, state: bytes):
        """Restore a checkpoint from save_state (mc_load_state)."""
        buf = ctypes.create_string_buffer(state, len(state))
        self._check(self._L.mc_load_state(self._h, buf, len(state)))

    def iteration(self) -> int:
        out = ctypes.c_uint64()
        self._check(self._L.mc_iteration(self._h, ctypes.addressof(out)))
        return out.value


def shared_load_peak(reps: int = 20):
    """Measured conflict-free 64-bit shared-load rate of the current device
    (mc_measure_shared_load_peak): dict with bytes_per_s, bytes_per_clk_per_sm,
    sm_ghz and sms, or None if the measurement failed."""
    out = np.zeros(3)
    st = lib().mc_measure_shared_load_peak(int(reps), out.ctypes.data)
    if st != 0:
        return None
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count \
        if torch is not None and torch.cuda.is_available() else None
    return {"bytes_per_s": float(out[0]), "bytes_per_clk_per_sm": float(out[1]), "sm_ghz": float(out[2]),
            "sms": sms}


def project_gate(ctx: Context, gate: int, x, field=None):
    """Differentiable A_i x = A D_{u_i} x on CUDA tensors (torch autograd).

    `field` (2 x n x n, dense-field contexts) replaces the gate's field first
    when given; gradients flow to x (A_i^* of the output gradient) and to the
    field (mc_vjp).  See autograd.GateProjection."""
    from .autograd import GateProjection
    return GateProjection.apply(ctx, gate, x, field)


def batch_spdhg_run(contexts, epochs: int, seeds, streams=None, ps=None):
    """SPDHG epochs on many independent slice contexts at once
    (mc_batch_spdhg_run): per context identical to ctx.spdhg_run(epochs,
    seed) but interleaved epoch by epoch across the contexts' streams.
    ps: None, or per context None / N sampling probabilities."""
    count = len(contexts)
    if streams is None:
        streams = [0] * count
    if ps is None:
        ps = [None] * count
    arr = (ctypes.c_void_p * count)(*[c._h for c in contexts])
    one = [c._sampling(s, t, p) for c, s, t, p in zip(contexts, seeds, streams, ps)]
    smp = (N.mc_sampling * count)(*[N.mc_sampling(o.seed, o.stream, o.p) for o in one])
    failed = ctypes.c_int32(-1)
    L = lib()
    if torch is not None and torch.cuda.is_available():
        cur = torch.cuda.current_stream()
        for c in contexts:
            if c._stream is not None and c._stream != cur:
                c._stream.wait_stream(cur)
    st = L.mc_batch_spdhg_run(arr, count, int(epochs), smp, ctypes.byref(failed))
    if st != 0:
        who = contexts[failed.value] if 0 <= failed.value < count else contexts[0]
        raise MCError(st, L.mc_last_error(who._h).decode())


class Batch:
    """Slices advanced together, one launch per stage of an SPDHG iteration
    over all of them (mc_batch_create / mc_batch_run).  Keeps the contexts
    alive; close() (or the context manager) releases the batch."""

    def __init__(self, contexts, stream: Optional[int] = None):
        L = lib()
        self._L = L
        self.contexts = list(contexts)
        count = len(self.contexts)
        arr = (ctypes.c_void_p * count)(*[c._h for c in self.contexts])
        out = ctypes.c_void_p()
        st = L.mc_batch_create(arr, count, ctypes.c_void_p(stream) if stream else None, ctypes.byref(out))
        if st != 0:
            msg = L.mc_last_error(self.contexts[0]._h).decode() if count else ""
            raise MCError(st, msg or "mc_batch_create failed")
        self._h = out.value

    def run(self, epochs: int, seeds, streams=None, ps=None):
        """`epochs` SPDHG epochs of every slice; per slice identical to
        ctx.spdhg_run(epochs, seed, stream, p=p)."""
        count = len(self.contexts)
        streams = [0] * count if streams is None else streams
        ps = [None] * count if ps is None else ps
        one = [c._sampling(s, t, p) for c, s, t, p in zip(self.contexts, seeds, streams, ps)]
        smp = (N.mc_sampling * count)(*[N.mc_sampling(o.seed, o.stream, o.p) for o in one])
        if torch is not None and torch.cuda.is_available():
            cur = torch.cuda.current_stream()
            for c in self.contexts:
                if c._stream is not None and c._stream != cur:
                    c._stream.wait_stream(cur)
        failed = ctypes.c_int32(-1)
        st = self._L.mc_batch_run(self._h, int(epochs), smp, ctypes.byref(failed))
        if st != 0:
            raise MCError(st, self._L.mc_batch_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            self._L.mc_batch_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
