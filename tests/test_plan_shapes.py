"""Host-side launch-shape rules (mc_plan_shapes, no GPU): the layouts' zero
guards cover the forward projector's clamp reach, the ring fits the shared
memory a block may use, every chosen shape has a compiled kernel, and the
choices at the benchmark's sizes are the measured ones."""
import ctypes
import math

import pytest

from paper_2410_10503_gb300 import _native as N

SMS = 152                       # the GB300's SMs
RING_BYTES = 221440             # shared memory of the forward's ring per block
# (lines per chunk, ring stages, lines per sampled part) the forward is compiled for
FORWARD_SHAPES = {(2, 5, 2), (4, 5, 4), (8, 5, 8), (8, 3, 8), (16, 3, 16), (16, 3, 8)}


def plan(n, na=180, nb=None, sms=SMS):
    nb = nb if nb is not None else n + 17
    lib = N.load()
    out = (ctypes.c_int32 * 10)()
    geom = N.mc_geometry(n, na, nb)
    st = lib.mc_plan_shapes(ctypes.byref(geom), sms, out)
    return st, dict(zip(("guard", "P", "lines", "lc", "cl", "ring", "pj", "Gb", "Pb", "warps"), list(out)))


def bp_window(pj):
    return (math.ceil(math.sqrt(31.0 * 31.0 + (pj - 1.0) ** 2)) + 7) & ~1


@pytest.mark.parametrize("n", list(range(2, 130)) + list(range(130, 2049, 37)) + [256, 384, 512, 520, 768, 1024, 2048])
def test_shape_invariants(n):
    st, s = plan(n)
    assert st == 0
    assert s["guard"] in (17, 33) and s["guard"] >= 2 * s["cl"] + 1       # the clamp's reach
    assert s["P"] % 4 == 0 and s["P"] >= n + 2 * s["guard"]               # guards after the data too
    assert s["lines"] >= n and s["lines"] % 8 == 0 and s["lines"] % s["lc"] == 0
    assert (s["lc"], s["ring"], s["cl"]) in FORWARD_SHAPES
    assert s["ring"] * s["lc"] * s["P"] * 8 <= RING_BYTES
    assert s["pj"] in (4, 8, 14, 16, 28)
    assert s["Pb"] >= n + 17 + 2 * s["Gb"] and bp_window(s["pj"]) <= s["Pb"]
    # two-part chunks carry two parts' state: fewer warps with more registers each
    assert s["warps"] == (15 if (s["lc"], s["cl"]) == (16, 8) else 23)
    assert 32 * (s["warps"] + 1) <= 1024


def test_measured_choices_at_the_benchmark_sizes():
    want = {
        128: dict(guard=33, lc=16, cl=16, ring=3),     # whole 16-line chunks (-9% per epoch)
        256: dict(guard=33, lc=16, cl=16, ring=3),
        384: dict(guard=33, lc=16, cl=16, ring=3),
        512: dict(guard=17, P=548, lc=16, cl=8, ring=3, pj=28, warps=15),   # two-part chunks, 28-row tiles
        768: dict(guard=17, lc=8, cl=8, ring=3, pj=16),
        1024: dict(guard=17, lc=8, cl=8, ring=3, pj=28),
        2048: dict(guard=17, lc=2, cl=2, ring=5),
        520: dict(guard=17, lc=8, cl=8, ring=5),       # 520 lines: no whole 16-line chunks
    }
    for n, w in want.items():
        st, s = plan(n, na=round(1.4 * n) if n != 512 else 720, nb=n + 17 if n != 512 else 729)
        assert st == 0
        for k, v in w.items():
            assert s[k] == v, (n, k, s)


def test_plan_refuses_what_create_refuses():
    for n, na, nb in ((1, 8, 8), (2049, 8, 8), (64, 0, 8), (64, 8, 8193)):
        st, _ = plan(n, na, nb)
        assert st == N.MC_EINVAL
    lib = N.load()
    out = (ctypes.c_int32 * 10)()
    assert lib.mc_plan_shapes(None, SMS, out) == N.MC_EINVAL
    assert lib.mc_plan_shapes(ctypes.byref(N.mc_geometry(64, 8, 8)), 0, out) == N.MC_EINVAL


def test_python_plan_shapes():
    import paper_2410_10503_gb300 as M
    sh = M.plan_shapes(512, 720, 729, SMS)
    assert sh == dict(zip(M.SHAPE_KEYS, plan(512, 720, 729)[1].values()))
    assert (sh["lines_per_chunk"], sh["lines_per_part"], sh["consumer_warps"], sh["rows_per_thread"]) == (16, 8, 15, 28)
    with pytest.raises(M.MCError):
        M.plan_shapes(4096, 8, 8, SMS)
