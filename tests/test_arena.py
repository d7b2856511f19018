"""Placement of served systems in the server's device arena (plss_arena.h,
plain C++ built here with g++ and a test shim): all-or-nothing placement in
the lowest free slot with first-fit ranges, no overlap between resident
systems, exact accounting, coalescing release, and the admission test of a
request that could never fit -- checked against a model kept in Python over
random place/release sequences."""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2207_07615_gb300", "csrc")
I64P = C.POINTER(C.c_int64)


@pytest.fixture(scope="module")
def L(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    out = str(tmp_path_factory.mktemp("arena") / "libarenashim.so")
    subprocess.run([gxx, "-std=c++17", "-O1", "-shared", "-fPIC", "-I" + CSRC,
                    os.path.join(ROOT, "tests", "host", "arena_shim.cpp"), "-o", out], check=True)
    lib = C.CDLL(out)
    lib.arena_new.restype = C.c_void_p
    lib.arena_new.argtypes = [C.c_int32] + [C.c_int64] * 8
    lib.arena_free.argtypes = [C.c_void_p]
    lib.arena_place.restype = C.c_int32
    lib.arena_place.argtypes = [C.c_void_p, I64P, I64P]
    lib.arena_release.argtypes = [C.c_void_p, I64P, I64P]
    lib.arena_ever_fits.restype = C.c_int32
    lib.arena_ever_fits.argtypes = [C.c_void_p, I64P]
    lib.arena_counters.argtypes = [C.c_void_p, I64P]
    lib.arena_free_ranges.restype = C.c_int64
    lib.arena_free_ranges.argtypes = [C.c_void_p, C.c_int32, I64P, C.c_int64]
    return lib


def arr(v):
    return (C.c_int64 * len(v))(*[int(x) for x in v])


class Model:
    """Live intervals per allocator (rows, cols, nnzs, slcs, els), slots and tiles."""

    def __init__(self, slots, caps, tiles):
        self.slots, self.caps, self.tmax = slots, list(caps), list(tiles)
        self.live = {}   # key -> (need, place)

    def lens(self, q):
        return [q[0] + 1, q[1] + 1, q[2], q[3], q[4]]

    def first_fit(self, w, length):
        if length <= 0:
            return 0
        taken = sorted((p[1 + w], self.lens(q)[w]) for q, p in self.live.values() if self.lens(q)[w] > 0)
        pos = 0
        for off, ln in taken:
            if off - pos >= length:
                return pos
            pos = max(pos, off + ln)
        return pos if self.caps[w] - pos >= length else None

    def predict(self, q):
        used = {p[0] for _, p in self.live.values()}
        free = [s for s in range(self.slots) if s not in used]
        if not free:
            return None
        tiles = [sum(v[0][5 + i] for v in self.live.values()) for i in range(3)]
        if any(tiles[i] + q[5 + i] > self.tmax[i] for i in range(3)):
            return None
        offs = []
        for w, ln in enumerate(self.lens(q)):
            o = self.first_fit(w, ln)
            if o is None:
                return None
            offs.append(o)
        return [free[0]] + offs


def counters(L, h):
    out = (C.c_int64 * 9)()
    L.arena_counters(h, out)
    return list(out)


def free_ranges(L, h, w):
    buf = (C.c_int64 * 4096)()
    k = L.arena_free_ranges(h, w, buf, 2048)
    return [(buf[2 * i], buf[2 * i + 1]) for i in range(k)]


@pytest.mark.parametrize("seed", range(6))
def test_random_place_release_against_model(L, seed):
    rng = np.random.default_rng(seed)
    slots = int(rng.integers(1, 9))
    caps = [int(rng.integers(50, 400)), int(rng.integers(50, 400)), int(rng.integers(200, 2000)),
            int(rng.integers(0, 60)) * (seed % 2), int(rng.integers(0, 3000)) * (seed % 2)]
    tiles = [int(rng.integers(5, 40)) for _ in range(3)]
    h = L.arena_new(slots, *caps, *tiles)
    model = Model(slots, caps, tiles)
    try:
        key = 0
        for step in range(600):
            if model.live and rng.random() < 0.45:
                k = list(model.live)[int(rng.integers(len(model.live)))]
                q, p = model.live.pop(k)
                L.arena_release(h, arr(q), arr(p))
            else:
                q = [int(rng.integers(0, 60)), int(rng.integers(0, 60)), int(rng.integers(0, 300)),
                     int(rng.integers(0, 8)) * (seed % 2), int(rng.integers(0, 400)) * (seed % 2),
                     int(rng.integers(1, 6)), int(rng.integers(1, 6)), int(rng.integers(1, 4))]
                before = counters(L, h), [free_ranges(L, h, w) for w in range(5)]
                want = model.predict(q)
                out = (C.c_int64 * 6)()
                ok = L.arena_place(h, arr(q), out)
                assert bool(ok) == (want is not None), (step, q, want)
                if ok:
                    assert list(out) == want, (step, q)          # lowest slot, first fit
                    model.live[key] = (q, list(out))
                    key += 1
                else:                                            # all or nothing
                    assert (counters(L, h), [free_ranges(L, h, w) for w in range(5)]) == before
            # accounting and disjointness
            c = counters(L, h)
            live = list(model.live.values())
            assert c[:3] == [sum(q[5 + i] for q, _ in live) for i in range(3)]
            assert c[3:8] == [sum(model.lens(q)[w] for q, _ in live) for w in range(5)]
            assert c[8] == len(live)
            for w in range(5):
                ivs = sorted((p[1 + w], model.lens(q)[w]) for q, p in live if model.lens(q)[w] > 0)
                for (o1, l1), (o2, _) in zip(ivs, ivs[1:]):
                    assert o1 + l1 <= o2
                assert all(0 <= o and o + ln <= caps[w] for o, ln in ivs)
                # free ranges are the exact complement, coalesced
                fr = free_ranges(L, h, w)
                assert all(a + la < b for (a, la), (b, _) in zip(fr, fr[1:]))
                assert sum(ln for _, ln in fr) + sum(ln for _, ln in ivs) == caps[w]
        for q, p in model.live.values():
            L.arena_release(h, arr(q), arr(p))
        assert counters(L, h) == [0] * 9
        for w in range(5):
            assert free_ranges(L, h, w) == ([(0, caps[w])] if caps[w] > 0 else [])
    finally:
        L.arena_free(h)


def test_ever_fits_is_the_empty_arena_test(L):
    caps, tiles = [100, 80, 500, 10, 900], [7, 6, 5]
    h = L.arena_new(2, *caps, *tiles)
    try:
        base = [99, 79, 500, 10, 900, 7, 6, 5]               # exactly the capacities
        assert L.arena_ever_fits(h, arr(base))
        for i in range(8):
            q = list(base)
            q[i] += 1
            assert not L.arena_ever_fits(h, arr(q)), i
        out = (C.c_int64 * 6)()
        assert L.arena_place(h, arr(base), out) == 1         # and it is placed at once
        assert L.arena_place(h, arr([0, 0, 0, 0, 0, 0, 0, 0]), out) == 0   # rows and columns are full
    finally:
        L.arena_free(h)
    h = L.arena_new(0, *caps, *tiles)                        # no slot at all
    try:
        assert not L.arena_ever_fits(h, arr([0] * 8))
    finally:
        L.arena_free(h)
