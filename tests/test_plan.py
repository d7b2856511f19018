"""Invariants of the host-side plan of the sweeps (tiles, sliced copies,
warp ranges), checked on the CPU: csrc/plss_plan.cu is plain C++ and is
built here with g++ together with a small test shim (tests/host)."""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_2207_07615_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2207_07615_gb300", "csrc")
K_SLICED, K_STAGED, K_MASK = 0x100, 0x200, 0xFF


@pytest.fixture(scope="module")
def shim(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    out = str(tmp_path_factory.mktemp("plan") / "libplanshim.so")
    subprocess.run([gxx, "-std=c++17", "-O1", "-shared", "-fPIC", "-I" + CSRC, "-x", "c++",
                    os.path.join(CSRC, "plss_plan.cu"), os.path.join(ROOT, "tests", "host", "plan_shim.cpp"),
                    "-o", out], check=True)
    L = C.CDLL(out)
    L.shim_plan.restype = C.c_void_p
    L.shim_plan.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_int64, C.c_int64, C.c_int64,
                            C.c_int32, C.c_int32, C.c_int32, C.c_int64, C.c_int32]
    L.shim_count.restype = C.c_int64
    L.shim_count.argtypes = [C.c_void_p, C.c_int32]
    L.shim_copy.argtypes = [C.c_void_p, C.c_int32, C.c_void_p]
    L.shim_free.argtypes = [C.c_void_p]
    L.shim_slice_lanes.restype = C.c_int32
    L.shim_slice_lanes.argtypes = [C.c_int64, C.c_int64]
    L.shim_tile_target.restype = C.c_int64
    L.shim_tile_target.argtypes = [C.c_int64, C.c_int64, C.c_int32, C.c_int32]
    return L


def plan(L, ptr, idx, val, f32, slice, g, nwarps=64, slots=(4864, 6080), shift=0):
    ptr = np.ascontiguousarray(ptr, dtype=np.int32)
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    val = np.ascontiguousarray(val, dtype=np.float64)
    h = L.shim_plan(ptr.ctypes.data, idx.ctypes.data, val.ctypes.data, len(ptr) - 1, int(ptr[-1]),
                    slots[0], slots[1], int(f32), int(slice), int(g), nwarps, int(shift))
    try:
        def get(which, dtype, width=1):
            n = L.shim_count(h, which if which != 6 else 4)
            a = np.empty(n * width, dtype=dtype)
            if n:
                L.shim_copy(h, which, a.ctypes.data)
            return a
        tiles = get(0, np.int32, 4).reshape(-1, 4)
        return dict(tiles=tiles, first=get(1, np.int32), ptr=get(2, np.int32), seg=get(3, np.int32),
                    idx=get(4, np.int32), val=get(6, np.float64), wr=get(5, np.int32))
    finally:
        L.shim_free(h)


def cases():
    out = {}
    A, _, _ = synth.overdetermined_scaled(m=20000, n=4000, per_row=8, seed=3, scale_decades=1.0)
    out["uniform_rows"] = (A.row_ptr, A.col_idx, A.val)
    At = A.scipy().T.tocsr()
    out["uniform_cols"] = (At.indptr, At.indices, At.data)          # ~40 per segment
    P, _, _ = synth.powerlaw_underdetermined(m=3000, n=30000, mean_len=20, max_len=5000, seed=4)
    out["powerlaw_rows"] = (P.row_ptr, P.col_idx, P.val)
    Pt = P.scipy().T.tocsr()
    out["powerlaw_cols"] = (Pt.indptr, Pt.indices, Pt.data)         # many empty columns
    out["tiny"] = (np.array([0, 2, 2, 3]), np.array([0, 1, 1]), np.array([1.0, 2.0, 3.0]))
    out["empty"] = (np.array([0]), np.array([], dtype=np.int32), np.array([]))
    return out


CASES = cases()


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("f32", [0, 1])
@pytest.mark.parametrize("slice_", [0, 1])
@pytest.mark.parametrize("shift", [-1, 0, 1])
def test_plan_invariants(shim, name, f32, slice_, shift):
    ptr, idx, val = (np.asarray(a) for a in CASES[name])
    nseg, nnz = len(ptr) - 1, int(ptr[-1])
    g = shim.shim_slice_lanes(max(nnz, 1), max(nseg, 1)) if slice_ else 1
    p = plan(shim, ptr, idx, val, f32, slice_, g, shift=shift)
    tiles = p["tiles"]
    lens = np.diff(ptr)
    # tiles partition [0, nseg) in order
    assert len(tiles) >= 1
    assert tiles[0, 1] == 0 and tiles[-1, 2] == nseg
    assert np.all(tiles[1:, 1] == tiles[:-1, 2]) and np.all(tiles[:, 2] >= tiles[:, 1])
    target = shim.shim_tile_target(max(nnz, 1), 6080 if f32 else 4864, f32, shift)
    assert (256 if shift < 0 else 1024) <= target <= (2048 if f32 else 16384)
    for sys, b, e, grp in tiles:
        tnz = int(ptr[e] - ptr[b])
        if (grp & K_MASK) == 0 and e > b:                    # one segment for the whole CTA
            assert e - b == 1
        if grp & K_STAGED:                                   # fits the shared-memory stage
            assert tnz <= 2048 and e - b <= 1024 and not grp & K_SLICED
        if f32 and e > b and not grp & K_SLICED and grp & K_MASK:
            assert grp & K_STAGED                            # FP32 tiles that are not sliced are staged
        if not slice_:
            assert not grp & K_SLICED
    # sliced copy: every nonzero of a sliced tile exactly once, where the layout says
    sl_ptr, seg, sidx, sval, first = p["ptr"], p["seg"], p["idx"], p["val"], p["first"]
    per = 32 // g
    seen = np.zeros(nseg, dtype=np.int64)
    for ti, (sys, b, e, grp) in enumerate(tiles):
        if not grp & K_SLICED:
            continue
        nsl = (e - b + per - 1) // per
        padded = 0
        for s in range(first[ti], first[ti] + nsl):
            off, width = sl_ptr[s], (sl_ptr[s + 1] - sl_ptr[s]) // 32
            assert (sl_ptr[s + 1] - sl_ptr[s]) % 32 == 0
            padded += 32 * width
            slots = seg[32 * s: 32 * s + 32]
            for q in range(per):
                grpslots = slots[q * g:(q + 1) * g]
                assert np.all(grpslots == grpslots[0])        # g lanes share a segment
                r = int(grpslots[0])
                if r < 0:
                    assert np.all(sidx[off + np.arange(width)[:, None] * 32 + q * g + np.arange(g)] == -1)
                    continue
                assert b <= r < e
                seen[r] += 1
                assert (lens[r] + g - 1) // g <= width
                for k in range(lens[r]):
                    pos = off + 32 * (k // g) + q * g + k % g
                    assert sidx[pos] == idx[ptr[r] + k] and sval[pos] == val[ptr[r] + k]
                for k in range(lens[r], width * g):               # padding
                    pos = off + 32 * (k // g) + q * g + k % g
                    assert sidx[pos] == -1 and sval[pos] == 0.0
        tnz = int(ptr[e] - ptr[b])
        assert padded * 4 <= tnz * 5 + 32 * g * 4            # at most 1/4 padding (sorted slices)
    sliced_rows = np.zeros(nseg, dtype=bool)
    for sys, b, e, grp in tiles:
        if grp & K_SLICED:
            sliced_rows[b:e] = True
    assert np.all(seen[sliced_rows] == 1) and np.all(seen[~sliced_rows] == 0)
    # warp ranges: only when every tile is sliced; monotone cover of all slices
    wr = p["wr"]
    if len(tiles) and np.all(tiles[:, 3] & K_SLICED):
        assert len(wr) == 64 + 1 and wr[0] == 0 and wr[-1] == len(sl_ptr) - 1
        assert np.all(np.diff(wr) >= 0)
        # balance: a slice costs its elements plus 256 (offsets, slot map,
        # results); no warp gets more than an equal share plus one slice
        cost = np.diff(sl_ptr).astype(np.int64) + 256
        prefix = np.concatenate([[0], np.cumsum(cost)])
        share = -(-int(prefix[-1]) // 64)
        per_warp = prefix[wr[1:]] - prefix[wr[:-1]]
        assert per_warp.max() <= share + (cost.max() if len(cost) else 0)
    else:
        assert len(wr) == 0


def test_slice_lanes(shim):
    assert shim.shim_slice_lanes(8_000_000, 1_000_000) == 1      # 8 per row
    assert shim.shim_slice_lanes(8_000_000, 200_000) == 4        # 40 per column
    assert shim.shim_slice_lanes(10**9, 1000) == 32              # capped


def test_tile_shift_scales_the_target(shim):
    """The autotuner's knob: 2^shift times the default target, clamped to
    [256, 16,384] (FP64) or [256, 2,048] (FP32, the staging limit)."""
    for nnz, slots in ((8_000_000, 4864), (40_000, 4864), (2_600_000, 608)):
        for f32 in (0, 1):
            base = shim.shim_tile_target(nnz, slots, f32, 0)
            cap = 2048 if f32 else 16384
            for shift in (-2, -1, 1, 2):
                want = base * 2 ** shift if shift > 0 else base >> -shift
                assert shim.shim_tile_target(nnz, slots, f32, shift) == min(cap, max(256, want))


def _check_sliced_vectorized(p, ptr, idx, val, g):
    """The sliced copy holds every nonzero of the sliced tiles exactly once,
    where the layout says, and padding elsewhere: numpy over all elements at
    once (the loop form above is for the small cases)."""
    tiles, sl_ptr, seg, sidx, sval, first = p["tiles"], p["ptr"], p["seg"], p["idx"], p["val"], p["first"]
    nseg = len(ptr) - 1
    lens = np.diff(ptr).astype(np.int64)
    per = 32 // g
    S = len(sl_ptr) - 1
    widths = np.diff(sl_ptr).astype(np.int64)
    assert np.all(widths % 32 == 0) and sl_ptr[0] == 0 and len(seg) == 32 * S
    widths //= 32
    # slices of each sliced tile, consecutive from first[ti]; rows inside the tile
    owner_b = np.full(S, -1, dtype=np.int64)
    owner_e = np.full(S, -1, dtype=np.int64)
    sliced_rows = np.zeros(nseg, dtype=bool)
    for ti, (sys, b, e, grp) in enumerate(tiles):
        if not grp & K_SLICED:
            continue
        nsl = (e - b + per - 1) // per
        sl = slice(first[ti], first[ti] + nsl)
        assert np.all(owner_b[sl] == -1)                      # no slice shared by two tiles
        owner_b[sl], owner_e[sl] = b, e
        sliced_rows[b:e] = True
        pad = int(32 * widths[sl].sum())
        assert pad * 4 <= int(ptr[e] - ptr[b]) * 5 + 32 * g * 4
    assert np.all(owner_b >= 0)                                # every slice belongs to a tile
    lanes = seg.reshape(S, per, g).astype(np.int64)
    assert np.all(lanes == lanes[:, :, :1])                   # g lanes share a segment
    r = lanes[:, :, 0]
    used = r >= 0
    rs = r[used]
    assert np.all((rs >= np.repeat(owner_b, per).reshape(S, per)[used]) &
                  (rs < np.repeat(owner_e, per).reshape(S, per)[used]))
    seen = np.bincount(rs, minlength=nseg)
    assert np.all(seen[sliced_rows] == 1) and np.all(seen[~sliced_rows] == 0)
    wide = np.repeat(widths, per).reshape(S, per)
    assert np.all((lens[rs] + g - 1) // g <= wide[used])
    # element by element: position -> (slice, step j, lane) -> (row, k)
    E = int(sl_ptr[-1])
    pos = np.arange(E, dtype=np.int64)
    s_of = np.repeat(np.arange(S, dtype=np.int64), 32 * widths)
    local = pos - sl_ptr[s_of]
    j, lane = local // 32, local % 32
    row = seg[32 * s_of + lane].astype(np.int64)
    k = j * g + lane % g
    real = row >= 0
    real[real] = k[real] < lens[row[real]]
    src = np.asarray(ptr, dtype=np.int64)[row[real]] + k[real]
    assert np.array_equal(sidx[real], np.asarray(idx)[src])
    assert np.array_equal(sval[real], np.asarray(val, dtype=np.float64)[src])
    assert np.all(sidx[~real] == -1) and np.all(sval[~real] == 0.0)
    assert int(real.sum()) == int(lens[sliced_rows].sum())


def _full_size(workload):
    if workload == "overdetermined_1e6x2e5":
        return synth.overdetermined_scaled(m=1_000_000, n=200_000, per_row=8, seed=0)[0]
    if workload == "powerlaw_1e5x1e6":
        return synth.powerlaw_underdetermined(m=100_000, n=1_000_000, mean_len=20.0, max_len=5000, seed=0)[0]
    return synth.laplacian7(126)


@pytest.mark.parametrize("workload,side", [("overdetermined_1e6x2e5", "rows"), ("overdetermined_1e6x2e5", "cols"),
                                           ("powerlaw_1e5x1e6", "rows"), ("powerlaw_1e5x1e6", "cols"),
                                           ("laplacian_126", "rows")])
@pytest.mark.parametrize("f32", [0, 1])
def test_plan_invariants_at_benchmark_size(shim, workload, side, f32):
    """The benchmark systems at full size -- 1,000,000 x 200,000 with 8
    nonzeros a row, 100,000 x 1,000,000 with Zipf row lengths up to 5,000,
    and the 7-point Laplacian on 126^3 points (symmetric: its columns are its
    rows) -- planned as a context on one GB300 plans them (152 SMs x 4 CTAs
    x 8 warps of warp ranges): tiles partition each side, the sliced copy
    holds every nonzero of the sliced tiles exactly once, and where every
    tile is sliced the warp ranges cover every slice in balanced shares."""
    A = _full_size(workload)
    if side == "rows":
        ptr, idx, val = np.asarray(A.row_ptr), np.asarray(A.col_idx), np.asarray(A.val)
    else:
        At = A.scipy().T.tocsr()
        ptr, idx, val = At.indptr, At.indices, At.data
    nseg, nnz = len(ptr) - 1, int(ptr[-1])
    nwarps = 152 * 4 * 8
    g = shim.shim_slice_lanes(nnz, nseg)
    p = plan(shim, ptr, idx, val, f32, 1, g, nwarps=nwarps)
    tiles = p["tiles"]
    assert tiles[0, 1] == 0 and tiles[-1, 2] == nseg and np.all(tiles[1:, 1] == tiles[:-1, 2])
    if workload != "powerlaw_1e5x1e6":
        assert np.all(tiles[:, 3] & K_SLICED)                # short uniform segments: all sliced
    _check_sliced_vectorized(p, ptr, idx, val, g)
    wr, sl_ptr = p["wr"], p["ptr"]
    if not np.all(tiles[:, 3] & K_SLICED):
        assert len(wr) == 0
        return
    assert len(wr) == nwarps + 1 and wr[0] == 0 and wr[-1] == len(sl_ptr) - 1 and np.all(np.diff(wr) >= 0)
    cost = np.diff(sl_ptr).astype(np.int64) + 256
    prefix = np.concatenate([[0], np.cumsum(cost)])
    share = -(-int(prefix[-1]) // nwarps)
    assert (prefix[wr[1:]] - prefix[wr[:-1]]).max() <= share + cost.max()


def test_vectorized_check_rejects_planted_defects(shim):
    """The whole-array check fails on a swapped element, a row sliced twice
    and a padding slot that holds an index."""
    ptr, idx, val = (np.asarray(a) for a in CASES["uniform_cols"])
    g = shim.shim_slice_lanes(int(ptr[-1]), len(ptr) - 1)
    p = plan(shim, ptr, idx, val, 0, 1, g, nwarps=64)
    _check_sliced_vectorized(p, ptr, idx, val, g)
    real = np.nonzero(p["idx"] >= 0)[0]
    pad = np.nonzero(p["idx"] < 0)[0]
    assert len(pad) > 0

    def planted(key, fn):
        q = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in p.items()}
        fn(q[key])
        with pytest.raises(AssertionError):
            _check_sliced_vectorized(q, ptr, idx, val, g)

    def swap(a):
        i, j = real[0], real[-1]
        a[i], a[j] = a[j], a[i]

    def twice(a):
        a[g:2 * g] = a[0]                       # the second lane group repeats the first's segment

    def fill(a):
        a[pad[0]] = 0

    planted("idx", swap)
    planted("seg", twice)
    planted("idx", fill)
