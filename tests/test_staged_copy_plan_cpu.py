"""Every bulk copy of the staged FP32 smoother, checked on the host against the rules of cp.async.bulk.

mg_staged_copy_plan runs the kernel's own copy planner (the code its producer thread executes) on the host and
returns every mbarrier arm and bulk copy of one block's CTAs.  For every staged shape offered at block edges 32, 64
and 128, the three coefficient modes (constant k: u and f staged; 1/k: with kappa; stored halved face coefficients:
with ax, ay, az) and both colours this test checks:
  * the size rule and 16-byte alignment of both addresses (global: the block stride keeps every block and half on a
    16-byte boundary; shared: the slots);
  * that each barrier is armed with exactly the bytes of the copies that complete it, below the 2^20 tx limit;
  * that every copy reads inside its block's slot of the pool and writes inside the ring area, below the barriers;
  * that each copy brings the plane segment the consumers read at that step (rows y0 - 1 .. y0 + TY of the other
    colour's padded plane, rows y0 .. y0 + TY - 1 of the own colour's) and holds it whole;
  * that a copy never lands on a slot whose plane a consumer warp may still read when the producer issues it.
No GPU is involved.
"""
import ctypes

import numpy as np
import pytest

from paper_2403_08063_gb300 import _lib

I64 = ctypes.c_int64


def _plan(lib, lg, coeff, colour, idx):
    shape = (ctypes.c_int32 * 5)()
    ns = ctypes.c_int32()
    smem, blk, nrec = I64(), I64(), I64()
    st = lib.mg_staged_copy_plan(lg, coeff, colour, idx, shape, ctypes.byref(ns), ctypes.byref(smem),
                                 ctypes.byref(blk), 0, None, ctypes.byref(nrec))
    assert st == 0
    if idx >= ns.value:
        return ns.value, None, None, None, None
    buf = (I64 * (10 * nrec.value))()
    st = lib.mg_staged_copy_plan(lg, coeff, colour, idx, shape, ctypes.byref(ns), ctypes.byref(smem),
                                 ctypes.byref(blk), nrec.value, buf, ctypes.byref(nrec))
    assert st == 0
    rec = np.frombuffer(buf, dtype=np.int64).reshape(-1, 10).copy()
    return ns.value, tuple(shape), smem.value, blk.value, rec


def _overlap(a, b):
    return a[0] < b[1] and b[0] < a[1]


def _check(lg, coeff, colour, shape, smem, blk, rec):
    n = 1 << lg
    P, H = n + 2, (n + 2) // 2
    HALF = P * P * H
    _, TY, TZ, D, R = shape
    G = D + 1
    assert rec.shape[0] > 0
    # shared memory: rings, then 2 G + 2 mbarriers (8 bytes each, 8-byte aligned)
    bar0 = smem - 8 * (2 * G + 2)
    assert bar0 % 8 == 0 and smem <= 200 * 1024
    assert blk % 16 == 0 and blk >= 4 * 2 * HALF
    other_arrays = {0: [0], 1: [0, 1], 2: [0, 1, 4, 5]}[coeff]
    own_arrays = {0: [2], 1: [2, 3], 2: [2, 3, 6, 7]}[coeff]
    half_start = {a: colour * HALF for a in (0, 1, 4, 5)}
    half_start.update({a: (colour ^ 1) * HALF for a in (2, 3, 6, 7)})
    tiles = (n // TY) * (n // TZ)
    assert set(rec[:, 0]) == set(range(tiles))
    for tile in range(tiles):
        ty, tz = tile % (n // TY), tile // (n // TY)
        y0, z0 = ty * TY, tz * TZ
        rt = rec[rec[:, 0] == tile]
        # issue order: first planes, then groups 0 .. TZ - 1, each an arm followed by its copies
        groups = list(dict.fromkeys(rt[:, 3].tolist()))
        assert groups == [-1] + list(range(TZ))
        other_slot, own_slot = {}, {}  # padded plane -> shared byte ranges of the copies holding it
        for g in groups:
            rg = rt[rt[:, 3] == g]
            assert rg[0, 1] == 0 and (rg[1:, 1] == 1).all()  # one arm, then copies
            bar = 0 if g < 0 else 1 + g % G
            assert (rg[:, 2] == bar).all()
            armed = int(rg[0, 7])
            copies = rg[1:]
            assert armed == copies[:, 7].sum() and 0 < armed < (1 << 20)
            want_arrays = other_arrays * (2 if g < 0 else 1) + ([] if g < 0 else own_arrays)
            assert sorted(copies[:, 5].tolist()) == sorted(want_arrays)
            new = []
            for c in copies:
                _, _, _, _, dst, arr, src, nbytes, lead, ln = (int(v) for v in c)
                assert nbytes > 0 and nbytes % 16 == 0 and dst % 16 == 0 and src % 16 == 0
                assert 0 <= src and src + nbytes <= blk  # reads stay inside the block's slot of the pool
                assert 0 <= dst and dst + nbytes <= bar0  # writes stay in the rings, below the barriers
                assert 0 <= lead <= 3 and lead + ln <= nbytes // 4  # the wanted segment is copied whole
                seg = src // 4 + lead - half_start[arr]
                assert 0 <= seg and seg + ln <= HALF
                if arr in other_arrays:  # other colour: rows y0 - 1 .. y0 + TY of one padded plane
                    assert ln == (TY + 2) * H and seg % (P * H) == y0 * H
                    zp = seg // (P * H)
                else:        # own colour: rows y0 .. y0 + TY - 1 of one padded plane
                    assert ln == TY * H and seg % (P * H) == (y0 + 1) * H
                    zp = seg // (P * H)
                new.append((arr, zp, (dst, dst + nbytes)))
            o_planes = sorted({zp for arr, zp, _ in new if arr in other_arrays})
            w_planes = sorted({zp for arr, zp, _ in new if arr in own_arrays})
            if g < 0:
                assert o_planes == [z0, z0 + 1] and not w_planes
            else:
                # the consumers at plane z0 + g read the other colour's plane z0 + g + 1 and their own plane z0 + g
                assert o_planes == [z0 + g + 2] and w_planes == [z0 + g + 1]
                # group g is issued once every warp is done with plane z0 + g - G (for g = G - 1: once the first
                # plane is in registers): warps may still read other planes z0 + g - G + 1 .. z0 + g (padded one
                # more) and own planes z0 + g - G + 1 .. z0 + g - 1; before that, the first two other planes too
                live_o = [p for p in other_slot if max(z0 + 1, z0 + g - G + 2) <= p <= z0 + g + 1]
                if g < G - 1:
                    live_o.append(z0)
                live_w = [p for p in own_slot if z0 + max(0, g - G + 1) + 1 <= p <= z0 + g]
                for arr, zp, rg_ in new:
                    for p in live_o:
                        for r2 in other_slot[p]:
                            assert not _overlap(rg_, r2), (shape, tile, g, p)
                    for p in live_w:
                        for r2 in own_slot[p]:
                            assert not _overlap(rg_, r2), (shape, tile, g, p)
            for arr, zp, rg_ in new:
                (other_slot if arr in other_arrays else own_slot).setdefault(zp, []).append(rg_)
            # copies of one group never overlap each other
            for i in range(len(new)):
                for k in range(i + 1, len(new)):
                    assert not _overlap(new[i][2], new[k][2])


@pytest.mark.parametrize("lg", [5, 6, 7])
@pytest.mark.parametrize("coeff", [0, 1, 2])
def test_every_staged_copy_follows_the_bulk_copy_rules(lg, coeff):
    lib = _lib.load()
    ns, *_ = _plan(lib, lg, coeff, 0, 1 << 30)
    assert ns > 0
    for colour in (0, 1):
        for idx in range(ns):
            _, shape, smem, blk, rec = _plan(lib, lg, coeff, colour, idx)
            _check(lg, coeff, colour, shape, smem, blk, rec)


def test_copy_plan_rejects_bad_arguments():
    lib = _lib.load()
    ns, nrec = ctypes.c_int32(), I64()
    for args in ((4, 0, 0), (8, 0, 0), (6, 3, 0), (6, 0, 2)):
        assert lib.mg_staged_copy_plan(*args, 0, None, ctypes.byref(ns), None, None, 0, None, ctypes.byref(nrec)) == 1
