"""Every bulk copy of the staged FP32 residual + restriction, checked on the host against the rules of cp.async.bulk.

mg_restrict_copy_plan runs the kernel's own copy planner (the code its producer thread executes) on the host and
returns every mbarrier arm and bulk copy of one block's CTAs.  For the tile the library launches and a few others,
fine block edges 64 and 128 and the three coefficient modes, this test checks:
  * the size rule and 16-byte alignment of both addresses;
  * that each plane's barrier is armed with exactly the bytes of its copies, below the 2^20 tx limit;
  * that every copy reads inside its block's slot of the pool and writes inside its plane's ring slot;
  * that each copy brings the plane segment the consumers read (rows y0 .. y0 + TY + 1 of the stencil arrays, rows
    y0 + 1 .. y0 + TY of f, f only for the tile's own planes) and holds it whole, the copies of a plane disjoint;
  * that the planes one coarse step reads sit in distinct slots, and that a plane is only written into a slot whose
    previous plane no step after its release reads.
No GPU is involved.
"""
import ctypes

import numpy as np
import pytest

from paper_2403_08063_gb300 import _lib

I64 = ctypes.c_int64


def _plan(lib, lg, coeff, shape):
    sh = (ctypes.c_int32 * 3)(*shape)
    smem, blk, nrec = I64(), I64(), I64()
    st = lib.mg_restrict_copy_plan(lg, coeff, sh, ctypes.byref(smem), ctypes.byref(blk), 0, None, ctypes.byref(nrec))
    assert st == 0
    buf = (I64 * (11 * nrec.value))()
    st = lib.mg_restrict_copy_plan(lg, coeff, sh, ctypes.byref(smem), ctypes.byref(blk), nrec.value, buf,
                                   ctypes.byref(nrec))
    assert st == 0
    return tuple(sh), smem.value, blk.value, np.frombuffer(buf, dtype=np.int64).reshape(-1, 11).copy()


def _check(lg, coeff, shape, smem, blk, rec):
    n = 1 << lg
    P, H = n + 2, (n + 2) // 2
    HALF = P * P * H
    TY, TZ, D = shape
    RS = 4 + 2 * D
    NU = {0: 1, 1: 2, 2: 4}[coeff]
    lo, lw = (TY + 2) * H, TY * H
    so, sw = (lo + 6) & ~3, (lw + 6) & ~3
    ss = 4 * (2 * NU * so + 2 * sw)  # bytes per ring slot
    assert smem == RS * ss + 8 * 2 * RS and smem <= 200 * 1024
    assert blk % 16 == 0 and blk >= 4 * 2 * HALF
    tiles = (n // TY) * (n // TZ)
    assert sorted(set(rec[:, 0].tolist())) == list(range(tiles))
    for tile in range(tiles):
        ty, tz = tile % (n // TY), tile // (n // TY)
        y0, z0 = ty * TY, tz * TZ
        rt = rec[rec[:, 0] == tile]
        assert list(dict.fromkeys(rt[:, 3].tolist())) == list(range(TZ + 2))
        for q in range(TZ + 2):
            rq = rt[rt[:, 3] == q]
            assert rq[0, 1] == 0 and (rq[1:, 1] == 1).all()  # one arm, then the copies
            slot = q % RS
            assert (rq[:, 2] == slot).all()
            copies = rq[1:]
            assert int(rq[0, 8]) == copies[:, 8].sum() and 0 < rq[0, 8] < (1 << 20)
            want = [(a, h) for a in range(NU) for h in (0, 1)] + ([(NU, 0), (NU, 1)] if 1 <= q <= TZ else [])
            assert sorted((int(c[5]), int(c[6])) for c in copies) == sorted(want)
            spans = []
            for c in copies:
                _, _, _, _, dst, arr, half, src, nbytes, lead, ln = (int(v) for v in c)
                assert nbytes > 0 and nbytes % 16 == 0 and dst % 16 == 0 and src % 16 == 0
                assert 0 <= src and src + nbytes <= blk  # inside the block's slot of the pool
                assert slot * ss <= dst and dst + nbytes <= (slot + 1) * ss  # inside the plane's ring slot
                assert 0 <= lead <= 3 and lead + ln <= nbytes // 4  # the wanted segment copied whole
                seg = src // 4 + lead - half * HALF
                assert 0 <= seg and seg + ln <= HALF and src // 4 >= half * HALF  # inside its half
                if arr < NU:
                    assert ln == lo and seg == ((z0 + q) * P + y0) * H
                else:
                    assert ln == lw and seg == ((z0 + q) * P + y0 + 1) * H
                spans.append((dst, dst + nbytes))
            spans.sort()
            assert all(a[1] <= b[0] for a, b in zip(spans, spans[1:]))
    # ring: step g reads planes 2g .. 2g + 3, releases 2g and 2g + 1; plane q >= RS is issued after plane q - RS is
    # released, i.e. after step (q - RS) // 2, when no step reads a plane below 2 ((q - RS) // 2 + 1)
    for g in range(TZ // 2):
        assert len({p % RS for p in range(2 * g, 2 * g + 4)}) == 4
    for q in range(RS, TZ + 2):
        first_live = 2 * ((q - RS) // 2 + 1)
        assert all(p % RS != q % RS for p in range(first_live, q))


@pytest.mark.parametrize("lg", [6, 7])
@pytest.mark.parametrize("coeff", [0, 1, 2])
def test_every_staged_restriction_copy_follows_the_bulk_copy_rules(lg, coeff):
    lib = _lib.load()
    shapes = [(0, 0, 0), (8, 16, 1), (16 if lg == 6 else 8, 8, 2), (2, 2, 0)]
    seen = set()
    for shape in shapes:
        sh, smem, blk, rec = _plan(lib, lg, coeff, shape)
        if sh in seen:
            continue
        seen.add(sh)
        _check(lg, coeff, sh, smem, blk, rec)
    assert len(seen) >= 3


def test_restriction_copy_plan_rejects_bad_arguments():
    lib = _lib.load()
    nrec = I64()
    for lg, coeff, shape in ((5, 0, (0, 0, 0)), (8, 0, (0, 0, 0)), (6, 3, (0, 0, 0)), (6, 1, (3, 32, 1)),
                             (6, 1, (16, 6, 1)), (6, 1, (16, 32, 9)), (6, 2, (64, 64, 4))):
        sh = (ctypes.c_int32 * 3)(*shape)
        assert lib.mg_restrict_copy_plan(lg, coeff, sh, None, None, 0, None, ctypes.byref(nrec)) == 1
    assert lib.mg_restrict_copy_plan(6, 0, None, None, None, 0, None, ctypes.byref(nrec)) == 1
