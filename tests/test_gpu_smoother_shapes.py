"""Launch shapes of the FP32 smoother: the column kernel (cells per thread along z, threads per CTA) and the
kernel whose other-colour planes are staged in shared memory by bulk copies (rows per CTA, planes per CTA, planes
in flight, rows per thread).

A shape only decides which thread updates which cell of a colour, and the half-sweep's cells are independent, so
every shape must give the same bits.  Checked on a refined forest with 32^3 blocks (C2F / F2C interfaces, boundary
reflection and same-level write-through on every level from 32^3 down to 4^3 blocks) and on a uniform forest of
32^3 blocks (no interface: only write-through ghosts), for constant and variable coefficients.
"""
import pytest
import torch

import synthetic as syn

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.mark.parametrize("coeff", [False, True])
@pytest.mark.parametrize("workload", ["sphere_2x32", "uniform_2x32"])
def test_every_smoother_shape_gives_identical_bits(coeff, workload):
    from paper_2403_08063_gb300 import Forest
    R, n, keys = syn.workload_forest(workload)
    dev = torch.device(DEV)
    f = syn.gaussian_bump_with_noise(R, n, keys, seed=31, device=dev)
    k = syn.lognormal_k_rff(R, n, keys, seed=32, device=dev) if coeff else None
    F = Forest(R, n, keys, coeff=coeff, precision=1, inner_cycles=2)
    F.set_rhs(f, k)
    nlev = len(F.levels())
    shapes = [F.smoother_shapes(l) for l in range(nlev)]
    assert all(shapes)
    # both kernels are offered on the 32^3 level, and the tuner picked an offered shape there
    assert {s[0] for s in shapes[0]} == {1, 2}
    assert F.smoother_shape(0) in shapes[0]
    ref = None
    for i in range(max(len(s) for s in shapes)):
        for l in range(nlev):
            sh = shapes[l][i % len(shapes[l])]
            F.set_smoother_shape(l, sh)
            assert F.smoother_shape(l) == sh
        u = torch.zeros_like(f)
        F.vcycle(u, 2)
        if ref is None:
            ref = u.clone()
            assert torch.isfinite(ref).all() and ref.abs().max() > 0
        else:
            assert torch.equal(u, ref), [shapes[l][i % len(shapes[l])] for l in range(nlev)]


@pytest.mark.parametrize("refined", [False, True])
def test_stored_face_levels_run_the_staged_smoother_with_identical_bits(refined):
    """Face-averaged coarse levels keep three halved face arrays (coefficient mode 3); with 32^3 blocks they are
    offered the staged kernel too, which stages the three arrays of both colours with u and f.  Every shape of such a
    level gives the bits of the column kernel.  64^3 leaf blocks, 4^3 uniform roots or 2^3 roots refined twice
    around a ball (interface ghosts on the 32^3 level)."""
    from paper_2403_08063_gb300 import Forest
    n = 64
    if refined:
        R = 2
        keys = syn.balance_2to1(syn.refine_ball(R, (0.5, 0.5, 0.5), 0.25, 2, open_ball=True), R, "26")
    else:
        R = 4
        keys = syn.uniform_leaves(R)
    dev = torch.device(DEV)
    f = syn.gaussian_bump_with_noise(R, n, keys, seed=33, device=dev)
    k = syn.lognormal_k_rff(R, n, keys, seed=34, device=dev)
    F = Forest(R, n, keys, coeff=True, precision=1, inner_cycles=2, coarse_coef="faces")
    F.set_rhs(f, k)
    lev = [l for l in range(len(F.levels())) if l > 0 and F.smoother_shapes(l)
           and {s[0] for s in F.smoother_shapes(l)} == {1, 2}]
    assert lev, "no face-averaged level with staged shapes"
    ref = None
    for l in lev:
        for sh in F.smoother_shapes(l):
            F.set_smoother_shape(l, sh)
            u = torch.zeros_like(f)
            F.vcycle(u, 2)
            if ref is None:
                ref = u.clone()
                assert torch.isfinite(ref).all() and ref.abs().max() > 0
            else:
                assert torch.equal(u, ref), (l, sh)
        F.set_smoother_shape(l, (1, 1, 256, 0, 0))


def test_smoother_shape_arguments_are_checked():
    from paper_2403_08063_gb300 import Forest, MGError
    R, n, keys = syn.workload_forest("uniform_2x4")
    F = Forest(R, n, keys, precision=1)
    offered = F.smoother_shapes(0)
    assert (1, 1, 256, 0, 0) in offered and all(s[0] == 1 for s in offered)  # column kernel only on 4^3 blocks
    for bad in ((1, 3, 256, 0, 0), (1, 1, 100, 0, 0), (1, 8, 256, 0, 0), (3, 1, 128, 0, 0), (2, 2, 4, 2, 1),
                (0, 0, 0, 0, 0)):
        with pytest.raises(MGError):
            F.set_smoother_shape(0, bad)
    with pytest.raises(MGError):
        F.set_smoother_shape(len(F.levels()), (1, 1, 256, 0, 0))
    F64 = Forest(R, n, keys, precision=0)
    assert F64.smoother_shape(0) == (0, 0, 0, 0, 0) and F64.smoother_shapes(0) == []
    with pytest.raises(MGError):
        F64.set_smoother_shape(0, (1, 1, 256, 0, 0))


@pytest.mark.parametrize("shape", [(2, 16, 16, 4, 4), (2, 16, 32, 4, 4)])
def test_staged_smoother_is_bit_reproducible_next_to_other_kernels(shape):
    """The staged smoother's shared-memory ring must not depend on how fast its warps run: with unrelated kernels
    occupying the SMs from another stream, one FP32-in-FP64 step of 4^3 roots of 64^3 cells (variable k, the 512^3
    workload's shapes) repeated eight times gives the same bits every time.  Before the first planes' loads were
    fenced against the bulk copy that refills their slot, most repeats here differed."""
    from paper_2403_08063_gb300 import Forest
    R, n = 4, 64
    keys = syn.uniform_leaves(R)
    dev = torch.device(DEV)
    k = syn.lognormal_k_rff(R, n, keys, seed=3, device=dev)
    f = syn.uniform_rhs(len(keys), n, seed=4).to(dev)
    F = Forest(R, n, keys, coeff=True, precision=1, inner_cycles=2)
    F.set_rhs(f, k)
    F.set_smoother_shape(0, shape)
    side = torch.cuda.Stream()
    busy = torch.randn(64 * 1024 * 1024, device=dev)
    outs = []
    for rep in range(8):
        u = torch.zeros_like(f)
        torch.cuda.synchronize()
        if rep % 2:
            with torch.cuda.stream(side):
                for _ in range(20):
                    busy.mul_(1.0000001).add_(1e-7)
        F.vcycle(u, 1)
        torch.cuda.synchronize()
        outs.append(u)
    for o in outs[1:]:
        assert torch.equal(o, outs[0])
    F.close()
