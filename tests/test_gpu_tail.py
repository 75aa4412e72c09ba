"""The persistent tail kernel: the FP32 V-cycle from a level down to the coarsest in one cooperative launch whose
resident CTAs walk the recorded step list with grid barriers.  It must reproduce the launched V-cycle bit for bit,
from any level it accepts, on a refined forest (interface exchanges, octet merging below 4^3) and a uniform one."""
import pytest
import torch

import synthetic as syn

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.mark.parametrize("name,coeff,coarse_coef", [("sphere_2x16", True, "k"), ("sphere_2x16", False, "k"),
                                                    ("uniform_4x16", True, "k"), ("sphere_2x16", True, "faces"),
                                                    ("uniform_4x16", True, "faces"), ("sphere_2x32", True, "faces"),
                                                    ("uniform_4x64", True, "faces"), ("uniform_4x64", False, "k")])
def test_tail_reproduces_the_launched_vcycle(name, coeff, coarse_coef):
    """Also with face-averaged coarse coefficients, whose coarse levels run the halved-face coefficient mode, and on
    32^3 and 64^3 blocks, where the launched V-cycle's prolongation runs the z-column kernel and the tail the
    cell-per-thread body."""
    from paper_2403_08063_gb300 import Forest
    R, n, keys = syn.workload_forest(name)
    dev = torch.device(DEV)
    f = syn.gaussian_bump_with_noise(R, n, keys, seed=51, device=dev)
    k = syn.lognormal_k_rff(R, n, keys, seed=52, device=dev) if coeff else None
    F = Forest(R, n, keys, coeff=coeff, precision=1, inner_cycles=2, coarse_coef=coarse_coef)
    F.set_rhs(f, k)
    nlev = len(F.levels())
    F.set_tail(-1)
    assert F.tail_level() == -1
    ref = torch.zeros_like(f)
    rel_ref = F.vcycle(ref, 3)
    for lt in range(nlev):
        F.set_tail(lt)
        assert F.tail_level() == lt
        u = torch.zeros_like(f)
        rel = F.vcycle(u, 3)
        assert torch.equal(u, ref), lt
        assert rel == rel_ref
    # a full solve with the tail from level 1 meets the tolerance in the same number of cycles
    F.set_tail(-1)
    u0 = torch.zeros_like(f)
    c0, r0 = F.solve(u0, rtol=1e-10, max_cycles=60)
    F.set_tail(1)
    u1 = torch.zeros_like(f)
    c1, r1 = F.solve(u1, rtol=1e-10, max_cycles=60)
    assert c1 == c0 and torch.equal(u1, u0)


def test_tail_arguments_are_checked():
    from paper_2403_08063_gb300 import Forest, MGError
    R, n, keys = syn.workload_forest("uniform_2x8")
    F64 = Forest(R, n, keys, precision=0)
    with pytest.raises(MGError):
        F64.set_tail(0)
    assert F64.tail_level() == -1
    F = Forest(R, n, keys, precision=1)
    with pytest.raises(MGError):
        F.set_tail(len(F.levels()))
    F.set_tail(0)
    assert F.tail_level() == 0
