"""mg_solve_host: the solve from host buffers (staging copies, k set-up overlapped with the f copy) gives the same bits
as mg_set_rhs + mg_solve on device copies of the same inputs, with a zero or a given initial guess, and rejects
bad arguments."""
import pytest
import torch

import synthetic as syn

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.mark.parametrize("coeff,precision", [(False, 0), (True, 1)])
def test_host_solve_matches_device_solve(coeff, precision):
    from paper_2403_08063_gb300 import Forest
    R, n, keys = syn.workload_forest("sphere_2x8")
    f = syn.gaussian_bump_with_noise(R, n, keys, seed=61)
    k = syn.lognormal_k_rff(R, n, keys, seed=62) if coeff else None
    u0 = 0.01 * syn.gaussian_bump_with_noise(R, n, keys, seed=63)
    F = Forest(R, n, keys, coeff=coeff, precision=precision, inner_cycles=3)
    for guess in (None, u0):
        F.set_rhs(f.to(DEV), k.to(DEV) if coeff else None)
        ud = torch.zeros_like(f, device=DEV) if guess is None else guess.to(DEV)
        cd, rd = F.solve(ud, rtol=1e-10)
        fh = f.pin_memory()
        kh = k.pin_memory() if coeff else None
        uh = torch.empty_like(f).pin_memory()
        u_out, ch, rh = F.solve_host(fh, kh, u=uh, u0=None if guess is None else guess, rtol=1e-10)
        assert u_out is uh and ch == cd and rh == rd
        assert torch.equal(uh, ud.cpu())
    # pageable buffers work as well
    u_out, ch, rh = F.solve_host(f, k, rtol=1e-10)
    assert rh <= 1e-10
    F.close()


def test_host_solve_arguments_are_checked():
    from paper_2403_08063_gb300 import Forest, MGError
    R, n, keys = syn.workload_forest("uniform_2x8")
    f = syn.gaussian_bump_with_noise(R, n, keys, seed=64)
    F = Forest(R, n, keys, coeff=True)
    with pytest.raises(MGError):
        F.solve_host(f)  # coeff == 1 needs k
    with pytest.raises(TypeError):
        F.solve_host(f.to(DEV), f)
    bad = syn.lognormal_k_rff(R, n, keys, seed=65)
    bad[3] = -1.0
    with pytest.raises(MGError):
        F.solve_host(f, bad)
    F.close()
