"""CUDA path vs the CPU oracle, element by element, through the C ABI.

Tolerances: single operator applications and exchanges agree to rounding (1e-13 relative); FP64 iterates after a
fixed number of V-cycles to 1e-10 relative L2 (the FP64 parity bar); converged solves are compared by the
oracle's own residual of the GPU solution; mixed-precision results state their error against the FP64 oracle.
"""
import numpy as np
import pytest
import torch

import synthetic as syn
from oracle.octree_mg import OracleMG

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _forest(*a, **kw):
    from paper_2403_08063_gb300 import Forest
    return Forest(*a, **kw)


def _inputs(name, coeff, seed=21):
    R, n, keys = syn.workload_forest(name)
    k = syn.lognormal_k_rff(R, n, keys, seed=seed) if coeff else None
    f = syn.gaussian_bump_with_noise(R, n, keys, seed=seed + 1)
    return R, n, keys, k, f


CASES = [
    ("uniform_2x8", False, "C"),
    ("sphere_2x8", False, "C"),
    ("sphere_2x8", False, "P"),
    ("sphere_2x8", True, "C"),
    ("sphere_2x8", True, "P"),
    ("sphere_2x4", True, "C"),
]


def _face_mask(n):
    P = n + 2
    z, y, x = np.meshgrid(np.arange(P), np.arange(P), np.arange(P), indexing="ij")
    inner = lambda a: (a >= 1) & (a <= n)  # noqa: E731
    cnt = (~inner(x)).astype(int) + (~inner(y)).astype(int) + (~inner(z)).astype(int)
    return cnt <= 1  # interior and face ghosts (edge / corner ghosts are never used)


@pytest.mark.parametrize("name,coeff,variant", CASES)
def test_exchange_every_level_matches_oracle(name, coeff, variant):
    R, n, keys, k, f = _inputs(name, coeff)
    F = _forest(R, n, keys, coeff=coeff, interface_flux=(variant == "C"))
    F.set_rhs(f.to(DEV), k.to(DEV) if coeff else None)
    ref = OracleMG(R, n, keys, k_user=None if k is None else k.numpy(), variant=variant)
    assert [(lv.nb, lv.n) for lv in ref.levels] == F.levels()
    rng = np.random.default_rng(5)
    for l, L in enumerate(ref.levels):
        gkeys = F.level_keys(l)
        assert sorted(gkeys) == sorted(L.keys)
        u = rng.normal(size=(L.nb, L.n ** 3))
        padded = F.exchange_level(l, torch.from_numpy(u).to(DEV)).cpu().numpy()
        perm = [L.index[key] for key in gkeys]  # GPU block b is oracle block perm[b]
        Uo = L.zeros()
        for b, ob in enumerate(perm):
            Uo[ob, 1:-1, 1:-1, 1:-1] = u[b].reshape(L.n, L.n, L.n)
        ref.exchange(l, Uo)
        mask = _face_mask(L.n)
        want = Uo[perm][:, mask]
        got = padded[:, mask]
        scale = np.abs(want).max()
        np.testing.assert_allclose(got, want, rtol=0, atol=1e-13 * scale, err_msg=f"level {l}")


@pytest.mark.parametrize("name,coeff,variant", CASES)
def test_apply_matches_oracle(name, coeff, variant):
    R, n, keys, k, f = _inputs(name, coeff)
    F = _forest(R, n, keys, coeff=coeff, interface_flux=(variant == "C"))
    F.set_rhs(f.to(DEV), k.to(DEV) if coeff else None)
    ref = OracleMG(R, n, keys, k_user=None if k is None else k.numpy(), variant=variant, operator_only=True)
    u = np.random.default_rng(6).normal(size=(len(keys), n ** 3))
    got = F.apply(torch.from_numpy(u).to(DEV)).cpu().numpy()
    want = ref.apply_A(u)
    assert np.linalg.norm(got - want) <= 1e-13 * np.linalg.norm(want)


@pytest.mark.parametrize("name,coeff,variant", CASES)
def test_fixed_vcycles_match_oracle(name, coeff, variant):
    R, n, keys, k, f = _inputs(name, coeff)
    F = _forest(R, n, keys, coeff=coeff, interface_flux=(variant == "C"))
    F.set_rhs(f.to(DEV), k.to(DEV) if coeff else None)
    u = torch.zeros_like(f, device=DEV)
    rel = F.vcycle(u, 3)
    ref = OracleMG(R, n, keys, k_user=None if k is None else k.numpy(), variant=variant)
    u_ref, hist = ref.solve(f.numpy(), cycles=3)
    got = u.cpu().numpy()
    assert np.linalg.norm(got - u_ref) <= 1e-10 * np.linalg.norm(u_ref)
    assert abs(rel - hist[-1]) <= 1e-6 * hist[-1]


def test_small_uniform_ten_cycles_manufactured():
    """2^3 blocks of 16^3, FP64, -Laplace with the sin-product manufactured solution, exactly 10 V(2,2) cycles."""
    R, n, keys = syn.workload_forest("uniform_2x16")
    f = syn.sin_product_rhs(R, n, keys)
    F = _forest(R, n, keys)
    assert F.levels() == [(8, 16), (8, 8), (8, 4)]
    F.set_rhs(f.to(DEV))
    u = torch.zeros_like(f, device=DEV)
    F.vcycle(u, 10)
    ref = OracleMG(R, n, keys)
    u_ref, hist = ref.solve(f.numpy(), cycles=10)
    got = u.cpu().numpy()
    assert np.linalg.norm(got - u_ref) <= 1e-10 * np.linalg.norm(u_ref)
    ue = syn.sin_product(R, n, keys).numpy()
    h = 1.0 / (R * n)
    err = np.sqrt(h ** 3 * np.sum((got - ue) ** 2))
    assert 2.5e-4 < err < 3.2e-4  # discretisation error of the 32^3 grid


@pytest.mark.parametrize("coeff,variant", [(False, "C"), (True, "C"), (True, "P")])
def test_coarsest_level_with_interfaces_matches_oracle(coeff, variant):
    """A coarsest level that keeps refinement interfaces: one root, seven level-1 blocks and the eight level-2 blocks
    of the eighth octant (n = 8), with max_coarse = 960 so that the 15 blocks of 4^3 are the coarsest level.  Its
    dense operator is then probed one unknown at a time through the C2F / F2C exchange (a coarsest level without
    interfaces is probed by colour classes instead); 4 FP64 V(2,2) cycles match the oracle's to 1e-10."""
    keys = [(1, i, j, k) for i in (0, 1) for j in (0, 1) for k in (0, 1) if (i, j, k) != (0, 0, 0)]
    keys += [(2, i, j, k) for i in (0, 1) for j in (0, 1) for k in (0, 1)]
    R, n = 1, 8
    k = syn.lognormal_k_rff(R, n, keys, seed=41) if coeff else None
    f = syn.gaussian_bump_with_noise(R, n, keys, seed=42)
    F = _forest(R, n, keys, coeff=coeff, interface_flux=variant == "C", max_coarse=960)
    assert F.levels() == [(15, 8), (15, 4)]
    F.set_rhs(f.to(DEV), k.to(DEV) if coeff else None)
    u = torch.zeros_like(f, device=DEV)
    F.vcycle(u, 4)
    ref = OracleMG(R, n, keys, k_user=None if k is None else k.numpy(), variant=variant, max_coarse=960)
    u_ref, _ = ref.solve(f.numpy(), cycles=4)
    got = u.cpu().numpy()
    assert np.linalg.norm(got - u_ref) <= 1e-10 * np.linalg.norm(u_ref)


@pytest.mark.parametrize("forest", ["sphere_2x8", "mixed_coarsest"])
def test_repeated_set_rhs_gives_the_same_cycles(forest):
    """mg_set_rhs records the coarsest-level probe and inversion as a CUDA graph at its second call and replays it
    afterwards: the V-cycles after the first and the third call with the same k give identical bits (colour probe on
    sphere_2x8's uniform coarsest level, column probe on a coarsest level with interfaces)."""
    if forest == "mixed_coarsest":
        keys = [(1, i, j, k) for i in (0, 1) for j in (0, 1) for k in (0, 1) if (i, j, k) != (0, 0, 0)]
        keys += [(2, i, j, k) for i in (0, 1) for j in (0, 1) for k in (0, 1)]
        R, n, mc = 1, 8, 960
    else:
        R, n, keys = syn.workload_forest(forest)
        mc = 512
    k1 = syn.lognormal_k_rff(R, n, keys, seed=51).to(DEV)
    k2 = syn.lognormal_k_rff(R, n, keys, seed=52).to(DEV)
    f = syn.gaussian_bump_with_noise(R, n, keys, seed=53).to(DEV)
    F = _forest(R, n, keys, coeff=True, max_coarse=mc)
    runs = []
    for kk in (k1, k2, k1):
        F.set_rhs(f, kk)
        u = torch.zeros_like(f)
        F.vcycle(u, 2)
        runs.append(u.clone())
    assert torch.isfinite(runs[0]).all() and not torch.equal(runs[0], runs[1])
    assert torch.equal(runs[0], runs[2])


@pytest.mark.parametrize("coeff", [False, True])
def test_refined_solve_to_1e10_property(coeff):
    """Refined forest (56 + 64 blocks of 16^3): the GPU solve's residual, recomputed by the oracle, is <= 1e-10."""
    R, _, keys = syn.workload_forest("sphere_2x16")
    n = 16
    k = syn.lognormal_k_rff(R, n, keys, seed=31) if coeff else None
    f = syn.gaussian_bump_with_noise(R, n, keys, seed=32)
    F = _forest(R, n, keys, coeff=coeff)
    F.set_rhs(f.to(DEV), k.to(DEV) if coeff else None)
    u = torch.zeros_like(f, device=DEV)
    cyc, rel = F.solve(u, rtol=1e-10, max_cycles=40)
    assert rel <= 1e-10 and cyc <= 16
    ref = OracleMG(R, n, keys, k_user=None if k is None else k.numpy(), operator_only=True)
    assert ref.rel_residual(u.cpu().numpy(), f.numpy()) <= 1.05e-10


@pytest.mark.parametrize("coeff,inner", [(False, 1), (True, 1), (True, 3)])
def test_mixed_precision_solve_error_vs_fp64_oracle(coeff, inner):
    R, n, keys, k, f = _inputs("sphere_2x8", coeff, seed=41)
    F = _forest(R, n, keys, coeff=coeff, precision=1, inner_cycles=inner)
    F.set_rhs(f.to(DEV), k.to(DEV) if coeff else None)
    u = torch.zeros_like(f, device=DEV)
    cyc, rel = F.solve(u, rtol=1e-10, max_cycles=40)
    assert rel <= 1e-10
    ref = OracleMG(R, n, keys, k_user=None if k is None else k.numpy())
    u_ref, hist = ref.solve(f.numpy(), rtol=1e-14, max_cycles=60)
    got = u.cpu().numpy()
    err = np.linalg.norm(got - u_ref) / np.linalg.norm(u_ref)
    print(f"mixed precision ({'k' if coeff else 'Laplace'}): {cyc} cycles, rel residual {rel:.2e}, "
          f"rel L2 error vs FP64 oracle {err:.2e}")
    assert ref.rel_residual(got, f.numpy()) <= 1.05e-10
    assert err < 1e-8


@pytest.mark.parametrize("name,variant", [("sphere_2x8", "C"), ("sphere_2x8", "P"), ("uniform_2x8", "C"),
                                          ("mixed_coarsest", "C")])
def test_face_averaged_coarse_coefficients_fp64_cycles_match_oracle(name, variant):
    """Face-averaged coarse coefficients (coarse_coef 'faces'): three FP64 V(2,2) cycles match the oracle's iterate to
    1e-10, on refined forests (both interface variants; merged octets below 4^3), a uniform one, and a coarsest
    level that keeps refinement interfaces; the adjoint on the same operator hierarchy matches the oracle's."""
    if name == "mixed_coarsest":
        keys = [(1, i, j, k) for i in (0, 1) for j in (0, 1) for k in (0, 1) if (i, j, k) != (0, 0, 0)]
        keys += [(2, i, j, k) for i in (0, 1) for j in (0, 1) for k in (0, 1)]
        R, n, mc = 1, 8, 960
    else:
        R, n, keys = syn.workload_forest(name)
        mc = 512
    k = syn.lognormal_k_rff(R, n, keys, seed=151)
    f = syn.gaussian_bump_with_noise(R, n, keys, seed=152)
    F = _forest(R, n, keys, coeff=True, interface_flux=(variant == "C"), max_coarse=mc, coarse_coef="faces")
    F.set_rhs(f.to(DEV), k.to(DEV))
    u = torch.zeros_like(f, device=DEV)
    F.vcycle(u, 3)
    ref = OracleMG(R, n, keys, k_user=k.numpy(), variant=variant, max_coarse=mc, coarse_coef="faces")
    u_ref, _ = ref.solve(f.numpy(), cycles=3)
    got = u.cpu().numpy()
    err = np.linalg.norm(got - u_ref) / np.linalg.norm(u_ref)
    print(f"face-averaged coarse coefficients, {name} {variant}: 3 FP64 cycles, rel L2 to the oracle {err:.2e}")
    assert err <= 1e-10
    g = np.random.default_rng(153).normal(size=u_ref.shape)
    lam, _ = F.adjoint(torch.from_numpy(u_ref).to(DEV), torch.from_numpy(g).to(DEV), want_k=False, rtol=1e-13,
                       max_cycles=60)
    lam_ref = ref.adjoint_solve(g, rtol=1e-13)
    assert np.linalg.norm(lam.cpu().numpy() - lam_ref) <= 1e-10 * np.linalg.norm(lam_ref)
    F.close()


@pytest.mark.parametrize("name,coeff,variant", [("sphere_2x8", True, "C"), ("sphere_2x8", False, "P"),
                                                ("uniform_2x8", True, "C")])
def test_diagonal_exchange_every_level_matches_oracle(name, coeff, variant):
    """Forests with the trilinear prolongation: mg_exchange_level also fills the edge and corner ghosts (copies from a
    same-level block across the edge or corner, else extrapolated from the face / edge ghosts).  Every entry of every
    padded block of every level (interior, face, edge and corner ghosts) matches the oracle's exchange followed by
    exchange_diagonal to 1e-13."""
    R, n, keys, k, f = _inputs(name, coeff)
    F = _forest(R, n, keys, coeff=coeff, interface_flux=(variant == "C"), prolongation="trilinear")
    F.set_rhs(f.to(DEV), k.to(DEV) if coeff else None)
    ref = OracleMG(R, n, keys, k_user=None if k is None else k.numpy(), variant=variant, prolongation="trilinear")
    rng = np.random.default_rng(6)
    for l, L in enumerate(ref.levels):
        gkeys = F.level_keys(l)
        u = rng.normal(size=(L.nb, L.n ** 3))
        padded = F.exchange_level(l, torch.from_numpy(u).to(DEV)).cpu().numpy()
        perm = [L.index[key] for key in gkeys]
        Uo = L.zeros()
        for b, ob in enumerate(perm):
            Uo[ob, 1:-1, 1:-1, 1:-1] = u[b].reshape(L.n, L.n, L.n)
        ref.exchange(l, Uo)
        ref.exchange_diagonal(l, Uo)
        want = Uo[perm].reshape(L.nb, -1)
        got = padded.reshape(L.nb, -1)
        np.testing.assert_allclose(got, want, rtol=0, atol=1e-13 * np.abs(want).max(), err_msg=f"level {l}")
    F.close()


@pytest.mark.parametrize("name,variant,coarse_coef", [("sphere_2x8", "C", "faces"), ("sphere_2x8", "P", "k"),
                                                      ("uniform_2x8", "C", "faces"), ("mixed_coarsest", "C", "k")])
def test_trilinear_prolongation_fp64_cycles_match_oracle(name, variant, coarse_coef):
    """The trilinear prolongation (edge and corner ghosts of the coarse correction, then the 8-point interpolation,
    then a full exchange): three FP64 V(2,2) cycles match the oracle's iterate to 1e-10 on refined forests (both
    interface variants, merged octets), a uniform one, and a coarsest level that keeps interfaces.  The adjoint,
    which transposes the face-neighbour prolongation only, refuses the forest."""
    from paper_2403_08063_gb300 import MGError
    if name == "mixed_coarsest":
        keys = [(1, i, j, k) for i in (0, 1) for j in (0, 1) for k in (0, 1) if (i, j, k) != (0, 0, 0)]
        keys += [(2, i, j, k) for i in (0, 1) for j in (0, 1) for k in (0, 1)]
        R, n, mc = 1, 8, 960
    else:
        R, n, keys = syn.workload_forest(name)
        mc = 512
    k = syn.lognormal_k_rff(R, n, keys, seed=161)
    f = syn.gaussian_bump_with_noise(R, n, keys, seed=162)
    F = _forest(R, n, keys, coeff=True, interface_flux=(variant == "C"), max_coarse=mc, coarse_coef=coarse_coef,
                prolongation="trilinear")
    F.set_rhs(f.to(DEV), k.to(DEV))
    u = torch.zeros_like(f, device=DEV)
    F.vcycle(u, 3)
    ref = OracleMG(R, n, keys, k_user=k.numpy(), variant=variant, max_coarse=mc, coarse_coef=coarse_coef,
                   prolongation="trilinear")
    u_ref, _ = ref.solve(f.numpy(), cycles=3)
    got = u.cpu().numpy()
    err = np.linalg.norm(got - u_ref) / np.linalg.norm(u_ref)
    print(f"trilinear prolongation, {name} {variant} {coarse_coef}: 3 FP64 cycles, rel L2 to the oracle {err:.2e}")
    assert err <= 1e-10
    with pytest.raises(MGError):
        F.adjoint(torch.from_numpy(u_ref).to(DEV), torch.from_numpy(u_ref).to(DEV), want_k=False)
    F.close()
