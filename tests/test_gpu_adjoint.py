"""Adjoint path on the GPU: A^T, the adjoint solve, dL/df and dL/dk against the oracle and against finite
differences.  L = 1/2 sum (u - u_t)^2; lambda solves A^T lambda = u - u_t; dL/df = lambda; dL/dk = -lambda^T dA/dk u.
"""
import numpy as np
import pytest
import torch

import synthetic as syn
from oracle.octree_mg import OracleMG

pytestmark = pytest.mark.gpu
DEV = "cuda:0"

CASES = [("sphere_2x8", False, "C"), ("sphere_2x8", True, "C"), ("sphere_2x8", True, "P"), ("uniform_2x8", True, "C")]


def _setup(name, coeff, variant, precision=0):
    from paper_2403_08063_gb300 import Forest
    R, n, keys = syn.workload_forest(name)
    k = syn.lognormal_k_rff(R, n, keys, seed=61) if coeff else None
    f = syn.gaussian_bump_with_noise(R, n, keys, seed=62)
    F = Forest(R, n, keys, coeff=coeff, interface_flux=(variant == "C"), precision=precision)
    F.set_rhs(f.to(DEV), k.to(DEV) if coeff else None)
    return R, n, keys, k, f, F


@pytest.mark.parametrize("name,coeff,variant", CASES)
def test_apply_transpose_matches_oracle_and_dot_product(name, coeff, variant):
    R, n, keys, k, f, F = _setup(name, coeff, variant)
    ref = OracleMG(R, n, keys, k_user=None if k is None else k.numpy(), variant=variant, operator_only=True)
    rng = np.random.default_rng(63)
    x = rng.normal(size=(len(keys), n ** 3))
    y = rng.normal(size=(len(keys), n ** 3))
    got = F.apply_transpose(torch.from_numpy(x).to(DEV)).cpu().numpy()
    want = ref.apply_AT(x)
    assert np.linalg.norm(got - want) <= 1e-13 * np.linalg.norm(want)
    Ay = F.apply(torch.from_numpy(y).to(DEV)).cpu().numpy()
    assert abs(np.sum(x * Ay) - np.sum(got * y)) <= 1e-12 * np.linalg.norm(x) * np.linalg.norm(Ay)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("name,coeff,variant", CASES)
def test_adjoint_solve_and_gradients_match_oracle(name, coeff, variant, precision):
    """lambda and dL/dk against the oracle's adjoint; precision 1 forests run FP32 transposed cycles inside FP64
    defect correction, precision 0 forests FP64 ones: both reach the FP64 result."""
    R, n, keys, k, f, F = _setup(name, coeff, variant, precision)
    ref = OracleMG(R, n, keys, k_user=None if k is None else k.numpy(), variant=variant)
    u_ref, _ = ref.solve(f.numpy(), rtol=1e-14, max_cycles=60)
    ut = syn.sin_target(R, n, keys, seed=64).numpy()
    g = u_ref - ut
    lam_ref = ref.adjoint_solve(g, rtol=1e-13)
    u_d = torch.from_numpy(u_ref).to(DEV)
    lam, gk = F.adjoint(u_d, torch.from_numpy(g).to(DEV), want_k=coeff, rtol=1e-13, max_cycles=60)
    lam = lam.cpu().numpy()
    assert np.linalg.norm(lam - lam_ref) <= 1e-10 * np.linalg.norm(lam_ref)
    if coeff:
        gk_ref = ref.grad_k(u_ref, lam_ref)
        assert np.linalg.norm(gk.cpu().numpy() - gk_ref) <= 1e-9 * np.linalg.norm(gk_ref)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("variant", ["C", "P"])
def test_adjoint_with_face_averaged_coarse_coefficients(variant, precision):
    """The transposed cycles with face-averaged coarse levels (FP64, and FP32 inside FP64 defect correction) reach
    the oracle's adjoint and gradient: the coarse operator changes the cycle, not lambda."""
    from paper_2403_08063_gb300 import Forest
    R, n, keys = syn.workload_forest("sphere_2x8")
    k = syn.lognormal_k_rff(R, n, keys, seed=61)
    f = syn.gaussian_bump_with_noise(R, n, keys, seed=62)
    F = Forest(R, n, keys, coeff=True, interface_flux=(variant == "C"), precision=precision, coarse_coef="faces")
    F.set_rhs(f.to(DEV), k.to(DEV))
    ref = OracleMG(R, n, keys, k_user=k.numpy(), variant=variant)
    u_ref, _ = ref.solve(f.numpy(), rtol=1e-14, max_cycles=60)
    g = u_ref - syn.sin_target(R, n, keys, seed=64).numpy()
    lam_ref = ref.adjoint_solve(g, rtol=1e-13)
    lam, gk = F.adjoint(torch.from_numpy(u_ref).to(DEV), torch.from_numpy(g).to(DEV), want_k=True, rtol=1e-13,
                        max_cycles=60)
    assert np.linalg.norm(lam.cpu().numpy() - lam_ref) <= 1e-10 * np.linalg.norm(lam_ref)
    gk_ref = ref.grad_k(u_ref, lam_ref)
    assert np.linalg.norm(gk.cpu().numpy() - gk_ref) <= 1e-9 * np.linalg.norm(gk_ref)
    F.close()


def _interface_cells(keys, n, count, rng):
    """(leaf, cell) pairs: cells on a block face that borders a coarser or a finer block."""
    index = set(keys)
    out = []
    for b, (l, i, j, k) in enumerate(keys):
        for axis in range(3):
            for side in (0, 1):
                p = [i, j, k]
                p[axis] += 1 if side else -1
                coarser = (l - 1, p[0] // 2, p[1] // 2, p[2] // 2) in index
                finer = any((l + 1, 2 * p[0] + a, 2 * p[1] + bb, 2 * p[2] + c) in index
                            for a in (0, 1) for bb in (0, 1) for c in (0, 1))
                if (l, *p) in index or not (coarser or finer):
                    continue
                t = rng.integers(0, n, size=2)
                cell = [0, 0, 0]
                cell[axis] = n - 1 if side else 0
                others = [d for d in range(3) if d != axis]
                cell[others[0]], cell[others[1]] = int(t[0]), int(t[1])
                out.append((b, (cell[2] * n + cell[1]) * n + cell[0]))
    sel = rng.choice(len(out), size=count, replace=False)
    return [out[s] for s in sel]


def test_gradients_match_finite_differences_on_refined_31m_cells():
    """Sphere-refined forest of 4^3 roots of 32^3 cells (448 + 512 blocks, 31,457,280 cells), log-normal k.

    Forward solves use FP32 cycles inside FP64 defect correction to 1e-11 (the FP64 rounding floor of f - A u for
    this coefficient contrast is near 3e-12); the adjoint solve runs FP32 transposed cycles inside FP64 defect
    correction to 1e-11.  Central
    differences on 10 seeded random cells and 10 seeded cells next to coarse-fine faces, evaluated through the
    difference solution delta = u+ - u- (exactly the central difference of L, without the cancellation of two
    nearly equal losses): step 1e-6 for f (L is quadratic in f); step 1e-4 relative for k, because at 1e-6 the
    k-difference sits at the FP64 noise of the solves (measured: worst 4e-5 at 1e-6, <= 5e-8 at 1e-4).
    """
    from paper_2403_08063_gb300 import Forest
    R, n, keys = syn.workload_forest("sphere_4x32")
    dev = torch.device(DEV)
    k = syn.lognormal_k_rff(R, n, keys, seed=71, device=dev)
    f = syn.gaussian_bump_with_noise(R, n, keys, seed=72, device=dev)
    ut = syn.sin_target(R, n, keys, seed=73, device=dev)
    Fm = Forest(R, n, keys, coeff=True, precision=1, inner_cycles=3)
    Fm.set_rhs(f, k)
    u = torch.zeros_like(f)
    Fm.solve(u, rtol=1e-11, max_cycles=60)
    lam, gk = Fm.adjoint(u, u - ut, want_k=True, rtol=1e-11, max_cycles=80)
    rng = np.random.default_rng(74)
    cells = [(int(b), int(c)) for b, c in zip(rng.integers(0, len(keys), 10), rng.integers(0, n ** 3, 10))]
    cells += _interface_cells(keys, n, 10, rng)
    eps = 1e-6
    # dL/df: delta = A^-1 (2 eps e_i); FD = delta . (u - u_t) / (2 eps)
    Fd = Forest(R, n, keys, coeff=True, precision=1, inner_cycles=3)
    worst_f = 0.0
    for b, c in cells:
        e = torch.zeros_like(f)
        e[b, c] = 2 * eps
        Fd.set_rhs(e, k)
        d = torch.zeros_like(f)
        Fd.solve(d, rtol=1e-11, max_cycles=60)
        fd = float((d * (u - ut)).sum()) / (2 * eps)
        an = float(lam[b, c])
        worst_f = max(worst_f, abs(fd - an) / abs(an))
    # dL/dk: A(k+) delta = (A(k-) - A(k+)) u-, u+ = u- + delta; FD = delta . ((u+ + u-)/2 - u_t) / (2 eps k_m)
    Fp = Forest(R, n, keys, coeff=True, precision=1, inner_cycles=3)
    worst_k = 0.0
    eps = 1e-4
    for b, c in cells:
        km = float(k[b, c])
        kp, kmn = k.clone(), k.clone()
        kp[b, c] = km * (1 + eps)
        kmn[b, c] = km * (1 - eps)
        Fd.set_rhs(f, kmn)
        um = torch.zeros_like(f)
        Fd.solve(um, rtol=1e-11, max_cycles=60)
        rhs = Fd.apply(um)
        Fp.set_rhs(f, kp)
        rhs = rhs - Fp.apply(um)
        Fp.set_rhs(rhs, kp)
        d = torch.zeros_like(f)
        Fp.solve(d, rtol=1e-11, max_cycles=60)
        fd = float((d * (um + 0.5 * d - ut)).sum()) / (2 * eps * km)
        an = float(gk[b, c])
        worst_k = max(worst_k, abs(fd - an) / abs(an))
    print(f"finite differences on 20 cells: worst relative error dL/df {worst_f:.2e}, dL/dk {worst_k:.2e}")
    assert worst_f < 1e-6 and worst_k < 1e-6


def test_autograd_function_matches_directional_differences():
    """MGSolveFn: gradients w.r.t. f and k of L = 1/2 ||u(f, k) - u_t||^2 through loss.backward()."""
    from paper_2403_08063_gb300 import Forest, MGSolveFn
    R, n, keys = syn.workload_forest("sphere_2x8")
    dev = torch.device(DEV)
    k = syn.lognormal_k_rff(R, n, keys, seed=81, device=dev)
    f = syn.gaussian_bump_with_noise(R, n, keys, seed=82, device=dev)
    ut = syn.sin_target(R, n, keys, seed=83, device=dev)
    F = Forest(R, n, keys, coeff=True)
    fr = f.clone().requires_grad_(True)
    kr = k.clone().requires_grad_(True)
    u = MGSolveFn.apply(fr, kr, F, 1e-13, 60)
    loss = 0.5 * ((u - ut) ** 2).sum()
    loss.backward()

    def L(ff, kk):
        uu = MGSolveFn.apply(ff, kk, F, 1e-13, 60)
        return float(0.5 * ((uu - ut) ** 2).sum())

    rng = np.random.default_rng(84)
    df = torch.from_numpy(rng.normal(size=f.shape)).to(dev)
    dk = torch.from_numpy(rng.normal(size=k.shape)).to(dev) * k
    # L is quadratic in f, so step 1e-6 is exact up to rounding; in k the loss difference at step 1e-6 is below the
    # FP64 noise of L itself, so the k direction uses step 1e-4 (truncation error ~1e-8 relative)
    eps, eps_k = 1e-6, 1e-4
    with torch.no_grad():
        fd_f = (L(f + eps * df, k) - L(f - eps * df, k)) / (2 * eps)
        fd_k = (L(f, k + eps_k * dk) - L(f, k - eps_k * dk)) / (2 * eps_k)
    an_f = float((fr.grad * df).sum())
    an_k = float((kr.grad * dk).sum())
    assert abs(fd_f - an_f) <= 1e-6 * abs(an_f)
    assert abs(fd_k - an_k) <= 1e-5 * abs(an_k)
