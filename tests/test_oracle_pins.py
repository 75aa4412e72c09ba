"""Pins of the CPU oracle against facts fixed by the paper and by mathematics, not by the oracle itself.

(a) 7-point exactness on polynomials; (b) O(h^2) convergence (kappa -> 0.25, Sec. 5 Eq. 3); (c) symmetry on
uniform forests; (d) a uniformly refined forest reproduces the exact single-grid solve (DST-II); (e) flux
conservation of the conservative interface variant; (f) dense direct solve on tiny forests; plus C2F
triquadratic exactness in all nine remap cases (Sec. 3.3.2), F2C multilinear exactness (Sec. 3.3.1), transfer
operators on linear functions, the transposed operator (dot-product test), the adjoint gradients against
finite differences of dense solves, harmonic-mean faces exact through a material jump, and constant k reducing
to the -Laplace cycle.
"""
import math

import numpy as np
import pytest
import scipy.fft

import synthetic as syn
from oracle.octree_mg import OracleMG, face_view, residual_from_stencil
from tests.helpers import (padded_centres, one_refined_root, poly3, neg_laplace_poly3, vw_norm, leaf_h)


def _fill_exact(mg, level, p):
    L = mg.levels[level]
    U = L.zeros()
    for b, key in enumerate(L.keys):
        U[b] = p(*padded_centres(L.R, L.n, key))
    return U


# ---------------------------------------------------------------- interpolation at refinement interfaces


@pytest.mark.parametrize("n", [4, 8])
def test_c2f_reproduces_triquadratic_all_nine_cases(n):
    R = 2
    keys = one_refined_root(R)
    mg = OracleMG(R, n, keys, operator_only=True)
    L = mg.levels[0]
    rng = np.random.default_rng(1)
    p = poly3(rng.normal(size=(3, 3, 3)))
    Ue = _fill_exact(mg, 0, p)
    U = Ue.copy()
    mg.exchange(0, U)
    cases = set()
    checked = 0
    for b in range(L.nb):
        for f in range(6):
            fc = L.faces[b][f]
            if fc[0] not in ("c2f", "same"):
                continue
            got = face_view(U[b], f // 2, f % 2)[0, 1:-1, 1:-1]
            want = face_view(Ue[b], f // 2, f % 2)[0, 1:-1, 1:-1]
            np.testing.assert_allclose(got, want, rtol=0, atol=1e-12 * np.abs(Ue).max())
            if fc[0] == "c2f":
                checked += 1
                for yf in range(n):
                    for zf in range(n):
                        yc, zc = fc[2][0] * n // 2 + yf // 2, fc[2][1] * n // 2 + zf // 2
                        cy = 1 if yc == 0 else (2 if yc == n - 1 else 0)
                        cz = 1 if zc == 0 else (2 if zc == n - 1 else 0)
                        cases.add((cy, cz))
    assert checked == 12  # 3 fine-block faces x 4 coarse neighbours... each of 3 coarse faces holds 4 segments
    assert cases == {(a, b) for a in range(3) for b in range(3)}


def test_c2f_is_not_exact_for_cubics():
    """Control: the scheme is quadratic, so a cubic in the normal direction is not reproduced."""
    R, n = 2, 8
    mg = OracleMG(R, n, one_refined_root(R), operator_only=True)
    coef = np.zeros((4, 1, 1))
    coef[3, 0, 0] = 1.0
    Ue = _fill_exact(mg, 0, poly3(coef))
    U = Ue.copy()
    mg.exchange(0, U)
    L = mg.levels[0]
    err = 0.0
    for b in range(L.nb):
        for f in (0, 1):
            if L.faces[b][f][0] == "c2f":
                err = max(err, np.abs(face_view(U[b], 0, f)[0] - face_view(Ue[b], 0, f)[0]).max())
    assert err > 1e-6


def test_f2c_mean_exact_for_multilinear():
    R, n = 2, 8
    mg = OracleMG(R, n, one_refined_root(R), variant="P", operator_only=True)
    L = mg.levels[0]
    rng = np.random.default_rng(2)
    p = poly3(rng.normal(size=(2, 2, 2)))
    Ue = _fill_exact(mg, 0, p)
    U = Ue.copy()
    mg.exchange(0, U)
    hits = 0
    for b in range(L.nb):
        for f in range(6):
            if L.faces[b][f][0] == "f2c":
                got = face_view(U[b], f // 2, f % 2)[0, 1:-1, 1:-1]
                want = face_view(Ue[b], f // 2, f % 2)[0, 1:-1, 1:-1]
                np.testing.assert_allclose(got, want, rtol=0, atol=1e-13 * np.abs(Ue).max())
                hits += 1
    assert hits == 3


# ---------------------------------------------------------------- (a) stencil exactness


@pytest.mark.parametrize("forest", ["uniform", "refined"])
def test_a_operator_exact_on_triquadratics(forest):
    R, n = 2, 8
    keys = syn.uniform_leaves(R) if forest == "uniform" else one_refined_root(R)
    mg = OracleMG(R, n, keys, operator_only=True)
    rng = np.random.default_rng(3)
    coef = rng.normal(size=(3, 3, 3))
    U = _fill_exact(mg, 0, poly3(coef))
    got = mg.apply_padded(0, U)
    want = np.stack([neg_laplace_poly3(coef)(*[c[1:-1, 1:-1, 1:-1] for c in padded_centres(R, n, key)])
                     for key in keys])
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-9 * np.abs(want).max())


# ---------------------------------------------------------------- (b) second-order convergence


def _manufactured_error(R, n, keys, variant="C"):
    mg = OracleMG(R, n, keys, variant=variant)
    f = syn.sin_product_rhs(R, n, keys).numpy()
    ue = syn.sin_product(R, n, keys).numpy()
    u, hist = mg.solve(f, rtol=1e-12, max_cycles=40)
    assert hist[-1] <= 1e-12
    return vw_norm(leaf_h(R, n, keys), u - ue)


def test_b_kappa_uniform():
    R = 2
    keys = syn.uniform_leaves(R)
    e = [_manufactured_error(R, n, keys) for n in (4, 8, 16)]
    kap = [e[i + 1] / e[i] for i in range(2)]
    assert 0.23 < kap[1] < 0.27, kap


def test_b_kappa_refined():
    R, _, keys = syn.workload_forest("sphere_2x4")
    e = [_manufactured_error(R, n, keys, "C") for n in (4, 8, 16)]
    kap = [e[i + 1] / e[i] for i in range(2)]
    assert 0.2 < kap[1] < 0.3, kap


def _golden_table():
    import os
    rows = {}
    with open(os.path.join(os.path.dirname(__file__), "golden", "paper_table_err_analysis.txt")) as fh:
        for line in fh:
            line = line.split("#")[0].split()
            if line:
                rows[int(line[0])] = [float(v) for v in line[1:]]
    return rows


def test_b_paper_error_table_second_order():
    """The paper's own accuracy problem with its ghost-only interface scheme (variant P), block sizes 16 and 32.

    Loose pin: the paper leaves the Dirichlet discretisation and norm unstated; with the reflection ghost
    2 g - u_i and the volume-weighted L2 norm the errors land within 12 % of the printed values and kappa near
    0.25, while a wrong interpolation order would give kappa near 0.5 or 1 (the table's other columns).
    """
    table = _golden_table()
    R, _, keys = syn.workload_forest("sphere_2x4")
    g = lambda x, y, z: np.sin(np.pi * x) * np.sin(np.pi * y) * np.sinh(np.sqrt(2) * np.pi * z)  # noqa: E731
    errs = {}
    for n in (16, 32):
        mg = OracleMG(R, n, keys, variant="P", bc=g)
        u, hist = mg.solve(np.zeros((len(keys), n ** 3)), rtol=1e-12, max_cycles=40)
        c = syn.cell_centres(R, n, keys).numpy().reshape(len(keys), -1, 3)
        errs[n] = vw_norm(leaf_h(R, n, keys), u - g(c[..., 0], c[..., 1], c[..., 2]))
        assert abs(errs[n] / table[n][2] - 1.0) < 0.12, (n, errs[n], table[n][2])
    assert 0.23 < errs[32] / errs[16] < 0.26


def test_b_kappa_variable_coefficient():
    """k = 1 + 1/2 sin(2 pi x) sin(2 pi y) sin(2 pi z), u = sin pi x sin pi y sin pi z, f = -div(k grad u)."""
    R, _, keys = syn.workload_forest("sphere_2x4")
    errs = []
    for n in (4, 8, 16):
        c = syn.cell_centres(R, n, keys).numpy().reshape(len(keys), -1, 3)
        x, y, z = c[..., 0], c[..., 1], c[..., 2]
        pi = math.pi
        k = 1 + 0.5 * np.sin(2 * pi * x) * np.sin(2 * pi * y) * np.sin(2 * pi * z)
        u = np.sin(pi * x) * np.sin(pi * y) * np.sin(pi * z)
        kx = pi * np.cos(2 * pi * x) * np.sin(2 * pi * y) * np.sin(2 * pi * z)
        ky = pi * np.sin(2 * pi * x) * np.cos(2 * pi * y) * np.sin(2 * pi * z)
        kz = pi * np.sin(2 * pi * x) * np.sin(2 * pi * y) * np.cos(2 * pi * z)
        ux = pi * np.cos(pi * x) * np.sin(pi * y) * np.sin(pi * z)
        uy = pi * np.sin(pi * x) * np.cos(pi * y) * np.sin(pi * z)
        uz = pi * np.sin(pi * x) * np.sin(pi * y) * np.cos(pi * z)
        f = 3 * pi ** 2 * k * u - (kx * ux + ky * uy + kz * uz)
        mg = OracleMG(R, n, keys, k_user=k)
        us, hist = mg.solve(f, rtol=1e-12, max_cycles=60)
        assert hist[-1] <= 1e-12
        errs.append(vw_norm(leaf_h(R, n, keys), us - u))
    kap = errs[2] / errs[1]
    assert 0.2 < kap < 0.3, errs


def _layered(axis, k1, k2):
    """k = k1 below the plane coord[axis] = 1/2, k2 above it; phi continuous, piecewise linear in coord[axis] with
    the same flux k phi' = 1 on both sides: the exact solution of -div(k grad u) = 0 through a material jump."""
    def phi(x, y, z):
        t = (x, y, z)[axis]
        return np.where(t <= 0.5, t / k1, 0.5 / k1 + (t - 0.5) / k2)
    def kf(x, y, z):
        return np.where((x, y, z)[axis] < 0.5, k1, k2)
    return phi, kf


@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("k1,k2", [(1.0, 10.0), (3.0, 0.25)])
def test_a_harmonic_faces_exact_through_a_material_jump(axis, k1, k2, monkeypatch):
    """Two-point flux with harmonic-mean faces is exact for a piecewise-linear, flux-continuous u when the jump
    lies on a cell face: A u = 0 in every cell, with the Dirichlet data u itself.  An arithmetic face mean fails."""
    import oracle.octree_mg as om
    R, n = 2, 8
    keys = syn.uniform_leaves(R)
    c = syn.cell_centres(R, n, keys).numpy().reshape(len(keys), -1, 3)
    phi, kf = _layered(axis, k1, k2)
    u = phi(c[..., 0], c[..., 1], c[..., 2])
    k = kf(c[..., 0], c[..., 1], c[..., 2])
    scale = 1.0 / (0.5 / n)  # |T (u_i - u_j)| / h^2 = flux / h
    Au = OracleMG(R, n, keys, k_user=k, operator_only=True, bc=phi).apply_A(u)
    assert np.abs(Au).max() <= 1e-12 * scale
    monkeypatch.setattr(om, "harmonic", lambda a, b: 0.5 * (a + b))
    Au_arith = OracleMG(R, n, keys, k_user=k, operator_only=True, bc=phi).apply_A(u)
    assert np.abs(Au_arith).max() > 0.1 * scale


@pytest.mark.parametrize("variant", ["C", "P"])
def test_constant_k_reduces_to_the_laplace_cycle(variant):
    """k = c everywhere: every level's operator is c times the -Laplace one (face means, coarse averages and ghost
    k all give c), and red-black Gauss-Seidel, the transfers and the dense coarsest solve commute with that
    scaling, so V-cycles on (A_k, c f) give the -Laplace V-cycles' iterates on (A, f)."""
    R, n, keys = 2, 8, one_refined_root()
    c = 2.5
    rng = np.random.default_rng(8)
    f = rng.uniform(-1.0, 1.0, size=(len(keys), n ** 3))
    mk = OracleMG(R, n, keys, k_user=np.full((len(keys), n ** 3), c), variant=variant)
    m1 = OracleMG(R, n, keys, variant=variant)
    assert len(mk.levels) == len(m1.levels) >= 3
    uk, _ = mk.solve(c * f, cycles=3)
    u1, _ = m1.solve(f, cycles=3)
    assert np.abs(uk - u1).max() <= 1e-13 * np.abs(u1).max()


# ---------------------------------------------------------------- (c) symmetry on uniform forests


@pytest.mark.parametrize("coeff", [False, True])
def test_c_symmetric_on_uniform_forest(coeff):
    R, n = 2, 8
    keys = syn.uniform_leaves(R)
    k = syn.lognormal_k_rff(R, n, keys, seed=4).numpy() if coeff else None
    mg = OracleMG(R, n, keys, k_user=k, operator_only=True)
    rng = np.random.default_rng(5)
    x = rng.normal(size=(len(keys), n ** 3))
    y = rng.normal(size=(len(keys), n ** 3))
    a, b = np.sum(x * mg.apply_A(y)), np.sum(y * mg.apply_A(x))
    assert abs(a - b) <= 1e-13 * np.linalg.norm(x) * np.linalg.norm(mg.apply_A(y))


# ---------------------------------------------------------------- (d) uniformly refined forest vs single grid


def _dst_poisson(fgrid, N):
    """Exact inverse of the cell-centred 7-point Laplacian with Dirichlet reflection on an N^3 grid, h = 1/N."""
    m = np.arange(1, N + 1)
    lam1 = (2.0 - 2.0 * np.cos(np.pi * m / N)) * N ** 2
    lam = lam1[:, None, None] + lam1[None, :, None] + lam1[None, None, :]
    return scipy.fft.idstn(scipy.fft.dstn(fgrid, type=2) / lam, type=2)


def test_d_uniformly_refined_forest_matches_single_grid():
    R, n = 2, 8
    keys = syn.uniform_leaves(R, level=1)  # 64 blocks of 8^3 = a 32^3 grid
    N = R * 2 * n
    rng = np.random.default_rng(6)
    f = rng.uniform(-1, 1, size=(len(keys), n ** 3))
    mg = OracleMG(R, n, keys)
    u, hist = mg.solve(f, rtol=1e-13, max_cycles=60)
    fg = np.zeros((N, N, N))
    for b, (_, i, j, k) in enumerate(keys):
        fg[k * n:(k + 1) * n, j * n:(j + 1) * n, i * n:(i + 1) * n] = f[b].reshape(n, n, n)
    ug = _dst_poisson(fg, N)
    ub = np.stack([ug[k * n:(k + 1) * n, j * n:(j + 1) * n, i * n:(i + 1) * n].reshape(-1) for (_, i, j, k) in keys])
    assert np.linalg.norm(u - ub) <= 1e-11 * np.linalg.norm(ub)


# ---------------------------------------------------------------- (e) conservation


def _boundary_flux(mg, u_user, k_user=None):
    """sum over domain-boundary faces of h T (u_i - ghost) with ghost = -u_i: 2 h T u_i, T = k_i (or 1)."""
    L = mg.levels[0]
    n = L.n
    U = mg.to_pad(u_user)
    K = mg.to_pad(k_user) if k_user is not None else None
    tot = 0.0
    for b in range(L.nb):
        for f in range(6):
            if L.faces[b][f][0] == "bnd":
                ui = face_view(U[b], f // 2, f % 2)[1, 1:-1, 1:-1]
                T = face_view(K[b], f // 2, f % 2)[1, 1:-1, 1:-1] if K is not None else 1.0
                tot += float(np.sum(2.0 * L.h[b] * T * ui))
    return tot


@pytest.mark.parametrize("coeff", [False, True])
def test_e_conservative_variant_telescopes(coeff):
    R, n, keys = syn.workload_forest("sphere_2x4")
    k = syn.lognormal_k_rff(R, n, keys, seed=7).numpy() if coeff else None
    rng = np.random.default_rng(8)
    u = rng.normal(size=(len(keys), n ** 3))
    h = leaf_h(R, n, keys)
    mgC = OracleMG(R, n, keys, k_user=k, variant="C", operator_only=True)
    total = float(np.sum(h[:, None] ** 3 * mgC.apply_A(u)))
    bnd = _boundary_flux(mgC, u, k)
    scale = float(np.sum(np.abs(h[:, None] ** 3 * mgC.apply_A(u))))
    assert abs(total - bnd) <= 1e-13 * scale
    mgP = OracleMG(R, n, keys, k_user=k, variant="P", operator_only=True)
    totalP = float(np.sum(h[:, None] ** 3 * mgP.apply_A(u)))
    assert abs(totalP - bnd) > 1e-6 * scale  # the paper's ghost-only scheme is not conservative


# ---------------------------------------------------------------- (f) dense direct solve on a tiny forest


def _dense(mg):
    L = mg.levels[0]
    N = L.nb * L.n ** 3
    A = np.zeros((N, N))
    for m in range(N):
        e = np.zeros(N)
        e[m] = 1.0
        A[:, m] = mg.apply_A(e.reshape(L.nb, -1)).reshape(-1)
    return A


@pytest.mark.parametrize("coeff", [False, True])
@pytest.mark.parametrize("variant", ["C", "P"])
def test_f_multigrid_matches_dense_solve(coeff, variant):
    R, n = 2, 4
    keys = one_refined_root(R)
    k = syn.lognormal_k_rff(R, n, keys, seed=9).numpy() if coeff else None
    mg = OracleMG(R, n, keys, k_user=k, variant=variant)
    assert [lv.nb for lv in mg.levels] == [15, 8]  # 8 children merged into their parent
    f = np.random.default_rng(10).uniform(-1, 1, size=(len(keys), n ** 3))
    u, hist = mg.solve(f, rtol=1e-14, max_cycles=80)
    A = _dense(mg)
    ud = np.linalg.solve(A, f.reshape(-1)).reshape(f.shape)
    assert np.linalg.norm(u - ud) <= 1e-11 * np.linalg.norm(ud)


# ---------------------------------------------------------------- transfer operators


def test_transfers_exact_on_linear_functions():
    R, _, keys = syn.workload_forest("sphere_2x4")
    mg = OracleMG(R, 8, keys)
    rng = np.random.default_rng(11)
    a = rng.normal(size=4)
    lin = lambda x, y, z: a[0] + a[1] * x + a[2] * y + a[3] * z  # noqa: E731
    kinds = set()
    for l in range(len(mg.levels) - 1):
        Lf, Lc = mg.levels[l], mg.levels[l + 1]
        kinds.update(t[0] for t in mg.transfer[l])
        Ec = _fill_exact(mg, l + 1, lin)
        Uf = Lf.zeros()
        mg._prolong_add(l, Ec, Uf)
        want = _fill_exact(mg, l, lin)[:, 1:-1, 1:-1, 1:-1]
        np.testing.assert_allclose(Uf[:, 1:-1, 1:-1, 1:-1], want, atol=1e-13)
        Xc = Lc.zeros()
        mg._restrict_into(l, _fill_exact(mg, l, lin), Xc)
        np.testing.assert_allclose(Xc[:, 1:-1, 1:-1, 1:-1], Ec[:, 1:-1, 1:-1, 1:-1], atol=1e-13)
    assert kinds == {"halve", "merge", "copy"}


def test_vcycle_convergence_factor():
    R, n, keys = syn.workload_forest("uniform_2x16")
    mg = OracleMG(R, n, keys)
    f = syn.sin_product_rhs(R, n, keys).numpy()
    _, hist = mg.solve(f, cycles=8)
    rates = [hist[i + 1] / hist[i] for i in range(len(hist) - 1)]
    assert max(rates) < 0.15, rates


# ---------------------------------------------------------------- adjoint


@pytest.mark.parametrize("variant", ["C", "P"])
@pytest.mark.parametrize("coeff", [False, True])
def test_transposed_operator_dot_product(variant, coeff):
    R, n, keys = syn.workload_forest("sphere_2x4")
    k = syn.lognormal_k_rff(R, n, keys, seed=12).numpy() if coeff else None
    mg = OracleMG(R, n, keys, k_user=k, variant=variant, operator_only=True)
    rng = np.random.default_rng(13)
    x = rng.normal(size=(len(keys), n ** 3))
    y = rng.normal(size=(len(keys), n ** 3))
    Ay = mg.apply_A(y)
    ATx = mg.apply_AT(x)
    lhs, rhs = np.sum(x * Ay), np.sum(ATx * y)
    assert abs(lhs - rhs) <= 1e-13 * np.linalg.norm(x) * np.linalg.norm(Ay)
    if variant == "C" or coeff:
        assert np.linalg.norm(ATx - mg.apply_A(x)) > 1e-6 * np.linalg.norm(ATx)  # refined: A is not symmetric


@pytest.mark.parametrize("variant", ["C", "P"])
def test_adjoint_solve_and_gradients_match_dense(variant):
    R, n = 2, 4
    keys = one_refined_root(R)
    rng = np.random.default_rng(14)
    k = syn.lognormal_k_rff(R, n, keys, seed=15).numpy()
    f = rng.uniform(-1, 1, size=(len(keys), n ** 3))
    ut = syn.sin_target(R, n, keys, seed=16).numpy()
    mg = OracleMG(R, n, keys, k_user=k, variant=variant)
    A = _dense(mg)
    u = np.linalg.solve(A, f.reshape(-1)).reshape(f.shape)
    g = u - ut
    lam = mg.adjoint_solve(g, rtol=1e-13)
    lam_d = np.linalg.solve(A.T, g.reshape(-1)).reshape(f.shape)
    assert np.linalg.norm(lam - lam_d) <= 1e-10 * np.linalg.norm(lam_d)
    grad = mg.grad_k(u, lam_d)

    def loss(kk):
        Ak = _dense(OracleMG(R, n, keys, k_user=kk, variant=variant, operator_only=True))
        uu = np.linalg.solve(Ak, f.reshape(-1))
        return 0.5 * np.sum((uu - ut.reshape(-1)) ** 2)

    # directional derivatives along random directions (relative perturbation of k), central differences
    for s in range(2):
        d = np.random.default_rng(100 + s).normal(size=k.shape) * k
        eps = 1e-6
        fd = (loss(k + eps * d) - loss(k - eps * d)) / (2 * eps)
        an = float(np.sum(grad * d))
        assert abs(fd - an) <= 1e-6 * abs(an), (fd, an)


@pytest.mark.parametrize("variant", ["C", "P"])
def test_transposed_vcycle_is_the_transpose(variant):
    """<x, M y> = <M^T x, y> for the forward V-cycle map M (zero initial guess) and its reverse sweep."""
    R, n, keys = syn.workload_forest("sphere_2x4")
    k = syn.lognormal_k_rff(R, n, keys, seed=17).numpy()
    mg = OracleMG(R, n, keys, k_user=k, variant=variant)
    L = mg.levels[0]
    rng = np.random.default_rng(18)
    x = rng.normal(size=(L.nb, n, n, n))
    y = rng.normal(size=(L.nb, n, n, n))
    U = L.zeros()
    mg.vcycle(0, U, y.copy())
    My = U[:, 1:-1, 1:-1, 1:-1]
    MTx = mg.vcycle_transposed(0, x)
    assert abs(np.sum(x * My) - np.sum(MTx * y)) <= 1e-13 * np.linalg.norm(x) * np.linalg.norm(My)


# ---------------------------------------------------------------- lower-order C2F, damped Jacobi (the paper's cycle)


@pytest.mark.parametrize("order,degree", [(0, 0), (1, 1)])
def test_lower_order_c2f_exact_for_its_degree(order, degree):
    """Order 0 (copy of the covering coarse cell) reproduces constants; order 1 (linear in the normal direction
    and along each tangential axis, the neighbour on the target's side or, at a coarse block edge, the other one)
    reproduces affine functions, in every remap case.  Control: order 1 does not reproduce a quadratic."""
    R, n = 2, 8
    mg = OracleMG(R, n, one_refined_root(R), operator_only=True, c2f_order=order)
    rng = np.random.default_rng(7)
    coef = np.zeros((2, 2, 2))
    coef[0, 0, 0] = rng.normal()
    if degree == 1:
        coef[1, 0, 0], coef[0, 1, 0], coef[0, 0, 1] = rng.normal(size=3)
    Ue = _fill_exact(mg, 0, poly3(coef))
    U = Ue.copy()
    mg.exchange(0, U)
    L = mg.levels[0]
    hits = 0
    for b in range(L.nb):
        for f in range(6):
            if L.faces[b][f][0] == "c2f":
                got = face_view(U[b], f // 2, f % 2)[0, 1:-1, 1:-1]
                want = face_view(Ue[b], f // 2, f % 2)[0, 1:-1, 1:-1]
                np.testing.assert_allclose(got, want, rtol=0, atol=1e-12 * np.abs(Ue).max())
                hits += 1
    assert hits == 12
    q = np.zeros((3, 1, 1))
    q[2, 0, 0] = 1.0
    Uq = _fill_exact(mg, 0, poly3(q))
    V = Uq.copy()
    mg.exchange(0, V)
    err = max(np.abs(face_view(V[b], 0, f)[0] - face_view(Uq[b], 0, f)[0]).max()
              for b in range(L.nb) for f in (0, 1) if L.faces[b][f][0] == "c2f")
    assert err > 1e-6


def test_paper_error_table_lower_orders_kappa():
    """Table err_analysis, constant- and first-order columns: the paper prints kappa near 1 (0.966, 0.984) and
    near 1/2 (0.493, 0.497).  The two schemes are named but not described, so the absolute errors of these
    readings differ from the printed ones (0.153 against 0.235 at 16^3 for order 0, 0.0158 against 0.0107 for
    order 1: within a factor two); the convergence orders, which the Table fixes, are pinned."""
    table = _golden_table()
    R, _, keys = syn.workload_forest("sphere_2x4")
    g = lambda x, y, z: np.sin(np.pi * x) * np.sin(np.pi * y) * np.sinh(np.sqrt(2) * np.pi * z)  # noqa: E731
    for order, lo, hi in ((0, 0.9, 1.1), (1, 0.4, 0.55)):
        errs = []
        for n in (8, 16):
            mg = OracleMG(R, n, keys, variant="P", bc=g, c2f_order=order)
            u, hist = mg.solve(np.zeros((len(keys), n ** 3)), rtol=1e-12, max_cycles=60)
            c = syn.cell_centres(R, n, keys).numpy().reshape(len(keys), -1, 3)
            errs.append(vw_norm(leaf_h(R, n, keys), u - g(c[..., 0], c[..., 1], c[..., 2])))
        assert lo < errs[1] / errs[0] < hi, (order, errs)
        assert 0.5 < errs[1] / table[16][order] < 2.0, (order, errs[1], table[16][order])


def _dense_operator(mg):
    L = mg.levels[0]
    N = L.nb * L.n ** 3
    A = np.zeros((N, N))
    for m in range(N):
        x = np.zeros(N)
        x[m] = 1.0
        A[:, m] = mg.apply_A(x.reshape(L.nb, -1)).reshape(-1)
    return A


def test_damped_jacobi_sweep_is_the_textbook_update():
    """One sweep of the paper's smoother with ghosts frozen at the exchanged values is u + w (h^2/6) (f - A u) for
    constant k (6 = the 7-point stencil's coefficient sum), on a refined forest, with A assembled densely."""
    R, n = 2, 4
    keys = one_refined_root(R)
    mg = OracleMG(R, n, keys, smoother="jacobi", omega=0.8)
    A = _dense_operator(OracleMG(R, n, keys, operator_only=True))
    rng = np.random.default_rng(8)
    L = mg.levels[0]
    u = rng.normal(size=(L.nb, n ** 3))
    f = rng.normal(size=(L.nb, n ** 3))
    U = mg.to_pad(u)
    F = mg.to_pad(f)[:, 1:-1, 1:-1, 1:-1].copy()
    mg.jacobi_sweep(0, U, F)
    h2 = np.repeat(L.h ** 2, n ** 3)
    want = u.reshape(-1) + 0.8 * h2 / 6.0 * (f.reshape(-1) - A @ u.reshape(-1))
    np.testing.assert_allclose(mg.from_pad(U).reshape(-1), want, rtol=1e-12, atol=1e-12)


def test_jacobi_coarsest_solve_converges_to_the_dense_solve():
    R, n, keys = 2, 8, syn.workload_forest("uniform_2x8")[2]
    dense = OracleMG(R, n, keys)
    jac = OracleMG(R, n, keys, coarse_iters=4000)
    rng = np.random.default_rng(9)
    Lc = dense.levels[-1]
    F = rng.normal(size=(Lc.nb, Lc.n, Lc.n, Lc.n))
    want = dense.coarse_solve(F)[:, 1:-1, 1:-1, 1:-1]
    got = jac.coarse_solve(F)[:, 1:-1, 1:-1, 1:-1]
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-9 * np.abs(want).max())


def test_paper_cycle_converges():
    """V(3,3) with damped Jacobi (w = 0.8) and 256 coarsest Jacobi sweeps, the paper's solver (Sec. 5), on the
    refined Table geometry: the residual falls by more than 8 orders in 30 cycles."""
    R, _, keys = syn.workload_forest("sphere_2x4")
    n = 8
    mg = OracleMG(R, n, keys, variant="P", nu1=3, nu2=3, smoother="jacobi", omega=0.8, coarse_iters=256)
    f = np.random.default_rng(10).normal(size=(len(keys), n ** 3))
    u, hist = mg.solve(f, cycles=30)
    assert hist[-1] < 1e-8, hist[-5:]


# ---------------------------------------------------------------- red-black Gauss-Seidel, ghost k, FP32 cycles


def _global_colour(R, n, keys, c):
    """Cells of colour c by the parity of their global index on their own refinement level (red = even), computed
    from the leaf coordinates alone."""
    out = []
    t = np.arange(n)
    z, y, x = np.meshgrid(t, t, t, indexing="ij")
    for (lev, i, j, k) in keys:
        out.append((((i * n + x) + (j * n + y) + (k * n + z)) % 2 == c).reshape(-1))
    return np.concatenate(out)


def _textbook_rbgs(A, D, colours, u, f):
    """One red-black Gauss-Seidel iteration in matrix form: every cell of one colour at once takes
    u_i + (f - A u)_i / D_i (D the stencil's diagonal sum_f T_f / h^2, ghosts as functions of the current u),
    red first, then black from the updated u."""
    for m in colours:
        u = u + np.where(m, (f - A @ u) / D, 0.0)
    return u


@pytest.mark.parametrize("variant", ["C", "P"])
def test_rbgs_iteration_is_the_textbook_update_refined(variant):
    """OracleMG.smooth (two half-sweeps, an exchange before each) against the red-black update written with the
    dense composite operator, constant k (D = 6 / h^2), on a forest with coarse-fine faces: a wrong colour order,
    a colour defined by local instead of global parity, a black sweep reading the ghosts exchanged before the red
    one, or a dropped h^2 f term fails it."""
    R, n = 2, 4
    keys = one_refined_root(R)
    mg = OracleMG(R, n, keys, variant=variant)
    A = _dense_operator(OracleMG(R, n, keys, variant=variant, operator_only=True))
    rng = np.random.default_rng(81)
    u = rng.normal(size=(len(keys), n ** 3))
    f = rng.normal(size=(len(keys), n ** 3))
    D = np.repeat(6.0 / leaf_h(R, n, keys) ** 2, n ** 3)
    red, black = _global_colour(R, n, keys, 0), _global_colour(R, n, keys, 1)
    want = _textbook_rbgs(A, D, (red, black), u.reshape(-1), f.reshape(-1))
    U = mg.to_pad(u)
    F = mg.to_pad(f)[:, 1:-1, 1:-1, 1:-1].copy()
    mg.smooth(0, U, F, 1)
    np.testing.assert_allclose(mg.from_pad(U).reshape(-1), want, rtol=0, atol=1e-12 * np.abs(want).max())


def test_rbgs_iteration_is_the_textbook_update_variable_k():
    """The same with a random k on a uniform forest; D_i = sum_f T_f / h^2 with T_f the harmonic mean of the two
    cells' k (the cell's own k on a domain face) is computed here on the global grid, independently of the
    oracle's ghost-k exchange and face-coefficient cache."""
    R, n = 2, 4
    keys = syn.uniform_leaves(R)
    N = R * n
    rng = np.random.default_rng(82)
    Kg = np.exp(rng.normal(size=(N, N, N)))  # [z, y, x] on the global grid
    k_user = np.stack([Kg[c * n:(c + 1) * n, b * n:(b + 1) * n, a * n:(a + 1) * n].reshape(-1)
                       for (_, a, b, c) in keys])
    mg = OracleMG(R, n, keys, k_user=k_user)
    A = _dense_operator(OracleMG(R, n, keys, k_user=k_user, operator_only=True))
    Tsum = np.zeros_like(Kg)
    for ax in range(3):
        for sh in (-1, 1):
            nb = np.roll(Kg, sh, axis=ax)
            edge = [slice(None)] * 3
            edge[ax] = 0 if sh == 1 else N - 1  # the rolled-in value came from the opposite face
            nb[tuple(edge)] = Kg[tuple(edge)]
            Tsum += 2.0 * Kg * nb / (Kg + nb)
    h = 1.0 / N
    D = np.stack([Tsum[c * n:(c + 1) * n, b * n:(b + 1) * n, a * n:(a + 1) * n].reshape(-1)
                  for (_, a, b, c) in keys]).reshape(-1) / h ** 2
    u = rng.normal(size=(len(keys), n ** 3))
    f = rng.normal(size=(len(keys), n ** 3))
    red, black = _global_colour(R, n, keys, 0), _global_colour(R, n, keys, 1)
    want = _textbook_rbgs(A, D, (red, black), u.reshape(-1), f.reshape(-1))
    U = mg.to_pad(u)
    F = mg.to_pad(f)[:, 1:-1, 1:-1, 1:-1].copy()
    mg.smooth(0, U, F, 1)
    np.testing.assert_allclose(mg.from_pad(U).reshape(-1), want, rtol=0, atol=1e-12 * np.abs(want).max())


@pytest.mark.parametrize("n", [4, 8])
def test_ghost_k_samples_a_field_constant_on_coarse_cells(n):
    """k constant on the cells of the coarse blocks' grid (edge 1 / (R n)) with independent random values, so it
    jumps across every refinement interface: every face ghost k inside the domain must equal the field at the
    ghost's centre (the fine ghost injects the coarse cell it lies in; the coarse ghost averages 8 fine cells of
    one coarse cell), and a domain-face ghost equals its cell's k.  A ghost taking its own cell's k, the wrong
    coarse cell or the wrong fine layers fails it."""
    R = 2
    keys = one_refined_root(R)
    M = R * n
    V = np.exp(np.random.default_rng(83).normal(size=(M, M, M)))  # [ix, iy, iz] of the coarse cells
    field = lambda x, y, z: V[np.floor(x * M).astype(int), np.floor(y * M).astype(int),  # noqa: E731
                              np.floor(z * M).astype(int)]
    c = syn.cell_centres(R, n, keys).numpy()
    k_user = field(c[..., 0], c[..., 1], c[..., 2]).reshape(len(keys), -1)
    mg = OracleMG(R, n, keys, k_user=k_user, operator_only=True)
    L = mg.levels[0]
    checked = {"inside": 0, "interface": 0, "boundary": 0}
    for b, key in enumerate(L.keys):
        x, y, z = padded_centres(R, n, key)
        for f in range(6):
            axis, side = f // 2, f % 2
            G = face_view(L.kpad[b], axis, side)[0, 1:-1, 1:-1]
            I = face_view(L.kpad[b], axis, side)[1, 1:-1, 1:-1]
            X = [face_view(a, axis, side)[0, 1:-1, 1:-1] for a in (x, y, z)]
            if L.faces[b][f][0] == "bnd":
                np.testing.assert_array_equal(G, I)
                checked["boundary"] += 1
                continue
            np.testing.assert_allclose(G, field(*X), rtol=1e-14, atol=0)
            checked["inside"] += 1
            checked["interface"] += L.faces[b][f][0] in ("c2f", "f2c")
    assert checked["interface"] >= 6 and checked["boundary"] > 0


def test_fp32_copy_computes_in_fp32():
    """with_dtype(np.float32): fields and face coefficients are FP32, and one V-cycle lands within FP32 rounding
    of the FP64 cycle (relative L2 between 1e-9 and 1e-5: far above FP64 rounding, far below any wrong step)."""
    from oracle.octree_mg import OracleMG as O
    R, n, keys = syn.workload_forest("sphere_2x4")
    k = syn.lognormal_k_rff(R, n, keys, seed=84).numpy()
    f = np.random.default_rng(85).normal(size=(len(keys), n ** 3))
    mg = O(R, n, keys, k_user=k)
    m32 = mg.with_dtype(np.float32)
    assert m32.levels[0].zeros().dtype == np.float32 and m32.levels[1].T[0].dtype == np.float32
    assert mg.levels[0].zeros().dtype == np.float64 and mg.levels[1].T[0].dtype == np.float64
    u64, _ = mg.solve(f, cycles=1)
    E = m32.levels[0].zeros()
    m32.vcycle(0, E, m32.to_pad(f)[:, 1:-1, 1:-1, 1:-1].astype(np.float32))
    assert E.dtype == np.float32
    rel = np.linalg.norm(m32.from_pad(E) - u64) / np.linalg.norm(u64)
    assert 1e-9 < rel < 1e-5, rel


@pytest.mark.parametrize("inner", [1, 3])
def test_mixed_solve_with_an_fp64_copy_is_plain_vcycles(inner):
    """Defect correction is exact algebra: with an FP64 copy as the inner solver, s steps of `inner` cycles give
    the iterate of s * inner FP64 V-cycles (the V-cycle is affine, u <- u + M (f - A u), and the power-of-two
    residual scale is exact), on a refined variable-k forest."""
    from oracle.octree_mg import mixed_solve
    R, n, keys = syn.workload_forest("sphere_2x4")
    k = syn.lognormal_k_rff(R, n, keys, seed=86).numpy()
    f = np.random.default_rng(87).normal(size=(len(keys), n ** 3))
    mg = OracleMG(R, n, keys, k_user=k)
    u_mix, _ = mixed_solve(mg, f, steps=2, inner=inner, mg32=mg.with_dtype(np.float64))
    u_ref, _ = mg.solve(f, cycles=2 * inner)
    assert np.linalg.norm(u_mix - u_ref) <= 1e-13 * np.linalg.norm(u_ref)


def test_mixed_solve_reaches_fp64_accuracy():
    """FP32 cycles inside FP64 defect correction reach a 1e-12 relative residual and the FP64 solution (dense
    solve of the composite operator) to 1e-10, although each FP32 cycle only resolves ~7 digits."""
    from oracle.octree_mg import mixed_solve
    R, n = 2, 4
    keys = one_refined_root(R)
    k = syn.lognormal_k_rff(R, n, keys, seed=88).numpy()
    f = np.random.default_rng(89).normal(size=(len(keys), n ** 3))
    mg = OracleMG(R, n, keys, k_user=k)
    u, hist = mixed_solve(mg, f, steps=8, inner=2)
    assert hist[-1] < 1e-12, hist
    A = _dense_operator(OracleMG(R, n, keys, k_user=k, operator_only=True))
    x = np.linalg.solve(A, f.reshape(-1))
    assert np.linalg.norm(u.reshape(-1) - x) <= 1e-10 * np.linalg.norm(x)


# ---------------------------------------------------------------- face-averaged coarse coefficients


def _level_operator(mg, l):
    """Dense operator of multigrid level l (its exchange with homogeneous data, then the 7-point rows)."""
    L = mg.levels[l]
    N = L.nb * L.n ** 3
    A = np.zeros((N, N))
    for m in range(N):
        X = np.zeros(N)
        X[m] = 1.0
        U = L.zeros()
        U[:, 1:-1, 1:-1, 1:-1] = X.reshape(L.nb, L.n, L.n, L.n)
        mg.exchange(l, U)
        A[:, m] = mg.apply_padded(l, U).reshape(-1)
    assert np.abs(A).max() > 0.0
    return A


def test_face_averaged_coarse_operator_is_symmetric():
    """On a uniform forest every level's operator with face-averaged coefficients is symmetric: the coarse cells on
    both sides of a coarse face must receive the same averaged value, so taking the finer cells of the wrong side
    (or the wrong pair of faces) for one of them makes A_c != A_c^T.  Checked on levels 1 and 2 (halving), random
    log-normal k."""
    R, n = 2, 8
    keys = syn.uniform_leaves(R)
    k = syn.lognormal_k_rff(R, n, keys, seed=91).numpy()
    mg = OracleMG(R, n, keys, k_user=k, coarse_coef="faces", max_coarse=64)
    for l in (1, 2):
        A = _level_operator(mg, l)
        assert np.abs(A - A.T).max() <= 1e-12 * np.abs(A).max(), l
    mg_k = OracleMG(R, n, keys, k_user=k, coarse_coef="k", max_coarse=64)
    assert np.abs(_level_operator(mg_k, 1) - _level_operator(mg, 1)).max() > 1e-3  # a different coarse operator


def test_face_averaged_merged_blocks_hold_one_coefficient_per_face():
    """On the refined sphere forest (8^3 blocks, interfaces on the finest levels, then a level of carried-over blocks
    and merged octets, then merged roots) every level's face coefficients have one value per face inside a block:
    the upper face of cell i equals the lower face of cell i + 1 along every axis, although the two children of a
    merged octet bring different values of their shared face where it was an interface or lay between a carried-over
    and a merged block.  On each merged block's mid-plane the two sides together keep a quarter of the sum of all the
    finer values on that face, from both children (the mean of the two sides' 2 x 2 averages: an average of one side
    only, or a missing 1/2, changes the sum).  The rediscretised coarse coefficients (coarse_coef='k') stay single
    valued too."""
    R, n, keys = syn.workload_forest("sphere_2x8")
    k = syn.lognormal_k_rff(R, n, keys, seed=97).numpy()
    mg = OracleMG(R, n, keys, k_user=k, coarse_coef="faces", operator_only=False, max_coarse=512)
    assert [tr[0] for tr in mg.transfer[-1]].count("merge") == len(mg.transfer[-1])
    merged_with_jump = 0
    for l, L in enumerate(mg.levels):
        for axis in range(3):
            a = 3 - axis  # numpy axis of the face normal in [b, z, y, x]
            up = np.take(L.T[2 * axis + 1], range(0, L.n - 1), axis=a)
            lo = np.take(L.T[2 * axis], range(1, L.n), axis=a)
            assert np.array_equal(up, lo), (l, axis)
        if l == 0:
            continue
        Lf = mg.levels[l - 1]
        h = L.n // 2
        for B, tr in enumerate(mg.transfer[l - 1]):
            if tr[0] != "merge":
                continue
            for axis in range(3):
                a = 2 - axis  # axis of the face normal in one block's [z, y, x]
                want = 0.0
                jump = 0.0
                for o, c in enumerate(tr[1]):
                    if (o >> axis) & 1:  # upper child: its lower face on its first layer
                        v = np.take(Lf.T[2 * axis][c], 0, axis=a)
                    else:  # lower child: its upper face on its last layer
                        v = np.take(Lf.T[2 * axis + 1][c], Lf.n - 1, axis=a)
                    want += v.sum()
                    jump += v.sum() * (1 if (o >> axis) & 1 else -1)
                got = np.take(L.T[2 * axis + 1][B], h - 1, axis=a).sum() + np.take(L.T[2 * axis][B], h, axis=a).sum()
                np.testing.assert_allclose(got, 0.25 * want, rtol=1e-13)
                merged_with_jump += abs(jump) > 1e-6 * want
    assert merged_with_jump > 0  # some merged faces really were two-valued on the finer level
    mg_k = OracleMG(R, n, keys, k_user=k, coarse_coef="k", operator_only=False, max_coarse=512)
    for L in mg_k.levels:
        for axis in range(3):
            up = np.take(L.T[2 * axis + 1], range(0, L.n - 1), axis=3 - axis)
            lo = np.take(L.T[2 * axis], range(1, L.n), axis=3 - axis)
            assert np.array_equal(up, lo)


def test_face_averaged_coefficients_obey_the_parallel_conductor_law():
    """k constant on layers y = const (one value per fine row): an x-face of a coarse cell is covered by fine x-faces
    of the two fine layers it contains, which conduct in parallel, so its coefficient is the arithmetic mean of the
    two layers' k; the same holds in z.  (Across the layers the coarse face keeps the finer face's harmonic mean.)"""
    R, n = 2, 8
    keys = syn.uniform_leaves(R)
    M = R * n
    ky = np.exp(np.random.default_rng(92).normal(size=M))
    c = syn.cell_centres(R, n, keys).numpy()
    k = ky[np.floor(c[..., 1] * M).astype(int)].reshape(len(keys), -1)
    mg = OracleMG(R, n, keys, k_user=k, coarse_coef="faces", operator_only=False, max_coarse=64)
    L1 = mg.levels[1]
    for b, (lev, i, j, kk) in enumerate(L1.keys):
        for Y in range(L1.n):
            yg = j * n + 2 * Y  # the two fine layers of coarse row Y
            want = 0.5 * (ky[yg] + ky[yg + 1])
            for q in (0, 1, 4, 5):  # x- and x+, z- and z+ faces
                np.testing.assert_allclose(L1.T[q][b][:, Y, :], want, rtol=1e-13)


def test_face_averaged_coarse_coefficients_converge_faster_and_to_the_same_solution():
    """With rough log-normal k the face-averaged coarse operator contracts much faster than the rediscretised one
    (2^3 roots of 16^3: 11 cycles to 1e-10 against 13; the gap grows with the block size), and on a refined forest
    with octet merging
    the solution is the dense solve of the finest operator (the coarse operator changes the cycle, not the
    solution)."""
    R, n = 2, 16
    keys = syn.uniform_leaves(R)
    k = syn.lognormal_k_rff(R, n, keys, seed=93).numpy()
    f = np.random.default_rng(94).normal(size=(len(keys), n ** 3))
    _, hk = OracleMG(R, n, keys, k_user=k, coarse_coef="k").solve(f, rtol=1e-10, max_cycles=40)
    _, hf = OracleMG(R, n, keys, k_user=k, coarse_coef="faces").solve(f, rtol=1e-10, max_cycles=40)
    assert len(hf) <= 11 and len(hk) >= len(hf) + 2, (len(hk), len(hf))
    R, n = 2, 4
    keys = one_refined_root(R)
    k = syn.lognormal_k_rff(R, n, keys, seed=95).numpy()
    f = np.random.default_rng(96).normal(size=(len(keys), n ** 3))
    for variant in ("C", "P"):
        mg = OracleMG(R, n, keys, k_user=k, variant=variant, coarse_coef="faces", max_coarse=64)
        assert any(tr[0] == "merge" for tr in mg.transfer[-1]) or len(mg.levels) > 1
        u, hist = mg.solve(f, rtol=1e-13, max_cycles=80)
        A = _dense_operator(OracleMG(R, n, keys, k_user=k, variant=variant, operator_only=True))
        x = np.linalg.solve(A, f.reshape(-1))
        assert np.linalg.norm(u.reshape(-1) - x) <= 1e-10 * np.linalg.norm(x), variant


# ---------------------------------------------------------------- edge / corner ghosts, trilinear prolongation


def _scatter_global(L, G, R, n):
    """Uniform level: the global array G [z, y, x] of (R n)^3 cells into padded blocks (interiors only)."""
    U = L.zeros()
    for b, (lev, i, j, k) in enumerate(L.keys):
        U[b, 1:-1, 1:-1, 1:-1] = G[k * n:(k + 1) * n, j * n:(j + 1) * n, i * n:(i + 1) * n]
    return U


def _diag_ghost_cells(n):
    """(z, y, x) padded indices of every edge and corner ghost cell of a block (two or three ghost coordinates)."""
    out = []
    for z in range(n + 2):
        for y in range(n + 2):
            for x in range(n + 2):
                if sum(c in (0, n + 1) for c in (x, y, z)) >= 2:
                    out.append((z, y, x))
    return out


def test_diagonal_ghosts_copy_same_level_blocks_and_are_exact_for_trilinear_data():
    """Uniform 3^3 roots of 4^3: after the face exchange and exchange_diagonal every edge and corner ghost inside the
    domain holds the global field's value there (the diagonal neighbour's cell; copying the wrong layer or the wrong
    neighbour fails).  Refined forest (one root split, ghost-only interfaces): for trilinear data every edge and
    corner ghost whose centre lies inside the domain equals the function there, for the copied ones and for those
    extrapolated where the diagonal block is coarser or finer (a wrong sign or weight fails, and so does the
    parallelogram rule g_a + g_b - u, which misses the cross terms)."""
    R, n = 3, 4
    keys = syn.uniform_leaves(R)
    mg = OracleMG(R, n, keys, operator_only=True, prolongation="trilinear")
    L = mg.levels[0]
    G = np.random.default_rng(71).normal(size=(R * n,) * 3)
    U = _scatter_global(L, G, R, n)
    mg.exchange(0, U)
    mg.exchange_diagonal(0, U)
    checked = 0
    for b, (lev, i, j, k) in enumerate(L.keys):
        for (z, y, x) in _diag_ghost_cells(n):
            gz, gy, gx = k * n + z - 1, j * n + y - 1, i * n + x - 1
            if all(0 <= c < R * n for c in (gz, gy, gx)):
                assert U[b, z, y, x] == G[gz, gy, gx], (b, z, y, x)
                checked += 1
    assert checked > 0
    R, n = 2, 4
    keys = one_refined_root(R)
    coef = np.random.default_rng(72).normal(size=(2, 2, 2))
    f = poly3(coef)
    mg = OracleMG(R, n, keys, variant="P", operator_only=True, prolongation="trilinear")
    L = mg.levels[0]
    U = L.zeros()
    for b, key in enumerate(L.keys):
        x, y, z = padded_centres(R, n, key)
        U[b, 1:-1, 1:-1, 1:-1] = f(x, y, z)[1:-1, 1:-1, 1:-1]
    mg.exchange(0, U)
    mg.exchange_diagonal(0, U)
    kinds = {"copy": 0, "extrapolated": 0}
    for b, key in enumerate(L.keys):
        lev, i, j, k = key
        x, y, z = padded_centres(R, n, key)
        ref = f(x, y, z)
        for (zz, yy, xx) in _diag_ghost_cells(n):
            c = (x[zz, yy, xx], y[zz, yy, xx], z[zz, yy, xx])
            if not all(0.0 < v < 1.0 for v in c):
                continue
            np.testing.assert_allclose(U[b, zz, yy, xx], ref[zz, yy, xx], rtol=0, atol=1e-12)
            d = [0 if q in range(1, n + 1) else (1 if q == n + 1 else -1) for q in (xx, yy, zz)]
            same = (lev, i + d[0], j + d[1], k + d[2]) in L.index
            kinds["copy" if same else "extrapolated"] += 1
    assert kinds["copy"] > 0 and kinds["extrapolated"] > 0, kinds


@pytest.mark.parametrize("R,max_coarse,transfer", [(2, 4096, "halve"), (4, 512, "merge")])
def test_trilinear_prolongation_is_exact_for_trilinear_corrections(R, max_coarse, transfer):
    """A trilinear coarse correction (ghosts from the face and diagonal exchanges) prolongates to the function's
    values at every fine cell whose coarse stencil stays inside the domain, across halving and octet-merging
    transfers; the face-neighbour linear prolongation misses the cross terms (xy, xz, yz, xyz) there."""
    n = 4 if transfer == "merge" else 8
    keys = syn.uniform_leaves(R)
    coef = np.random.default_rng(73).normal(size=(2, 2, 2))
    coef[1, 1, 0] = 1.0  # a real xy term
    f = poly3(coef)
    errs = {}
    for pr in ("trilinear", "linear"):
        mg = OracleMG(R, n, keys, max_coarse=max_coarse, prolongation=pr)
        assert any(t[0] == transfer for t in mg.transfer[0])
        Lf, Lc = mg.levels[0], mg.levels[1]
        Ec = Lc.zeros()
        for B, key in enumerate(Lc.keys):
            x, y, z = padded_centres(R, Lc.n, key)
            Ec[B, 1:-1, 1:-1, 1:-1] = f(x, y, z)[1:-1, 1:-1, 1:-1]
        mg.exchange(1, Ec)
        if pr == "trilinear":
            mg.exchange_diagonal(1, Ec)
        Uf = Lf.zeros()
        mg._prolong_add(0, Ec, Uf)
        worst = 0.0
        for b, key in enumerate(Lf.keys):
            x, y, z = padded_centres(R, n, key)
            hf = 1.0 / (R * 2 ** key[0] * n)
            x, y, z = (c[1:-1, 1:-1, 1:-1] for c in (x, y, z))  # interior cells; at least two coarse cells inside
            inner = np.ones_like(x, dtype=bool)
            for c in (x, y, z):
                inner &= (c > 4 * hf) & (c < 1 - 4 * hf)
            diff = np.abs(Uf[b, 1:-1, 1:-1, 1:-1] - f(x, y, z))[inner]
            worst = max(worst, float(diff.max()) if diff.size else 0.0)
        errs[pr] = worst
    assert errs["trilinear"] <= 1e-12, errs
    assert errs["linear"] > 1e-3, errs


@pytest.mark.parametrize("variant", ["C", "P"])
def test_trilinear_prolongation_solves_to_the_dense_solution(variant):
    """With the trilinear prolongation the cycle still solves the finest operator: on a refined forest with log-normal
    k it reaches the dense solution (the prolongation changes the cycle, not the solution)."""
    R, n = 2, 4
    keys = one_refined_root(R)
    k = syn.lognormal_k_rff(R, n, keys, seed=74).numpy()
    f = np.random.default_rng(75).normal(size=(len(keys), n ** 3))
    mg = OracleMG(R, n, keys, k_user=k, variant=variant, max_coarse=64, prolongation="trilinear")
    u, hist = mg.solve(f, rtol=1e-13, max_cycles=80)
    A = _dense_operator(OracleMG(R, n, keys, k_user=k, variant=variant, operator_only=True))
    x = np.linalg.solve(A, f.reshape(-1))
    assert np.linalg.norm(u.reshape(-1) - x) <= 1e-10 * np.linalg.norm(x)
    assert len(hist) < 60


@pytest.mark.parametrize("variant", ["C", "P"])
def test_rbgs_leaves_zero_residual_on_second_colour_away_from_boundary_and_interfaces(variant):
    """After a red-black iteration (red, then black, an exchange before each half-sweep and before the residual),
    every black cell satisfies its equation, unless one of its ghosts was rewritten after its update: a reflection
    ghost on the domain boundary (it mirrors the cell itself) or a ghost across a refinement interface (interpolated
    again from the neighbour's new values).  Checked on a refined forest with variable k, with both exceptions
    shown to be real: a swapped colour order, a black sweep on stale red ghosts or a wrong diagonal fails it."""
    R, n = 2, 8
    keys = one_refined_root(R)
    rng = np.random.default_rng(83)
    k_user = np.exp(rng.normal(size=(len(keys), n ** 3)))
    mg = OracleMG(R, n, keys, k_user=k_user, variant=variant)
    L = mg.levels[0]
    U = mg.to_pad(rng.normal(size=(len(keys), n ** 3)))
    F = rng.normal(size=(len(keys), n, n, n))
    mg.smooth(0, U, F, 1)
    r = mg.residual(0, U, F)
    scale = np.abs(r).max()
    black = L.colour_mask(1)
    t = np.arange(n)
    z, y, x = np.meshgrid(t, t, t, indexing="ij")
    on_face = [x == 0, x == n - 1, y == 0, y == n - 1, z == 0, z == n - 1]
    seen = {"bnd": 0.0, "iface": 0.0}
    for b in range(L.nb):
        changed = np.zeros((n, n, n), dtype=bool)
        for f in range(6):
            kind = L.faces[b][f][0]
            if kind == "same":
                continue
            changed |= on_face[f]
            m = black & on_face[f]
            tag = "bnd" if kind == "bnd" else "iface"
            seen[tag] = max(seen[tag], float(np.abs(r[b][m]).max()))
        quiet = black & ~changed
        assert np.abs(r[b][quiet]).max() <= 1e-12 * scale, (b, np.abs(r[b][quiet]).max(), scale)
    # the exceptions: black cells on boundary faces and on interface faces do carry a residual
    assert seen["bnd"] > 1e-3 * scale and seen["iface"] > 1e-3 * scale, (seen, scale)
    # and the first colour's residual is not zero anywhere near as often
    assert np.abs(r[:, ~black]).max() > 1e-3 * scale


# ---------------------------------------------------------------- per-cell residual (sampled checks of large solves)


def _grid_stencils(N, ufun, kfun):
    """Every cell of the uniform N^3 grid on [0, 1]^3 as a 7-point stencil (cell, x-, x+, y-, y+, z-, z+): values of
    ufun / kfun at the cell centres (a boundary neighbour gets a placeholder), the boundary flags, and g = ufun at
    each boundary face's centre."""
    h = 1.0 / N
    t = (np.arange(N) + 0.5) * h
    z, y, x = np.meshgrid(t, t, t, indexing="ij")
    pts = np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1)
    idx = np.stack(np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")[::-1], axis=-1).reshape(-1, 3)
    u7 = np.empty((len(pts), 7))
    k7 = np.empty((len(pts), 7))
    bnd = np.zeros((len(pts), 6), dtype=bool)
    g = np.zeros((len(pts), 6))
    u7[:, 0] = ufun(*pts.T)
    k7[:, 0] = kfun(*pts.T)
    for face in range(6):
        axis, side = face // 2, face % 2
        d = np.zeros(3)
        d[axis] = h if side else -h
        q = pts + d
        bnd[:, face] = idx[:, axis] == (N - 1 if side else 0)
        u7[:, 1 + face] = np.where(bnd[:, face], 0.0, ufun(*q.T))
        k7[:, 1 + face] = np.where(bnd[:, face], 0.0, kfun(*q.T))
        fc = pts + d / 2
        g[:, face] = ufun(*fc.T)
    return u7, k7, bnd, g, h, idx


def test_stencil_residual_linear_and_quadratic():
    """k = 1: a linear u with its own boundary values is reproduced exactly by the operator, reflection ghosts
    included (A u = 0 at every cell); u = x^2 + y^2 - 3 z^2 / 2 gives A u = -lap u = -1 at every interior cell.  A sign
    error in the reflection, the neighbour's k on a boundary face or a missing 1/h^2 fails one of them."""
    one = lambda x, y, z: np.ones_like(x)
    lin = lambda x, y, z: 1.0 + 2.0 * x - 3.0 * y + 0.5 * z
    u7, k7, bnd, g, h, idx = _grid_stencils(8, lin, one)
    au, r, s = residual_from_stencil(u7, k7, bnd, np.zeros(len(u7)), h, g)
    np.testing.assert_allclose(au, 0.0, atol=1e-12 * s.max())
    quad = lambda x, y, z: x ** 2 + y ** 2 - 1.5 * z ** 2
    u7, k7, bnd, g, h, idx = _grid_stencils(8, quad, one)
    au, r, s = residual_from_stencil(u7, k7, bnd, np.full(len(u7), -1.0), h, g)
    inner = ~bnd.any(axis=1)
    np.testing.assert_allclose(au[inner], -1.0, rtol=0, atol=1e-11 * s.max())
    np.testing.assert_allclose(r[inner], 0.0, rtol=0, atol=1e-11 * s.max())


def test_stencil_residual_material_jump_is_exact():
    """k jumps from 1 to 10 across the plane x = 1/2 (a cell face); u is linear on each side with continuous flux
    (k u' equal).  The harmonic face mean makes the discrete flux exact, so A u = 0 at every cell; an arithmetic face
    mean, or the neighbour's k on a boundary face, fails it."""
    k1, k2, a1 = 1.0, 10.0, 3.0
    a2 = k1 * a1 / k2
    kfun = lambda x, y, z: np.where(x < 0.5, k1, k2)
    ufun = lambda x, y, z: np.where(x < 0.5, a1 * x, a1 * 0.5 + a2 * (x - 0.5))
    u7, k7, bnd, g, h, idx = _grid_stencils(8, ufun, kfun)
    au, r, s = residual_from_stencil(u7, k7, bnd, np.zeros(len(u7)), h, g)
    np.testing.assert_allclose(au, 0.0, atol=1e-12 * s.max())


def test_stencil_residual_agrees_with_the_forest_operator():
    """Random u and k on 2^3 roots of 4^3 cells: the per-cell residual equals the forest operator's (OracleMG.apply_A)
    at every cell."""
    R, n = 2, 4
    N = R * n
    keys = syn.uniform_leaves(R)
    rng = np.random.default_rng(84)
    Ug = rng.normal(size=(N, N, N))
    Kg = np.exp(rng.normal(size=(N, N, N)))
    blocks = lambda G: np.stack([G[c * n:(c + 1) * n, b * n:(b + 1) * n, a * n:(a + 1) * n].reshape(-1)
                                 for (_, a, b, c) in keys])
    mg = OracleMG(R, n, keys, k_user=blocks(Kg))
    want = mg.apply_A(blocks(Ug))
    at = lambda G: (lambda x, y, z: G[np.minimum((z * N).astype(int), N - 1), np.minimum((y * N).astype(int), N - 1),
                                      np.minimum((x * N).astype(int), N - 1)])
    u7, k7, bnd, _, h, idx = _grid_stencils(N, at(Ug), at(Kg))
    au, _, s = residual_from_stencil(u7, k7, bnd, np.zeros(len(u7)), h, 0.0)
    got = blocks(au.reshape(N, N, N))
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-13 * s.max())


def test_batch_stencil_sampler_matches_the_forest_operator():
    """The sampler behind the full-size batch check (tests.helpers.batch_stencils) on a small batch of refined
    problems: at every sampled cell, the per-cell operator built from the sampled stencil equals the forest
    operator of that problem (OracleMG.apply_A).  So the flat offsets, the neighbour blocks across block faces and
    the boundary flags it returns are right, and cells next to refinement interfaces are left out."""
    from tests.helpers import batch_stencils
    problems = syn.batch_problems(count=6, seed=3, sizes=(4, 8), max_depth=2, box=(0.2, 0.5))
    assert any(len(keys) > 1 for _, keys in problems)
    rng = np.random.default_rng(87)
    us, ks, want = [], [], []
    for n, keys in problems:
        k = np.exp(rng.normal(size=(len(keys), n ** 3)))
        u = rng.normal(size=(len(keys), n ** 3))
        want.append(OracleMG(1, n, keys, k_user=k).apply_A(u).reshape(-1))
        us.append(u.reshape(-1))
        ks.append(k.reshape(-1))
    u, k, want = np.concatenate(us), np.concatenate(ks), np.concatenate(want)
    idx, bnd, pid, h = batch_stencils(problems, np.random.default_rng(88), per_problem=200)
    assert len(idx) > 600 and bnd.any() and len(np.unique(pid)) == len(problems)
    au, _, s = residual_from_stencil(u[idx], k[idx], bnd, np.zeros(len(idx)), h, 0.0)
    np.testing.assert_allclose(au, want[idx[:, 0]], rtol=0, atol=1e-12 * s.max())
