"""Plain, slow FP64 CPU oracle for the octree-block multigrid method of arXiv 2403.08063.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or execute this module; only the tests,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` use it.  It shares no code with the CUDA
path: its forest tables, interpolation weights, transfer operators and solver are written here from the paper.

What it computes
----------------
* Discretisation (Sec. 5, Eq. 1-2): -div(k grad u) = f on [0,1]^3, cell-centred finite volumes on a forest of
  octree blocks (Sec. 2), every block holding n^3 cells plus one ghost layer (Sec. 3.3: "half of the ghost layers").
  Point form: (A u)_i = (1/h_i^2) sum_faces T_f (u_i - u_f), u_f the neighbour or ghost value.
  T_f = 1 for constant k, else the harmonic mean 2 k_i k_g / (k_i + k_g) (variable coefficients are future work
  in Sec. 8; harmonic mean is the standard finite-volume reading).
* Ghost exchange (Sec. 3.1): same-level copy; domain boundary Dirichlet reflection ghost = 2 g - u_i (g = 0);
  coarse-to-fine (Sec. 3.3.2) quadratic Lagrange extrapolation: first along the normal through the current coarse
  cell and two cells inward, then along each orthogonal axis through {-1, 0, +1}, with any base that falls in the
  coarse block's ghost region remapped by -2o, targets at -h/4 (downwind) and +h/4 (upwind); fine-to-coarse
  (Sec. 3.3.1) mean of the 2x2x2 fine inner cells overlapping a coarse ghost cell (weight 0.125).
* Interface variants: 'P' is the paper's ghost-only scheme (coarse ghosts from the F2C mean).  'C' replaces the
  coarse cell's interface flux by the sum of the four fine sub-face fluxes (coarse ghost written so that
  T_C (u_C - G) = 1/2 sum_j T_j (g_j - u_j)), which makes the composite operator conservative.  The paper states
  no conservation property; 'C' is this project's reading, 'P' reproduces the paper.
* Multigrid (Sec. 5: block-local coarsening down to 4^3 cells per block): V(nu1, nu2) with red-black Gauss-Seidel,
  colour (x+y+z) mod 2 of the block-local cell index (blocks have even n, so this is the global parity), red
  first, an exchange before every half-sweep; residual restricted by the mean of the 8 children; prolongation
  e_f = 1/4 (e_C + e_{C+sx} + e_{C+sy} + e_{C+sz}) with s_d towards the child's side (or, optionally, the 8-point
  trilinear interpolation, which reads the coarse correction's edge and corner ghosts: copies from a same-level
  diagonal neighbour, else linear extrapolation from the neighbouring face (edge) ghosts, exact for trilinear data;
  Sec. 8 names diagonal ghosts for wider stencils as future work); coarse levels rediscretised
  with homogeneous Dirichlet data and k averaged over the 8 children; when the 4^3 level has more than
  ``max_coarse`` unknowns, complete sibling octets at the deepest level are merged into their parent (a
  coarsening step the paper does not need, since it smooths on the coarsest level); the coarsest level is solved
  by a dense LU factorisation.
* The paper's own cycle (Sec. 5), for its accuracy and benchmark experiments: damped Jacobi smoothing (omega
  = 0.8, one sweep per smoothing step, ghosts frozen at the exchanged values) and damped Jacobi sweeps as the
  coarsest solver; coarse-to-fine interpolation of order 2 (above), or the Table's lower orders: order 1 linear
  along the normal (the current coarse cell and the next one inward) and along each orthogonal axis (the
  neighbour on the fine cell's side, the other one at a coarse block edge), order 0 a copy of the covering coarse
  cell.  The paper names the lower orders without describing them; these are this project's readings.
* Stopping: volume-weighted L2 norm sqrt(sum h^3 r^2) of the residual relative to that of f (Sec. 5 says only
  "L2 residual norm"; a normalised norm is the reading that gives the printed kappa near 0.25).
* Adjoint: A^T applied matrix-free as the transposed stencil followed by the transposed ghost exchange; dL/df =
  lambda and dL/dk = -lambda^T (dA/dk) u for L = 1/2 sum (u - u_t)^2.
* Mixed precision (not in the paper, which computes in FP64): ``OracleMG.with_dtype(np.float32)`` is a copy whose
  level fields, face coefficients and cycle arithmetic are FP32 while its set-up (hierarchy, FP64 coefficient
  pyramid, LU factors of the FP64 coarsest operator) stays FP64; ``mixed_solve`` runs such FP32 V-cycles inside FP64
  defect correction, so that the error an FP32 cycle should have can be stated against the FP64 oracle.

User layout: leaf-major in the order of the leaf list, each leaf n^3 interior cells with x fastest.
"""
from __future__ import annotations

import copy
import functools
import itertools
from fractions import Fraction

import numpy as np
import scipy.linalg

# ----------------------------------------------------------------------------------------------------------
# Lagrange weights (Sec. 3.3.2: w_i(x) = prod_{j != i} (x - x_j) / (x_i - x_j))
# ----------------------------------------------------------------------------------------------------------


def lagrange_weights(nodes, x):
    """Exact Lagrange basis weights at x for the given nodes (Sec. 3.3.2 weight formula)."""
    nodes = [Fraction(v) for v in nodes]
    x = Fraction(x)
    out = []
    for i, xi in enumerate(nodes):
        w = Fraction(1)
        for j, xj in enumerate(nodes):
            if j != i:
                w *= (x - xj) / (xi - xj)
        out.append(w)
    return out


# Normal step: bases at the current coarse cell and the two cells inward (the -d_comm direction), measured in
# coarse cells inward; the fine ghost centre lies h_c/4 outward of the current coarse centre.
NORMAL_NODES = (0, 1, 2)
NORMAL_TARGET = Fraction(-1, 4)
NORMAL_W = [float(w) for w in lagrange_weights(NORMAL_NODES, NORMAL_TARGET)]


def normal_weights(order):
    """Weights of the coarse cells 0, 1, .. inward (the -d_comm direction) for the fine ghost at -1/4: the quadratic
    rule of Sec. 3.3.2 (order 2, bases 0, 1, 2) and the Table's lower orders (order 1: bases 0, 1; order 0: the
    covering coarse cell alone)."""
    return [float(w) for w in lagrange_weights(tuple(range(order + 1)), NORMAL_TARGET)]


def tangential_nodes_order(yc, n, target, order):
    """Bases along an orthogonal axis for the given interpolation order.

    Order 2: tangential_nodes.  Order 1 (the paper names the first-order scheme without describing it; reading):
    the current coarse cell and its neighbour on the target's side, or the neighbour on the other side when that
    one lies outside the coarse block's interior.  Order 0: the covering coarse cell.
    """
    if order == 2:
        return tangential_nodes(yc, n)
    if order == 0:
        return [0]
    o = -1 if target < 0 else 1
    if not (0 <= yc + o <= n - 1):
        o = -o
    return [0, o]


def tangential_nodes(yc, n):
    """Bases along an orthogonal axis for coarse cell yc of a block with n cells on that axis (Sec. 3.3.2).

    Start from {-1, 0, +1}; a neighbour o in {-1, +1} lying in the ghost region (outside 0..n-1) is remapped to
    the inner cell at -2o.
    """
    nodes = []
    for o in (-1, 0, 1):
        if o != 0 and not (0 <= yc + o <= n - 1):
            nodes.append(-2 * o)
        else:
            nodes.append(o)
    return nodes


@functools.lru_cache(maxsize=None)
def _tangential_matrix_cached(n, offset, order):
    """Read-only cached copy of tangential_matrix_uncached (Sec. 3.3.2)."""
    M = tangential_matrix_uncached(n, offset, order)
    M.setflags(write=False)
    return M


def tangential_matrix(n, offset, order=2):
    """The C2F tangential interpolation matrix of one axis (Sec. 3.3.2), cached."""
    return _tangential_matrix_cached(n, offset, order)


def tangential_matrix_uncached(n, offset, order=2):
    """(n x n) map from the coarse cells of one tangential axis to the n fine ghost cells of a segment.

    Fine index yf belongs to coarse cell yc = offset + yf // 2; even yf sits at -1/4 (downwind), odd at +1/4.
    """
    M = np.zeros((n, n))
    for yf in range(n):
        yc = offset + yf // 2
        target = Fraction(-1, 4) if yf % 2 == 0 else Fraction(1, 4)
        nodes = tangential_nodes_order(yc, n, target, order)
        for node, w in zip(nodes, lagrange_weights(nodes, target)):
            M[yf, yc + node] += float(w)
    return M


def harmonic(a, b):
    """Face coefficient between cells with k = a and k = b: the harmonic mean (this project's reading for the
    variable coefficients that Sec. 8 leaves to future work)."""
    return 2.0 * a * b / (a + b)


def residual_from_stencil(u7, k7, bnd, f, h, g=0.0):
    """r = f - A u at cells taken one by one, each from its own 7-point stencil (Sec. 5, Eq. 1-2, in the point form
    of this module's header), for cells whose six face neighbours lie on the same refinement level or on the domain
    boundary: large problems can be checked at sampled cells without building the forest.

    u7, k7: (m, 7) FP64 arrays, column 0 the cell, columns 1..6 its x-, x+, y-, y+, z-, z+ neighbours (ignored where
    ``bnd`` is set); bnd: (m, 6) bool, the face lies on the domain boundary, whose Dirichlet reflection ghost is
    2 g - u_i with the cell's own k (harmonic(k_i, k_i) = k_i), g a scalar or (m, 6) per face; f: (m,); h: cell
    width (scalar or (m,)).
    Returns (A u, r, s), s = sum_f T_f (|u_i| + |u_f|) / h^2 the size of the terms, for rounding bounds."""
    u7 = np.asarray(u7, dtype=np.float64)
    k7 = np.asarray(k7, dtype=np.float64)
    bnd = np.asarray(bnd, dtype=bool)
    uc, kc = u7[:, 0], k7[:, 0]
    h2 = np.asarray(h, dtype=np.float64) ** 2
    au = np.zeros_like(uc)
    s = np.zeros_like(uc)
    for face in range(6):
        b = bnd[:, face]
        gf = np.asarray(g, dtype=np.float64)[:, face] if np.ndim(g) == 2 else g
        uf = np.where(b, 2.0 * gf - uc, u7[:, 1 + face])
        kf = np.where(b, kc, k7[:, 1 + face])
        T = harmonic(kc, kf)
        au += T * (uc - uf)
        s += T * (np.abs(uc) + np.abs(uf))
    au = au / h2
    return au, np.asarray(f, dtype=np.float64) - au, s / h2


# ----------------------------------------------------------------------------------------------------------
# Forest geometry and neighbour tables (Sec. 2, Sec. 3.1: N_neigh = 4 finer neighbours per face in 3D)
# ----------------------------------------------------------------------------------------------------------


def face_view(a, axis, side):
    """View of a padded block array a[z, y, x] as [depth, t1, t2] for face (axis, side).

    depth 0 is the ghost layer of that face, depth 1 the first interior layer, and so on; t1 < t2 are the two
    other spatial axes in increasing order, in their original orientation.
    """
    t1, t2 = [d for d in range(3) if d != axis]
    v = np.moveaxis(a, (2 - axis, 2 - t1, 2 - t2), (0, 1, 2))
    return v[::-1] if side == 1 else v


class Level:
    """One multigrid level: a list of blocks (level, i, j, k) all holding n^3 cells."""

    dtype = np.dtype(np.float64)  # working precision of the level's fields (OracleMG.with_dtype changes it)

    def __init__(self, R, n, keys):
        """Blocks of one level of the forest (Sec. 2: octree blocks over R^3 roots), with their face neighbours."""
        self.R, self.n, self.keys = R, n, list(keys)
        self.index = {key: b for b, key in enumerate(self.keys)}
        self.nb = len(self.keys)
        self.h = np.array([1.0 / (R * 2.0 ** key[0] * n) for key in self.keys])
        self.faces = [[self._face(key, f // 2, f % 2) for f in range(6)] for key in self.keys]
        self.kpad = None
        self.T = None  # cached face coefficients (6 arrays (nb, n, n, n)) for variable k

    def blocks_per_axis(self, lev):
        """R 2^lev: blocks per axis at refinement level lev (Sec. 2)."""
        m = self.R * 2.0 ** lev
        assert m == int(m) and m >= 1, "level below the root grid"
        return int(m)

    def _face(self, key, axis, side):
        """Neighbour relation across one block face (Sec. 3.1): boundary, same level, coarser (C2F, with the
        segment of the coarse face) or finer (F2C, the four fine blocks and their segments)."""
        lev = key[0]
        idx = list(key[1:])
        m = self.blocks_per_axis(lev)
        p = idx.copy()
        p[axis] += 1 if side == 1 else -1
        if not (0 <= p[axis] < m):
            return ("bnd",)
        same = (lev, *p)
        if same in self.index:
            return ("same", self.index[same])
        t1, t2 = [d for d in range(3) if d != axis]
        parent = (lev - 1, p[0] // 2, p[1] // 2, p[2] // 2)
        if parent in self.index:
            return ("c2f", self.index[parent], (idx[t1] % 2, idx[t2] % 2))
        segs = []
        for s2 in (0, 1):
            for s1 in (0, 1):
                c = [0, 0, 0]
                c[axis] = 2 * p[axis] + (1 if side == 0 else 0)
                c[t1] = 2 * p[t1] + s1
                c[t2] = 2 * p[t2] + s2
                ck = (lev + 1, *c)
                if ck not in self.index:
                    raise ValueError(f"block {key} face {(axis, side)}: neighbourhood is not 2:1 balanced or has holes")
                segs.append((self.index[ck], s1, s2))
        return ("f2c", segs)

    def zeros(self):
        """A zero field with one ghost layer per block (Sec. 3.3: one ghost layer)."""
        n = self.n
        return np.zeros((self.nb, n + 2, n + 2, n + 2), dtype=self.dtype)

    def colour_mask(self, c):
        """Interior cells of colour c, (x + y + z) mod 2 of the block-local index (red-black ordering)."""
        n = self.n
        z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
        return ((x + y + z) % 2) == c


def check_forest(R, keys):
    """The leaves tile the unit cube: no leaf is an ancestor of another and the volumes sum to 1."""
    keyset = set(keys)
    if len(keyset) != len(keys):
        raise ValueError("duplicate leaves")
    vol = Fraction(0)
    for (l, i, j, k) in keys:
        m = R * 2 ** l
        if not (0 <= i < m and 0 <= j < m and 0 <= k < m):
            raise ValueError("leaf outside the domain")
        vol += Fraction(1, m ** 3)
        a = (l, i, j, k)
        while a[0] > 0:
            a = (a[0] - 1, a[1] // 2, a[2] // 2, a[3] // 2)
            if a in keyset:
                raise ValueError("overlapping leaves")
    if vol != 1:
        raise ValueError("leaves do not cover the domain")


# ----------------------------------------------------------------------------------------------------------
# The solver
# ----------------------------------------------------------------------------------------------------------


class OracleMG:
    """FP64 octree-block multigrid on one forest.

    R: root blocks per axis; n: cells per block edge on the finest level (power of two, >= 4);
    keys: leaf list (level, i, j, k); k_user: None for -Laplace, else (n_leaves, n^3) coefficient values.
    """

    dtype = np.dtype(np.float64)  # working precision of the cycles (with_dtype makes an FP32 copy)

    def __init__(self, R, n, keys, k_user=None, variant="C", nu1=2, nu2=2, max_coarse=512, operator_only=False,
                 bc=None, c2f_order=2, smoother="rbgs", omega=0.8, coarse_iters=None, coarse_coef="k",
                 prolongation="linear"):
        """operator_only builds the finest level alone (for applying A, A^T and dA/dk; no solver).

        bc: None for homogeneous Dirichlet data, else a vectorised g(x, y, z) giving the Dirichlet value at
        boundary face centres of the finest level (Sec. 5, Eq. 2); coarse levels always use g = 0.
        c2f_order: 2 the paper's quadratic coarse-to-fine scheme, 1 / 0 the lower orders of its Table err_analysis.
        smoother: 'rbgs' (red-black Gauss-Seidel) or 'jacobi' (damped by omega, the paper's own smoother, Sec. 5;
        one sweep per smoothing step).  coarse_iters: None for the dense direct coarsest solve, else that many damped
        Jacobi sweeps from zero on the coarsest level (the paper's coarsest solver, Sec. 5).
        coarse_coef (variable k): 'k' rediscretises every coarse level from its k, the mean of the 8 children's
        (the reading of Sec. 5's rediscretisation); 'faces' gives every coarse face the mean of the 2 x 2 finer
        face coefficients it covers (an operator-aware coarsening the paper does not discuss; far fewer cycles for
        rough k).  The finest level's coefficients are the harmonic means either way.
        prolongation: 'linear' the face-neighbour linear interpolation (each fine cell from its coarse cell and the
        three face neighbours towards it), 'trilinear' the 8-point tensor-product interpolation, which also needs the
        coarse correction's edge and corner ghosts (exchange_diagonal; Sec. 8 lists such diagonal ghosts for wider
        stencils as future work).
        """
        if n < 4 or n & (n - 1):
            raise ValueError("n must be a power of two >= 4")
        check_forest(R, list(keys))
        self.R, self.n, self.variant = R, n, variant
        self.nu1, self.nu2 = nu1, nu2
        if c2f_order not in (0, 1, 2) or smoother not in ("rbgs", "jacobi") or coarse_coef not in ("k", "faces"):
            raise ValueError("c2f_order must be 0, 1 or 2, smoother 'rbgs' or 'jacobi', coarse_coef 'k' or 'faces'")
        self.coarse_coef = coarse_coef
        if prolongation not in ("linear", "trilinear"):
            raise ValueError("prolongation must be 'linear' or 'trilinear'")
        self.prolongation = prolongation
        self.c2f_order, self.smoother, self.omega, self.coarse_iters = c2f_order, smoother, omega, coarse_iters
        self.normal_w = normal_weights(c2f_order)
        self.levels = [Level(R, n, keys)]
        self.transfer = []  # transfer[l]: per coarse block of level l+1, ('halve', b) | ('copy', b) | ('merge', [8 b])
        while self.levels[-1].n > 4 and not operator_only:
            L = self.levels[-1]
            self.levels.append(Level(R, L.n // 2, L.keys))
            self.transfer.append([("halve", b) for b in range(L.nb)])
        while self.levels[-1].nb * self.levels[-1].n ** 3 > max_coarse and not operator_only:
            nxt = self._merge_deepest(self.levels[-1])
            if nxt is None:
                break
            self.levels.append(nxt[0])
            self.transfer.append(nxt[1])
        self.gface = {}
        if bc is not None:
            L0 = self.levels[0]
            for b, key in enumerate(L0.keys):
                for f in range(6):
                    if L0.faces[b][f][0] == "bnd":
                        self.gface[(b, f)] = _boundary_face_values(R, n, key, f // 2, f % 2, bc)
        self.coeff = k_user is not None
        if self.coeff:
            L0 = self.levels[0]
            L0.kpad = self.to_pad(np.asarray(k_user, dtype=np.float64))
            self.exchange_k(0)
            for l in range(len(self.levels) - 1):
                kc = self.levels[l + 1].zeros()
                self._restrict_into(l, self.levels[l].kpad, kc)
                self.levels[l + 1].kpad = kc
                self.exchange_k(l + 1)
            for l in range(len(self.levels)):
                if l == 0 or coarse_coef == "k":
                    self._cache_T(l)
                else:
                    self._average_faces(l - 1)
        if not operator_only and coarse_iters is None:
            self._factor_coarsest()

    # -- hierarchy -------------------------------------------------------------------------------------
    def _merge_deepest(self, L):
        """Merge complete sibling octets of 4^3 blocks at the deepest level into their parent (a coarsening step
        below Sec. 5's block-local coarsening, used when the coarsest level is too large for a dense solve)."""
        deepest = max(key[0] for key in L.keys)
        m_parent = L.R * 2.0 ** (deepest - 1)
        if m_parent != int(m_parent) or m_parent < 1:
            return None
        groups = {}
        for key in L.keys:
            if key[0] == deepest:
                groups.setdefault((deepest - 1, key[1] // 2, key[2] // 2, key[3] // 2), []).append(key)
        parents = {p for p, ch in groups.items() if len(ch) == 8}
        if not parents:
            return None
        merged = set()
        for p in parents:
            merged.update(groups[p])
        keys = [k for k in L.keys if k not in merged] + sorted(parents, key=lambda t: (t[3], t[2], t[1]))
        C = Level(L.R, L.n, keys)
        tr = []
        for key in C.keys:
            if key in parents:
                l, i, j, k = key
                ch = [L.index[(l + 1, 2 * i + a, 2 * j + b, 2 * k + c)] for c in (0, 1) for b in (0, 1) for a in (0, 1)]
                tr.append(("merge", ch))
            else:
                tr.append(("copy", L.index[key]))
        return C, tr

    # -- layout ----------------------------------------------------------------------------------------
    def to_pad(self, x_user, level=0):
        """User layout (leaf-major, n^3 per leaf, x fastest) -> blocks with a zero ghost layer."""
        L = self.levels[level]
        n = L.n
        U = L.zeros()
        U[:, 1:-1, 1:-1, 1:-1] = np.asarray(x_user, dtype=np.float64).reshape(L.nb, n, n, n)
        return U

    def from_pad(self, U):
        """Blocks with ghosts -> user layout (interior only)."""
        return U[:, 1:-1, 1:-1, 1:-1].reshape(U.shape[0], -1).copy()

    def with_dtype(self, dtype):
        """A copy of this oracle whose cycles compute in ``dtype``: level fields, ghost exchange, smoother,
        residual, transfers and face coefficients (the harmonic means of the FP64 k pyramid rounded to dtype).  The
        set-up stays this oracle's: hierarchy, FP64 k pyramid and the LU factors of the FP64 coarsest operator, whose
        solves run in FP64 on the rounded right-hand side and are stored in dtype.  np.float32 gives the FP32
        V-cycles of the mixed-precision solve (not in the paper; its FP64 cycle is this oracle's default)."""
        other = copy.copy(self)
        other.dtype = np.dtype(dtype)
        other.levels = []
        for L in self.levels:
            M = copy.copy(L)
            M.dtype = other.dtype
            if L.kpad is not None:
                M.kpad = L.kpad.astype(other.dtype)
            other.levels.append(M)
        if self.coeff:
            for l in range(len(other.levels)):
                if l == 0 or self.coarse_coef == "k":
                    other._cache_T(l)
                else:  # averaged set-up data: the FP64 coefficients rounded
                    other.levels[l].T = [t.astype(other.dtype) for t in self.levels[l].T]
        return other

    def _h2(self, l):
        """h^2 of every block of level l in the working precision, broadcast over a block's cells."""
        return (self.levels[l].h ** 2).astype(self.dtype)[:, None, None, None]

    # -- ghost exchange --------------------------------------------------------------------------------
    def _c2f_values(self, Vc, n, seg):
        """Fine ghost face (n x n, [t1, t2]) from the coarse view Vc (Sec. 3.3.2, 3D scheme)."""
        E = sum(w * Vc[1 + a, 1:-1, 1:-1] for a, w in enumerate(self.normal_w))
        M1 = tangential_matrix(n, seg[0] * n // 2, self.c2f_order).astype(self.dtype)
        M2 = tangential_matrix(n, seg[1] * n // 2, self.c2f_order).astype(self.dtype)
        return M1 @ E @ M2.T

    def exchange(self, l, U):
        """Fill every ghost face of level l's field U (homogeneous Dirichlet on the domain boundary)."""
        L = self.levels[l]
        n, h2 = L.n, n_half(L.n)
        for b in range(L.nb):
            for f in range(6):
                axis, side = f // 2, f % 2
                fc = L.faces[b][f]
                V = face_view(U[b], axis, side)
                if fc[0] == "bnd":
                    g = self.gface.get((b, f)) if l == 0 else None
                    V[0, 1:-1, 1:-1] = -V[1, 1:-1, 1:-1] if g is None else 2.0 * g - V[1, 1:-1, 1:-1]
                elif fc[0] == "same":
                    W = face_view(U[fc[1]], axis, 1 - side)
                    V[0, 1:-1, 1:-1] = W[1, 1:-1, 1:-1]
                elif fc[0] == "c2f":
                    Vc = face_view(U[fc[1]], axis, 1 - side)
                    V[0, 1:-1, 1:-1] = self._c2f_values(Vc, n, fc[2])
                elif fc[0] == "f2c" and self.variant == "P":
                    for (fb, s1, s2) in fc[1]:
                        Vf = face_view(U[fb], axis, 1 - side)
                        o1, o2 = s1 * h2, s2 * h2
                        V[0, 1 + o1:1 + o1 + h2, 1 + o2:1 + o2 + h2] = \
                            Vf[1:3, 1:-1, 1:-1].reshape(2, h2, 2, h2, 2).mean(axis=(0, 2, 4))
        if self.variant == "C":
            for b in range(L.nb):
                for f in range(6):
                    fc = L.faces[b][f]
                    if fc[0] == "f2c":
                        self._f2c_flux(l, U, b, f // 2, f % 2, fc[1])

    def _f2c_flux(self, l, U, b, axis, side, segs):
        """Coarse ghost G with T_C (u_C - G) = 1/2 sum_j T_j (g_j - u_j) over the 4 fine cells j of each coarse face."""
        L = self.levels[l]
        h2 = n_half(L.n)
        V = face_view(U[b], axis, side)
        for (fb, s1, s2) in segs:
            Vf = face_view(U[fb], axis, 1 - side)
            o1, o2 = s1 * h2, s2 * h2
            g = Vf[0, 1:-1, 1:-1]
            u = Vf[1, 1:-1, 1:-1]
            uc = V[1, 1 + o1:1 + o1 + h2, 1 + o2:1 + o2 + h2]
            if self.coeff:
                Tj = self._face_T(l, fb, axis, 1 - side)
                Tc = self._face_T(l, b, axis, side)[o1:o1 + h2, o2:o2 + h2]
            else:
                Tj = np.ones_like(g)
                Tc = np.ones_like(uc)
            flux = (Tj * (g - u)).reshape(h2, 2, h2, 2).sum(axis=(1, 3))
            V[0, 1 + o1:1 + o1 + h2, 1 + o2:1 + o2 + h2] = uc - flux / (2.0 * Tc)

    def exchange_k(self, l):
        """Ghost k: boundary k_g = k_i; same level copy; fine ghosts inject the overlapping coarse cell's k;
        coarse ghosts take the mean of the 8 overlapping fine k."""
        L = self.levels[l]
        K = L.kpad
        h2 = n_half(L.n)
        for b in range(L.nb):
            for f in range(6):
                axis, side = f // 2, f % 2
                fc = L.faces[b][f]
                V = face_view(K[b], axis, side)
                if fc[0] == "bnd":
                    V[0, 1:-1, 1:-1] = V[1, 1:-1, 1:-1]
                elif fc[0] == "same":
                    V[0, 1:-1, 1:-1] = face_view(K[fc[1]], axis, 1 - side)[1, 1:-1, 1:-1]
                elif fc[0] == "c2f":
                    Vc = face_view(K[fc[1]], axis, 1 - side)
            # injection: fine ghost (yf, zf) lies in coarse cell (o1 + yf//2, o2 + zf//2) of the first layer
                    o1, o2 = fc[2][0] * h2, fc[2][1] * h2
                    seg = Vc[1, 1 + o1:1 + o1 + h2, 1 + o2:1 + o2 + h2]
                    V[0, 1:-1, 1:-1] = np.repeat(np.repeat(seg, 2, axis=0), 2, axis=1)
                elif fc[0] == "f2c":
                    for (fb, s1, s2) in fc[1]:
                        Vf = face_view(K[fb], axis, 1 - side)
                        o1, o2 = s1 * h2, s2 * h2
                        V[0, 1 + o1:1 + o1 + h2, 1 + o2:1 + o2 + h2] = \
                            Vf[1:3, 1:-1, 1:-1].reshape(2, h2, 2, h2, 2).mean(axis=(0, 2, 4))

    def _cache_T(self, l):
        """Face coefficients T_f of level l from its ghost-filled k (Sec. 5, Eq. 1 with a per-cell k)."""
        L = self.levels[l]
        K = L.kpad
        kc = K[:, 1:-1, 1:-1, 1:-1]
        L.T = [harmonic(kc, nb) for nb in _neighbours(K)]

    def _face_T(self, l, b, axis, side):
        """Face coefficients of block b's face (axis, side) at its first interior layer, [t1, t2] (n x n)."""
        return _interior_view(self.levels[l].T[2 * axis + side][b], axis, side)[0]

    def _average_faces(self, l):
        """Face coefficients of level l + 1 averaged from level l's (coarse_coef='faces'): a coarse cell's face is
        covered by 2 x 2 faces of the finer level (the finer cells next to it on that side), and its coefficient is
        their mean.  Blocks carried over unchanged keep their coefficients; merged octets are assembled first."""
        Lf, Lc = self.levels[l], self.levels[l + 1]
        out = [np.zeros((Lc.nb, Lc.n, Lc.n, Lc.n), dtype=self.dtype) for _ in range(6)]
        for B, tr in enumerate(self.transfer[l]):
            for q in range(6):
                if tr[0] == "copy":
                    out[q][B] = Lf.T[q][tr[1]]
                    continue
                fine = Lf.T[q][tr[1]] if tr[0] == "halve" else _assemble_octets([Lf.T[q][c] for c in tr[1]])
                axis, side = q // 2, q % 2
                sel = [slice(None)] * 3  # [z, y, x]
                sel[2 - axis] = slice(side, None, 2)  # the finer cells on the face's side of each coarse cell
                v = fine[tuple(sel)]
                for d in range(3):
                    if d == axis:
                        continue
                    a = 2 - d
                    lo = [slice(None)] * 3
                    hi = [slice(None)] * 3
                    lo[a], hi[a] = slice(0, None, 2), slice(1, None, 2)
                    v = 0.5 * (v[tuple(lo)] + v[tuple(hi)])
                out[q][B] = v
            if tr[0] == "merge":
                # Inside a merged block each face has one coefficient.  The two children meeting at a face between
                # them each bring their own average, and these differ where that face was a refinement interface
                # or lay between a copied and a merged block on the finer level: both sides take the mean of the two.
                h = Lc.n // 2
                for axis in range(3):
                    up = [slice(None)] * 3
                    dn = [slice(None)] * 3
                    up[2 - axis], dn[2 - axis] = h - 1, h  # coarse cells below / above the children's shared face
                    m = 0.5 * (out[2 * axis + 1][B][tuple(up)] + out[2 * axis][B][tuple(dn)])
                    out[2 * axis + 1][B][tuple(up)] = m
                    out[2 * axis][B][tuple(dn)] = m
        Lc.T = out

    # -- stencil ---------------------------------------------------------------------------------------
    def _T(self, l):
        """The six face-coefficient arrays of level l (1 for -Laplace)."""
        return self.levels[l].T if self.coeff else [1.0] * 6

    def apply_padded(self, l, U):
        """(A u) on the interior of level l, ghosts of U already filled."""
        L = self.levels[l]
        T = self._T(l)
        uc = U[:, 1:-1, 1:-1, 1:-1]
        acc = np.zeros_like(uc)
        for Tf, nb in zip(T, _neighbours(U)):
            acc += Tf * (uc - nb)
        return acc / self._h2(l)

    def residual(self, l, U, F):
        """r = f - A u on level l after a ghost exchange (Sec. 5, Eq. 1-2)."""
        self.exchange(l, U)
        return F - self.apply_padded(l, U)

    def half_sweep(self, l, U, F, colour):
        """Gauss-Seidel update of one colour: u_i = (h^2 f_i + sum_f T_f u_f) / sum_f T_f."""
        L = self.levels[l]
        self.exchange(l, U)
        T = self._T(l)
        num = self._h2(l) * F
        den = 0.0
        for Tf, nb in zip(T, _neighbours(U)):
            num = num + Tf * nb
            den = den + Tf
        new = num / den
        mask = L.colour_mask(colour)[None]
        uc = U[:, 1:-1, 1:-1, 1:-1]
        U[:, 1:-1, 1:-1, 1:-1] = np.where(mask, new, uc)

    def jacobi_sweep(self, l, U, F):
        """Damped Jacobi with ghosts frozen at the exchanged values: u_i <- (1 - w) u_i + w (h^2 f_i + sum_f T_f u_f)
        / sum_f T_f for every cell at once (the paper's smoother, Sec. 5, omega = 0.8)."""
        self.exchange(l, U)
        T = self._T(l)
        num = self._h2(l) * F
        den = 0.0
        for Tf, nb in zip(T, _neighbours(U)):
            num = num + Tf * nb
            den = den + Tf
        uc = U[:, 1:-1, 1:-1, 1:-1]
        U[:, 1:-1, 1:-1, 1:-1] = (1.0 - self.omega) * uc + self.omega * (num / den)

    def smooth(self, l, U, F, iters):
        """iters smoothing steps (Sec. 5): red-black Gauss-Seidel, or the paper's damped Jacobi, each after an
        exchange."""
        for _ in range(iters):
            if self.smoother == "jacobi":
                self.jacobi_sweep(l, U, F)
            else:
                self.half_sweep(l, U, F, 0)
                self.half_sweep(l, U, F, 1)

    # -- transfers -------------------------------------------------------------------------------------
    def _restrict_into(self, l, Xf, Xc_pad):
        """Mean of the 8 children (8:1 restriction) from level l (padded or interior) into level l+1's interior."""
        Lf, Lc = self.levels[l], self.levels[l + 1]
        nf, nc = Lf.n, Lc.n
        Xi = Xf[:, 1:-1, 1:-1, 1:-1] if Xf.shape[1] == nf + 2 else Xf
        for B, tr in enumerate(self.transfer[l]):
            if tr[0] == "copy":
                Xc_pad[B, 1:-1, 1:-1, 1:-1] = Xi[tr[1]]
                continue
            fine = Xi[tr[1]] if tr[0] == "halve" else _assemble_octets([Xi[c] for c in tr[1]])
            Xc_pad[B, 1:-1, 1:-1, 1:-1] = fine.reshape(nc, 2, nc, 2, nc, 2).mean(axis=(1, 3, 5))

    def exchange_diagonal(self, l, U):
        """Edge and corner ghosts of level l, after the face exchange: the cells of a same-level block across the edge
        or corner where there is one; else linear extrapolation, along each of the edge's (corner's) ghost axes in
        turn, from the two ghosts next to it on that axis (face ghosts for an edge, edge ghosts for a corner), and the
        mean of the two (three) results.  Data linear along each axis (trilinear data) is reproduced exactly.  Edges
        first, then corners.  The paper defines no diagonal ghosts (Sec. 8 lists them as future work for wider
        stencils); this is the reading used for the trilinear prolongation."""
        L = self.levels[l]
        n = L.n

        def at(sel):  # sel: per axis (x, y, z) an index or a slice; array order [b, z, y, x]
            return (sel[2], sel[1], sel[0])

        def ghost(side):
            return 0 if side < 0 else n + 1

        def inner(side, depth):  # the interior index `depth` cells in from the ghost (depth 1 or 2)
            return depth if side < 0 else n + 1 - depth

        for b, key in enumerate(L.keys):
            lev, idx = key[0], list(key[1:])
            m = L.blocks_per_axis(lev)
            V = U[b]
            for corner in (False, True):
                axes_sets = [(0, 1, 2)] if corner else [(0, 1), (0, 2), (1, 2)]
                for axes in axes_sets:
                    for signs in np.ndindex(*([2] * len(axes))):
                        sg = [1 if q else -1 for q in signs]
                        p = idx.copy()
                        for a_, s_ in zip(axes, sg):
                            p[a_] += s_
                        nb = L.index.get((lev, *p)) if all(0 <= v < m for v in p) else None
                        sel = [slice(1, n + 1)] * 3
                        for a_, s_ in zip(axes, sg):
                            sel[a_] = ghost(s_)
                        if nb is not None:
                            src = [slice(1, n + 1)] * 3
                            for a_, s_ in zip(axes, sg):
                                src[a_] = 1 if s_ > 0 else n  # the neighbour's cells next to the edge / corner
                            V[at(sel)] = U[nb][at(src)]
                            continue
                        acc = 0.0
                        for a_, s_ in zip(axes, sg):  # extrapolate along a_ from the two ghosts next to it
                            s1, s2 = list(sel), list(sel)
                            s1[a_], s2[a_] = inner(s_, 1), inner(s_, 2)
                            acc = acc + (2.0 * V[at(s1)] - V[at(s2)])
                        V[at(sel)] = acc / len(axes)

    def _prolong_add(self, l, Ec_pad, Uf):
        """u_f += P e_c, P the face-neighbour linear cell-centred interpolation; Ec_pad has its ghosts filled."""
        Lf, Lc = self.levels[l], self.levels[l + 1]
        nc = Lc.n
        for B, tr in enumerate(self.transfer[l]):
            E = Ec_pad[B]
            if tr[0] == "copy":
                Uf[tr[1], 1:-1, 1:-1, 1:-1] += E[1:-1, 1:-1, 1:-1]
                continue
            P = np.zeros((2 * nc,) * 3, dtype=E.dtype)
            c = E[1:-1, 1:-1, 1:-1]
            for sz in (0, 1):
                for sy in (0, 1):
                    for sx in (0, 1):
                        if self.prolongation == "trilinear":
                            # weights (3/4)^(3-d) (1/4)^d of the coarse cells d steps (0..3 axes) towards the fine cell
                            acc = np.zeros_like(c)
                            for dz in (0, 1):
                                for dy in (0, 1):
                                    for dx in (0, 1):
                                        oz, oy, ox = (dz if sz else -dz), (dy if sy else -dy), (dx if sx else -dx)
                                        w = 0.75 ** (3 - dx - dy - dz) * 0.25 ** (dx + dy + dz)
                                        acc = acc + w * E[1 + oz:nc + 1 + oz, 1 + oy:nc + 1 + oy, 1 + ox:nc + 1 + ox]
                            P[sz::2, sy::2, sx::2] = acc
                            continue
                        ex = E[1:-1, 1:-1, 2:] if sx else E[1:-1, 1:-1, :-2]
                        ey = E[1:-1, 2:, 1:-1] if sy else E[1:-1, :-2, 1:-1]
                        ez = E[2:, 1:-1, 1:-1] if sz else E[:-2, 1:-1, 1:-1]
                        P[sz::2, sy::2, sx::2] = 0.25 * (c + ex + ey + ez)
            if tr[0] == "halve":
                Uf[tr[1], 1:-1, 1:-1, 1:-1] += P
            else:
                for o, cb in enumerate(tr[1]):
                    a, bb, cc = o % 2, (o // 2) % 2, o // 4
                    Uf[cb, 1:-1, 1:-1, 1:-1] += P[cc * nc:(cc + 1) * nc, bb * nc:(bb + 1) * nc, a * nc:(a + 1) * nc]

    # -- coarsest solve --------------------------------------------------------------------------------
    def _factor_coarsest(self):
        """Dense LU of the coarsest level's operator, assembled column by column (this project's direct coarsest
        solver; the paper's is damped Jacobi, Sec. 5, available through coarse_iters)."""
        l = len(self.levels) - 1
        L = self.levels[l]
        N = L.nb * L.n ** 3
        A = np.zeros((N, N))
        for m in range(N):
            X = np.zeros(N)
            X[m] = 1.0
            U = L.zeros()
            U[:, 1:-1, 1:-1, 1:-1] = X.reshape(L.nb, L.n, L.n, L.n)
            self.exchange(l, U)
            A[:, m] = self.apply_padded(l, U).reshape(-1)
        self.A_coarse = A
        self.lu = scipy.linalg.lu_factor(A)

    def coarse_solve(self, F):
        """Coarsest-level solve: dense LU, or coarse_iters damped Jacobi sweeps from zero (Sec. 5)."""
        l = len(self.levels) - 1
        L = self.levels[l]
        U = L.zeros()
        if self.coarse_iters is not None:
            for _ in range(self.coarse_iters):
                self.jacobi_sweep(l, U, F)
            return U
        U[:, 1:-1, 1:-1, 1:-1] = scipy.linalg.lu_solve(self.lu, F.reshape(-1)).reshape(F.shape)
        return U

    # -- cycle -----------------------------------------------------------------------------------------
    def vcycle(self, l, U, F):
        """One V(nu1, nu2) cycle from level l (Sec. 5): smooth, restrict the residual, recurse, prolongate and
        correct, smooth."""
        if l == len(self.levels) - 1:
            U[...] = self.coarse_solve(F)
            return
        self.smooth(l, U, F, self.nu1)
        r = self.residual(l, U, F)
        Fc = self.levels[l + 1].zeros()
        self._restrict_into(l, r, Fc)
        Fc = Fc[:, 1:-1, 1:-1, 1:-1].copy()
        Ec = self.levels[l + 1].zeros()
        self.vcycle(l + 1, Ec, Fc)
        self.exchange(l + 1, Ec)
        if self.prolongation == "trilinear":
            self.exchange_diagonal(l + 1, Ec)
        self._prolong_add(l, Ec, U)
        self.smooth(l, U, F, self.nu2)

    def norm(self, l, X):
        """Volume-weighted L2 norm sqrt(sum h^3 x^2) (Sec. 5's L2 norm, in the reading that gives its kappa)."""
        L = self.levels[l]
        return float(np.sqrt(np.sum((L.h ** 3)[:, None, None, None] * X ** 2)))

    def solve(self, f_user, u0_user=None, cycles=None, rtol=None, max_cycles=100):
        """V-cycles from u0 (default 0): exactly ``cycles`` of them, or until ||r|| / ||r_0|| <= rtol.

        r_0 is the residual of the zero guess, i.e. f itself under homogeneous Dirichlet data.
        Returns (u_user, list of relative residuals after each cycle).
        """
        F = self.to_pad(f_user)[:, 1:-1, 1:-1, 1:-1].copy()
        U = self.to_pad(u0_user) if u0_user is not None else self.levels[0].zeros()
        fn = self.norm(0, self.residual(0, self.levels[0].zeros(), F))
        hist = []
        ncyc = cycles if cycles is not None else max_cycles
        for _ in range(ncyc):
            self.vcycle(0, U, F)
            rel = self.norm(0, self.residual(0, U, F)) / fn
            hist.append(rel)
            if rtol is not None and rel <= rtol:
                break
        return self.from_pad(U), hist

    # -- plain operator in user layout -----------------------------------------------------------------
    def apply_A(self, u_user, level=0):
        """A u in user layout (Sec. 5, Eq. 1-2), ghosts from the exchange of Sec. 3."""
        U = self.to_pad(u_user, level)
        self.exchange(level, U)
        return self.apply_padded(level, U).reshape(U.shape[0], -1)

    def rel_residual(self, u_user, f_user):
        """||f - A u|| / ||f|| in the volume-weighted norm (Sec. 5)."""
        F = self.to_pad(f_user)[:, 1:-1, 1:-1, 1:-1]
        U = self.to_pad(u_user)
        return self.norm(0, self.residual(0, U, F)) / self.norm(0, F)

    # -- adjoint ---------------------------------------------------------------------------------------
    def apply_AT(self, y_user):
        """A^T y on the finest level, in user layout."""
        L = self.levels[0]
        return self.apply_AT_level(0, y_user.reshape(L.nb, L.n, L.n, L.n)).reshape(L.nb, -1)

    def apply_AT_level(self, l, Y_int):
        """A^T y on level l (interior arrays): transposed stencil into a padded adjoint array, then the transposed
        ghost exchange."""
        L = self.levels[l]
        Y = Y_int / (L.h ** 2)[:, None, None, None]
        T = self._T(l)
        G = L.zeros()
        for Tf, sl in zip(T, _neighbour_slices()):
            G[:, 1:-1, 1:-1, 1:-1] += Tf * Y
            G[(slice(None),) + sl] -= Tf * Y
        self.exchange_T(l, G)
        return G[:, 1:-1, 1:-1, 1:-1].copy()

    def exchange_T(self, l, G):
        """Transpose of the (linear part of the) ghost exchange, in place on a padded adjoint array G: every ghost
        adjoint is added into the interior cells its ghost value was computed from.  Reverse order of the forward
        exchange: the flux-carrying coarse ghosts (variant C) first, then copies, reflections, C2F and F2C."""
        if self.c2f_order != 2:
            raise NotImplementedError("the transposed exchange is written for the quadratic coarse-to-fine scheme")
        L = self.levels[l]
        n = L.n
        h2 = n_half(n)
        if self.variant == "C":
            for b in range(L.nb):
                for f in range(6):
                    fc = L.faces[b][f]
                    if fc[0] != "f2c":
                        continue
                    axis, side = f // 2, f % 2
                    V = face_view(G[b], axis, side)
                    for (fb, s1, s2) in fc[1]:
                        o1, o2 = s1 * h2, s2 * h2
                        Gg = V[0, 1 + o1:1 + o1 + h2, 1 + o2:1 + o2 + h2]
                        if self.coeff:
                            Tj = self._face_T(l, fb, axis, 1 - side)
                            Tc = self._face_T(l, b, axis, side)[o1:o1 + h2, o2:o2 + h2]
                        else:
                            Tj, Tc = np.ones((n, n)), np.ones((h2, h2))
                        V[1, 1 + o1:1 + o1 + h2, 1 + o2:1 + o2 + h2] += Gg
                        cj = Tj / (2.0 * np.repeat(np.repeat(Tc, 2, axis=0), 2, axis=1))
                        Gj = np.repeat(np.repeat(Gg, 2, axis=0), 2, axis=1)
                        Vf = face_view(G[fb], axis, 1 - side)
                        Vf[0, 1:-1, 1:-1] -= cj * Gj
                        Vf[1, 1:-1, 1:-1] += cj * Gj
        for b in range(L.nb):
            for f in range(6):
                axis, side = f // 2, f % 2
                fc = L.faces[b][f]
                V = face_view(G[b], axis, side)
                gadj = V[0, 1:-1, 1:-1]
                if fc[0] == "bnd":
                    V[1, 1:-1, 1:-1] -= gadj
                elif fc[0] == "same":
                    face_view(G[fc[1]], axis, 1 - side)[1, 1:-1, 1:-1] += gadj
                elif fc[0] == "c2f":
                    seg = fc[2]
                    M1 = tangential_matrix(n, seg[0] * n // 2)
                    M2 = tangential_matrix(n, seg[1] * n // 2)
                    back = M1.T @ gadj @ M2
                    Vc = face_view(G[fc[1]], axis, 1 - side)
                    for a in range(3):
                        Vc[1 + a, 1:-1, 1:-1] += NORMAL_W[a] * back
                elif fc[0] == "f2c" and self.variant == "P":
                    for (fb, s1, s2) in fc[1]:
                        o1, o2 = s1 * h2, s2 * h2
                        Gg = V[0, 1 + o1:1 + o1 + h2, 1 + o2:1 + o2 + h2]
                        Vf = face_view(G[fb], axis, 1 - side)
                        Vf[1:3, 1:-1, 1:-1] += np.repeat(np.repeat(Gg, 2, axis=0), 2, axis=1)[None] / 8.0

    def _diag_lagged(self, l):
        """sum_f T_f / h^2: the diagonal the ghost-lagged smoother divides by."""
        L = self.levels[l]
        T = self._T(l)
        D = sum(np.broadcast_to(Tf, (L.nb, L.n, L.n, L.n)) for Tf in T)
        return D / (L.h ** 2)[:, None, None, None]

    def _restrict_T(self, l, Fc_bar):
        """Transpose of the 8:1 mean restriction: each fine cell receives 1/8 of its parent's adjoint."""
        Lf, Lc = self.levels[l], self.levels[l + 1]
        nc = Lc.n
        out = np.zeros((Lf.nb, Lf.n, Lf.n, Lf.n))
        for B, tr in enumerate(self.transfer[l]):
            x = Fc_bar[B]
            if tr[0] == "copy":
                out[tr[1]] += x
                continue
            big = np.repeat(np.repeat(np.repeat(x, 2, 0), 2, 1), 2, 2) / 8.0
            if tr[0] == "halve":
                out[tr[1]] += big
            else:
                for o, cb in enumerate(tr[1]):
                    a, bb, cc = o % 2, (o // 2) % 2, o // 4
                    out[cb] += big[cc * nc:(cc + 1) * nc, bb * nc:(bb + 1) * nc, a * nc:(a + 1) * nc]
        return out

    def _prolong_T(self, l, Ubar_int):
        """Transpose of u_f += P e_c: the padded coarse adjoint of the interpolation stencil, then the transposed
        coarse exchange (P reads coarse ghosts).  Returns the coarse interior adjoint."""
        Lf, Lc = self.levels[l], self.levels[l + 1]
        nc = Lc.n
        Eb = Lc.zeros()
        for B, tr in enumerate(self.transfer[l]):
            if tr[0] == "copy":
                Eb[B, 1:-1, 1:-1, 1:-1] += Ubar_int[tr[1]]
                continue
            Q = Ubar_int[tr[1]] if tr[0] == "halve" else _assemble_octets([Ubar_int[c] for c in tr[1]])
            E = Eb[B]
            for sz in (0, 1):
                for sy in (0, 1):
                    for sx in (0, 1):
                        q = 0.25 * Q[sz::2, sy::2, sx::2]
                        E[1:-1, 1:-1, 1:-1] += q
                        E[1:-1, 1:-1, (slice(2, None) if sx else slice(0, -2))] += q
                        E[1:-1, (slice(2, None) if sy else slice(0, -2)), 1:-1] += q
                        E[(slice(2, None) if sz else slice(0, -2)), 1:-1, 1:-1] += q
        self.exchange_T(l + 1, Eb)
        return Eb[:, 1:-1, 1:-1, 1:-1].copy()

    def _smooth_steps(self, nu):
        """Colour order of nu red-black Gauss-Seidel iterations (red first)."""
        return [c for _ in range(nu) for c in (0, 1)]

    def vcycle_transposed(self, l, Ubar):
        """M_l^T: the exact transpose of the forward V-cycle map f -> u (zero initial guess) on level l.
        Written for red-black Gauss-Seidel and the dense coarsest solve.

        The forward cycle is a sequence of linear steps (half-sweeps u += Pi_c D^-1 (f - A u), residual,
        restriction, coarse cycle, prolongation); its transpose runs them in reverse with each step transposed.
        A half-sweep's transpose is: z = Pi_c D^-1 ubar; fbar += z; ubar -= A^T z.
        Returns fbar (interior array of level l)."""
        if self.smoother != "rbgs" or self.coarse_iters is not None:
            raise NotImplementedError("the transposed cycle is written for red-black Gauss-Seidel and a dense "
                                      "coarsest solve")
        L = self.levels[l]
        if l == len(self.levels) - 1:
            return scipy.linalg.lu_solve(self.lu, Ubar.reshape(-1), trans=1).reshape(Ubar.shape)
        D = self._diag_lagged(l)
        masks = [L.colour_mask(0)[None], L.colour_mask(1)[None]]
        ub = Ubar.copy()
        fb = np.zeros_like(ub)

        def smooth_T(steps):
            nonlocal ub, fb
            for c in reversed(steps):
                z = np.where(masks[c], ub / D, 0.0)
                fb += z
                ub = ub - self.apply_AT_level(l, z)

        smooth_T(self._smooth_steps(self.nu2))
        ecb = self._prolong_T(l, ub)
        fcb = self.vcycle_transposed(l + 1, ecb)
        rb = self._restrict_T(l, fcb)
        fb += rb
        ub = ub - self.apply_AT_level(l, rb)
        smooth_T(self._smooth_steps(self.nu1))
        return fb

    def adjoint_solve(self, g_user, rtol=1e-13, max_cycles=100, return_history=False):
        """lambda with A^T lambda = g, by defect correction lambda += M^T (g - A^T lambda), M the forward V-cycle.

        The error propagator is (I - M A)^T, so it converges at the forward cycle's rate.
        """
        L = self.levels[0]
        n = L.n
        G = np.asarray(g_user, dtype=np.float64).reshape(L.nb, n, n, n)
        lam = np.zeros_like(G)
        gn = self.norm(0, G)
        hist = []
        for _ in range(max_cycles):
            lam = lam + self.vcycle_transposed(0, G - self.apply_AT_level(0, lam))
            rel = self.norm(0, G - self.apply_AT_level(0, lam)) / gn
            hist.append(rel)
            if rel <= rtol:
                break
        else:
            raise RuntimeError(f"adjoint multigrid did not reach {rtol} in {max_cycles} cycles: {hist[-3:]}")
        lam = lam.reshape(L.nb, -1)
        return (lam, hist) if return_history else lam

    def grad_k(self, u_user, lam_user):
        """dL/dk = -lambda^T (dA/dk) u, face by face through the harmonic-mean coefficients and ghost k maps."""
        if not self.coeff:
            raise ValueError("constant-coefficient problem has no k")
        L = self.levels[0]
        n = L.n
        h2 = n_half(n)
        U = self.to_pad(u_user)
        self.exchange(0, U)
        K = L.kpad
        kc = K[:, 1:-1, 1:-1, 1:-1]
        lam = lam_user.reshape(L.nb, n, n, n) / (L.h ** 2)[:, None, None, None]
        uc = U[:, 1:-1, 1:-1, 1:-1]
        grad = np.zeros_like(kc)
        gadj = L.zeros()  # adjoint of the k value at neighbour/ghost positions
        # mask out coarse-side interface faces in variant C (their row term is handled below)
        skip = np.zeros((6,) + kc.shape, dtype=bool)
        if self.variant == "C":
            for b in range(L.nb):
                for f in range(6):
                    if L.faces[b][f][0] == "f2c":
                        m = np.zeros((n + 2,) * 3, dtype=bool)
                        face_view(m, f // 2, f % 2)[1, 1:-1, 1:-1] = True
                        skip[f, b] = m[1:-1, 1:-1, 1:-1]
        for f, (nb, sl) in enumerate(zip(_neighbours(K), _neighbour_slices())):
            unb = _neighbours(U)[f]
            d = uc - unb
            dTa = 2.0 * nb ** 2 / (kc + nb) ** 2
            dTb = 2.0 * kc ** 2 / (kc + nb) ** 2
            w = np.where(skip[f], 0.0, -lam * d)
            grad += w * dTa
            gadj[(slice(None),) + sl] += w * dTb
        grad += gadj[:, 1:-1, 1:-1, 1:-1]  # neighbours inside the block: their own k
        for b in range(L.nb):
            for f in range(6):
                axis, side = f // 2, f % 2
                fc = L.faces[b][f]
                Vg = face_view(gadj[b], axis, side)
                gr = _interior_view(grad[b], axis, side)
                if fc[0] == "bnd":
                    gr[0] += Vg[0, 1:-1, 1:-1]
                elif fc[0] == "same":
                    _interior_view(grad[fc[1]], axis, 1 - side)[0] += Vg[0, 1:-1, 1:-1]
                elif fc[0] == "c2f":
                    o1, o2 = fc[2][0] * h2, fc[2][1] * h2
                    s = Vg[0, 1:-1, 1:-1].reshape(h2, 2, h2, 2).sum(axis=(1, 3))
                    _interior_view(grad[fc[1]], axis, 1 - side)[0, o1:o1 + h2, o2:o2 + h2] += s
                elif fc[0] == "f2c" and self.variant == "P":
                    for (fb, s1, s2) in fc[1]:
                        o1, o2 = s1 * h2, s2 * h2
                        a = Vg[0, 1 + o1:1 + o1 + h2, 1 + o2:1 + o2 + h2] / 8.0
                        gi = _interior_view(grad[fb], axis, 1 - side)
                        gi[0:2] += np.repeat(np.repeat(a, 2, axis=0), 2, axis=1)[None]
                elif fc[0] == "f2c" and self.variant == "C":
                    # row C term: (1/h_c^2) 1/2 sum_j T_j (g_j - u_j), T_j = harmonic(k_j, k_C)
                    for (fb, s1, s2) in fc[1]:
                        o1, o2 = s1 * h2, s2 * h2
                        Vf = face_view(U[fb], axis, 1 - side)
                        Kf = face_view(K[fb], axis, 1 - side)
                        kj = Kf[1, 1:-1, 1:-1]
                        kC = np.repeat(np.repeat(face_view(K[b], axis, side)[1, 1 + o1:1 + o1 + h2, 1 + o2:1 + o2 + h2],
                                                 2, axis=0), 2, axis=1)
                        lC = np.repeat(np.repeat(_interior_view(lam[b], axis, side, padded=False)[0, o1:o1 + h2, o2:o2 + h2],
                                                 2, axis=0), 2, axis=1)
                        dd = 0.5 * (Vf[0, 1:-1, 1:-1] - Vf[1, 1:-1, 1:-1])
                        w = -lC * dd
                        _interior_view(grad[fb], axis, 1 - side)[0] += w * 2.0 * kC ** 2 / (kj + kC) ** 2
                        s = (w * 2.0 * kj ** 2 / (kj + kC) ** 2).reshape(h2, 2, h2, 2).sum(axis=(1, 3))
                        _interior_view(grad[b], axis, side)[0, o1:o1 + h2, o2:o2 + h2] += s
        return grad.reshape(L.nb, -1)


def pow2_near(x):
    """The power of two nearest to x > 0 in the log scale (2^round(log2 x)); scaling by it is exact in binary
    floating point."""
    return float(2.0 ** np.round(np.log2(x)))


def mixed_solve(mg64, f_user, steps, inner=1, mg32=None, u0_user=None):
    """FP32 V-cycles inside FP64 defect correction (the mixed-precision solve; the paper itself computes in FP64).

    Every step: r = f - A u in FP64 (the finest operator with its exchange); s = pow2_near(1 / ||r||) with the
    volume-weighted norm; rhs = FP32(s r); ``inner`` V-cycles of the FP32 copy mg32 (default
    mg64.with_dtype(np.float32)) on A e = rhs from e = 0; u += e / s in FP64.  Because s is a power of two the
    scaling adds no rounding, and with an FP64 copy in place of mg32 a step equals ``inner`` FP64 V-cycles on u.
    Returns (u_user, [||f - A u|| / ||f|| after every step]).
    """
    if mg32 is None:
        mg32 = mg64.with_dtype(np.float32)
    L0 = mg64.levels[0]
    F = mg64.to_pad(f_user)[:, 1:-1, 1:-1, 1:-1].copy()
    U = mg64.to_pad(u0_user) if u0_user is not None else L0.zeros()
    fn = mg64.norm(0, mg64.residual(0, L0.zeros(), F))
    hist = []
    for _ in range(steps):
        r = mg64.residual(0, U, F)
        rn = mg64.norm(0, r)
        if rn == 0.0:
            hist.append(0.0)
            break
        s = pow2_near(1.0 / rn)
        rhs = (s * r).astype(mg32.dtype)
        E = mg32.levels[0].zeros()
        for _ in range(inner):
            mg32.vcycle(0, E, rhs)
        U[:, 1:-1, 1:-1, 1:-1] += E[:, 1:-1, 1:-1, 1:-1].astype(np.float64) / s
        hist.append(mg64.norm(0, mg64.residual(0, U, F)) / fn)
    return mg64.from_pad(U), hist


# ----------------------------------------------------------------------------------------------------------
# small helpers
# ----------------------------------------------------------------------------------------------------------


def n_half(n):
    """Coarse cells along a block edge covered by one coarse-fine segment (Sec. 3.3: a fine face covers half)."""
    return n // 2


def _boundary_face_values(R, n, key, axis, side, g):
    """g at the n x n face centres of a block's boundary face, in face_view order [t1, t2]."""
    lev = key[0]
    ext = 1.0 / (R * 2.0 ** lev)
    h = ext / n
    org = np.array(key[1:], dtype=np.float64) * ext
    t1, t2 = [d for d in range(3) if d != axis]
    c1 = org[t1] + (np.arange(n) + 0.5) * h
    c2 = org[t2] + (np.arange(n) + 0.5) * h
    A, B = np.meshgrid(c1, c2, indexing="ij")
    X = [None, None, None]
    X[axis] = np.full_like(A, org[axis] + (ext if side == 1 else 0.0))
    X[t1], X[t2] = A, B
    return g(X[0], X[1], X[2])


def _neighbour_slices():
    """Padded-array slices of the 6 face neighbours of every interior cell, order x-, x+, y-, y+, z-, z+."""
    I = slice(1, -1)
    return [
        (I, I, slice(0, -2)), (I, I, slice(2, None)),
        (I, slice(0, -2), I), (I, slice(2, None), I),
        (slice(0, -2), I, I), (slice(2, None), I, I),
    ]


def _neighbours(U):
    """The six face-neighbour views of every interior cell of padded blocks U (the 7-point stencil)."""
    return [U[(slice(None),) + sl] for sl in _neighbour_slices()]


def _interior_view(a, axis, side, padded=False):
    """View [depth, t1, t2] of an interior-only block array (n, n, n) for face (axis, side); depth 0 = first layer."""
    t1, t2 = [d for d in range(3) if d != axis]
    v = np.moveaxis(a, (2 - axis, 2 - t1, 2 - t2), (0, 1, 2))
    return v[::-1] if side == 1 else v


def _assemble_octets(children):
    """8 child blocks (n^3 each, octant order x fastest) -> one (2n)^3 array."""
    n = children[0].shape[0]
    out = np.zeros((2 * n,) * 3, dtype=children[0].dtype)
    for o, c in enumerate(children):
        a, b, cc = o % 2, (o // 2) % 2, o // 4
        out[cc * n:(cc + 1) * n, b * n:(b + 1) * n, a * n:(a + 1) * n] = c
    return out
