"""Test-side helpers: geometry of padded blocks and small forests.  No solver arithmetic lives here."""
import numpy as np


def padded_centres(R, n, key):
    """Cell-centre coordinates (x, y, z), each (n+2)^3 indexed [z, y, x], of a padded block (ghosts included)."""
    lev, i, j, k = key
    ext = 1.0 / (R * 2.0 ** lev)
    h = ext / n
    t = (np.arange(n + 2) - 0.5) * h
    z, y, x = np.meshgrid(k * ext + t, j * ext + t, i * ext + t, indexing="ij")
    return x, y, z


def one_refined_root(R=2, root=(0, 0, 0)):
    """R^3 roots with one root split into its 8 children."""
    keys = [(0, i, j, k) for k in range(R) for j in range(R) for i in range(R) if (i, j, k) != tuple(root)]
    i, j, k = root
    keys += [(1, 2 * i + a, 2 * j + b, 2 * k + c) for c in (0, 1) for b in (0, 1) for a in (0, 1)]
    return keys


def poly3(coef):
    """p(x, y, z) = sum coef[a, b, c] x^a y^b z^c."""
    def p(x, y, z):
        out = np.zeros_like(x)
        for a in range(coef.shape[0]):
            for b in range(coef.shape[1]):
                for c in range(coef.shape[2]):
                    out = out + coef[a, b, c] * x ** a * y ** b * z ** c
        return out
    return p


def neg_laplace_poly3(coef):
    """-Laplace(p) for p = poly3(coef), analytic."""
    def q(x, y, z):
        out = np.zeros_like(x)
        A, B, C = coef.shape
        for a in range(A):
            for b in range(B):
                for c in range(C):
                    w = coef[a, b, c]
                    if a >= 2:
                        out = out - w * a * (a - 1) * x ** (a - 2) * y ** b * z ** c
                    if b >= 2:
                        out = out - w * b * (b - 1) * x ** a * y ** (b - 2) * z ** c
                    if c >= 2:
                        out = out - w * c * (c - 1) * x ** a * y ** b * z ** (c - 2)
        return out
    return q


def vw_norm(h_per_leaf, x):
    """Volume-weighted L2 norm sqrt(sum h^3 x^2) of a (n_leaves, n^3) field."""
    return float(np.sqrt(np.sum(np.asarray(h_per_leaf)[:, None] ** 3 * np.asarray(x) ** 2)))


def leaf_h(R, n, keys):
    return np.array([1.0 / (R * 2.0 ** key[0] * n) for key in keys])


def batch_stencils(problems, rng, per_problem=64):
    """Sampled cells of a batch whose six face neighbours are in the same block, in a same-level leaf or on the
    domain boundary (cells next to a refinement interface are drawn and dropped): flat indices (m, 7) into the
    batch layout (a boundary face's column repeats the cell), boundary flags (m, 6), problem ids and cell widths."""
    idx, bnds, pids, hs = [], [], [], []
    off = 0
    for p, (n, keys) in enumerate(problems):
        where = {key: b for b, key in enumerate(keys)}
        for _ in range(per_problem):
            b = int(rng.integers(0, len(keys)))
            lev, bi, bj, bk = keys[b]
            c = rng.integers(0, n, size=3)
            row, flags, ok = [off + b * n ** 3 + int(c[0] + n * (c[1] + n * c[2]))], [], True
            for face in range(6):
                axis, side = face // 2, face % 2
                q = c.copy()
                q[axis] += 1 if side else -1
                if 0 <= q[axis] < n:
                    row.append(off + b * n ** 3 + int(q[0] + n * (q[1] + n * q[2])))
                    flags.append(False)
                    continue
                nb = [bi, bj, bk]
                nb[axis] += 1 if side else -1
                if not 0 <= nb[axis] < 2 ** lev:
                    row.append(row[0])
                    flags.append(True)
                    continue
                key = (lev, *nb)
                if key not in where:
                    ok = False  # a refinement interface: not a same-level stencil
                    break
                q[axis] %= n
                row.append(off + where[key] * n ** 3 + int(q[0] + n * (q[1] + n * q[2])))
                flags.append(False)
            if ok:
                idx.append(row)
                bnds.append(flags)
                pids.append(p)
                hs.append(1.0 / (n * 2 ** lev))
        off += len(keys) * n ** 3
    return np.array(idx), np.array(bnds), np.array(pids), np.array(hs)
