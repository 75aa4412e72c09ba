"""Seeded cell-centred fields on a block forest, in the solver's user layout.

Layout: leaf-major in the order of the leaf list; each leaf holds its n^3 interior cells with x fastest, i.e.
element [leaf, (z * n + y) * n + x].  Every function returns a float64 torch tensor of shape (n_leaves, n^3) on
the requested device (plain torch arithmetic: these are inputs, not solver work).  Random draws use
``numpy.random.default_rng(seed)`` in the order stated in each docstring.
"""
from __future__ import annotations

import math

import numpy as np
import torch

F64 = torch.float64


def _leaf_geometry(R: int, keys, device):
    lv = torch.tensor([k[0] for k in keys], dtype=F64, device=device)
    ijk = torch.tensor([[k[1], k[2], k[3]] for k in keys], dtype=F64, device=device)
    ext = 1.0 / (R * torch.pow(torch.tensor(2.0, dtype=F64, device=device), lv))
    return ijk * ext[:, None], ext


def cell_centres(R: int, n: int, keys, device="cpu", leaf_slice=slice(None)):
    """Cell-centre coordinates, shape (L, n, n, n, 3) indexed [leaf, z, y, x, axis] with axis 0 = x."""
    keys = list(keys)[leaf_slice]
    org, ext = _leaf_geometry(R, keys, device)
    h = ext / n
    t = torch.arange(n, dtype=F64, device=device) + 0.5
    L = len(keys)
    xs = org[:, 0, None] + h[:, None] * t[None, :]
    ys = org[:, 1, None] + h[:, None] * t[None, :]
    zs = org[:, 2, None] + h[:, None] * t[None, :]
    out = torch.empty((L, n, n, n, 3), dtype=F64, device=device)
    out[..., 0] = xs[:, None, None, :]
    out[..., 1] = ys[:, None, :, None]
    out[..., 2] = zs[:, :, None, None]
    return out


def _chunks(keys, chunk):
    for s in range(0, len(keys), chunk):
        yield slice(s, min(s + chunk, len(keys)))


def sin_product(R, n, keys, device="cpu"):
    """u(x, y, z) = sin(pi x) sin(pi y) sin(pi z) at cell centres."""
    c = cell_centres(R, n, keys, device)
    return (torch.sin(math.pi * c[..., 0]) * torch.sin(math.pi * c[..., 1]) *
            torch.sin(math.pi * c[..., 2])).reshape(len(keys), -1)


def sin_product_rhs(R, n, keys, device="cpu"):
    """f = -Laplace(u) = 3 pi^2 sin(pi x) sin(pi y) sin(pi z) at cell centres."""
    return 3.0 * math.pi ** 2 * sin_product(R, n, keys, device)


def gaussian_bump_with_noise(R, n, keys, seed=0, center=(0.5, 0.5, 0.5), sigma=0.05, amplitude=1.0,
                             noise=1e-3, device="cpu"):
    """amplitude * exp(-|x - c|^2 / (2 sigma^2)) + U(-noise, noise); one uniform draw per cell in layout order."""
    keys = list(keys)
    rng = np.random.default_rng(seed)
    eta = torch.from_numpy(rng.uniform(-noise, noise, size=len(keys) * n ** 3)).to(device).reshape(len(keys), -1)
    out = torch.empty((len(keys), n ** 3), dtype=F64, device=device)
    cc = torch.tensor(center, dtype=F64, device=device)
    for sl in _chunks(keys, 64):
        c = cell_centres(R, n, keys, device, sl)
        r2 = ((c - cc) ** 2).sum(-1)
        out[sl] = (amplitude * torch.exp(-r2 / (2.0 * sigma ** 2))).reshape(c.shape[0], -1)
    return out + eta


def lognormal_k_rff(R, n, keys, seed=0, sigma=1.0, ell=0.1, features=512, device="cpu", dtype=F64):
    """k = exp(g), g a stationary Gaussian random field with covariance sigma^2 exp(-r^2 / (2 ell^2)).

    g is drawn by random Fourier features, g(x) = sigma sqrt(2/M) sum_m cos(w_m . x + phi_m), with the M
    frequencies w_m ~ N(0, ell^-2 I) drawn first (shape (M, 3)) and the phases phi_m ~ U(0, 2 pi) second.
    It can be evaluated at any point, so refined forests sample the same field.  dtype=torch.float32 evaluates the
    features in single precision (for very large inputs); the returned field is float64 either way.
    """
    keys = list(keys)
    rng = np.random.default_rng(seed)
    w = torch.from_numpy(rng.normal(0.0, 1.0 / ell, size=(features, 3))).to(device)
    phi = torch.from_numpy(rng.uniform(0.0, 2.0 * math.pi, size=features)).to(device)
    wd, phid = w.to(dtype), phi.to(dtype)
    amp = sigma * math.sqrt(2.0 / features)
    out = torch.empty((len(keys), n ** 3), dtype=F64, device=device)
    per = max(1, (1 << 20) // n ** 3)
    for sl in _chunks(keys, per):
        c = cell_centres(R, n, keys, device, sl).reshape(-1, 3).to(dtype)
        g = amp * torch.cos(c @ wd.T + phid).sum(-1)
        out[sl] = torch.exp(g.to(F64)).reshape(-1, n ** 3)
    return out


def uniform_rhs(n_leaves, n, seed=0, lo=-1.0, hi=1.0, device="cpu"):
    """U(lo, hi) per cell, one draw per cell in layout order."""
    rng = np.random.default_rng(seed)
    return torch.from_numpy(rng.uniform(lo, hi, size=(n_leaves, n ** 3))).to(device)


def sin_target(R, n, keys, seed=0, device="cpu"):
    """u_t = sin(m1 pi x) sin(m2 pi y) sin(m3 pi z), with (m1, m2, m3) drawn uniformly from {1, 2, 3}."""
    rng = np.random.default_rng(seed)
    m = rng.integers(1, 4, size=3)
    c = cell_centres(R, n, keys, device)
    return (torch.sin(m[0] * math.pi * c[..., 0]) * torch.sin(m[1] * math.pi * c[..., 1]) *
            torch.sin(m[2] * math.pi * c[..., 2])).reshape(len(list(keys)), -1)


def batch_fields(problems, seed=0, device="cpu", sigma=1.0, ell=0.1):
    """(f, k) of a batch in its flat layout (problems in order, each leaf n^3 cells): per problem p, k is the
    log-normal random-Fourier-feature field with seed `seed + p` (features in FP32) and f ~ U(-1, 1) drawn with
    torch's Philox generator seeded `seed + 100000 + p` on `device`."""
    total = sum(len(keys) * n ** 3 for n, keys in problems)
    f = torch.empty(total, dtype=F64, device=device)
    k = torch.empty(total, dtype=F64, device=device)
    off = 0
    for p, (n, keys) in enumerate(problems):
        cnt = len(keys) * n ** 3
        k[off:off + cnt] = lognormal_k_rff(1, n, keys, seed=seed + p, sigma=sigma, ell=ell, device=device,
                                           dtype=torch.float32).reshape(-1)
        gen = torch.Generator(device=device)
        gen.manual_seed(seed + 100000 + p)
        f[off:off + cnt] = torch.rand(cnt, generator=gen, device=device, dtype=F64) * 2.0 - 1.0
        off += cnt
    return f, k


def boundary_values(R, n, keys, g, device="cpu"):
    """Dirichlet data at the face centres of every leaf face, shape (n_leaves, 6, n^2) float64: face 2 axis + side
    (side 1 the upper face), entry i2 * n + i1 at interior coordinates (i1, i2) along the two other axes in
    increasing axis order.  g is a vectorised function of (x, y, z); faces inside the domain get values too (they
    are ignored by the solver)."""
    keys = list(keys)
    out = np.empty((len(keys), 6, n * n))
    t = (np.arange(n) + 0.5) / n
    for b, (lev, i, j, k) in enumerate(keys):
        ext = 1.0 / (R * 2.0 ** lev)
        org = np.array([i, j, k], dtype=np.float64) * ext
        for axis in range(3):
            t1, t2 = [d for d in range(3) if d != axis]
            i2g, i1g = np.meshgrid(t, t, indexing="ij")  # [i2][i1]
            X = [None, None, None]
            X[t1] = org[t1] + i1g * ext
            X[t2] = org[t2] + i2g * ext
            for side in range(2):
                X[axis] = np.full_like(i1g, org[axis] + side * ext)
                out[b, 2 * axis + side] = np.asarray(g(X[0], X[1], X[2]), dtype=np.float64).reshape(-1)
    return torch.from_numpy(out).to(device)
