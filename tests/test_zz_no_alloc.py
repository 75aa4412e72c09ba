"""mg_exchange_level_noalloc against mg_exchange_level.

The no-allocation variant is for callers that cannot allocate device memory when they need an exchange (inside a
stream capture, with all memory owned by a caching allocator, in allocation-free loops).  It must return exactly
what the allocating entry point returns, on consecutive calls (its static scratch array keeps the previous call's
contents), and refuse levels larger than its fixed scratch.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest
import torch

import synthetic as syn

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _noalloc(F, level, u):
    nb, n = F.levels()[level]
    out = torch.full((nb * (n + 2) ** 3,), float("nan"), dtype=torch.float64, device=u.device)
    st = F.lib.mg_exchange_level_noalloc(F.h, int(level), ctypes.c_void_p(u.data_ptr()),
                                         ctypes.c_void_p(out.data_ptr()))
    return st, out.view(nb, n + 2, n + 2, n + 2)


@pytest.mark.parametrize("coeff,flux", [(False, True), (True, True), (True, False)])
def test_noalloc_exchange_matches_allocating_entry_point(coeff, flux):
    from paper_2403_08063_gb300 import Forest
    R, n, keys = syn.workload_forest("sphere_2x8")
    k = syn.lognormal_k_rff(R, n, keys, seed=51).to(DEV) if coeff else None
    f = syn.gaussian_bump_with_noise(R, n, keys, seed=52).to(DEV)
    F = Forest(R, n, keys, coeff=coeff, interface_flux=flux)
    F.set_rhs(f, k)
    rng = np.random.default_rng(53)
    for level, (nb, nl) in enumerate(F.levels()):
        for call in range(2):  # two calls in a row: the shared scratch must not leak the previous call's values
            u = torch.from_numpy(rng.normal(size=(nb, nl ** 3))).to(DEV)
            want = F.exchange_level(level, u)
            st, got = _noalloc(F, level, u)
            assert st == 0, F.lib.mg_last_error().decode()
            scale = float(want.abs().max())
            assert torch.allclose(got, want, rtol=0.0, atol=1e-13 * scale), (level, call)
    F.close()


def test_noalloc_rejects_levels_beyond_its_scratch():
    from paper_2403_08063_gb300 import Forest
    # 4^3 roots of 32^3: level 0 needs 64 x 39,328 doubles (too many); level 1 (16^3) needs 64 x 5,856 (fits)
    F = Forest(4, 32, syn.uniform_leaves(4))
    F.set_rhs(torch.zeros(64 * 32 ** 3, dtype=torch.float64, device=DEV).view(64, -1))
    u = torch.zeros(64, 32 ** 3, dtype=torch.float64, device=DEV)
    st, _ = _noalloc(F, 0, u)
    assert st == 1
    assert "static scratch" in F.lib.mg_last_error().decode()
    st, got = _noalloc(F, 1, u.view(-1)[: 64 * 16 ** 3].view(64, -1))  # level 1 (16^3 blocks) fits
    assert st == 0
    F.close()
