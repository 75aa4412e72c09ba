"""mg_exchange_level_noalloc against mg_exchange_level.

The no-allocation variant is for callers that cannot let a library allocate device memory when they need an
exchange (all device memory owned by a caching allocator or reserved at start-up, loops that must not enter CUDA's
allocator).  It must return exactly
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


def _noalloc(F, level, u, out=None):
    nb, n = F.levels()[level]
    if out is None:
        out = torch.full((nb * (n + 2) ** 3,), float("nan"), dtype=torch.float64, device=u.device)
    else:
        out.fill_(float("nan"))
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


def test_noalloc_never_allocates_on_fp32_cycle_forests():
    """A variable-k forest with FP32 cycles (the mixed-precision configuration) keeps FP64 face coefficients only on
    its finest level (the FP64 outer residual) and its coarsest; the intermediate levels get them when an FP64 path
    first needs them, and creating them allocates.  The no-allocation entry point must not do that: on level 0 it
    works at once, on level 1 (which has conservative fine-to-coarse ghosts) it returns MG_ERR_STATE until an
    allocating call has created the coefficients, and the device's free memory never changes across its calls.
    Each level's result matches mg_exchange_level on two calls in a row."""
    from paper_2403_08063_gb300 import Forest
    from oracle.octree_mg import OracleMG
    R, n, keys = syn.workload_forest("sphere_2x8")
    k = syn.lognormal_k_rff(R, n, keys, seed=61).to(DEV)
    f = syn.gaussian_bump_with_noise(R, n, keys, seed=62).to(DEV)
    F = Forest(R, n, keys, coeff=True, interface_flux=True, precision=1)
    F.set_rhs(f, k)
    levels = F.levels()
    assert len(levels) > 2 and any(fc[0] == "f2c" for b in OracleMG(R, n, keys).levels[1].faces for fc in b)
    rng = np.random.default_rng(63)
    us = [torch.from_numpy(rng.normal(size=(nb, nl ** 3))).to(DEV) for nb, nl in levels[:2]]
    outs = [[torch.empty(nb * (nl + 2) ** 3, dtype=torch.float64, device=DEV) for _ in range(2)]
            for nb, nl in levels[:2]]  # allocated before measuring: one output per call
    # the first call in a process loads the library's device code with its static array (CUDA loads modules
    # lazily); that happens before the measurement
    assert _noalloc(F, 0, us[0], outs[0][0])[0] == 0, F.lib.mg_last_error().decode()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    st0 = [_noalloc(F, 0, us[0], o)[0] for o in outs[0]]
    st1 = _noalloc(F, 1, us[1], outs[1][0])[0]
    msg1 = F.lib.mg_last_error().decode()
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] >= free0 - (1 << 20)
    assert st0 == [0, 0], F.lib.mg_last_error().decode()
    assert st1 == 9 and "face coefficients" in msg1, (st1, msg1)  # MG_ERR_STATE
    wants = [F.exchange_level(l, us[l]) for l in range(2)]  # allocating entry point: creates the coefficients
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    st1 = [_noalloc(F, 1, us[1], o)[0] for o in outs[1]]
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] >= free1 - (1 << 20)
    assert st1 == [0, 0], F.lib.mg_last_error().decode()
    for l in range(2):
        scale = float(wants[l].abs().max())
        for call, o in enumerate(outs[l]):
            got = o.view_as(wants[l])
            assert torch.allclose(got, wants[l], rtol=0.0, atol=1e-13 * scale), (l, call)
    F.close()
