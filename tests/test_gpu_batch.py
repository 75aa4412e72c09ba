"""Several independent problems solved together (one forest per block size, problems sharing it).

Each problem's converged GPU solution is checked against the oracle run on that problem alone: the oracle's own
residual of the GPU solution, and the distance to the oracle's converged solution.
"""
import numpy as np
import pytest
import torch

import synthetic as syn
from oracle.octree_mg import OracleMG

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.mark.parametrize("precision,coeff", [(0, False), (1, True)])
def test_multi_problem_forest_matches_single_problem_oracle(precision, coeff):
    from paper_2403_08063_gb300 import Forest
    problems = syn.batch_problems(count=5, seed=3, sizes=(8,))
    leaves, ns = syn.batch_leaves(problems)
    n = 8
    rng = np.random.default_rng(4)
    fs, ks = [], []
    for p, (_, keys) in enumerate(problems):
        fs.append(rng.uniform(-1, 1, size=(len(keys), n ** 3)))
        ks.append(syn.lognormal_k_rff(1, n, keys, seed=10 + p).numpy() if coeff else None)
    f = torch.from_numpy(np.concatenate(fs)).to(DEV)
    k = torch.from_numpy(np.concatenate(ks)).to(DEV) if coeff else None
    F = Forest(1, n, leaves, coeff=coeff, precision=precision, inner_cycles=3, max_coarse=64)
    assert F.n_problems == 5
    F.set_rhs(f, k)
    u = torch.zeros_like(f)
    cyc, rel = F.solve(u, rtol=1e-11, max_cycles=60)
    assert max(rel) <= 1e-11
    got = u.cpu().numpy()
    off = 0
    for p, (_, keys) in enumerate(problems):
        nb = len(keys)
        ref = OracleMG(1, n, keys, k_user=ks[p], max_coarse=64)
        up = got[off:off + nb]
        assert ref.rel_residual(up, fs[p]) <= 1.05e-11
        u_ref, _ = ref.solve(fs[p], rtol=1e-13, max_cycles=80)
        assert np.linalg.norm(up - u_ref) <= 1e-8 * np.linalg.norm(u_ref)
        off += nb


def test_batch_with_mixed_block_sizes_matches_single_problem_oracle():
    """Problems with block sizes 8 and 16 (refined 0-2 times in random boxes) in one batch, FP32-in-FP64 solves
    captured in CUDA graphs, each to 1e-8 (the batched workload's tolerance), checked per problem by the oracle.

    k is a log-normal field resolved on 8^3 blocks (correlation length 0.3, sigma 0.5): with the workload's
    length 0.1 and sigma 1 an isolated 8^3 root block sees cell-to-cell contrasts near e^8, where averaged coarse
    coefficients make multigrid slow whether the problem is batched or alone (measured: 7e-4 after 30 cycles)."""
    from paper_2403_08063_gb300 import Batch
    problems = syn.batch_problems(count=8, seed=5, sizes=(8, 16))
    leaves, ns = syn.batch_leaves(problems)
    rng = np.random.default_rng(6)
    fs, ks = [], []
    for p, (n, keys) in enumerate(problems):
        fs.append(rng.uniform(-1, 1, size=len(keys) * n ** 3))
        ks.append(syn.lognormal_k_rff(1, n, keys, seed=20 + p, sigma=0.5, ell=0.3).numpy().reshape(-1))
    f = torch.from_numpy(np.concatenate(fs)).to(DEV)
    k = torch.from_numpy(np.concatenate(ks)).to(DEV)
    B = Batch(leaves, ns, coeff=True, inner_cycles=3)
    info = B.info()
    assert sorted(g[0] for g in info["groups"]) == [8, 16] and info["cells"] == f.numel()
    B.set_rhs(f, k)
    u = torch.zeros_like(f)
    for rep in range(2):  # the second solve replays the captured graph from the converged guess
        cyc, rel = B.solve(u, rtol=1e-8, max_cycles=40)
        assert max(rel) <= 1e-8
    got = u.cpu().numpy()
    off = 0
    for p, (n, keys) in enumerate(problems):
        cnt = len(keys) * n ** 3
        ref = OracleMG(1, n, keys, k_user=ks[p].reshape(len(keys), -1), max_coarse=64, operator_only=True)
        assert ref.rel_residual(got[off:off + cnt].reshape(len(keys), -1), fs[p].reshape(len(keys), -1)) <= 1.05e-8
        off += cnt
    B.close()


def test_converged_problems_stop_where_they_would_stop_alone():
    """Per-problem done-mask: once a problem meets rtol its blocks are skipped by every kernel of the later
    defect-correction steps, so the batch returns, for each problem, the iterate and the cycle count of a solve of
    that problem alone (same hierarchy, same inner cycles), although the batch keeps cycling for the slower ones."""
    from paper_2403_08063_gb300 import Batch, Forest
    problems = syn.batch_problems(count=6, seed=11, sizes=(8, 16))
    leaves, ns = syn.batch_leaves(problems)
    rng = np.random.default_rng(12)
    fs, ks = [], []
    for p, (n, keys) in enumerate(problems):
        fs.append(rng.uniform(-1, 1, size=len(keys) * n ** 3))
        sigma = 0.2 if p % 2 else 0.6  # different coefficient contrasts: different cycle counts
        ks.append(syn.lognormal_k_rff(1, n, keys, seed=40 + p, sigma=sigma, ell=0.3).numpy().reshape(-1))
    f = torch.from_numpy(np.concatenate(fs)).to(DEV)
    k = torch.from_numpy(np.concatenate(ks)).to(DEV)
    B = Batch(leaves, ns, coeff=True, inner_cycles=2, max_coarse=64)
    B.set_rhs(f, k)
    u = torch.zeros_like(f)
    cyc, rel = B.solve(u, rtol=1e-9, max_cycles=60)
    assert max(rel) <= 1e-9
    assert len(set(cyc)) > 1, cyc  # the problems converge at different cycles
    off = 0
    for p, (n, keys) in enumerate(problems):
        cnt = len(keys) * n ** 3
        lv = [(0, lev, i, j, kk) for (lev, i, j, kk) in keys]
        F = Forest(1, n, lv, coeff=True, precision=1, inner_cycles=2, max_coarse=64)
        F.set_rhs(f[off:off + cnt].clone(), k[off:off + cnt].clone())
        ua = torch.zeros(cnt, dtype=torch.float64, device=DEV)
        ca, ra = F.solve(ua, rtol=1e-9, max_cycles=60)
        assert ca == cyc[p], (p, ca, cyc[p])
        assert abs(ra - rel[p]) <= 1e-4 * ra  # the squared norm is accumulated in FP32 per thread
        assert torch.allclose(u[off:off + cnt], ua, rtol=0, atol=1e-12 * float(ua.abs().max()))
        F.close()
        off += cnt
    B.close()
