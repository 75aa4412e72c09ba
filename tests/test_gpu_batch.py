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


def test_batch_tail_modes_give_identical_solves():
    """The three ways of running the coarse levels of a batch -- every level launched, each block-size group's own
    persistent tail, one joint persistent tail per V-cycle over all groups -- run the same device code per step, so
    the solves are bit-identical (iterate, cycle counts and residuals).  Groups of block size 8, 16 and 32 with
    refined problems (interface exchanges inside the tails), FP32 cycles in FP64 defect correction, graph-launched
    steps."""
    from paper_2403_08063_gb300 import Batch
    problems = syn.batch_problems(count=9, seed=7, sizes=(8, 16, 32))
    leaves, ns = syn.batch_leaves(problems)
    rng = np.random.default_rng(8)
    fs, ks = [], []
    for p, (n, keys) in enumerate(problems):
        fs.append(rng.uniform(-1, 1, size=len(keys) * n ** 3))
        ks.append(syn.lognormal_k_rff(1, n, keys, seed=30 + p, sigma=0.5, ell=0.3).numpy().reshape(-1))
    f = torch.from_numpy(np.concatenate(fs)).to(DEV)
    k = torch.from_numpy(np.concatenate(ks)).to(DEV)
    B = Batch(leaves, ns, coeff=True, inner_cycles=4, coarse_coef="faces")
    B.set_rhs(f, k)
    assert B.tail_mode() in (0, 1, 2)
    assert any(lv >= 0 for lv in B.tail_levels()) or B.tail_mode() == 0
    out = {}
    for mode in (0, 1, 2):
        B.set_tail_mode(mode)
        assert B.tail_mode() == mode
        u = torch.zeros_like(f)
        cyc, rel = B.solve(u, rtol=1e-9, max_cycles=60)
        assert max(rel) <= 1e-9
        out[mode] = (u.cpu().numpy(), list(cyc), list(rel))
    for mode in (1, 2):
        assert np.array_equal(out[mode][0], out[0][0]), mode
        assert out[mode][1] == out[0][1] and out[mode][2] == out[0][2], mode
    B.set_tail_mode(2)  # the profiled (launched, not graph-replayed) path of the joint tail counts its launches
    B.profile(True)
    u = torch.zeros_like(f)
    B.solve(u, rtol=1e-9, max_cycles=60)
    prof = B.profile_read()
    B.profile(False)
    assert np.array_equal(u.cpu().numpy(), out[0][0])
    tails = [lv for lv in B.tail_levels() if lv >= 0]
    if tails:
        assert prof.get("tail_f32", (0.0, 0))[1] > 0
    with pytest.raises(Exception):
        B.set_tail_mode(3)
    B.close()


def test_concurrent_groups_give_bit_reproducible_solves():
    """Block-size groups run concurrently on their own streams, so the staged smoothers of one group share SMs with
    the other groups' kernels.  Exactly 10 cycles of the same batch, repeated, must give bit-identical iterates: a
    shared-memory slot refilled by a bulk copy before every read of it had landed made some problems differ at the
    1e-12 level from one solve to the next (and in every problem's FP32 cycles)."""
    from paper_2403_08063_gb300 import Batch, MGError
    problems = [p for p in syn.batch_problems(count=256, seed=0) if p[0] in (16, 32, 64)][:120]
    leaves, ns = syn.batch_leaves(problems)
    f, k = syn.batch_fields(problems, seed=0, device=torch.device(DEV))
    B = Batch(leaves, ns, coeff=True, inner_cycles=5)
    B.set_rhs(f, k)
    outs = []
    for rep in range(3):
        u = torch.zeros_like(f)
        with pytest.raises(MGError):  # rtol 0 is never met: exactly max_cycles cycles
            B.solve(u, rtol=0.0, max_cycles=10)
        outs.append(u.cpu().numpy())
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])
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
