"""Python front end of the C ABI: torch tensors in, device pointers and the current stream out."""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib

F64 = torch.float64


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _host_f64(t, numel, name):
    if not isinstance(t, torch.Tensor) or t.is_cuda or t.dtype != F64:
        raise TypeError(f"{name} must be a CPU float64 tensor")
    if t.numel() != numel or not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous with {numel} elements")
    return t


def _dev_f64(t, numel, name):
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != F64:
        raise TypeError(f"{name} must be a CUDA float64 tensor")
    if t.numel() != numel or not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous with {numel} elements")
    return t


class Forest:
    """A forest of octree blocks with its multigrid hierarchy (wraps mg_forest_create / mg_forest_destroy).

    R: root blocks per axis; n: cells per block edge; leaves: (n_leaves, 5) int32 rows (problem, level, i, j, k)
    or a list of (level, i, j, k) keys.  Fields are (n_leaves, n^3) float64 CUDA tensors in leaf order, x fastest.
    """

    def __init__(self, R, n, leaves, coeff=False, interface_flux=True, precision=0, nu1=2, nu2=2, max_coarse=512,
                 inner_cycles=1, n_problems=None, stream=None, c2f_variant=0, smoother="rbgs", omega=0.8,
                 coarse_iters=0, coarse_coef="k", prolongation="linear"):
        self.lib = _lib.load()
        arr = np.asarray(leaves, dtype=np.int32)
        if arr.ndim == 2 and arr.shape[1] == 4:
            arr = np.concatenate([np.zeros((arr.shape[0], 1), np.int32), arr], axis=1)
        self._leaves = np.ascontiguousarray(arr, dtype=np.int32)
        self.R, self.n, self.n_leaves = int(R), int(n), int(self._leaves.shape[0])
        self.coeff = bool(coeff)
        self.precision = int(precision)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        cfg = _lib.MGConfig()
        cfg.roots, cfg.n, cfg.n_leaves = self.R, self.n, self.n_leaves
        cfg.leaves = self._leaves.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        cfg.coeff, cfg.interface_flux, cfg.precision = int(coeff), int(interface_flux), int(precision)
        cfg.nu1, cfg.nu2, cfg.max_coarse = int(nu1), int(nu2), int(max_coarse)
        cfg.inner_cycles = int(inner_cycles)
        cfg.c2f_variant = int(c2f_variant)
        cfg.smoother = {"rbgs": 0, "jacobi": 1}[smoother]
        cfg.omega = float(omega)
        cfg.coarse_iters = int(coarse_iters)
        cfg.coarse_coef = {"k": 0, "faces": 1}[coarse_coef]
        cfg.prolongation = {"linear": 0, "trilinear": 1}[prolongation]
        self.n_problems = int(n_problems) if n_problems else int(self._leaves[:, 0].max()) + 1
        cfg.n_problems = self.n_problems
        cfg.stream = ctypes.c_void_p(self.stream.cuda_stream)
        h = ctypes.c_void_p()
        _lib.check(self.lib.mg_forest_create(ctypes.byref(cfg), ctypes.byref(h)))
        self.h = h
        self.numel = self.n_leaves * self.n ** 3
        self.version = 0  # bumped by set_rhs; the autograd function re-sets (f, k) if it changed

    # -- lifetime ----------------------------------------------------------------------------------------
    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.lib.mg_forest_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- structure ---------------------------------------------------------------------------------------
    def levels(self):
        nl = ctypes.c_int32()
        _lib.check(self.lib.mg_forest_levels(self.h, ctypes.byref(nl), None, None))
        nb = (ctypes.c_int32 * nl.value)()
        nn = (ctypes.c_int32 * nl.value)()
        _lib.check(self.lib.mg_forest_levels(self.h, ctypes.byref(nl), nb, nn))
        return [(nb[i], nn[i]) for i in range(nl.value)]

    def level_keys(self, level):
        nb = self.levels()[level][0]
        keys = np.zeros((nb, 4), dtype=np.int32)
        _lib.check(self.lib.mg_level_keys(self.h, level, keys.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))))
        return [tuple(int(v) for v in r) for r in keys]

    # -- solver ------------------------------------------------------------------------------------------
    def set_rhs(self, f, k=None):
        _dev_f64(f, self.numel, "f")
        if self.coeff:
            _dev_f64(k, self.numel, "k")
        _lib.check(self.lib.mg_set_rhs(self.h, _ptr(f), _ptr(k) if self.coeff else None))
        self.version += 1

    def set_boundary(self, g=None):
        """Dirichlet data on the finest level's boundary faces: g of shape (n_leaves, 6, n^2) (face 2 axis + side,
        index i2 * n + i1 along the two other axes in increasing order), or None for g = 0."""
        if g is None:
            _lib.check(self.lib.mg_set_boundary(self.h, None))
            self._g = None
            return
        _dev_f64(g, self.n_leaves * 6 * self.n ** 2, "g")
        self._g = g
        _lib.check(self.lib.mg_set_boundary(self.h, _ptr(g)))

    def vcycle(self, u, ncycles=1):
        """ncycles V-cycles on u in place; returns the relative residual (a list with several problems)."""
        _dev_f64(u, self.numel, "u")
        rel = (ctypes.c_double * self.n_problems)()
        _lib.check(self.lib.mg_vcycle(self.h, _ptr(u), int(ncycles), rel))
        return rel[0] if self.n_problems == 1 else list(rel)

    def solve(self, u, rtol=1e-10, max_cycles=100, raise_on_failure=True):
        """Cycle on u (initial guess in place) until ||f - A u|| / ||f|| <= rtol for every problem.

        Returns (cycles, rel), or (list of cycles, list of rel) with several problems."""
        _dev_f64(u, self.numel, "u")
        cyc = (ctypes.c_int32 * self.n_problems)()
        rel = (ctypes.c_double * self.n_problems)()
        st = self.lib.mg_solve(self.h, _ptr(u), float(rtol), int(max_cycles), cyc, rel)
        if st != 0 and (raise_on_failure or st != 6):
            _lib.check(st)
        if self.n_problems == 1:
            return cyc[0], rel[0]
        return list(cyc), list(rel)

    def solve_host(self, f, k=None, u=None, u0=None, rtol=1e-10, max_cycles=100, raise_on_failure=True):
        """mg_set_rhs + mg_solve from CPU float64 tensors (page-locked ones give the fastest copies): f, k (coeff),
        u0 the initial guess (None: zero); the solution is written into u (allocated when None, may be u0).

        Returns (u, cycles, rel), with lists of cycles and rel for several problems."""
        _host_f64(f, self.numel, "f")
        if k is not None:
            _host_f64(k, self.numel, "k")
        if u0 is not None:
            _host_f64(u0, self.numel, "u0")
        if u is None:
            u = torch.empty_like(f)
        _host_f64(u, self.numel, "u")
        cyc = (ctypes.c_int32 * self.n_problems)()
        rel = (ctypes.c_double * self.n_problems)()
        st = self.lib.mg_solve_host(self.h, _ptr(f), _ptr(k), _ptr(u0), _ptr(u), float(rtol), int(max_cycles), cyc,
                                    rel)
        if st != 0 and (raise_on_failure or st != 6):
            _lib.check(st)
        if self.n_problems == 1:
            return u, cyc[0], rel[0]
        return u, list(cyc), list(rel)

    def apply(self, u):
        _dev_f64(u, self.numel, "u")
        out = torch.empty_like(u)
        _lib.check(self.lib.mg_apply(self.h, _ptr(u), _ptr(out)))
        return out

    def apply_transpose(self, y):
        _dev_f64(y, self.numel, "y")
        out = torch.empty_like(y)
        _lib.check(self.lib.mg_apply_transpose(self.h, _ptr(y), _ptr(out)))
        return out

    def adjoint(self, u, dLdu, want_k=True, rtol=1e-12, max_cycles=100):
        """lambda = A^-T dL/du (= dL/df) and, for coeff problems, dL/dk.  Returns (lambda, dLdk or None)."""
        _dev_f64(u, self.numel, "u")
        _dev_f64(dLdu, self.numel, "dLdu")
        lam = torch.empty_like(u)
        gk = torch.empty_like(u) if (want_k and self.coeff) else None
        _lib.check(self.lib.mg_adjoint_solve(self.h, _ptr(u), _ptr(dLdu), _ptr(lam), _ptr(gk), float(rtol),
                                             int(max_cycles)))
        return lam, gk

    def exchange_level(self, level, u):
        nb, n = self.levels()[level]
        _dev_f64(u, nb * n ** 3, "u")
        out = torch.empty(nb * (n + 2) ** 3, dtype=F64, device=u.device)
        _lib.check(self.lib.mg_exchange_level(self.h, int(level), _ptr(u), _ptr(out)))
        return out.view(nb, n + 2, n + 2, n + 2)

    def tail_level(self):
        """Level from which the persistent tail kernel runs the FP32 V-cycle (-1: off)."""
        lv = ctypes.c_int32()
        _lib.check(self.lib.mg_get_tail(self.h, ctypes.byref(lv)))
        return lv.value

    def set_tail(self, level):
        _lib.check(self.lib.mg_set_tail(self.h, int(level)))

    def smoother_shapes(self, level):
        """The FP32 smoother launch shapes offered on `level` (5-tuples; empty where it is not used)."""
        cnt = ctypes.c_int32()
        _lib.check(self.lib.mg_smoother_shapes(self.h, int(level), 0, None, ctypes.byref(cnt)))
        buf = (ctypes.c_int32 * (5 * max(1, cnt.value)))()
        _lib.check(self.lib.mg_smoother_shapes(self.h, int(level), cnt.value, buf, ctypes.byref(cnt)))
        return [tuple(buf[5 * i:5 * i + 5]) for i in range(cnt.value)]

    def smoother_shape(self, level):
        """The FP32 smoother launch shape of `level`; (0, 0, 0, 0, 0) where it is not used."""
        buf = (ctypes.c_int32 * 5)()
        _lib.check(self.lib.mg_get_smoother_shape(self.h, int(level), buf))
        return tuple(buf)

    def set_smoother_shape(self, level, shape):
        buf = (ctypes.c_int32 * 5)(*[int(v) for v in shape])
        _lib.check(self.lib.mg_set_smoother_shape(self.h, int(level), buf))

    # -- accounting --------------------------------------------------------------------------------------
    def profile(self, enable=True):
        _lib.check(self.lib.mg_profile(self.h, int(bool(enable))))

    def profile_read(self):
        """{family: (milliseconds, launches)} of the kernel families since the last profile(True)."""
        return _profile_read_handle(self.lib, self.h)


class Batch:
    """Independent problems with per-problem block sizes solved together (wraps mg_batch_*).

    leaves: (n_leaves, 5) int32 rows (problem, level, i, j, k); problem_n: block size per problem.  Fields are flat
    float64 CUDA tensors: the leaves in order, each with its problem's n^3 cells, x fastest.
    """

    def __init__(self, leaves, problem_n, R=1, coeff=True, interface_flux=True, inner_cycles=3, nu1=2, nu2=2,
                 max_coarse=64, stream=None, coarse_coef="k", prolongation="linear"):
        self.lib = _lib.load()
        self._leaves = np.ascontiguousarray(np.asarray(leaves, dtype=np.int32))
        self._pn = np.ascontiguousarray(np.asarray(problem_n, dtype=np.int32))
        self.n_problems = int(self._pn.shape[0])
        self.coeff = bool(coeff)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        cfg = _lib.MGConfig()
        cfg.roots, cfg.n, cfg.n_leaves = int(R), int(self._pn[0]), int(self._leaves.shape[0])
        cfg.leaves = self._leaves.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        cfg.coeff, cfg.interface_flux, cfg.precision = int(coeff), int(interface_flux), 1
        cfg.nu1, cfg.nu2, cfg.max_coarse, cfg.inner_cycles = int(nu1), int(nu2), int(max_coarse), int(inner_cycles)
        cfg.coarse_coef = {"k": 0, "faces": 1}[coarse_coef]
        cfg.prolongation = {"linear": 0, "trilinear": 1}[prolongation]
        cfg.n_problems = self.n_problems
        cfg.stream = ctypes.c_void_p(self.stream.cuda_stream)
        h = ctypes.c_void_p()
        _lib.check(self.lib.mg_batch_create(ctypes.byref(cfg), self._pn.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                            ctypes.byref(h)))
        self.h = h
        self.numel = int(sum(int(self._pn[p]) ** 3 for p in self._leaves[:, 0]))

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.lib.mg_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self):
        ng = ctypes.c_int32()
        tot = ctypes.c_int64()
        _lib.check(self.lib.mg_batch_info(self.h, ctypes.byref(ng), ctypes.byref(tot), None, None))
        gn = (ctypes.c_int32 * ng.value)()
        gp = (ctypes.c_int32 * ng.value)()
        _lib.check(self.lib.mg_batch_info(self.h, ctypes.byref(ng), ctypes.byref(tot), gn, gp))
        return {"groups": [(gn[i], gp[i]) for i in range(ng.value)], "cells": tot.value}

    def set_rhs(self, f, k=None):
        _dev_f64(f, self.numel, "f")
        if self.coeff:
            _dev_f64(k, self.numel, "k")
        _lib.check(self.lib.mg_batch_set_rhs(self.h, _ptr(f), _ptr(k) if self.coeff else None))

    def solve(self, u, rtol=1e-8, max_cycles=100, raise_on_failure=True):
        """Cycle on u in place until every problem meets rtol; returns (cycles per problem, rel per problem)."""
        _dev_f64(u, self.numel, "u")
        cyc = (ctypes.c_int32 * self.n_problems)()
        rel = (ctypes.c_double * self.n_problems)()
        st = self.lib.mg_batch_solve(self.h, _ptr(u), float(rtol), int(max_cycles), cyc, rel)
        if st != 0 and (raise_on_failure or st != 6):
            _lib.check(st)
        return list(cyc), list(rel)

    def tail_levels(self):
        """Per group, the level from which its persistent tail kernel runs the FP32 V-cycle (-1: off)."""
        out = []
        for g in range(len(self.info()["groups"])):
            lv = ctypes.c_int32()
            _lib.check(self.lib.mg_get_tail(ctypes.c_void_p(self.lib.mg_batch_group(self.h, g)), ctypes.byref(lv)))
            out.append(lv.value)
        return out

    def set_tail_off(self):
        """Runs every group's FP32 V-cycle as separate launches (no persistent tail)."""
        self.set_tail_mode(0)

    def tail_mode(self):
        """0: every level launched; 1: each group's own persistent tail; 2: one joint persistent tail per V-cycle."""
        m = ctypes.c_int32()
        _lib.check(self.lib.mg_batch_get_tail_mode(self.h, ctypes.byref(m)))
        return m.value

    def set_tail_mode(self, mode):
        """Overrides the tuned tail mode (see tail_mode); after set_rhs."""
        _lib.check(self.lib.mg_batch_set_tail_mode(self.h, int(mode)))

    def profile(self, enable=True):
        _lib.check(self.lib.mg_batch_profile(self.h, int(bool(enable))))

    def profile_read(self):
        """Per kernel family (milliseconds, launches), summed over the groups (the group forests stay owned by
        the batch: they are read through their handles, never wrapped in a Forest that would destroy them)."""
        out = {}
        for g in range(len(self.info()["groups"])):
            fh = ctypes.c_void_p(self.lib.mg_batch_group(self.h, g))
            for k, (ms, n) in _profile_read_handle(self.lib, fh).items():
                a = out.get(k, (0.0, 0))
                out[k] = (a[0] + ms, a[1] + n)
        return out


def alu_peaks():
    """Measured FMA throughput of the current device, (FP64, FP32) in TFLOP/s (mg_alu_peaks; synchronises it)."""
    lib = _lib.load()
    a, b = ctypes.c_double(), ctypes.c_double()
    _lib.check(lib.mg_alu_peaks(ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def _profile_read_handle(lib, h):
    nf = ctypes.c_int32()
    _lib.check(lib.mg_profile_read(h, 0, None, None, None, ctypes.byref(nf)))
    m = nf.value
    names = ctypes.create_string_buffer(32 * m)
    ms = (ctypes.c_double * m)()
    cnt = (ctypes.c_int64 * m)()
    _lib.check(lib.mg_profile_read(h, m, names, ms, cnt, ctypes.byref(nf)))
    out = {}
    for i in range(m):
        nm = names.raw[32 * i:32 * (i + 1)].split(b"\0")[0].decode()
        out[nm] = (ms[i], int(cnt[i]))
    return out


class MGSolveFn(torch.autograd.Function):
    """u = A(k)^-1 f through the forest's multigrid solve, differentiable in f and k.

    backward re-runs multigrid on the transposed operator (mg_adjoint_solve): lambda = A^-T grad_u is dL/df and
    dL/dk = -lambda^T (dA/dk) u.  The checkpointed forward state is u itself plus the forest's set-up hierarchy
    (coefficient pyramid, coarsest inverse); if the forest was re-used with other inputs in between, backward
    restores (f, k) first.  Usage: u = MGSolveFn.apply(f, k, forest, rtol, max_cycles) (k may be None).
    """

    @staticmethod
    def forward(ctx, f, k, forest, rtol=1e-10, max_cycles=100):
        fd = f.detach().contiguous()
        kd = k.detach().contiguous() if k is not None else None
        forest.set_rhs(fd, kd)
        u = torch.zeros_like(fd)
        forest.solve(u, rtol=rtol, max_cycles=max_cycles)
        ctx.forest, ctx.version, ctx.rtol, ctx.max_cycles = forest, forest.version, rtol, max_cycles
        ctx.save_for_backward(u, fd, kd if kd is not None else torch.empty(0, device=fd.device))
        ctx.has_k = kd is not None
        return u

    @staticmethod
    def backward(ctx, grad_u):
        u, fd, kd = ctx.saved_tensors
        forest = ctx.forest
        if forest.version != ctx.version:
            forest.set_rhs(fd, kd if ctx.has_k else None)
        want_k = ctx.has_k and ctx.needs_input_grad[1]
        lam, gk = forest.adjoint(u, grad_u.contiguous().to(torch.float64), want_k=want_k,
                                 rtol=min(ctx.rtol, 1e-10), max_cycles=max(ctx.max_cycles, 100))
        return lam, gk, None, None, None
