"""PyTorch-facing wrapper of the C ABI: a ``Plan`` holding a native plan,
and autograd Functions whose backward calls the native adjoints.

PyTorch supplies device memory and the current CUDA stream; every step of
every transform runs in the library's kernels.
"""
import ctypes

import torch

from . import _native
from ._native import PRECISION, SHTError, check, lib


def _stream_ptr(device):
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


class Plan:
    """Spherical-harmonic transform plan on the J x I Clenshaw-Curtis grid
    (``grid="cc"``), on the shifted grid of Fejer's first rule
    (``grid="fejer1"``, Sec. 3.3), or on a reduced Clenshaw-Curtis grid
    (``grid="reduced"``) with ``lat_points[j]`` longitudes on latitude j
    (I is then ignored; see ``reduced_grid_sizes``).

    Layouts: grid ``[nfields, J, I]`` real (reduced: ``[nfields, sum of
    lat_points]``, rows packed); spectrum ``[ncoef, nfields]`` complex
    (packed m-major, m >= 0 only).  ``precision`` is one of "fp64",
    "bf16x2", "bf16x3", "fp16x2", "fp16x3"; FP64 plans use float64/complex128
    tensors, split plans float32/complex64."""

    def __init__(self, N, J, I, nfields, precision="fp64", device=None, grid="cc",
                 lat_points=None, half_shift=None):
        if precision not in PRECISION:
            raise ValueError("precision must be one of %s" % list(PRECISION))
        if grid not in _native.GRID and grid != "reduced":
            raise ValueError("grid must be one of %s" % (list(_native.GRID) + ["reduced"]))
        if (grid == "reduced") != (lat_points is not None):
            raise ValueError("lat_points goes with grid='reduced' and only with it")
        if half_shift is not None and grid != "reduced":
            raise ValueError("half_shift goes with grid='reduced'")
        self.grid = grid
        self.device = torch.device("cuda", torch.cuda.current_device()
                                   if device is None else torch.device(device).index or 0)
        self.N, self.J, self.I, self.F = N, J, I, nfields
        self.precision = precision
        self.real_dtype = torch.float64 if precision == "fp64" else torch.float32
        self.complex_dtype = torch.complex128 if precision == "fp64" else torch.complex64
        self.ncoef = (N + 1) * (N + 2) // 2
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            if grid == "reduced":
                pts = [int(v) for v in lat_points]
                if len(pts) != J:
                    raise ValueError("lat_points needs J = %d entries" % J)
                arr = (ctypes.c_int * J)(*pts)
                if half_shift is None:
                    rc = check(lib.sht_plan_create_reduced(N, J, arr, nfields,
                                                           PRECISION[precision],
                                                           ctypes.byref(h)))
                else:
                    sh = [int(v) for v in half_shift]
                    if len(sh) != J:
                        raise ValueError("half_shift needs J = %d entries" % J)
                    rc = check(lib.sht_plan_create_reduced_shifted(
                        N, J, arr, (ctypes.c_int * J)(*sh), nfields, PRECISION[precision],
                        ctypes.byref(h)))
                self.half_shift = None if half_shift is None else [int(v) for v in half_shift]
                self.lat_points = pts
                self.I = max(pts)
            else:
                rc = check(lib.sht_plan_create_grid(N, J, I, nfields, PRECISION[precision],
                                                    _native.GRID[grid], ctypes.byref(h)))
                self.lat_points = None
                self.half_shift = None
        self.exact = rc == _native.SHT_OK
        self._h = h
        npts = ctypes.c_longlong()
        check(lib.sht_plan_grid_points(h, ctypes.byref(npts)))
        self.npts = npts.value
        self.grid_shape = ((self.F, self.npts) if grid == "reduced"
                           else (self.F, self.J, self.I))

    # -- buffers ----------------------------------------------------------
    def _check(self, t, shape, dtype, name):
        if not isinstance(t, torch.Tensor) or t.device != self.device:
            raise ValueError("%s must be a tensor on %s" % (name, self.device))
        if tuple(t.shape) != tuple(shape) or t.dtype != dtype:
            raise ValueError("%s must be %s %s, got %s %s" % (
                name, dtype, tuple(shape), t.dtype, tuple(t.shape)))
        if not t.is_contiguous():
            raise ValueError("%s must be contiguous" % name)

    def empty_grid(self):
        return torch.empty(self.grid_shape, dtype=self.real_dtype, device=self.device)

    def empty_spec(self):
        return torch.empty((self.ncoef, self.F), dtype=self.complex_dtype,
                           device=self.device)

    # -- transforms -----------------------------------------------------------
    def forward(self, grid, out=None):
        """Analysis: grid (``grid_shape``) -> spectrum [ncoef, F]."""
        self._check(grid, self.grid_shape, self.real_dtype, "grid")
        out = self.empty_spec() if out is None else out
        self._check(out, (self.ncoef, self.F), self.complex_dtype, "spec")
        check(lib.sht_forward(self._h, ctypes.c_void_p(grid.data_ptr()),
                              ctypes.c_void_p(out.data_ptr()),
                              _stream_ptr(self.device)))
        return out

    def inverse(self, spec, out=None):
        """Synthesis: spectrum [ncoef, F] -> grid (``grid_shape``)."""
        self._check(spec, (self.ncoef, self.F), self.complex_dtype, "spec")
        out = self.empty_grid() if out is None else out
        self._check(out, self.grid_shape, self.real_dtype, "grid")
        check(lib.sht_inverse(self._h, ctypes.c_void_p(spec.data_ptr()),
                              ctypes.c_void_p(out.data_ptr()),
                              _stream_ptr(self.device)))
        return out

    def adjoint(self, which, x, out=None):
        """which=0: adjoint of forward (spectrum -> grid);
        which=1: adjoint of inverse (grid -> spectrum)."""
        if which == 0:
            self._check(x, (self.ncoef, self.F), self.complex_dtype, "spec")
            out = self.empty_grid() if out is None else out
            self._check(out, self.grid_shape, self.real_dtype, "grid")
        elif which == 1:
            self._check(x, self.grid_shape, self.real_dtype, "grid")
            out = self.empty_spec() if out is None else out
            self._check(out, (self.ncoef, self.F), self.complex_dtype, "spec")
        else:
            raise ValueError("which must be 0 or 1")
        check(lib.sht_adjoint(self._h, which, ctypes.c_void_p(x.data_ptr()),
                              ctypes.c_void_p(out.data_ptr()),
                              _stream_ptr(self.device)))
        return out

    def alias_products(self, spec_u, spec_v, spec_w, grids=None, out=None):
        """Quadratic and cubic terms of the aliasing experiment (Sec. 4.2):
        the analyses of U V and U V W, with U, V, W synthesised from their
        spectra on this plan's grid.  ``grids``: two work grids (returned
        holding U V and U V W); ``out``: two spectra.  Returns (spec_q,
        spec_c)."""
        for t, nm in ((spec_u, "spec_u"), (spec_v, "spec_v"), (spec_w, "spec_w")):
            self._check(t, (self.ncoef, self.F), self.complex_dtype, nm)
        grids = [self.empty_grid(), self.empty_grid()] if grids is None else grids
        out = [self.empty_spec(), self.empty_spec()] if out is None else out
        for g in grids:
            self._check(g, self.grid_shape, self.real_dtype, "grid")
        for o in out:
            self._check(o, (self.ncoef, self.F), self.complex_dtype, "spec")
        ptr = lambda t: ctypes.c_void_p(t.data_ptr())
        check(lib.sht_alias_products(self._h, ptr(spec_u), ptr(spec_v), ptr(spec_w),
                                     ptr(grids[0]), ptr(grids[1]), ptr(out[0]),
                                     ptr(out[1]), _stream_ptr(self.device)))
        return out[0], out[1]

    def restrict_nested(self, fine_grid, k, out=None):
        """Coarse spectrum of a fine grid with J_f = 2^k (J+1) - 1, I_f = 2^k I."""
        Jf, If = 2 ** k * (self.J + 1) - 1, 2 ** k * self.I
        self._check(fine_grid, (self.F, Jf, If), self.real_dtype, "fine_grid")
        out = self.empty_spec() if out is None else out
        self._check(out, (self.ncoef, self.F), self.complex_dtype, "spec")
        check(lib.sht_restrict_nested(self._h, ctypes.c_void_p(fine_grid.data_ptr()),
                                      k, ctypes.c_void_p(out.data_ptr()),
                                      _stream_ptr(self.device)))
        return out

    def prolong_spectral(self, coarse_spec, Nc, out=None, add=False):
        """Grid of a spectrum truncated at Nc <= N, zero-padded to this plan's
        N (multigrid prolongation in spectral space, Appendix C).  With
        add=True the grid is added onto ``out`` (required), the V-cycle's
        correction step."""
        self._check(coarse_spec, ((Nc + 1) * (Nc + 2) // 2, self.F), self.complex_dtype,
                    "coarse_spec")
        if add and out is None:
            raise ValueError("add=True needs the grid to add onto (out)")
        out = self.empty_grid() if out is None else out
        self._check(out, self.grid_shape, self.real_dtype, "grid")
        fn = lib.sht_prolong_spectral_add if add else lib.sht_prolong_spectral
        check(fn(self._h, ctypes.c_void_p(coarse_spec.data_ptr()), Nc,
                 ctypes.c_void_p(out.data_ptr()), _stream_ptr(self.device)))
        return out

    def inject_nested(self, fine_grid, k, out=None):
        """This plan's grid sampled from a nested fine grid (every 2^k-th
        latitude and longitude: restriction by injection, Appendix C)."""
        Jf, If = 2 ** k * (self.J + 1) - 1, 2 ** k * self.I
        self._check(fine_grid, (self.F, Jf, If), self.real_dtype, "fine_grid")
        out = self.empty_grid() if out is None else out
        self._check(out, self.grid_shape, self.real_dtype, "grid")
        check(lib.sht_inject_nested(self._h, ctypes.c_void_p(fine_grid.data_ptr()), k,
                                    ctypes.c_void_p(out.data_ptr()),
                                    _stream_ptr(self.device)))
        return out

    def reduced_grid_sizes(self, rule="smooth"):
        """Longitudes per latitude (J ints) of the reduced grid that the
        1e-16 reduction rule of Sec. 6 gives on this plan's latitudes, capped
        at its I.  ``rule``: "smooth" (any even 2-3-5-smooth count) or "fast"
        (counts with compile-time FFT kernels); see ``sht_reduced_grid_sizes``."""
        if rule not in _native.REDUCED_RULE:
            raise ValueError("rule must be one of %s" % list(_native.REDUCED_RULE))
        out = (ctypes.c_int * self.J)()
        check(lib.sht_reduced_grid_sizes(self._h, _native.REDUCED_RULE[rule], out))
        return list(out)

    def tables(self):
        """(w [J], mu [J], pnm [ncoef, (J+1)/2]) copied from the device."""
        import numpy as np
        Jh = (self.J + 1) // 2
        w = np.empty(self.J)
        mu = np.empty(self.J)
        pnm = np.empty((self.ncoef, Jh))
        dp = ctypes.POINTER(ctypes.c_double)
        check(lib.sht_plan_copy_tables(self._h, w.ctypes.data_as(dp),
                                       mu.ctypes.data_as(dp), pnm.ctypes.data_as(dp)))
        return w, mu, pnm

    def status(self):
        """Synchronise; raise SHTError if a kernel of this plan gave up on a
        bounded wait since the last check."""
        check(lib.sht_plan_status(self._h))

    # -- launch shapes ----------------------------------------------------
    @property
    def tuning(self):
        """{"fields_per_cta": G, "tile_width": TN} (TN is 0 for FP64 plans)."""
        g, t = ctypes.c_int(), ctypes.c_int()
        check(lib.sht_plan_get_tuning(self._h, ctypes.byref(g), ctypes.byref(t)))
        return {"fields_per_cta": g.value, "tile_width": t.value}

    def set_tuning(self, fields_per_cta=0, tile_width=0):
        """Set the FFT fields per CTA and/or the split GEMM tile width (64 or
        128); 0 leaves a shape unchanged.  Results do not depend on either."""
        with torch.cuda.device(self.device):
            check(lib.sht_plan_set_tuning(self._h, int(fields_per_cta), int(tile_width)))

    def set_reduced(self, on=True):
        """Reduced transform (Sec. 4.1): neglect |P~| < 1e-16, per tile."""
        with torch.cuda.device(self.device):
            check(lib.sht_plan_set_reduced(self._h, 1 if on else 0))

    def autotune(self, reps=3):
        """Time the candidate launch shapes on this plan and keep the fastest;
        returns the choice and the mean ms of an inverse + forward pair."""
        g, t, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_float()
        with torch.cuda.device(self.device):
            check(lib.sht_plan_autotune(self._h, int(reps), _stream_ptr(self.device),
                                        ctypes.byref(g), ctypes.byref(t), ctypes.byref(ms)))
        return {"fields_per_cta": g.value, "tile_width": t.value,
                "ms_per_pair": ms.value}

    def profile(self, on=True):
        """Turn per-launch event timing on or off."""
        check(lib.sht_profile_enable(self._h, 1 if on else 0))

    def profile_read(self, kernels=False):
        """{stage: (total_ms, runs)} since the last read (synchronises); with
        kernels=True {stage: (total_ms, runs, kernels launched)}."""
        ms = (ctypes.c_double * _native.PROFILE_STAGES)()
        n = (ctypes.c_longlong * _native.PROFILE_STAGES)()
        kn = (ctypes.c_longlong * _native.PROFILE_STAGES)()
        check(lib.sht_profile_read_kernels(self._h, ms, n, kn))
        return {_native.STAGE_NAMES[k]: ((ms[k], n[k], kn[k]) if kernels else (ms[k], n[k]))
                for k in range(_native.PROFILE_STAGES) if n[k]}

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib.sht_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Group:
    """Several plans transformed by one launch per kernel stage.

    ``forward(grids)`` / ``inverse(specs)`` take and return lists with one
    tensor per plan (each plan's own layouts).  The plans must outlive the
    group."""

    def __init__(self, plans):
        plans = list(plans)
        if not 1 <= len(plans) <= 8:
            raise ValueError("a group holds 1..8 plans")
        self.plans = plans
        arr = (ctypes.c_void_p * len(plans))(*[p._h.value for p in plans])
        h = ctypes.c_void_p()
        with torch.cuda.device(plans[0].device):
            check(lib.sht_group_create(arr, len(plans), ctypes.byref(h)))
        self._h = h

    def _ptrs(self, ts):
        return (ctypes.c_void_p * len(ts))(*[t.data_ptr() for t in ts])

    def forward(self, grids, out=None):
        if len(grids) != len(self.plans):
            raise ValueError("one grid per plan")
        out = [p.empty_spec() for p in self.plans] if out is None else out
        for p, g, o in zip(self.plans, grids, out):
            p._check(g, (p.F, p.J, p.I), p.real_dtype, "grid")
            p._check(o, (p.ncoef, p.F), p.complex_dtype, "spec")
        check(lib.sht_group_forward(self._h, self._ptrs(grids), self._ptrs(out),
                                    _stream_ptr(self.plans[0].device)))
        return out

    def inverse(self, specs, out=None):
        if len(specs) != len(self.plans):
            raise ValueError("one spectrum per plan")
        out = [p.empty_grid() for p in self.plans] if out is None else out
        for p, a, o in zip(self.plans, specs, out):
            p._check(a, (p.ncoef, p.F), p.complex_dtype, "spec")
            p._check(o, (p.F, p.J, p.I), p.real_dtype, "grid")
        check(lib.sht_group_inverse(self._h, self._ptrs(specs), self._ptrs(out),
                                    _stream_ptr(self.plans[0].device)))
        return out

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib.sht_group_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def octahedral_grid_sizes(J, first=20, step=4):
    """Longitudes per latitude of the octahedral Clenshaw-Curtis grid
    (Sec. 6): first + step (j - 1) on the j-th latitude from either pole."""
    out = (ctypes.c_int * J)()
    check(lib.sht_octahedral_grid_sizes(J, first, step, out))
    return list(out)


def icositetrahedral_grid_sizes(J):
    """(longitudes per latitude, half-spacing shift per latitude) of the
    icositetrahedral Clenshaw-Curtis grid (Sec. 6), for
    ``Plan(..., grid="reduced", lat_points=..., half_shift=...)``."""
    pts, sh = (ctypes.c_int * J)(), (ctypes.c_int * J)()
    check(lib.sht_icositetrahedral_grid_sizes(J, pts, sh))
    return list(pts), list(sh)


class Analysis(torch.autograd.Function):
    """grid -> spectrum with the native adjoint as backward."""

    @staticmethod
    def forward(ctx, grid, plan):
        ctx.plan = plan
        return plan.forward(grid.contiguous())

    @staticmethod
    def backward(ctx, g):
        return ctx.plan.adjoint(0, g.contiguous()), None


class Synthesis(torch.autograd.Function):
    """spectrum -> grid with the native adjoint as backward."""

    @staticmethod
    def forward(ctx, spec, plan):
        ctx.plan = plan
        return plan.inverse(spec.contiguous())

    @staticmethod
    def backward(ctx, g):
        return ctx.plan.adjoint(1, g.contiguous()), None


def analysis(grid, plan):
    return Analysis.apply(grid, plan)


def synthesis(spec, plan):
    return Synthesis.apply(spec, plan)


__all__ = ["Plan", "Group", "Analysis", "Synthesis", "analysis", "synthesis",
           "octahedral_grid_sizes", "icositetrahedral_grid_sizes", "SHTError"]
