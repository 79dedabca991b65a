"""B300-native layered-medium elastic multiple-scattering solver (arxiv 2608.26875).

Python face of the C ABI in include/ms_b300.h.  `Solver` owns one library handle; its methods
take and return torch CUDA tensors in the library layout (M, 2, 2p+1, nrhs) complex128, with
b = 0 the compressional (alpha / a) and b = 1 the shear (beta / b) coefficients of order n = -p..p.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _native as nat
from ._native import (MS_PART_R, MS_PART_S, MS_PART_T, MS_PART_T_FAR, MS_PART_T_NEAR, MS_PREC_BF16,
                      MS_PREC_FP32, MS_PREC_FP64, MsError)

__all__ = ["Solver", "Solver3", "MsError", "MS_PREC_FP64", "MS_PREC_FP32", "MS_PREC_BF16", "MS_PART_T", "MS_PART_R", "MS_PART_S",
           "MS_PART_T_NEAR", "MS_PART_T_FAR", "default_options"]


def _dp(a: np.ndarray):
    return a.ctypes.data_as(nat.c_dp)


def _ip(a: np.ndarray):
    return a.ctypes.data_as(nat.c_ip)


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def tensor_peak(prec: int = MS_PREC_FP32, iters: int = 200000):
    """Measured dense tensor-core rate (TFLOP/s) for the operand kind of prec (ms_tensor_peak)."""
    tf, ms = ctypes.c_double(), ctypes.c_double()
    nat.check(nat.lib().ms_tensor_peak(prec, int(iters), ctypes.byref(tf), ctypes.byref(ms)), "ms_tensor_peak")
    return float(tf.value), float(ms.value)


def default_options() -> nat.Options:
    o = nat.Options()
    nat.lib().ms_default_options(ctypes.byref(o))
    return o


class Solver:
    """One geometry, medium, frequency omega and expansion order p (ms_setup)."""

    def __init__(self, centres, radius, bc, media, omega: float, p: int, proto=None, rotation=None,
                 proto_S=None, n_panels: int = 32, nodes_per_panel: int = 16, t_max: float = 20.0,
                 restart: int = 50, max_iters: int = 2000, check_geometry: bool = True,
                 use_fmm: bool = True, leaf_target: int = 10, depth: float = 0.5, grade: int = 0,
                 tensor_cores: bool = True, inner_tol: float = 0.0, block_krylov: bool = True,
                 cuda_graph: bool = True, tc_wait_test: int = 0, store_near: int = 0, precond_group: int = 0):
        L = nat.lib()
        self._keep = []
        c = np.ascontiguousarray(centres, dtype=np.float64)
        r = np.ascontiguousarray(radius, dtype=np.float64)
        b = np.ascontiguousarray(bc, dtype=np.int32)
        M = int(c.shape[0])
        g = nat.Geometry()
        g.M = M
        g.centres, g.radius, g.bc = _dp(c), _dp(r), _ip(b)
        self._keep += [c, r, b]
        if proto is not None:
            pr = np.ascontiguousarray(proto, dtype=np.int32)
            g.proto = _ip(pr)
            self._keep.append(pr)
        if rotation is not None:
            ro = np.ascontiguousarray(rotation, dtype=np.float64)
            g.rotation = _dp(ro)
            self._keep.append(ro)
        if proto_S is not None:
            ps = np.ascontiguousarray(np.asarray(proto_S, dtype=np.complex128)).view(np.float64)
            g.n_proto = int(np.asarray(proto_S).shape[0])
            g.proto_S = _dp(ps)
            self._keep.append(ps)
        md = nat.Media(float(media.lam_u), float(media.mu_u), float(media.lam_l), float(media.mu_l))
        o = default_options()
        o.n_panels, o.nodes_per_panel, o.t_max = n_panels, nodes_per_panel, float(t_max)
        o.restart, o.max_iters, o.check_geometry = restart, max_iters, int(bool(check_geometry))
        o.use_fmm, o.leaf_target = int(bool(use_fmm)), int(leaf_target)
        o.depth, o.grade = float(depth), int(grade)
        o.tensor_cores = int(bool(tensor_cores))
        o.inner_tol = float(inner_tol)
        o.block_krylov = int(bool(block_krylov))
        o.cuda_graph = int(bool(cuda_graph))
        o.tc_wait_test = int(tc_wait_test)
        o.store_near = int(store_near)
        o.precond_group = int(precond_group)
        h = ctypes.c_void_p()
        nat.check(L.ms_setup(ctypes.byref(g), ctypes.byref(md), float(omega), int(p), ctypes.byref(o),
                             ctypes.byref(h)), "ms_setup")
        self._h = h
        self.M, self.p, self.nc = M, int(p), 2 * int(p) + 1
        self.has_proto = proto is not None and bool((np.asarray(proto) >= 0).any())
        nn, lev, npair = nat.c_int(), nat.c_int(), ctypes.c_int64()
        L.ms_info(h, None, None, ctypes.byref(nn), ctypes.byref(lev), ctypes.byref(npair))
        self.n_nodes = int(nn.value)
        self.fmm_levels = int(lev.value)
        self.near_pairs = int(npair.value)
        self._keep = []

    @classmethod
    def from_workload(cls, wl, proto_S=None, **kw):
        """Handle for a synthetic.Workload: closed-form discs, and for a workload with star particles
        (wl.proto) the prototype scattering matrices proto_S (Q, 2nc, 2nc), which the caller supplies."""
        proto = getattr(wl, "proto", None)
        if proto is not None and (np.asarray(proto) >= 0).any():
            if proto_S is None:
                raise ValueError(f"workload {wl.name} has prototype particles: pass proto_S")
            kw.update(proto=proto, proto_S=proto_S)
        return cls(wl.centres, wl.radius, wl.bc, wl.media, wl.omega, wl.p, rotation=wl.rotation,
                   n_panels=wl.n_panels, nodes_per_panel=wl.nodes_per_panel, t_max=wl.t_max,
                   depth=wl.depth, grade=wl.grade, **kw)

    # ------------------------------------------------------------------ helpers
    def _check_vec(self, x: torch.Tensor, nrhs=None) -> int:
        if not (x.is_cuda and x.dtype == torch.complex128 and x.is_contiguous()):
            raise ValueError("expected a contiguous complex128 CUDA tensor")
        if x.dim() != 4 or tuple(x.shape[:3]) != (self.M, 2, self.nc):
            raise ValueError(f"expected shape ({self.M}, 2, {self.nc}, nrhs), got {tuple(x.shape)}")
        return int(x.shape[3])

    def empty(self, nrhs: int, device=None) -> torch.Tensor:
        return torch.empty((self.M, 2, self.nc, nrhs), dtype=torch.complex128, device=device or "cuda")

    # ------------------------------------------------------------------ entry points
    def apply(self, x: torch.Tensor, prec: int = MS_PREC_FP64, out=None, stream=None) -> torch.Tensor:
        """y = x - S (T + R) x (ms_apply)."""
        nrhs = self._check_vec(x)
        y = out if out is not None else torch.empty_like(x)
        nat.check(nat.lib().ms_apply(self._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                     nrhs, prec, _stream(stream)), "ms_apply")
        return y

    def apply_adjoint(self, x: torch.Tensor, prec: int = MS_PREC_FP64, out=None, stream=None) -> torch.Tensor:
        """y = A^H x (ms_apply_adjoint)."""
        nrhs = self._check_vec(x)
        y = out if out is not None else torch.empty_like(x)
        nat.check(nat.lib().ms_apply_adjoint(self._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                             nrhs, prec, _stream(stream)), "ms_apply_adjoint")
        return y

    def operator(self, x: torch.Tensor, parts: int, prec: int = MS_PREC_FP64, stream=None) -> torch.Tensor:
        """y = [S] (T_sel + R_sel) x (ms_operator)."""
        nrhs = self._check_vec(x)
        y = torch.empty_like(x)
        nat.check(nat.lib().ms_operator(self._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                        nrhs, prec, parts, _stream(stream)), "ms_operator")
        return y

    def _incidence(self, kinds, angles):
        k = np.ascontiguousarray(kinds, dtype=np.int32)
        a = np.ascontiguousarray(angles, dtype=np.float64)
        inc = nat.Incidence(int(k.size), _ip(k), _dp(a))
        return inc, (k, a)

    def rhs(self, kinds, angles, stream=None) -> torch.Tensor:
        """b = S a0 for plane-wave incidences from the upper layer (ms_rhs)."""
        inc, keep = self._incidence(kinds, angles)
        b = self.empty(inc.nrhs)
        nat.check(nat.lib().ms_rhs(self._h, ctypes.byref(inc), ctypes.c_void_p(b.data_ptr()), _stream(stream)),
                  "ms_rhs")
        return b

    def solve(self, kinds, angles, tol: float = 1e-12, prec: int = MS_PREC_FP64, stream=None, out=None):
        """gamma solving A gamma = S a0 (ms_solve).  Returns (gamma, info), info a dict with the
        iterations, refinements, mat-vecs, worst relative residual, seconds and the status (MS_OK, or
        MS_NOT_CONVERGED when a column missed tol within the iteration cap)."""
        inc, keep = self._incidence(kinds, angles)
        g = out if out is not None else self.empty(inc.nrhs)
        info = nat.SolveInfo()
        st = nat.check(nat.lib().ms_solve(self._h, ctypes.byref(inc), float(tol), prec,
                                          ctypes.c_void_p(g.data_ptr()), ctypes.byref(info), _stream(stream)),
                       "ms_solve", allow_warning=True)
        return g, {"iterations": info.iterations, "refinements": info.refinements, "matvecs": info.matvecs,
                   "max_rel_residual": info.max_rel_residual, "seconds": info.seconds, "status": st}

    def solve_rhs(self, b: torch.Tensor, tol: float = 1e-12, prec: int = MS_PREC_FP64, x0=None, stream=None,
                  out=None):
        """gamma solving A gamma = b for a caller right-hand side b (ms_solve_rhs), from the initial
        guess x0 (zero if None).  Returns (gamma, info) like solve()."""
        nrhs = self._check_vec(b)
        g = out if out is not None else torch.empty_like(b)
        if x0 is not None:
            self._check_vec(x0)
            g.copy_(x0)
        info = nat.SolveInfo()
        st = nat.check(nat.lib().ms_solve_rhs(self._h, ctypes.c_void_p(b.data_ptr()), nrhs, float(tol), prec,
                                              ctypes.c_void_p(g.data_ptr()), int(x0 is not None), ctypes.byref(info),
                                              _stream(stream)), "ms_solve_rhs", allow_warning=True)
        return g, {"iterations": info.iterations, "refinements": info.refinements, "matvecs": info.matvecs,
                   "max_rel_residual": info.max_rel_residual, "seconds": info.seconds, "status": st}

    def rhs_point(self, sources, forces, stream=None) -> torch.Tensor:
        """b = S a0 for point forces in the upper layer (ms_rhs_point): sources (n, 2) with y > 0,
        forces (n, 2)."""
        src = np.ascontiguousarray(sources, dtype=np.float64)
        fo = np.ascontiguousarray(forces, dtype=np.float64)
        if src.shape != fo.shape or src.ndim != 2 or src.shape[1] != 2:
            raise ValueError("sources and forces must both be (n, 2)")
        b = self.empty(int(src.shape[0]))
        nat.check(nat.lib().ms_rhs_point(self._h, _dp(src), _dp(fo), int(src.shape[0]), ctypes.c_void_p(b.data_ptr()),
                                         _stream(stream)), "ms_rhs_point")
        return b

    def fields_upper(self, gamma: torch.Tensor, receivers, stream=None) -> torch.Tensor:
        """Scattered displacement (nrhs, R, 2) at receivers (R, 2) in the upper layer (ms_fields_upper)."""
        nrhs = self._check_vec(gamma)
        rx = torch.as_tensor(np.ascontiguousarray(receivers, dtype=np.float64), device=gamma.device)
        R = int(rx.shape[0])
        u = torch.empty((nrhs, R, 2), dtype=torch.complex128, device=gamma.device)
        nat.check(nat.lib().ms_fields_upper(self._h, ctypes.c_void_p(gamma.data_ptr()), nrhs,
                                            ctypes.c_void_p(rx.data_ptr()), R, ctypes.c_void_p(u.data_ptr()),
                                            _stream(stream)), "ms_fields_upper")
        return u

    def time_reversal(self, mirror, tol: float = 1e-10, prec: int = MS_PREC_FP64, stream=None):
        """DORT (ms_time_reversal) for mirror points (n, 2) in the upper layer: returns (F, eigenvalues of
        conj(F)^T F descending, eigenvectors as columns, info) as numpy arrays."""
        trm = np.ascontiguousarray(mirror, dtype=np.float64)
        nr = 2 * int(trm.shape[0])
        F = np.zeros((nr, nr), np.complex128)
        ev = np.zeros(nr)
        V = np.zeros((nr, nr), np.complex128)
        info = nat.SolveInfo()
        st = nat.check(nat.lib().ms_time_reversal(self._h, _dp(trm), int(trm.shape[0]), float(tol), prec,
                                                  F.view(np.float64).ctypes.data_as(nat.c_dp), _dp(ev),
                                                  V.view(np.float64).ctypes.data_as(nat.c_dp), ctypes.byref(info),
                                                  _stream(stream)), "ms_time_reversal", allow_warning=True)
        return F, ev, V, {"iterations": info.iterations, "refinements": info.refinements,
                          "max_rel_residual": info.max_rel_residual, "seconds": info.seconds, "status": st}

    def fields(self, gamma: torch.Tensor, receivers, stream=None) -> torch.Tensor:
        """Scattered displacement (nrhs, R, 2) complex128 at receivers (R, 2) in the lower layer (ms_fields)."""
        nrhs = self._check_vec(gamma)
        rx = torch.as_tensor(np.ascontiguousarray(receivers, dtype=np.float64), device=gamma.device)
        R = int(rx.shape[0])
        u = torch.empty((nrhs, R, 2), dtype=torch.complex128, device=gamma.device)
        nat.check(nat.lib().ms_fields(self._h, ctypes.c_void_p(gamma.data_ptr()), nrhs,
                                      ctypes.c_void_p(rx.data_ptr()), R, ctypes.c_void_p(u.data_ptr()),
                                      _stream(stream)), "ms_fields")
        return u

    def grad(self, kinds, angles, gamma: torch.Tensor, w: torch.Tensor, receivers, tol: float = 1e-10,
             prec: int = MS_PREC_FP64, want_omega: bool = True, stream=None):
        """Adjoint gradient (ms_grad) of a real loss with dL = Re sum conj(w) du at the receivers.
        Returns (dL/dcentres (M,2), dL/dradii (M,), dL/domega or None, info) as float64 tensors."""
        inc, keep = self._incidence(kinds, angles)
        nrhs = self._check_vec(gamma)
        rx = torch.as_tensor(np.ascontiguousarray(receivers, dtype=np.float64), device=gamma.device)
        R = int(rx.shape[0])
        if tuple(w.shape) != (nrhs, R, 2) or w.dtype != torch.complex128 or not w.is_contiguous():
            raise ValueError(f"w must be a contiguous ({nrhs}, {R}, 2) complex128 CUDA tensor")
        gc = torch.empty((self.M, 2), dtype=torch.float64, device=gamma.device)
        gr = torch.empty((self.M,), dtype=torch.float64, device=gamma.device)
        go = ctypes.c_double(0.0)
        info = nat.SolveInfo()
        st = nat.check(nat.lib().ms_grad(self._h, ctypes.byref(inc), ctypes.c_void_p(gamma.data_ptr()),
                                         ctypes.c_void_p(w.data_ptr()), ctypes.c_void_p(rx.data_ptr()), R,
                                         float(tol), prec, ctypes.c_void_p(gc.data_ptr()),
                                         ctypes.c_void_p(gr.data_ptr()), ctypes.byref(go) if want_omega else None,
                                         ctypes.byref(info), _stream(stream)), "ms_grad", allow_warning=True)
        return gc, gr, (go.value if want_omega else None), {
            "iterations": info.iterations, "refinements": info.refinements, "matvecs": info.matvecs,
            "max_rel_residual": info.max_rel_residual, "seconds": info.seconds, "status": st}

    def fields_noalloc(self, gamma: torch.Tensor, rx: torch.Tensor, out: torch.Tensor, stream=None) -> torch.Tensor:
        """ms_fields without any allocation: rx (R, 2) float64 and out (nrhs, R, 2) complex128 are
        caller-owned CUDA tensors; scratch lives in the library's fixed device arrays."""
        nrhs = self._check_vec(gamma)
        if not (rx.is_cuda and rx.dtype == torch.float64 and rx.is_contiguous() and rx.dim() == 2):
            raise ValueError("rx must be a contiguous (R, 2) float64 CUDA tensor")
        R = int(rx.shape[0])
        if tuple(out.shape) != (nrhs, R, 2) or out.dtype != torch.complex128 or not out.is_contiguous():
            raise ValueError(f"out must be a contiguous ({nrhs}, {R}, 2) complex128 CUDA tensor")
        nat.check(nat.lib().ms_fields_noalloc(self._h, ctypes.c_void_p(gamma.data_ptr()), nrhs,
                                              ctypes.c_void_p(rx.data_ptr()), R, ctypes.c_void_p(out.data_ptr()),
                                              _stream(stream)), "ms_fields_noalloc")
        return out

    def work(self):
        """ms_work: algorithmic complex multiply-adds per column of one application, by part."""
        v = [ctypes.c_double() for _ in range(4)]
        nat.check(nat.lib().ms_work(self._h, *[ctypes.byref(x) for x in v]), "ms_work")
        return dict(zip(("near", "far", "refl", "sapply"), (x.value for x in v)))

    def near_stored_bytes(self) -> int:
        """ms_near_stored: device bytes of the stored near-pair operator (0: generated per application)."""
        v = ctypes.c_int64()
        nat.check(nat.lib().ms_near_stored(self._h, ctypes.byref(v)), "ms_near_stored")
        return int(v.value)

    def autotune(self, nrhs: int = 64, prec: int = MS_PREC_FP32, stream=None):
        """ms_autotune: time the candidate FMM leaf levels and multipole-to-Sommerfeld split sizes and keep
        the fastest.  Returns (leaf target, rows per split, ms per application)."""
        leaf, rows, ms = nat.c_int(), nat.c_int(), ctypes.c_double()
        nat.check(nat.lib().ms_autotune(self._h, int(nrhs), prec, ctypes.byref(leaf), ctypes.byref(rows),
                                        ctypes.byref(ms), _stream(stream)), "ms_autotune")
        lev = nat.c_int()
        npair = ctypes.c_int64()
        nat.lib().ms_info(self._h, None, None, None, ctypes.byref(lev), ctypes.byref(npair))
        self.fmm_levels, self.near_pairs = int(lev.value), int(npair.value)
        return int(leaf.value), int(rows.value), float(ms.value)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            nat.lib().ms_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Solver3:
    """3D handle (include/ms3_b300.h): spheres below the interface, vector spherical wave expansions,
    polar Sommerfeld rule.  Blocks are torch CUDA tensors (M, T, nrhs) complex128, T = 2p(p+2) + (p+1)^2,
    coefficients in the order [alpha (n = 1..p) | beta (n = 1..p) | gamma (n = 0..p)], (n, m) at
    n^2 + n + m (minus one for alpha and beta)."""

    def __init__(self, centres, radius, bc, media, omega: float, p: int, n_r: int = 128, n_theta: int = 64,
                 n_panels: int = 4, t_max: float = 10.0, alpha: float = 1.0, beta: float = 1.0, restart: int = 60,
                 max_iters: int = 1000):
        L = nat.lib()
        c = np.ascontiguousarray(centres, dtype=np.float64)
        r = np.ascontiguousarray(radius, dtype=np.float64)
        b = np.ascontiguousarray(bc, dtype=np.int32)
        g = nat.Geometry3()
        g.M = int(r.shape[0])
        g.centres, g.radius, g.bc = _dp(c), _dp(r), _ip(b)
        md = nat.Media(float(media.lam_u), float(media.mu_u), float(media.lam_l), float(media.mu_l))
        o = nat.Options3()
        L.ms3_default_options(ctypes.byref(o))
        o.n_r, o.n_theta, o.n_panels = int(n_r), int(n_theta), int(n_panels)
        o.t_max, o.alpha, o.beta = float(t_max), float(alpha), float(beta)
        o.restart, o.max_iters = int(restart), int(max_iters)
        h = ctypes.c_void_p()
        nat.check(L.ms3_setup(ctypes.byref(g), ctypes.byref(md), float(omega), int(p), ctypes.byref(o),
                              ctypes.byref(h)), "ms3_setup")
        self._h = h
        self.M, self.p = g.M, int(p)
        self.T = 2 * self.p * (self.p + 2) + (self.p + 1) ** 2
        nn = nat.c_int()
        L.ms3_info(h, None, None, None, ctypes.byref(nn))
        self.n_nodes = int(nn.value)

    def _check(self, x):
        if not (x.is_cuda and x.dtype == torch.complex128 and x.is_contiguous()) or x.dim() != 3 or \
                tuple(x.shape[:2]) != (self.M, self.T):
            raise ValueError(f"expected a contiguous complex128 CUDA tensor ({self.M}, {self.T}, nrhs)")
        return int(x.shape[2])

    def apply(self, x: torch.Tensor, prec: int = MS_PREC_FP64, out=None, stream=None) -> torch.Tensor:
        """y = x - S (T + R) x (ms3_apply), FP64 or FP32 arithmetic."""
        return self.operator(x, nat.MS3_PART_T | nat.MS3_PART_R | nat.MS3_PART_S, prec, out, stream)

    def operator(self, x: torch.Tensor, parts: int, prec: int = MS_PREC_FP64, out=None, stream=None) -> torch.Tensor:
        """The selected parts (ms3_operator): with MS3_PART_S, x - S (parts) x; else (parts) x."""
        nrhs = self._check(x)
        y = out if out is not None else torch.empty_like(x)
        nat.check(nat.lib().ms3_operator(self._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()), nrhs,
                                         int(parts), int(prec), _stream(stream)), "ms3_operator")
        return y

    @staticmethod
    def _incidence(kinds, thetas, phis):
        k = np.ascontiguousarray(kinds, dtype=np.int32)
        t = np.ascontiguousarray(thetas, dtype=np.float64)
        f = np.ascontiguousarray(phis, dtype=np.float64)
        inc = nat.Incidence3(int(k.shape[0]), _ip(k), _dp(t), _dp(f))
        return inc, (k, t, f)

    def rhs(self, kinds, thetas, phis, stream=None) -> torch.Tensor:
        """b = S a0 for plane waves from the upper layer (kind 0 P, 1 SV, 2 SH; angle from the downward
        vertical; azimuth) (ms3_rhs)."""
        inc, keep = self._incidence(kinds, thetas, phis)
        b = torch.empty((self.M, self.T, inc.nrhs), dtype=torch.complex128, device="cuda")
        nat.check(nat.lib().ms3_rhs(self._h, ctypes.byref(inc), ctypes.c_void_p(b.data_ptr()), _stream(stream)),
                  "ms3_rhs")
        return b

    def solve(self, kinds, thetas, phis, tol: float = 1e-10, prec: int = MS_PREC_FP64, stream=None):
        """tau solving A tau = S a0 (ms3_solve): FP64, or FP32 inner solves with FP64 refinement.
        Returns (tau, info)."""
        inc, keep = self._incidence(kinds, thetas, phis)
        g = torch.empty((self.M, self.T, inc.nrhs), dtype=torch.complex128, device="cuda")
        info = nat.SolveInfo()
        st = nat.check(nat.lib().ms3_solve(self._h, ctypes.byref(inc), float(tol), int(prec),
                                           ctypes.c_void_p(g.data_ptr()), ctypes.byref(info), _stream(stream)),
                       "ms3_solve", allow_warning=True)
        return g, {"iterations": info.iterations, "refinements": info.refinements, "matvecs": info.matvecs,
                   "max_rel_residual": info.max_rel_residual, "seconds": info.seconds, "status": st}

    def close(self):
        if getattr(self, "_h", None):
            nat.lib().ms3_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
