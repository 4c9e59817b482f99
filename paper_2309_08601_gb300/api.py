"""Torch-facing wrapper of the mp3pcf C ABI.

PyTorch provides device memory and the CUDA stream; every step of the estimator runs in the
library's CUDA kernels. Tensors passed in must be contiguous CUDA tensors of the documented
dtypes; outputs are allocated with torch on the estimator's device.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass
from typing import Optional

import numpy as np

from . import native


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("mp3pcf needs a CUDA device; there is no CPU fallback")
    return torch


def _ptr(t) -> Optional[int]:
    return None if t is None else t.data_ptr()


def _need(t, dtype, name, n=None):
    torch = _torch()
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("%s must be a CUDA tensor" % name)
    if t.dtype != dtype:
        raise ValueError("%s must be %s, got %s" % (name, dtype, t.dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if n is not None and t.numel() != n:
        raise ValueError("%s must have %d entries" % (name, n))
    return t


@dataclass
class Measurement:
    upsilon: object  # [n_z^3][4][n_max+1][nb][nb] complex128
    norm: object     # [n_z^3][2n_max+1][nb][nb] complex128
    gamma_n: object  # [n_z^3][4][2n_max+1][nb][nb] complex128
    n_singular: int
    gamma_x: object    # [n_z^3][4][nb][nb][n_phi]
    gamma_cen: object  # [n_z^3][4][nb][nb][n_phi]
    corr: object       # [n_z^3][n_ap][4] complex128
    m8: object         # [n_z^3][n_ap][8] float64


class Estimator:
    """One library context: a measurement setup bound to a device and a stream."""

    def __init__(self, n_bins, theta_min, theta_max, n_max, *, n_phi=100, n_z=1,
                 quantum=2.0 ** -13, precision="fp32", norm_truncate=False,
                 radial_nodes="arithmetic", cell_occupancy=0, contract_slices=0,
                 exclude_degenerate=False, grid_fft=False, stream=None):
        torch = _torch()
        self.cfg = native.make_config(n_bins, theta_min, theta_max, n_max, n_phi, n_z, quantum,
                                      precision, norm_truncate, radial_nodes, cell_occupancy,
                                      contract_slices, exclude_degenerate, grid_fft)
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.precision = precision
        self._ctx = C.c_void_p()
        native.check(native.lib().mp3pcf_create(C.byref(self.cfg), C.c_void_p(self.stream.cuda_stream),
                                                C.byref(self._ctx)), "mp3pcf_create")

    # ------------------------------------------------------------------ lifetime
    def close(self):
        if self._ctx:
            native.lib().mp3pcf_destroy(self._ctx)
            self._ctx = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ------------------------------------------------------------------ shapes
    @property
    def n_bins(self):
        return self.cfg.n_bins

    @property
    def n_max(self):
        return self.cfg.n_max

    @property
    def n_z(self):
        return self.cfg.n_z

    @property
    def z3(self):
        return self.cfg.n_z ** 3

    def bin_edges(self):
        e = np.zeros(self.n_bins + 1)
        e2 = np.zeros(self.n_bins + 1, dtype=np.int64)
        native.check(native.lib().mp3pcf_bin_edges(C.byref(self.cfg), e.ctypes.data_as(C.c_void_p),
                                                   e2.ctypes.data_as(C.c_void_p)), "mp3pcf_bin_edges")
        return e, e2

    # ------------------------------------------------------------------ stage (a)
    def accumulate_moments(self, xq, yq, g1, g2, w, zbin=None, centre_mask=None):
        self._generation = getattr(self, "_generation", 0) + 1
        torch = _torch()
        n = int(xq.numel())
        _need(xq, torch.int32, "xq", n)
        _need(yq, torch.int32, "yq", n)
        _need(g1, torch.float32, "g1", n)
        _need(g2, torch.float32, "g2", n)
        _need(w, torch.float32, "w", n)
        _need(zbin, torch.uint8, "zbin", n)
        _need(centre_mask, torch.uint8, "centre_mask", n)
        st = native.lib().mp3pcf_accumulate_moments(self._ctx, n, _ptr(xq), _ptr(yq), _ptr(g1),
                                                    _ptr(g2), _ptr(w), _ptr(zbin), _ptr(centre_mask))
        native.check(st, "mp3pcf_accumulate_moments", self._ctx)

    def accumulate_moments_combined(self, xq, yq, g1, g2, w, zbin=None, centre_mask=None, levels=()):
        """The combined estimator's moments (Sec. 3.3) through mp3pcf_accumulate_moments_combined:
        levels is a sequence of (b_start, pixel_q); bins below the first b_start are the galaxies'
        discrete moments, bins from b_start[l] on (up to the next level's) the moments of the
        pixel catalog of side pixel_q quanta at each centre galaxy's pixel. contract() then gives
        the combined multipoles."""
        self._generation = getattr(self, "_generation", 0) + 1
        torch = _torch()
        n = int(xq.numel())
        _need(xq, torch.int32, "xq", n)
        _need(yq, torch.int32, "yq", n)
        _need(g1, torch.float32, "g1", n)
        _need(g2, torch.float32, "g2", n)
        _need(w, torch.float32, "w", n)
        _need(zbin, torch.uint8, "zbin", n)
        _need(centre_mask, torch.uint8, "centre_mask", n)
        L = len(levels)
        bs = (C.c_int32 * max(L, 1))(*[int(b) for b, _ in levels])
        pq = (C.c_int64 * max(L, 1))(*[int(q) for _, q in levels])
        st = native.lib().mp3pcf_accumulate_moments_combined(self._ctx, n, _ptr(xq), _ptr(yq), _ptr(g1), _ptr(g2),
                                                             _ptr(w), _ptr(zbin), _ptr(centre_mask), L, bs, pq)
        native.check(st, "mp3pcf_accumulate_moments_combined", self._ctx)

    def counts(self):
        nc = C.c_int64()
        npairs = C.c_int64()
        native.check(native.lib().mp3pcf_counts(self._ctx, C.byref(nc), C.byref(npairs)),
                     "mp3pcf_counts", self._ctx)
        return nc.value, npairs.value

    def moments(self):
        torch = _torch()
        nc, _ = self.counts()
        dt = torch.complex128 if self.precision == "fp64" else torch.complex64
        G = torch.empty((nc, self.n_z, self.n_bins, 2 * self.n_max + 3), dtype=dt, device=self.device)
        W = torch.empty((nc, self.n_z, self.n_bins, 2 * self.n_max + 1), dtype=dt, device=self.device)
        native.check(native.lib().mp3pcf_copy_moments(self._ctx, _ptr(G), _ptr(W)),
                     "mp3pcf_copy_moments", self._ctx)
        return G, W

    # ------------------------------------------------------------------ stage (b)
    def new_multipoles(self):
        torch = _torch()
        ups = torch.zeros((self.z3, 4, self.n_max + 1, self.n_bins, self.n_bins),
                          dtype=torch.complex128, device=self.device)
        norm = torch.zeros((self.z3, 2 * self.n_max + 1, self.n_bins, self.n_bins),
                           dtype=torch.complex128, device=self.device)
        return ups, norm

    def contract(self, ups=None, norm=None):
        """Adds this catalog's multipoles into (ups, norm) (fresh zero buffers if None)."""
        if ups is None or norm is None:
            ups, norm = self.new_multipoles()
        native.check(native.lib().mp3pcf_contract_multipoles(self._ctx, _ptr(ups), _ptr(norm)),
                     "mp3pcf_contract_multipoles", self._ctx)
        return ups, norm

    # ------------------------------------------------------------------ FP64 post-processing
    def edge_correct(self, ups, norm, report_singular=True):
        torch = _torch()
        gam = torch.empty((self.z3, 4, 2 * self.n_max + 1, self.n_bins, self.n_bins),
                          dtype=torch.complex128, device=self.device)
        ns = C.c_int64(0)
        st = native.lib().mp3pcf_edge_correct(self._ctx, _ptr(ups), _ptr(norm), _ptr(gam),
                                              C.byref(ns) if report_singular else None)
        native.check(st, "mp3pcf_edge_correct", self._ctx, ok=(native.OK, native.ESINGULAR))
        return gam, int(ns.value)

    def to_gamma(self, gamma_n, projection: int):
        torch = _torch()
        out = torch.empty((self.z3, 4, self.n_bins, self.n_bins, self.cfg.n_phi),
                          dtype=torch.complex128, device=self.device)
        native.check(native.lib().mp3pcf_to_gamma(self._ctx, _ptr(gamma_n), int(projection), _ptr(out)),
                     "mp3pcf_to_gamma", self._ctx)
        return out

    def to_map3(self, gamma_cen, theta_ap):
        torch = _torch()
        th = torch.as_tensor(np.atleast_2d(np.asarray(theta_ap, dtype=np.float64)),
                             device=self.device).contiguous()
        n_ap = th.shape[0]
        corr = torch.empty((self.z3, n_ap, 4), dtype=torch.complex128, device=self.device)
        m8 = torch.empty((self.z3, n_ap, 8), dtype=torch.float64, device=self.device)
        native.check(native.lib().mp3pcf_to_map3(self._ctx, _ptr(gamma_cen), n_ap, _ptr(th),
                                                 _ptr(corr), _ptr(m8)), "mp3pcf_to_map3", self._ctx)
        return corr, m8

    def to_map3_four(self, gamma_cen, theta_ap):
        """m4 [n_z^3][n_ap][4] = (Map^3, <Map^2 Mx>, <Map Mx^2>, <Mx^3>) by the four-equation form
        of App. C (mp3pcf_to_map3_four), a cross-check of to_map3's eight-equation form."""
        torch = _torch()
        th = torch.as_tensor(np.atleast_2d(np.asarray(theta_ap, dtype=np.float64)),
                             device=self.device).contiguous()
        n_ap = th.shape[0]
        m4 = torch.empty((self.z3, n_ap, 4), dtype=torch.float64, device=self.device)
        native.check(native.lib().mp3pcf_to_map3_four(self._ctx, _ptr(gamma_cen), n_ap, _ptr(th), _ptr(m4)),
                     "mp3pcf_to_map3_four", self._ctx)
        return m4

    # ------------------------------------------------------------------ batching
    def set_extent(self, extent):
        """Fixed patch extent (x0, y0, x1, y1) in position quanta, or None."""
        if extent is None:
            native.check(native.lib().mp3pcf_set_extent(self._ctx, None), "mp3pcf_set_extent", self._ctx)
            return
        e = (C.c_int64 * 4)(*[int(v) for v in extent])
        native.check(native.lib().mp3pcf_set_extent(self._ctx, e), "mp3pcf_set_extent", self._ctx)

    def run_batch(self, catalogs, extent, theta_ap, use_graphs=True):
        """m8 [n_cats][n_z^3][n_ap][8] for a list of device catalogs (xq, yq, g1, g2, w[, zbin]) of
        any sizes inside a common extent, through mp3pcf_run_batch (CUDA graphs by default)."""
        torch = _torch()
        th = torch.as_tensor(np.atleast_2d(np.asarray(theta_ap, dtype=np.float64)),
                             device=self.device).contiguous()
        views = (native.CatalogView * max(1, len(catalogs)))()
        for i, cat in enumerate(catalogs):
            xq, yq, g1, g2, w = cat[:5]
            zb = cat[5] if len(cat) > 5 else None
            n = int(xq.numel())
            for t, dt, nm in ((xq, torch.int32, "xq"), (yq, torch.int32, "yq"), (g1, torch.float32, "g1"),
                              (g2, torch.float32, "g2"), (w, torch.float32, "w")):
                _need(t, dt, nm, n)
            _need(zb, torch.uint8, "zbin", n)
            views[i] = native.CatalogView(n, _ptr(xq), _ptr(yq), _ptr(g1), _ptr(g2), _ptr(w), _ptr(zb))
        m8 = torch.empty((len(catalogs), self.z3, th.shape[0], 8), dtype=torch.float64, device=self.device)
        e = (C.c_int64 * 4)(*[int(v) for v in extent])
        native.check(native.lib().mp3pcf_run_batch(self._ctx, views, len(catalogs), e, th.shape[0], _ptr(th),
                                                   _ptr(m8), int(bool(use_graphs))),
                     "mp3pcf_run_batch", self._ctx)
        return m8

    def last_error(self) -> str:
        r = native.lib().mp3pcf_last_error(self._ctx)
        return r.decode() if r else ""

    def graph_stats(self):
        """(CUDA-graph launches, instantiations) made by run_batch so far."""
        a, b = C.c_int64(), C.c_int64()
        native.check(native.lib().mp3pcf_graph_stats(self._ctx, C.byref(a), C.byref(b)), "mp3pcf_graph_stats")
        return int(a.value), int(b.value)

    # ------------------------------------------------------------------ grid-based approximation
    def grid_catalog(self, xq, yq, g1, g2, w, zbin=None, pixel_arcmin=1.0, origin=None, shape=None):
        """The pixel catalog of the grid-based approximation (Sec. 3.2) through mp3pcf_grid_catalog:
        device tensors (xq, yq, g1, g2, w, zbin-or-None) of the non-empty pixels, in (z, iy, ix)
        order, of side pixel_arcmin (rounded to whole quanta); origin (quanta) and shape (npx, npy) default to
        the catalog's bounding box. Its moments and multipoles (measure, accumulate_moments, ...)
        are the grid estimator's (Eq. UpsilonmuGrid)."""
        torch = _torch()
        n = int(xq.numel())
        for t, dt, nm in ((xq, torch.int32, "xq"), (yq, torch.int32, "yq"), (g1, torch.float32, "g1"),
                          (g2, torch.float32, "g2"), (w, torch.float32, "w")):
            _need(t, dt, nm, n)
        _need(zbin, torch.uint8, "zbin", n)
        pq = max(1, int(round(float(pixel_arcmin) / float(self.cfg.quantum))))
        if origin is None:
            origin = (int(xq.min()), int(yq.min())) if n else (0, 0)
        if shape is None:
            npx = (int(xq.max()) - int(origin[0])) // pq + 1 if n else 1
            npy = (int(yq.max()) - int(origin[1])) // pq + 1 if n else 1
        else:
            npx, npy = int(shape[0]), int(shape[1])
        nz = int(self.cfg.n_z)
        m = nz * npx * npy
        out = (torch.empty(m, dtype=torch.int32, device=self.device), torch.empty(m, dtype=torch.int32, device=self.device),
               torch.empty(m, dtype=torch.float32, device=self.device), torch.empty(m, dtype=torch.float32, device=self.device),
               torch.empty(m, dtype=torch.float32, device=self.device),
               torch.empty(m, dtype=torch.uint8, device=self.device) if nz > 1 else None)
        org = (C.c_int64 * 2)(int(origin[0]), int(origin[1]))
        cnt = C.c_int64()
        native.check(native.lib().mp3pcf_grid_catalog(self._ctx, n, _ptr(xq), _ptr(yq), _ptr(g1), _ptr(g2), _ptr(w),
                                                      _ptr(zbin), org, pq, npx, npy, *[_ptr(t) for t in out],
                                                      C.byref(cnt)),
                     "mp3pcf_grid_catalog", self._ctx)
        k = int(cnt.value)
        return tuple(None if t is None else t[:k] for t in out)

    # ------------------------------------------------------------------ direct estimator
    def map3_direct(self, xq, yq, g1, g2, w, theta_ap, centres, rcut_factor=4.0):
        """Numerator and denominator [n_centres][n_ap][2] (float64) of the direct estimator of
        <M_ap^3> (Sec. 5.3, Eq. MapDirectEstimator) at the aperture centres [n_centres][2]
        (arcmin, x = xq * quantum) for the radii triples theta_ap [n_ap][3] (arcmin); galaxies
        beyond rcut_factor * max(theta) from a centre are left out."""
        torch = _torch()
        n = int(xq.numel())
        for t, dt, nm in ((xq, torch.int32, "xq"), (yq, torch.int32, "yq"), (g1, torch.float32, "g1"),
                          (g2, torch.float32, "g2"), (w, torch.float32, "w")):
            _need(t, dt, nm, n)
        th = torch.as_tensor(np.atleast_2d(np.asarray(theta_ap, dtype=np.float64)),
                             device=self.device).contiguous()
        cen = torch.as_tensor(np.asarray(centres, dtype=np.float64).reshape(-1, 2), device=self.device).contiguous()
        out = torch.empty((cen.shape[0], th.shape[0], 2), dtype=torch.float64, device=self.device)
        native.check(native.lib().mp3pcf_map3_direct(self._ctx, n, _ptr(xq), _ptr(yq), _ptr(g1), _ptr(g2), _ptr(w),
                                                     cen.shape[0], _ptr(cen), th.shape[0], _ptr(th),
                                                     float(rcut_factor), _ptr(out)),
                     "mp3pcf_map3_direct", self._ctx)
        return out

    # ------------------------------------------------------------------ adjoints
    def to_map3_adjoint(self, theta_ap, grad_m8=None, grad_corr=None):
        """dL/dGamma^cen from dL/dm8 and/or dL/dcorr (complex gradients: dL/dRe + i dL/dIm)."""
        torch = _torch()
        th = torch.as_tensor(np.atleast_2d(np.asarray(theta_ap, dtype=np.float64)),
                             device=self.device).contiguous()
        n_ap = th.shape[0]
        if grad_m8 is not None:
            grad_m8 = _need(grad_m8.contiguous(), torch.float64, "grad_m8", self.z3 * n_ap * 8)
        if grad_corr is not None:
            grad_corr = _need(grad_corr.contiguous(), torch.complex128, "grad_corr", self.z3 * n_ap * 4)
        out = torch.empty((self.z3, 4, self.n_bins, self.n_bins, self.cfg.n_phi),
                          dtype=torch.complex128, device=self.device)
        native.check(native.lib().mp3pcf_to_map3_adjoint(self._ctx, n_ap, _ptr(th), _ptr(grad_corr),
                                                         _ptr(grad_m8), _ptr(out)),
                     "mp3pcf_to_map3_adjoint", self._ctx)
        return out

    def to_gamma_adjoint(self, grad_gamma_phi, projection: int):
        torch = _torch()
        g = _need(grad_gamma_phi.contiguous(), torch.complex128, "grad_gamma_phi")
        out = torch.empty((self.z3, 4, 2 * self.n_max + 1, self.n_bins, self.n_bins),
                          dtype=torch.complex128, device=self.device)
        native.check(native.lib().mp3pcf_to_gamma_adjoint(self._ctx, int(projection), _ptr(g), _ptr(out)),
                     "mp3pcf_to_gamma_adjoint", self._ctx)
        return out

    def edge_correct_adjoint(self, norm, gamma_n, grad_gamma_n):
        """(dL/dUpsilon, dL/dN) of the edge-correction solve."""
        torch = _torch()
        g = _need(grad_gamma_n.contiguous(), torch.complex128, "grad_gamma_n")
        gu, gn = self.new_multipoles()
        native.check(native.lib().mp3pcf_edge_correct_adjoint(self._ctx, _ptr(norm), _ptr(gamma_n), _ptr(g),
                                                              _ptr(gu), _ptr(gn)),
                     "mp3pcf_edge_correct_adjoint", self._ctx)
        return gu, gn

    def moments_adjoint(self, grad_ups, grad_norm, g1, g2, w):
        """(dL/dgamma_1, dL/dgamma_2, dL/dw) per galaxy for the catalog of the last
        accumulate_moments call, given dL/dUpsilon and dL/dN."""
        torch = _torch()
        n = g1.numel()
        for t, nm in ((g1, "g1"), (g2, "g2"), (w, "w")):
            _need(t, torch.float32, nm, n)
        out = [torch.zeros(n, dtype=torch.float32, device=self.device) for _ in range(3)]
        native.check(native.lib().mp3pcf_moments_adjoint(
            self._ctx, _ptr(grad_ups.contiguous()), _ptr(grad_norm.contiguous()), n, _ptr(g1), _ptr(g2),
            _ptr(w), _ptr(out[0]), _ptr(out[1]), _ptr(out[2])), "mp3pcf_moments_adjoint", self._ctx)
        return tuple(out)

    # ------------------------------------------------------------------ tracing
    STAGES = ("sort", "moments", "contract", "edge_correct", "to_gamma", "to_map3")

    def set_timing(self, on: bool = True):
        native.check(native.lib().mp3pcf_set_timing(self._ctx, int(bool(on))), "mp3pcf_set_timing")

    def stage_times(self, reset: bool = True):
        """{stage: (device ms, kernel launches)} since the last reset (synchronises)."""
        ms = np.zeros(6)
        nl = np.zeros(6, dtype=np.int64)
        native.check(native.lib().mp3pcf_stage_times(self._ctx, ms.ctypes.data_as(C.c_void_p),
                                                     nl.ctypes.data_as(C.c_void_p), int(reset)),
                     "mp3pcf_stage_times", self._ctx)
        return {k: (float(ms[i]), int(nl[i])) for i, k in enumerate(self.STAGES)}

    # ------------------------------------------------------------------ whole path
    def measure(self, xq, yq, g1, g2, w, theta_ap, zbin=None, centre_mask=None,
                report_singular=True, levels=None) -> Measurement:
        """The whole path for one catalog; with levels ((b_start, pixel_q), ...) the moments are
        the combined estimator's (accumulate_moments_combined)."""
        if levels:
            self.accumulate_moments_combined(xq, yq, g1, g2, w, zbin, centre_mask, levels=levels)
        else:
            self.accumulate_moments(xq, yq, g1, g2, w, zbin, centre_mask)
        ups, norm = self.contract()
        gam, ns = self.edge_correct(ups, norm, report_singular)
        gx = self.to_gamma(gam, 0)
        gc = self.to_gamma(gam, 1)
        corr, m8 = self.to_map3(gc, theta_ap)
        return Measurement(ups, norm, gam, ns, gx, gc, corr, m8)


def aperture_centres(xq, yq, quantum, theta_ap, spacing=None, rcut_factor=4.0):
    """Aperture centres [n][2] (arcmin) on a square grid over the catalog's bounding box, at
    least rcut_factor * max(theta) from its edges (the direct estimator's apertures must lie
    inside the field, Sec. 5.3); the grid spacing defaults to the smallest radius."""
    x = np.asarray(xq.cpu() if hasattr(xq, "cpu") else xq, dtype=np.float64) * quantum
    y = np.asarray(yq.cpu() if hasattr(yq, "cpu") else yq, dtype=np.float64) * quantum
    th = np.asarray(theta_ap, dtype=np.float64)
    margin = float(rcut_factor) * float(th.max())
    step = float(spacing) if spacing else float(th.min())
    gx = np.arange(x.min() + margin, x.max() - margin + 1e-9, step)
    gy = np.arange(y.min() + margin, y.max() - margin + 1e-9, step)
    if gx.size == 0 or gy.size == 0:
        return np.zeros((0, 2))
    X, Y = np.meshgrid(gx, gy, indexing="ij")
    return np.stack([X.ravel(), Y.ravel()], axis=1)


def map3_from_direct(out):
    """<M_ap^3> per radii triple from mp3pcf_map3_direct's output: the mean over the apertures
    of numerator / denominator (apertures with a zero denominator left out)."""
    o = out.double().cpu().numpy() if hasattr(out, "cpu") else np.asarray(out, dtype=np.float64)
    num, den = o[..., 0], o[..., 1]
    ok = den != 0
    return np.array([(num[ok[:, a], a] / den[ok[:, a], a]).mean() for a in range(o.shape[1])])


def catalog_to_device(cat, device=None):
    """Copies a synth.Catalog to CUDA tensors (xq, yq, g1, g2, w, zbin-or-None)."""
    torch = _torch()
    dev = device or torch.device("cuda", torch.cuda.current_device())
    zb = None if cat.zbin is None else torch.as_tensor(np.ascontiguousarray(cat.zbin, np.uint8), device=dev)
    return (torch.as_tensor(np.ascontiguousarray(cat.xq, np.int32), device=dev),
            torch.as_tensor(np.ascontiguousarray(cat.yq, np.int32), device=dev),
            torch.as_tensor(np.ascontiguousarray(cat.g1, np.float32), device=dev),
            torch.as_tensor(np.ascontiguousarray(cat.g2, np.float32), device=dev),
            torch.as_tensor(np.ascontiguousarray(cat.w, np.float32), device=dev), zb)


# ---------------------------------------------------------------------- differentiation form

def _map3_function():
    torch = _torch()

    class Map3Function(torch.autograd.Function):
        """m8 = Map^3 measures of a catalog, differentiable in (gamma_1, gamma_2, w) through the
        library's hand-written adjoint kernels. The forward keeps the catalog's moments in the
        estimator's context; if the context has been used for another catalog before backward
        runs, the moments are recomputed from the saved inputs first."""

        @staticmethod
        def forward(ctx, g1, g2, w, est, xq, yq, theta_ap, zbin, centre_mask):
            m = est.measure(xq, yq, g1, g2, w, theta_ap, zbin, centre_mask, report_singular=False)
            ctx.est, ctx.theta = est, theta_ap
            ctx.geom = (xq, yq, zbin, centre_mask)
            ctx.generation = est._generation
            ctx.save_for_backward(g1, g2, w, m.norm, m.gamma_n)
            return m.m8

        @staticmethod
        def backward(ctx, grad_m8):
            g1, g2, w, norm, gam = ctx.saved_tensors
            est = ctx.est
            xq, yq, zbin, cmask = ctx.geom
            if est._generation != ctx.generation:
                est.accumulate_moments(xq, yq, g1, g2, w, zbin, cmask)  # recompute G, W
                ctx.generation = est._generation
            ggc = est.to_map3_adjoint(ctx.theta, grad_m8=grad_m8.to(torch.float64))
            ggn = est.to_gamma_adjoint(ggc, 1)
            gu, gn = est.edge_correct_adjoint(norm, gam, ggn)
            d1, d2, dw = est.moments_adjoint(gu, gn, g1.detach(), g2.detach(), w.detach())
            return d1, d2, dw, None, None, None, None, None, None

    return Map3Function


_MAP3_FN = None


def map3(est, xq, yq, g1, g2, w, theta_ap, zbin=None, centre_mask=None):
    """Differentiable <Map^3> measures m8 [n_z^3][n_ap][8] (float64) of a catalog: backward gives
    dL/dgamma_1, dL/dgamma_2, dL/dw (float32, per galaxy) through the library's adjoint kernels
    (to_map3 -> to_gamma -> edge_correct -> contraction -> moments, all on the GPU)."""
    global _MAP3_FN
    if _MAP3_FN is None:
        _MAP3_FN = _map3_function()
    return _MAP3_FN.apply(g1, g2, w, est, xq, yq, theta_ap, zbin, centre_mask)
