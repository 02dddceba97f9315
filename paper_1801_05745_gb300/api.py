"""Python binding of the C ABI in ``include/ufalcon.h`` (libufalcon_gb300.so).

Argument marshalling only: every step of the hot path runs in the CUDA
library.  Device buffers are torch tensors on the context's device; the
calls are enqueued on torch's current CUDA stream.  There is no CPU
fallback: importing this module raises if the library is missing.
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# UFC_CHECKED=1 loads the checked build (index tests in the kernels), made
# by build.build(checked=True)
CHECKED = os.environ.get("UFC_CHECKED", "0") == "1"
LIB_PATH = os.path.join(_HERE, "_build", "libufalcon_gb300_checked.so" if CHECKED
                        else "libufalcon_gb300.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{os.path.basename(LIB_PATH)} is not built ({LIB_PATH}); run "
                      "paper_1801_05745_gb300.build.build(checked=...) or __graft_entry__.build()")

_lib = ctypes.CDLL(LIB_PATH)

P = ctypes.c_void_p
I32 = ctypes.c_int32
I64 = ctypes.c_int64
D = ctypes.c_double
DP = ctypes.POINTER(ctypes.c_double)

UFC_OK = 0
UFC_BIN_ACCUMULATE = 1
UFC_BIN_FORCE_DIRECT = 2
UFC_BIN_FORCE_DENSE = 4
UFC_BATCH_GRAPH = 1
UFC_BATCH_LAUNCHES = 2
NMOMENTS = 10
MOMENT_NAMES = ("mean", "mu2", "mu3", "mu4", "skew", "kurt", "s2_expect", "var_s2",
                "s2_over_var_s2", "n")


class Tuning(ctypes.Structure):
    """ufc_tuning: chunk size and blocks per SM of the persistent batch kernel (0 = default)."""
    _fields_ = [("batch_chunk", I32), ("batch_blocks_per_sm", I32)]


class Cosmo(ctypes.Structure):
    """ufc_cosmo: flat LambdaCDM (omega_m, h), lengths in Mpc/h if units_mpc_over_h;
    density_volume = 1 averages the density factor over the shell volume."""
    _fields_ = [("omega_m", D), ("h", D), ("units_mpc_over_h", I32), ("density_volume", I32)]


class Box(ctypes.Structure):
    """ufc_box: one box of the nesting scheme (observer, owned shells, n_total)."""
    _fields_ = [("L", D), ("obs", D * 3), ("n_total", I64), ("shell_lo", I32),
                ("shell_hi", I32), ("replicate", I32)]


class Source(ctypes.Structure):
    """ufc_source: kind 0 = plane at z_s, kind 1 = n(z) ~ z^alpha exp(-(z/z0)^beta)."""
    _fields_ = [("kind", I32), ("z_s", D), ("alpha", D), ("beta", D), ("z0", D), ("z_max", D)]


def make_cosmo(omega_m=0.3, h=0.7, units_mpc_over_h=1, density_volume=0) -> Cosmo:
    return Cosmo(float(omega_m), float(h), int(units_mpc_over_h), int(density_volume))


def make_box(L, obs, n_total, shell_lo, shell_hi, replicate=0) -> Box:
    b = Box()
    b.L = float(L)
    for i in range(3):
        b.obs[i] = float(obs[i])
    b.n_total, b.shell_lo, b.shell_hi, b.replicate = int(n_total), int(shell_lo), int(shell_hi), int(replicate)
    return b


def make_source(kind=0, z_s=1.5, alpha=2.0, beta=1.5, z0=0.5, z_max=1.5) -> Source:
    return Source(int(kind), float(z_s), float(alpha), float(beta), float(z0), float(z_max))


_SIGS = {
    "ufc_create": [ctypes.POINTER(P), I32],
    "ufc_destroy": [P],
    "ufc_set_stream": [P, P],
    "ufc_synchronize": [P],
    "ufc_wait_selftest": [P, I64],
    "ufc_reserve": [P, I32, I32, I64],
    "ufc_chi_edges": [ctypes.POINTER(Cosmo), P, I32, P],
    "ufc_z_of_chi": [ctypes.POINTER(Cosmo), P, I32, P],
    "ufc_kappa_coeffs": [ctypes.POINTER(Cosmo), P, I32, P, I32, I32, ctypes.POINTER(Source),
                         P, P, P, P, P],
    "ufc_delta_coeffs": [ctypes.POINTER(Cosmo), P, I32, P, I32, I32, P, P, P, P],
    "ufc_keys": [P, P, I64, ctypes.POINTER(Box), P, I32, I32, P],
    "ufc_bin": [P, P, P, P, I32, P, I32, I32, I32, P],
    "ufc_bin_host": [P, P, P, P, I32, P, I32, I32, I32, P],
    "ufc_bin_host_stream": [P, P, P, P, I32, P, I32, I32, I32, I64, P],
    "ufc_bin_info": [P, P],
    "ufc_snapshot_assign": [P, I32, P, I32, P],
    "ufc_bin_snapshots": [P, P, P, P, I32, P, P, I32, I32, I32, P],
    "ufc_bin_snapshots_host": [P, P, P, P, I32, P, P, I32, I32, I32, I64, P],
    "ufc_kappa_stats": [P, P, I32, I32, P, D, D, D, I32, P, P, P],
    "ufc_kappa_backward": [P, P, I32, I32, P, D, D, D, P, P, P, P, P, P],
    "ufc_kappa_stats_backward": [P, P, I32, I32, P, D, D, D, I32, D, D, P, P, P, P, P, P, P, P, P],
    "ufc_welford_update": [P, P, I32, I32, P],
    "ufc_welford_merge": [P, P, P, I32],
    "ufc_welford_finalize": [P, P, I32, I32, P, P, P],
    "ufc_stats_vector": [P, P, P, I32, P],
    "ufc_batched_stats": [P, I32, I32, P, P, P, P, I32, I32, P, P, D, D, I32, P, P, P, P, P, P, I32],
    "ufc_kappa_stats_noalloc": [P, P, I32, I32, P, D, D, D, I32, P, P, P],
    "ufc_map2alm": [P, P, I32, I32, P],
    "ufc_alm2cl": [P, P, I32, P],
    "ufc_cl_bin": [P, P, I32, I32, I32, I32, P],
    "ufc_alm2map": [P, P, I32, I32, P],
    "ufc_alm_beam": [P, P, I32, D, P],
    "ufc_map_stats": [P, P, I32, D, D, I32, P, P],
    "ufc_profile_enable": [P, I32],
    "ufc_profile_read": [P, I32, P, P, P, P],
    "ufc_workspace_bytes": [P, P],
    "ufc_welford_update_host": [P, I32, I32, P],
    "ufc_set_tuning": [P, P],
    "ufc_get_tuning": [P, P],
    "ufc_welford_merge_host": [P, P, I32],
    "ufc_check_selftest": [P, I64, I64],
    "ufc_kappa_partial": [P, P, I32, I32, P, P],
    "ufc_kappa_stats_partial": [P, P, I32, D, D, D, I32, P, P, P],
    "ufc_kappa_adjoint_sums": [P, P, I32, I32, P, D, P, D, D, I32, P, P, P, P],
    "ufc_kappa_grad_from_sums": [P, I32, I32, D, D, P, P, P, P, P],
}
for _name, _args in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = ctypes.c_int
_lib.ufc_last_error.argtypes = [P]
_lib.ufc_last_error.restype = ctypes.c_char_p


class UfcError(RuntimeError):
    pass


def _np_ptr(a: np.ndarray):
    return a.ctypes.data_as(P)


def _check(status: int, ctx=None, what=""):
    if status != UFC_OK:
        msg = _lib.ufc_last_error(ctx).decode() if ctx else ""
        raise UfcError(f"{what} failed with status {status}: {msg}")


# ---- host cosmology ---------------------------------------------------------------
def chi_edges(cosmo: Cosmo, z_edges) -> np.ndarray:
    """chi(z) of the shell edges (Delta chi_b of Sec. 2.4), FP64."""
    z = np.ascontiguousarray(z_edges, dtype=np.float64)
    out = np.empty_like(z)
    _check(_lib.ufc_chi_edges(ctypes.byref(cosmo), _np_ptr(z), len(z) - 1, _np_ptr(out)),
           what="ufc_chi_edges")
    return out


def z_of_chi(cosmo: Cosmo, chi) -> np.ndarray:
    c = np.ascontiguousarray(np.atleast_1d(chi), dtype=np.float64)
    out = np.empty_like(c)
    _check(_lib.ufc_z_of_chi(ctypes.byref(cosmo), _np_ptr(c), len(c), _np_ptr(out)),
           what="ufc_z_of_chi")
    return out


def snapshot_assign(z_edges, z_snap) -> np.ndarray:
    """int32 snapshot index of every shell in snapshot mode (the last snapshot
    at or below the shell's lower-edge redshift, -1 if none)."""
    z = np.ascontiguousarray(z_edges, dtype=np.float64)
    zs = np.ascontiguousarray(z_snap, dtype=np.float64)
    out = np.empty(len(z) - 1, dtype=np.int32)
    _check(_lib.ufc_snapshot_assign(_np_ptr(z), len(z) - 1, _np_ptr(zs), len(zs), _np_ptr(out)),
           what="ufc_snapshot_assign")
    return out


def delta_coeffs(cosmo: Cosmo, boxes, z_edges, nside: int, derivs=False):
    """(A, C[, dA, dC]) of the overdensity map delta_p = sum_b A_b n_bp - C
    (Eq. 7); the map and its statistics come from Context.kappa_stats."""
    z = np.ascontiguousarray(z_edges, dtype=np.float64)
    S = len(z) - 1
    arr = (Box * len(boxes))(*boxes)
    A = np.empty(S)
    C = ctypes.c_double()
    dA = np.empty((5, S)) if derivs else None
    dC = np.empty(5) if derivs else None
    _check(_lib.ufc_delta_coeffs(ctypes.byref(cosmo), ctypes.cast(arr, P), len(boxes), _np_ptr(z),
                                 S, nside, _np_ptr(A), ctypes.byref(C),
                                 _np_ptr(dA) if derivs else None,
                                 _np_ptr(dC) if derivs else None), what="ufc_delta_coeffs")
    if derivs:
        return A, C.value, dA, dC
    return A, C.value


def kappa_coeffs(cosmo: Cosmo, boxes, z_edges, nside: int, source: Source, derivs=False):
    """(A, B, C[, dA, dC]) of kappa_p = sum_b A_b n_bp - C (Eq. 6)."""
    z = np.ascontiguousarray(z_edges, dtype=np.float64)
    S = len(z) - 1
    arr = (Box * len(boxes))(*boxes)
    A, B = np.empty(S), np.empty(S)
    C = ctypes.c_double()
    dA = np.empty((5, S)) if derivs else None
    dC = np.empty(5) if derivs else None
    _check(_lib.ufc_kappa_coeffs(ctypes.byref(cosmo), ctypes.cast(arr, P), len(boxes), _np_ptr(z),
                                 S, nside, ctypes.byref(source), _np_ptr(A), _np_ptr(B),
                                 ctypes.byref(C), _np_ptr(dA) if derivs else None,
                                 _np_ptr(dC) if derivs else None), what="ufc_kappa_coeffs")
    if derivs:
        return A, B, C.value, dA, dC
    return A, B, C.value


# ---- device context ---------------------------------------------------------------
class Context:
    """A library context on one CUDA device (owns the device workspace)."""

    def __init__(self, device: int = 0):
        import torch  # noqa: F401  (device memory and streams)
        self.device = int(device)
        h = P()
        st = _lib.ufc_create(ctypes.byref(h), self.device)
        if st != UFC_OK:
            raise UfcError(f"ufc_create({device}) failed with status {st}")
        self.h = h

    def close(self):
        if self.h:
            _lib.ufc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _stream(self):
        import torch
        s = torch.cuda.current_stream(self.device).cuda_stream
        _lib.ufc_set_stream(self.h, P(s))

    def _ck(self, st, what):
        _check(st, self.h, what)

    def synchronize(self):
        self._ck(_lib.ufc_synchronize(self.h), "ufc_synchronize")

    def wait_selftest(self, limit: int = 1000):
        """Makes one device-side bounded wait run out (ufc_wait_selftest); the
        next synchronize() raises UfcError with status UFC_ERR_TIMEOUT."""
        self._stream()
        self._ck(_lib.ufc_wait_selftest(self.h, int(limit)), "ufc_wait_selftest")

    def check_selftest(self, index: int, bound: int):
        """ufc_check_selftest: one failed index test (reported by the next
        synchronize as UFC_ERR_INTERNAL)."""
        self._stream()
        self._ck(_lib.ufc_check_selftest(self.h, int(index), int(bound)), "ufc_check_selftest")

    def profile(self, on: bool = True):
        """Bracket every library kernel launch with CUDA events (tracing)."""
        self._ck(_lib.ufc_profile_enable(self.h, 1 if on else 0), "ufc_profile_enable")

    def profile_read(self) -> dict:
        """{kernel name: (total ms, launches)} since the last read (synchronises)."""
        mx = 64
        names = ctypes.create_string_buffer(32 * mx)
        ms = np.zeros(mx)
        cnt = np.zeros(mx, dtype=np.int64)
        n = ctypes.c_int32()
        self._stream()
        self._ck(_lib.ufc_profile_read(self.h, mx, names, _np_ptr(ms), _np_ptr(cnt), ctypes.byref(n)),
                 "ufc_profile_read")
        out = {}
        for i in range(min(n.value, mx)):
            nm = names.raw[32 * i:32 * i + 32].split(b"\0", 1)[0].decode()
            out[nm] = (float(ms[i]), int(cnt[i]))
        return out

    def workspace_bytes(self) -> int:
        """Device bytes the context holds (ufc_workspace_bytes)."""
        out = ctypes.c_int64()
        self._ck(_lib.ufc_workspace_bytes(self.h, ctypes.byref(out)), "ufc_workspace_bytes")
        return int(out.value)

    def reserve(self, nside: int, nshell: int, n_max: int):
        self._ck(_lib.ufc_reserve(self.h, nside, nshell, n_max), "ufc_reserve")

    # -- binning --
    def keys(self, xyz, box: Box, chi_edges, nside: int, out=None):
        import torch
        xyz = _dev_f32(xyz, self.device)
        n = xyz.numel() // 3
        if out is None:
            out = torch.empty(n, dtype=torch.int32, device=xyz.device)
        chi = np.ascontiguousarray(chi_edges, dtype=np.float64)
        self._stream()
        self._ck(_lib.ufc_keys(self.h, P(xyz.data_ptr()), n, ctypes.byref(box), _np_ptr(chi),
                               len(chi) - 1, nside, P(out.data_ptr())), "ufc_keys")
        return out

    def bin(self, xyz_list, boxes, chi_edges, nside: int, counts=None, accumulate=False,
            path: str | None = None):
        """int32 [nshell, 12 nside^2] count maps of the lightcone (Eq. 5, 8).
        path: None (the autotuner's cached choice for this shape if there is
        one, else the library's), "direct" or "dense" (UFC_BIN_FORCE_*)."""
        import torch
        chi = np.ascontiguousarray(chi_edges, dtype=np.float64)
        S = len(chi) - 1
        npix = 12 * nside * nside
        xs = [_dev_f32(x, self.device) for x in xyz_list]
        if path is None:
            from . import autotune
            path = autotune.cached_bin_path(self, nside, S, sum(x.numel() // 3 for x in xs))
        if counts is None:
            counts = torch.empty((S, npix), dtype=torch.int32, device=f"cuda:{self.device}")
        assert counts.dtype == torch.int32 and counts.is_contiguous() and counts.numel() == S * npix
        ptrs = (P * len(xs))(*[P(x.data_ptr()) for x in xs])
        ns = (I64 * len(xs))(*[x.numel() // 3 for x in xs])
        arr = (Box * len(boxes))(*boxes)
        self._stream()
        flags = _bin_flags(accumulate, path)
        self._ck(_lib.ufc_bin(self.h, ctypes.cast(ptrs, P), ctypes.cast(ns, P), ctypes.cast(arr, P),
                              len(boxes), _np_ptr(chi), S, nside, flags, P(counts.data_ptr())),
                 "ufc_bin")
        return counts

    def bin_host(self, xyz_list, boxes, chi_edges, nside: int, counts=None, accumulate=False,
                 path: str | None = None):
        """bin() with the positions in host memory (ufc_bin_host): float32
        [n, 3] CPU tensors (page-locked for overlapped copies) or numpy
        arrays.  They must stay unchanged until the stream has finished."""
        import torch
        chi = np.ascontiguousarray(chi_edges, dtype=np.float64)
        S = len(chi) - 1
        npix = 12 * nside * nside
        xs = [_host_f32(x) for x in xyz_list]
        if counts is None:
            counts = torch.empty((S, npix), dtype=torch.int32, device=f"cuda:{self.device}")
        assert counts.dtype == torch.int32 and counts.is_contiguous() and counts.numel() == S * npix
        ptrs = (P * len(xs))(*[P(a) for a, _ in xs])
        ns = (I64 * len(xs))(*[m // 3 for _, m in xs])
        arr = (Box * len(boxes))(*boxes)
        self._stream()
        self._ck(_lib.ufc_bin_host(self.h, ctypes.cast(ptrs, P), ctypes.cast(ns, P),
                                   ctypes.cast(arr, P), len(boxes), _np_ptr(chi), S, nside,
                                   _bin_flags(accumulate, path), P(counts.data_ptr())),
                 "ufc_bin_host")
        return counts

    def bin_host_stream(self, xyz_list, boxes, chi_edges, nside: int, chunk: int, counts=None,
                        accumulate=False, path: str | None = None):
        """bin_host through two device buffers of `chunk` particles
        (ufc_bin_host_stream): particle sets beyond device memory."""
        import torch
        chi = np.ascontiguousarray(chi_edges, dtype=np.float64)
        S = len(chi) - 1
        npix = 12 * nside * nside
        xs = [_host_f32(x) for x in xyz_list]
        if counts is None:
            counts = torch.empty((S, npix), dtype=torch.int32, device=f"cuda:{self.device}")
        assert counts.dtype == torch.int32 and counts.is_contiguous() and counts.numel() == S * npix
        ptrs = (P * len(xs))(*[P(a) for a, _ in xs])
        ns = (I64 * len(xs))(*[m // 3 for _, m in xs])
        arr = (Box * len(boxes))(*boxes)
        self._stream()
        self._ck(_lib.ufc_bin_host_stream(self.h, ctypes.cast(ptrs, P), ctypes.cast(ns, P),
                                          ctypes.cast(arr, P), len(boxes), _np_ptr(chi), S, nside,
                                          _bin_flags(accumulate, path), int(chunk),
                                          P(counts.data_ptr())), "ufc_bin_host_stream")
        return counts

    def bin_snapshots(self, xyz_list, geoms, snap_of_shell, chi_edges, nside: int, counts=None,
                      accumulate=False, path: str | None = None):
        """Count maps of a snapshot-mode lightcone (ufc_bin_snapshots): shell b
        from the particles xyz_list[s] of snapshot s = snap_of_shell[b], in the
        box geoms[s] (its shell range is ignored)."""
        import torch
        chi = np.ascontiguousarray(chi_edges, dtype=np.float64)
        S = len(chi) - 1
        npix = 12 * nside * nside
        sos = np.ascontiguousarray(snap_of_shell, dtype=np.int32)
        assert len(sos) == S and len(geoms) == len(xyz_list)
        xs = [_dev_f32(x, self.device) for x in xyz_list]
        if counts is None:
            counts = torch.empty((S, npix), dtype=torch.int32, device=f"cuda:{self.device}")
        assert counts.dtype == torch.int32 and counts.is_contiguous() and counts.numel() == S * npix
        ptrs = (P * len(xs))(*[P(x.data_ptr()) for x in xs])
        ns = (I64 * len(xs))(*[x.numel() // 3 for x in xs])
        arr = (Box * len(geoms))(*geoms)
        self._stream()
        self._ck(_lib.ufc_bin_snapshots(self.h, ctypes.cast(ptrs, P), ctypes.cast(ns, P),
                                        ctypes.cast(arr, P), len(geoms), _np_ptr(sos),
                                        _np_ptr(chi), S, nside, _bin_flags(accumulate, path),
                                        P(counts.data_ptr())), "ufc_bin_snapshots")
        return counts

    def bin_snapshots_host(self, xyz_list, geoms, snap_of_shell, chi_edges, nside: int,
                           chunk: int, counts=None, accumulate=False, path: str | None = None):
        """bin_snapshots with the snapshots in host memory, streamed through two
        device buffers of `chunk` particles (ufc_bin_snapshots_host)."""
        import torch
        chi = np.ascontiguousarray(chi_edges, dtype=np.float64)
        S = len(chi) - 1
        npix = 12 * nside * nside
        sos = np.ascontiguousarray(snap_of_shell, dtype=np.int32)
        assert len(sos) == S and len(geoms) == len(xyz_list)
        xs = [_host_f32(x) for x in xyz_list]
        if counts is None:
            counts = torch.empty((S, npix), dtype=torch.int32, device=f"cuda:{self.device}")
        assert counts.dtype == torch.int32 and counts.is_contiguous() and counts.numel() == S * npix
        ptrs = (P * len(xs))(*[P(a) for a, _ in xs])
        ns = (I64 * len(xs))(*[m // 3 for _, m in xs])
        arr = (Box * len(geoms))(*geoms)
        self._stream()
        self._ck(_lib.ufc_bin_snapshots_host(self.h, ctypes.cast(ptrs, P), ctypes.cast(ns, P),
                                             ctypes.cast(arr, P), len(geoms), _np_ptr(sos),
                                             _np_ptr(chi), S, nside, _bin_flags(accumulate, path),
                                             int(chunk), P(counts.data_ptr())),
                 "ufc_bin_snapshots_host")
        return counts

    def bin_info(self):
        out = np.zeros(4, dtype=np.int64)
        self._stream()
        self._ck(_lib.ufc_bin_info(self.h, _np_ptr(out)), "ufc_bin_info")
        return dict(invalid=int(out[0]), keyed=int(out[1]), refined=int(out[2]), exact=int(out[3]))

    # -- kappa, moments, PDF --
    def kappa_stats(self, counts, A, C, pdf_lo, pdf_hi, nbins=200, kappa=None, want_stats=True):
        """(kappa FP32 [npix], moments FP64 [10], pdf int64 [nbins+3]) on the device."""
        import torch
        S, npix = counts.shape
        nside = int(round((npix / 12) ** 0.5))
        dev = counts.device
        if kappa is None:
            kappa = torch.empty(npix, dtype=torch.float32, device=dev)
        mom = torch.empty(NMOMENTS, dtype=torch.float64, device=dev) if want_stats else None
        pdf = torch.empty(nbins + 3, dtype=torch.int64, device=dev) if want_stats else None
        A = np.ascontiguousarray(A, dtype=np.float64)
        self._stream()
        self._ck(_lib.ufc_kappa_stats(self.h, P(counts.data_ptr()), S, nside, _np_ptr(A), float(C),
                                      float(pdf_lo), float(pdf_hi), nbins, P(kappa.data_ptr()),
                                      P(mom.data_ptr()) if want_stats else None,
                                      P(pdf.data_ptr()) if want_stats else None),
                 "ufc_kappa_stats")
        return kappa, mom, pdf

    def kappa_backward(self, counts, A, C, dA, dC, w_var=0.0, w_skew=0.0, g_kappa=None):
        """(dL/dtheta [5], G [nshell], H) for L = w_var var + w_skew skew + <g, kappa>."""
        S, npix = counts.shape
        nside = int(round((npix / 12) ** 0.5))
        A = np.ascontiguousarray(A, dtype=np.float64)
        dA = np.ascontiguousarray(dA, dtype=np.float64)
        dC = np.ascontiguousarray(dC, dtype=np.float64)
        grad = np.empty(5)
        G = np.empty(S)
        H = ctypes.c_double()
        gp = None
        if g_kappa is not None:
            g_kappa = _dev_f32(g_kappa, self.device)
            if g_kappa.data_ptr() % 16:          # the adjoint reads g with 16-byte loads
                g_kappa = g_kappa.clone()
            gp = P(g_kappa.data_ptr())
        self._stream()
        self._ck(_lib.ufc_kappa_backward(self.h, P(counts.data_ptr()), S, nside, _np_ptr(A),
                                         float(C), float(w_var), float(w_skew), gp, _np_ptr(dA),
                                         _np_ptr(dC), _np_ptr(grad), _np_ptr(G), ctypes.byref(H)),
                 "ufc_kappa_backward")
        return grad, G, H.value

    def kappa_stats_backward(self, counts, A, C, dA, dC, pdf_lo, pdf_hi, nbins=200,
                             w_var=0.0, w_skew=0.0, g_kappa=None, kappa=None):
        """kappa_stats and kappa_backward in one read of the counts
        (ufc_kappa_stats_backward): (kappa, moments, pdf, grad [5], G, H)."""
        import torch
        S, npix = counts.shape
        nside = int(round((npix / 12) ** 0.5))
        dev = counts.device
        if kappa is None:
            kappa = torch.empty(npix, dtype=torch.float32, device=dev)
        mom = torch.empty(NMOMENTS, dtype=torch.float64, device=dev)
        pdf = torch.empty(nbins + 3, dtype=torch.int64, device=dev)
        A = np.ascontiguousarray(A, dtype=np.float64)
        dA = np.ascontiguousarray(dA, dtype=np.float64)
        dC = np.ascontiguousarray(dC, dtype=np.float64)
        grad, G, H = np.empty(5), np.empty(S), ctypes.c_double()
        gp = None
        if g_kappa is not None:
            g_kappa = _dev_f32(g_kappa, self.device)
            if g_kappa.data_ptr() % 16:
                g_kappa = g_kappa.clone()
            gp = P(g_kappa.data_ptr())
        self._stream()
        self._ck(_lib.ufc_kappa_stats_backward(
            self.h, P(counts.data_ptr()), S, nside, _np_ptr(A), float(C), float(pdf_lo),
            float(pdf_hi), nbins, float(w_var), float(w_skew), gp, _np_ptr(dA), _np_ptr(dC),
            P(kappa.data_ptr()), P(mom.data_ptr()), P(pdf.data_ptr()), _np_ptr(grad), _np_ptr(G),
            ctypes.byref(H)), "ufc_kappa_stats_backward")
        return kappa, mom, pdf, grad, G, H.value

    # -- subvolume combination (Sec. 2.4) --
    def kappa_partial(self, counts, A, out=None):
        """ufc_kappa_partial: FP64 [npix] partial sum sum_b A_b n_bp of one
        subvolume's counts (no -C), to be summed over subvolumes."""
        import torch
        S, npix = counts.shape
        nside = int(round((npix / 12) ** 0.5))
        if out is None:
            out = torch.empty(npix, dtype=torch.float64, device=counts.device)
        A = np.ascontiguousarray(A, dtype=np.float64)
        self._stream()
        self._ck(_lib.ufc_kappa_partial(self.h, P(counts.data_ptr()), S, nside, _np_ptr(A),
                                        P(out.data_ptr())), "ufc_kappa_partial")
        return out

    def kappa_stats_partial(self, partial, C, pdf_lo, pdf_hi, nbins=200, kappa=None):
        """ufc_kappa_stats_partial: (kappa, moments, pdf) of the map from the
        summed partials."""
        import torch
        npix = partial.shape[0]
        nside = int(round((npix / 12) ** 0.5))
        dev = partial.device
        if kappa is None:
            kappa = torch.empty(npix, dtype=torch.float32, device=dev)
        mom = torch.empty(NMOMENTS, dtype=torch.float64, device=dev)
        pdf = torch.empty(nbins + 3, dtype=torch.int64, device=dev)
        self._stream()
        self._ck(_lib.ufc_kappa_stats_partial(self.h, P(partial.data_ptr()), nside, float(C),
                                              float(pdf_lo), float(pdf_hi), nbins,
                                              P(kappa.data_ptr()), P(mom.data_ptr()),
                                              P(pdf.data_ptr())), "ufc_kappa_stats_partial")
        return kappa, mom, pdf

    def kappa_adjoint_sums(self, counts, partial, C, g_kappa=None, pdf_lo=None, pdf_hi=None,
                           nbins=200, kappa=None, want_map=False):
        """ufc_kappa_adjoint_sums: the adjoint sums (FP64 [4 nshell + 4], the
        per-shell part this subvolume's share) of the summed partials'
        map; with want_map also (kappa, moments, pdf) from the same read.
        Returns (sums, kappa, moments, pdf), the last three None without
        want_map."""
        import torch
        S, npix = counts.shape
        nside = int(round((npix / 12) ** 0.5))
        dev = counts.device
        sums = np.empty(4 * S + 4)
        mom = pdf = None
        if want_map:
            if kappa is None:
                kappa = torch.empty(npix, dtype=torch.float32, device=dev)
            mom = torch.empty(NMOMENTS, dtype=torch.float64, device=dev)
            pdf = torch.empty(nbins + 3, dtype=torch.int64, device=dev)
        else:
            kappa = None
        gp = None
        if g_kappa is not None:
            g_kappa = _dev_f32(g_kappa, self.device)
            if g_kappa.data_ptr() % 16:
                g_kappa = g_kappa.clone()
            gp = P(g_kappa.data_ptr())
        self._stream()
        self._ck(_lib.ufc_kappa_adjoint_sums(
            self.h, P(counts.data_ptr()), S, nside, P(partial.data_ptr()), float(C), gp,
            float(pdf_lo if want_map else 0.0), float(pdf_hi if want_map else 1.0), nbins,
            P(kappa.data_ptr()) if want_map else None, P(mom.data_ptr()) if want_map else None,
            P(pdf.data_ptr()) if want_map else None, _np_ptr(sums)), "ufc_kappa_adjoint_sums")
        return sums, kappa, mom, pdf

    # -- batched realisations --
    def set_tuning(self, batch_chunk: int = 0, batch_blocks_per_sm: int = 0):
        """ufc_set_tuning (0 = library default)."""
        t = Tuning(int(batch_chunk), int(batch_blocks_per_sm))
        self._ck(_lib.ufc_set_tuning(self.h, ctypes.byref(t)), "ufc_set_tuning")

    def get_tuning(self) -> dict:
        t = Tuning()
        self._ck(_lib.ufc_get_tuning(self.h, ctypes.byref(t)), "ufc_get_tuning")
        return dict(batch_chunk=t.batch_chunk, batch_blocks_per_sm=t.batch_blocks_per_sm)

    def batched_stats(self, xyz, boxes, chi_edges, nside, A, C, pdf_lo, pdf_hi, nbins,
                      state, graph=True, counts=None, kappa=None, launches=False):
        """Statistics of many realisations in one call (ufc_batched_stats).
        xyz[r][k]: particles of realisation r, box k; boxes[r][k]: its box;
        A [nreal, nshell], C [nreal].  Returns (moments [nreal,10],
        pdf [nreal, nbins+3], stats [nreal, 6+nbins]); updates `state`.
        launches=True: one launch sequence per realisation instead of the
        persistent kernel (UFC_BATCH_LAUNCHES).  The autotuner's cached
        tuning for this shape, if any, is applied first (autotune.tune_batch
        makes it)."""
        import torch
        nreal, nbox = len(xyz), len(xyz[0])
        if not launches:
            from . import autotune
            tuned = autotune.cached_batch_tuning(self, nside, len(chi_edges) - 1, nreal,
                                                 sum(x.numel() // 3 for row in xyz for x in row))
            if tuned:
                self.set_tuning(*tuned)
        chi = np.ascontiguousarray(chi_edges, dtype=np.float64)
        S = len(chi) - 1
        npix = 12 * nside * nside
        dev = torch.device("cuda", self.device)
        flat = [_dev_f32(x, self.device) for row in xyz for x in row]
        ptrs = (P * len(flat))(*[P(x.data_ptr()) for x in flat])
        ns = (I64 * len(flat))(*[x.numel() // 3 for x in flat])
        bx = (Box * len(flat))(*[b for row in boxes for b in row])
        A = np.ascontiguousarray(A, dtype=np.float64).reshape(nreal, S)
        C = np.ascontiguousarray(C, dtype=np.float64).reshape(nreal)
        if counts is None:
            counts = torch.empty((S, npix), dtype=torch.int32, device=dev)
        if kappa is None:
            kappa = torch.empty(npix, dtype=torch.float32, device=dev)
        mom = torch.empty((nreal, NMOMENTS), dtype=torch.float64, device=dev)
        pdf = torch.empty((nreal, nbins + 3), dtype=torch.int64, device=dev)
        stats = torch.empty((nreal, 6 + nbins), dtype=torch.float64, device=dev)
        self._stream()
        self._ck(_lib.ufc_batched_stats(self.h, nreal, nbox, ctypes.cast(ptrs, P), ctypes.cast(ns, P),
                                        ctypes.cast(bx, P), _np_ptr(chi), S, nside, _np_ptr(A),
                                        _np_ptr(C), float(pdf_lo), float(pdf_hi), nbins,
                                        P(counts.data_ptr()), P(kappa.data_ptr()), P(mom.data_ptr()),
                                        P(pdf.data_ptr()), P(stats.data_ptr()), P(state.data_ptr()),
                                        (UFC_BATCH_GRAPH if graph else 0) |
                                        (UFC_BATCH_LAUNCHES if launches else 0)),
                 "ufc_batched_stats")
        return mom, pdf, stats

    # -- full-sky power spectrum --
    def map2alm(self, m, nside: int, lmax: int, out=None):
        """complex128 a_lm [(lmax+1)(lmax+2)/2], m-major, of a FP32 RING map."""
        import torch
        m = _dev_f32(m, self.device)
        nalm = (lmax + 1) * (lmax + 2) // 2
        if out is None:
            out = torch.empty(nalm, dtype=torch.complex128, device=m.device)
        self._stream()
        self._ck(_lib.ufc_map2alm(self.h, P(m.data_ptr()), nside, lmax, P(out.data_ptr())),
                 "ufc_map2alm")
        return out

    def alm2cl(self, alm, lmax: int, out=None):
        import torch
        if out is None:
            out = torch.empty(lmax + 1, dtype=torch.float64, device=alm.device)
        self._stream()
        self._ck(_lib.ufc_alm2cl(self.h, P(alm.data_ptr()), lmax, P(out.data_ptr())), "ufc_alm2cl")
        return out

    def alm2map(self, alm, nside: int, lmax: int, out=None):
        """FP32 RING map of the real field with coefficients a_lm."""
        import torch
        if out is None:
            out = torch.empty(12 * nside * nside, dtype=torch.float32, device=alm.device)
        self._stream()
        self._ck(_lib.ufc_alm2map(self.h, P(alm.data_ptr()), nside, lmax, P(out.data_ptr())),
                 "ufc_alm2map")
        return out

    def alm_beam(self, alm, lmax: int, sigma: float, out=None):
        """a_lm times the Gaussian beam of r.m.s. radius sigma (radians)."""
        import torch
        if out is None:
            out = torch.empty_like(alm)
        self._stream()
        self._ck(_lib.ufc_alm_beam(self.h, P(alm.data_ptr()), lmax, float(sigma), P(out.data_ptr())),
                 "ufc_alm_beam")
        return out

    def map_stats(self, m, nside: int, lo: float, hi: float, nbins: int):
        """(moments [10], pdf [nbins + 3]) of an FP32 map."""
        import torch
        m = _dev_f32(m, self.device)
        mom = torch.empty(NMOMENTS, dtype=torch.float64, device=m.device)
        pdf = torch.empty(nbins + 3, dtype=torch.int64, device=m.device)
        self._stream()
        self._ck(_lib.ufc_map_stats(self.h, P(m.data_ptr()), nside, float(lo), float(hi), nbins,
                                    P(mom.data_ptr()), P(pdf.data_ptr())), "ufc_map_stats")
        return mom, pdf

    def smoothed_moments(self, m, nside: int, lmax: int, sigmas, lo: float, hi: float,
                         nbins: int):
        """Moments and PDF of the map smoothed by Gaussian beams of r.m.s.
        radii sigmas (radians): one analysis, then per scale beam + synthesis
        + statistics, all on the device."""
        alm = self.map2alm(m, nside, lmax)
        work = alm.clone()
        sm = None
        out = []
        for s in sigmas:
            self.alm_beam(alm, lmax, s, out=work)
            sm = self.alm2map(work, nside, lmax, out=sm)
            out.append(self.map_stats(sm, nside, lo, hi, nbins))
        return out

    def cl_bin(self, cl, lmax: int, lmin: int, dl: int, nbins: int, out=None):
        """Band powers: means of C_l over [lmin + b dl, lmin + (b+1) dl)."""
        import torch
        if out is None:
            out = torch.empty(nbins, dtype=torch.float64, device=cl.device)
        self._stream()
        self._ck(_lib.ufc_cl_bin(self.h, P(cl.data_ptr()), lmax, lmin, dl, nbins,
                                 P(out.data_ptr())), "ufc_cl_bin")
        return out

    # -- covariance --
    def stats_vector(self, moments, pdf, out=None):
        """(mean, mu2, mu3, mu4, skew, kurt, pdf/N) of one map, FP64 on the device."""
        import torch
        nbins = pdf.numel() - 3
        if out is None:
            out = torch.empty(6 + nbins, dtype=torch.float64, device=moments.device)
        self._stream()
        self._ck(_lib.ufc_stats_vector(self.h, P(moments.data_ptr()), P(pdf.data_ptr()), nbins,
                                       P(out.data_ptr())), "ufc_stats_vector")
        return out

    def welford_update(self, v, state):
        v = v.contiguous()
        nvec, d = v.shape
        self._stream()
        self._ck(_lib.ufc_welford_update(self.h, P(v.data_ptr()), nvec, d, P(state.data_ptr())),
                 "ufc_welford_update")

    def welford_merge(self, a, b, d):
        self._stream()
        self._ck(_lib.ufc_welford_merge(self.h, P(a.data_ptr()), P(b.data_ptr()), d),
                 "ufc_welford_merge")

    def welford_finalize(self, state, d, ddof=1):
        import torch
        dev = state.device
        mean = torch.empty(d, dtype=torch.float64, device=dev)
        cov = torch.empty((d, d), dtype=torch.float64, device=dev)
        corr = torch.empty((d, d), dtype=torch.float64, device=dev)
        self._stream()
        self._ck(_lib.ufc_welford_finalize(self.h, P(state.data_ptr()), d, ddof, P(mean.data_ptr()),
                                           P(cov.data_ptr()), P(corr.data_ptr())),
                 "ufc_welford_finalize")
        return mean, cov, corr


def welford_update_host(v: np.ndarray, state: np.ndarray):
    """ufc_welford_update on host memory: adds the rows of v [nvec, d] to a
    float64 state of 1 + d + d*d doubles (in place)."""
    v = np.ascontiguousarray(v, dtype=np.float64)
    assert state.dtype == np.float64 and state.flags.c_contiguous
    nvec, d = v.shape
    _check(_lib.ufc_welford_update_host(_np_ptr(v), nvec, d, _np_ptr(state)),
           what="ufc_welford_update_host")


def welford_merge_host(a: np.ndarray, b: np.ndarray, d: int):
    """ufc_welford_merge on host memory: state b merged into state a (in place)."""
    assert a.dtype == np.float64 and b.dtype == np.float64
    assert a.flags.c_contiguous and b.flags.c_contiguous
    _check(_lib.ufc_welford_merge_host(_np_ptr(a), _np_ptr(np.ascontiguousarray(b)), d),
           what="ufc_welford_merge_host")


def kappa_grad_from_sums(sums: np.ndarray, nshell: int, nside: int, dA, dC, w_var=0.0,
                         w_skew=0.0):
    """ufc_kappa_grad_from_sums (host only): (dL/dtheta [5], G [nshell], H)
    from adjoint sums whose per-shell part is summed over subvolumes."""
    sums = np.ascontiguousarray(sums, dtype=np.float64)
    dA = np.ascontiguousarray(dA, dtype=np.float64)
    dC = np.ascontiguousarray(dC, dtype=np.float64)
    assert sums.shape == (4 * nshell + 4,) and dA.size == 5 * nshell and dC.size == 5
    grad, G, H = np.empty(5), np.empty(nshell), ctypes.c_double()
    _check(_lib.ufc_kappa_grad_from_sums(_np_ptr(sums), nshell, nside, float(w_var),
                                         float(w_skew), _np_ptr(dA), _np_ptr(dC), _np_ptr(grad),
                                         _np_ptr(G), ctypes.byref(H)),
           what="ufc_kappa_grad_from_sums")
    return grad, G, H.value


def welford_state(d: int, device="cuda"):
    import torch
    return torch.zeros(1 + d + d * d, dtype=torch.float64, device=device)


def _bin_flags(accumulate, path):
    flags = UFC_BIN_ACCUMULATE if accumulate else 0
    if path == "direct":
        flags |= UFC_BIN_FORCE_DIRECT
    elif path == "dense":
        flags |= UFC_BIN_FORCE_DENSE
    elif path is not None:
        raise ValueError(f"unknown binning path {path!r}")
    return flags


def _host_f32(x):
    """(address, element count) of a contiguous float32 host array."""
    import torch
    if isinstance(x, torch.Tensor):
        if x.is_cuda or x.dtype != torch.float32 or not x.is_contiguous():
            raise TypeError("expected a contiguous float32 CPU tensor")
        return x.data_ptr(), x.numel()
    if isinstance(x, np.ndarray):
        if x.dtype != np.float32 or not x.flags.c_contiguous:
            raise TypeError("expected a C-contiguous float32 array")
        return x.ctypes.data, x.size
    raise TypeError("expected a float32 CPU tensor or numpy array")


def _dev_f32(x, device):
    import torch
    if not isinstance(x, torch.Tensor) or not x.is_cuda:
        raise TypeError("expected a CUDA float32 tensor")
    if x.dtype != torch.float32 or not x.is_contiguous():
        raise TypeError("expected a contiguous float32 tensor")
    return x


_ctx_lock = threading.Lock()
_ctxs: dict[int, Context] = {}


def context(device: int = 0) -> Context:
    """Process-wide default context of a device."""
    with _ctx_lock:
        if device not in _ctxs:
            _ctxs[device] = Context(device)
        return _ctxs[device]
