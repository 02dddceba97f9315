"""Plain, slow FP64 CPU oracle for the UFalcon lightcone hot path.

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may use it; the library product never does.
It shares no code with the CUDA library.  The C sources here are compiled with
``-O2 -ffp-contract=off`` so that every floating-point step is one IEEE
binary64 operation in the written order.

Sections of Sgier et al. followed: Sec. 2.3 (Eq. 1-7), Sec. 2.4 (Eq. 8,
nesting, HEALPix), Sec. 3.2 (Eq. 10-11) and Sec. 3.3 (Eq. 12-13, PDF).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SOURCES = ["healpix.c", "lightcone.c", "cosmo.c", "stats.c", "sht.c"]
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, no contraction, no fast-math)."""
    srcs = [os.path.join(_HERE, s) for s in _SOURCES] + [os.path.join(_HERE, "oracle.h")]
    newest = max(os.path.getmtime(s) for s in srcs)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= newest:
        return _LIB_PATH
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-fopenmp", "-std=c11", "-o", tmp] + [os.path.join(_HERE, s) for s in _SOURCES] + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Box(ctypes.Structure):
    """or_box: a simulation box of the nesting scheme (Sec. 2.4, Table 1)."""
    _fields_ = [("L", ctypes.c_double), ("obs", ctypes.c_double * 3),
                ("n_total", ctypes.c_int64), ("shell_lo", ctypes.c_int32),
                ("shell_hi", ctypes.c_int32), ("replicate", ctypes.c_int32)]


class Source(ctypes.Structure):
    """or_source: kind 0 = single source plane at z_s, 1 = n(z)."""
    _fields_ = [("kind", ctypes.c_int32), ("z_s", ctypes.c_double),
                ("alpha", ctypes.c_double), ("beta", ctypes.c_double),
                ("z0", ctypes.c_double), ("z_max", ctypes.c_double)]


def make_box(L, obs, n_total, shell_lo, shell_hi, replicate=0) -> Box:
    b = Box()
    b.L = float(L)
    for i in range(3):
        b.obs[i] = float(obs[i])
    b.n_total = int(n_total)
    b.shell_lo, b.shell_hi, b.replicate = int(shell_lo), int(shell_hi), int(replicate)
    return b


def make_source(kind=0, z_s=1.5, alpha=2.0, beta=1.5, z0=0.5, z_max=1.5) -> Source:
    s = Source()
    s.kind, s.z_s, s.alpha, s.beta, s.z0, s.z_max = int(kind), z_s, alpha, beta, z0, z_max
    return s


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            _declare(_lib)
        return _lib


P = ctypes.c_void_p
D = ctypes.c_double
I32 = ctypes.c_int32
I64 = ctypes.c_int64


def _declare(L):
    sig = {
        "or_nside2npix": (I64, [I64]),
        "or_vec2pix_ring": (I64, [I64, D, D, D, D]),
        "or_azimuth_t": (D, [D, D]),
        "or_vec2pix_batch": (None, [I64, P, I64, P]),
        "or_pix2ang_ring": (None, [I64, I64, P, P]),
        "or_keys": (None, [P, I64, P, P, I32, I64, P]),
        "or_bin": (I64, [P, I64, P, P, I32, I64, P]),
        "or_bin_omp": (I64, [P, I64, P, P, I32, I64, P, P]),
        "or_snapshot_assign": (None, [P, I32, P, I32, P]),
        "or_bin_snapshots": (I64, [P, P, P, P, P, I32, I64, P]),
        "or_comoving_distance": (D, [D, D, ctypes.c_int, D]),
        "or_chi_edges": (None, [D, D, ctypes.c_int, P, I32, P]),
        "or_z_of_chi": (D, [D, D, ctypes.c_int, D]),
        "or_shell_weights": (None, [D, P, I32, P, P]),
        "or_kappa_coeffs": (None, [D, D, ctypes.c_int, ctypes.c_int, P, I32, P, I32, I64, P, P, P, P]),
        "or_delta_coeffs": (None, [D, D, ctypes.c_int, ctypes.c_int, P, I32, P, I32, I64, P, P]),
        "or_alm_index": (I64, [I32, I32, I32]),
        "or_lambda_lm": (None, [D, D, I32, P]),
        "or_map2alm": (None, [P, I64, I32, P, P]),
        "or_alm2cl": (None, [P, P, I32, P]),
        "or_alm2map": (None, [P, P, I64, I32, P]),
        "or_gauss_beam": (None, [D, I32, P]),
        "or_kappa_map": (None, [P, I32, I64, P, D, P]),
        "or_moments": (None, [P, I64, P]),
        "or_pdf": (None, [P, I64, D, D, I32, P]),
        "or_covariance": (None, [P, I64, I32, I32, P, P, P]),
        "or_kappa_stat_grads": (None, [P, I32, I64, D, D, ctypes.c_int, P, I32, P, P, P, P]),
        "or_kappa_stats_f64": (None, [P, I32, I64, D, D, ctypes.c_int, P, I32, P, P, P, P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _boxes(boxes):
    arr = (Box * len(boxes))(*boxes)
    return arr, ctypes.cast(arr, ctypes.c_void_p)


# ---- HEALPix ------------------------------------------------------------------
def nside2npix(nside: int) -> int:
    return 12 * nside * nside


def vec2pix(nside: int, dx: float, dy: float, dz: float) -> int:
    """RING pixel of one observer-relative FP64 vector (fixed FP64 procedure)."""
    r = float(np.sqrt((dx * dx + dy * dy) + dz * dz))
    return int(lib().or_vec2pix_ring(nside, dx, dy, dz, r))


def vec2pix_many(nside: int, d: np.ndarray) -> np.ndarray:
    d = np.ascontiguousarray(d, dtype=np.float64).reshape(-1, 3)
    out = np.empty(len(d), dtype=np.int64)
    lib().or_vec2pix_batch(nside, _ptr(d), len(d), _ptr(out))
    return out


def azimuth_t(dx: float, dy: float) -> float:
    return float(lib().or_azimuth_t(dx, dy))


def pix2ang(nside: int, pix: int):
    z = ctypes.c_double()
    phi = ctypes.c_double()
    lib().or_pix2ang_ring(nside, pix, ctypes.byref(z), ctypes.byref(phi))
    return z.value, phi.value


def pix2vec(nside: int, pix: int) -> np.ndarray:
    z, phi = pix2ang(nside, pix)
    s = np.sqrt((1.0 - z) * (1.0 + z))
    return np.array([s * np.cos(phi), s * np.sin(phi), z])


# ---- lightcone ------------------------------------------------------------------
def keys(xyz: np.ndarray, box: Box, chi_edges: np.ndarray, nside: int) -> np.ndarray:
    xyz = np.ascontiguousarray(xyz, dtype=np.float32).reshape(-1, 3)
    chi = np.ascontiguousarray(chi_edges, dtype=np.float64)
    out = np.empty(len(xyz), dtype=np.int64)
    lib().or_keys(_ptr(xyz), len(xyz), ctypes.byref(box), _ptr(chi), len(chi) - 1, nside, _ptr(out))
    return out


def bin_counts(xyz: np.ndarray, box: Box, chi_edges: np.ndarray, nside: int,
               counts: np.ndarray | None = None):
    """Per-shell count maps int32[nshell, npix] (Eq. 5, Eq. 8); returns (counts, n_invalid)."""
    xyz = np.ascontiguousarray(xyz, dtype=np.float32).reshape(-1, 3)
    chi = np.ascontiguousarray(chi_edges, dtype=np.float64)
    nshell = len(chi) - 1
    if counts is None:
        counts = np.zeros((nshell, nside2npix(nside)), dtype=np.int32)
    assert counts.dtype == np.int32 and counts.flags.c_contiguous
    inv = lib().or_bin(_ptr(xyz), len(xyz), ctypes.byref(box), _ptr(chi), nshell, nside, _ptr(counts))
    return counts, int(inv)


def bin_counts_omp(xyz: np.ndarray, box: Box, chi_edges: np.ndarray, nside: int,
                   counts: np.ndarray | None = None):
    """bin_counts on all host cores (OpenMP); returns (counts, n_invalid, threads)."""
    xyz = np.ascontiguousarray(xyz, dtype=np.float32).reshape(-1, 3)
    chi = np.ascontiguousarray(chi_edges, dtype=np.float64)
    nshell = len(chi) - 1
    if counts is None:
        counts = np.zeros((nshell, nside2npix(nside)), dtype=np.int32)
    assert counts.dtype == np.int32 and counts.flags.c_contiguous
    th = np.zeros(1, dtype=np.int32)
    inv = lib().or_bin_omp(_ptr(xyz), len(xyz), ctypes.byref(box), _ptr(chi), nshell, nside,
                           _ptr(counts), _ptr(th))
    return counts, int(inv), int(th[0])


def snapshot_assign(z_edges, z_snap) -> np.ndarray:
    """Snapshot of each shell in snapshot mode (Sec. 2.1, 2.4), -1 if none."""
    z = np.ascontiguousarray(z_edges, dtype=np.float64)
    zs = np.ascontiguousarray(z_snap, dtype=np.float64)
    out = np.empty(len(z) - 1, dtype=np.int32)
    lib().or_snapshot_assign(_ptr(z), len(z) - 1, _ptr(zs), len(zs), _ptr(out))
    return out


def bin_snapshots(xyz_list, geoms, snap_of_shell, chi_edges, nside: int):
    """Count maps int32[nshell, npix] of a snapshot-mode lightcone: shell b
    from the particles of snapshot snap_of_shell[b]; returns (counts, n_invalid)."""
    xs = [np.ascontiguousarray(x, dtype=np.float32).reshape(-1, 3) for x in xyz_list]
    chi = np.ascontiguousarray(chi_edges, dtype=np.float64)
    nshell = len(chi) - 1
    sos = np.ascontiguousarray(snap_of_shell, dtype=np.int32)
    assert len(sos) == nshell and len(geoms) == len(xs)
    counts = np.zeros((nshell, nside2npix(nside)), dtype=np.int32)
    ptrs = (ctypes.c_void_p * len(xs))(*[x.ctypes.data for x in xs])
    ns = np.array([len(x) for x in xs], dtype=np.int64)
    arr = (Box * len(geoms))(*geoms)
    inv = lib().or_bin_snapshots(ctypes.cast(ptrs, ctypes.c_void_p), _ptr(ns),
                                 ctypes.cast(arr, ctypes.c_void_p), _ptr(sos), _ptr(chi), nshell,
                                 nside, _ptr(counts))
    return counts, int(inv)


# ---- cosmology -------------------------------------------------------------------
def comoving_distance(omega_m, h, units_mpc_over_h, z) -> float:
    return float(lib().or_comoving_distance(omega_m, h, units_mpc_over_h, z))


def chi_edges(omega_m, h, units_mpc_over_h, z_edges) -> np.ndarray:
    z = np.ascontiguousarray(z_edges, dtype=np.float64)
    out = np.empty_like(z)
    lib().or_chi_edges(omega_m, h, units_mpc_over_h, _ptr(z), len(z) - 1, _ptr(out))
    return out


def z_of_chi(omega_m, h, units_mpc_over_h, chi) -> float:
    return float(lib().or_z_of_chi(omega_m, h, units_mpc_over_h, chi))


def shell_weights(omega_m, z_edges, src: Source) -> np.ndarray:
    z = np.ascontiguousarray(z_edges, dtype=np.float64)
    out = np.empty(len(z) - 1)
    lib().or_shell_weights(omega_m, _ptr(z), len(z) - 1, ctypes.byref(src), _ptr(out))
    return out


def kappa_coeffs(omega_m, h, units_mpc_over_h, boxes, z_edges, nside, src, dens_volume=0):
    z = np.ascontiguousarray(z_edges, dtype=np.float64)
    ns = len(z) - 1
    A, B, C = np.empty(ns), np.empty(ns), ctypes.c_double()
    arr, bp = _boxes(boxes)
    lib().or_kappa_coeffs(omega_m, h, units_mpc_over_h, dens_volume, bp, len(boxes), _ptr(z), ns,
                          nside, ctypes.byref(src), _ptr(A), _ptr(B), ctypes.byref(C))
    return A, B, C.value


def delta_coeffs(omega_m, h, units_mpc_over_h, boxes, z_edges, nside, dens_volume=0):
    """(A, C) of the overdensity map delta_p = sum_b A_b n_bp - C (Eq. 7);
    the map itself is kappa_map(counts, A, C)."""
    z = np.ascontiguousarray(z_edges, dtype=np.float64)
    ns = len(z) - 1
    A, C = np.empty(ns), ctypes.c_double()
    arr, bp = _boxes(boxes)
    lib().or_delta_coeffs(omega_m, h, units_mpc_over_h, dens_volume, bp, len(boxes), _ptr(z), ns,
                          nside, _ptr(A), ctypes.byref(C))
    return A, C.value


# ---- spherical-harmonic analysis --------------------------------------------------
def alm_size(lmax: int) -> int:
    return (lmax + 1) * (lmax + 2) // 2


def alm_index(lmax: int, l: int, m: int) -> int:
    """m-major index of a_lm: m (2 lmax + 1 - m) / 2 + l."""
    return int(lib().or_alm_index(lmax, l, m))


def lambda_lm(z: float, lmax: int) -> np.ndarray:
    """Orthonormal associated Legendre functions lambda_lm(z) (m-major)."""
    out = np.empty(alm_size(lmax))
    lib().or_lambda_lm(float(z), float(np.sqrt((1.0 - z) * (1.0 + z))), lmax, _ptr(out))
    return out


def map2alm(m: np.ndarray, nside: int, lmax: int) -> np.ndarray:
    """complex128 a_lm (m-major) of a RING map by the direct sum over pixels."""
    mp = np.ascontiguousarray(m, dtype=np.float32)
    re, im = np.empty(alm_size(lmax)), np.empty(alm_size(lmax))
    lib().or_map2alm(_ptr(mp), nside, lmax, _ptr(re), _ptr(im))
    return re + 1j * im


def alm2map(alm: np.ndarray, nside: int, lmax: int) -> np.ndarray:
    """FP64 RING map of the real field with coefficients a_lm (m >= 0)."""
    re = np.ascontiguousarray(alm.real, dtype=np.float64)
    im = np.ascontiguousarray(alm.imag, dtype=np.float64)
    out = np.empty(12 * nside * nside)
    lib().or_alm2map(_ptr(re), _ptr(im), nside, lmax, _ptr(out))
    return out


def gauss_beam(sigma: float, lmax: int) -> np.ndarray:
    out = np.empty(lmax + 1)
    lib().or_gauss_beam(float(sigma), lmax, _ptr(out))
    return out


def alm2cl(alm: np.ndarray, lmax: int) -> np.ndarray:
    re = np.ascontiguousarray(alm.real, dtype=np.float64)
    im = np.ascontiguousarray(alm.imag, dtype=np.float64)
    out = np.empty(lmax + 1)
    lib().or_alm2cl(_ptr(re), _ptr(im), lmax, _ptr(out))
    return out


# ---- statistics --------------------------------------------------------------------
def kappa_map(counts: np.ndarray, A: np.ndarray, C: float) -> np.ndarray:
    counts = np.ascontiguousarray(counts, dtype=np.int32)
    ns, npix = counts.shape
    A = np.ascontiguousarray(A, dtype=np.float64)
    out = np.empty(npix, dtype=np.float32)
    lib().or_kappa_map(_ptr(counts), ns, npix, _ptr(A), C, _ptr(out))
    return out


def moments(kappa: np.ndarray) -> np.ndarray:
    k = np.ascontiguousarray(kappa, dtype=np.float32)
    out = np.empty(10)
    lib().or_moments(_ptr(k), len(k), _ptr(out))
    return out


def pdf(kappa: np.ndarray, lo: float, hi: float, nbins: int) -> np.ndarray:
    k = np.ascontiguousarray(kappa, dtype=np.float32)
    out = np.empty(nbins + 3, dtype=np.int64)
    lib().or_pdf(_ptr(k), len(k), lo, hi, nbins, _ptr(out))
    return out


def covariance(v: np.ndarray, ddof: int = 1):
    v = np.ascontiguousarray(v, dtype=np.float64)
    R, d = v.shape
    mean, cov, corr = np.empty(d), np.empty((d, d)), np.empty((d, d))
    lib().or_covariance(_ptr(v), R, d, ddof, _ptr(mean), _ptr(cov), _ptr(corr))
    return mean, cov, corr


def kappa_stat_grads(counts, nside, omega_m, h, units_mpc_over_h, boxes, z_edges, src, g=None):
    """Complex-step d(var, skew, <g,kappa>)/d(omega_m, h, alpha, beta, z0), shape [3, 5]."""
    counts = np.ascontiguousarray(counts, dtype=np.int32)
    z = np.ascontiguousarray(z_edges, dtype=np.float64)
    out = np.empty((3, 5))
    arr, bp = _boxes(boxes)
    gp = None
    if g is not None:
        g = np.ascontiguousarray(g, dtype=np.float32)
        gp = _ptr(g)
    lib().or_kappa_stat_grads(_ptr(counts), counts.shape[0], nside, omega_m, h, units_mpc_over_h,
                              bp, len(boxes), _ptr(z), ctypes.byref(src), gp, _ptr(out))
    return out


def kappa_stats_f64(counts, nside, omega_m, h, units_mpc_over_h, boxes, z_edges, src, g=None):
    """(var, skew, <g,kappa>) of the unrounded FP64 map."""
    counts = np.ascontiguousarray(counts, dtype=np.int32)
    z = np.ascontiguousarray(z_edges, dtype=np.float64)
    out = np.empty(3)
    arr, bp = _boxes(boxes)
    gp = None
    if g is not None:
        g = np.ascontiguousarray(g, dtype=np.float32)
        gp = _ptr(g)
    lib().or_kappa_stats_f64(_ptr(counts), counts.shape[0], nside, omega_m, h, units_mpc_over_h,
                             bp, len(boxes), _ptr(z), ctypes.byref(src), gp, _ptr(out))
    return out
