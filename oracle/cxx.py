"""ctypes wrapper of the C++/OpenMP CPU oracle (``oracle/cpp/snd_oracle.cpp``).

TEST INFRASTRUCTURE ONLY, like the rest of this package. The C++ oracle states the same
definitions and readings as the numpy modules here (delays, encoder, SND tree per DM with no
deduplication, direct dedispersion, matched filter, closing and labelling, streaming), in
plain loops parallelised over trial-DM rows with OpenMP, so that the full 1024-channel /
2048-DM stream can be checked cell by cell and candidate by candidate. It shares no code
with the CUDA library. ``tests/test_oracle_cxx.py`` pins it to the numpy oracle and to the
paper's invariants.

The shared library is built on first use (g++ -O3 -fopenmp -ffp-contract=off) next to its
source, or by ``__graft_entry__.build()``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "cpp", "snd_oracle.cpp")
LIB = os.path.join(HERE, "cpp", "libsnd_oracle.so")

BINARY, GRADED, FLOAT = 0, 1, 2

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle library if it is missing or older than its source."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + f".{os.getpid()}.tmp"
    cmd = ["g++", "-O3", "-std=c++17", "-fopenmp", "-fPIC", "-shared", "-ffp-contract=off", "-o", tmp, SRC]
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError("oracle build failed:\n" + " ".join(cmd) + "\n" + r.stdout)
    os.replace(tmp, LIB)
    return LIB


class _Config(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("cluster", ctypes.c_int32), ("branching", ctypes.c_int32),
                ("k_leaf", ctypes.c_int32), ("k_internal", ctypes.c_int32), ("cap", ctypes.c_int32),
                ("closing", ctypes.c_int32), ("n_min", ctypes.c_int32), ("enc_theta", ctypes.c_double),
                ("det_theta", ctypes.c_double), ("sigma_min", ctypes.c_double), ("mf_alpha", ctypes.c_double)]


CAND_DTYPE = np.dtype([("dm_index", "<i4"), ("width", "<i4"), ("npix", "<i4"), ("pad", "<i4"),
                       ("dm", "<f4"), ("snr", "<f4"), ("t", "<i8")])

_P = ctypes.c_void_p


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            i32, i64, f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
            sig = {
                "osnd_max_threads": (i32, []),
                "osnd_set_threads": (None, [i32]),
                "osnd_delay_table": (i32, [_P, i32, f64, _P, i32, _P]),
                "osnd_channel_stats": (None, [_P, i64, i64, _P]),
                "osnd_encode_chunk": (None, [_P, i32, i32, f64, _P, _P]),
                "osnd_snd_rows": (i32, [_P, i32, i64, i64, _P, _P, i32, i64, i32, i32, i32, i32, i32, i32, i32, _P]),
                "osnd_brute_rows": (i32, [_P, i32, i64, i64, _P, _P, i32, i64, i32, _P]),
                "osnd_row_widths": (i32, [_P, i32, f64, f64, f64, _P]),
                "osnd_row_mf": (None, [_P, i32, _P, i32, f64, f64, _P, _P, _P, _P]),
                "osnd_closing": (None, [_P, i32, i32, i32, _P]),
                "osnd_block_candidates": (i32, [_P, _P, _P, i32, i32, _P, i64, i32, i32, _P, i32]),
                "osnd_stream_new": (_P, [_P, i32, f64, _P, i32, _P]),
                "osnd_stream_free": (None, [_P]),
                "osnd_stream_max_delay": (i32, [_P]),
                "osnd_stream_max_width": (i32, [_P]),
                "osnd_stream_nemit": (i64, [_P, i32]),
                "osnd_stream_push": (i32, [_P, _P, i32, _P, _P, _P]),
                "osnd_stream_candidates": (i32, [_P, _P, i32]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _p(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


def max_threads() -> int:
    return int(lib().osnd_max_threads())


def set_threads(n: int) -> None:
    lib().osnd_set_threads(int(n))


def delay_table(freqs, dt: float, dms) -> np.ndarray:
    f = np.ascontiguousarray(freqs, dtype=np.float64)
    d = np.ascontiguousarray(dms, dtype=np.float64)
    out = np.zeros((d.size, f.size), dtype=np.int32)
    if lib().osnd_delay_table(_p(f), f.size, float(dt), _p(d), d.size, _p(out)) != 0:
        raise ValueError("delay out of range")
    return out


def channel_stats(values) -> tuple:
    v = np.ascontiguousarray(values, dtype=np.uint8)
    out = np.zeros(4, dtype=np.float64)
    lib().osnd_channel_stats(_p(v), v.size, 1, _p(out))
    return tuple(float(x) for x in out)


def encode_chunk(chunk, theta: float) -> tuple:
    """(x uint8[nchan][nsamp], levels int32[nchan])."""
    ch = np.ascontiguousarray(chunk, dtype=np.uint8)
    n, nchan = ch.shape
    x = np.zeros((nchan, n), dtype=np.uint8)
    lev = np.zeros(nchan, dtype=np.int32)
    lib().osnd_encode_chunk(_p(ch), n, nchan, float(theta), _p(x), _p(lev))
    return x, lev


def snd_rows(x, x_t0: int, delays, rows, t_start: int, nout: int, mode: int, cluster: int, branching: int,
             k_leaf: int = 0, k_internal: int = 0, cap: int = 255) -> np.ndarray:
    xr = np.ascontiguousarray(x, dtype=np.uint8)
    dl = np.ascontiguousarray(delays, dtype=np.int32)
    rw = np.ascontiguousarray(list(rows), dtype=np.int32)
    out = np.zeros((rw.size, max(nout, 0)), dtype=np.int32)
    rc = lib().osnd_snd_rows(_p(xr), xr.shape[0], xr.shape[1], int(x_t0), _p(dl), _p(rw), rw.size, int(t_start),
                             int(nout), int(mode), int(cluster), int(branching), int(k_leaf), int(k_internal),
                             int(cap), _p(out))
    if rc != 0:
        raise IndexError("raster does not cover the requested output times")
    return out


def brute_rows(x, x_t0: int, delays, rows, t_start: int, nout: int) -> np.ndarray:
    xr = np.ascontiguousarray(x, dtype=np.uint8)
    dl = np.ascontiguousarray(delays, dtype=np.int32)
    rw = np.ascontiguousarray(list(rows), dtype=np.int32)
    out = np.zeros((rw.size, max(nout, 0)), dtype=np.int32)
    if lib().osnd_brute_rows(_p(xr), xr.shape[0], xr.shape[1], int(x_t0), _p(dl), _p(rw), rw.size, int(t_start),
                             int(nout), _p(out)) != 0:
        raise IndexError("raster does not cover the requested output times")
    return out


def row_widths(freqs, dt: float, dm: float, alpha: float) -> list:
    f = np.ascontiguousarray(freqs, dtype=np.float64)
    w = np.zeros(16, dtype=np.int32)
    n = lib().osnd_row_widths(_p(f), f.size, float(dt), float(dm), float(alpha), _p(w))
    return [int(v) for v in w[:n]]


def row_mf(y_concat, nb: int, widths, theta: float, sigma_floor=None) -> tuple:
    """Same contract as ``oracle.mf.row_mf``: (mask, snr, width, mu, sigma)."""
    y = np.ascontiguousarray(y_concat, dtype=np.int64)
    if y.size < nb + max(widths) - 1:
        raise ValueError("row too short for its widths")
    w = np.ascontiguousarray(widths, dtype=np.int32)
    mask = np.zeros(nb, dtype=np.uint8)
    snr = np.zeros(nb, dtype=np.float64)
    wid = np.zeros(nb, dtype=np.int32)
    ms = np.zeros(2, dtype=np.float64)
    lib().osnd_row_mf(_p(y), int(nb), _p(w), w.size, float(theta), -1.0 if sigma_floor is None else float(sigma_floor),
                      _p(mask), _p(snr), _p(wid), _p(ms))
    return mask.astype(bool), snr, wid.astype(np.int64), float(ms[0]), float(ms[1])


def closing(mask, size: int = 9) -> np.ndarray:
    m = np.ascontiguousarray(mask, dtype=np.uint8)
    out = np.zeros_like(m)
    lib().osnd_closing(_p(m), m.shape[0], m.shape[1], int(size), _p(out))
    return out.astype(bool)


def _cand_list(arr) -> list:
    return [(int(c["dm_index"]), np.float32(c["dm"]), int(c["t"]), np.float32(c["snr"]), int(c["width"]),
             int(c["npix"])) for c in arr]


def block_candidates(mask, snr, width, dms, t_base: int, size: int = 9, n_min: int = 10) -> list:
    """Same contract as ``oracle.candidates.block_candidates``."""
    m = np.ascontiguousarray(mask, dtype=np.uint8)
    s = np.ascontiguousarray(snr, dtype=np.float64)
    w = np.ascontiguousarray(width, dtype=np.int32)
    d = np.ascontiguousarray(dms, dtype=np.float64)
    h, wd = m.shape
    cap = 1024
    while True:
        out = np.zeros(cap, dtype=CAND_DTYPE)
        n = lib().osnd_block_candidates(_p(m), _p(s), _p(w), h, wd, _p(d), int(t_base), int(size), int(n_min),
                                        _p(out), cap)
        if n <= cap:
            return _cand_list(out[:n])
        cap = n


class Stream:
    """The whole hot path on the CPU, chunk by chunk, with the contract of
    ``oracle.stream.OracleStream.push`` (keys levels, e_prev, e_new, plane, f_prev, nb,
    candidates, and plane_float in Mode C; no mask/snr/width arrays)."""

    def __init__(self, freqs, dt: float, dms, cfg):
        self.freqs = np.ascontiguousarray(freqs, dtype=np.float64)
        self.dms = np.ascontiguousarray(dms, dtype=np.float64)
        self.nchan = self.freqs.size
        self.cfg = cfg
        c = _Config(cfg.mode, cfg.cluster, cfg.branching, cfg.k_leaf, cfg.k_internal, cfg.cap, cfg.closing, cfg.n_min,
                    cfg.enc_theta, cfg.det_theta, cfg.sigma_min, cfg.mf_alpha)
        self._h = lib().osnd_stream_new(_p(self.freqs), self.nchan, float(dt), _p(self.dms), self.dms.size,
                                        ctypes.byref(c))
        if not self._h:
            raise ValueError("oracle stream rejected its configuration")
        self.D = int(lib().osnd_stream_max_delay(self._h))
        self.wmax = int(lib().osnd_stream_max_width(self._h))
        self._ncand = 0

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.osnd_stream_free(h)
            self._h = None

    def nemit_next(self, nsamp: int) -> int:
        return int(lib().osnd_stream_nemit(self._h, int(nsamp)))

    def push(self, chunk, want_plane: bool = True) -> dict:
        ch = np.ascontiguousarray(chunk, dtype=np.uint8)
        nout = self.nemit_next(ch.shape[0])
        plane = np.zeros((self.dms.size, max(nout, 0)), dtype=np.int32) if want_plane else None
        lev = np.zeros(self.nchan, dtype=np.int32)
        info = np.zeros(5, dtype=np.int64)
        rc = lib().osnd_stream_push(self._h, _p(ch), ch.shape[0], _p(plane) if nout > 0 else None, _p(lev), _p(info))
        if rc != 0:
            raise RuntimeError("oracle stream push failed")
        e_prev, e_new, f_prev, nb, nc = (int(v) for v in info)
        total = self._ncand + nc
        out = np.zeros(max(total, 1), dtype=CAND_DTYPE)
        got = lib().osnd_stream_candidates(self._h, _p(out), max(total, 1))
        assert got == total
        cands = _cand_list(out[self._ncand:total])
        self._ncand = total
        r = dict(levels=lev.astype(np.int64), e_prev=e_prev, e_new=e_new, f_prev=f_prev, nb=nb, candidates=cands,
                 plane=plane)
        if want_plane and self.cfg.mode == FLOAT:
            r["plane_float"] = plane.astype(np.float64) / np.sqrt(float(self.nchan))
        return r
