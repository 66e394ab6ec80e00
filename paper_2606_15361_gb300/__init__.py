"""Python binding of the GB300 SND library (``libsnd.so``, C ABI in ``include/snd.h``).

Argument marshalling only: every step of the hot path runs in the library's CUDA kernels.
PyTorch supplies device memory (the workspace, chunks and planes) and streams. Importing
this module loads the in-tree library and fails loudly if it has not been built; there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsnd.so")

MODE_BINARY, MODE_GRADED, MODE_FLOAT, MODE_ZFLOAT = 0, 1, 2, 3
FLAG_REFERENCE_TREE = 1
FLAG_FP16_PARTIALS = 2
FLAG_LEAF_SHARING = 4
FLAG_UNIT_PAYLOAD = 16
FLAG_LEVEL_RATES = 32
TREE_KERNELS = {0: "leaf-sharing k_tree", 1: "direct k_snd", 2: "reference k_tree_ref", 3: "labelled-payload k_tree_z"}

STATUS = {
    0: "SND_OK", -1: "SND_ERR_ARG", -2: "SND_ERR_FREQ_ORDER", -3: "SND_ERR_DM",
    -4: "SND_ERR_WORKSPACE", -5: "SND_ERR_CHUNK", -6: "SND_ERR_CUDA", -7: "SND_ERR_STATE",
    -8: "SND_ERR_TIMEOUT", -9: "SND_ERR_OVERFLOW", -10: "SND_ERR_NOMEM", -11: "SND_ERR_UNSUPPORTED",
}
ERR = {v: k for k, v in STATUS.items()}


class SndOptions(ctypes.Structure):
    _fields_ = [
        ("cluster_size", ctypes.c_int32), ("k_leaf", ctypes.c_int32), ("k_internal", ctypes.c_int32),
        ("graded_cap", ctypes.c_int32), ("enc_theta", ctypes.c_double), ("det_theta", ctypes.c_double),
        ("sigma_min", ctypes.c_double), ("mf_alpha", ctypes.c_double), ("closing_size", ctypes.c_int32),
        ("n_min_pixels", ctypes.c_int32), ("max_chunk", ctypes.c_int32), ("cand_capacity", ctypes.c_int32),
        ("cell_capacity", ctypes.c_int32), ("run_capacity", ctypes.c_int32), ("flags", ctypes.c_int32),
        ("plane_dtype", ctypes.c_int32), ("tree_warps", ctypes.c_int32), ("tree_round", ctypes.c_int32),
    ]


class SndCandidate(ctypes.Structure):
    _fields_ = [("dm_index", ctypes.c_int32), ("dm", ctypes.c_float), ("t", ctypes.c_int64),
                ("snr", ctypes.c_float), ("width", ctypes.c_int32), ("npix", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class SndPlanStats(ctypes.Structure):
    _fields_ = [
        ("nchan", ctypes.c_int32), ("ndm", ctypes.c_int32), ("mode", ctypes.c_int32),
        ("branching", ctypes.c_int32), ("cluster_size", ctypes.c_int32), ("max_delay", ctypes.c_int32),
        ("nlevels", ctypes.c_int32), ("nodes_per_level", ctypes.c_int32 * 24),
        ("unique_per_level", ctypes.c_int64 * 24), ("adds_per_dm_sample", ctypes.c_double),
        ("wmax", ctypes.c_int32), ("ring_words", ctypes.c_int32), ("hist_mem_bytes", ctypes.c_int64),
        ("workspace_bytes", ctypes.c_size_t), ("samples_in", ctypes.c_int64), ("emitted", ctypes.c_int64),
        ("scored", ctypes.c_int64), ("candidates_pending", ctypes.c_int32), ("tree_tile_dms", ctypes.c_int32),
        ("tree_tile_words", ctypes.c_int32), ("tree_group_leaves", ctypes.c_int32),
        ("tree_smem_bytes", ctypes.c_int32), ("max_patterns_per_group", ctypes.c_int32),
        ("kernel_launches", ctypes.c_int64), ("tree_kernel", ctypes.c_int32), ("device_status", ctypes.c_int32),
    ]


CANDIDATE_DTYPE = np.dtype([("dm_index", "<i4"), ("dm", "<f4"), ("t", "<i8"), ("snr", "<f4"),
                            ("width", "<i4"), ("npix", "<i4"), ("reserved", "<i4")])
assert CANDIDATE_DTYPE.itemsize == ctypes.sizeof(SndCandidate) == 32

EXPORTS = ("snd_options_init", "snd_plan", "snd_plan_ex", "snd_workspace_size", "snd_bind_workspace",
           "snd_execute", "snd_execute_host", "snd_candidates", "snd_plan_stats", "snd_delay_table",
           "snd_profile", "snd_profile_read", "snd_encode_static", "snd_debug_fail_host_alloc", "snd_debug_loop_limit", "snd_level_rates",
           "snd_destroy",
           "snd_error_string",
           "snd_multirate_plan", "snd_multirate_info", "snd_multirate_band_plan", "snd_multirate_workspace_size",
           "snd_multirate_bind_workspace", "snd_multirate_execute", "snd_multirate_execute_host",
           "snd_multirate_candidates", "snd_multirate_destroy", "snd_multirate_set_graph",
           "snd_sifter_create", "snd_sifter_num_params", "snd_sifter_workspace_size", "snd_sifter_bind_workspace",
           "snd_sifter_set_params", "snd_sifter_get_params", "snd_sifter_forward", "snd_sifter_gradients",
           "snd_sifter_train_step", "snd_sifter_status", "snd_sifter_launches", "snd_sifter_destroy", "snd_snippets",
           "snd_gemm_bf16", "snd_batch_create", "snd_batch_set_graph", "snd_batch_execute", "snd_batch_graph_stats",
           "snd_batch_destroy")
STAGES = ("encode", "tree", "mf", "candidates")


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libsnd.so not built at {LIB_PATH}: run __graft_entry__.build()")
    lib = ctypes.CDLL(LIB_PATH)
    P, I32, I64, D, SZ, V = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double,
                             ctypes.c_size_t, ctypes.c_void_p)
    dp = ctypes.POINTER(ctypes.c_double)
    lib.snd_options_init.argtypes = [I32, ctypes.POINTER(SndOptions)]
    lib.snd_plan.argtypes = [dp, I32, D, dp, I32, I32, I32, ctypes.POINTER(P)]
    lib.snd_plan_ex.argtypes = [dp, I32, D, dp, I32, I32, I32, ctypes.POINTER(SndOptions), ctypes.POINTER(P)]
    lib.snd_workspace_size.argtypes = [P]
    lib.snd_workspace_size.restype = SZ
    lib.snd_bind_workspace.argtypes = [P, V, SZ, V]
    lib.snd_execute.argtypes = [P, V, I32, V, V, ctypes.POINTER(I32)]
    lib.snd_execute_host.argtypes = [P, V, I32, V, V, ctypes.POINTER(I32)]
    lib.snd_candidates.argtypes = [P, ctypes.POINTER(SndCandidate), I32, ctypes.POINTER(I32)]
    lib.snd_plan_stats.argtypes = [P, ctypes.POINTER(SndPlanStats)]
    lib.snd_delay_table.argtypes = [P, ctypes.POINTER(ctypes.c_int32), I64]
    lib.snd_profile.argtypes = [P, ctypes.c_int]
    lib.snd_profile_read.argtypes = [P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)]
    lib.snd_encode_static.argtypes = [V, I32, I32, D, V, V]
    lib.snd_debug_fail_host_alloc.argtypes = [I32]
    lib.snd_debug_loop_limit.argtypes = [P, I64, I64]
    lib.snd_level_rates.argtypes = [P, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_double), I32,
                                    ctypes.POINTER(I32)]
    lib.snd_level_rates.restype = ctypes.c_int
    lib.snd_debug_loop_limit.restype = ctypes.c_int
    lib.snd_debug_fail_host_alloc.restype = ctypes.c_int
    lib.snd_destroy.argtypes = [P]
    lib.snd_destroy.restype = None
    lib.snd_error_string.argtypes = [ctypes.c_int]
    lib.snd_error_string.restype = ctypes.c_char_p
    ip = ctypes.POINTER(I32)
    lib.snd_multirate_plan.argtypes = [dp, I32, D, dp, I32, I32, I32, ctypes.POINTER(SndOptions), I32,
                                       ctypes.POINTER(P)]
    lib.snd_multirate_info.argtypes = [P, ip, ip, ip, I32]
    lib.snd_multirate_band_plan.argtypes = [P, I32, ctypes.POINTER(P)]
    lib.snd_multirate_workspace_size.argtypes = [P]
    lib.snd_multirate_workspace_size.restype = SZ
    lib.snd_multirate_bind_workspace.argtypes = [P, V, SZ, V]
    lib.snd_multirate_execute.argtypes = [P, V, I32, V]
    lib.snd_multirate_execute_host.argtypes = [P, V, I32, V]
    lib.snd_multirate_candidates.argtypes = [P, ctypes.POINTER(SndCandidate), I32, ip]
    lib.snd_multirate_set_graph.argtypes = [P, I32]
    lib.snd_multirate_set_graph.restype = ctypes.c_int
    lib.snd_multirate_destroy.argtypes = [P]
    lib.snd_multirate_destroy.restype = None
    fp = ctypes.POINTER(ctypes.c_float)
    lib.snd_sifter_create.argtypes = [I32, I32, ctypes.c_uint64, ctypes.POINTER(P)]
    lib.snd_sifter_num_params.argtypes = []
    lib.snd_sifter_num_params.restype = I64
    lib.snd_sifter_workspace_size.argtypes = [P]
    lib.snd_sifter_workspace_size.restype = SZ
    lib.snd_sifter_bind_workspace.argtypes = [P, V, SZ, V]
    lib.snd_sifter_set_params.argtypes = [P, fp, I64, V]
    lib.snd_sifter_get_params.argtypes = [P, fp, I64]
    lib.snd_sifter_forward.argtypes = [P, V, I32, V, V]
    lib.snd_sifter_gradients.argtypes = [P, V, V, I32, V, V, V]
    lib.snd_sifter_train_step.argtypes = [P, V, V, I32, ctypes.c_float, V, V]
    lib.snd_sifter_status.argtypes = [P]
    lib.snd_sifter_launches.argtypes = [P]
    lib.snd_sifter_launches.restype = I64
    lib.snd_sifter_destroy.argtypes = [P]
    lib.snd_sifter_destroy.restype = None
    lib.snd_snippets.argtypes = [V, I64, I32, I64, V, V, I32, V, V]
    lib.snd_gemm_bf16.argtypes = [V, I64, V, I64, I32, I32, I64, V, I64, I32, V, V]
    lib.snd_batch_create.argtypes = [ctypes.POINTER(P), I32, ctypes.POINTER(P)]
    lib.snd_batch_set_graph.argtypes = [P, I32]
    lib.snd_batch_execute.argtypes = [P, ctypes.POINTER(P), ctypes.POINTER(I32), V]
    lib.snd_batch_graph_stats.argtypes = [P, ctypes.POINTER(I64), ctypes.POINTER(I64)]
    lib.snd_batch_destroy.argtypes = [P]
    lib.snd_batch_destroy.restype = None
    for name in ("snd_batch_create", "snd_batch_set_graph", "snd_batch_execute", "snd_batch_graph_stats"):
        getattr(lib, name).restype = ctypes.c_int
    for name in ("snd_sifter_create", "snd_sifter_bind_workspace", "snd_sifter_set_params", "snd_sifter_get_params",
                 "snd_sifter_forward", "snd_sifter_gradients", "snd_sifter_train_step", "snd_sifter_status",
                 "snd_snippets", "snd_gemm_bf16"):
        getattr(lib, name).restype = ctypes.c_int
    for name in ("snd_options_init", "snd_plan", "snd_plan_ex", "snd_bind_workspace", "snd_execute",
                 "snd_execute_host", "snd_candidates", "snd_plan_stats", "snd_delay_table", "snd_profile",
                 "snd_profile_read", "snd_encode_static", "snd_multirate_plan", "snd_multirate_info",
                 "snd_multirate_band_plan", "snd_multirate_bind_workspace", "snd_multirate_execute",
                 "snd_multirate_execute_host", "snd_multirate_candidates"):
        getattr(lib, name).restype = ctypes.c_int
    return lib


lib = _load()


class SndError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        msg = lib.snd_error_string(code).decode()
        super().__init__(f"{where}: {STATUS.get(code, code)} ({msg})")


def _check(code: int, where: str) -> int:
    if code != 0:
        raise SndError(code, where)
    return code


def options(mode: int, **kw) -> SndOptions:
    o = SndOptions()
    _check(lib.snd_options_init(mode, ctypes.byref(o)), "snd_options_init")
    for k, v in kw.items():
        if not hasattr(o, k):
            raise AttributeError(k)
        setattr(o, k, v)
    return o


def _stream_ptr(stream) -> ctypes.c_void_p:
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(int(getattr(stream, "cuda_stream", stream)))


class Plan:
    """One SND plan (snd_plan_ex) plus a torch-allocated device workspace."""

    def __init__(self, freqs, dt: float, dms, branching: int, mode: int, opts: SndOptions | None = None,
                 bind: bool = True, device=None, stream=None):
        self.freqs = np.ascontiguousarray(freqs, dtype=np.float64)
        self.dms = np.ascontiguousarray(dms, dtype=np.float64)
        self.dt = float(dt)
        self.mode = int(mode)
        self.nchan = self.freqs.size
        self.ndm = self.dms.size
        self.opts = opts if opts is not None else options(mode)
        h = ctypes.c_void_p()
        dp = ctypes.POINTER(ctypes.c_double)
        _check(lib.snd_plan_ex(self.freqs.ctypes.data_as(dp), self.nchan, self.dt, self.dms.ctypes.data_as(dp),
                               self.ndm, int(branching), self.mode, ctypes.byref(self.opts), ctypes.byref(h)),
               "snd_plan_ex")
        self.handle = h
        self.workspace = None
        if bind:
            self.bind(device=device, stream=stream)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value and getattr(self, "_owned", True):
            lib.snd_destroy(h)
            self.handle = None

    @property
    def workspace_bytes(self) -> int:
        return int(lib.snd_workspace_size(self.handle))

    def bind(self, device=None, stream=None, workspace=None):
        import torch
        n = self.workspace_bytes
        if workspace is None:
            workspace = torch.empty(n + 256, dtype=torch.uint8, device=device or "cuda")
        ptr = workspace.data_ptr()
        off = (-ptr) % 256
        self.workspace = workspace
        _check(lib.snd_bind_workspace(self.handle, ctypes.c_void_p(ptr + off), n, _stream_ptr(stream)),
               "snd_bind_workspace")

    def execute(self, chunk, plane_out=None, stream=None) -> int:
        """chunk: device uint8 tensor [nsamp][nchan]; plane_out: optional device tensor
        [ndm][nemit] (int32, or float32 in float mode). Returns nemit."""
        assert chunk.is_cuda and chunk.dtype.itemsize == 1 and chunk.is_contiguous()
        nsamp = int(chunk.shape[0])
        ne = ctypes.c_int32(0)
        out = ctypes.c_void_p(plane_out.data_ptr()) if plane_out is not None else None
        _check(lib.snd_execute(self.handle, ctypes.c_void_p(chunk.data_ptr()), nsamp, _stream_ptr(stream), out,
                               ctypes.byref(ne)), "snd_execute")
        return int(ne.value)

    def execute_host(self, chunk, plane_out=None, stream=None) -> int:
        """chunk: host uint8 array/tensor [nsamp][nchan] (pinned for an asynchronous copy)."""
        if hasattr(chunk, "data_ptr"):
            ptr, nsamp = chunk.data_ptr(), int(chunk.shape[0])
        else:
            chunk = np.ascontiguousarray(chunk, dtype=np.uint8)
            ptr, nsamp = chunk.ctypes.data, chunk.shape[0]
        ne = ctypes.c_int32(0)
        out = ctypes.c_void_p(plane_out.data_ptr()) if plane_out is not None else None
        _check(lib.snd_execute_host(self.handle, ctypes.c_void_p(ptr), nsamp, _stream_ptr(stream), out,
                                    ctypes.byref(ne)), "snd_execute_host")
        return int(ne.value)

    def nemit_next(self, nsamp: int) -> int:
        s = self.stats()
        return max(0, s.samples_in + nsamp - s.max_delay) - s.emitted

    def candidates(self, cap: int | None = None, check: bool = True):
        """Synchronise and return (structured numpy array of candidates, status)."""
        cap = int(self.opts.cand_capacity if cap is None else cap)
        buf = (SndCandidate * max(cap, 1))()
        n = ctypes.c_int32(0)
        rc = lib.snd_candidates(self.handle, buf, cap, ctypes.byref(n))
        if check:
            _check(rc, "snd_candidates")
        arr = np.frombuffer(bytes(buf)[: n.value * CANDIDATE_DTYPE.itemsize], dtype=CANDIDATE_DTYPE).copy()
        return arr, rc

    def stats(self) -> SndPlanStats:
        s = SndPlanStats()
        _check(lib.snd_plan_stats(self.handle, ctypes.byref(s)), "snd_plan_stats")
        return s

    def profile(self, enable: bool = True):
        _check(lib.snd_profile(self.handle, int(enable)), "snd_profile")

    def profile_read(self) -> dict:
        """{stage: (milliseconds summed, timed launches)} since the last read."""
        ms = (ctypes.c_double * 4)()
        cnt = (ctypes.c_int64 * 4)()
        _check(lib.snd_profile_read(self.handle, ms, cnt), "snd_profile_read")
        return {STAGES[i]: (ms[i], cnt[i]) for i in range(4)}

    def level_rates(self):
        """(fires uint64[nlev], rates float64[nlev]) of a plan made with FLAG_LEVEL_RATES."""
        fires = np.zeros(24, dtype=np.uint64)
        rates = np.zeros(24, dtype=np.float64)
        n = ctypes.c_int32(0)
        _check(lib.snd_level_rates(self.handle, fires.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                                   rates.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 24, ctypes.byref(n)),
               "snd_level_rates")
        return fires[:n.value], rates[:n.value]

    def delay_table(self) -> np.ndarray:
        out = np.zeros((self.ndm, self.nchan), dtype=np.int32)
        _check(lib.snd_delay_table(self.handle, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), out.size),
               "snd_delay_table")
        return out


class _BandPlan(Plan):
    """A band plan owned by a MultiRatePlan: statistics, profiling and the delay table only."""

    def __init__(self, handle, freqs, dt, dms, mode, opts):
        self.freqs, self.dms, self.dt, self.mode = freqs, dms, dt, mode
        self.nchan, self.ndm, self.opts = freqs.size, dms.size, opts
        self.handle = handle
        self._owned = False
        self.workspace = None


class MultiRatePlan:
    """Multi-rate search (snd_multirate_*): one plan per scrunch band, candidates merged on the GPU."""

    def __init__(self, freqs, dt: float, dms, branching: int, mode: int, opts: SndOptions | None = None,
                 s_max: int = 64, bind: bool = True, device=None, stream=None):
        self.freqs = np.ascontiguousarray(freqs, dtype=np.float64)
        self.dms = np.ascontiguousarray(dms, dtype=np.float64)
        self.dt = float(dt)
        self.mode = int(mode)
        self.nchan = self.freqs.size
        self.opts = opts if opts is not None else options(mode)
        h = ctypes.c_void_p()
        dp = ctypes.POINTER(ctypes.c_double)
        _check(lib.snd_multirate_plan(self.freqs.ctypes.data_as(dp), self.nchan, self.dt,
                                      self.dms.ctypes.data_as(dp), self.dms.size, int(branching), self.mode,
                                      ctypes.byref(self.opts), int(s_max), ctypes.byref(h)), "snd_multirate_plan")
        self.handle = h
        nb = ctypes.c_int32(0)
        _check(lib.snd_multirate_info(h, ctypes.byref(nb), None, None, 0), "snd_multirate_info")
        sc = (ctypes.c_int32 * max(nb.value, 1))()
        nd = (ctypes.c_int32 * max(nb.value, 1))()
        _check(lib.snd_multirate_info(h, ctypes.byref(nb), sc, nd, nb.value), "snd_multirate_info")
        self.scrunch = [int(sc[i]) for i in range(nb.value)]
        self.band_ndm = [int(nd[i]) for i in range(nb.value)]
        self.workspace = None
        if bind:
            self.bind(device=device, stream=stream)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            lib.snd_multirate_destroy(h)
            self.handle = None

    @property
    def workspace_bytes(self) -> int:
        return int(lib.snd_multirate_workspace_size(self.handle))

    def set_graph(self, enable: bool):
        _check(lib.snd_multirate_set_graph(self.handle, int(bool(enable))), "snd_multirate_set_graph")

    def band_plan(self, i: int) -> Plan:
        """Borrowed view of band i's plan (stats, profile, delay table)."""
        h = ctypes.c_void_p()
        _check(lib.snd_multirate_band_plan(self.handle, int(i), ctypes.byref(h)), "snd_multirate_band_plan")
        s = self.scrunch[i]
        return _BandPlan(h, self.freqs, self.dt * s, np.zeros(self.band_ndm[i]), self.mode, self.opts)

    def bind(self, device=None, stream=None, workspace=None):
        import torch
        n = self.workspace_bytes
        if workspace is None:
            workspace = torch.empty(n + 256, dtype=torch.uint8, device=device or "cuda")
        ptr = workspace.data_ptr()
        off = (-ptr) % 256
        self.workspace = workspace
        _check(lib.snd_multirate_bind_workspace(self.handle, ctypes.c_void_p(ptr + off), n, _stream_ptr(stream)),
               "snd_multirate_bind_workspace")

    def execute(self, chunk, stream=None):
        assert chunk.is_cuda and chunk.dtype.itemsize == 1 and chunk.is_contiguous()
        _check(lib.snd_multirate_execute(self.handle, ctypes.c_void_p(chunk.data_ptr()), int(chunk.shape[0]),
                                         _stream_ptr(stream)), "snd_multirate_execute")

    def execute_host(self, chunk, stream=None):
        if hasattr(chunk, "data_ptr"):
            ptr, nsamp = chunk.data_ptr(), int(chunk.shape[0])
        else:
            chunk = np.ascontiguousarray(chunk, dtype=np.uint8)
            ptr, nsamp = chunk.ctypes.data, chunk.shape[0]
        _check(lib.snd_multirate_execute_host(self.handle, ctypes.c_void_p(ptr), nsamp, _stream_ptr(stream)),
               "snd_multirate_execute_host")

    def candidates(self, cap: int | None = None, check: bool = True):
        """Merged candidates since the last call: (structured numpy array, status)."""
        cap = int(self.opts.cand_capacity * len(self.scrunch) if cap is None else cap)
        buf = (SndCandidate * max(cap, 1))()
        n = ctypes.c_int32(0)
        rc = lib.snd_multirate_candidates(self.handle, buf, cap, ctypes.byref(n))
        if check:
            _check(rc, "snd_multirate_candidates")
        arr = np.frombuffer(bytes(buf)[: n.value * CANDIDATE_DTYPE.itemsize], dtype=CANDIDATE_DTYPE).copy()
        return arr, rc


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


class Sifter:
    """The learned candidate sifter (snd_sifter_*) with a torch-allocated workspace."""

    NUM_PARAMS = None

    def __init__(self, max_batch: int, training: bool = True, seed: int = 1, device=None, stream=None):
        h = ctypes.c_void_p()
        _check(lib.snd_sifter_create(int(max_batch), int(bool(training)), int(seed), ctypes.byref(h)),
               "snd_sifter_create")
        self.handle = h
        self.max_batch = int(max_batch)
        self.num_params = int(lib.snd_sifter_num_params())
        import torch
        n = int(lib.snd_sifter_workspace_size(h))
        self.workspace = torch.empty(n + 256, dtype=torch.uint8, device=device or "cuda")
        ptr = self.workspace.data_ptr()
        _check(lib.snd_sifter_bind_workspace(h, ctypes.c_void_p(ptr + (-ptr) % 256), n, _stream_ptr(stream)),
               "snd_sifter_bind_workspace")

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            lib.snd_sifter_destroy(h)
            self.handle = None

    def set_params(self, params, stream=None):
        p = np.ascontiguousarray(params, dtype=np.float32)
        _check(lib.snd_sifter_set_params(self.handle, p.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), p.size,
                                         _stream_ptr(stream)), "snd_sifter_set_params")

    def get_params(self) -> np.ndarray:
        p = np.zeros(self.num_params, dtype=np.float32)
        _check(lib.snd_sifter_get_params(self.handle, p.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), p.size),
               "snd_sifter_get_params")
        return p

    def forward(self, x, logits=None, stream=None):
        """x: device float32 [n][64][256] -> device float32 logits [n]."""
        import torch
        assert x.is_cuda and x.dtype == torch.float32 and x.is_contiguous()
        n = int(x.shape[0])
        if logits is None:
            logits = torch.empty(n, dtype=torch.float32, device=x.device)
        _check(lib.snd_sifter_forward(self.handle, _ptr(x), n, _ptr(logits), _stream_ptr(stream)),
               "snd_sifter_forward")
        return logits

    def gradients(self, x, y, stream=None):
        """(loss, gradient vector) on device tensors x [n][64][256], y [n] (no update)."""
        import torch
        n = int(x.shape[0])
        g = torch.empty(self.num_params, dtype=torch.float32, device=x.device)
        loss = torch.empty(1, dtype=torch.float32, device=x.device)
        _check(lib.snd_sifter_gradients(self.handle, _ptr(x), _ptr(y), n, _ptr(g), _ptr(loss), _stream_ptr(stream)),
               "snd_sifter_gradients")
        return loss, g

    def train_step(self, x, y, lr: float, loss=None, stream=None):
        n = int(x.shape[0])
        _check(lib.snd_sifter_train_step(self.handle, _ptr(x), _ptr(y), n, float(lr),
                                         _ptr(loss) if loss is not None else None, _stream_ptr(stream)),
               "snd_sifter_train_step")

    def status(self):
        _check(lib.snd_sifter_status(self.handle), "snd_sifter_status")

    @property
    def launches(self) -> int:
        return int(lib.snd_sifter_launches(self.handle))


def snippets(plane, rows, cols, out=None, stream=None):
    """Standardised 64 x 256 snippets of a device float32 plane [ndm][ncols] around
    (rows[i], cols[i]) (device int32 / int64 tensors)."""
    import torch
    n = int(rows.shape[0])
    if out is None:
        out = torch.empty((n, 64, 256), dtype=torch.float32, device=plane.device)
    _check(lib.snd_snippets(_ptr(plane), plane.stride(0), plane.shape[0], plane.shape[1], _ptr(rows), _ptr(cols), n,
                            _ptr(out), _stream_ptr(stream)), "snd_snippets")
    return out


def gemm_bf16(a, b, k=None, splits=1, out=None, stream=None):
    """FP32 C = A . B^T on the tensor cores (A [m][lda], B [n][ldb] BF16 device tensors)."""
    import torch
    m, n = int(a.shape[0]), int(b.shape[0])
    k = int(a.shape[1] if k is None else k)
    if out is None:
        out = torch.zeros((m, n), dtype=torch.float32, device=a.device)
    err = torch.zeros(1, dtype=torch.int32, device=a.device)
    _check(lib.snd_gemm_bf16(_ptr(a), a.stride(0), _ptr(b), b.stride(0), m, n, k, _ptr(out), out.stride(0),
                             int(splits), _ptr(err), _stream_ptr(stream)), "snd_gemm_bf16")
    return out, err


class Batch:
    """Advance several bound plans (beams) by one chunk each per call (snd_batch_*)."""

    def __init__(self, plans, graph: bool = False):
        self.plans = list(plans)
        arr = (ctypes.c_void_p * len(self.plans))(*[p.handle.value for p in self.plans])
        h = ctypes.c_void_p()
        _check(lib.snd_batch_create(arr, len(self.plans), ctypes.byref(h)), "snd_batch_create")
        self.handle = h
        self.set_graph(graph)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            lib.snd_batch_destroy(h)
            self.handle = None

    def set_graph(self, enable: bool):
        _check(lib.snd_batch_set_graph(self.handle, int(bool(enable))), "snd_batch_set_graph")

    def execute(self, chunks, stream=None):
        """chunks: one contiguous device uint8 tensor [nsamp_i][nchan_i] per plan."""
        n = len(self.plans)
        ptrs = (ctypes.c_void_p * n)(*[c.data_ptr() for c in chunks])
        ns = (ctypes.c_int32 * n)(*[int(c.shape[0]) for c in chunks])
        _check(lib.snd_batch_execute(self.handle, ptrs, ns, _stream_ptr(stream)), "snd_batch_execute")

    def graph_stats(self):
        a, b = ctypes.c_int64(0), ctypes.c_int64(0)
        _check(lib.snd_batch_graph_stats(self.handle, ctypes.byref(a), ctypes.byref(b)), "snd_batch_graph_stats")
        return int(a.value), int(b.value)
