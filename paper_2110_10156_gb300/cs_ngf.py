"""Thin Python binding of ``libcs_ngf.so`` (C ABI in ``include/cs_ngf.h``).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Device arrays are passed as torch CUDA tensors (their data pointers
and the current torch stream); quaternions are host float64.  If the library
has not been built the import fails loudly; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcs_ngf.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with "
                      "`python -m paper_2110_10156_gb300.build` (needs nvcc)")

_lib = ctypes.CDLL(LIB_PATH)

OK, EINVAL, ENOMEM, ECUDA, ENOVALID, EUNSUPPORTED, ECANCELED, ETIMEOUT, EBUSY = range(9)

EXPORTED = (
    "cs_ngf_default_config", "cs_ngf_prepare_fixed", "cs_ngf_score_rotations",
    "cs_ngf_score_rotations_host", "cs_ngf_align", "cs_ngf_score_map", "cs_ngf_resample",
    "cs_ngf_get_info", "cs_ngf_release", "cs_ngf_status_string", "cs_ngf_last_error",
    "cs_ngf_auto_pad", "cs_ngf_update_fixed", "cs_ngf_set_profiling", "cs_ngf_stage_times",
    "cs_ngf_launch_count", "cs_ngf_score_rotations_noalloc",
    "cs_ngf_server_default_config", "cs_ngf_server_create", "cs_ngf_server_submit",
    "cs_ngf_server_cancel", "cs_ngf_server_wait", "cs_ngf_server_stats", "cs_ngf_server_destroy",
    "cs_ngf_search_default_config", "cs_ngf_global_align", "cs_ngf_length_sets",
    "cs_ngf_tuning", "cs_ngf_tuning_reset", "cs_ngf_plan_lengths",
)

MAX_LEVELS = 8

STAGES = ("resample", "fwd_x", "fwd_y", "zmac", "inv_y", "inv_x", "fixed", "other")


class Config(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_float), ("gamma", ctypes.c_float),
                ("pad", ctypes.c_int32 * 3), ("batch", ctypes.c_int32), ("measure", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("pad_mode", ctypes.c_int32), ("autotune", ctypes.c_int32),
                ("tensor_cores", ctypes.c_int32)]


class TuningEntry(ctypes.Structure):
    _fields_ = [("pass_", ctypes.c_int32), ("length", ctypes.c_int32), ("half_input", ctypes.c_int32),
                ("storage", ctypes.c_int32), ("variant", ctypes.c_int32), ("split", (ctypes.c_int32 * 2) * 2),
                ("ms", ctypes.c_float * 2)]


PASS_NAMES = ("fwd_x", "fwd_y", "zmac", "inv_y", "inv_x")


MEASURES = {"squared": 0, "unsquared": 1}
PRECISIONS = {"fp32": 0, "bf16": 1, "fp16": 2}
PAD_MODES = {"full": 0, "bound": 1}


class Info(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int32 * 3), ("pad", ctypes.c_int32 * 3),
                ("batch", ctypes.c_int32), ("sum_mask_a", ctypes.c_int64),
                ("fixed_bytes", ctypes.c_int64), ("workspace_bytes", ctypes.c_int64),
                ("max_pad", ctypes.c_int32 * 3), ("pad_mode", ctypes.c_int32),
                ("length_sets", ctypes.c_int32), ("reserved_", ctypes.c_int32)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("memory_budget_bytes", ctypes.c_int64), ("max_active_jobs", ctypes.c_int32),
                ("max_inflight", ctypes.c_int32), ("batch", ctypes.c_int32),
                ("policy", ctypes.c_int32), ("inject_admission_failure", ctypes.c_int64)]


class JobResult(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("rotations", ctypes.c_int32), ("scored", ctypes.c_int32),
                ("score", ctypes.c_float), ("rot_index", ctypes.c_int32), ("shift", ctypes.c_int32 * 3),
                ("latency_ms", ctypes.c_double), ("queue_ms", ctypes.c_double)]


class ServerInfo(ctypes.Structure):
    _fields_ = [("pending", ctypes.c_int32), ("active", ctypes.c_int32), ("slots", ctypes.c_int32),
                ("reserved_", ctypes.c_int32), ("admitted", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("bytes_in_use", ctypes.c_int64), ("memory_budget_bytes", ctypes.c_int64)]


class SearchConfig(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int32), ("sigma", ctypes.c_float * 8),
                ("downsample", ctypes.c_int32 * 8), ("max_step_deg", ctypes.c_float * 8),
                ("random_rotations", ctypes.c_int32 * 8), ("starting_points", ctypes.c_int32 * 8),
                ("start_euler_deg", ctypes.c_float * 3), ("seed", ctypes.c_uint64)]


class SearchResult(ctypes.Structure):
    _fields_ = [("score", ctypes.c_float), ("level_best", ctypes.c_float * 8),
                ("euler_deg", ctypes.c_double * 3), ("quat", ctypes.c_double * 4),
                ("shift", ctypes.c_int32 * 3), ("rotations_scored", ctypes.c_int64)]


_vp, _i32, _p = ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER
_lib.cs_ngf_default_config.argtypes = [_p(Config)]
_lib.cs_ngf_default_config.restype = None
_lib.cs_ngf_prepare_fixed.argtypes = [_vp, _vp, _p(_i32), _p(Config), _vp, _p(_vp)]
_lib.cs_ngf_score_rotations.argtypes = [_vp, _vp, _vp, _vp, _i32, _vp, _vp, _vp]
_lib.cs_ngf_score_rotations_host.argtypes = [_vp, _vp, _vp, _vp, _i32, _vp, _vp, _vp]
_lib.cs_ngf_align.argtypes = [_vp, _vp, _vp, _vp, _i32, _p(ctypes.c_float), _p(_i32), _p(_i32), _vp]
_lib.cs_ngf_score_map.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp]
_lib.cs_ngf_resample.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp, _vp]
_lib.cs_ngf_get_info.argtypes = [_vp, _p(Info)]
_lib.cs_ngf_release.argtypes = [_vp]
_lib.cs_ngf_release.restype = None
_lib.cs_ngf_status_string.argtypes = [_i32]
_lib.cs_ngf_status_string.restype = ctypes.c_char_p
_lib.cs_ngf_last_error.argtypes = []
_lib.cs_ngf_last_error.restype = ctypes.c_char_p
_lib.cs_ngf_plan_lengths.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, _i32,
                                     ctypes.c_void_p, _i32, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_void_p]
_lib.cs_ngf_plan_lengths.restype = _i32
_lib.cs_ngf_tuning.argtypes = [_i32, ctypes.c_void_p]
_lib.cs_ngf_tuning.restype = _i32
_lib.cs_ngf_tuning_reset.argtypes = []
_lib.cs_ngf_tuning_reset.restype = None
_lib.cs_ngf_length_sets.argtypes = [ctypes.c_void_p, _i32, ctypes.c_void_p, ctypes.c_void_p]
_lib.cs_ngf_length_sets.restype = _i32
_lib.cs_ngf_auto_pad.argtypes = [_i32]
_lib.cs_ngf_auto_pad.restype = _i32
_lib.cs_ngf_update_fixed.argtypes = [_vp, _vp, _vp, _vp]
_lib.cs_ngf_set_profiling.argtypes = [_vp, _i32]
_lib.cs_ngf_stage_times.argtypes = [_vp, _p(ctypes.c_double), _p(ctypes.c_int64)]
_lib.cs_ngf_score_rotations_noalloc.argtypes = [_vp, _vp, _vp, _vp, _p(_i32), ctypes.c_float,
                                                 ctypes.c_float, _vp, _i32, _vp, _vp, _vp]
_lib.cs_ngf_score_rotations_noalloc.restype = _i32
_lib.cs_ngf_server_default_config.argtypes = [_p(ServerConfig)]
_lib.cs_ngf_server_default_config.restype = None
_lib.cs_ngf_server_create.argtypes = [_p(ServerConfig), _p(_vp)]
_lib.cs_ngf_server_submit.argtypes = [_vp, _vp, _vp, _vp, _vp, _p(_i32), _vp, _i32, _p(Config),
                                      _p(ctypes.c_int64)]
_lib.cs_ngf_server_cancel.argtypes = [_vp, ctypes.c_int64]
_lib.cs_ngf_server_wait.argtypes = [_vp, ctypes.c_int64, ctypes.c_double, _p(JobResult), _vp, _vp]
_lib.cs_ngf_server_stats.argtypes = [_vp, _p(ServerInfo)]
_lib.cs_ngf_server_destroy.argtypes = [_vp]
_lib.cs_ngf_server_destroy.restype = None
for _name in ("cs_ngf_server_create", "cs_ngf_server_submit", "cs_ngf_server_cancel",
              "cs_ngf_server_wait", "cs_ngf_server_stats"):
    getattr(_lib, _name).restype = _i32
_lib.cs_ngf_search_default_config.argtypes = [_p(SearchConfig)]
_lib.cs_ngf_search_default_config.restype = None
_lib.cs_ngf_global_align.argtypes = [_vp, _vp, _vp, _vp, _p(_i32), _p(Config), _p(SearchConfig), _vp,
                                     _p(SearchResult)]
_lib.cs_ngf_global_align.restype = _i32
_lib.cs_ngf_launch_count.argtypes = []
_lib.cs_ngf_launch_count.restype = ctypes.c_int64
for _name in ("cs_ngf_update_fixed", "cs_ngf_set_profiling", "cs_ngf_stage_times",
              "cs_ngf_prepare_fixed", "cs_ngf_score_rotations", "cs_ngf_score_rotations_host",
              "cs_ngf_align", "cs_ngf_score_map", "cs_ngf_resample", "cs_ngf_get_info"):
    getattr(_lib, _name).restype = _i32


class CsNgfError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = _lib.cs_ngf_status_string(status).decode()
        detail = _lib.cs_ngf_last_error().decode()
        super().__init__(f"{where}: {msg}" + (f" ({detail})" if detail else ""))


def _check(status: int, where: str):
    if status != OK:
        raise CsNgfError(status, where)


def library():
    """The loaded ctypes library (for symbol checks)."""
    return _lib


def launch_count() -> int:
    """Kernel launches made by the library in this process."""
    return int(_lib.cs_ngf_launch_count())


def plan_lengths(dims, max_pad, bounds, cur_pad=None):
    """Length classes of bound-limited padding for per-rotation shift bounds
    [R][6] (cs_ngf_plan_lengths, host only): ([((Pz, Py, Px), count)], order)."""
    b = np.ascontiguousarray(bounds, dtype=np.int32).reshape(-1, 6)
    R = b.shape[0]
    d = (ctypes.c_int32 * 3)(*dims)
    m = (ctypes.c_int32 * 3)(*max_pad)
    c = (ctypes.c_int32 * 3)(*cur_pad) if cur_pad is not None else None
    pads = (ctypes.c_int32 * 24)()
    counts = (ctypes.c_int32 * 8)()
    order = np.zeros(R, np.int32)
    n = int(_lib.cs_ngf_plan_lengths(d, m, c, R, b.ctypes.data_as(ctypes.c_void_p), 8, pads, counts,
                                     order.ctypes.data_as(ctypes.c_void_p)))
    if n < 0:
        raise CsNgfError(EINVAL, "cs_ngf_plan_lengths")
    return [((pads[3 * k], pads[3 * k + 1], pads[3 * k + 2]), int(counts[k])) for k in range(n)], order


def tuning():
    """The process's autotuning choices (cs_ngf_tuning): one dict per FFT pass,
    length, input kind and storage form timed so far."""
    n = int(_lib.cs_ngf_tuning(0, None))
    arr = (TuningEntry * max(n, 1))()
    _lib.cs_ngf_tuning(n, arr)
    store = {v: k for k, v in PRECISIONS.items()}
    return [dict(stage=PASS_NAMES[e.pass_], length=e.length, half_input=bool(e.half_input),
                 storage=store.get(e.storage, e.storage), variant=e.variant,
                 splits=[tuple(e.split[v]) for v in range(2)], ms=[float(e.ms[0]), float(e.ms[1])])
            for e in arr[:n]]


def tuning_reset():
    _lib.cs_ngf_tuning_reset()


def auto_pad(n: int) -> int:
    return int(_lib.cs_ngf_auto_pad(int(n)))


def _stream_ptr(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dev_ptr(t, dtype, name):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _check_shapes(dims, named):
    """Every (tensor, name) must have shape ``dims`` (checked before any pointer
    reaches the library, which reads them with those dims)."""
    for t, name in named:
        if tuple(t.shape) != tuple(dims):
            raise ValueError(f"{name} must have shape {tuple(dims)}, got {tuple(t.shape)}")


def _check_outputs(out_score, out_shift, R):
    """Caller-given outputs must hold R scores and R x 3 shifts."""
    if out_score is not None and tuple(out_score.shape) != (R,):
        raise ValueError(f"best_score must have shape ({R},), got {tuple(out_score.shape)}")
    if out_shift is not None and tuple(out_shift.shape) != (R, 3):
        raise ValueError(f"best_shift must have shape ({R}, 3), got {tuple(out_shift.shape)}")


def _same_device(device, named):
    for t, name in named:
        if t.device != device:
            raise ValueError(f"{name} is on {t.device}, expected {device}")


def _quats(q) -> np.ndarray:
    q = np.ascontiguousarray(np.asarray(q, dtype=np.float64).reshape(-1, 4))
    return q


class Fixed:
    """Handle on the device-resident fixed-volume spectra (cs_ngf_prepare_fixed)."""

    def __init__(self, A, MA, eps=1e-5, gamma=0.5, pad=None, batch=0, stream=None,
                 measure="squared", precision="fp32", pad_mode="bound", autotune=False,
                 tensor_cores=True):
        """autotune: False (built-in radix splits), True (timed on first use
        at new lengths) or "alternative" (the second split wherever a length
        has one).  tensor_cores: the BF16 and FP16 forms run the z-axis
        forward DFT of the channel fields on the tensor cores (False: CUDA-core
        FFTs throughout)."""
        import torch
        _dev_ptr(A, torch.float32, "A")
        _dev_ptr(MA, torch.uint8, "maskA")
        if A.dim() != 3:
            raise ValueError("A must be [nz][ny][nx]")
        self.dims = tuple(int(d) for d in A.shape)
        if tuple(MA.shape) != self.dims:
            raise ValueError("maskA must have A's shape")
        cfg = Config()
        _lib.cs_ngf_default_config(ctypes.byref(cfg))
        cfg.eps = float(eps)
        cfg.gamma = float(gamma)
        if pad is not None:
            for i, p in enumerate(pad):
                cfg.pad[i] = int(p)
        cfg.batch = int(batch)
        cfg.measure = MEASURES[measure]
        cfg.precision = PRECISIONS[precision]
        cfg.pad_mode = PAD_MODES[pad_mode]
        cfg.autotune = 2 if autotune == "alternative" else (1 if autotune else 0)
        cfg.tensor_cores = 1 if tensor_cores else 0
        self.measure = measure
        self.precision = precision
        self.pad_mode = pad_mode
        # everything besides A and maskA that decides the handle's results
        self.settings = dict(eps=float(eps), gamma=float(gamma), measure=measure,
                             precision=precision, pad_mode=pad_mode, batch=int(batch),
                             tensor_cores=bool(tensor_cores),
                             pad=tuple(int(v) for v in pad) if pad is not None else None)
        dims = (ctypes.c_int32 * 3)(*self.dims)
        h = ctypes.c_void_p()
        st = _check(_lib.cs_ngf_prepare_fixed(_dev_ptr(A, torch.float32, "A"),
                                              _dev_ptr(MA, torch.uint8, "maskA"), dims,
                                              ctypes.byref(cfg), _stream_ptr(stream),
                                              ctypes.byref(h)), "cs_ngf_prepare_fixed")
        self._h = h
        self._keep = (A, MA)
        info = self._info()
        self.max_pad = tuple(info.max_pad)
        self.batch = int(info.batch)
        self.sum_mask_a = int(info.sum_mask_a)
        self.fixed_bytes = int(info.fixed_bytes)
        self.workspace_bytes = int(info.workspace_bytes)

    def _info(self):
        info = Info()
        _check(_lib.cs_ngf_get_info(self._h, ctypes.byref(info)), "cs_ngf_get_info")
        return info

    @property
    def pad(self):
        """FFT lengths (z, y, x) in use: those of the last call (bound-limited
        padding may shorten them below max_pad)."""
        return tuple(self._info().pad)

    def length_classes(self):
        """[((Pz, Py, Px), rotations)] of the last scoring call, in the order scored."""
        n = int(_lib.cs_ngf_length_sets(self._h, 0, None, None))
        pads = (ctypes.c_int32 * (3 * max(n, 1)))()
        counts = (ctypes.c_int32 * max(n, 1))()
        _lib.cs_ngf_length_sets(self._h, n, pads, counts)
        return [((pads[3 * c], pads[3 * c + 1], pads[3 * c + 2]), int(counts[c])) for c in range(n)]

    @property
    def length_sets(self):
        """Sets of FFT lengths the last scoring call used (rotations regrouped
        by the lengths they need under bound-limited padding)."""
        return int(self._info().length_sets)

    @property
    def handle(self):
        return self._h

    def _check_vol(self, B, MB):
        import torch
        if tuple(B.shape) != self.dims or tuple(MB.shape) != self.dims:
            raise ValueError("B and maskB must have the fixed volume's shape")
        pb, pm = _dev_ptr(B, torch.float32, "B"), _dev_ptr(MB, torch.uint8, "maskB")
        _same_device(self._keep[0].device, ((B, "B"), (MB, "maskB")))
        return pb, pm

    def score_rotations(self, B, MB, quats, out_score=None, out_shift=None, stream=None):
        """Per-rotation best score [R] (float32) and shift [R, 3] (int32, z y x)."""
        import torch
        q = _quats(quats)
        R = q.shape[0]
        pb, pm = self._check_vol(B, MB)
        _check_outputs(out_score, out_shift, R)
        if out_score is None:
            out_score = torch.empty(R, dtype=torch.float32, device=B.device)
        if out_shift is None:
            out_shift = torch.empty((R, 3), dtype=torch.int32, device=B.device)
        _check(_lib.cs_ngf_score_rotations(self._h, pb, pm, q.ctypes.data_as(ctypes.c_void_p), R,
                                           _dev_ptr(out_score, torch.float32, "best_score"),
                                           _dev_ptr(out_shift, torch.int32, "best_shift"),
                                           _stream_ptr(stream)), "cs_ngf_score_rotations")
        self._last_q = q          # keep the host array alive until the call returned
        return out_score, out_shift

    def score_rotations_host(self, B_host: np.ndarray, MB_host: np.ndarray, quats,
                             out_score: np.ndarray | None = None,
                             out_shift: np.ndarray | None = None, stream=None):
        """Same, from HOST arrays (copies inside the call); returns numpy arrays."""
        q = _quats(quats)
        R = q.shape[0]
        for name, arr, dt in (("B", B_host, np.float32), ("maskB", MB_host, np.uint8)):
            if arr.dtype != dt or not arr.flags.c_contiguous or tuple(arr.shape) != self.dims:
                raise ValueError(f"{name} must be a C-contiguous {dt.__name__} array of the fixed shape")
        if out_score is None:
            out_score = np.empty(R, np.float32)
        if out_shift is None:
            out_shift = np.empty((R, 3), np.int32)
        _check(_lib.cs_ngf_score_rotations_host(
            self._h, ctypes.c_void_p(B_host.ctypes.data), ctypes.c_void_p(MB_host.ctypes.data),
            q.ctypes.data_as(ctypes.c_void_p), R, ctypes.c_void_p(out_score.ctypes.data),
            ctypes.c_void_p(out_shift.ctypes.data), _stream_ptr(stream)),
            "cs_ngf_score_rotations_host")
        return out_score, out_shift

    def align(self, B, MB, quats, stream=None):
        """(score, rotation index, (cz, cy, cx)); index -1 if nothing is valid."""
        q = _quats(quats)
        pb, pm = self._check_vol(B, MB)
        sc = ctypes.c_float()
        ri = ctypes.c_int32()
        sh = (ctypes.c_int32 * 3)()
        st = _lib.cs_ngf_align(self._h, pb, pm, q.ctypes.data_as(ctypes.c_void_p), q.shape[0],
                               ctypes.byref(sc), ctypes.byref(ri), sh, _stream_ptr(stream))
        if st not in (OK, ENOVALID):
            _check(st, "cs_ngf_align")
        return float(sc.value), int(ri.value), tuple(int(v) for v in sh)

    def score_map(self, B, MB, quat, stream=None):
        """Full CSNGF map over shifts for one rotation (-inf where invalid)."""
        import torch
        q = _quats(quat)
        pb, pm = self._check_vol(B, MB)
        shape = tuple(2 * n - 1 for n in self.dims)
        out = torch.empty(shape, dtype=torch.float32, device=B.device)
        _check(_lib.cs_ngf_score_map(self._h, pb, pm, q.ctypes.data_as(ctypes.c_void_p),
                                     _dev_ptr(out, torch.float32, "map"), _stream_ptr(stream)),
               "cs_ngf_score_map")
        torch.cuda.current_stream().synchronize() if stream is None else stream.synchronize()
        return out

    def resample(self, B, MB, quat, stream=None):
        """B_hat (float32) and M_hat (uint8) for one rotation."""
        import torch
        q = _quats(quat)
        pb, pm = self._check_vol(B, MB)
        Bh = torch.empty(self.dims, dtype=torch.float32, device=B.device)
        Mh = torch.empty(self.dims, dtype=torch.uint8, device=B.device)
        _check(_lib.cs_ngf_resample(self._h, pb, pm, q.ctypes.data_as(ctypes.c_void_p),
                                    _dev_ptr(Bh, torch.float32, "Bhat"),
                                    _dev_ptr(Mh, torch.uint8, "Mhat"), _stream_ptr(stream)),
               "cs_ngf_resample")
        torch.cuda.current_stream().synchronize() if stream is None else stream.synchronize()
        return Bh, Mh

    def update_fixed(self, A, MA, stream=None):
        """Recompute the fixed spectra from a new A / maskA of the same shape."""
        import torch
        if tuple(A.shape) != self.dims or tuple(MA.shape) != self.dims:
            raise ValueError("A and maskA must keep the handle's shape")
        _check(_lib.cs_ngf_update_fixed(self._h, _dev_ptr(A, torch.float32, "A"),
                                        _dev_ptr(MA, torch.uint8, "maskA"), _stream_ptr(stream)),
               "cs_ngf_update_fixed")
        self._keep = (A, MA)

    def set_profiling(self, on: bool):
        _check(_lib.cs_ngf_set_profiling(self._h, 1 if on else 0), "cs_ngf_set_profiling")

    def stage_times(self):
        """{stage: (milliseconds, launches)} since the previous call (synchronises)."""
        ms = (ctypes.c_double * len(STAGES))()
        n = (ctypes.c_int64 * len(STAGES))()
        _check(_lib.cs_ngf_stage_times(self._h, ms, n), "cs_ngf_stage_times")
        return {name: (float(ms[i]), int(n[i])) for i, name in enumerate(STAGES)}

    def release(self):
        if getattr(self, "_h", None):
            _lib.cs_ngf_release(self._h)
            self._h = None

    def __del__(self):
        try:
            self.release()
        except Exception:
            pass


def score_rotations_noalloc(A, MA, B, MB, quats, eps=1e-5, gamma=0.5, out_score=None,
                            out_shift=None, stream=None):
    """Allocation-free scoring for volumes up to 32 per axis
    (cs_ngf_score_rotations_noalloc): the library allocates no device memory;
    its scratch is a fixed static device array shared by all calls, so calls
    must not overlap on the GPU.  The outputs are allocated here by torch
    unless given."""
    import torch
    if len(A.shape) != 3:
        raise ValueError("A must be [nz][ny][nx]")
    dims = tuple(int(d) for d in A.shape)
    _check_shapes(dims, ((MA, "maskA"), (B, "B"), (MB, "maskB")))
    q = _quats(quats)
    R = q.shape[0]
    _check_outputs(out_score, out_shift, R)
    for t, dt, name in ((A, torch.float32, "A"), (MA, torch.uint8, "maskA"),
                        (B, torch.float32, "B"), (MB, torch.uint8, "maskB")):
        _dev_ptr(t, dt, name)
    named = [(MA, "maskA"), (B, "B"), (MB, "maskB")]
    named += [(t, n) for t, n in ((out_score, "best_score"), (out_shift, "best_shift")) if t is not None]
    _same_device(A.device, named)
    # the library scores on the current device with that device's scratch
    with torch.cuda.device(A.device):
        if out_score is None:
            out_score = torch.empty(R, dtype=torch.float32, device=A.device)
        if out_shift is None:
            out_shift = torch.empty((R, 3), dtype=torch.int32, device=A.device)
        d = (ctypes.c_int32 * 3)(*dims)
        _check(_lib.cs_ngf_score_rotations_noalloc(
            _dev_ptr(A, torch.float32, "A"), _dev_ptr(MA, torch.uint8, "maskA"),
            _dev_ptr(B, torch.float32, "B"), _dev_ptr(MB, torch.uint8, "maskB"), d,
            float(eps), float(gamma), q.ctypes.data_as(ctypes.c_void_p), R,
            _dev_ptr(out_score, torch.float32, "best_score"),
            _dev_ptr(out_shift, torch.int32, "best_shift"), _stream_ptr(stream)),
            "cs_ngf_score_rotations_noalloc")
    return out_score, out_shift


class Server:
    """Continuous-batching request loop (cs_ngf_server_*): submit host arrays,
    wait for per-job results.  Runs on the current CUDA device."""

    POLICIES = {"arrival": 0, "shortest": 1}

    def __init__(self, memory_budget_bytes=0, max_active_jobs=4, max_inflight=2, batch=16,
                 inject_admission_failure=0, policy="arrival"):
        if policy not in self.POLICIES:
            raise ValueError(f"policy must be one of {sorted(self.POLICIES)}")
        cfg = ServerConfig()
        _lib.cs_ngf_server_default_config(ctypes.byref(cfg))
        cfg.memory_budget_bytes = int(memory_budget_bytes)
        cfg.max_active_jobs = int(max_active_jobs)
        cfg.max_inflight = int(max_inflight)
        cfg.batch = int(batch)
        cfg.policy = self.POLICIES[policy]
        cfg.inject_admission_failure = int(inject_admission_failure)
        h = ctypes.c_void_p()
        _check(_lib.cs_ngf_server_create(ctypes.byref(cfg), ctypes.byref(h)), "cs_ngf_server_create")
        self._h = h
        self._R = {}

    def submit(self, A, MA, B, MB, quats, eps=1e-5, gamma=0.5, pad=None, batch=0,
               measure="squared", precision="fp32", pad_mode="bound", tensor_cores=True) -> int:
        arrs = []
        for name, a, dt in (("A", A, np.float32), ("maskA", MA, np.uint8), ("B", B, np.float32),
                            ("maskB", MB, np.uint8)):
            a = np.ascontiguousarray(a, dtype=dt)
            if a.ndim != 3 or a.shape != tuple(np.shape(A)):
                raise ValueError(f"{name} must be 3-D with A's shape")
            arrs.append(a)
        q = _quats(quats)
        cfg = Config()
        _lib.cs_ngf_default_config(ctypes.byref(cfg))
        cfg.eps, cfg.gamma, cfg.batch = float(eps), float(gamma), int(batch)
        cfg.measure = MEASURES[measure]
        cfg.precision = PRECISIONS[precision]
        cfg.pad_mode = PAD_MODES[pad_mode]
        cfg.tensor_cores = 1 if tensor_cores else 0
        if pad is not None:
            for i, p in enumerate(pad):
                cfg.pad[i] = int(p)
        dims = (ctypes.c_int32 * 3)(*arrs[0].shape)
        jid = ctypes.c_int64()
        _check(_lib.cs_ngf_server_submit(self._h, *[ctypes.c_void_p(a.ctypes.data) for a in arrs], dims,
                                         q.ctypes.data_as(ctypes.c_void_p), q.shape[0], ctypes.byref(cfg),
                                         ctypes.byref(jid)), "cs_ngf_server_submit")
        self._R[jid.value] = q.shape[0]
        return int(jid.value)

    def cancel(self, job: int):
        _check(_lib.cs_ngf_server_cancel(self._h, int(job)), "cs_ngf_server_cancel")

    def wait(self, job: int, timeout_s: float = -1.0, per_rotation: bool = True):
        """dict with status, score, rot_index, shift, latency_ms, queue_ms and,
        if per_rotation, the per-rotation scores [R] and shifts [R, 3]."""
        R = self._R.get(int(job), 0)
        res = JobResult()
        sc = np.full(R, -np.inf, np.float32) if per_rotation else None
        sh = np.zeros((R, 3), np.int32) if per_rotation else None
        _check(_lib.cs_ngf_server_wait(self._h, int(job), float(timeout_s), ctypes.byref(res),
                                       ctypes.c_void_p(sc.ctypes.data) if per_rotation else None,
                                       ctypes.c_void_p(sh.ctypes.data) if per_rotation else None),
               "cs_ngf_server_wait")
        self._R.pop(int(job), None)
        out = dict(status=int(res.status), rotations=int(res.rotations), scored=int(res.scored),
                   score=float(res.score), rot_index=int(res.rot_index), shift=tuple(res.shift),
                   latency_ms=float(res.latency_ms), queue_ms=float(res.queue_ms))
        if per_rotation:                    # -inf / (0, 0, 0) where a rotation was not scored
            out["scores"], out["shifts"] = sc, sh
        return out

    def stats(self):
        info = ServerInfo()
        _check(_lib.cs_ngf_server_stats(self._h, ctypes.byref(info)), "cs_ngf_server_stats")
        return {f: getattr(info, f) for f, _ in ServerInfo._fields_ if f != "reserved_"}

    def close(self):
        if getattr(self, "_h", None):
            _lib.cs_ngf_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def global_align(A, MA, B, MB, schedule=None, seed=0x5EED, start=(0.0, 0.0, 0.0), eps=1e-5,
                 gamma=0.5, measure="squared", stream=None, pad_mode="bound"):
    """Pyramid random search of Section 3.2 (cs_ngf_global_align) on device
    volumes.  schedule: list of (sigma, d, u_deg, a, p) per level, p being the
    number of starting points of that level (the first level's p is 1); None
    = the paper's schedule.  Returns a dict with score, euler_deg, quat, shift,
    level_best and rotations_scored."""
    import torch
    sc = SearchConfig()
    _lib.cs_ngf_search_default_config(ctypes.byref(sc))
    if schedule is not None:
        if not 1 <= len(schedule) <= MAX_LEVELS:
            raise ValueError("1 to 8 levels")
        sc.levels = len(schedule)
        for k, (sigma, d, u, a, p) in enumerate(schedule):
            sc.sigma[k], sc.downsample[k], sc.max_step_deg[k] = float(sigma), int(d), float(u)
            sc.random_rotations[k], sc.starting_points[k] = int(a), int(p)
    sc.seed = int(seed)
    for i in range(3):
        sc.start_euler_deg[i] = float(start[i])
    cfg = Config()
    _lib.cs_ngf_default_config(ctypes.byref(cfg))
    cfg.eps, cfg.gamma, cfg.measure = float(eps), float(gamma), MEASURES[measure]
    cfg.pad_mode = PAD_MODES[pad_mode]
    dims = (ctypes.c_int32 * 3)(*tuple(A.shape))
    res = SearchResult()
    _check(_lib.cs_ngf_global_align(_dev_ptr(A, torch.float32, "A"), _dev_ptr(MA, torch.uint8, "maskA"),
                                    _dev_ptr(B, torch.float32, "B"), _dev_ptr(MB, torch.uint8, "maskB"),
                                    dims, ctypes.byref(cfg), ctypes.byref(sc), _stream_ptr(stream),
                                    ctypes.byref(res)), "cs_ngf_global_align")
    return dict(score=float(res.score), euler_deg=tuple(res.euler_deg), quat=tuple(res.quat),
                shift=tuple(res.shift), level_best=[float(res.level_best[k]) for k in range(sc.levels)],
                rotations_scored=int(res.rotations_scored))


def prepare_fixed(A, MA, **kw) -> Fixed:
    return Fixed(A, MA, **kw)
