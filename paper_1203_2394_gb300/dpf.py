"""Python binding of the C ABI in ``include/dpf.h`` (argument marshalling only).

Every step of the filter runs in the CUDA library ``_lib/libdpf.so``; this
module only converts arguments. There is no CPU fallback: if the library is not
built, importing the binding's functions raises ``DpfLibraryMissing``.
PyTorch, when used, supplies device memory and streams.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "libdpf.so")

DPF_OK, DPF_E_INVALID, DPF_E_NOMEM, DPF_E_CUDA, DPF_E_TIMEOUT, DPF_E_NUMERIC, DPF_E_UNSUPPORTED = range(7)
DPF_F32, DPF_F64 = 0, 1
DPF_MODEL_CLG = 1
DPF_SYS_GLOBAL, DPF_SYS_LOCAL = 0, 1
STATUS_NAMES = {0: "DPF_OK", 1: "DPF_E_INVALID", 2: "DPF_E_NOMEM", 3: "DPF_E_CUDA",
                4: "DPF_E_TIMEOUT", 5: "DPF_E_NUMERIC", 6: "DPF_E_UNSUPPORTED"}


class DpfLibraryMissing(ImportError):
    pass


class DpfError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class ModelDesc(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int32), ("d", ctypes.c_int32), ("dy", ctypes.c_int32),
        ("precision", ctypes.c_int32), ("growth_x", ctypes.c_int32), ("quad_obs", ctypes.c_int32),
        ("perm", ctypes.c_void_p), ("A", ctypes.c_void_p), ("Q", ctypes.c_void_p),
        ("H", ctypes.c_void_p), ("R", ctypes.c_void_p), ("m0", ctypes.c_void_p),
        ("P0", ctypes.c_void_p), ("growth", ctypes.c_double * 4), ("qc", ctypes.c_double),
    ]


_lib = None

# (name, restype, argtypes) of every entry point of include/dpf.h
_P, _I32, _I64, _U64, _SZ = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_size_t
SIGNATURES = [
    ("dpf_create", ctypes.c_int, [_P, _I32, _I32, _I64, _I32, _I32, _U64, _P, _P]),
    ("dpf_step", ctypes.c_int, [_P, _P, _I32, _P, _P]),
    ("dpf_step_async", ctypes.c_int, [_P, _P, _P, _P]),
    ("dpf_sync", ctypes.c_int, [_P]),
    ("dpf_resample", ctypes.c_int, [_P, _I32, _I64, _I64, _I32, _P, _P, _P]),
    ("dpf_resample_noalloc", ctypes.c_int, [_P, _I32, _I64, _P, _P, _P]),
    ("dpf_box_muller", ctypes.c_int, [_P, _I64, _I32, _P, _P]),
    ("dpf_tc_matmul", ctypes.c_int, [_P, _P, _P, _I32, _I32, _I32, _I32, _P]),
    ("dpf_diag", ctypes.c_int, [_P, _P, _P, _P]),
    ("dpf_read", ctypes.c_int, [_P, ctypes.c_char_p, _P, _SZ]),
    ("dpf_set_tensor_cores", ctypes.c_int, [_P, _I32]),
    ("dpf_set_debug", ctypes.c_int, [_P, _I32]),
    ("dpf_profile", ctypes.c_int, [_P, _I32]),
    ("dpf_profile_read", ctypes.c_int, [_P, _P, _P]),
    ("dpf_memory", ctypes.c_int, [_P, _P]),
    ("dpf_batch_create", ctypes.c_int, [_P, _P, _P, _P, _I32, _P, _I32, _P, _P]),
    ("dpf_batch_step", ctypes.c_int, [_P, _P, _P, _P]),
    ("dpf_batch_run", ctypes.c_int, [_P, _P, _I64, _P, _P, _I32]),
    ("dpf_batch_autotune", ctypes.c_int, [_P, _I32, ctypes.c_char_p, _SZ]),
    ("dpf_batch_filter", ctypes.c_int, [_P, _I32, _P]),
    ("dpf_batch_sync", ctypes.c_int, [_P]),
    ("dpf_batch_profile", ctypes.c_int, [_P, _I32]),
    ("dpf_batch_profile_read", ctypes.c_int, [_P, _P, _P]),
    ("dpf_batch_destroy", None, [_P]),
    ("dpf_destroy", None, [_P]),
    ("dpf_last_error", ctypes.c_char_p, []),
]


def lib():
    """Load ``libdpf.so`` (raises DpfLibraryMissing when it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise DpfLibraryMissing(
                f"{LIB_PATH} is missing: build it with paper_1203_2394_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, res, args in SIGNATURES:
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def check(status: int):
    if status != DPF_OK:
        raise DpfError(status, lib().dpf_last_error().decode())


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)  # a torch.cuda.Stream


class Model:
    """Model descriptor; arrays are kept alive for the lifetime of this object."""

    def __init__(self, d, dy, A, Q, H, R, m0, P0, precision=DPF_F32, growth=None, qc=None,
                 perm=None):
        f = lambda a: np.ascontiguousarray(a, dtype=np.float64)
        self.arrays = [f(A), f(Q), f(H), f(R), f(m0), f(P0)]
        self.perm = None if perm is None else np.ascontiguousarray(perm, dtype=np.int32)
        self.d, self.dy, self.precision = int(d), int(dy), int(precision)
        ptr = lambda a: a.ctypes.data
        g = (ctypes.c_double * 4)(*(growth if growth is not None else (0.0, 0.0, 0.0, 0.0)))
        self.desc = ModelDesc(DPF_MODEL_CLG, self.d, self.dy, self.precision,
                              int(growth is not None), int(qc is not None),
                              None if self.perm is None else ptr(self.perm),
                              *[ptr(a) for a in self.arrays], g,
                              float(qc if qc is not None else 0.0))

    @classmethod
    def from_spec(cls, spec, precision=DPF_F32, perm=None):
        return cls(spec.d, spec.dy, spec.A, spec.Q, spec.H, spec.R, spec.m0, spec.P0, precision,
                   spec.growth, spec.qc, perm)


class Filter:
    """One LA-DPF filter (``dpf_create`` ... ``dpf_destroy``)."""

    def __init__(self, model: Model, d1: int, d2: int, N: int, M: int, L: int, seed: int = 0,
                 stream=None):
        self.model = model
        self.d1, self.d2, self.N, self.M, self.L = int(d1), int(d2), int(N), int(M), int(L)
        self.d, self.dy = model.d, model.dy
        self.dtype = np.float64 if model.precision == DPF_F64 else np.float32
        self._lib = lib()
        h = ctypes.c_void_p()
        check(self._lib.dpf_create(ctypes.byref(model.desc), self.d1, self.d2, self.N, self.M,
                                   self.L, ctypes.c_uint64(seed), _stream_ptr(stream),
                                   ctypes.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self._lib.dpf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, y):
        """Host observation in, host outputs back (synchronises)."""
        y = np.ascontiguousarray(y, dtype=self.dtype)
        mean = np.zeros(self.d)
        logz = ctypes.c_double()
        check(self._lib.dpf_step(self.h, y.ctypes.data, 0, mean.ctypes.data, ctypes.byref(logz)))
        return mean, logz.value

    def step_device(self, y_ptr: int, mean_ptr: int | None = None, logz_ptr: int | None = None):
        """Device observation and device outputs (stream-ordered, no synchronisation)."""
        check(self._lib.dpf_step_async(self.h, y_ptr, mean_ptr, logz_ptr))

    def sync(self):
        check(self._lib.dpf_sync(self.h))

    def diag(self):
        ess = ctypes.c_double(); st = ctypes.c_int64(); lz = ctypes.c_double()
        check(self._lib.dpf_diag(self.h, ctypes.byref(ess), ctypes.byref(st), ctypes.byref(lz)))
        return dict(ess=ess.value, step=st.value, logZ_step=lz.value)

    _SHAPES = {
        "lw": lambda s: (s.N,), "lwhat": lambda s: (s.N, s.L), "xbb": lambda s: (s.N, s.L, s.d1),
        "anc": lambda s: (s.N,), "sel": lambda s: (s.N,), "wout": lambda s: (s.N,),
        "x": lambda s: (s.N, s.d1), "z": lambda s: (s.d2, s.N, s.M), "lq": lambda s: (s.N, s.M),
        "bidx": lambda s: (s.N, s.M),
    }

    def read(self, which: str) -> np.ndarray:
        shape = self._SHAPES[which](self)
        dt = np.int32 if which in ("anc", "sel", "bidx") else self.dtype
        out = np.zeros(shape, dtype=dt)
        check(self._lib.dpf_read(self.h, which.encode(), out.ctypes.data, out.nbytes))
        return out

    def set_debug(self, on=True):
        check(self._lib.dpf_set_debug(self.h, int(on)))

    def set_tensor_cores(self, on=True):
        check(self._lib.dpf_set_tensor_cores(self.h, int(on)))

    def profile(self, on=True):
        check(self._lib.dpf_profile(self.h, int(on)))

    def profile_read(self):
        ms = ctypes.c_double(); n = ctypes.c_int64()
        check(self._lib.dpf_profile_read(self.h, ctypes.byref(ms), ctypes.byref(n)))
        return ms.value, n.value

    def memory(self) -> int:
        b = ctypes.c_size_t()
        check(self._lib.dpf_memory(self.h, ctypes.byref(b)))
        return b.value


class _Borrowed(Filter):
    """A batch member's context viewed as a Filter (owned by the batch)."""

    def __init__(self, h, model, d1, d2, N, M, L):
        self.model = model
        self.d1, self.d2, self.N, self.M, self.L = d1, d2, N, M, L
        self.d, self.dy = model.d, model.dy
        self.dtype = np.float64 if model.precision == DPF_F64 else np.float32
        self._lib = lib()
        self.h = h

    def close(self):
        self.h = None


class Batch:
    """Many filters stepped together (``dpf_batch_*``)."""

    def __init__(self, models, d1s, Ns, Ms, L, seeds, stream=None):
        self.models = list(models)
        F = len(self.models)
        self.F, self.L = F, int(L)
        self.d, self.dy = self.models[0].d, self.models[0].dy
        self.d1s = [int(v) for v in d1s]
        self.Ns = [int(v) for v in Ns]
        self.Ms = [int(v) for v in Ms]
        descs = (ctypes.c_void_p * F)(*[ctypes.addressof(m.desc) for m in self.models])
        d1a = (ctypes.c_int32 * F)(*self.d1s)
        Na = (ctypes.c_int64 * F)(*self.Ns)
        Ma = (ctypes.c_int32 * F)(*self.Ms)
        Sa = (ctypes.c_uint64 * F)(*[int(s) for s in seeds])
        self._lib = lib()
        h = ctypes.c_void_p()
        check(self._lib.dpf_batch_create(descs, d1a, Na, Ma, self.L, Sa, F, _stream_ptr(stream),
                                         ctypes.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self._lib.dpf_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step_device(self, y_ptr, means_ptr=None, logz_ptr=None):
        check(self._lib.dpf_batch_step(self.h, y_ptr, means_ptr, logz_ptr))

    def run_device(self, ys_ptr, T, means_ptr=None, logz_ptr=None, graph=True):
        check(self._lib.dpf_batch_run(self.h, ys_ptr, int(T), means_ptr, logz_ptr, int(bool(graph))))

    def sync(self):
        check(self._lib.dpf_batch_sync(self.h))

    def autotune(self, reps=3):
        buf = ctypes.create_string_buffer(1 << 16)
        check(self._lib.dpf_batch_autotune(self.h, int(reps), buf, len(buf)))
        import json
        return json.loads(buf.value.decode())

    def profile(self, on=True):
        check(self._lib.dpf_batch_profile(self.h, int(on)))

    def profile_read(self):
        ms = ctypes.c_double(); n = ctypes.c_int64()
        check(self._lib.dpf_batch_profile_read(self.h, ctypes.byref(ms), ctypes.byref(n)))
        return ms.value, n.value

    def filter(self, f) -> Filter:
        h = ctypes.c_void_p()
        check(self._lib.dpf_batch_filter(self.h, int(f), ctypes.byref(h)))
        return _Borrowed(h, self.models[f], self.d1s[f], self.d - self.d1s[f], self.Ns[f],
                         self.Ms[f], self.L)


def resample(w, u, rule=DPF_SYS_GLOBAL, n_seg=1, out=None, stream=None):
    """Systematic resampling of device tensors (torch): w (float32/float64), u (uint32 words
    as int32/uint32 tensor of n_seg entries); returns int32 indices (segment-local)."""
    import torch
    assert w.is_cuda and u.is_cuda and w.is_contiguous() and u.is_contiguous()
    dtype = {torch.float32: DPF_F32, torch.float64: DPF_F64}[w.dtype]
    if out is None:
        out = torch.empty(w.numel(), dtype=torch.int32, device=w.device)
    s = stream if stream is not None else torch.cuda.current_stream(w.device)
    check(lib().dpf_resample(w.data_ptr(), dtype, w.numel(), int(n_seg), int(rule), u.data_ptr(),
                             out.data_ptr(), _stream_ptr(s)))
    return out


def resample_noalloc(w, u, out=None, stream=None):
    """Global systematic resampling through the allocation-free entry point (scratch in a
    fixed per-device array; at most 4,194,304 weights; calls must not overlap on the GPU)."""
    import torch
    assert w.is_cuda and u.is_cuda and w.is_contiguous() and u.is_contiguous()
    dtype = {torch.float32: DPF_F32, torch.float64: DPF_F64}[w.dtype]
    if out is None:
        out = torch.empty(w.numel(), dtype=torch.int32, device=w.device)
    s = stream if stream is not None else torch.cuda.current_stream(w.device)
    check(lib().dpf_resample_noalloc(w.data_ptr(), dtype, w.numel(), u.data_ptr(), out.data_ptr(),
                                     _stream_ptr(s)))
    return out


def box_muller(words, dtype="float32", stream=None):
    """The library's normal transform on device words (torch int32 tensor holding the
    uint32 bit patterns, 2 per pair); returns a device tensor of 2 n_pairs normals."""
    import torch
    assert words.is_cuda and words.dtype == torch.int32 and words.numel() % 2 == 0
    tdt = {"float32": torch.float32, "float64": torch.float64}[dtype]
    out = torch.empty(words.numel(), dtype=tdt, device=words.device)
    s = stream if stream is not None else torch.cuda.current_stream(words.device)
    check(lib().dpf_box_muller(words.data_ptr(), words.numel() // 2,
                               DPF_F32 if dtype == "float32" else DPF_F64, out.data_ptr(),
                               _stream_ptr(s)))
    return out


DPF_TC_TF32, DPF_TC_TF32X3, DPF_TC_BF16 = 0, 1, 2


def tc_matmul(A, B, mode=DPF_TC_TF32X3, stream=None):
    """D = A B^T on the tensor cores (see ``dpf_tc_matmul``). A: (M, K), B: (N, K)
    CUDA tensors, float32 (TF32 modes) or bfloat16 (DPF_TC_BF16); returns D (M, N) float32."""
    import torch
    M, K = A.shape
    N = B.shape[0]
    D = torch.empty((M, N), dtype=torch.float32, device=A.device)
    s = stream if stream is not None else torch.cuda.current_stream().cuda_stream
    check(lib().dpf_tc_matmul(A.data_ptr(), B.data_ptr(), D.data_ptr(), M, N, K, int(mode), s))
    return D
