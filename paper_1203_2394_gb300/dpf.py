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
DPF_MODEL_CLG, DPF_MODEL_PAPER1, DPF_MODEL_PAPER2 = 1, 2, 3
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
    ("dpf_check_bounded_wait", ctypes.c_int, [_P]),
    ("dpf_fail_allocation_after", ctypes.c_int, [ctypes.c_int64]),
    ("dpf_diag", ctypes.c_int, [_P, _P, _P, _P]),
    ("dpf_diag_inner", ctypes.c_int, [_P, _P, _P]),
    ("dpf_create_pf", ctypes.c_int, [_P, _I32, _I32, _I64, _U64, _P, _P]),
    ("dpf_create_std", ctypes.c_int, [_P, _I32, _I32, _I64, _I32, _U64, _P, _P]),
    ("dpf_set_gaussian_approx", ctypes.c_int, [_P, _I32]),
    ("dpf_read", ctypes.c_int, [_P, ctypes.c_char_p, _P, _SZ]),
    ("dpf_proposal_create", ctypes.c_int, [_I32, _I32, _I32, _I32, _I32, _P, _P]),
    ("dpf_proposal_create_amortised", ctypes.c_int, [_I32, _I32, _I32, _I32, _P, _P, _P]),
    ("dpf_proposal_num_params", ctypes.c_int, [_P, _P]),
    ("dpf_proposal_set_weights", ctypes.c_int, [_P, _P, _I64]),
    ("dpf_proposal_get_weights", ctypes.c_int, [_P, _P, _I64]),
    ("dpf_proposal_set_bf16", ctypes.c_int, [_P, _I32]),
    ("dpf_proposal_set_centre", ctypes.c_int, [_P, _I32]),
    ("dpf_proposal_loss_grad", ctypes.c_int, [_P, _P, _P, _P, _I64, _P, _P]),
    ("dpf_proposal_adam_step", ctypes.c_int, [_P, _P, ctypes.c_float]),
    ("dpf_proposal_train", ctypes.c_int, [_P, _P, _P, _P, _I64, _I32, _I32, ctypes.c_float, _U64, _P]),
    ("dpf_proposal_forward", ctypes.c_int, [_P, _P, _I64, _P]),
    ("dpf_proposal_destroy", None, [_P]),
    ("dpf_set_proposal", ctypes.c_int, [_P, _P]),
    ("dpf_record_tuples", ctypes.c_int, [_P, _I64, _I64, _P, _P, _P]),
    ("dpf_record_tuples_amortised", ctypes.c_int, [_P, _I64, _I64, _P, _P, _P]),
    ("dpf_state_bytes", ctypes.c_int, [_P, _P]),
    ("dpf_get_state", ctypes.c_int, [_P, _P, _SZ]),
    ("dpf_set_state", ctypes.c_int, [_P, _P, _SZ]),
    ("dpf_set_fallback", ctypes.c_int, [_P, ctypes.c_double]),
    ("dpf_bandit_create", ctypes.c_int, [_I32, _I32, ctypes.c_double, ctypes.c_double, _U64, _P]),
    ("dpf_bandit_probs", ctypes.c_int, [_P, _P]),
    ("dpf_bandit_choose", ctypes.c_int, [_P, _P]),
    ("dpf_bandit_update", ctypes.c_int, [_P, _P]),
    ("dpf_bandit_reward", ctypes.c_int, [_P, _P, _I32, ctypes.c_double, _P]),
    ("dpf_bandit_destroy", None, [_P]),
    ("dpf_set_tensor_cores", ctypes.c_int, [_P, _I32]),
    ("dpf_set_debug", ctypes.c_int, [_P, _I32]),
    ("dpf_profile", ctypes.c_int, [_P, _I32]),
    ("dpf_profile_read", ctypes.c_int, [_P, _P, _P]),
    ("dpf_memory", ctypes.c_int, [_P, _P]),
    ("dpf_batch_create", ctypes.c_int, [_P, _P, _P, _P, _I32, _P, _I32, _P, _P]),
    ("dpf_batch_step", ctypes.c_int, [_P, _P, _P, _P]),
    ("dpf_batch_run", ctypes.c_int, [_P, _P, _I64, _P, _P, _I32]),
    ("dpf_batch_autotune", ctypes.c_int, [_P, _I32, ctypes.c_char_p, _SZ]),
    ("dpf_batch_set_split", ctypes.c_int, [_P, _I32]),
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


class PaperModel(Model):
    """The paper's benchmark model 1 (d = 2) or 2 (d = 4) of Table 1, FP32; the filter is
    created with d1 = d2 = d / 2 (the matrices of the descriptor are not used). perm = (1, 0)
    decomposes model 1 the other way: the table's z outer, its x inner."""

    def __init__(self, kind: int, perm=None):
        if kind not in (1, 2):
            raise ValueError("kind must be 1 or 2")
        self.arrays = []
        self.perm = None if perm is None else np.ascontiguousarray(perm, dtype=np.int32)
        self.d, self.dy, self.precision = (2 if kind == 1 else 4), 1, DPF_F32
        self.d1 = self.d2 = self.d // 2
        g = (ctypes.c_double * 4)(0.0, 0.0, 0.0, 0.0)
        self.desc = ModelDesc(DPF_MODEL_PAPER1 if kind == 1 else DPF_MODEL_PAPER2, self.d, self.dy,
                              self.precision, 0, 0, None if self.perm is None else self.perm.ctypes.data,
                              None, None, None, None, None, None, g, 0.0)


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
        "xm": lambda s: (s.d1, s.N), "zm": lambda s: (s.d2, s.N),
        "x": lambda s: (s.N, s.d1), "z": lambda s: (s.d2, s.N, s.M), "lq": lambda s: (s.N, s.M),
        "bidx": lambda s: (s.N, s.M), "fallback": lambda s: (s.N,), "jla": lambda s: (s.N, s.L),
        "head": lambda s: (s.N, s.M, s.proposal.dout),
        "afeat": lambda s: (s.N, 2 * s.d1 + s.dy + 2 * s.d2),
        "ahead": lambda s: (s.N, 2 * s.d2),
    }

    def diag_inner(self):
        """Minimum and mean over the groups of the inner effective sample size."""
        lo = ctypes.c_double(); mean = ctypes.c_double()
        check(self._lib.dpf_diag_inner(self.h, ctypes.byref(lo), ctypes.byref(mean)))
        return dict(ess_inner_min=lo.value, ess_inner_mean=mean.value)

    def read(self, which: str) -> np.ndarray:
        shape = self._SHAPES[which](self)
        dt = np.int32 if which in ("anc", "sel", "bidx", "fallback", "jla") else self.dtype
        out = np.zeros(shape, dtype=dt)
        check(self._lib.dpf_read(self.h, which.encode(), out.ctypes.data, out.nbytes))
        return out

    def set_debug(self, on=True):
        check(self._lib.dpf_set_debug(self.h, int(on)))

    def set_fallback(self, frac):
        """Learned proposal: groups with inner ESS below frac * M redo the plain update."""
        check(self._lib.dpf_set_fallback(self.h, float(frac)))

    def set_tensor_cores(self, on=True):
        check(self._lib.dpf_set_tensor_cores(self.h, int(on)))

    def state_bytes(self) -> int:
        n = ctypes.c_size_t()
        check(self._lib.dpf_state_bytes(self.h, ctypes.byref(n)))
        return n.value

    def get_state(self):
        """A checkpoint of the filter (a device uint8 tensor)."""
        import torch
        buf = torch.empty(self.state_bytes(), dtype=torch.uint8, device="cuda")
        check(self._lib.dpf_get_state(self.h, buf.data_ptr(), buf.numel()))
        return buf

    def set_state(self, buf):
        check(self._lib.dpf_set_state(self.h, buf.data_ptr(), buf.numel()))

    def set_proposal(self, proposal):
        """Use a learned inner proposal from the next step on (None: the prior)."""
        check(self._lib.dpf_set_proposal(self.h, proposal.h if proposal is not None else None))
        self.proposal = proposal

    def record_amortised(self, i0=0, n_outer=None):
        """Training rows of the last inner update for the outer-amortised proposal: device
        tensors G (n, 2 d1 + dy + 2 d2), Z (n, 3 d2), w (n)."""
        import torch
        n_outer = self.N - i0 if n_outer is None else n_outer
        din = 2 * self.d1 + self.dy + 2 * self.d2
        n = n_outer * self.M
        G = torch.empty((n, din), dtype=torch.float32, device="cuda")
        Z = torch.empty((n, 3 * self.d2), dtype=torch.float32, device="cuda")
        w = torch.empty((n,), dtype=torch.float32, device="cuda")
        check(self._lib.dpf_record_tuples_amortised(self.h, int(i0), int(n_outer), G.data_ptr(), Z.data_ptr(),
                                                    w.data_ptr()))
        return G, Z, w

    def record(self, i0=0, n_outer=None):
        """Training rows of the last inner update (see ``dpf_record_tuples``): device
        tensors F (n, din), Z (n, d2), w (n)."""
        import torch
        n_outer = self.N - i0 if n_outer is None else n_outer
        din = 2 * self.d1 + self.d2 + self.dy
        n = n_outer * self.M
        F = torch.empty((n, din), dtype=torch.float32, device="cuda")
        Z = torch.empty((n, self.d2), dtype=torch.float32, device="cuda")
        w = torch.empty((n,), dtype=torch.float32, device="cuda")
        check(self._lib.dpf_record_tuples(self.h, int(i0), int(n_outer), F.data_ptr(), Z.data_ptr(),
                                          w.data_ptr()))
        return F, Z, w

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


class ParticleFilter(Filter):
    """The bootstrap particle filter over the full state (``dpf_create_pf``): N
    particles; ``step`` returns the weighted mean and the cumulative log-evidence."""

    def __init__(self, model: Model, d1: int, d2: int, N: int, seed: int = 0, stream=None):
        self.model = model
        self.d1, self.d2, self.N, self.M, self.L = int(d1), int(d2), int(N), 1, 1
        self.d, self.dy = model.d, model.dy
        self.dtype = np.float64 if model.precision == DPF_F64 else np.float32
        self._lib = lib()
        h = ctypes.c_void_p()
        check(self._lib.dpf_create_pf(ctypes.byref(model.desc), self.d1, self.d2, self.N,
                                      ctypes.c_uint64(seed), _stream_ptr(stream), ctypes.byref(h)))
        self.h = h


class StandardDPF(Filter):
    """The decentralized particle filter without look-ahead (``dpf_create_std``): N outer
    particles with M inner particles each."""

    def __init__(self, model: Model, d1: int, d2: int, N: int, M: int, seed: int = 0, stream=None):
        self.model = model
        self.d1, self.d2, self.N, self.M, self.L = int(d1), int(d2), int(N), int(M), 1
        self.d, self.dy = model.d, model.dy
        self.dtype = np.float64 if model.precision == DPF_F64 else np.float32
        self._lib = lib()
        h = ctypes.c_void_p()
        check(self._lib.dpf_create_std(ctypes.byref(model.desc), self.d1, self.d2, self.N, self.M,
                                       ctypes.c_uint64(seed), _stream_ptr(stream), ctypes.byref(h)))
        self.h = h

    def set_gaussian_approx(self, on=True):
        """Draw x_t from the mixture's moment-matched Gaussian (Section 4.2)."""
        check(self._lib.dpf_set_gaussian_approx(self.h, int(on)))


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

    def set_split(self, split=True):
        """Every class of several filters as one launch a filter (True) or one launch
        (False), by hand; the results do not depend on it."""
        check(self._lib.dpf_batch_set_split(self.h, int(bool(split))))

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


class Proposal:
    """The learned inner proposal (``dpf_proposal_*``): an MLP of three hidden ReLU layers
    with a Gaussian-mixture head (per inner particle), or with the Qz given, the
    outer-amortised form (one row per outer particle, a diagonal affine map of the
    group's prior draws); trained on the GPU by the library's kernels."""

    def __init__(self, d1, d2, dy, hidden=256, components=4, stream=None, amortised_Qz=None):
        self.d1, self.d2, self.dy = int(d1), int(d2), int(dy)
        self.hidden = int(hidden)
        self._lib = lib()
        h = ctypes.c_void_p()
        if amortised_Qz is None:
            self.kind, self.C = 0, int(components)
            self.din = 2 * self.d1 + self.d2 + self.dy
            self.dout = self.C * (1 + 2 * self.d2)
            check(self._lib.dpf_proposal_create(self.d1, self.d2, self.dy, self.hidden, self.C,
                                                _stream_ptr(stream), ctypes.byref(h)))
        else:
            self.kind, self.C = 1, 1
            self.din = 2 * self.d1 + self.dy + 2 * self.d2
            self.dout = 2 * self.d2
            q = np.ascontiguousarray(amortised_Qz, dtype=np.float64)
            check(self._lib.dpf_proposal_create_amortised(self.d1, self.d2, self.dy, self.hidden,
                                                          q.ctypes.data, _stream_ptr(stream),
                                                          ctypes.byref(h)))
        self.h = h
        n = ctypes.c_int64()
        check(self._lib.dpf_proposal_num_params(self.h, ctypes.byref(n)))
        self.nparams = n.value

    def close(self):
        if getattr(self, "h", None):
            self._lib.dpf_proposal_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def layout(self):
        """(name, shape) of every parameter block in the library's order."""
        H, out = [], []
        sizes = [(self.hidden, self.din), (self.hidden, self.hidden), (self.hidden, self.hidden),
                 (self.dout, self.hidden)]
        for l, (r, c) in enumerate(sizes, 1):
            out += [(f"W{l}", (r, c)), (f"b{l}", (r,))]
        return out

    def flatten(self, W):
        return np.concatenate([np.asarray(W[k], np.float32).ravel() for k, _ in self.layout()])

    def unflatten(self, flat):
        W, o = {}, 0
        for k, shp in self.layout():
            n = int(np.prod(shp))
            W[k] = flat[o:o + n].reshape(shp).astype(np.float64)
            o += n
        return W

    def set_weights(self, W):
        flat = np.ascontiguousarray(self.flatten(W))
        check(self._lib.dpf_proposal_set_weights(self.h, flat.ctypes.data, flat.size))

    def get_weights(self):
        flat = np.zeros(self.nparams, np.float32)
        check(self._lib.dpf_proposal_get_weights(self.h, flat.ctypes.data, flat.size))
        return self.unflatten(flat)

    def set_bf16(self, on=True):
        check(self._lib.dpf_proposal_set_bf16(self.h, int(on)))

    def set_centre(self, per_particle=True):
        """The outer-amortised map's centre: the particle's own prior mean (True) or the
        group's mean prior mean (False, the default); see ``dpf_proposal_set_centre``."""
        check(self._lib.dpf_proposal_set_centre(self.h, int(per_particle)))
        self.centre = "particle" if per_particle else "group"

    def loss_grad(self, F, Z, w, grad=True):
        """Weighted NLL and (optionally) its gradient (device tensor of num_params)."""
        import torch
        loss = ctypes.c_double()
        g = torch.empty(self.nparams, dtype=torch.float32, device=F.device) if grad else None
        check(self._lib.dpf_proposal_loss_grad(self.h, F.data_ptr(), Z.data_ptr(), w.data_ptr(),
                                               F.shape[0], ctypes.byref(loss),
                                               g.data_ptr() if g is not None else None))
        return loss.value, g

    def adam_step(self, grad, lr):
        check(self._lib.dpf_proposal_adam_step(self.h, grad.data_ptr(), ctypes.c_float(lr)))

    def train(self, F, Z, w, batch=1024, epochs=1, lr=1e-3, seed=0):
        losses = np.zeros(epochs)
        check(self._lib.dpf_proposal_train(self.h, F.data_ptr(), Z.data_ptr(), w.data_ptr(),
                                           F.shape[0], int(batch), int(epochs), ctypes.c_float(lr),
                                           ctypes.c_uint64(seed), losses.ctypes.data))
        return losses

    def forward(self, F):
        """Head outputs by the tensor-core pass (device tensor (n, dout))."""
        import torch
        out = torch.empty((F.shape[0], self.dout), dtype=torch.float32, device=F.device)
        check(self._lib.dpf_proposal_forward(self.h, F.data_ptr(), F.shape[0], out.data_ptr()))
        return out


def check_bounded_wait(stream=None):
    """Run the scan whose look-back can never finish (see ``dpf_check_bounded_wait``);
    raises DpfError with status DPF_E_TIMEOUT when the waits give up as designed."""
    import torch
    s = stream if stream is not None else torch.cuda.current_stream().cuda_stream
    check(lib().dpf_check_bounded_wait(s))


def fail_allocation_after(n: int):
    """Arm the library's allocation-failure countdown (``dpf_fail_allocation_after``): the
    n-th device allocation of a context, batch or proposal from now fails; 0 disarms."""
    check(lib().dpf_fail_allocation_after(int(n)))


DPF_HEDGE, DPF_EXP3 = 0, 1


class Bandit:
    """Hedge or Exp3 over K decompositions (``dpf_bandit_*``)."""

    def __init__(self, kind, K, eta, gamma=0.0, seed=0):
        self.kind, self.K = int(kind), int(K)
        self._lib = lib()
        h = ctypes.c_void_p()
        check(self._lib.dpf_bandit_create(self.kind, self.K, float(eta), float(gamma),
                                          ctypes.c_uint64(seed), ctypes.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self._lib.dpf_bandit_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def probs(self):
        p = np.zeros(self.K)
        check(self._lib.dpf_bandit_probs(self.h, p.ctypes.data))
        return p

    def choose(self):
        a = ctypes.c_int32()
        check(self._lib.dpf_bandit_choose(self.h, ctypes.byref(a)))
        return a.value

    def update(self, rewards):
        r = np.ascontiguousarray(np.atleast_1d(rewards), dtype=np.float64)
        check(self._lib.dpf_bandit_update(self.h, r.ctypes.data))


def bandit_reward(y, yhat, alpha):
    """``dpf_bandit_reward``: alpha / (alpha + |y - yhat|^2)."""
    y = np.ascontiguousarray(y, dtype=np.float64).ravel()
    yh = np.ascontiguousarray(yhat, dtype=np.float64).ravel()
    r = ctypes.c_double()
    check(lib().dpf_bandit_reward(y.ctypes.data, yh.ctypes.data, y.size, float(alpha), ctypes.byref(r)))
    return r.value
