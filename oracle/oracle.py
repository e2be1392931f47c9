"""ctypes wrapper of the FP64 C oracle (``dpf_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may use this module; the library path never
does. It imports nothing from the CUDA package.

Arrays follow the oracle's array-of-structures layout (see the C file header):
``x[N, d1]``, ``z[N, M, d2]``, ``lq[N, M]``, ``xbb[N, L, d1]``, ``lwhat[N, L]``.
Model matrices are given in the x-first coordinate order.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dpf_oracle.c")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

P_INIT_X, P_INIT_Z, P_LA_J, P_LA_X, P_LA_Z, P_OUTER, P_SEL, P_INNER, P_PROP = range(1, 10)
P_LCOMP = 10  # mixture-component draw of the learned inner proposal


def build(force: bool = False, extra_flags: tuple = ()) -> str:
    """Compile the oracle with gcc (plain -O2, OpenMP); returns the .so path."""
    out = _OUT
    if extra_flags:
        tag = "_".join(f.strip("-").replace("=", "") for f in extra_flags)
        out = os.path.join(_HERE, "_build", f"liboracle_{tag}.so")
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
        return out
    os.makedirs(os.path.dirname(out), exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fopenmp", *extra_flags, _SRC,
           "-o", tmp, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, out)
    return out


class ModelIn(ctypes.Structure):
    _fields_ = [
        ("d1", ctypes.c_int32), ("d2", ctypes.c_int32), ("dy", ctypes.c_int32),
        ("growth_x", ctypes.c_int32), ("quad_obs", ctypes.c_int32), ("reserved", ctypes.c_int32),
        ("ga", ctypes.c_double), ("gb", ctypes.c_double), ("gc", ctypes.c_double),
        ("gw", ctypes.c_double), ("qc", ctypes.c_double),
        ("A", ctypes.c_void_p), ("Q", ctypes.c_void_p), ("H", ctypes.c_void_p),
        ("R", ctypes.c_void_p), ("m0", ctypes.c_void_p), ("P0", ctypes.c_void_p),
    ]


class Dims(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int64), ("M", ctypes.c_int32), ("L", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("filter_id", ctypes.c_uint32),
                ("nthreads", ctypes.c_int32)]


def load(path: str | None = None):
    global _lib
    with _lock:
        if path is not None:
            lib = ctypes.CDLL(path)
        else:
            if _lib is not None:
                return _lib
            lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        lib.ora_philox4x32_10.argtypes = [P, P, P]
        lib.ora_u01.argtypes = [ctypes.c_uint32]
        lib.ora_u01.restype = ctypes.c_double
        lib.ora_box_muller.argtypes = [ctypes.c_uint32, ctypes.c_uint32, P, P]
        lib.ora_normals.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                    ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                    ctypes.c_int, P]
        lib.ora_normals_many.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                         ctypes.c_int64, P, ctypes.c_uint32, P, ctypes.c_int, P]
        lib.ora_sys_global.argtypes = [P, ctypes.c_int64, ctypes.c_uint32, P]
        lib.ora_sys_local.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_uint32, P]
        lib.ora_init.argtypes = [P, P, P, P, P]
        lib.ora_lookahead.argtypes = [P, P, ctypes.c_uint32, P, ctypes.c_int64, P, P, P, P, P, P,
                                      P, P, P]
        lib.ora_finalize.argtypes = [P, P, ctypes.c_uint32, P, ctypes.c_int64, P, P, P, P, P, P,
                                     P, P, P, P, P]
        lib.ora_step.argtypes = [P, P, ctypes.c_uint32, P] + [P] * 19
        if path is None:
            _lib = lib
        return lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class OracleModel:
    """Model in the x-first coordinate order, kept alive for the ctypes pointers."""

    def __init__(self, d1, d2, dy, A, Q, H, R, m0, P0, growth=None, qc=None):
        self.d1, self.d2, self.dy = int(d1), int(d2), int(dy)
        self.A, self.Q, self.H, self.R = _f64(A), _f64(Q), _f64(H), _f64(R)
        self.m0, self.P0 = _f64(m0), _f64(P0)
        self.growth, self.qc = growth, qc
        g = growth if growth is not None else (0.0, 0.0, 0.0, 0.0)
        self.s = ModelIn(self.d1, self.d2, self.dy, int(growth is not None), int(qc is not None), 0,
                         float(g[0]), float(g[1]), float(g[2]), float(g[3]),
                         float(qc if qc is not None else 0.0),
                         _ptr(self.A).value, _ptr(self.Q).value, _ptr(self.H).value,
                         _ptr(self.R).value, _ptr(self.m0).value, _ptr(self.P0).value)

    @classmethod
    def from_spec(cls, spec, d1=None):
        """Build from a workload spec (see ``workloads.ModelSpec``), permuted x-first."""
        p = np.asarray(spec.perm(d1))
        A = spec.A[np.ix_(p, p)]
        Q = spec.Q[np.ix_(p, p)]
        H = spec.H[:, p]
        P0 = spec.P0[np.ix_(p, p)]
        m0 = spec.m0[p]
        dd1 = spec.d1 if d1 is None else d1
        return cls(dd1, spec.d - dd1, spec.dy, A, Q, H, spec.R, m0, P0, spec.growth, spec.qc)


class Oracle:
    """Stateless calls into the C oracle for one model and filter size."""

    def __init__(self, model: OracleModel, N, M, L, seed, filter_id=0, nthreads=1, lib=None):
        self.m = model
        self.N, self.M, self.L = int(N), int(M), int(L)
        self.dims = Dims(self.N, self.M, self.L, int(seed), int(filter_id), int(nthreads))
        self.lib = lib if lib is not None else load()

    def _check(self, st, what):
        if st != 0:
            raise RuntimeError(f"oracle {what} failed with status {st}")

    def init(self):
        m, N, M = self.m, self.N, self.M
        x = np.zeros((N, m.d1)); z = np.zeros((N, M, m.d2)); lq = np.zeros((N, M))
        self._check(self.lib.ora_init(ctypes.byref(m.s), ctypes.byref(self.dims), _ptr(x), _ptr(z),
                                      _ptr(lq)), "init")
        return x, z, lq

    def step(self, t, y, x, z, lq, anc=None, sel=None, bidx=None):
        """One full step from the state at t-1. anc, sel, bidx (optional): replay the
        given outer ancestors (N), selected draws (N) and local resampling indices
        (N, M) instead of drawing them."""
        m, N, M, L = self.m, self.N, self.M, self.L
        y = _f64(y); x = _f64(x); z = _f64(z); lq = _f64(lq)
        anc_in = None if anc is None else np.ascontiguousarray(anc, dtype=np.int32)
        sel_in = None if sel is None else np.ascontiguousarray(sel, dtype=np.int32)
        bidx_in = None if bidx is None else np.ascontiguousarray(bidx, dtype=np.int32)
        out = dict(
            x=np.zeros((N, m.d1)), z=np.zeros((N, M, m.d2)), lq=np.zeros((N, M)),
            lw=np.zeros(N), lwhat=np.zeros((N, L)), xbb=np.zeros((N, L, m.d1)),
            jla=np.zeros((N, L), np.int32), anc=np.zeros(N, np.int32), sel=np.zeros(N, np.int32),
            bidx=np.zeros((N, M), np.int32), mean=np.zeros(m.d1 + m.d2))
        logZ = np.zeros(1); ess = np.zeros(1)
        st = self.lib.ora_step(ctypes.byref(m.s), ctypes.byref(self.dims), int(t), _ptr(y), _ptr(x),
                               _ptr(z), _ptr(lq), _ptr(out["x"]), _ptr(out["z"]), _ptr(out["lq"]),
                               _ptr(out["lw"]), _ptr(out["lwhat"]), _ptr(out["xbb"]),
                               _ptr(out["jla"]), _ptr(out["anc"]), _ptr(out["sel"]),
                               _ptr(out["bidx"]), _ptr(out["mean"]), _ptr(logZ), _ptr(ess),
                               _ptr(anc_in), _ptr(sel_in), _ptr(bidx_in))
        self._check(st, "step")
        out["logZ"] = float(logZ[0]); out["ess"] = float(ess[0])
        return out

    def lookahead(self, t, y, idx, x, z, lq):
        m, M, L = self.m, self.M, self.L
        idx = np.ascontiguousarray(idx, dtype=np.int64)
        n = len(idx)
        y = _f64(y); x = _f64(x); z = _f64(z); lq = _f64(lq)
        lw = np.zeros(n); jla = np.zeros((n, L), np.int32); xbb = np.zeros((n, L, m.d1))
        lwhat = np.zeros((n, L)); mu = np.zeros((n, L, m.d2))
        st = self.lib.ora_lookahead(ctypes.byref(m.s), ctypes.byref(self.dims), int(t), _ptr(y), n,
                                    _ptr(idx), _ptr(x), _ptr(z), _ptr(lq), _ptr(lw), _ptr(jla),
                                    _ptr(xbb), _ptr(lwhat), _ptr(mu))
        self._check(st, "lookahead")
        return dict(lw=lw, jla=jla, xbb=xbb, lwhat=lwhat, mu=mu)

    def finalize(self, t, y, idx, anc, x_prev, z_prev, lq_prev, x_new, bidx=None):
        """Step 4 (local resampling, propagation, measurement update) for the outer
        particles idx with ancestors anc. bidx (optional, (n, M)): replay these local
        resampling indices. The result also holds alpha, the local resampling weights."""
        m, M = self.m, self.M
        idx = np.ascontiguousarray(idx, dtype=np.int64)
        anc = np.ascontiguousarray(anc, dtype=np.int32)
        n = len(idx)
        y = _f64(y); x_prev = _f64(x_prev); z_prev = _f64(z_prev); lq_prev = _f64(lq_prev)
        x_new = _f64(x_new)
        bidx_in = None if bidx is None else np.ascontiguousarray(bidx, dtype=np.int32)
        z = np.zeros((n, M, m.d2)); lq = np.zeros((n, M)); bidx = np.zeros((n, M), np.int32)
        alpha = np.zeros((n, M))
        st = self.lib.ora_finalize(ctypes.byref(m.s), ctypes.byref(self.dims), int(t), _ptr(y), n,
                                   _ptr(idx), _ptr(anc), _ptr(x_prev), _ptr(z_prev), _ptr(lq_prev),
                                   _ptr(x_new), _ptr(z), _ptr(lq), _ptr(bidx), _ptr(bidx_in),
                                   _ptr(alpha))
        self._check(st, "finalize")
        return dict(z=z, lq=lq, bidx=bidx, alpha=alpha)

    def run(self, ys, steps=None):
        """Free-running filter over ys[0..T-1] (y_1..y_T); returns per-step outputs."""
        x, z, lq = self.init()
        T = len(ys) if steps is None else steps
        outs = []
        for t in range(1, T + 1):
            o = self.step(t, ys[t - 1], x, z, lq)
            x, z, lq = o["x"], o["z"], o["lq"]
            outs.append(o)
        return outs


def philox(ctr, key, lib=None):
    lib = lib or load()
    c = np.asarray(ctr, dtype=np.uint32); k = np.asarray(key, dtype=np.uint32)
    o = np.zeros(4, np.uint32)
    lib.ora_philox4x32_10(_ptr(c), _ptr(k), _ptr(o))
    return o


def normals(seed, filter_id, t, i, purpose, sub, n, lib=None):
    lib = lib or load()
    o = np.zeros(n)
    lib.ora_normals(seed, filter_id, t, i, purpose, sub, n, _ptr(o))
    return o


def normals_many(seed, filter_id, t, idx, purpose, sub, n, lib=None):
    """Row q: the n normals of (t, idx[q], purpose, sub[q])."""
    lib = lib or load()
    idx = np.ascontiguousarray(idx, dtype=np.uint32)
    sub = np.ascontiguousarray(np.broadcast_to(np.asarray(sub, dtype=np.uint32), idx.shape))
    o = np.zeros((len(idx), n))
    lib.ora_normals_many(seed, filter_id, t, len(idx), _ptr(idx), purpose, _ptr(sub), n, _ptr(o))
    return o


def sys_global(W, u, lib=None):
    lib = lib or load()
    W = _f64(W)
    out = np.zeros(len(W), np.int32)
    st = lib.ora_sys_global(_ptr(W), len(W), int(u), _ptr(out))
    if st:
        raise RuntimeError(f"sys_global status {st}")
    return out


def sys_local(W, n_out, u, lib=None):
    lib = lib or load()
    W = _f64(W)
    out = np.zeros(n_out, np.int32)
    st = lib.ora_sys_local(_ptr(W), len(W), int(n_out), int(u), _ptr(out))
    if st:
        raise RuntimeError(f"sys_local status {st}")
    return out
