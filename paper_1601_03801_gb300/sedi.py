"""Thin ctypes binding of libsedi.so (include/sedi.h).

Argument marshalling only: every step of the hot path runs in the library's
CUDA kernels.  numpy arrays are passed as host memory, CUDA torch tensors as
device memory (the C ABI's `mem` flag).  There is no CPU fallback: if the
library is missing or no GPU is present the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsedi.so")

_D, _I, _L, _P = C.c_double, C.c_int32, C.c_int64, C.c_void_p

SEDI_FORM_SPLIT, SEDI_FORM_PLAIN_FP32, SEDI_FORM_FP64 = 0, 1, 2
FORMS = {"split": SEDI_FORM_SPLIT, "plain": SEDI_FORM_PLAIN_FP32, "fp64": SEDI_FORM_FP64}
MEM_HOST, MEM_DEVICE = 0, 1

ERRORS = {
    -1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "EOVERFLOW", -5: "ERANGE", -6: "EDIVERGED",
    -7: "ENONFINITE", -8: "ETIMEOUT", -9: "ESTATE", -10: "EIO",
}

# every entry point declared in include/sedi.h
EXPORTS = [
    "sedi_default_params", "sedi_create", "sedi_destroy", "sedi_set_stream", "sedi_set_particles",
    "sedi_set_fluid", "sedi_set_eps", "sedi_step", "sedi_average", "sedi_deposit", "sedi_smooth",
    "sedi_get_particles", "sedi_compute_forces", "sedi_get_neighbors", "sedi_get_contacts",
    "sedi_save_state", "sedi_load_state", "sedi_get_timings", "sedi_get_stats", "sedi_sync",
    "sedi_last_error", "sedi_smooth_static", "sedi_cnn_set_params", "sedi_cnn_get_params",
    "sedi_cnn_forward", "sedi_cnn_loss_grad", "sedi_cnn_train", "sedi_set_bed",
    "sedi_set_contacts", "sedi_set_accel", "sedi_get_wall_springs", "sedi_set_wall_springs",
    "sedi_average_deposit",
]
ALL_BEDS = -1  # SEDI_ALL_BEDS


class SediParams(C.Structure):
    _fields_ = [
        ("contact_law", _I),
        ("E", _D), ("poisson", _D), ("restitution", _D), ("friction", _D),
        ("kn_linear", _D), ("kt_ratio", _D),
        ("rho_f", _D), ("nu_f", _D), ("g", _D * 3),
        ("lo", _D * 3), ("hi", _D * 3),
        ("periodic", _I * 3), ("wall_lo", _I * 3), ("wall_hi", _I * 3),
        ("dt", _D), ("skin", _D),
        ("lubrication", _I), ("drag", _I), ("pressure_grad", _I), ("added_mass", _I),
        ("lift", _I), ("lub_tangential", _I),
        ("lub_h_in_frac", _D), ("lub_h_out_frac", _D), ("c_add", _D), ("c_lift", _D), ("eps_max", _D),
        ("ncell", _I * 3), ("z_grading", _D),
        ("bandwidth", _D * 3), ("n_tau", _I), ("tau_scheme", _I), ("cg_rtol", _D), ("cg_max_iter", _I),
        ("shift_eps", _I), ("shift_mom", _I), ("shift_force", _I),
        ("precision_form", _I), ("nbr_capacity", _I), ("use_graphs", _I), ("substep_variant", _I),
        ("n_beds", _I), ("profile", _I), ("use_cnn_guess", _I), ("ens_persistent", _I),
        ("bin_order", _I), ("bins_per_cutoff", _I), ("cnn_scale", _D * 4),
        ("seed", C.c_uint64),
    ]


class SediStats(C.Structure):
    _fields_ = [("substeps", _L), ("rebuilds", _L), ("averages", _L), ("cg_iterations", _L),
                ("max_neighbors", _I), ("nbr_capacity", _I), ("substep_variant", _I),
                ("substep_block", _I), ("bins_per_cutoff", _I), ("bin_order", _I)]


class SediError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


_lib = None


def lib():
    """Load libsedi.so (built in-tree by __graft_entry__.build())."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
        L = C.CDLL(LIB_PATH)
        sig = {
            "sedi_default_params": (None, [C.POINTER(SediParams)]),
            "sedi_create": (C.c_int, [C.POINTER(SediParams), C.POINTER(_P)]),
            "sedi_destroy": (None, [_P]),
            "sedi_set_stream": (C.c_int, [_P, _P]),
            "sedi_set_particles": (C.c_int, [_P, _I, _L, _P, _P, _P, _P, _P, _P, _I]),
            "sedi_set_fluid": (C.c_int, [_P, _I, _P, _P, _P, _P, _I]),
            "sedi_set_eps": (C.c_int, [_P, _I, _P, _I]),
            "sedi_step": (C.c_int, [_P, _I]),
            "sedi_average": (C.c_int, [_P, _I, _P, _P, _P, _I]),
            "sedi_deposit": (C.c_int, [_P, _I, _P, _I]),
            "sedi_smooth": (C.c_int, [_P, _I, _I, _P, _P, _P, _P, _I]),
            "sedi_get_particles": (C.c_int, [_P, _I, _P, _P, _P, _P, _I]),
            "sedi_compute_forces": (C.c_int, [_P, _I, _P, _P, _P, _P, _I]),
            "sedi_get_neighbors": (_L, [_P, _I, _P, _P, _L]),
            "sedi_get_contacts": (_L, [_P, _I, _L, _P, _P]),
            "sedi_save_state": (C.c_int, [_P, C.c_char_p]),
            "sedi_load_state": (C.c_int, [_P, C.c_char_p]),
            "sedi_get_timings": (C.c_int, [_P, _P, _I]),
            "sedi_get_stats": (C.c_int, [_P, C.POINTER(SediStats)]),
            "sedi_sync": (C.c_int, [_P]),
            "sedi_last_error": (C.c_char_p, [_P]),
            "sedi_smooth_static": (C.c_int, [C.POINTER(SediParams), _I, _P, _P, _P, _P, C.c_char_p, _I]),
            "sedi_set_contacts": (C.c_int, [_P, _I, _L, _P, _P, _I]),
            "sedi_set_accel": (C.c_int, [_P, _I, _P, _I]),
            "sedi_get_wall_springs": (C.c_int, [_P, _I, _P, _I]),
            "sedi_set_wall_springs": (C.c_int, [_P, _I, _P, _I]),
            "sedi_average_deposit": (C.c_int, [_P, _I, _P, _P, _P, _P, _I]),
            "sedi_cnn_set_params": (C.c_int, [_P, _P, _L]),
            "sedi_cnn_get_params": (C.c_int, [_P, _P, _L]),
            "sedi_cnn_forward": (C.c_int, [_P, _P, _P, _I]),
            "sedi_cnn_loss_grad": (C.c_int, [_P, _P, _P, _P, _P, _I]),
            "sedi_cnn_train": (C.c_int, [_P, _I, _P, _P, _I, _D, _P, _I]),
            "sedi_set_bed": (C.c_int, [_P, _I, _P, _P, _P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def default_params() -> dict:
    p = SediParams()
    lib().sedi_default_params(C.byref(p))
    return {name: (list(getattr(p, name)) if hasattr(t, "_length_") else getattr(p, name))
            for name, t in SediParams._fields_}


def make_params(prm: dict) -> SediParams:
    """sedi_params from the library defaults overridden by the keys of prm that it
    knows (unknown keys are ignored so one dict can feed several consumers)."""
    p = SediParams()
    lib().sedi_default_params(C.byref(p))
    fields = dict(SediParams._fields_)
    for k, v in prm.items():
        if k == "precision_form" and isinstance(v, str):
            v = FORMS[v]
        if k not in fields:
            continue
        t = fields[k]
        setattr(p, k, t(*v) if hasattr(t, "_length_") else v)
    return p


STATIC_MAX_WORDS = 1 << 20  # SEDI_STATIC_MAX_WORDS of include/sedi.h


def smooth_static(params: dict, phi, out, stream=None):
    """sedi_smooth_static: smoothing with the library's static scratch (no device
    allocation).  phi and out are CUDA tensors [n_fields, C] of float64."""
    import torch
    p = make_params(params)
    cells = int(np.prod([p.ncell[0], p.ncell[1], p.ncell[2]]))
    for name, t in (("phi", phi), ("out", out)):
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise ValueError(f"smooth_static: {name} must be a CUDA tensor")
        if t.dtype != torch.float64 or not t.is_contiguous():
            raise ValueError(f"smooth_static: {name} must be contiguous float64")
    if phi.dim() != 2 or not 1 <= phi.shape[0] <= 8 or phi.shape[1] != cells:
        raise ValueError(f"smooth_static: phi must be [n_fields <= 8, {cells}], got {tuple(phi.shape)}")
    if tuple(out.shape) != tuple(phi.shape) or out.device != phi.device:
        raise ValueError("smooth_static: out must match phi's shape and device")
    nf = int(phi.shape[0])
    iters = np.zeros(nf, dtype=np.int32)
    msg = C.create_string_buffer(256)
    sptr = 0 if stream is None else (stream if isinstance(stream, int) else stream.cuda_stream)
    rc = lib().sedi_smooth_static(C.byref(p), nf, phi.data_ptr(), out.data_ptr(), iters.ctypes.data,
                                  sptr, msg, 256)
    if rc:
        raise SediError(rc, msg.value.decode())
    return iters


def _is_torch(a):
    return type(a).__module__.startswith("torch")


class _Arg:
    """Pointer + mem flag for a numpy array or a CUDA torch tensor."""

    def __init__(self, a, dtype, shape=None, writable=False):
        self.keep = None
        if a is None:
            self.ptr, self.mem = None, None
            return
        if _is_torch(a):
            import torch
            tdt = {np.float64: torch.float64, np.int64: torch.int64, np.int32: torch.int32}[dtype]
            if a.dtype != tdt or not a.is_contiguous():
                if writable:
                    raise ValueError("output tensors must be contiguous and of the right dtype")
                a = a.to(tdt).contiguous()
            if shape is not None and a.numel() != int(np.prod(shape)):
                raise ValueError(f"expected {shape} elements, got {tuple(a.shape)}")
            self.keep = a
            self.ptr = a.data_ptr()
            self.mem = MEM_DEVICE if a.is_cuda else MEM_HOST
        else:
            if writable:
                if a.dtype != dtype or not a.flags.c_contiguous:
                    raise ValueError("output arrays must be C-contiguous and of the right dtype")
            else:
                a = np.ascontiguousarray(a, dtype=dtype)
            if shape is not None and a.size != int(np.prod(shape)):
                raise ValueError(f"expected {shape} elements, got {a.shape}")
            self.keep = a
            self.ptr = a.ctypes.data
            self.mem = MEM_HOST


def _mem(*args):
    mems = {a.mem for a in args if a.mem is not None}
    if len(mems) > 1:
        raise ValueError("mix of host arrays and device tensors in one call")
    return mems.pop() if mems else MEM_HOST


class Sedi:
    """One handle of the library (see include/sedi.h for the semantics).  With
    params["n_beds"] > 1 it is an ensemble: the per-bed methods take `bed`."""

    def __init__(self, params: dict, stream=None):
        self._p = make_params(params)
        h = _P()
        rc = lib().sedi_create(C.byref(self._p), C.byref(h))
        if rc:
            raise SediError(rc, "sedi_create rejected the parameters")
        self.h = h
        self.n_beds = int(self._p.n_beds)
        c0 = int(np.prod(list(self._p.ncell)))
        self._C = {b: c0 for b in range(self.n_beds)}
        self._nc = {b: tuple(self._p.ncell) for b in range(self.n_beds)}
        self._n = {b: 0 for b in range(self.n_beds)}
        if stream is not None:
            self.set_stream(stream)

    # bed 0 (single-bed handles)
    @property
    def n(self):
        return self._n[0]

    @n.setter
    def n(self, value):  # after load_state, which restores a particle count the binding cannot see
        self._n[0] = int(value)

    @property
    def C(self):
        return self._C[0]

    def close(self):
        if getattr(self, "h", None):
            lib().sedi_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc < 0:
            raise SediError(rc, lib().sedi_last_error(self.h).decode())
        return rc

    def set_stream(self, stream):
        ptr = stream if isinstance(stream, int) else stream.cuda_stream
        self._check(lib().sedi_set_stream(self.h, ptr))

    def set_bed(self, bed, lo, hi, ncell):
        """Box and mesh of ensemble bed `bed` (resets its particles)."""
        lo_a = (C.c_double * 3)(*lo); hi_a = (C.c_double * 3)(*hi)
        nc = (C.c_int32 * 3)(*[int(v) for v in ncell])
        self._check(lib().sedi_set_bed(self.h, int(bed), lo_a, hi_a, nc))
        self._C[bed] = int(np.prod(ncell))
        self._nc[bed] = tuple(int(v) for v in ncell)
        self._n[bed] = 0

    def set_particles(self, x, v=None, w=None, d=None, rho=None, ids=None, bed=0):
        n = (x.shape[0] if hasattr(x, "shape") else len(x))
        ax = _Arg(x, np.float64, (n, 3)); av = _Arg(v, np.float64, (n, 3))
        aw = _Arg(w, np.float64, (n, 3)); ad = _Arg(d, np.float64, (n,))
        ar = _Arg(rho, np.float64, (n,)); ai = _Arg(ids, np.int64, (n,))
        mem = _mem(ax, av, aw, ad, ar, ai)
        self._check(lib().sedi_set_particles(self.h, int(bed), n, ai.ptr, ax.ptr, av.ptr, aw.ptr,
                                             ad.ptr, ar.ptr, mem))
        self._n[bed] = n

    def set_fluid(self, U=None, grad_p=None, DUDt=None, bed=0):
        Cb = self._C[bed]
        nc = (C.c_int32 * 3)(*self._nc[bed])
        au = _Arg(U, np.float64, (Cb, 3)); ag = _Arg(grad_p, np.float64, (Cb, 3))
        ad = _Arg(DUDt, np.float64, (Cb, 3))
        self._check(lib().sedi_set_fluid(self.h, int(bed), nc, au.ptr, ag.ptr, ad.ptr, _mem(au, ag, ad)))

    def set_eps(self, eps, bed=0):
        a = _Arg(eps, np.float64, (self._C[bed],))
        self._check(lib().sedi_set_eps(self.h, int(bed), a.ptr, a.mem))

    def step(self, n_substeps=1):
        self._check(lib().sedi_step(self.h, int(n_substeps)))

    def sync(self):
        self._check(lib().sedi_sync(self.h))

    def average(self, eps=None, Us=None, F=None, bed=0):
        """Into given outputs (numpy or CUDA tensors), else new numpy arrays."""
        Cb = self._C[bed]
        if eps is None and Us is None and F is None:
            eps = np.zeros(Cb); Us = np.zeros((Cb, 3)); F = np.zeros((Cb, 3))
        a = [_Arg(o, np.float64, s, writable=True) for o, s in
             ((eps, (Cb,)), (Us, (Cb, 3)), (F, (Cb, 3)))]
        self._check(lib().sedi_average(self.h, int(bed), a[0].ptr, a[1].ptr, a[2].ptr, _mem(*a)))
        return eps, Us, F

    def average_inplace(self):
        """Averaging whose only output is the drag's solid fraction on the device
        (every bed of an ensemble)."""
        bed = ALL_BEDS if self.n_beds > 1 else 0
        self._check(lib().sedi_average(self.h, bed, None, None, None, MEM_HOST))

    def deposit(self, bed=0):
        q = np.zeros((7, self._C[bed]), dtype=np.int64)
        self._check(lib().sedi_deposit(self.h, int(bed), q.ctypes.data, MEM_HOST))
        return q

    def smooth(self, phi, guess=None, bed=0):
        Cb = self._C[bed]
        phi = np.ascontiguousarray(phi, dtype=np.float64).reshape(-1, Cb)
        nf = phi.shape[0]
        out = np.zeros_like(phi)
        g = None if guess is None else np.ascontiguousarray(guess, dtype=np.float64).reshape(nf, Cb)
        iters = np.zeros(nf, dtype=np.int32)
        self._check(lib().sedi_smooth(self.h, int(bed), nf, phi.ctypes.data, out.ctypes.data,
                                      None if g is None else g.ctypes.data, iters.ctypes.data,
                                      MEM_HOST))
        return out, iters

    def get_particles(self, bed=0):
        n = self._n[bed]
        x, v, w, a = (np.zeros((n, 3)) for _ in range(4))
        self._check(lib().sedi_get_particles(self.h, int(bed), x.ctypes.data, v.ctypes.data,
                                             w.ctypes.data, a.ctypes.data, MEM_HOST))
        return x, v, w, a

    def get_positions(self, out, bed=0):
        a = _Arg(out, np.float64, (self._n[bed], 3), writable=True)
        self._check(lib().sedi_get_particles(self.h, int(bed), a.ptr, None, None, None, a.mem))
        return out

    def compute_forces(self, bed=0):
        n = self._n[bed]
        out = {k: np.zeros((n, 3)) for k in ("contact", "lub", "fluid", "torque")}
        self._check(lib().sedi_compute_forces(self.h, int(bed), out["contact"].ctypes.data,
                                              out["lub"].ctypes.data, out["fluid"].ctypes.data,
                                              out["torque"].ctypes.data, MEM_HOST))
        return out

    def neighbors(self, bed=0):
        off = np.zeros(self._n[bed] + 1, dtype=np.int64)
        tot = self._check(lib().sedi_get_neighbors(self.h, int(bed), off.ctypes.data, None, 0))
        ids = np.zeros(max(tot, 1), dtype=np.int64)
        tot = self._check(lib().sedi_get_neighbors(self.h, int(bed), off.ctypes.data, ids.ctypes.data, tot))
        return off, ids[:tot]

    def contacts(self, bed=0):
        cap = max(16, 8 * self._n[bed])
        while True:
            ij = np.zeros((cap, 2), dtype=np.int64); xi = np.zeros((cap, 3))
            rc = lib().sedi_get_contacts(self.h, int(bed), cap, ij.ctypes.data, xi.ctypes.data)
            if rc == -4:
                cap *= 4
                continue
            m = self._check(rc)
            return ij[:m], xi[:m]

    def set_contacts(self, ij, xi, bed=0):
        """Springs of the given pairs (caller indices i < j, xi as seen from i)."""
        ij = np.ascontiguousarray(ij, dtype=np.int64).reshape(-1, 2)
        xi = np.ascontiguousarray(xi, dtype=np.float64).reshape(-1, 3)
        if len(ij) != len(xi):
            raise ValueError("ij and xi differ in length")
        self._check(lib().sedi_set_contacts(self.h, int(bed), len(ij), ij.ctypes.data if len(ij) else None,
                                            xi.ctypes.data if len(xi) else None, MEM_HOST))

    def set_accel(self, a, bed=0):
        a = _Arg(a, np.float64, (self._n[bed], 3))
        self._check(lib().sedi_set_accel(self.h, int(bed), a.ptr, a.mem))

    def wall_springs(self, bed=0):
        out = np.zeros((self._n[bed], 6, 3))
        self._check(lib().sedi_get_wall_springs(self.h, int(bed), out.ctypes.data, MEM_HOST))
        return out

    def set_wall_springs(self, xw, bed=0):
        a = _Arg(xw, np.float64, (self._n[bed], 6, 3))
        self._check(lib().sedi_set_wall_springs(self.h, int(bed), a.ptr, a.mem))

    def average_deposit(self, q, bed=0):
        """sedi_average_deposit: the averaging from a given deposition [7][C] (int64)."""
        Cb = self._C[bed]
        q = np.ascontiguousarray(q, dtype=np.int64).reshape(7, Cb)
        eps = np.zeros(Cb); Us = np.zeros((Cb, 3)); F = np.zeros((Cb, 3))
        self._check(lib().sedi_average_deposit(self.h, int(bed), q.ctypes.data, eps.ctypes.data,
                                               Us.ctypes.data, F.ctypes.data, MEM_HOST))
        return eps, Us, F

    def save_state(self, path):
        self._check(lib().sedi_save_state(self.h, str(path).encode()))

    def load_state(self, path):
        self._check(lib().sedi_load_state(self.h, str(path).encode()))

    # ---- learned warm start
    CNN_PARAMS = 34628  # SEDI_CNN_PARAMS

    def cnn_set_params(self, params):
        p = np.ascontiguousarray(params, dtype=np.float64)
        self._check(lib().sedi_cnn_set_params(self.h, p.ctypes.data, p.size))

    def cnn_get_params(self):
        p = np.zeros(self.CNN_PARAMS)
        self._check(lib().sedi_cnn_get_params(self.h, p.ctypes.data, p.size))
        return p

    def cnn_forward(self, x):
        x = np.ascontiguousarray(x, dtype=np.float64).reshape(4, self.C)
        y = np.zeros_like(x)
        self._check(lib().sedi_cnn_forward(self.h, x.ctypes.data, y.ctypes.data, MEM_HOST))
        return y

    def cnn_loss_grad(self, x, target):
        x = np.ascontiguousarray(x, dtype=np.float64).reshape(4, self.C)
        t = np.ascontiguousarray(target, dtype=np.float64).reshape(4, self.C)
        g = np.zeros(self.CNN_PARAMS)
        loss = C.c_double()
        self._check(lib().sedi_cnn_loss_grad(self.h, x.ctypes.data, t.ctypes.data, g.ctypes.data,
                                             C.byref(loss), MEM_HOST))
        return loss.value, g

    def cnn_train(self, x, target, steps, lr=1e-3):
        x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 4, self.C)
        t = np.ascontiguousarray(target, dtype=np.float64).reshape(-1, 4, self.C)
        losses = np.zeros(steps)
        self._check(lib().sedi_cnn_train(self.h, x.shape[0], x.ctypes.data, t.ctypes.data, int(steps),
                                         float(lr), losses.ctypes.data, MEM_HOST))
        return losses

    def timings(self) -> dict:
        ms = (C.c_double * 8)()
        n = self._check(lib().sedi_get_timings(self.h, ms, 8))
        keys = ("rebuild_ms", "substep_ms", "deposit_ms", "smooth_ms",
                "rebuild_n", "substep_n", "deposit_n", "smooth_n")
        return {k: ms[i] for i, k in enumerate(keys[:n])}

    def stats(self) -> dict:
        s = SediStats()
        self._check(lib().sedi_get_stats(self.h, C.byref(s)))
        return {k: getattr(s, k) for k, _ in SediStats._fields_}
