"""ctypes binding of the FP64 CPU oracle (test infrastructure only).

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg import this
module.  It builds oracle/liborc.so on first use.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

_D = C.c_double
_I = C.c_int32
_L = C.c_int64
_P = C.c_void_p


class OrcParams(C.Structure):
    _fields_ = [
        ("E", _D), ("poisson", _D), ("restitution", _D), ("friction", _D),
        ("rho_f", _D), ("nu_f", _D), ("g", _D * 3),
        ("lo", _D * 3), ("hi", _D * 3),
        ("periodic", _I * 3), ("wall_lo", _I * 3), ("wall_hi", _I * 3),
        ("dt", _D),
        ("lubrication", _I), ("drag", _I), ("pressure_grad", _I), ("added_mass", _I),
        ("lub_h_in_frac", _D), ("lub_h_out_frac", _D), ("c_add", _D), ("eps_max", _D),
        ("ncell", _I * 3),
        ("bandwidth", _D * 3), ("n_tau", _I), ("cg_rtol", _D), ("cg_max_iter", _I),
        ("shift_eps", _I), ("shift_mom", _I), ("shift_force", _I),
        ("contact_law", _I), ("kn_linear", _D), ("kt_ratio", _D), ("tau_scheme", _I),
        ("lift", _I), ("c_lift", _D), ("lub_tangential", _I), ("z_grading", _D),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        L.orc_create.restype = _P
        L.orc_create.argtypes = [C.POINTER(OrcParams)]
        L.orc_destroy.argtypes = [_P]
        for name, args in {
            "orc_set_particles": [_P, _L, _P, _P, _P, _P, _P],
            "orc_set_accel": [_P, _P],
            "orc_set_fluid": [_P, _P, _P, _P],
            "orc_set_eps": [_P, _P],
            "orc_step": [_P, _I],
            "orc_set_threads": [_P, _I],
            "orc_set_contacts": [_P, _L, _P, _P],
            "orc_set_wall_history": [_P, _P],
            "orc_average_fixed": [_P, _P, _P, _P, _P],
            "orc_forces": [_P, _P, _P, _P, _P],
            "orc_get_particles": [_P, _P, _P, _P, _P],
            "orc_get_contacts": [_P, _L, _P, _P],
            "orc_get_wall_history": [_P, _P],
            "orc_deposit": [_P, _P],
            "orc_smooth": [_P, _I, _P, _P, _P],
            "orc_average": [_P, _P, _P, _P],
        }.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = C.c_int
        L.orc_num_contacts.argtypes = [_P]
        L.orc_num_contacts.restype = _L
        L.orc_neighbors.argtypes = [_P, _D, _I, _P, _P, _L]
        L.orc_neighbors.restype = _L
        L.orc_drag.argtypes = [C.POINTER(OrcParams), _D, _P, _D, _P, _P, _P]
        L.orc_drag.restype = None
        L.orc_vr.argtypes = [_D, _D]
        L.orc_vr.restype = _D
        L.orc_z_faces.argtypes = [C.POINTER(OrcParams), _P]
        L.orc_z_faces.restype = None
        L.orc_smooth_operator.argtypes = [C.POINTER(OrcParams), _P, _P]
        L.orc_smooth_operator.restype = None
        L.orc_curl.argtypes = [C.POINTER(OrcParams), _P, _P]
        L.orc_curl.restype = None
        L.orc_lift.argtypes = [C.POINTER(OrcParams), _P, _P, _D, _P]
        L.orc_lift.restype = None
        L.orc_lub_pair.argtypes = [C.POINTER(OrcParams), _P, _D, _D, _P, _P, _P, _P, _P, _P, _P]
        L.orc_lub_pair.restype = None
        L.orc_hm_pair.argtypes = [C.POINTER(OrcParams), _P, _D, _D, _D, _D, _P, _P, _P, _P, _P,
                                  _P, _P, _P, _P]
        L.orc_hm_pair.restype = C.c_int
        L.orc_lub_wall.argtypes = [C.POINTER(OrcParams), _P, _D, _D, _P, _P, _P, _P]
        L.orc_lub_wall.restype = None
        L.orc_cnn_num_params.argtypes = []
        L.orc_cnn_num_params.restype = _L
        L.orc_cnn_forward.argtypes = [C.c_int, C.c_int, C.c_int, _P, _P, _P, _P, _P, _P, _I]
        L.orc_cnn_forward.restype = C.c_int
        L.orc_cnn_loss_grad.argtypes = [C.c_int, C.c_int, C.c_int, _P, _P, _P, _P, _P]
        L.orc_cnn_loss_grad.restype = _D
        L.orc_adam.argtypes = [_L, _P, _P, _P, _P, _L, _D, _D, _D, _D]
        L.orc_adam.restype = None
        _lib = L
    return _lib


def make_params(prm: dict) -> OrcParams:
    """Fill the oracle's own parameter struct from a plain dict of physical inputs."""
    p = OrcParams()
    # the contact law defaults to Hertz-Mindlin (the linear law's inputs then unused)
    optional = {"contact_law": 0, "kn_linear": 800.0, "kt_ratio": 2.0 / 7.0, "tau_scheme": 0,
                "lift": 0, "c_lift": 1.6, "lub_tangential": 0, "z_grading": 1.0}
    for name, ctype in OrcParams._fields_:
        if name not in prm and name not in optional:
            raise KeyError(f"oracle parameter {name!r} missing")
        val = prm.get(name, optional.get(name))
        if hasattr(ctype, "_length_"):
            setattr(p, name, ctype(*val))
        else:
            setattr(p, name, val)
    return p


def _ptr(a):
    return None if a is None else a.ctypes.data


def _f64(a, shape=None):
    if a is None:
        return None
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


class Oracle:
    """One oracle instance: particles, fluid fields and contact history."""

    def __init__(self, prm: dict, threads: int = 1):
        self.prm = dict(prm)
        self._p = make_params(prm)
        self.C = int(np.prod(prm["ncell"]))
        self.h = lib().orc_create(C.byref(self._p))
        self.n = 0
        self.set_threads(threads)

    def set_threads(self, threads: int):
        """Threads of the particle loops and of the smoothing (same results for any count)."""
        self.threads = max(1, int(threads))
        lib().orc_set_threads(self.h, self.threads)

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_destroy(self.h)
            self.h = None

    def set_particles(self, x, v, w, d, rho):
        x = _f64(x, (-1, 3)); n = x.shape[0]
        v = _f64(v, (n, 3)); w = _f64(w, (n, 3))
        d = _f64(d, (n,)); rho = _f64(rho, (n,))
        self.n = n
        self._keep = (x, v, w, d, rho)
        assert lib().orc_set_particles(self.h, n, _ptr(x), _ptr(v), _ptr(w), _ptr(d), _ptr(rho)) == 0

    def set_accel(self, a):
        a = _f64(a, (self.n, 3))
        lib().orc_set_accel(self.h, _ptr(a))

    def set_fluid(self, U=None, grad_p=None, DUDt=None):
        U = _f64(U, (self.C, 3)); gp = _f64(grad_p, (self.C, 3)); du = _f64(DUDt, (self.C, 3))
        lib().orc_set_fluid(self.h, _ptr(U), _ptr(gp), _ptr(du))

    def set_eps(self, eps):
        e = _f64(eps, (self.C,))
        lib().orc_set_eps(self.h, _ptr(e))

    def step(self, n_sub=1):
        assert lib().orc_step(self.h, int(n_sub)) == 0

    def forces(self):
        out = {k: np.zeros((self.n, 3)) for k in ("contact", "lub", "fluid", "torque")}
        lib().orc_forces(self.h, _ptr(out["contact"]), _ptr(out["lub"]), _ptr(out["fluid"]),
                         _ptr(out["torque"]))
        return out

    def get_particles(self):
        x, v, w, a = (np.zeros((self.n, 3)) for _ in range(4))
        lib().orc_get_particles(self.h, _ptr(x), _ptr(v), _ptr(w), _ptr(a))
        return x, v, w, a

    def contacts(self):
        m = lib().orc_num_contacts(self.h)
        ij = np.zeros((m, 2), dtype=np.int64); xi = np.zeros((m, 3))
        if m:
            assert lib().orc_get_contacts(self.h, m, _ptr(ij), _ptr(xi)) == 0
        return ij, xi

    def set_contacts(self, ij, xi):
        ij = np.ascontiguousarray(ij, dtype=np.int64).reshape(-1, 2)
        xi = np.ascontiguousarray(xi, dtype=np.float64).reshape(-1, 3)
        assert lib().orc_set_contacts(self.h, len(ij), _ptr(ij), _ptr(xi)) == 0

    def set_wall_history(self, xw):
        xw = _f64(xw, (self.n, 6, 3))
        lib().orc_set_wall_history(self.h, _ptr(xw))

    def average_fixed(self, q):
        q = np.ascontiguousarray(q, dtype=np.int64).reshape(7, self.C)
        eps = np.zeros(self.C); Us = np.zeros((self.C, 3)); F = np.zeros((self.C, 3))
        st = lib().orc_average_fixed(self.h, _ptr(q), _ptr(eps), _ptr(Us), _ptr(F))
        if st:
            raise RuntimeError(f"oracle average failed ({st})")
        return eps, Us, F

    def wall_history(self):
        xw = np.zeros((self.n, 6, 3))
        lib().orc_get_wall_history(self.h, _ptr(xw))
        return xw

    def neighbors(self, skin, brute=True):
        cap = max(64, self.n * 64)
        while True:
            off = np.zeros(self.n + 1, dtype=np.int64); idx = np.zeros(cap, dtype=np.int64)
            tot = lib().orc_neighbors(self.h, float(skin), int(bool(brute)), _ptr(off), _ptr(idx), cap)
            if tot >= 0:
                return off, idx[:tot]
            cap *= 4

    def deposit(self):
        q = np.zeros((7, self.C), dtype=np.int64)
        st = lib().orc_deposit(self.h, _ptr(q))
        if st:
            raise RuntimeError(f"oracle deposit failed ({st})")
        return q

    def smooth(self, phi, guess=None, check=True):
        phi = np.array(phi, dtype=np.float64, copy=True).reshape(-1, self.C)
        nf = phi.shape[0]
        g = _f64(guess, (nf, self.C))
        iters = np.zeros(nf, dtype=np.int32)
        st = lib().orc_smooth(self.h, nf, _ptr(phi), _ptr(g), _ptr(iters))
        if st and check:
            raise RuntimeError(f"oracle smoothing did not converge ({st})")
        return phi, iters

    def average(self):
        eps = np.zeros(self.C); Us = np.zeros((self.C, 3)); F = np.zeros((self.C, 3))
        st = lib().orc_average(self.h, _ptr(eps), _ptr(Us), _ptr(F))
        if st:
            raise RuntimeError(f"oracle average failed ({st})")
        return eps, Us, F


def drag(prm: dict, eps_s, w, d):
    """Single-particle drag of the oracle: (force, V_r, C_d |w|)."""
    p = make_params(prm)
    w = np.ascontiguousarray(w, dtype=np.float64)
    f = np.zeros(3); vr = C.c_double(); cdw = C.c_double()
    lib().orc_drag(C.byref(p), float(eps_s), _ptr(w), float(d), _ptr(f), C.byref(vr), C.byref(cdw))
    return f, vr.value, cdw.value


def vr(eps_f, Re):
    return lib().orc_vr(float(eps_f), float(Re))


def z_faces(prm: dict):
    """Faces of the oracle's z mesh (n_z + 1 values)."""
    p = make_params(prm)
    out = np.zeros(prm["ncell"][2] + 1)
    lib().orc_z_faces(C.byref(p), _ptr(out))
    return out


def smooth_operator(prm: dict, x):
    """y = A x, the operator of one backward-Euler smoothing step, on one field [C]."""
    p = make_params(prm)
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.zeros_like(x)
    lib().orc_smooth_operator(C.byref(p), _ptr(x), _ptr(y))
    return y


def curl(prm: dict, U):
    """Cell-centred vorticity of the oracle from U [C, 3]."""
    p = make_params(prm)
    U = np.ascontiguousarray(U, dtype=np.float64).reshape(-1, 3)
    out = np.zeros_like(U)
    lib().orc_curl(C.byref(p), _ptr(U), _ptr(out))
    return out


def lift(prm: dict, w, omega, d):
    """Single-particle lift of the oracle for slip w = U_f - u_p and vorticity omega."""
    p = make_params(prm)
    w = np.ascontiguousarray(w, dtype=np.float64)
    om = np.ascontiguousarray(omega, dtype=np.float64)
    f = np.zeros(3)
    lib().orc_lift(C.byref(p), _ptr(w), _ptr(om), float(d), _ptr(f))
    return f


def lub_pair(prm: dict, dx, ra, rb, va, vb, wa, wb):
    """Lubrication of the pair (a, b), dx = x_b - x_a: (force on a, torque on a, torque on b)."""
    p = make_params(prm)
    a = [np.ascontiguousarray(v, dtype=np.float64) for v in (dx, va, vb, wa, wb)]
    F, Ta, Tb = np.zeros(3), np.zeros(3), np.zeros(3)
    lib().orc_lub_pair(C.byref(p), _ptr(a[0]), float(ra), float(rb), _ptr(a[1]), _ptr(a[2]),
                       _ptr(a[3]), _ptr(a[4]), _ptr(F), _ptr(Ta), _ptr(Tb))
    return F, Ta, Tb


def hm_pair(prm: dict, dx, ra, rb, ma, mb, va, vb, wa, wb, xi_old):
    """Contact of the pair (a, b), dx = x_b - x_a, with spring xi_old: (active, force on a,
    torque on a, torque on b, updated spring)."""
    p = make_params(prm)
    a = [np.ascontiguousarray(v, dtype=np.float64) for v in (dx, va, vb, wa, wb, xi_old)]
    F, Ta, Tb, xi = np.zeros(3), np.zeros(3), np.zeros(3), np.zeros(3)
    act = lib().orc_hm_pair(C.byref(p), _ptr(a[0]), float(ra), float(rb), float(ma), float(mb),
                            _ptr(a[1]), _ptr(a[2]), _ptr(a[3]), _ptr(a[4]), _ptr(a[5]),
                            _ptr(F), _ptr(Ta), _ptr(Tb), _ptr(xi))
    return bool(act), F, Ta, Tb, xi


def lub_wall(prm: dict, n, dist, r, v, w):
    """Lubrication of a sphere against a wall (n towards the wall): (force, torque)."""
    p = make_params(prm)
    a = [np.ascontiguousarray(x, dtype=np.float64) for x in (n, v, w)]
    F, T = np.zeros(3), np.zeros(3)
    lib().orc_lub_wall(C.byref(p), _ptr(a[0]), float(dist), float(r), _ptr(a[1]), _ptr(a[2]),
                       _ptr(F), _ptr(T))
    return F, T


# ---------------------------------------------------------------- learned warm start
def cnn_num_params():
    return int(lib().orc_cnn_num_params())


def cnn_forward(params, x, ncell, periodic, round_bf16=False, activations=False):
    """x [4, nz, ny, nx] (or [4, C]) -> y of the same shape."""
    nx, ny, nz = ncell
    N = nx * ny * nz
    p = np.ascontiguousarray(params, dtype=np.float64)
    xi = np.ascontiguousarray(x, dtype=np.float64).reshape(4, N)
    y = np.zeros((4, N))
    a1 = np.zeros((32, N)) if activations else None
    a2 = np.zeros((32, N)) if activations else None
    per = np.asarray(periodic, dtype=np.int32)
    lib().orc_cnn_forward(nx, ny, nz, per.ctypes.data, p.ctypes.data, xi.ctypes.data, y.ctypes.data,
                          _ptr(a1), _ptr(a2), int(bool(round_bf16)))
    return (y, a1, a2) if activations else y


def cnn_loss_grad(params, x, target, ncell, periodic):
    nx, ny, nz = ncell
    N = nx * ny * nz
    p = np.ascontiguousarray(params, dtype=np.float64)
    xi = np.ascontiguousarray(x, dtype=np.float64).reshape(4, N)
    ti = np.ascontiguousarray(target, dtype=np.float64).reshape(4, N)
    g = np.zeros_like(p)
    per = np.asarray(periodic, dtype=np.int32)
    loss = lib().orc_cnn_loss_grad(nx, ny, nz, per.ctypes.data, p.ctypes.data, xi.ctypes.data,
                                   ti.ctypes.data, g.ctypes.data)
    return loss, g


def adam(params, grad, m, v, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """In place on float64 numpy arrays."""
    lib().orc_adam(params.size, params.ctypes.data, grad.ctypes.data, m.ctypes.data, v.ctypes.data,
                   int(t), lr, beta1, beta2, eps)
