"""FP64 CPU oracle of the reduced polyatomic ES-BGK lattice-Boltzmann step.

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package. The CUDA library in
``paper_2201_05280_gb300`` never imports it and shares no code with it.

The arithmetic lives in ``rpk_oracle.c`` (plain C, double precision, single
thread, written in the order of the paper's Sec. 5); this module builds it with
gcc, loads it with ctypes and marshals numpy arrays. ``params`` holds the
host-side parameter mapping of Sec. 4 written out independently of the
library's own.

Functions whose result has no independent pin are marked "parity unpinned" in
their docstring; at present there are none: every C entry point is pinned by a
``-m "not gpu"`` test (see ``tests/test_oracle_*.py``).
"""
import ctypes
import os
import subprocess

import numpy as np

from . import params  # noqa: F401  (re-exported)

Q = 41
_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rpk_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle.so")


def build(force=False):
    """Compile the oracle with gcc (IEEE double, no FMA contraction, so that
    x86-64 and aarch64 hosts give the same bits)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Params(ctypes.Structure):
    """Mirror of ``ora_params`` in rpk_oracle.c."""
    _fields_ = [("delta", ctypes.c_double), ("tau", ctypes.c_double),
                ("tau1", ctypes.c_double), ("b", ctypes.c_double),
                ("kr", ctypes.c_double), ("dt", ctypes.c_double),
                ("nsub", ctypes.c_int), ("bcx", ctypes.c_int), ("diff", ctypes.c_int),
                ("rot_mode", ctypes.c_int), ("bcy", ctypes.c_int),
                ("wall", ctypes.c_double * 8), ("xwall", ctypes.c_double * 8)]

    def __repr__(self):
        return ("Params(delta=%g, tau=%g, tau1=%g, b=%g, kr=%g, dt=%g, nsub=%d, bcx=%d, diff=%d, "
                "rot_mode=%d, bcy=%d, wall=%s)" % (self.delta, self.tau, self.tau1, self.b, self.kr,
                                                   self.dt, self.nsub, self.bcx, self.diff,
                                                   self.rot_mode, self.bcy, list(self.wall)))


_lib = None
_dp = ctypes.POINTER(ctypes.c_double)


def _configure(lib):
    P = ctypes.POINTER(Params)
    i, l, d = ctypes.c_int, ctypes.c_long, ctypes.c_double
    sig = {
        "ora_theta0": (d, []),
        "ora_lattice": (None, [_dp, _dp]),
        "ora_target": (None, [d, _dp, _dp, _dp]),
        "ora_point_init": (None, [P, d, _dp, d, d, _dp, _dp]),
        "ora_point_moments": (None, [P, _dp, d, _dp]),
        "ora_point_collide": (None, [P, _dp, _dp]),
        "ora_point_f": (None, [P, _dp, d, _dp]),
        "ora_init": (i, [P, i, i, i, _dp, _dp, _dp, _dp, _dp, _dp]),
        "ora_step": (i, [P, i, i, i, _dp, _dp, _dp, _dp, l]),
        "ora_diffuse_be_line": (i, [i, d, d, _dp, _dp, _dp, d, d, d, d]),
        "ora_fields": (None, [P, i, i, i, _dp, _dp, _dp, _dp, _dp, _dp, _dp]),
        "ora_diag": (None, [P, i, i, i, _dp, _dp, _dp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


def _load():
    global _lib
    if _lib is None:
        _lib = _configure(ctypes.CDLL(build()))
    return _lib


class using_library:
    """Context manager that routes every oracle call to another build of the
    oracle source (used by the mutation tests to plant mistakes on the CPU)."""

    def __init__(self, path):
        self.path = path

    def __enter__(self):
        global _lib
        self.saved = _load()
        _lib = _configure(ctypes.CDLL(self.path))
        return self

    def __exit__(self, *exc):
        global _lib
        _lib = self.saved


def compile_variant(source_text, out_path):
    """Compile a modified copy of the oracle source with the same flags."""
    src = out_path + ".c"
    with open(src, "w") as f:
        f.write(source_text)
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math",
                           "-fPIC", "-shared", "-o", out_path, src, "-lm"])
    return out_path


def source():
    with open(_SRC) as f:
        return f.read()


def _ptr(a):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_dp)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def theta0():
    """Sec. 5, Table 1: lattice reference temperature."""
    return _load().ora_theta0()


THETA0 = 0.2948964908710633  # Sec. 5, Table 1 caption


def lattice():
    """(c, w): the 41 RD3Q41 velocities (41x3) and weights (Sec. 5, Table 1)."""
    c = np.zeros((Q, 3))
    w = np.zeros(Q)
    _load().ora_lattice(_ptr(c), _ptr(w))
    return c, w


def target(rho, u, Lam):
    """Discrete Gaussian f_i(rho, u, Lam), third-order Hermite expansion."""
    f = np.zeros(Q)
    _load().ora_target(float(rho), _ptr(_f64(u)), _ptr(_f64(np.asarray(Lam).reshape(9))), _ptr(f))
    return f


def make_params(delta, tau, tau1, b=0.0, kr=0.0, dt=1.0, nsub=1, bcx=0, diff=0, rot_mode=0,
                walls=None, xwalls=None):
    """diff = 0: FTCS sub-steps of the rotational diffusion (Sec. 5); 1: one
    backward-Euler step per sublattice line (variant for quasi-1-D tubes).
    rot_mode = 0: conservative form on the auxiliary energy Er; 1: the paper's
    four-step theta_R solver (Sec. 5), the state then holds theta_R.
    walls: None (periodic in y) or 8 numbers, ux, uy, uz, theta of the low-y
    and then of the high-y diffuse wall (uy must be 0). xwalls: the same for
    diffuse walls normal to x (ux must be 0; sets bcx = 2)."""
    P = Params(float(delta), float(tau), float(tau1), float(b), float(kr), float(dt),
               int(nsub), int(bcx), int(diff), int(rot_mode), 0)
    if walls is not None:
        w = np.asarray(walls, dtype=np.float64).reshape(8)
        P.bcy = 1
        for k in range(8):
            P.wall[k] = float(w[k])
    if xwalls is not None:
        w = np.asarray(xwalls, dtype=np.float64).reshape(8)
        P.bcx = 2
        for k in range(8):
            P.xwall[k] = float(w[k])
    return P


def diffuse_be_line(delta, dt, rho, kap, Er, thl, kl, thr, kr):
    """The backward-Euler diffusion stage on one line (ora_diffuse_be_line);
    returns the new Er."""
    Er = _f64(Er).copy()
    rc = _load().ora_diffuse_be_line(len(Er), float(delta), float(dt), _ptr(_f64(rho)),
                                     _ptr(_f64(kap)), _ptr(Er), float(thl), float(kl),
                                     float(thr), float(kr))
    if rc:
        raise MemoryError("ora_diffuse_be_line")
    return Er


def point_init(P, rho, u, T, R):
    g = np.zeros(Q)
    Er = ctypes.c_double(0.0)
    _load().ora_point_init(ctypes.byref(P), float(rho), _ptr(_f64(u)), float(T), float(R),
                           _ptr(g), ctypes.cast(ctypes.byref(Er), _dp))
    return g, Er.value


def point_moments(P, g, Er):
    """dict of rho, u, T, R, theta, thetaTg, sigma (3x3) of the f-level state."""
    out = np.zeros(17)
    _load().ora_point_moments(ctypes.byref(P), _ptr(_f64(g)), float(Er), _ptr(out))
    return {"rho": out[0], "u": out[1:4].copy(), "T": out[4], "R": out[5],
            "theta": out[6], "thetaTg": out[7], "sigma": out[8:17].reshape(3, 3).copy()}


def point_collide(P, g, Er):
    g = _f64(g).copy()
    e = ctypes.c_double(float(Er))
    _load().ora_point_collide(ctypes.byref(P), _ptr(g), ctypes.cast(ctypes.byref(e), _dp))
    return g, e.value


def point_f(P, g, Er):
    f = np.zeros(Q)
    _load().ora_point_f(ctypes.byref(P), _ptr(_f64(g)), float(Er), _ptr(f))
    return f


class State:
    """Grid state of the oracle: g (npts x 41, point-major) and Er (npts)."""

    def __init__(self, P, nx, ny, nz, reservoirs=None):
        self.P = P
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.npts = 2 * self.nx * self.ny * self.nz
        self.g = np.zeros((self.npts, Q))
        self.Er = np.zeros(self.npts)
        self.uprev = np.zeros(3 * self.npts)  # u of the previous step (advection)
        self.res = None if reservoirs is None else _f64(reservoirs).reshape(12).copy()
        self.t = 0

    def init_fields(self, rho, u, T, R):
        n = self.npts
        rho, T, R = _f64(rho).reshape(n), _f64(T).reshape(n), _f64(R).reshape(n)
        u = _f64(u).reshape(3 * n)
        _load().ora_init(ctypes.byref(self.P), self.nx, self.ny, self.nz, _ptr(rho), _ptr(u),
                         _ptr(T), _ptr(R), _ptr(self.g), _ptr(self.Er))
        self.uprev[:] = u  # the first step advects with u(0)
        self.t = 0
        return self

    def step(self, n=1):
        res = self.res if self.res is not None else np.zeros(12)
        if self.P.bcx == 1 and self.res is None:
            raise ValueError("bcx=1 needs reservoir states")
        rc = _load().ora_step(ctypes.byref(self.P), self.nx, self.ny, self.nz, _ptr(res),
                              _ptr(self.g), _ptr(self.Er), _ptr(self.uprev), int(n))
        if rc == 2:
            raise ValueError("unsupported setting: the backward-Euler diffusion variant needs "
                             "ny = nz = 1, bcx = 1 and the conservative rotational form; walls "
                             "need at least 2 cells across, zero normal wall velocity, no x "
                             "reservoirs and no backward-Euler variant")
        if rc != 0:
            raise MemoryError("oracle step could not allocate its work arrays")
        self.t += int(n)
        return self

    def fields(self):
        """dict rho, u (3 x npts), T, R, Erot (each npts)."""
        n = self.npts
        rho, T, R, E = (np.zeros(n) for _ in range(4))
        u = np.zeros(3 * n)
        _load().ora_fields(ctypes.byref(self.P), self.nx, self.ny, self.nz, _ptr(self.g),
                           _ptr(self.Er), _ptr(rho), _ptr(u), _ptr(T), _ptr(R), _ptr(E))
        return {"rho": rho, "u": u.reshape(3, n), "T": T, "R": R, "Erot": E}

    def diag(self):
        """dict M, J (3), E, H1, min_g."""
        out = np.zeros(7)
        _load().ora_diag(ctypes.byref(self.P), self.nx, self.ny, self.nz, _ptr(self.g),
                         _ptr(self.Er), _ptr(out))
        return {"M": out[0], "J": out[1:4].copy(), "E": out[4], "H1": out[5], "min_g": out[6]}
