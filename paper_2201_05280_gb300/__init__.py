"""Python binding of librpk: the GB300 (sm_103a) lattice-Boltzmann step of the
reduced polyatomic ES-BGK model (Kolluru, Atif & Ansumali, arXiv 2201.05280).

This module only marshals arguments to the C interface declared in
``include/rpk.h``; every step of the computation runs in the CUDA kernels of
``librpk.so``. There is no CPU fallback: if the library is missing or cannot
be loaded, ``load_library`` raises.

Arrays: host numpy float64 arrays, or CUDA float64 torch tensors (then the
device path of the C interface is used and nothing crosses PCIe/C2C). A scalar
field has 2*nx*ny*nz entries indexed p = ((s*nz + z)*ny + y)*nx + x; u has
shape (3, npts).
"""
import ctypes
import os

import numpy as np

__all__ = ["Lattice", "RpkError", "load_library", "theta0", "map_gas", "auto_nsub",
           "gas_from_nondim", "sound_speed", "auto_nsub_fields", "tube_reservoirs",
           "field_totals_noalloc", "Batch", "Net", "Rollout", "SurConfig", "SurSeq",
           "sur_pack", "sur_apply", "PRECISIONS", "library_path"]

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "librpk.so")

PRECISIONS = {"f64": 0, "f32": 1, "f16dev": 2, "bf16dev": 3}
_BC = {"periodic": 0, "reservoir": 1}
_STATUS = {0: "OK", 1: "ERR_ARG", 2: "ERR_PARAM", 3: "ERR_CUDA", 4: "ERR_NUMERIC",
           5: "ERR_STATE", 6: "ERR_OOM", 7: "ERR_IO"}


class RpkError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s: %s" % (_STATUS.get(code, code), msg))
        self.code = code


class Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("precision", ctypes.c_int), ("bc_x", ctypes.c_int)]


class Relax(ctypes.Structure):
    _fields_ = [("delta", ctypes.c_double), ("tau", ctypes.c_double),
                ("tau1", ctypes.c_double), ("b", ctypes.c_double), ("k_r", ctypes.c_double),
                ("dt", ctypes.c_double), ("nsub", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Tube(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("nsteps", ctypes.c_int), ("relax", Relax),
                ("res", ctypes.c_double * 12)]


class SurConfig(ctypes.Structure):
    _fields_ = [("jump", ctypes.c_int), ("pad", ctypes.c_int), ("spot_every", ctypes.c_int),
                ("project", ctypes.c_int), ("anchor", ctypes.c_int), ("drift_tol", ctypes.c_double),
                ("l1_tol", ctypes.c_double), ("in_shift", ctypes.c_float * 4),
                ("in_scale", ctypes.c_float * 4), ("out_scale", ctypes.c_float * 4),
                ("in_dscale", ctypes.c_float * 4),
                ("lbm_threads", ctypes.c_int), ("lbm_ctas_per_sm", ctypes.c_int),
                ("lbm_diffusion", ctypes.c_int)]

    @classmethod
    def make(cls, **kw):
        c = cls()
        c.jump, c.pad, c.spot_every, c.project, c.anchor = 32, 128, 8, 1, 1
        c.drift_tol, c.l1_tol = 1e-4, 1e-2
        for k in range(4):
            c.in_scale[k] = c.out_scale[k] = c.in_dscale[k] = 1.0
        for k, v in kw.items():
            if k in ("in_shift", "in_scale", "out_scale", "in_dscale"):
                for i in range(4):
                    getattr(c, k)[i] = float(v[i])
            else:
                setattr(c, k, v)
        return c


class SurSeq(ctypes.Structure):
    _fields_ = [("src", ctypes.c_int64), ("tgt", ctypes.c_int64), ("prev", ctypes.c_int64),
                ("out", ctypes.c_int64),
                ("nx", ctypes.c_int), ("len", ctypes.c_int), ("crop", ctypes.c_int),
                ("pad_", ctypes.c_int), ("res", (ctypes.c_float * 4) * 2),
                ("cond", ctypes.c_float * 2)]


class Diag(ctypes.Structure):
    _fields_ = [("mass", ctypes.c_double), ("mom", ctypes.c_double * 3),
                ("energy", ctypes.c_double), ("H1", ctypes.c_double),
                ("min_g", ctypes.c_double), ("status", ctypes.c_uint32),
                ("pad", ctypes.c_uint32), ("steps", ctypes.c_int64)]


_lib = None
_dp = ctypes.POINTER(ctypes.c_double)


def library_path():
    return _LIB_PATH


def load_library(path=None):
    """Load librpk.so (built by ``build.build()``); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _LIB_PATH
    if not os.path.exists(path):
        raise ImportError("librpk.so not found at %s: build it with "
                          "`python -c 'import __graft_entry__ as g; g.build()'`" % path)
    lib = ctypes.CDLL(path)
    vp, i, d, i64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int64
    sig = {
        "rpk_abi_version": (i, []),
        "rpk_theta0": (d, []),
        "rpk_last_error": (ctypes.c_char_p, []),
        "rpk_map_gas": (i, [d, d, d, d, d, d, ctypes.POINTER(Relax)]),
        "rpk_auto_nsub": (i, [ctypes.POINTER(Relax), d, i]),
        "rpk_gas_from_nondim": (i, [d, d, d, d, d, ctypes.POINTER(d)]),
        "rpk_sound_speed": (d, [d]),
        "rpk_auto_nsub_fields": (i, [ctypes.POINTER(Relax), _dp, _dp, i64, _dp, i]),
        "rpk_sur_reservoirs": (i, [ctypes.POINTER(Tube), ctypes.POINTER(ctypes.c_float)]),
        "rpk_create": (i, [ctypes.POINTER(Grid), vp, ctypes.POINTER(vp)]),
        "rpk_destroy": (None, [vp]),
        "rpk_set_relax": (i, [vp, ctypes.POINTER(Relax)]),
        "rpk_set_gas": (i, [vp, d, d, d, d, d]),
        "rpk_set_reservoirs": (i, [vp, _dp]),
        "rpk_set_rot_mode": (i, [vp, i]),
        "rpk_set_walls": (i, [vp, _dp]),
        "rpk_set_x_walls": (i, [vp, _dp]),
        "rpk_init_fields": (i, [vp, vp, vp, vp, vp, i]),
        "rpk_step": (i, [vp, i64]),
        "rpk_read_moments": (i, [vp, vp, vp, vp, vp, vp, i]),
        "rpk_diagnostics": (i, [vp, ctypes.POINTER(Diag)]),
        "rpk_save": (i, [vp, ctypes.c_char_p]),
        "rpk_load": (i, [vp, ctypes.c_char_p]),
        "rpk_get_info": (i, [vp, ctypes.POINTER(i64)]),
        "rpk_timing": (i, [vp, i]),
        "rpk_timing_read": (i, [vp, ctypes.POINTER(d), ctypes.POINTER(i64)]),
        "rpk_field_totals_noalloc": (i, [vp, vp, vp, vp, i64, d, vp, vp]),
        "rpk_batch_max_nx": (i, [i]),
        "rpk_batch_create": (i, [i, i, ctypes.POINTER(Tube), i, vp, ctypes.POINTER(vp)]),
        "rpk_batch_destroy": (None, [vp]),
        "rpk_batch_init": (i, [vp, vp, vp, vp, vp]),
        "rpk_batch_set_config": (i, [vp, i, i]),
        "rpk_batch_set_diffusion": (i, [vp, i]),
        "rpk_batch_autotune": (i, [vp, ctypes.POINTER(i64)]),
        "rpk_batch_run": (i, [vp]),
        "rpk_batch_read_moments": (i, [vp, vp, vp, vp, vp, vp]),
        "rpk_batch_snapshots": (i, [vp, vp, ctypes.POINTER(i64)]),
        "rpk_batch_init_device": (i, [vp, vp]),
        "rpk_batch_set_steps": (i, [vp, ctypes.POINTER(i)]),
        "rpk_batch_moments_device": (i, [vp, vp]),
        "rpk_sur_pack": (i, [ctypes.POINTER(SurConfig), vp, vp, i, i, i, ctypes.POINTER(ctypes.c_float),
                             ctypes.c_uint64, vp, vp, vp, vp]),
        "rpk_sur_apply": (i, [ctypes.POINTER(SurConfig), vp, vp, vp, i, vp, vp, vp, vp]),
        "rpk_rollout_create": (i, [vp, ctypes.POINTER(SurConfig), i, ctypes.POINTER(Tube),
                                   ctypes.POINTER(ctypes.c_float), vp, ctypes.POINTER(vp)]),
        "rpk_rollout_destroy": (None, [vp]),
        "rpk_rollout_run": (i, [vp, vp, ctypes.POINTER(i64), ctypes.POINTER(d), ctypes.POINTER(d)]),
        "rpk_rollout_errors": (i, [vp, vp, ctypes.POINTER(i)]),
        "rpk_net_create": (i, [i, i, i, i, ctypes.c_uint64, vp, ctypes.POINTER(vp)]),
        "rpk_net_destroy": (None, [vp]),
        "rpk_net_num_params": (i64, [vp]),
        "rpk_net_get_params": (i, [vp, vp, i]),
        "rpk_net_set_params": (i, [vp, vp]),
        "rpk_net_forward": (i, [vp, vp, i, i, vp]),
        "rpk_net_forward_ragged": (i, [vp, vp, i, ctypes.POINTER(i), vp]),
        "rpk_net_loss_grad": (i, [vp, vp, vp, vp, i, i, ctypes.POINTER(d)]),
        "rpk_net_adam": (i, [vp, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if lib.rpk_abi_version() != 1:
        raise ImportError("librpk ABI version mismatch")
    _lib = lib
    return lib


def _check(code):
    if code != 0:
        raise RpkError(code, load_library().rpk_last_error().decode())


def theta0():
    """Lattice reference temperature (Sec. 5, Table 1)."""
    return load_library().rpk_theta0()


def map_gas(gamma, eta, eta_B, kappa, b=0.0, rho0=1.0):
    """(gamma, eta, eta_B, kappa, b) -> raw relaxation parameters (rpk_map_gas)."""
    r = Relax()
    _check(load_library().rpk_map_gas(gamma, eta, eta_B, kappa, b, rho0, ctypes.byref(r)))
    return r.as_dict()


def auto_nsub(relax, theta_max, ndim):
    r = Relax(**{k: relax.get(k, 0) for k, _ in Relax._fields_})
    return load_library().rpk_auto_nsub(ctypes.byref(r), float(theta_max), int(ndim))


def gas_from_nondim(gamma, nu, lam, Pr, rho0=1.0):
    """(eta, eta_B, kappa) from kinematic viscosity nu, eta_B/eta = lam and
    the Prandtl number (rpk_gas_from_nondim)."""
    out = (ctypes.c_double * 3)()
    _check(load_library().rpk_gas_from_nondim(float(gamma), float(nu), float(lam), float(Pr),
                                              float(rho0), out))
    return out[0], out[1], out[2]


def sound_speed(gamma):
    """Adiabatic sound speed of the lattice reference state (rpk_sound_speed)."""
    return load_library().rpk_sound_speed(float(gamma))


def auto_nsub_fields(relax, T, R, res=None, ndim=1):
    """FTCS sub-steps at the hottest of the fields T, R (host arrays) and the
    optional 12 reservoir values (rpk_auto_nsub_fields)."""
    r = Relax(**{k: relax.get(k, 0) for k, _ in Relax._fields_})
    T = np.ascontiguousarray(T, dtype=np.float64).reshape(-1)
    R = np.ascontiguousarray(R, dtype=np.float64).reshape(-1)
    if T.size != R.size:
        raise ValueError("T and R differ in size")
    rs = None if res is None else np.ascontiguousarray(res, dtype=np.float64).reshape(12)
    return load_library().rpk_auto_nsub_fields(
        ctypes.byref(r), T.ctypes.data_as(_dp), R.ctypes.data_as(_dp), T.size,
        None if rs is None else rs.ctypes.data_as(_dp), int(ndim))


def tube_reservoirs(tube):
    """(2, 4) float32 moment-block values (rho, u_x, theta_T, E_R) of a tube
    dict's reservoirs (rpk_sur_reservoirs)."""
    t = _tube_struct(tube)
    out = np.zeros(8, dtype=np.float32)
    _check(load_library().rpk_sur_reservoirs(ctypes.byref(t),
                                             out.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
    return out.reshape(2, 4)


def field_totals_noalloc(rho, u, T, R, delta, out, stream=None):
    """Conserved totals (sum rho, sum rho u (3), E_T + E_R) of CUDA float64
    tensors, written into the CUDA float64 tensor ``out`` (5 values) on
    ``stream``; allocates nothing (rpk_field_totals_noalloc). For callers
    that may not allocate device memory at that point (an application whose
    memory manager owns all device memory, or a loop that must not stall on
    cudaMalloc). Every tensor and the stream must be on the current CUDA
    device. Asynchronous: synchronise the stream before reading ``out``."""
    import torch
    cur = torch.cuda.current_device()
    n = rho.numel()
    ptrs = []
    for name, a, m in (("rho", rho, n), ("u", u, 3 * n), ("T", T, n), ("R", R, n), ("out", out, 5)):
        p, dev, _ = _arg(a, m)
        if dev != 1:
            raise ValueError("field_totals_noalloc takes CUDA tensors only (%s)" % name)
        if a.device.index != cur:
            raise ValueError("%s is on cuda:%d, not on the current device cuda:%d"
                             % (name, a.device.index, cur))
        ptrs.append(p)
    if stream is not None and not isinstance(stream, int) and stream.device.index != cur:
        raise ValueError("the stream is on cuda:%d, not on the current device cuda:%d"
                         % (stream.device.index, cur))
    _check(load_library().rpk_field_totals_noalloc(ptrs[0], ptrs[1], ptrs[2], ptrs[3], n,
                                                   float(delta), _stream_handle(stream),
                                                   ptrs[4]))
    return out


def _tube_struct(d):
    """rpk_tube of a tube dict (nx, nsteps, relax, res)."""
    t = Tube()
    t.nx, t.nsteps = int(d["nx"]), int(d["nsteps"])
    r = d["relax"]
    t.relax = Relax(r["delta"], r["tau"], r["tau1"], r.get("b", 0.0), r.get("k_r", 0.0),
                    r.get("dt", 1.0), int(r.get("nsub", 0)))
    for k in range(12):
        t.res[k] = float(d["res"][k])
    return t


def _is_torch(a):
    return type(a).__module__.startswith("torch")


def _arg(a, n):
    """(pointer, on_device, keepalive) for a float64 array of n values."""
    if _is_torch(a):
        import torch
        if a.dtype != torch.float64 or not a.is_contiguous() or a.numel() != n:
            raise ValueError("expected a contiguous float64 tensor of %d values" % n)
        return ctypes.c_void_p(a.data_ptr()), 1 if a.is_cuda else 0, a
    arr = np.ascontiguousarray(a, dtype=np.float64)
    if arr.size != n:
        raise ValueError("expected %d values, got %d" % (n, arr.size))
    return arr.ctypes.data_as(ctypes.c_void_p), 0, arr


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)  # torch.cuda.Stream


class Lattice:
    """One lattice on the current CUDA device, driven through librpk."""

    def __init__(self, nx, ny, nz, precision="f32", bc_x="periodic", stream=None):
        lib = load_library()
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.npts = 2 * self.nx * self.ny * self.nz
        self.precision = precision
        g = Grid(self.nx, self.ny, self.nz, PRECISIONS[precision], _BC[bc_x])
        h = ctypes.c_void_p()
        _check(lib.rpk_create(ctypes.byref(g), _stream_handle(stream), ctypes.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            load_library().rpk_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_relax(self, delta, tau, tau1, b=0.0, k_r=0.0, nsub=0, dt=1.0):
        r = Relax(delta, tau, tau1, b, k_r, dt, int(nsub))
        _check(load_library().rpk_set_relax(self._h, ctypes.byref(r)))
        return self

    def set_gas(self, gamma, eta, eta_B, kappa, b=0.0):
        _check(load_library().rpk_set_gas(self._h, gamma, eta, eta_B, kappa, b))
        return self

    def set_reservoirs(self, states12):
        s = np.ascontiguousarray(states12, dtype=np.float64).reshape(12)
        _check(load_library().rpk_set_reservoirs(self._h, s.ctypes.data_as(_dp)))
        return self

    def set_walls(self, low=None, high=None):
        """Diffuse walls normal to y at y = -1/4 and y = ny - 1/4 (rpk_set_walls):
        low and high are (ux, uy, uz, theta) of each wall, uy = 0; no arguments
        makes y periodic again."""
        if low is None and high is None:
            _check(load_library().rpk_set_walls(self._h, None))
            return self
        w = np.ascontiguousarray(np.concatenate([np.ravel(low), np.ravel(high)]), dtype=np.float64)
        if w.size != 8:
            raise ValueError("each wall is (ux, uy, uz, theta)")
        _check(load_library().rpk_set_walls(self._h, w.ctypes.data_as(_dp)))
        return self

    def set_x_walls(self, low=None, high=None):
        """Diffuse walls normal to x at x = -1/4 and x = nx - 1/4
        (rpk_set_x_walls): low and high are (ux, uy, uz, theta), ux = 0; no
        arguments makes x periodic again."""
        if low is None and high is None:
            _check(load_library().rpk_set_x_walls(self._h, None))
            return self
        w = np.ascontiguousarray(np.concatenate([np.ravel(low), np.ravel(high)]), dtype=np.float64)
        if w.size != 8:
            raise ValueError("each wall is (ux, uy, uz, theta)")
        _check(load_library().rpk_set_x_walls(self._h, w.ctypes.data_as(_dp)))
        return self

    def set_rot_mode(self, mode):
        """'conservative' (default) or 'paper' (the four-step theta_R solver of
        Sec. 5); discards the state."""
        _check(load_library().rpk_set_rot_mode(self._h, {"conservative": 0, "paper": 1}[mode]))
        return self

    def init_fields(self, rho, u, T, R):
        n = self.npts
        args = [_arg(rho, n), _arg(u, 3 * n), _arg(T, n), _arg(R, n)]
        dev = {a[1] for a in args}
        if len(dev) != 1:
            raise ValueError("all fields must be on the host or all on the device")
        _check(load_library().rpk_init_fields(self._h, *[a[0] for a in args], dev.pop()))
        return self

    def step(self, n=1):
        _check(load_library().rpk_step(self._h, int(n)))
        return self

    def read_moments(self, out=None, check=True):
        """dict rho, u (3, npts), T, R, Erot. ``out`` may hold preallocated
        numpy arrays or CUDA float64 tensors with those keys."""
        n = self.npts
        if out is None:
            out = {"rho": np.empty(n), "u": np.empty((3, n)), "T": np.empty(n),
                   "R": np.empty(n), "Erot": np.empty(n)}
        sizes = {"rho": n, "u": 3 * n, "T": n, "R": n, "Erot": n}
        args = {k: _arg(out[k], sizes[k]) if k in out else (None, None, None) for k in sizes}
        dev = {a[1] for a in args.values() if a[1] is not None}
        if len(dev) != 1:
            raise ValueError("outputs must be all host or all device")
        code = load_library().rpk_read_moments(self._h, args["rho"][0], args["u"][0],
                                               args["T"][0], args["R"][0], args["Erot"][0],
                                               dev.pop())
        if check:
            _check(code)
        res = {}
        for k in sizes:
            if k in out:
                a = args[k][2]
                res[k] = a.reshape(3, n) if k == "u" else a
        return res

    def diagnostics(self, check=True):
        d = Diag()
        code = load_library().rpk_diagnostics(self._h, ctypes.byref(d))
        if check:
            _check(code)
        return {"M": d.mass, "J": np.array(d.mom[:]), "E": d.energy, "H1": d.H1,
                "min_g": d.min_g, "status": d.status, "steps": d.steps}

    def save(self, path):
        _check(load_library().rpk_save(self._h, os.fsencode(path)))

    def load(self, path):
        _check(load_library().rpk_load(self._h, os.fsencode(path)))
        return self

    def timing(self, enable=True):
        """Start (clearing the counters) or stop per-kernel-class CUDA-event timing."""
        _check(load_library().rpk_timing(self._h, 1 if enable else 0))
        return self

    def timing_read(self):
        """{class: (ms, launches)} for 'collide' and 'transport' since the last start."""
        ms = (ctypes.c_double * 2)()
        n = (ctypes.c_int64 * 2)()
        _check(load_library().rpk_timing_read(self._h, ms, n))
        return {name: (ms[i], n[i]) for i, name in enumerate(("collide", "transport"))}

    def info(self):
        out = (ctypes.c_int64 * 4)()
        _check(load_library().rpk_get_info(self._h, out))
        return {"nsub": out[0], "steps": out[1], "npts": out[2], "bytes": out[3]}


class Batch:
    """Many quasi-1-D tubes (nx x 1 x 1 lattices with x reservoirs) advanced in
    one persistent launch (rpk_batch_*). ``tubes`` is a sequence of dicts with
    keys nx, nsteps, relax (dict of rpk_relax fields) and res (12 reservoir
    values). Fields are concatenated tube after tube (2 nx points each)."""

    def __init__(self, tubes, precision="f32", save_every=32, stream=None):
        lib = load_library()
        arr = (Tube * len(tubes))(*[_tube_struct(d) for d in tubes])
        self.tubes = [dict(d) for d in tubes]
        self.save_every = int(save_every)
        self.offsets = np.cumsum([0] + [2 * int(d["nx"]) for d in tubes])
        self.total_pts = int(self.offsets[-1])
        h = ctypes.c_void_p()
        _check(lib.rpk_batch_create(PRECISIONS[precision], len(tubes), arr, self.save_every,
                                    _stream_handle(stream), ctypes.byref(h)))
        self._h = h

    @staticmethod
    def max_nx(precision="f32"):
        return load_library().rpk_batch_max_nx(PRECISIONS[precision])

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            load_library().rpk_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init_fields(self, rho, u, T, R):
        n = self.total_pts
        a = [np.ascontiguousarray(x, dtype=np.float64).reshape(-1) for x in (rho, u, T, R)]
        if [x.size for x in a] != [n, 3 * n, n, n]:
            raise ValueError("concatenated fields of %d points expected" % n)
        _check(load_library().rpk_batch_init(self._h, *[x.ctypes.data_as(ctypes.c_void_p)
                                                        for x in a]))
        self._keep = a
        return self

    def set_diffusion(self, mode):
        """'ftcs' (the paper's sub-stepped scheme, default) or 'implicit'
        (one backward-Euler step per time step)."""
        _check(load_library().rpk_batch_set_diffusion(self._h, {"ftcs": 0, "implicit": 1}[mode]))
        return self

    def set_config(self, threads, ctas_per_sm=1):
        _check(load_library().rpk_batch_set_config(self._h, int(threads), int(ctas_per_sm)))
        return self

    def autotune(self):
        out = (ctypes.c_int64 * 3)()
        _check(load_library().rpk_batch_autotune(self._h, out))
        return {"threads": out[0], "ctas_per_sm": out[1], "sample_ms": out[2] / 1000.0}

    def run(self):
        _check(load_library().rpk_batch_run(self._h))
        return self

    def read_moments(self, check=True):
        n = self.total_pts
        out = {"rho": np.empty(n), "u": np.empty((3, n)), "T": np.empty(n), "R": np.empty(n),
               "Erot": np.empty(n)}
        code = load_library().rpk_batch_read_moments(
            self._h, *[out[k].ctypes.data_as(ctypes.c_void_p) for k in ("rho", "u", "T", "R", "Erot")])
        if check:
            _check(code)
        return out

    @property
    def block_offsets(self):
        """Float offset of each tube's moment block [4][2 nx] (8 nx floats per tube)."""
        return 4 * self.offsets[:-1]

    def init_device(self, state):
        """Initialise from moment blocks (CUDA float32 tensor of 4 * total_pts)."""
        _check(load_library().rpk_batch_init_device(self._h, _dev_f32(state, (4 * self.total_pts,), "state")))
        return self

    def set_steps(self, nsteps):
        arr = (ctypes.c_int * len(self.tubes))(*[int(v) for v in nsteps])
        _check(load_library().rpk_batch_set_steps(self._h, arr))
        return self

    def moments_device(self, out=None):
        """Current moments as moment blocks (CUDA float32 tensor of 4 * total_pts)."""
        import torch
        if out is None:
            out = torch.empty(4 * self.total_pts, device="cuda", dtype=torch.float32)
        _check(load_library().rpk_batch_moments_device(self._h, _dev_f32(out, (4 * self.total_pts,), "out")))
        return out

    def snapshots(self):
        """List per tube of float32 arrays (nsnap, 4, 2 nx): rho, u_x, theta_T, E_R at
        steps 0, save_every, ... of the last run."""
        lib = load_library()
        cnt = ctypes.c_int64()
        _check(lib.rpk_batch_snapshots(self._h, None, ctypes.byref(cnt)))
        buf = np.empty(cnt.value, dtype=np.float32)
        _check(lib.rpk_batch_snapshots(self._h, buf.ctypes.data_as(ctypes.c_void_p), ctypes.byref(cnt)))
        res, off = [], 0
        for d in self.tubes:
            np2 = 2 * int(d["nx"])
            ns = (int(d["nsteps"]) + self.save_every - 1) // self.save_every
            res.append(buf[off:off + ns * 4 * np2].reshape(ns, 4, np2))
            off += ns * 4 * np2
        return res


def _dev_f32(t, shape=None, name="tensor"):
    """Device pointer of a contiguous CUDA float32 torch tensor."""
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32
            and t.is_contiguous()):
        raise TypeError("%s must be a contiguous CUDA float32 tensor" % name)
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError("%s has shape %s, expected %s" % (name, tuple(t.shape), tuple(shape)))
    return ctypes.c_void_p(t.data_ptr())


class Net:
    """The surrogate network of the C interface (rpk_net_*): a 1-D convolutional
    operator on position-major tensors [sequence][point][channel], trained and
    evaluated by the library's BF16 tensor-core kernels. Tensors are contiguous
    CUDA float32 torch tensors; parameters cross as host numpy float32 vectors."""

    def __init__(self, cin, cout, width=128, nblocks=6, seed=0, stream=None):
        h = ctypes.c_void_p()
        _check(load_library().rpk_net_create(int(cin), int(cout), int(width), int(nblocks),
                                             int(seed), _stream_handle(stream), ctypes.byref(h)))
        self._h = h
        self.cin, self.cout, self.width, self.nblocks = int(cin), int(cout), int(width), int(nblocks)

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            load_library().rpk_net_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def num_params(self):
        return int(load_library().rpk_net_num_params(self._h))

    def params(self, grads=False):
        out = np.empty(self.num_params, dtype=np.float32)
        _check(load_library().rpk_net_get_params(self._h, out.ctypes.data_as(ctypes.c_void_p),
                                                 1 if grads else 0))
        return out

    def set_params(self, v):
        v = np.ascontiguousarray(v, dtype=np.float32)
        if v.size != self.num_params:
            raise ValueError("expected %d parameters" % self.num_params)
        _check(load_library().rpk_net_set_params(self._h, v.ctypes.data_as(ctypes.c_void_p)))

    def forward(self, x, out=None):
        import torch
        nseq, length, cin = x.shape
        if cin != self.cin:
            raise ValueError("expected %d input channels" % self.cin)
        if out is None:
            out = torch.empty((nseq, length, self.cout), device=x.device, dtype=torch.float32)
        _check(load_library().rpk_net_forward(self._h, _dev_f32(x, name="x"), nseq, length,
                                              _dev_f32(out, (nseq, length, self.cout), "out")))
        return out

    def forward_ragged(self, x, lens, out=None):
        """x [sum(lens)][cin]: sequences of the given lengths (multiples of 4) back to back."""
        import torch
        lens = [int(v) for v in lens]
        n = sum(lens)
        if out is None:
            out = torch.empty((n, self.cout), device=x.device, dtype=torch.float32)
        arr = (ctypes.c_int * len(lens))(*lens)
        _check(load_library().rpk_net_forward_ragged(self._h, _dev_f32(x, (n, self.cin), "x"),
                                                     len(lens), arr,
                                                     _dev_f32(out, (n, self.cout), "out")))
        return out

    def loss_grad(self, x, target, mask):
        nseq, length, _ = x.shape
        loss = ctypes.c_double()
        _check(load_library().rpk_net_loss_grad(
            self._h, _dev_f32(x, (nseq, length, self.cin), "x"),
            _dev_f32(target, (nseq, length, self.cout), "target"),
            _dev_f32(mask, (nseq, length), "mask"), nseq, length, ctypes.byref(loss)))
        return loss.value

    def adam(self, lr, beta1=0.9, beta2=0.999, eps=1e-8):
        _check(load_library().rpk_net_adam(self._h, lr, beta1, beta2, eps))


def _seq_array(seqs):
    """Sequence descriptors (dicts with src, tgt, prev, out, nx, len, crop, res
    (2x4), cond (2)) -> a CUDA uint8 tensor holding the rpk_sur_seq array."""
    import torch
    arr = (SurSeq * len(seqs))()
    for a, d in zip(arr, seqs):
        a.src, a.tgt, a.out = int(d["src"]), int(d.get("tgt", -1)), int(d["out"])
        a.prev = int(d.get("prev", -1))
        a.nx, a.len, a.crop = int(d["nx"]), int(d["len"]), int(d.get("crop", 0))
        for side in range(2):
            for k in range(4):
                a.res[side][k] = float(d["res"][side][k])
        a.cond[0], a.cond[1] = float(d["cond"][0]), float(d["cond"][1])
    raw = np.frombuffer(bytes(arr), dtype=np.uint8).copy()
    return torch.from_numpy(raw).cuda()


def sur_pack(cfg, store, seqs, margin=0, x=None, target=None, mask=None, noise=None, seed=0,
             stream=None):
    """Network inputs (and targets / mask when sequences carry tgt >= 0) for
    the sequences; returns (x, target, mask) as CUDA float32 tensors."""
    import torch
    total = max(int(d["out"]) + int(d["len"]) for d in seqs)
    maxlen = max(int(d["len"]) for d in seqs)
    with_t = any(int(d.get("tgt", -1)) >= 0 for d in seqs)
    if x is None:
        x = torch.zeros((total, 11), device="cuda", dtype=torch.float32)
    if with_t and target is None:
        target = torch.zeros((total, 4), device="cuda", dtype=torch.float32)
    if with_t and mask is None:
        mask = torch.zeros(total, device="cuda", dtype=torch.float32)
    dseq = _seq_array(seqs)
    vp = ctypes.c_void_p
    nz = (ctypes.c_float * 4)(*[float(v) for v in noise]) if noise is not None else None
    _check(load_library().rpk_sur_pack(
        ctypes.byref(cfg), _dev_f32(store, name="store"), vp(dseq.data_ptr()), len(seqs), maxlen,
        int(margin), nz, int(seed), _dev_f32(x, name="x"), _dev_f32(target, name="target") if with_t else None,
        _dev_f32(mask, name="mask") if with_t else None, _stream_handle(stream)))
    torch.cuda.synchronize()
    return x, target, mask


def sur_apply(cfg, state, y, seqs, stream=None):
    """One conservative network update of the tubes in seqs: returns (next state
    tensor, flags (numpy int), totals (numpy (n, 2)))."""
    import torch
    nxt = state.clone()
    n = len(seqs)
    flags = torch.zeros(n, device="cuda", dtype=torch.int32)
    tot = torch.zeros((n, 2), device="cuda", dtype=torch.float64)
    dseq = _seq_array(seqs)
    vp = ctypes.c_void_p
    _check(load_library().rpk_sur_apply(ctypes.byref(cfg), _dev_f32(state, name="state"),
                                        _dev_f32(y, name="y"), vp(dseq.data_ptr()), n,
                                        _dev_f32(nxt, name="next"), vp(flags.data_ptr()),
                                        vp(tot.data_ptr()), _stream_handle(stream)))
    torch.cuda.synchronize()
    return nxt, flags.cpu().numpy(), tot.cpu().numpy()


class Rollout:
    """Surrogate rollout with LBM fallback (rpk_rollout_*): ``net`` a Net,
    ``tubes`` as for Batch (every relax must carry nsub > 0), ``cond`` (ntubes,
    2) conditioning features, ``cfg`` a SurConfig."""

    def __init__(self, net, cfg, tubes, cond, stream=None):
        lib = load_library()
        arr = (Tube * len(tubes))(*[_tube_struct(d) for d in tubes])
        c = np.ascontiguousarray(cond, dtype=np.float32).reshape(-1)
        if c.size != 2 * len(tubes):
            raise ValueError("cond must have 2 values per tube")
        h = ctypes.c_void_p()
        _check(lib.rpk_rollout_create(net._h, ctypes.byref(cfg), len(tubes), arr,
                                      c.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                      _stream_handle(stream), ctypes.byref(h)))
        self._h, self._net, self.cfg = h, net, cfg
        self.ntubes = len(tubes)

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            load_library().rpk_rollout_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def run(self, state):
        """Advance the moment blocks ``state`` (CUDA float32 tensor) in place.
        Returns a dict: fail_step, windows, checks, lbm_steps, rerun (per
        tube), est (estimated L1 error per tube), ms (network, spot checks,
        final LBM, repeated runs)."""
        n = self.ntubes
        stats = np.zeros(5 * n, dtype=np.int64)
        est = np.zeros(n)
        ms = np.zeros(4)
        _check(load_library().rpk_rollout_run(
            self._h, _dev_f32(state, name="state"),
            stats.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
            est.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
            ms.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        st = stats.reshape(n, 5)
        return {"fail_step": st[:, 0], "windows": st[:, 1], "checks": st[:, 2],
                "lbm_steps": st[:, 3], "rerun": st[:, 4], "est": est, "ms": ms}

    def errors(self):
        """(ntubes, windows) spot-check L1 errors of the last run (NaN: unchecked)."""
        w = ctypes.c_int()
        _check(load_library().rpk_rollout_errors(self._h, None, ctypes.byref(w)))
        out = np.full((self.ntubes, max(w.value, 1)), np.nan)
        _check(load_library().rpk_rollout_errors(self._h, out.ctypes.data_as(ctypes.c_void_p),
                                                 ctypes.byref(w)))
        return out[:, :w.value]
