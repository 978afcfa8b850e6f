"""Python binding of the lbmh C ABI (include/lbmh.h): argument marshalling only.

Every step of the method runs in the CUDA library ``_lbmh.so`` built from
``csrc/`` for sm_103a.  There is no fallback: if the library is missing or no
CUDA device is present, the calls raise.

Device arrays are passed as torch tensors (their data pointers); host arrays
as numpy arrays.  The CUDA stream is torch's current stream unless one is
given.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# LBMH_LIBRARY=checked selects the bounds-checked build (debug runs of the tests)
LIB_PATH = os.path.join(HERE, "_lbmh_checked.so" if os.environ.get("LBMH_LIBRARY") == "checked" else "_lbmh.so")

OK, ERR_INVALID_ARG, ERR_OOM, ERR_NONPHYSICAL, ERR_TIMEOUT, ERR_CUDA, ERR_UNSUPPORTED = 0, -1, -2, -3, -4, -5, -6
ERR_BOUNDS = -7  # bounds-checked build only: an index left its array
KERNEL_AUTO, KERNEL_FUSED, KERNEL_UNFUSED = 0, 1, 2
FP64, FP32 = 0, 1


class LbmhError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"lbmh error {code}: {msg}")
        self.code = code


class _Problem(ctypes.Structure):
    _fields_ = [
        ("system", ctypes.c_int), ("dim", ctypes.c_int),
        ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("x0", ctypes.c_double), ("x1", ctypes.c_double),
        ("y0", ctypes.c_double), ("y1", ctypes.c_double),
        ("bc", ctypes.c_int * 4),
        ("cfl", ctypes.c_double), ("eps", ctypes.c_double),
        ("adv", ctypes.c_double * 2),
        ("gamma", ctypes.c_double), ("g", ctypes.c_double),
        ("bed_amp", ctypes.c_double), ("bed_w2", ctypes.c_double),
        ("bed_xc", ctypes.c_double), ("bed_yc", ctypes.c_double),
        ("K", ctypes.c_double), ("Ti", ctypes.c_double), ("q", ctypes.c_double),
        ("m_linear", ctypes.c_int),
        ("A", ctypes.POINTER(ctypes.c_double)),
        ("omega_mode", ctypes.c_int), ("omega_fixed", ctypes.c_double),
        ("h_dry", ctypes.c_double),
        ("precision", ctypes.c_int), ("kernel", ctypes.c_int),
        ("cuda_stream", ctypes.c_void_p),
        ("sponge_width", ctypes.c_double),
        ("u_in", ctypes.c_double * 8),
        ("nz", ctypes.c_int),
        ("z0", ctypes.c_double), ("z1", ctypes.c_double),
        ("bc_z", ctypes.c_int * 2),
        ("adv_z", ctypes.c_double),
    ]


class Info(ctypes.Structure):
    _fields_ = [
        ("t", ctypes.c_double), ("steps", ctypes.c_int64),
        ("abar", ctypes.c_double * 2),
        ("last_dt", ctypes.c_double), ("last_lambda", ctypes.c_double),
        ("sum_U", ctypes.c_double * 8),
        ("status", ctypes.c_uint32), ("m", ctypes.c_int), ("Q", ctypes.c_int),
        ("kernel", ctypes.c_int), ("device_bytes", ctypes.c_int64),
        ("abar_z", ctypes.c_double),
        ("halo_bytes", ctypes.c_int64), ("halo_rows", ctypes.c_int * 2), ("row0", ctypes.c_int),
    ]

    def as_dict(self):
        return {"t": self.t, "steps": self.steps, "abar": list(self.abar),
                "last_dt": self.last_dt, "last_lambda": self.last_lambda,
                "sum_U": list(self.sum_U)[: self.m], "status": self.status, "m": self.m,
                "Q": self.Q, "kernel": self.kernel, "device_bytes": self.device_bytes, "abar_z": self.abar_z,
                "halo_bytes": self.halo_bytes, "halo_rows": list(self.halo_rows), "row0": self.row0}


_lib = None

# (name, restype, argtypes) of every entry point declared in include/lbmh.h
_H = ctypes.c_void_p
_DP = ctypes.c_void_p
SIGNATURES = [
    ("lbmh_create", ctypes.c_int, [ctypes.POINTER(_Problem), ctypes.POINTER(ctypes.c_void_p)]),
    ("lbmh_set_state", ctypes.c_int, [_H, _DP, ctypes.c_int]),
    ("lbmh_step", ctypes.c_int, [_H, ctypes.c_int64]),
    ("lbmh_advance_to", ctypes.c_int, [_H, ctypes.c_double, ctypes.c_int64]),
    ("lbmh_moments", ctypes.c_int, [_H, _DP, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                    ctypes.POINTER(ctypes.c_int64)]),
    ("lbmh_get_f", ctypes.c_int, [_H, _DP, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                  ctypes.POINTER(ctypes.c_int64)]),
    ("lbmh_set_f", ctypes.c_int, [_H, _DP, ctypes.c_int, ctypes.c_double, ctypes.c_int64]),
    ("lbmh_omega", ctypes.c_int, [_H, _DP, ctypes.c_int]),
    ("lbmh_get_info", ctypes.c_int, [_H, ctypes.POINTER(Info)]),
    ("lbmh_destroy", ctypes.c_int, [_H]),
    ("lbmh_step_static", ctypes.c_int, [ctypes.POINTER(_Problem), _DP, _DP, ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(ctypes.c_uint32)]),
    ("lbmh_create_slab", ctypes.c_int, [ctypes.POINTER(_Problem), ctypes.c_int, ctypes.c_int,
                                        ctypes.POINTER(ctypes.c_void_p)]),
    ("lbmh_state_speed_bound", ctypes.c_int, [_H, _DP, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
    ("lbmh_set_state_bound", ctypes.c_int, [_H, _DP, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
    ("lbmh_get_speed_bound", ctypes.c_int, [_H, ctypes.POINTER(ctypes.c_double)]),
    ("lbmh_set_speed_bound", ctypes.c_int, [_H, ctypes.POINTER(ctypes.c_double)]),
    ("lbmh_halo_get", ctypes.c_int, [_H, ctypes.c_int, _DP, ctypes.c_int]),
    ("lbmh_halo_set", ctypes.c_int, [_H, ctypes.c_int, _DP, ctypes.c_int]),
    ("lbmh_batch_create", ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p,
                                         ctypes.POINTER(ctypes.c_void_p)]),
    ("lbmh_batch_footprint", ctypes.c_int64, [ctypes.POINTER(_Problem)]),
    ("lbmh_batch_add", ctypes.c_int, [_H, ctypes.POINTER(_Problem), _DP, ctypes.c_int, ctypes.c_int64,
                                      ctypes.c_double, ctypes.POINTER(ctypes.c_int)]),
    ("lbmh_batch_remove", ctypes.c_int, [_H, ctypes.c_int]),
    ("lbmh_batch_step", ctypes.c_int, [_H, ctypes.c_int64]),
    ("lbmh_batch_autotune", ctypes.c_int, [_H, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
    ("lbmh_batch_poll", ctypes.c_int, [_H, _DP, _DP, _DP, _DP]),
    ("lbmh_batch_moments", ctypes.c_int, [_H, ctypes.c_int, _DP, ctypes.c_int]),
    ("lbmh_batch_info", ctypes.c_int, [_H, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                                       ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                       ctypes.POINTER(ctypes.c_int)]),
    ("lbmh_batch_destroy", ctypes.c_int, [_H]),
    ("lbmh_batch_last_error", ctypes.c_char_p, [_H]),
    ("lbmh_last_error", ctypes.c_char_p, [_H]),
    ("lbmh_version", ctypes.c_char_p, []),
]


def load(path=LIB_PATH):
    """Load the CUDA library; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"lbmh CUDA library not built ({path}); run "
                          "python -m paper_2609_18177_b300.build")
    lib = ctypes.CDLL(path)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _c_problem(pb, precision, kernel, stream):
    s = _Problem()
    s.system, s.dim, s.nx = int(pb.system), int(pb.dim), int(pb.nx)
    s.ny = int(pb.ny) if pb.dim >= 2 else 1
    s.x0, s.x1, s.y0, s.y1 = float(pb.x0), float(pb.x1), float(pb.y0), float(pb.y1)
    for i in range(4):
        s.bc[i] = int(pb.bc[i])
    s.cfl, s.eps = float(pb.cfl), float(pb.eps)
    s.adv[0], s.adv[1] = float(pb.adv[0]), float(pb.adv[1])
    s.gamma, s.g = float(pb.gamma), float(pb.g)
    s.bed_amp, s.bed_w2, s.bed_xc, s.bed_yc = (float(pb.bed_amp), float(pb.bed_w2),
                                               float(pb.bed_xc), float(pb.bed_yc))
    s.K, s.Ti, s.q = float(pb.K), float(pb.Ti), float(pb.q)
    s.m_linear = int(getattr(pb, "m_linear", 0))
    s.omega_mode, s.omega_fixed = int(pb.omega_mode), float(pb.omega_fixed)
    s.h_dry = float(pb.h_dry)
    s.precision, s.kernel = int(precision), int(kernel)
    s.cuda_stream = stream
    s.sponge_width = float(getattr(pb, "sponge_width", 0.0))
    for i, v in enumerate(tuple(getattr(pb, "u_in", ()))[:8]):
        s.u_in[i] = float(v)
    if pb.dim == 3:
        s.nz = int(pb.nz)
        s.z0, s.z1 = float(pb.z0), float(pb.z1)
        s.bc_z[0], s.bc_z[1] = int(pb.bc_z[0]), int(pb.bc_z[1])
        s.adv_z = float(pb.adv[2]) if len(pb.adv) > 2 else 0.0
    else:
        s.nz = 1
    return s


def _current_stream():
    import torch
    return torch.cuda.current_stream().cuda_stream


def _ptr(a):
    """(pointer, on_device) of a numpy array or a torch tensor (FP64, contiguous)."""
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags.c_contiguous:
            raise TypeError("host arrays must be C-contiguous float64")
        return a.ctypes.data, 0
    import torch
    if isinstance(a, torch.Tensor):
        if a.dtype != torch.float64 or not a.is_contiguous():
            raise TypeError("tensors must be contiguous float64")
        return a.data_ptr(), 1 if a.is_cuda else 0
    raise TypeError(f"unsupported array type {type(a)}")


class Solver:
    """One lattice held on the GPU (a handle of the C ABI)."""

    def __init__(self, pb, precision=None, kernel=KERNEL_AUTO, stream=None):
        lib = load()
        self.pb = pb
        self.precision = pb.precision if precision is None else precision
        self._stream = _current_stream() if stream is None else stream
        self._s = _c_problem(pb, self.precision, kernel, self._stream)
        h = ctypes.c_void_p()
        rc = lib.lbmh_create(ctypes.byref(self._s), ctypes.byref(h))
        if rc != OK:
            raise LbmhError(rc, lib.lbmh_last_error(None).decode())
        self._h = h
        self.m = pb.nfields
        self.Q = 2 * pb.dim + 1

    def _check(self, rc):
        if rc != OK:
            raise LbmhError(rc, load().lbmh_last_error(self._h).decode())

    @property
    def shape_U(self):
        return (self.m,) + self.pb.shape()

    @property
    def shape_f(self):
        return (self.Q, self.m) + self.pb.shape()

    def set_state(self, U):
        if isinstance(U, np.ndarray):
            U = np.ascontiguousarray(U, dtype=np.float64).reshape(self.shape_U)
        p, dev = _ptr(U)
        self._check(load().lbmh_set_state(self._h, p, dev))
        return self

    def step(self, n=1):
        self._check(load().lbmh_step(self._h, int(n)))
        return self

    def advance_to(self, T, max_steps=2**62):
        self._check(load().lbmh_advance_to(self._h, float(T), int(max_steps)))
        return self

    def moments(self, out=None, check=True):
        if out is None:
            out = np.empty(self.shape_U)
        p, dev = _ptr(out)
        t = ctypes.c_double()
        n = ctypes.c_int64()
        rc = load().lbmh_moments(self._h, p, dev, ctypes.byref(t), ctypes.byref(n))
        if check or rc != ERR_NONPHYSICAL:
            self._check(rc)
        self.t, self.nsteps = t.value, n.value
        return out

    def get_f(self, out=None):
        if out is None:
            out = np.empty(self.shape_f)
        p, dev = _ptr(out)
        t = ctypes.c_double()
        n = ctypes.c_int64()
        self._check(load().lbmh_get_f(self._h, p, dev, ctypes.byref(t), ctypes.byref(n)))
        self.t, self.nsteps = t.value, n.value
        return out

    def set_f(self, f, t=0.0, steps=0):
        if isinstance(f, np.ndarray):
            f = np.ascontiguousarray(f, dtype=np.float64)
        p, dev = _ptr(f)
        self._check(load().lbmh_set_f(self._h, p, dev, float(t), int(steps)))
        return self

    def omega(self, out=None):
        if out is None:
            out = np.empty(self.pb.shape())
        p, dev = _ptr(out)
        self._check(load().lbmh_omega(self._h, p, dev))
        return out

    def info(self):
        inf = Info()
        self._check(load().lbmh_get_info(self._h, ctypes.byref(inf)))
        return inf.as_dict()

    def close(self):
        if getattr(self, "_h", None):
            load().lbmh_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def _raw_ptr(a):
    """(pointer, on_device) of a contiguous numpy array or torch tensor of any dtype."""
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            raise TypeError("host arrays must be C-contiguous")
        return a.ctypes.data, 0
    import torch
    if isinstance(a, torch.Tensor):
        if not a.is_contiguous():
            raise TypeError("tensors must be contiguous")
        return a.data_ptr(), 1 if a.is_cuda else 0
    raise TypeError(f"unsupported array type {type(a)}")


def _vec(values, n=3):
    v = (ctypes.c_double * n)()
    for i, x in enumerate(list(values)[:n]):
        v[i] = float(x)
    return v


class Slab(Solver):
    """Rows [row_begin, row_end) of a 2D lattice decomposed along y (a slab
    handle of the C ABI): the local lattice holds those rows plus three halo
    rows on each side that borders another slab.  U and f arrays cover the
    local lattice, halo rows included."""

    def __init__(self, pb, row_begin, row_end, precision=None, stream=None):
        lib = load()
        self.pb_global = pb
        self.precision = pb.precision if precision is None else precision
        self._stream = _current_stream() if stream is None else stream
        self._s = _c_problem(pb, self.precision, KERNEL_FUSED, self._stream)
        h = ctypes.c_void_p()
        rc = lib.lbmh_create_slab(ctypes.byref(self._s), int(row_begin), int(row_end), ctypes.byref(h))
        if rc != OK:
            raise LbmhError(rc, lib.lbmh_last_error(None).decode())
        self._h = h
        self.m = pb.nfields
        self.Q = 2 * pb.dim + 1
        inf = Info()
        self._check(lib.lbmh_get_info(self._h, ctypes.byref(inf)))
        self.halo = tuple(inf.halo_rows)
        self.row0 = inf.row0
        self.halo_bytes = inf.halo_bytes
        self.rows = (row_begin, row_end)
        ny_local = row_end - row_begin + self.halo[0] + self.halo[1]
        self.pb = pb.with_(ny=ny_local, y1=pb.y0 + ny_local * pb.dx)

    def state_speed_bound(self, U):
        U = np.ascontiguousarray(U, dtype=np.float64).reshape(self.shape_U) if isinstance(U, np.ndarray) else U
        p, dev = _ptr(U)
        out = (ctypes.c_double * 3)()
        self._check(load().lbmh_state_speed_bound(self._h, p, dev, out))
        return list(out)[: self.pb.dim]

    def set_state_bound(self, U, abar):
        U = np.ascontiguousarray(U, dtype=np.float64).reshape(self.shape_U) if isinstance(U, np.ndarray) else U
        p, dev = _ptr(U)
        self._check(load().lbmh_set_state_bound(self._h, p, dev, _vec(abar)))
        return self

    def get_speed_bound(self):
        out = (ctypes.c_double * 3)()
        self._check(load().lbmh_get_speed_bound(self._h, out))
        return list(out)[: self.pb.dim]

    def set_speed_bound(self, abar):
        self._check(load().lbmh_set_speed_bound(self._h, _vec(abar)))
        return self

    def halo_get(self, side, out):
        p, dev = _raw_ptr(out)
        self._check(load().lbmh_halo_get(self._h, int(side), p, dev))
        return out

    def halo_set(self, side, rows):
        p, dev = _raw_ptr(rows)
        self._check(load().lbmh_halo_set(self._h, int(side), p, dev))
        return self


class Batch:
    """Many 2D lattices of one system and precision advanced together (a batch
    of the C ABI).  Lattices are admitted into a fixed device arena."""

    def __init__(self, system, precision=FP32, capacity_bytes=1 << 30, max_instances=1024, stream=None):
        lib = load()
        self._stream = _current_stream() if stream is None else stream
        h = ctypes.c_void_p()
        rc = lib.lbmh_batch_create(int(system), int(precision), int(capacity_bytes), int(max_instances),
                                   self._stream, ctypes.byref(h))
        if rc != OK:
            raise LbmhError(rc, lib.lbmh_batch_last_error(None).decode())
        self._h = h
        self.system, self.precision, self.max_instances = system, precision, max_instances
        self.problems = {}

    def _check(self, rc):
        if rc != OK:
            raise LbmhError(rc, load().lbmh_batch_last_error(self._h).decode())

    @staticmethod
    def footprint(pb, precision=FP32):
        s = _c_problem(pb, precision, KERNEL_AUTO, None)
        return int(load().lbmh_batch_footprint(ctypes.byref(s)))

    def add(self, pb, U0, max_steps=0, T=0.0):
        """Admit a lattice; returns its slot, or None if the arena or the slots are full."""
        s = _c_problem(pb, self.precision, KERNEL_AUTO, self._stream)
        if isinstance(U0, np.ndarray):
            U0 = np.ascontiguousarray(U0, dtype=np.float64)
        p, dev = _ptr(U0)
        slot = ctypes.c_int(-1)
        rc = load().lbmh_batch_add(self._h, ctypes.byref(s), p, dev, int(max_steps), float(T), ctypes.byref(slot))
        if rc == ERR_OOM:
            return None
        self._check(rc)
        self.problems[slot.value] = pb
        return slot.value

    def remove(self, slot):
        self._check(load().lbmh_batch_remove(self._h, int(slot)))
        self.problems.pop(slot, None)

    def step(self, n=1):
        self._check(load().lbmh_batch_step(self._h, int(n)))
        return self

    def autotune(self, steps_per_candidate=3):
        ms = ctypes.c_double(0.0)
        self._check(load().lbmh_batch_autotune(self._h, int(steps_per_candidate), ctypes.byref(ms)))
        return ms.value

    def poll(self):
        n = self.max_instances
        done = np.zeros(n, dtype=np.int32)
        t = np.zeros(n)
        steps = np.zeros(n, dtype=np.int64)
        status = np.zeros(n, dtype=np.uint32)
        self._check(load().lbmh_batch_poll(self._h, done.ctypes.data, t.ctypes.data, steps.ctypes.data,
                                           status.ctypes.data))
        return done, t, steps, status

    def moments(self, slot, out=None):
        pb = self.problems[slot]
        if out is None:
            out = np.empty((pb.nfields,) + pb.shape())
        p, dev = _ptr(out)
        self._check(load().lbmh_batch_moments(self._h, int(slot), p, dev))
        return out

    def info(self):
        used, cap = ctypes.c_int64(), ctypes.c_int64()
        act, grid, var = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        self._check(load().lbmh_batch_info(self._h, ctypes.byref(used), ctypes.byref(cap), ctypes.byref(act),
                                           ctypes.byref(grid), ctypes.byref(var)))
        return {"used_bytes": used.value, "capacity_bytes": cap.value, "active": act.value,
                "grid": grid.value, "variant": var.value}

    def close(self):
        if getattr(self, "_h", None):
            load().lbmh_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _check_static_arrays(pb, f_in, f_out):
    """The C entry point cannot see array sizes: before any launch, require two
    contiguous FP64 tensors of exactly the lattice's shape [Q][m][ny][nx] on the
    current CUDA device, with storage that does not overlap."""
    import torch
    shape = (pb.nvel, pb.nfields, pb.ny if pb.dim == 2 else 1, pb.nx)
    for name, a in (("f_in", f_in), ("f_out", f_out)):
        if not isinstance(a, torch.Tensor):
            raise TypeError(f"step_static: {name} must be a torch tensor")
        if tuple(a.shape) != shape and not (pb.dim == 1 and tuple(a.shape) == shape[:2] + shape[3:]):
            raise TypeError(f"step_static: {name} has shape {tuple(a.shape)}, the lattice needs {shape}")
    for name, a in (("f_in", f_in), ("f_out", f_out)):
        if a.dtype != torch.float64 or not a.is_contiguous():
            raise TypeError(f"step_static: {name} must be contiguous float64")
        if not a.is_cuda:
            raise TypeError(f"step_static: {name} must be a CUDA tensor")
        if a.device.index != torch.cuda.current_device():
            raise TypeError(f"step_static: {name} is on {a.device}, the current device is "
                            f"cuda:{torch.cuda.current_device()}")
    nbytes = f_in.numel() * 8
    a0, b0 = f_in.data_ptr(), f_out.data_ptr()
    if a0 < b0 + nbytes and b0 < a0 + nbytes:
        raise TypeError("step_static: f_in and f_out overlap")


def step_static(pb, f_in, f_out, stream=None, want_dt=True, want_status=False):
    """One FP64 step f_in -> f_out on device tensors [Q][m][ny][nx] through the
    allocation-free entry point (scratch in the library's static device
    array).  Returns dt when want_dt, (dt, status bits) when want_status too
    (either synchronises the stream)."""
    if pb.dim not in (1, 2):
        raise TypeError("step_static serves 1D and 2D lattices")
    _check_static_arrays(pb, f_in, f_out)
    lib = load()
    s = _c_problem(pb, FP64, KERNEL_UNFUSED, _current_stream() if stream is None else stream)
    dt = ctypes.c_double(0.0)
    st = ctypes.c_uint32(0)
    rc = lib.lbmh_step_static(ctypes.byref(s), f_in.data_ptr(), f_out.data_ptr(),
                              ctypes.byref(dt) if (want_dt or want_status) else None,
                              ctypes.byref(st) if want_status else None)
    if rc != OK:
        raise LbmhError(rc, lib.lbmh_last_error(None).decode())
    if want_status:
        return dt.value, st.value
    return dt.value if want_dt else None


def version():
    return load().lbmh_version().decode()
