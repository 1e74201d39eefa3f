"""Thin ctypes binding of the C ABI declared in include/seird.h.

Argument marshalling only: every step of the SEIRD Newton-Krylov-Schwarz path
runs in the CUDA library.  Importing this module loads ``_lib/libseird.so`` and
raises ``ImportError`` when it is missing; there is no fallback.

Device buffers may be passed as torch CUDA tensors (float64, contiguous), host
buffers as numpy arrays; the ``on_device`` flag of the C ABI is set from the
argument's type.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libseird.so")

if not os.path.exists(LIB_PATH):
    raise ImportError("libseird.so is not built (run __graft_entry__.build() or "
                      "python -m paper_2208_01839_gb300.build): %s" % LIB_PATH)
_lib = C.CDLL(LIB_PATH)

OK = 0
ERRORS = {-1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "ENEWTON_DIVERGED", -5: "ENEWTON_MAXIT",
          -6: "EGMRES", -7: "ENONFINITE", -8: "ETIMEOUT", -9: "ESINGULAR"}

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int32)


class Mesh(C.Structure):
    _fields_ = [("n_nodes", C.c_int64), ("n_tris", C.c_int64), ("xy", _dp), ("tri", _ip)]


class Params(C.Structure):
    _fields_ = [("A", C.c_double), ("beta_i", C.c_double), ("beta_e", C.c_double), ("sigma", C.c_double),
                ("gamma_e", C.c_double), ("gamma_r", C.c_double), ("gamma_d", C.c_double),
                ("alpha", C.c_double), ("mu", C.c_double), ("nu", C.c_double * 4), ("beta_field", _dp)]


class Options(C.Structure):
    _fields_ = [("dt", C.c_double), ("newton_rtol", C.c_double), ("newton_atol", C.c_double),
                ("newton_maxit", C.c_int32), ("ls_maxit", C.c_int32), ("gmres_restart", C.c_int32),
                ("gmres_maxit", C.c_int32), ("gmres_rtol", C.c_double), ("gmres_atol", C.c_double),
                ("gmres_dtol", C.c_double), ("n_subdomains", C.c_int32), ("overlap", C.c_int32),
                ("coarse", C.c_int32), ("precision", C.c_int32), ("quadrature", C.c_int32),
                ("pc_lag", C.c_int32), ("owner", _ip), ("seed", C.c_uint64), ("stream", C.c_void_p),
                ("timing", C.c_int32), ("gmres_forcing", C.c_int32), ("nonlinear", C.c_int32),
                ("gmres_one_pass", C.c_int32), ("picard_tol", C.c_double), ("pc_keep_steps", C.c_int32),
                ("coarse_group", C.c_int32), ("predictor", C.c_int32), ("autotune", C.c_int32),
                ("graph", C.c_int32), ("forcing_first", C.c_double), ("ilu_fill", C.c_int32)]


class BetaSchedule(C.Structure):
    """Sigmoid transmission schedule, Eq. beta_ie and Eq. beta_x."""
    _fields_ = [(k, C.c_double) for k in ("b0", "b1", "t_mid", "beta_central", "beta_eastern", "beta_western",
                                          "x_eastern", "x_western", "k_eastern", "k_western")]


KERNEL_CLASSES = ["residual", "jacobian", "ilu_factor", "coarse_setup", "spmv", "ilu_solve", "coarse_apply", "krylov"]


class Stats(C.Structure):
    _fields_ = [("newton_its", C.c_int32), ("gmres_its", C.c_int32), ("ls_halvings", C.c_int32),
                ("pc_setups", C.c_int32), ("res0", C.c_double), ("res_final", C.c_double),
                ("eps_update", C.c_double), ("ms_assemble", C.c_double), ("ms_setup", C.c_double),
                ("ms_solve", C.c_double), ("ms_total", C.c_double), ("kernel_ms", C.c_double * 8),
                ("kernel_calls", C.c_int32 * 8), ("alg_bytes", C.c_double * 8)]

    def as_dict(self):
        arrays = ("kernel_ms", "kernel_calls", "alg_bytes")
        d = {k: getattr(self, k) for k, _ in self._fields_ if k not in arrays}
        for a in arrays:
            d[a] = {KERNEL_CLASSES[i]: getattr(self, a)[i] for i in range(8)}
        return d


class Misfit(C.Structure):
    _fields_ = [("n_steps", C.c_int32), ("checkpoint_every", C.c_int32), ("n_obs_nodes", C.c_int32),
                ("obs_nodes", _ip), ("n_obs_steps", C.c_int32), ("obs_steps", _ip), ("I_hat", _dp),
                ("D_hat", _dp), ("lin_rtol", C.c_double)]


PARAM_NAMES = ("beta_i", "beta_e", "sigma", "gamma_e", "gamma_r", "gamma_d", "nu_S", "nu_E", "nu_I", "nu_R")


class Info(C.Structure):
    _fields_ = [("n_nodes", C.c_int64), ("n_tris", C.c_int64), ("nnzb", C.c_int64), ("n_subdomains", C.c_int32),
                ("subdomain_rows", C.c_int64), ("subdomain_blocks", C.c_int64), ("max_levels", C.c_int32),
                ("coarse_band", C.c_int32), ("device_bytes", C.c_int64), ("coarse_units", C.c_int32),
                ("spmv_threads", C.c_int32), ("cgs_ctas", C.c_int32), ("cgs_tile", C.c_int32),
                ("ilu_batch", C.c_int32), ("ilu_warps", C.c_int32), ("ilu_ring", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def _sig(name, res, args):
    f = getattr(_lib, name)
    f.restype = res
    f.argtypes = args
    return f


_vp = C.c_void_p
_default_options = _sig("seird_default_options", None, [C.POINTER(Options)])
_create = _sig("seird_create", C.c_int, [C.POINTER(Mesh), C.POINTER(Params), C.POINTER(Options), C.POINTER(_vp)])
_destroy = _sig("seird_destroy", None, [_vp])
_last_error = _sig("seird_last_error", C.c_char_p, [_vp])
_set_state = _sig("seird_set_state", C.c_int, [_vp, _vp, C.c_int, C.c_double])
_get_state = _sig("seird_get_state", C.c_int, [_vp, _vp, C.c_int, C.POINTER(C.c_double)])
_step = _sig("seird_step", C.c_int, [_vp, C.POINTER(Stats)])
_run = _sig("seird_run", C.c_int, [_vp, C.c_int32, C.POINTER(Stats)])
_get_info = _sig("seird_get_info", C.c_int, [_vp, C.POINTER(Info)])
_eval_residual = _sig("seird_eval_residual", C.c_int, [_vp, _vp, _vp, _vp, C.c_int])
_eval_jacobian = _sig("seird_eval_jacobian", C.c_int, [_vp, _vp, C.c_int])
_get_jacobian = _sig("seird_get_jacobian", C.c_int, [_vp, _vp, _vp, _vp])
_apply_jacobian = _sig("seird_apply_jacobian", C.c_int, [_vp, _vp, _vp, C.c_int])
_precond_setup = _sig("seird_precond_setup", C.c_int, [_vp])
_precond_apply = _sig("seird_precond_apply", C.c_int, [_vp, _vp, _vp, C.c_int])
_linear_solve = _sig("seird_linear_solve", C.c_int, [_vp, _vp, _vp, C.c_int, C.POINTER(C.c_int32)])
_bsr_spmv = _sig("seird_bsr_spmv", C.c_int, [C.c_int64, _vp, _vp, _vp, _vp, _vp, _vp])
_bsr_spmv_f32 = _sig("seird_bsr_spmv_f32val", C.c_int, [C.c_int64, _vp, _vp, _vp, _vp, _vp, _vp])
_launch_count = _sig("seird_launch_count", C.c_int64, [])
_setup_check = _sig("seird_setup_check", C.c_int, [C.POINTER(Mesh), C.POINTER(Options), C.POINTER(C.c_int64)])
_create_ensemble = _sig("seird_create_ensemble", C.c_int,
                        [C.POINTER(Mesh), C.c_int32, C.POINTER(Params), C.POINTER(Options), C.POINTER(_vp)])
_set_params = _sig("seird_set_params", C.c_int, [_vp, C.POINTER(Params)])
_set_beta_schedule = _sig("seird_set_beta_schedule", C.c_int, [_vp, C.POINTER(BetaSchedule)])
_adjoint = _sig("seird_adjoint", C.c_int, [_vp, C.POINTER(Misfit), C.POINTER(C.c_double), _vp, _vp])
_set_wait_limit = _sig("seird_set_wait_limit", C.c_int, [_vp, C.c_int32])
_set_launch_shapes = _sig("seird_set_launch_shapes", C.c_int,
                          [_vp, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int32])
_residual_noalloc = _sig("seird_residual_noalloc", C.c_int,
                         [C.c_int64, C.c_int64, _vp, _vp, _vp, _vp, C.POINTER(Params), _vp, C.c_double, C.c_int32,
                          _vp, _vp, _vp, _vp, _vp])
NOALLOC_MAX_TRIS = 65536
NOALLOC_MAX_NODES = 65536


class SeirdError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (ERRORS.get(code, "E?"), code, msg))
        self.code = code


def default_options(**over) -> Options:
    o = Options()
    _default_options(C.byref(o))
    for k, v in over.items():
        setattr(o, k, v)
    return o


def launch_count() -> int:
    return int(_launch_count())


def setup_check(xy, tri, owner=None, **options) -> dict:
    """Host-only check of the set-up the kernels rely on (seird_setup_check):
    raises SeirdError on a violated invariant, else returns the set-up's sizes."""
    xy = np.ascontiguousarray(xy, dtype=np.float64)
    tri = np.ascontiguousarray(tri, dtype=np.int32)
    mesh = Mesh(len(xy), len(tri), xy.ctypes.data_as(_dp), tri.ctypes.data_as(_ip))
    o = default_options(**options)
    own = None
    if owner is not None:
        own = np.ascontiguousarray(owner, dtype=np.int32)
        o.owner = own.ctypes.data_as(_ip)
        o.n_subdomains = int(own.max()) + 1
    st = (C.c_int64 * 8)()
    rc = _setup_check(C.byref(mesh), C.byref(o), st)
    if rc != OK:
        raise SeirdError(rc, _last_error(None).decode())
    keys = ("n_nodes", "n_tris", "nnzb", "n_subdomains", "subdomain_rows", "forward_stages", "backward_stages",
            "violations")
    return {k: int(st[i]) for i, k in enumerate(keys)}


def _ptr(a):
    """(address, on_device) of a numpy array or a torch tensor."""
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data, 0
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr(), int(a.is_cuda)
    raise TypeError("expected a numpy array or a torch tensor")


def _arr(a, count, dtype, name):
    """(address, on_device) of a contiguous numpy array or torch tensor holding
    exactly ``count`` values of ``dtype`` ("float64" or "int32"): the library
    reads and writes that many values behind the pointer, so a wrong size or
    type is refused here, before the call."""
    p, dev = _ptr(a)
    dt = str(a.dtype)
    if dt not in (dtype, "torch." + dtype):
        raise TypeError("%s: expected %s values, got %s" % (name, dtype, dt))
    size = a.size if isinstance(a, np.ndarray) else a.numel()
    if size != count:
        raise ValueError("%s: expected %d values, got %d" % (name, count, size))
    return p, dev


def _same_place(devs, names):
    if len(set(devs)) != 1:
        raise ValueError("%s must all be host arrays or all device tensors" % ", ".join(names))
    return devs[0]


def _stream_handle(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


def bsr_spmv(row_ptr, col, val, x, y, stream=None):
    """y = A x for 5x5-block BSR device tensors (val float64 or float32)."""
    n_rows = row_ptr.numel() - 1
    nnzb = col.numel()
    f32 = str(val.dtype).endswith("float32")
    fn = _bsr_spmv_f32 if f32 else _bsr_spmv
    args = [_arr(row_ptr, n_rows + 1, "int32", "row_ptr"), _arr(col, nnzb, "int32", "col"),
            _arr(val, 25 * nnzb, "float32" if f32 else "float64", "val"), _arr(y, 5 * n_rows, "float64", "y")]
    if not all(dev for _, dev in args) or not (hasattr(x, "is_cuda") and x.is_cuda):
        raise ValueError("bsr_spmv: every array must be a CUDA tensor")
    if str(x.dtype) != "torch.float64":
        raise TypeError("x: expected float64 values, got %s" % x.dtype)
    rc = fn(n_rows, row_ptr.data_ptr(), col.data_ptr(), val.data_ptr(), x.data_ptr(), y.data_ptr(),
            _stream_handle(stream))
    if rc != OK:
        raise SeirdError(rc, "bsr_spmv launch failed")


def params_struct(params) -> Params:
    """Params structure from an object with ``as_dict()`` or a mapping (beta_field left NULL)."""
    p = Params()
    pd = params.as_dict() if hasattr(params, "as_dict") else dict(params)
    for k in ("A", "beta_i", "beta_e", "sigma", "gamma_e", "gamma_r", "gamma_d", "alpha", "mu"):
        setattr(p, k, float(pd[k]))
    for c in range(4):
        p.nu[c] = float(pd["nu"][c])
    return p


def residual_noalloc(xy, tri, inc_ptr, inc, params, u, u_prev, F, dt, quadrature=0, beta_field=None, norm2=None,
                     stream=None):
    """F(u; u_prev) on a mesh held in caller-owned device tensors, without any
    device allocation by the library (see seird_residual_noalloc in seird.h).
    All array arguments are CUDA tensors on one device; ``inc_ptr``/``inc`` give
    each node's incident (3*t + a) entries, ascending in t.  The call runs with
    that device current, on ``stream`` or, by default, on torch's current stream
    of that device (so it is ordered after the work that wrote the inputs)."""
    import torch
    p = params_struct(params)
    n, m = xy.shape[0], tri.shape[0]
    checks = [(xy, 2 * n, "float64", "xy"), (tri, 3 * m, "int32", "tri"), (inc_ptr, n + 1, "int32", "inc_ptr"),
              (inc, 3 * m, "int32", "inc"), (u, 5 * n, "float64", "u"), (u_prev, 5 * n, "float64", "u_prev"),
              (F, 5 * n, "float64", "F")]
    if beta_field is not None:
        checks.append((beta_field, n, "float64", "beta_field"))
    if norm2 is not None:
        checks.append((norm2, 1, "float64", "norm2"))
    if not all(_arr(*ck)[1] for ck in checks):
        raise ValueError("residual_noalloc: every array must be a CUDA tensor")
    # the library launches on the current device: every tensor must live there
    devs = {ck[0].device for ck in checks}
    if len(devs) != 1:
        raise ValueError("residual_noalloc: tensors on several devices: %s" % sorted(str(d) for d in devs))
    dev = devs.pop()
    with torch.cuda.device(dev):
        sh = _stream_handle(stream) if stream is not None else torch.cuda.current_stream(dev).cuda_stream
        rc = _residual_noalloc(xy.shape[0], tri.shape[0], xy.data_ptr(), tri.data_ptr(), inc_ptr.data_ptr(),
                               inc.data_ptr(), C.byref(p), None if beta_field is None else beta_field.data_ptr(),
                               float(dt), int(quadrature), u.data_ptr(), u_prev.data_ptr(), F.data_ptr(),
                               None if norm2 is None else norm2.data_ptr(), sh)
    if rc != OK:
        raise SeirdError(rc, _last_error(None).decode())


class Solver:
    """One SEIRD context: mesh, parameters and options live on the device.

    ``params`` may be a list of parameter sets: the context is then an ensemble
    (seird_create_ensemble) with one sample per entry, and states have
    len(params) * n_nodes rows, sample-major."""

    def __init__(self, xy, tri, params, options: Options | None = None, beta_field=None, owner=None, stream=None,
                 **opt_over):
        self._xy = np.ascontiguousarray(xy, dtype=np.float64)
        self._tri = np.ascontiguousarray(tri, dtype=np.int32)
        if self._xy.ndim != 2 or self._xy.shape[1] != 2 or self._tri.ndim != 2 or self._tri.shape[1] != 3:
            raise ValueError("xy must be [n, 2] and tri [m, 3], got %s and %s" % (self._xy.shape, self._tri.shape))
        mesh = Mesh(len(self._xy), len(self._tri), self._xy.ctypes.data_as(_dp), self._tri.ctypes.data_as(_ip))
        samples = list(params) if isinstance(params, (list, tuple)) else None
        self.n_samples = len(samples) if samples is not None else 1
        self.n = len(self._xy) * self.n_samples
        if samples is not None:
            p = (Params * len(samples))(*[params_struct(q) for q in samples])
        else:
            p = params_struct(params)
        p0 = p[0] if samples is not None else p
        self._bf = None
        if beta_field is not None:
            self._bf = np.ascontiguousarray(beta_field, dtype=np.float64)
            _arr(self._bf, len(self._xy), "float64", "beta_field")
            p0.beta_field = self._bf.ctypes.data_as(_dp)
        o = options if options is not None else default_options()
        for k, v in opt_over.items():
            setattr(o, k, v)
        self._owner = None
        if owner is not None:
            self._owner = np.ascontiguousarray(owner, dtype=np.int32)
            _arr(self._owner, len(self._xy), "int32", "owner")
            o.owner = self._owner.ctypes.data_as(_ip)
        if stream is not None:
            o.stream = _stream_handle(stream)
        self.options = o
        h = _vp()
        if samples is not None:
            rc = _create_ensemble(C.byref(mesh), len(samples), p, C.byref(o), C.byref(h))
        else:
            rc = _create(C.byref(mesh), C.byref(p), C.byref(o), C.byref(h))
        if rc != OK:
            raise SeirdError(rc, _last_error(None).decode())
        self._h = h

    # -- lifetime
    def close(self):
        if getattr(self, "_h", None):
            _destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _check(self, rc):
        if rc != OK:
            raise SeirdError(rc, _last_error(self._h).decode())

    # -- state
    def set_state(self, u, t=0.0):
        p, dev = _arr(u, 5 * self.n, "float64", "u")
        self._check(_set_state(self._h, p, dev, float(t)))

    def get_state(self, out=None):
        if out is None:
            out = np.empty((self.n, 5))
        p, dev = _arr(out, 5 * self.n, "float64", "out")
        t = C.c_double()
        self._check(_get_state(self._h, p, dev, C.byref(t)))
        self.t = t.value
        return out

    def step(self):
        st = Stats()
        self._check(_step(self._h, C.byref(st)))
        return st.as_dict()

    def run(self, n_steps):
        arr = (Stats * max(1, n_steps))()
        self._check(_run(self._h, int(n_steps), arr))
        return [arr[k].as_dict() for k in range(n_steps)]

    def set_params(self, params, beta_field=None):
        p = params_struct(params)
        if beta_field is not None:
            self._bf = np.ascontiguousarray(beta_field, dtype=np.float64)
            _arr(self._bf, self.n, "float64", "beta_field")
            p.beta_field = self._bf.ctypes.data_as(_dp)
        self._check(_set_params(self._h, C.byref(p)))

    def set_beta_schedule(self, sched):
        """Turns the sigmoid schedule on (a dict with the BetaSchedule fields) or off (None)."""
        if sched is None:
            self._check(_set_beta_schedule(self._h, None))
        else:
            s = BetaSchedule(**{k: float(v) for k, v in sched.items()})
            self._check(_set_beta_schedule(self._h, C.byref(s)))

    def adjoint(self, n_steps, obs_nodes, obs_steps, I_hat, D_hat, checkpoint_every=1, lin_rtol=0.0,
                field=True):
        """(misfit, gradient over PARAM_NAMES [10] (ensembles: [n_samples, 10]),
        gradient over the per-node transmission field [n] or None) by the discrete
        adjoint, from the current state; the state is left unchanged."""
        nodes = np.ascontiguousarray(obs_nodes, dtype=np.int32)
        steps = np.ascontiguousarray(obs_steps, dtype=np.int32)
        Ih = np.ascontiguousarray(I_hat, dtype=np.float64)
        Dh = np.ascontiguousarray(D_hat, dtype=np.float64)
        _arr(Ih, len(steps) * len(nodes), "float64", "I_hat")
        _arr(Dh, len(steps) * len(nodes), "float64", "D_hat")
        spec = Misfit(int(n_steps), int(checkpoint_every), len(nodes), nodes.ctypes.data_as(_ip), len(steps),
                      steps.ctypes.data_as(_ip), Ih.ctypes.data_as(_dp), Dh.ctypes.data_as(_dp), float(lin_rtol))
        j = C.c_double()
        g = np.zeros(10 * self.n_samples)
        gf = np.zeros(self.n) if field else None
        self._check(_adjoint(self._h, C.byref(spec), C.byref(j), g.ctypes.data,
                             None if gf is None else gf.ctypes.data))
        return j.value, (g if self.n_samples == 1 else g.reshape(self.n_samples, 10)), gf

    def set_launch_shapes(self, spmv_threads=0, cgs_ctas=0, cgs_tile=0, ilu_batch=0, ilu_warps=0, ilu_ring=0):
        """Pins launch shapes (seird_set_launch_shapes); 0 keeps a shape as it is."""
        self._check(_set_launch_shapes(self._h, int(spmv_threads), int(cgs_ctas), int(cgs_tile), int(ilu_batch),
                                       int(ilu_warps), int(ilu_ring)))

    def set_wait_limit(self, polls):
        """Polls of each bounded wait in the subdomain solves (seird_set_wait_limit):
        0 restores the default, a negative value makes every wait give up at once."""
        self._check(_set_wait_limit(self._h, int(polls)))

    def info(self):
        inf = Info()
        self._check(_get_info(self._h, C.byref(inf)))
        return inf.as_dict()

    # -- components
    def residual(self, u, u_prev, out=None):
        if out is None:
            out = np.empty((self.n, 5)) if isinstance(u, np.ndarray) else u.new_empty(u.shape)
        a, d0 = _arr(u, 5 * self.n, "float64", "u")
        b, d1 = _arr(u_prev, 5 * self.n, "float64", "u_prev")
        c, d2 = _arr(out, 5 * self.n, "float64", "out")
        dev = _same_place((d0, d1, d2), ("u", "u_prev", "out"))
        self._check(_eval_residual(self._h, a, b, c, dev))
        return out

    def jacobian(self, u):
        a, dev = _arr(u, 5 * self.n, "float64", "u")
        self._check(_eval_jacobian(self._h, a, dev))

    def get_jacobian(self):
        nnzb = self.info()["nnzb"]
        rp = np.empty(self.n + 1, dtype=np.int32)
        col = np.empty(nnzb, dtype=np.int32)
        val = np.empty((nnzb, 5, 5))
        self._check(_get_jacobian(self._h, rp.ctypes.data, col.ctypes.data, val.ctypes.data))
        return rp, col, val

    def apply_jacobian(self, x, out=None):
        if out is None:
            out = np.empty_like(x) if isinstance(x, np.ndarray) else x.new_empty(x.shape)
        a, d0 = _arr(x, 5 * self.n, "float64", "x")
        b, d1 = _arr(out, 5 * self.n, "float64", "out")
        dev = _same_place((d0, d1), ("x", "out"))
        self._check(_apply_jacobian(self._h, a, b, dev))
        return out

    def precond_setup(self):
        self._check(_precond_setup(self._h))

    def precond_apply(self, r, out=None):
        if out is None:
            out = np.empty_like(r) if isinstance(r, np.ndarray) else r.new_empty(r.shape)
        a, d0 = _arr(r, 5 * self.n, "float64", "r")
        b, d1 = _arr(out, 5 * self.n, "float64", "out")
        dev = _same_place((d0, d1), ("r", "out"))
        self._check(_precond_apply(self._h, a, b, dev))
        return out

    def linear_solve(self, b, out=None):
        if out is None:
            out = np.empty_like(b) if isinstance(b, np.ndarray) else b.new_empty(b.shape)
        a, d0 = _arr(b, 5 * self.n, "float64", "b")
        c, d1 = _arr(out, 5 * self.n, "float64", "out")
        dev = _same_place((d0, d1), ("b", "out"))
        its = C.c_int32()
        self._check(_linear_solve(self._h, a, c, dev, C.byref(its)))
        return out, its.value


def declared_functions(header_path=None):
    """Names of the functions declared in include/seird.h."""
    import re
    header_path = header_path or os.path.join(_HERE, "..", "include", "seird.h")
    txt = open(header_path).read()
    return sorted(set(re.findall(r"\b(seird_[a-z0-9_]+)\s*\(", txt)))
