"""Thin Python binding of libstrm.so (include/strm.h): argument marshalling only.

Every step of the right-hand side and of the RK update runs in the library's CUDA kernels; this
module converts a workload description into the ABI structs, allocates the caller-owned
workspace and state buffers with torch on the current CUDA device, and passes raw pointers and
the current torch stream. It raises if the library has not been built: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
# STRM_LIBRARY=debug selects the bounds-checking build (libstrm_debug.so)
LIB_PATH = os.path.join(HERE, "libstrm_debug.so" if os.environ.get("STRM_LIBRARY") == "debug" else "libstrm.so")

STRM_OK = 0
_STATUS = {-1: "EINVAL", -2: "ECUDA", -3: "ENONFINITE", -4: "ENOMEM", -5: "ETIMEOUT"}
WENO_MODES = {"off": 0, "sensor": 1, "all": 2}
VISC_LAWS = {"power": 0, "sutherland": 1}
PRECISIONS = {"fp64": 0, "mixed": 1}
Y_MAPS = {"uniform": 0, "tanh": 1, "tanh1": 2, "erf": 3, "sinh1": 4}
FACES = {"xmin": 1, "xmax": 2, "ymin": 3, "ymax": 4}
BC_KINDS = {"periodic": 0, "wall": 1, "char": 2, "recycle": 3, "shock": 4, "df": 5}


class DF(ctypes.Structure):
    _fields_ = [("p_ref", ctypes.c_double), ("ny_filter", ctypes.c_int), ("nz_filter", ctypes.c_int),
                ("tau", ctypes.c_double), ("seed", ctypes.c_ulonglong)]


class StrmError(RuntimeError):
    def __init__(self, fn, code, msg):
        super().__init__(f"{fn} -> {_STATUS.get(code, code)}: {msg}")
        self.code = code


class Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("lx", ctypes.c_double), ("ly", ctypes.c_double), ("lz", ctypes.c_double),
                ("y_map", ctypes.c_int), ("beta", ctypes.c_double)]


class Phys(ctypes.Structure):
    _fields_ = [("gamma", ctypes.c_double), ("prandtl", ctypes.c_double),
                ("r_gas", ctypes.c_double), ("visc_law", ctypes.c_int),
                ("mu_ref", ctypes.c_double), ("t_ref", ctypes.c_double),
                ("visc_exp", ctypes.c_double), ("suth_s", ctypes.c_double),
                ("t_wall", ctypes.c_double), ("forcing", ctypes.c_int)]


class Scheme(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int), ("weno_mode", ctypes.c_int),
                ("theta_thr", ctypes.c_double), ("weno_eps", ctypes.c_double),
                ("u0", ctypes.c_double), ("l0", ctypes.c_double),
                ("convective", ctypes.c_int), ("viscous", ctypes.c_int),
                ("precision", ctypes.c_int)]


_lib = None

# every symbol include/strm.h declares, with its ctypes signature
_P = ctypes.POINTER
_vp, _d, _i, _sz = ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_size_t
SIGNATURES = {
    "strm_last_error": ([], ctypes.c_char_p),
    "strm_workspace_bytes": ([_P(Grid), _P(Scheme)], _sz),
    "strm_init_grid": ([_P(_vp), _P(Grid), _P(Phys), _P(Scheme), _vp, _sz, _vp], _i),
    "strm_set_bc": ([_vp, _i, _i, _vp, _i], _i),
    "strm_compute_rhs": ([_vp, _vp, _vp], _i),
    "strm_rk_step": ([_vp, _vp, _vp, _d, _d], _i),
    "strm_advance_n": ([_vp, _vp, _vp, _i, _d, _d], _i),
    "strm_advance_n_host": ([_vp, _vp, _vp, _vp, _i, _d, _d], _i),
    "strm_conserved_totals": ([_vp, _vp, _P(_d)], _i),
    "strm_get_time": ([_vp, _P(_d), _P(_d)], _i),
    "strm_set_time": ([_vp, _d], _i),
    "strm_sensor": ([_vp, _vp, _vp, _vp, _vp, _vp, _vp], _i),
    "strm_weno_counts": ([_vp, _P(ctypes.c_longlong)], _i),
    "strm_inflow_df_bytes": ([_vp, _P(DF)], _sz),
    "strm_set_inflow_df": ([_vp, _P(DF), _P(_d), _vp, _sz], _i),
    "strm_set_overlap": ([_vp, _i], _i),
    "strm_set_theta": ([_vp, _vp], _i),
    "strm_debug_build": ([], _i),
    "strm_debug_flags": ([_vp, _P(ctypes.c_uint)], _i),
    "strm_stats_bytes": ([_vp, _i], _sz),
    "strm_stats_bind": ([_vp, _i, _vp, _sz], _i),
    "strm_stats_sample": ([_vp, _vp], _i),
    "strm_stats_every": ([_vp, _i], _i),
    "strm_stats_read": ([_vp, _P(_d), _P(ctypes.c_longlong)], _i),
    "strm_kernel_name": ([_i], ctypes.c_char_p),
    "strm_timing": ([_vp, _i], _i),
    "strm_timing_read": ([_vp, _P(_d), _P(ctypes.c_longlong), _P(ctypes.c_longlong)], _i),
    "strm_launch_count": ([_vp, _P(ctypes.c_longlong)], _i),
    "strm_conserved_totals_static": ([_P(Grid), _vp, _P(_d), _vp], _i),
    "strm_peak_fma": ([_i, _i, _vp, _P(_d), _P(_d)], _i),
    "strm_convert_f64_f32": ([_vp, _vp, ctypes.c_longlong, _vp], _i),
    "strm_convert_f32_f64": ([_vp, _vp, ctypes.c_longlong, _vp], _i),
    "strm_ensemble_workspace_bytes": ([_i, _P(Grid), _P(Scheme)], _sz),
    "strm_ensemble_create": ([_P(_vp), _i, _P(Grid), _P(Phys), _P(Scheme), _P(_i), _vp, _sz, _vp], _i),
    "strm_ensemble_set_bc": ([_vp, _i, _i, _i, _vp, _i], _i),
    "strm_ensemble_debug_flags": ([_vp, _P(ctypes.c_uint)], _i),
    "strm_ensemble_inflow_df_bytes": ([_vp, _i, _P(DF)], _sz),
    "strm_ensemble_set_inflow_df": ([_vp, _i, _P(DF), _P(_d), _vp, _sz], _i),
    "strm_ensemble_advance": ([_vp, _P(_vp), _P(_vp), _i, _d, _d], _i),
    "strm_ensemble_tune": ([_vp, _P(_vp), _P(_vp), _P(_i)], _i),
    "strm_ensemble_set_schedule": ([_vp, _P(_i)], _i),
    "strm_ensemble_set_barrier_limit": ([_vp, _d], _i),
    "strm_ensemble_totals": ([_vp, _P(_vp), _P(_d)], _i),
    "strm_ensemble_times": ([_vp, _P(_d)], _i),
    "strm_ensemble_destroy": ([_vp], None),
    "strm_destroy": ([_vp], None),
}
K_COUNT = 14


def lib():
    """Load libstrm.so (built by ``__graft_entry__.build()``); raise if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} not found: build the CUDA library first "
                               "(python -c 'import __graft_entry__ as g; g.build()')")
        L = ctypes.CDLL(LIB_PATH)
        for name, (args, res) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def _check(fn, rc):
    if rc != STRM_OK:
        raise StrmError(fn, rc, lib().strm_last_error().decode())


def structs(case):
    """ABI structs for a workload (``inputs.Case`` or an object with the same attributes)."""
    beta = getattr(case, "beta", 0.0) or 0.0
    ymap = Y_MAPS[getattr(case, "y_map", "tanh")] if beta > 0 else 0
    g = Grid(case.nx, case.ny, case.nz, case.lx, case.ly, case.lz, ymap, beta)
    p = Phys(case.gamma, case.prandtl, case.r_gas, VISC_LAWS[getattr(case, "visc_law", "power")],
             case.mu_ref, getattr(case, "t_ref", 1.0), getattr(case, "visc_exp", 0.76),
             getattr(case, "suth_s", 0.0), getattr(case, "t_wall", 1.0),
             int(bool(getattr(case, "forcing", False))))
    wm = getattr(case, "weno_mode", "sensor")
    s = Scheme(getattr(case, "L", 3), WENO_MODES[wm] if isinstance(wm, str) else int(wm),
               getattr(case, "theta_thr", 0.05), getattr(case, "weno_eps", 1e-6),
               getattr(case, "u0", 1.0), getattr(case, "l0", 1.0),
               int(bool(getattr(case, "convective", True))),
               int(bool(getattr(case, "viscous", True))),
               PRECISIONS[getattr(case, "precision", "fp64")])
    return g, p, s


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def face_settings(case):
    """(face, kind, params) calls that give a context the boundary kinds of a workload."""
    ywall = getattr(case, "y_wall", False)
    kinds = {
        "xmin": getattr(case, "bc_xmin", None) or "periodic",
        "xmax": getattr(case, "bc_xmax", None) or "periodic",
        "ymin": getattr(case, "bc_ymin", None) or ("wall" if ywall else "periodic"),
        "ymax": getattr(case, "bc_ymax", None) or ("wall" if ywall else "periodic"),
    }
    ref = list(getattr(case, "ref", None) or (1.0, 0.0, 0.0, 0.0, 1.0))
    out = []
    for face, kind in kinds.items():
        if kind == "df":
            continue  # set with the inflow profiles (Solver.set_inflow_df)
        if kind in ("periodic", "wall"):
            out.append((FACES[face], BC_KINDS[kind], None))
        elif kind == "char" and face == "ymax" and getattr(case, "shock", False):
            out.append((FACES[face], BC_KINDS["shock"], ref + [case.shock_theta, case.shock_ximp]))
        elif kind == "char":
            out.append((FACES[face], BC_KINDS[kind], ref))
        elif kind == "recycle":
            out.append((FACES[face], BC_KINDS[kind], ref + [float(case.i_recycle), case.delta_in]))
        else:
            raise ValueError(f"unknown boundary kind {kind!r}")
    return out


def apply_faces(lib_, ctx, case):
    for face, kind, params in face_settings(case):
        if params is None:
            rc = lib_.strm_set_bc(ctx, face, kind, None, 0)
        else:
            arr = (ctypes.c_double * len(params))(*params)
            rc = lib_.strm_set_bc(ctx, face, kind, arr, len(params))
        _check("strm_set_bc", rc)


def conserved_totals_static(case, w, stream=None):
    """Totals of a device state through the entry point that allocates nothing (no context,
    no workspace); for callers that cannot allocate device memory. ``w`` must be a contiguous
    float64 CUDA tensor of shape [5, nz, ny, nx]; the call runs with w's device current."""
    shape = (5, case.nz, case.ny, case.nx)
    if not (isinstance(w, torch.Tensor) and w.is_cuda and w.dtype == torch.float64
            and w.is_contiguous() and tuple(w.shape) == shape):
        raise ValueError(f"state must be a contiguous float64 CUDA tensor of shape {shape}")
    g, _, _ = structs(case)
    out = (ctypes.c_double * 5)()
    with torch.cuda.device(w.device):
        st = stream if stream is not None else torch.cuda.current_stream(w.device)
        _check("strm_conserved_totals_static",
               lib().strm_conserved_totals_static(ctypes.byref(g), _ptr(w), out,
                                                  ctypes.c_void_p(st.cuda_stream)))
    return list(out)


def peak_fma(precision="fp64", launches=10, device=None):
    """Measured FMA rate of the current GPU in TFLOP/s (FP64 or, with "fp32", FP32) and the best
    launch's milliseconds, on the current torch stream (strm_peak_fma)."""
    dev = torch.device(device if device is not None else "cuda")
    tf, ms = ctypes.c_double(), ctypes.c_double()
    with torch.cuda.device(dev):
        st = ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
        _check("strm_peak_fma", lib().strm_peak_fma(0 if precision == "fp64" else 1, int(launches), st,
                                                    ctypes.byref(tf), ctypes.byref(ms)))
    return tf.value, ms.value


def convert(x):
    """The FP64 <-> FP32 conversions of the mixed-precision kernels, elementwise on a contiguous
    CUDA tensor (float64 -> float32 or float32 -> float64), on the current stream."""
    if not (x.is_cuda and x.is_contiguous() and x.dtype in (torch.float64, torch.float32)):
        raise ValueError("need a contiguous float64 or float32 CUDA tensor")
    st = ctypes.c_void_p(torch.cuda.current_stream(x.device).cuda_stream)
    if x.dtype == torch.float64:
        y = torch.empty(x.shape, dtype=torch.float32, device=x.device)
        _check("strm_convert_f64_f32", lib().strm_convert_f64_f32(_ptr(x), _ptr(y), x.numel(), st))
    else:
        y = torch.empty(x.shape, dtype=torch.float64, device=x.device)
        _check("strm_convert_f32_f64", lib().strm_convert_f32_f64(_ptr(x), _ptr(y), x.numel(), st))
    return y


class Solver:
    """A context of the CUDA library on the current device and torch stream.

    State tensors are float64 CUDA tensors of shape [5, nz, ny, nx] (contiguous).
    """

    def __init__(self, case, device=None, stream=None, inflow=None):
        """`inflow`: the [7, ny] profiles (U, V, T, R11, R12, R22, R33) of a digital-filter
        inflow face, required when case.bc_xmin == "df"."""
        if getattr(case, "bc_xmin", None) == "df" and inflow is None:
            raise ValueError("a digital-filter inflow face needs its profiles (inflow=...)")
        self.case = case
        self.device = torch.device(device if device is not None else "cuda")
        self.g, self.p, self.s = structs(case)
        L = lib()
        nbytes = L.strm_workspace_bytes(ctypes.byref(self.g), ctypes.byref(self.s))
        if nbytes == 0:
            raise StrmError("strm_workspace_bytes", -1, "invalid grid or scheme")
        # torch's caching allocator returns 512-byte aligned blocks
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        ctx = ctypes.c_void_p()
        _check("strm_init_grid", L.strm_init_grid(
            ctypes.byref(ctx), ctypes.byref(self.g), ctypes.byref(self.p), ctypes.byref(self.s),
            _ptr(self.workspace), nbytes, ctypes.c_void_p(self.stream.cuda_stream)))
        self.ctx = ctx
        apply_faces(L, self.ctx, case)
        if getattr(case, "bc_xmin", None) == "df":
            self.set_inflow_df(inflow)

    def set_inflow_df(self, prof):
        """Make the x-min face a digital-filter inflow with the case's filter parameters."""
        c = self.case
        prof = np.ascontiguousarray(prof, dtype=np.float64)
        if prof.shape != (7, c.ny):
            raise ValueError("inflow profiles must be [7, ny]")
        df = DF(c.ref[4], c.df_ny, c.df_nz, c.df_tau, c.df_seed)
        nbytes = lib().strm_inflow_df_bytes(self.ctx, ctypes.byref(df))
        if nbytes == 0:
            raise StrmError("strm_inflow_df_bytes", -1, "invalid inflow parameters")
        self._df_buf = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        _check("strm_set_inflow_df", lib().strm_set_inflow_df(
            self.ctx, ctypes.byref(df), prof.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
            _ptr(self._df_buf), nbytes))

    @property
    def shape(self):
        return (5, self.case.nz, self.case.ny, self.case.nx)

    def _state(self, w):
        if not (w.is_cuda and w.dtype == torch.float64 and w.is_contiguous()
                and tuple(w.shape) == self.shape):
            raise ValueError(f"state must be a contiguous float64 CUDA tensor of shape {self.shape}")
        return w

    def empty(self):
        return torch.empty(self.shape, dtype=torch.float64, device=self.device)

    def compute_rhs(self, w, out=None):
        out = self.empty() if out is None else out
        _check("strm_compute_rhs", lib().strm_compute_rhs(self.ctx, _ptr(self._state(w)),
                                                          _ptr(self._state(out))))
        return out

    def rk_step(self, w, r_old, dt=0.0, cfl=None):
        cfl = self.case.cfl if cfl is None else cfl
        _check("strm_rk_step", lib().strm_rk_step(self.ctx, _ptr(self._state(w)),
                                                  _ptr(self._state(r_old)), dt, cfl))

    def advance_n(self, w, r_old, nsteps, dt=0.0, cfl=None):
        cfl = self.case.cfl if cfl is None else cfl
        _check("strm_advance_n", lib().strm_advance_n(self.ctx, _ptr(self._state(w)),
                                                      _ptr(self._state(r_old)), nsteps, dt, cfl))

    def advance_n_host(self, w_host, w, r_old, nsteps, dt=0.0, cfl=None):
        """Host-buffer path: w_host (CPU float64, ideally pinned) -> device -> n steps -> w_host."""
        cfl = self.case.cfl if cfl is None else cfl
        if (w_host.device.type != "cpu" or w_host.dtype != torch.float64 or not w_host.is_contiguous()
                or w_host.numel() != int(np.prod(self.shape))):
            raise ValueError(f"w_host must be a contiguous CPU float64 tensor of {int(np.prod(self.shape))} elements")
        _check("strm_advance_n_host", lib().strm_advance_n_host(
            self.ctx, _ptr(w_host), _ptr(self._state(w)), _ptr(self._state(r_old)), nsteps, dt, cfl))

    def totals(self, w):
        out = (ctypes.c_double * 5)()
        _check("strm_conserved_totals", lib().strm_conserved_totals(self.ctx, _ptr(self._state(w)), out))
        return list(out)

    def set_overlap(self, mode=3):
        """Concurrency inside a right-hand side (bit-identical results): bit 1 the ghost fill
        beside the inner part of the sensor, bit 2 the x/y/z face stages as concurrent branches;
        True means both, False or 0 the sequential order."""
        mode = 3 if mode is True else int(mode)
        _check("strm_set_overlap", lib().strm_set_overlap(self.ctx, mode))

    def set_theta(self, theta=None):
        """Prescribe the sensor field the hybrid switch reads ([nz, ny, nx] float64 CUDA tensor,
        kept alive here while set), or None to return to the computed sensor."""
        if theta is not None:
            c = self.case
            if not (theta.is_cuda and theta.dtype == torch.float64 and theta.is_contiguous()
                    and tuple(theta.shape) == (c.nz, c.ny, c.nx)):
                raise ValueError("theta must be a contiguous float64 CUDA tensor of shape [nz, ny, nx]")
        self._theta = theta
        _check("strm_set_theta", lib().strm_set_theta(self.ctx, None if theta is None else _ptr(theta)))

    def time(self):
        t, dt = ctypes.c_double(), ctypes.c_double()
        _check("strm_get_time", lib().strm_get_time(self.ctx, ctypes.byref(t), ctypes.byref(dt)))
        return t.value, dt.value

    def set_time(self, t):
        _check("strm_set_time", lib().strm_set_time(self.ctx, float(t)))

    def sensor(self, w):
        """(theta, div, flags_x, flags_y, flags_z) as CUDA tensors (flag layout of strm.h)."""
        c = self.case
        th = torch.empty((c.nz, c.ny, c.nx), dtype=torch.float64, device=self.device)
        dv = torch.empty_like(th)
        fx = torch.empty((c.nz, c.ny, c.nx + 1), dtype=torch.uint8, device=self.device)
        fy = torch.empty((c.nz, c.ny + 1, c.nx), dtype=torch.uint8, device=self.device)
        fz = torch.empty((c.nz + 1, c.ny, c.nx), dtype=torch.uint8, device=self.device)
        _check("strm_sensor", lib().strm_sensor(self.ctx, _ptr(self._state(w)), _ptr(th), _ptr(dv),
                                                _ptr(fx), _ptr(fy), _ptr(fz)))
        return th, dv, fx, fy, fz

    def weno_counts(self):
        out = (ctypes.c_longlong * 3)()
        _check("strm_weno_counts", lib().strm_weno_counts(self.ctx, out))
        return list(out)

    STATS_MODES = {"xz": 0, "z": 1}
    STAT_NAMES = ["rho", "u", "v", "w", "p", "T", "rho_u", "rho_v", "rho_w", "rho_T", "rho_uu",
                  "rho_vv", "rho_ww", "rho_uv", "rho_uw", "rho_vw", "uu", "vv", "ww", "uv", "pp",
                  "TT", "rhorho", "mu"]

    def stats_bind(self, mode="xz", every=0):
        """Allocate and attach a statistics accumulator ("xz": means over x and z per wall-normal
        row; "z": means over z per (x, y) column) and sample after every `every`-th step."""
        m = self.STATS_MODES[mode]
        nbytes = lib().strm_stats_bytes(self.ctx, m)
        self._stats_buf = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self._stats_mode = mode
        _check("strm_stats_bind", lib().strm_stats_bind(self.ctx, m, _ptr(self._stats_buf), nbytes))
        _check("strm_stats_every", lib().strm_stats_every(self.ctx, int(every)))

    def stats_sample(self, w):
        _check("strm_stats_sample", lib().strm_stats_sample(self.ctx, _ptr(self._state(w))))

    def stats_read(self):
        """(means [24, ny] or [24, ny, nx] as numpy, number of samples)."""
        c = self.case
        shape = (len(self.STAT_NAMES), c.ny) if self._stats_mode == "xz" else (len(self.STAT_NAMES), c.ny, c.nx)
        out = np.empty(shape)
        ns = ctypes.c_longlong()
        _check("strm_stats_read", lib().strm_stats_read(
            self.ctx, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(ns)))
        return out, ns.value

    def debug_flags(self):
        """The bounds-checking build's error word (0: no violation; always 0 in the release
        build)."""
        out = ctypes.c_uint()
        _check("strm_debug_flags", lib().strm_debug_flags(self.ctx, ctypes.byref(out)))
        return out.value

    def timing(self, enable=True):
        _check("strm_timing", lib().strm_timing(self.ctx, int(bool(enable))))

    def timing_read(self):
        """{kernel name: (total ms, launches)} and WENO faces per direction since timing()."""
        ms = (ctypes.c_double * K_COUNT)()
        n = (ctypes.c_longlong * K_COUNT)()
        wf = (ctypes.c_longlong * 3)()
        _check("strm_timing_read", lib().strm_timing_read(self.ctx, ms, n, wf))
        names = [lib().strm_kernel_name(k).decode() for k in range(K_COUNT)]
        return {names[k]: (ms[k], n[k]) for k in range(K_COUNT)}, list(wf)

    def launch_count(self):
        v = ctypes.c_longlong()
        _check("strm_launch_count", lib().strm_launch_count(self.ctx, ctypes.byref(v)))
        return v.value

    def close(self):
        if getattr(self, "ctx", None):
            lib().strm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Ensemble:
    """Many independent grids advanced together by the batched kernels of the library.

    ``cases`` is a list of workload descriptions sharing L and precision: channels and
    boundary layers alike (every face kind of a single context). ``inflows`` maps the index of
    an instance with a digital-filter inflow to its [7, ny] profiles. State tensors are lists of
    float64 CUDA tensors, one [5, nz, ny, nx] tensor per instance.
    """

    def __init__(self, cases, device=None, stream=None, inflows=None):
        self.cases = list(cases)
        n = len(self.cases)
        self.device = torch.device(device if device is not None else "cuda")
        parts = [structs(c) for c in self.cases]
        self.grids = (Grid * n)(*[p[0] for p in parts])
        self.phys = (Phys * n)(*[p[1] for p in parts])
        self.schemes = (Scheme * n)(*[p[2] for p in parts])
        self.bc = (ctypes.c_int * n)(*[1 if getattr(c, "y_wall", False) else 0 for c in self.cases])
        L = lib()
        nbytes = L.strm_ensemble_workspace_bytes(n, self.grids, self.schemes)
        if nbytes == 0:
            raise StrmError("strm_ensemble_workspace_bytes", -1, "invalid grid or scheme")
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        ens = ctypes.c_void_p()
        _check("strm_ensemble_create", L.strm_ensemble_create(
            ctypes.byref(ens), n, self.grids, self.phys, self.schemes, self.bc,
            _ptr(self.workspace), nbytes, ctypes.c_void_p(self.stream.cuda_stream)))
        self.ens = ens
        self._df_bufs = {}
        inflows = inflows or {}
        for e, c in enumerate(self.cases):
            for face, kind, params in face_settings(c):
                arr = (ctypes.c_double * len(params))(*params) if params else None
                _check("strm_ensemble_set_bc", L.strm_ensemble_set_bc(
                    self.ens, e, face, kind, arr, len(params) if params else 0))
            if getattr(c, "bc_xmin", None) == "df":
                if e not in inflows:
                    raise ValueError(f"instance {e} has a digital-filter inflow but no profiles")
                prof = np.ascontiguousarray(inflows[e], dtype=np.float64)
                df = DF(c.ref[4], c.df_ny, c.df_nz, c.df_tau, c.df_seed)
                nb = L.strm_ensemble_inflow_df_bytes(self.ens, e, ctypes.byref(df))
                if nb == 0:
                    raise StrmError("strm_ensemble_inflow_df_bytes", -1, "invalid inflow parameters")
                buf = torch.empty(nb, dtype=torch.uint8, device=self.device)
                self._df_bufs[e] = buf
                _check("strm_ensemble_set_inflow_df", L.strm_ensemble_set_inflow_df(
                    self.ens, e, ctypes.byref(df), prof.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                    _ptr(buf), nb))

    def empty(self):
        return [torch.empty((5, c.nz, c.ny, c.nx), dtype=torch.float64, device=self.device)
                for c in self.cases]

    def _ptrs(self, ts):
        if len(ts) != len(self.cases):
            raise ValueError("one state tensor per instance")
        for t, c in zip(ts, self.cases):
            if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()
                    and tuple(t.shape) == (5, c.nz, c.ny, c.nx)):
                raise ValueError("state tensors must be contiguous float64 CUDA [5, nz, ny, nx]")
        return (ctypes.c_void_p * len(ts))(*[t.data_ptr() for t in ts])

    def advance(self, ws, rs, nsteps, dt=0.0, cfl=0.8):
        _check("strm_ensemble_advance", lib().strm_ensemble_advance(
            self.ens, self._ptrs(ws), self._ptrs(rs), nsteps, dt, cfl))

    def debug_flags(self):
        out = ctypes.c_uint()
        _check("strm_ensemble_debug_flags", lib().strm_ensemble_debug_flags(self.ens, ctypes.byref(out)))
        return out.value

    SCHEDULE = ("weno_block", "weno_per_sm", "central_per_sm", "persistent", "slab_cap")

    def tune(self, ws, rs):
        """Run the autotuner; returns the chosen schedule as a dict (keys SCHEDULE): WENO block
        size, WENO and central-list blocks per SM, persistent stage (1) or one launch per kernel
        type (0), and the slab-height cap of the slab traversal order (0: natural order)."""
        out = (ctypes.c_int * 5)()
        _check("strm_ensemble_tune", lib().strm_ensemble_tune(self.ens, self._ptrs(ws), self._ptrs(rs), out))
        return dict(zip(self.SCHEDULE, list(out)))

    def set_barrier_limit(self, seconds):
        """How long a grid-wide barrier of the persistent stage waits before giving up (0: the
        first block that has to wait gives up, which exercises the failure path)."""
        _check("strm_ensemble_set_barrier_limit", lib().strm_ensemble_set_barrier_limit(self.ens, float(seconds)))

    def set_schedule(self, weno_block=128, weno_per_sm=8, central_per_sm=16, persistent=0, slab_cap=32):
        """Set the schedule the autotuner would choose (see tune)."""
        c = (ctypes.c_int * 5)(weno_block, weno_per_sm, central_per_sm, persistent, slab_cap)
        _check("strm_ensemble_set_schedule", lib().strm_ensemble_set_schedule(self.ens, c))

    def totals(self, ws):
        out = (ctypes.c_double * (5 * len(self.cases)))()
        _check("strm_ensemble_totals", lib().strm_ensemble_totals(self.ens, self._ptrs(ws), out))
        return [list(out[5 * e:5 * e + 5]) for e in range(len(self.cases))]

    def times(self):
        out = (ctypes.c_double * len(self.cases))()
        _check("strm_ensemble_times", lib().strm_ensemble_times(self.ens, out))
        return list(out)

    def close(self):
        if getattr(self, "ens", None):
            lib().strm_ensemble_destroy(self.ens)
            self.ens = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
