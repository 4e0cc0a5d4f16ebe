"""Python binding of libhmg.so (C ABI in include/hmg.h): argument marshalling only.

Every numerical step runs in the CUDA library. PyTorch is used for device memory and the
stream (tensors are passed by data_ptr()). If the library has not been built this module
raises on first use; there is no CPU fallback.

Low-level functions carry the C names (hmg_create, hmg_solve, ...); `Solver` wraps one
context for a mesh hierarchy + coefficients produced by `paper_2210_11797_gb300.inputs`.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

HMG_OK = 0
STATUS_NAMES = {0: "ok", 1: "invalid_arg", 2: "cuda", 3: "not_ready", 4: "not_converged",
                5: "breakdown", 6: "nonfinite", 7: "timeout", 8: "out_of_memory"}
PRECISION = {"fp64": 0, "mixed": 1}
PRECOND = {"none": 0, "linesmooth": 1, "nonnested": 2, "schur": 3}
COARSE = {"vcycle": 0, "learned": 1, "learned_vcycle": 2, "exact": 3, "approx": 4}
KRYLOV = {"bicgstab": 0, "fgmres": 1}
_NAMED = {"precision": PRECISION, "precond": PRECOND, "coarse": COARSE, "krylov": KRYLOV}
MAX_HISTORY = 512
NCOMP = 8
COMPONENTS = ["trace_rhs", "trace_apply", "presmooth", "line_sweep", "residual_restrict",
              "pressure_vcycle", "prolong", "krylov_vectors"]


class HmgError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class MeshLevel(C.Structure):
    _fields_ = [("geometry", C.c_int32), ("ncol", C.c_int32), ("nlev", C.c_int32), ("nedge", C.c_int32),
                ("radius", C.c_double), ("corners", C.c_void_p), ("z_levels", C.c_void_p),
                ("col_edges", C.c_void_p), ("edge_cols", C.c_void_p), ("edge_face", C.c_void_p),
                ("parent", C.c_void_p)]


class Background(C.Structure):
    _fields_ = [("theta_lev", C.c_void_p), ("exner_lev", C.c_void_p), ("exner", C.c_void_p)]


class Scalars(C.Structure):
    _fields_ = [("dt", C.c_double), ("tau_u", C.c_double), ("tau_rho", C.c_double),
                ("tau_theta", C.c_double), ("cp", C.c_double), ("kappa", C.c_double),
                ("preset", C.c_int32), ("sigma", C.c_double), ("omega", C.c_double)]


class Options(C.Structure):
    _fields_ = [("precision", C.c_int32), ("precond", C.c_int32), ("n_pre", C.c_int32),
                ("n_post", C.c_int32), ("n_smooth", C.c_int32), ("omega", C.c_double),
                ("mg_npre", C.c_int32), ("mg_npost", C.c_int32), ("mg_ncoarse", C.c_int32),
                ("mg_omega", C.c_double), ("tol", C.c_double), ("max_iter", C.c_int32),
                ("divergence", C.c_double), ("profile", C.c_int32), ("graph", C.c_int32),
                ("coarse", C.c_int32), ("krylov", C.c_int32), ("restart", C.c_int32),
                ("stall_ratio", C.c_double), ("mg_fused", C.c_int32), ("warm_start", C.c_int32),
                ("mg_fuse_cells", C.c_int32), ("async_stats", C.c_int32), ("degree", C.c_int32)]


class SolveStats(C.Structure):
    _fields_ = [("status", C.c_int32), ("iterations", C.c_int32), ("rel_residual", C.c_double),
                ("true_rel_residual", C.c_double), ("solve_ms", C.c_double), ("n_history", C.c_int32),
                ("history", C.c_double * MAX_HISTORY), ("comp_ms", C.c_double * NCOMP),
                ("comp_calls", C.c_int32 * NCOMP), ("coarse_fallback", C.c_int32)]

    def as_dict(self):
        return {"status": STATUS_NAMES.get(self.status, self.status), "iterations": self.iterations,
                "rel_residual": self.rel_residual, "true_rel_residual": self.true_rel_residual,
                "solve_ms": self.solve_ms, "history": list(self.history[: self.n_history]),
                "coarse_fallback": bool(self.coarse_fallback),
                "components": {n: {"ms": self.comp_ms[i], "launches": self.comp_calls[i]}
                               for i, n in enumerate(COMPONENTS)}}


_LIB = None
_P = C.c_void_p
_SIGS = {
    "hmg_default_options": ([C.POINTER(Options)], C.c_int),
    "hmg_create": ([C.POINTER(_P), C.POINTER(Options), _P], C.c_int),
    "hmg_set_options": ([_P, C.POINTER(Options)], C.c_int),
    "hmg_set_mesh": ([_P, C.c_int32, C.POINTER(MeshLevel)], C.c_int),
    "hmg_set_coefficients": ([_P, C.POINTER(Scalars), C.POINTER(Background)], C.c_int),
    "hmg_assemble_trace": ([_P], C.c_int),
    "hmg_sizes": ([_P, C.POINTER(C.c_int64), C.POINTER(C.c_int64)], C.c_int),
    "hmg_destroy": ([_P], None),
    "hmg_status_string": ([C.c_int], C.c_char_p),
    "hmg_last_error": ([_P], C.c_char_p),
    "hmg_trace_rhs": ([_P, _P, _P, _P], C.c_int),
    "hmg_solve": ([_P, _P, _P, _P, C.POINTER(SolveStats)], C.c_int),
    "hmg_solve_stats_get": ([_P, C.POINTER(SolveStats)], C.c_int),
    "hmg_solve_host": ([_P, _P, _P, _P, C.POINTER(SolveStats)], C.c_int),
    "hmg_reconstruct": ([_P, _P, _P, _P, _P, _P], C.c_int),
    "hmg_apply_trace": ([_P, _P, _P], C.c_int),
    "hmg_precond_apply": ([_P, _P, _P], C.c_int),
    "hmg_line_smooth": ([_P, _P, _P, C.c_int32], C.c_int),
    "hmg_line_smooth_noalloc": ([_P, _P, _P, C.c_int32], C.c_int),
    "hmg_apply_pressure": ([_P, C.c_int32, _P, _P], C.c_int),
    "hmg_pressure_vcycle": ([_P, _P, _P], C.c_int),
    "hmg_get_gamma": ([_P, _P], C.c_int),
    "hmg_get_trace_operator": ([_P, _P], C.c_int),
    "hmg_solve_batched": ([C.POINTER(_P), C.c_int32, C.POINTER(_P), C.POINTER(_P), C.POINTER(_P),
                           C.POINTER(SolveStats)], C.c_int),
    "hmg_autotune": ([_P], C.c_int),
    "hmg_get_launch_shapes": ([_P, _P, _P, C.c_int32], C.c_int),
    "hmg_set_launch_shapes": ([_P, _P, _P, C.c_int32], C.c_int),
    "hmg_solve_mixed": ([_P, _P, _P, _P, _P, C.POINTER(SolveStats)], C.c_int),
    "hmg_apply_mixed": ([_P, _P, _P], C.c_int),
    "hmg_coarse_model_size": ([], C.c_int32),
    "hmg_check_device_wait": ([_P, C.c_int32], C.c_int),
    "hmg_set_coarse_model": ([_P, _P, C.c_int32], C.c_int),
    "hmg_get_coarse_model": ([_P, _P, C.c_int32], C.c_int),
    "hmg_apply_coarse_model": ([_P, _P, _P, C.c_int32], C.c_int),
    "hmg_coarse_model_grad": ([_P, _P, _P, C.c_int32, C.c_int32, C.c_int32, C.c_int32, _P,
                               C.POINTER(C.c_double)], C.c_int),
    "hmg_train_coarse_model": ([_P, _P, _P, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int32,
                                C.c_double, C.c_uint64, _P], C.c_int),
    "hmg_adam_step": ([_P, _P, _P, _P, _P, C.c_int32, C.c_int32, C.c_double, C.c_double, C.c_double,
                       C.c_double], C.c_int),
    "hmg_collect_coarse_pairs": ([_P, _P, _P, _P, C.c_int32, _P, _P, C.POINTER(C.c_int32),
                                  C.POINTER(SolveStats)], C.c_int),
    "hmg_extract_patches": ([_P, _P, _P, C.c_int32, _P, _P, C.c_int32, C.c_int32, _P, _P], C.c_int),
}


def solve_batched(solvers, Rubs, Rpis, lams=None, check=True):
    """n independent solves (one per Solver, each with its own mesh) in one graph launch.
    Returns (list of lambda tensors, list of stats dicts)."""
    n = len(solvers)
    lams = lams or [s._empty(s.ntrace) for s in solvers]
    P = C.c_void_p
    ctxs = (P * n)(*[s.ctx.value for s in solvers])
    rub = (P * n)(*[s._dev(r, 6 * s.ncell, "Rub").value for s, r in zip(solvers, Rubs)])
    rpi = (P * n)(*[s._dev(r, s.ncell, "Rpi").value for s, r in zip(solvers, Rpis)])
    lam = (P * n)(*[s._dev(l, s.ntrace, "lambda").value for s, l in zip(solvers, lams)])
    stats = (SolveStats * n)()
    rc = lib().hmg_solve_batched(ctxs, n, rub, rpi, lam, stats)
    if check:
        _check(solvers[0].ctx, rc)
    return lams, [st.as_dict() for st in stats]


def header_symbols():
    """Names of the functions declared in include/hmg.h."""
    import re
    path = os.path.join(_build.INCLUDE, "hmg.h")
    src = open(path).read()
    return sorted(set(re.findall(r"^\s*(?:int|int32_t|void|const char \*)\s*(hmg_\w+)\s*\(", src, re.M)))


def lib():
    """Load libhmg.so (built in-tree by paper_2210_11797_gb300.build)."""
    global _LIB
    if _LIB is None:
        path = _build.library_path()
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with `python -m paper_2210_11797_gb300.build` "
                               "(there is no CPU fallback)")
        L = C.CDLL(path)
        for name, (args, res) in _SIGS.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _LIB = L
    return _LIB


def _check(ctx, st):
    if st != HMG_OK:
        msg = lib().hmg_last_error(ctx).decode() if ctx else lib().hmg_status_string(st).decode()
        raise HmgError(st, msg)


def _ptr(t):
    return C.c_void_p(t.data_ptr())


def _option_value(k, v):
    return _NAMED[k][v] if k in _NAMED and isinstance(v, str) else v


def default_options(**kw) -> Options:
    o = Options()
    lib().hmg_default_options(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, _option_value(k, v))
    return o


class Solver:
    """One library context: mesh hierarchy, coefficients, assembled operators, workspace."""

    def __init__(self, hier, coeffs, stream=None, **options):
        import torch
        self.torch = torch
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.opts = default_options(**options)
        self.ctx = C.c_void_p()
        _check(None, lib().hmg_create(C.byref(self.ctx), C.byref(self.opts), C.c_void_p(self.stream.cuda_stream)))
        self._keep = []
        self._set_mesh(hier)
        self._set_coefficients(coeffs)
        _check(self.ctx, lib().hmg_assemble_trace(self.ctx))
        self._fp32_built = self.opts.precision == PRECISION["mixed"]   # FP32 operator copies exist
        self._sizes()
        self._keep = []

    def _sizes(self):
        """Cells, trace unknowns and the cell residual dofs of the assembled degree p (velocity:
        3 (p+1)^2 (p+2) = 6, 36, 108, 240; pressure: (p+1)^3 = 1, 8, 27, 64)."""
        nc, nt = C.c_int64(), C.c_int64()
        _check(self.ctx, lib().hmg_sizes(self.ctx, C.byref(nc), C.byref(nt)))
        self.ncell, self.ntrace = nc.value, nt.value
        self.degree = p = self.opts.degree
        self.nu, self.npr = 3 * (p + 1) ** 2 * (p + 2), (p + 1) ** 3

    def _arr(self, a, dtype):
        a = np.ascontiguousarray(a, dtype=dtype)
        self._keep.append(a)
        return a.ctypes.data_as(C.c_void_p)

    def _set_mesh(self, hier):
        levels = (MeshLevel * hier.nmg)()
        for l, m in enumerate(hier.meshes):
            lv = levels[l]
            lv.geometry, lv.ncol, lv.nlev, lv.nedge = m.geometry, m.ncol, m.nlev, m.nedge
            lv.radius = m.radius
            lv.corners = self._arr(m.corners, np.float64)
            lv.z_levels = self._arr(m.z_levels, np.float64)
            lv.col_edges = self._arr(m.col_edges, np.int32)
            lv.edge_cols = self._arr(m.edge_cols, np.int32)
            lv.edge_face = self._arr(m.edge_face, np.int8)
            lv.parent = self._arr(hier.parents[l], np.int32) if l + 1 < hier.nmg else None
        _check(self.ctx, lib().hmg_set_mesh(self.ctx, hier.nmg, levels))
        self.nmg = hier.nmg
        self.ncol, self.nlev = hier.meshes[0].ncol, hier.meshes[0].nlev
        self.level_cells = [m.ncell for m in hier.meshes]

    def _set_coefficients(self, co):
        sc = Scalars(co.dt, co.tau_u, co.tau_rho, co.tau_theta, co.cp, co.kappa, co.preset, co.sigma,
                     getattr(co, "omega", 0.0))
        bgs = (Background * len(co.levels))()
        for l, bg in enumerate(co.levels):
            bgs[l].theta_lev = self._arr(bg.theta_lev, np.float64)
            bgs[l].exner_lev = self._arr(bg.exner_lev, np.float64)
            bgs[l].exner = self._arr(bg.exner, np.float64)
        _check(self.ctx, lib().hmg_set_coefficients(self.ctx, C.byref(sc), bgs))

    # -- helpers --------------------------------------------------------------------------
    def _dev(self, t, n, name):
        torch = self.torch
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
            raise TypeError(f"{name}: expected a contiguous float64 CUDA tensor")
        if t.numel() != n:
            raise ValueError(f"{name}: expected {n} elements, got {t.numel()}")
        return _ptr(t)

    def _empty(self, n):
        return self.torch.empty(n, dtype=self.torch.float64, device=self.device)

    def set_options(self, **kw):
        for k, v in kw.items():
            setattr(self.opts, k, _option_value(k, v))
        # (hmg_set_options makes the FP32 copies of the operators when the precision becomes
        # mixed, and rebuilds them with the factors when a relaxation weight changes)
        _check(self.ctx, lib().hmg_set_options(self.ctx, C.byref(self.opts)))
        if self.opts.precision == PRECISION["mixed"]:
            self._fp32_built = True
        if self.opts.degree != self.degree:       # a new discretisation: assemble it
            _check(self.ctx, lib().hmg_assemble_trace(self.ctx))
            self._sizes()

    # -- the calls ------------------------------------------------------------------------
    def trace_rhs(self, Rub, Rpi):
        B = self._empty(self.ntrace)
        _check(self.ctx, lib().hmg_trace_rhs(self.ctx, self._dev(Rub, self.nu * self.ncell, "Rub"),
                                             self._dev(Rpi, self.npr * self.ncell, "Rpi"), _ptr(B)))
        return B

    def solve(self, Rub, Rpi, lam=None, check=True):
        """(lambda, stats dict). With async_stats = 1 a graph-launched solve is only enqueued:
        stats is None and solve_stats() gives them later."""
        lam = self._empty(self.ntrace) if lam is None else lam
        st = SolveStats()
        rc = lib().hmg_solve(self.ctx, self._dev(Rub, self.nu * self.ncell, "Rub"),
                             self._dev(Rpi, self.npr * self.ncell, "Rpi"),
                             self._dev(lam, self.ntrace, "lambda"), C.byref(st))
        if check:
            _check(self.ctx, rc)
        if rc == HMG_OK and st.status == 3:   # async_stats: enqueued, stats from solve_stats()
            return lam, None
        return lam, st.as_dict()

    def solve_stats(self, check=True):
        """Stats of the last solve enqueued with async_stats = 1 (waits for it)."""
        st = SolveStats()
        rc = lib().hmg_solve_stats_get(self.ctx, C.byref(st))
        if check:
            _check(self.ctx, rc)
        return st.as_dict()

    def solve_mixed(self, Rub, Rpi, check=True):
        """Configuration 1: returns (u [ntrace], Pi [ncell], stats)."""
        u, pi = self._empty(self.ntrace), self._empty(self.ncell)
        st = SolveStats()
        rc = lib().hmg_solve_mixed(self.ctx, self._dev(Rub, 6 * self.ncell, "Rub"), self._dev(Rpi, self.ncell, "Rpi"),
                                   _ptr(u), _ptr(pi), C.byref(st))
        if check:
            _check(self.ctx, rc)
        return u, pi, st.as_dict()

    def apply_mixed(self, x):
        n = self.ntrace + self.ncell
        y = self._empty(n)
        _check(self.ctx, lib().hmg_apply_mixed(self.ctx, self._dev(x, n, "x"), _ptr(y)))
        return y

    def solve_host(self, Rub, Rpi, check=True, out=None):
        """Host buffers in and out; `out` (float64 [ntrace], e.g. a view of pinned memory)
        receives lambda, else a new array."""
        Rub = np.ascontiguousarray(Rub, np.float64)
        Rpi = np.ascontiguousarray(Rpi, np.float64)
        if Rub.size != self.nu * self.ncell or Rpi.size != self.npr * self.ncell:
            raise ValueError("Rub / Rpi size")
        lam = np.empty(self.ntrace) if out is None else out
        if lam.dtype != np.float64 or lam.size != self.ntrace or not lam.flags.c_contiguous:
            raise ValueError("out: contiguous float64 [ntrace]")
        st = SolveStats()
        rc = lib().hmg_solve_host(self.ctx, Rub.ctypes.data_as(C.c_void_p), Rpi.ctypes.data_as(C.c_void_p),
                                  lam.ctypes.data_as(C.c_void_p), C.byref(st))
        if check:
            _check(self.ctx, rc)
        return lam, st.as_dict()

    def assemble(self):
        """Rebuild the operators (cell matrices, S, factors, H per level, Gamma) from the
        coefficients on the device (hmg_assemble_trace)."""
        _check(self.ctx, lib().hmg_assemble_trace(self.ctx))
        self._fp32_built = self.opts.precision == PRECISION["mixed"] or self._fp32_built

    def reconstruct(self, lam, Rub, Rpi):
        ub, pi = self._empty(self.nu * self.ncell), self._empty(self.npr * self.ncell)
        _check(self.ctx, lib().hmg_reconstruct(self.ctx, self._dev(lam, self.ntrace, "lambda"),
                                               self._dev(Rub, self.nu * self.ncell, "Rub"),
                                               self._dev(Rpi, self.npr * self.ncell, "Rpi"), _ptr(ub), _ptr(pi)))
        return ub, pi

    def apply_trace(self, x):
        y = self._empty(self.ntrace)
        _check(self.ctx, lib().hmg_apply_trace(self.ctx, self._dev(x, self.ntrace, "x"), _ptr(y)))
        return y

    def precond(self, r):
        n = self.ntrace + (self.ncell if self.opts.precond == PRECOND["schur"] else 0)
        z = self._empty(n)
        _check(self.ctx, lib().hmg_precond_apply(self.ctx, self._dev(r, n, "r"), _ptr(z)))
        return z

    def line_smooth(self, b, lam, nsweeps):
        _check(self.ctx, lib().hmg_line_smooth(self.ctx, self._dev(b, self.ntrace, "b"),
                                               self._dev(lam, self.ntrace, "lambda"), nsweeps))
        return lam

    def apply_pressure(self, level, x):
        n = self.level_cells[level]
        y = self._empty(n)
        _check(self.ctx, lib().hmg_apply_pressure(self.ctx, level, self._dev(x, n, "x"), _ptr(y)))
        return y

    def vcycle(self, b):
        x = self._empty(self.ncell)
        _check(self.ctx, lib().hmg_pressure_vcycle(self.ctx, self._dev(b, self.ncell, "b"), _ptr(x)))
        return x

    def gamma(self):
        g = self._empty(self.ncell)
        _check(self.ctx, lib().hmg_get_gamma(self.ctx, _ptr(g)))
        return g

    def autotune(self):
        _check(self.ctx, lib().hmg_autotune(self.ctx))

    def launch_shapes(self):
        """((sweep columns, threads), [(smoother columns, threads) per level]); 0 = default."""
        sw = np.zeros(2, np.int32)
        mg = np.zeros(2 * self.nmg, np.int32)
        _check(self.ctx, lib().hmg_get_launch_shapes(self.ctx, sw.ctypes.data_as(C.c_void_p),
                                                     mg.ctypes.data_as(C.c_void_p), self.nmg))
        return (int(sw[0]), int(sw[1])), [(int(mg[2 * l]), int(mg[2 * l + 1])) for l in range(self.nmg)]

    def set_launch_shapes(self, sweep, mg):
        sw = np.asarray(sweep, np.int32).ravel()
        mgs = np.asarray(mg, np.int32).ravel()
        _check(self.ctx, lib().hmg_set_launch_shapes(self.ctx, sw.ctypes.data_as(C.c_void_p),
                                                     mgs.ctypes.data_as(C.c_void_p), self.nmg))

    def trace_operator_slots(self):
        out = self.torch.empty((11, self.ntrace), dtype=self.torch.float64, device=self.device)
        _check(self.ctx, lib().hmg_get_trace_operator(self.ctx, _ptr(out)))
        return out

    # -- learned coarse correction ----------------------------------------------------------
    def _f32(self, t, name):
        torch = self.torch
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
            raise TypeError(f"{name}: expected a contiguous float32 CUDA tensor")
        return _ptr(t)

    def check_device_wait(self, polls=1000):
        """Status of the bounded-wait self-test (expected: 7, HMG_ERR_TIMEOUT)."""
        return lib().hmg_check_device_wait(self.ctx, polls)

    def set_coarse_model(self, params):
        p = np.ascontiguousarray(params, np.float32).ravel()
        _check(self.ctx, lib().hmg_set_coarse_model(self.ctx, p.ctypes.data_as(C.c_void_p), p.size))

    def get_coarse_model(self):
        p = np.empty(lib().hmg_coarse_model_size(), np.float32)
        _check(self.ctx, lib().hmg_get_coarse_model(self.ctx, p.ctypes.data_as(C.c_void_p), p.size))
        return p

    MODEL_MODES = {"tensor": 0, "fp32": 1, "bf16": 2}

    def apply_coarse_model(self, bbar, mode="tensor"):
        """mode: "tensor" (BF16 on the tensor cores, the solver's form), "fp32" or "bf16" (CUDA cores)."""
        out = self._empty(self.ncell)
        _check(self.ctx, lib().hmg_apply_coarse_model(self.ctx, self._dev(bbar, self.ncell, "bbar"), _ptr(out),
                                                      self.MODEL_MODES[mode]))
        return out

    def _patches(self, x, t, nx, ny):
        if x.shape != t.shape or x.ndim != 3 or x.shape[1] != nx * ny:
            raise ValueError("x, t: expected [nsamp, nx*ny, nlev]")
        return self._f32(x, "x"), self._f32(t, "t"), x.shape[0]

    def coarse_model_grad(self, x, t, nx, ny, fp32=False):
        px, pt, ns = self._patches(x, t, nx, ny)
        g = np.empty(lib().hmg_coarse_model_size(), np.float32)
        loss = C.c_double()
        _check(self.ctx, lib().hmg_coarse_model_grad(self.ctx, px, pt, ns, nx, ny, 1 if fp32 else 0,
                                                     g.ctypes.data_as(C.c_void_p), C.byref(loss)))
        return loss.value, g

    def train_coarse_model(self, x, t, nx, ny, batch, epochs, lr, seed=0):
        px, pt, ns = self._patches(x, t, nx, ny)
        hist = np.zeros(max(epochs, 1))
        _check(self.ctx, lib().hmg_train_coarse_model(self.ctx, px, pt, ns, nx, ny, batch, epochs, lr, seed,
                                                      hist.ctypes.data_as(C.c_void_p)))
        return hist[:epochs]

    def adam_step(self, w, g, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
        """One Adam update of the FP32 device tensors w, m, v (in place) with gradient g."""
        n = w.numel()
        for name, t in (("w", w), ("g", g), ("m", m), ("v", v)):
            if t.dtype != self.torch.float32 or not t.is_cuda or not t.is_contiguous() or t.numel() != n:
                raise ValueError(f"{name}: a contiguous CUDA float32 tensor of {n} values is required")
        _check(self.ctx, lib().hmg_adam_step(self.ctx, _ptr(w), _ptr(g), _ptr(m), _ptr(v), n, step, lr, beta1,
                                             beta2, eps))

    def collect_coarse_pairs(self, Rub, Rpi, max_pairs, check=True):
        torch = self.torch
        xs = torch.empty((max_pairs, self.ncell), dtype=torch.float32, device=self.device)
        ts = torch.empty_like(xs)
        lam = self._empty(self.ntrace)
        n = C.c_int32()
        st = SolveStats()
        rc = lib().hmg_collect_coarse_pairs(self.ctx, self._dev(Rub, 6 * self.ncell, "Rub"),
                                            self._dev(Rpi, self.ncell, "Rpi"), _ptr(lam), max_pairs,
                                            _ptr(xs), _ptr(ts), C.byref(n), C.byref(st))
        if check:
            _check(self.ctx, rc)
        return xs[: n.value], ts[: n.value], lam, st.as_dict()

    def extract_patches(self, xs, ts, pair, cols):
        """pair [npatch], cols [npatch, P] (int32 CUDA tensors) -> x, t [npatch, P, nlev]."""
        torch = self.torch
        npatch, P = cols.shape
        xo = torch.empty((npatch, P, self.nlev), dtype=torch.float32, device=self.device)
        to = torch.empty_like(xo)
        for a, nm in ((pair, "pair"), (cols, "cols")):
            if not (a.is_cuda and a.dtype == torch.int32 and a.is_contiguous()):
                raise TypeError(f"{nm}: expected a contiguous int32 CUDA tensor")
        _check(self.ctx, lib().hmg_extract_patches(self.ctx, self._f32(xs, "xs"), self._f32(ts, "ts"), xs.shape[0],
                                                   _ptr(pair), _ptr(cols), npatch, P, _ptr(xo), _ptr(to)))
        return xo, to

    def close(self):
        if self.ctx:
            lib().hmg_destroy(self.ctx)
            self.ctx = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
