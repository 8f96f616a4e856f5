"""ctypes binding of libthermo.so (argument marshalling only).

Every numerical step runs in the CUDA library; this module only converts
numpy arrays / torch CUDA tensors into pointers and status codes into
exceptions. The library must have been built (python -m
paper_1902_00095_gb300.build); importing fails loudly otherwise.
"""
import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libthermo.so")

TP_OK, TP_EINVAL, TP_ENOMEM, TP_ECUDA, TP_ENONFINITE, TP_SETUP_FAILED, TP_ESTATE = 0, -1, -2, -3, -4, -5, -6
TP_NOT_CONVERGED, TP_BREAKDOWN = 1, 2

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)
_sp = C.POINTER(C.c_byte)


class Grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double), ("g", C.c_double)]


class Fluid(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("rho0", "c", "beta", "p0", "T0", "mu0", "T_mu0",
                                          "mu_coef", "cv", "rho_r", "cr", "kTf")] + [
        ("kT_mix", C.c_int), ("mu_law", C.c_int), ("api", C.c_double)]


class Well(C.Structure):
    _fields_ = [("i", C.c_int), ("j", C.c_int), ("k0", C.c_int), ("k1", C.c_int), ("kind", C.c_int),
                ("value", C.c_double), ("T_inj", C.c_double), ("U", C.c_double)]


class PrecondOpts(C.Structure):
    _fields_ = [("schur", C.c_int), ("variant", C.c_int), ("precision", C.c_int),
                ("interp", C.c_int), ("smoother", C.c_int), ("nu_pre", C.c_int),
                ("nu_post", C.c_int), ("cheb_degree", C.c_int), ("theta", C.c_double),
                ("max_levels", C.c_int), ("coarse_size", C.c_int), ("seed", C.c_ulonglong),
                ("use_graphs", C.c_int), ("interp_S", C.c_int), ("max_levels_S", C.c_int),
                ("nu_S", C.c_int), ("pmax", C.c_int), ("smoother_S", C.c_int),
                ("tail_rows", C.c_int), ("nu_line", C.c_int),
                ("sell_rows", C.c_int)]


class SolveInfo(C.Structure):
    _fields_ = [("iters", C.c_int), ("restarts", C.c_int), ("status", C.c_int),
                ("levels_pp", C.c_int), ("levels_S", C.c_int), ("rel_res", C.c_double),
                ("rel_res_unscaled", C.c_double), ("rel_res_p", C.c_double),
                ("rel_res_T", C.c_double), ("opc_pp", C.c_double), ("opc_S", C.c_double),
                ("t_solve_ms", C.c_double)]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


class NewtonOpts(C.Structure):
    _fields_ = [("max_newton", C.c_int), ("tol_f", C.c_double), ("tol_dx", C.c_double),
                ("rtol", C.c_double), ("maxit", C.c_int), ("restart", C.c_int), ("reuse", C.c_int),
                ("line_search", C.c_int)]


class NewtonInfo(C.Structure):
    _fields_ = [("newton_iters", C.c_int), ("linear_iters", C.c_int), ("status", C.c_int),
                ("last_linear_status", C.c_int), ("rel_f", C.c_double), ("rel_dx", C.c_double),
                ("t_ms", C.c_double), ("line_search_halvings", C.c_int)]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


# name -> (restype, argtypes)
SIGNATURES = {
    "tp_default_opts": (None, [C.POINTER(PrecondOpts)]),
    "tp_status_string": (C.c_char_p, [C.c_int]),
    "tp_last_error": (C.c_char_p, []),
    "tp_kernel_launches": (C.c_longlong, []),
    "tp_create": (C.c_int, [C.POINTER(C.c_void_p), C.POINTER(Grid), C.POINTER(Fluid), C.c_void_p]),
    "tp_destroy": (None, [C.c_void_p]),
    "tp_get_sizes": (C.c_int, [C.c_void_p, _ip, _ip]),
    "tp_set_fields": (C.c_int, [C.c_void_p] + [C.c_void_p] * 5 + [C.c_int]),
    "tp_set_wells": (C.c_int, [C.c_void_p, C.POINTER(Well), C.c_int]),
    "tp_assemble": (C.c_int, [C.c_void_p] + [C.c_void_p] * 4 + [C.c_double] + [C.c_void_p] * 2 + [C.c_int]),
    "tp_build_preconditioner": (C.c_int, [C.c_void_p, C.POINTER(PrecondOpts)]),
    "tp_solve": (C.c_int, [C.c_void_p] + [C.c_void_p] * 4 + [C.c_double, C.c_int, C.c_int,
                                                             C.POINTER(SolveInfo), C.c_int]),
    "tp_spmv": (C.c_int, [C.c_void_p] + [C.c_void_p] * 4 + [C.c_int]),
    "tp_newton_step": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.c_void_p,
                                 C.c_void_p, C.POINTER(PrecondOpts), C.POINTER(NewtonOpts),
                                 C.POINTER(NewtonInfo), C.c_int]),
    "tp_probe_enable": (C.c_int, [C.c_void_p, C.c_int]),
    "tp_probe_read": (C.c_int, [C.c_void_p, _dp, C.POINTER(C.c_longlong), _dp, C.c_int]),
    "tp_apply_preconditioner": (C.c_int, [C.c_void_p] + [C.c_void_p] * 4 + [C.c_int]),
    "tp_export_system": (C.c_int, [C.c_void_p, _ip, _ip, _dp, _dp, _dp]),
    "tp_hierarchy_info": (C.c_int, [C.c_void_p, C.c_int, _ip, _ip, _ip, C.c_int]),
    "tp_vcycle_measure": (C.c_int, [C.c_void_p, C.c_int, C.c_int, _dp, _dp, _dp]),
    "tp_setup_timings": (C.c_int, [C.c_void_p, C.c_int, _dp]),
    "tp_export_level": (C.c_int, [C.c_void_p, C.c_int, C.c_int, _ip, _ip, _dp, _sp, _sp, _ip,
                                  _ip, _ip, _dp]),
    "tp_amg_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_int, C.c_void_p, C.c_void_p,
                                C.c_void_p, C.POINTER(PrecondOpts), C.c_void_p, C.c_int]),
    "tp_amg_destroy": (None, [C.c_void_p]),
    "tp_mlp_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_void_p, C.c_void_p]),
    "tp_mlp_destroy": (None, [C.c_void_p]),
    "tp_mlp_set_params": (C.c_int, [C.c_void_p, C.c_void_p]),
    "tp_mlp_get_params": (C.c_int, [C.c_void_p, C.c_void_p]),
    "tp_mlp_forward": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_int]),
    "tp_mlp_gradient": (C.c_int, [C.c_void_p, C.c_int] + [C.c_void_p] * 7 + [C.c_int]),
    "tp_mlp_train_step": (C.c_int, [C.c_void_p, C.c_int] + [C.c_void_p] * 5 +
                          [C.c_double, C.c_void_p, C.c_int]),
    "tp_learned_features": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    "tp_set_schur_model": (C.c_int, [C.c_void_p, C.c_void_p]),
    "tp_learned_status": (C.c_int, [C.c_void_p, _ip, _ip]),
    "tp_probe_schur_columns": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_double,
                                         C.c_void_p, C.c_void_p, _ip]),
    "tp_equation_scales_noalloc": (C.c_int, [C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                                             C.c_void_p, C.c_void_p]),
    "tp_amg_vcycle": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]),
    "tp_amg_info": (C.c_int, [C.c_void_p, _ip, _ip, _ip, C.c_int]),
    "tp_amg_level_storage": (C.c_int, [C.c_void_p, C.c_int, _ip, C.POINTER(C.c_longlong)]),
    "tp_level_storage": (C.c_int, [C.c_void_p, C.c_int, C.c_int, _ip,
                                   C.POINTER(C.c_longlong)]),
    "tp_amg_export_level": (C.c_int, [C.c_void_p, C.c_int, _ip, _ip, _dp, _sp, _sp, _ip, _ip,
                                      _ip, _dp]),
}

_lib = None


def load():
    """The loaded library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -m paper_1902_00095_gb300.build`")
        lib = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


class ThermoError(RuntimeError):
    def __init__(self, status, where):
        lib = load()
        msg = lib.tp_status_string(status).decode()
        detail = lib.tp_last_error().decode()
        super().__init__(f"{where}: {msg} ({status}) {detail}")
        self.status = status


def _check(status, where, warn_ok=False):
    if status < 0 or (status > 0 and not warn_ok):
        raise ThermoError(status, where)
    return status


def _is_torch(a):
    return type(a).__module__.startswith("torch")


def _arg(a, dtype=np.float64):
    """(pointer, is_device, keepalive) for a numpy array or a torch tensor."""
    if a is None:
        return None, None, None
    if _is_torch(a):
        import torch
        want = torch.float64 if dtype == np.float64 else torch.int32
        if a.dtype != want or not a.is_contiguous():
            raise TypeError(f"expected a contiguous {want} tensor")
        return C.c_void_p(a.data_ptr()), 1 if a.is_cuda else 0, a
    arr = np.ascontiguousarray(a, dtype=dtype)
    return C.c_void_p(arr.ctypes.data), 0, arr


def _args(*arrays):
    ptrs, devs, keep = [], set(), []
    for a in arrays:
        p, d, k = _arg(a)
        ptrs.append(p)
        keep.append(k)
        if d is not None:
            devs.add(d)
    if len(devs) > 1:
        raise ValueError("mixing host and device arrays in one call")
    return ptrs, (devs.pop() if devs else 0), keep


def kernel_launches():
    """Kernels launched by the library so far in this process."""
    return int(load().tp_kernel_launches())


def default_opts(**kw):
    o = PrecondOpts()
    load().tp_default_opts(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def fluid_struct(fl):
    return Fluid(**{n: float(fl[n]) for n, _ in Fluid._fields_
                    if n not in ("kT_mix", "mu_law", "api")},
                 kT_mix=int(fl.get("kT_mix", 0)), mu_law=int(fl.get("mu_law", 0)),
                 api=float(fl.get("api", 0.0)))


class Solver:
    """One context of the CUDA solver for a Cartesian grid."""

    def __init__(self, nx, ny, nz, fluid, dx=10.0, dy=10.0, dz=10.0, g=9.81, stream=None):
        lib = load()
        self._lib = lib
        self._h = C.c_void_p()
        grid = Grid(nx, ny, nz, dx, dy, dz, g)
        fl = fluid_struct(fluid)
        _check(lib.tp_create(C.byref(self._h), C.byref(grid), C.byref(fl),
                             C.c_void_p(stream) if stream else None), "tp_create")
        n, nnzb = C.c_int(), C.c_int()
        lib.tp_get_sizes(self._h, C.byref(n), C.byref(nnzb))
        self.N, self.nnzb = n.value, nnzb.value

    @classmethod
    def from_problem(cls, prob, **kw):
        s = cls(prob["nx"], prob["ny"], prob["nz"], prob["fluid"], prob["dx"], prob["dy"],
                prob["dz"], prob["g"], **kw)
        s.set_fields(prob["Kx"], prob["Ky"], prob["Kz"], prob["phi"], prob["kTr"])
        s.set_wells(prob["wells"])
        return s

    def close(self):
        if self._h:
            self._lib.tp_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_fields(self, Kx, Ky, Kz, phi, kTr):
        p, d, keep = _args(Kx, Ky, Kz, phi, kTr)
        _check(self._lib.tp_set_fields(self._h, *p, d), "tp_set_fields")

    def set_wells(self, wells):
        arr = (Well * max(1, len(wells)))()
        for q, w in enumerate(wells):
            arr[q] = Well(int(w["i"]), int(w["j"]), int(w["k0"]), int(w["k1"]), int(w["kind"]),
                          float(w["value"]), float(w.get("T_inj", 0.0)), float(w.get("U", 0.0)))
        _check(self._lib.tp_set_wells(self._h, arr, len(wells)), "tp_set_wells")

    def assemble(self, p_k, T_k, p_n, T_n, dt, R_m=None, R_e=None):
        """Assemble at (p_k, T_k); returns (R_m, R_e) host arrays unless
        output buffers are given."""
        host_out = R_m is None
        if host_out and not _is_torch(p_k):
            R_m, R_e = np.empty(self.N), np.empty(self.N)
        p, d, keep = _args(p_k, T_k, p_n, T_n, R_m, R_e)
        _check(self._lib.tp_assemble(self._h, p[0], p[1], p[2], p[3], float(dt), p[4], p[5], d),
               "tp_assemble")
        return (keep[4], keep[5]) if R_m is not None else None

    def build(self, opts=None, **kw):
        o = opts if opts is not None else default_opts(**kw)
        _check(self._lib.tp_build_preconditioner(self._h, C.byref(o)), "tp_build_preconditioner")

    def solve(self, b_p=None, b_T=None, rtol=1e-8, maxit=300, restart=30, out=None):
        """Solve A x = b (b = -G(x_k) when b is None). Returns (x_p, x_T, info)."""
        info = SolveInfo()
        if out is None:
            like = b_p
            if like is not None and _is_torch(like):
                import torch
                out = (torch.empty_like(like), torch.empty_like(like))
            else:
                out = (np.empty(self.N), np.empty(self.N))
        p, d, keep = _args(b_p, b_T, out[0], out[1])
        st = self._lib.tp_solve(self._h, p[0], p[1], p[2], p[3], float(rtol), int(maxit),
                                int(restart), C.byref(info), d)
        _check(st, "tp_solve", warn_ok=True)
        return keep[2], keep[3], info.as_dict()

    def newton_step(self, p_n, T_n, dt, max_newton=3, tol_f=1e-8, tol_dx=1e-8, rtol=1e-8,
                    maxit=500, restart=30, reuse=True, line_search=True, opts=None, out=None,
                    **kw):
        """One backward-Euler step by Newton's method from (p_n, T_n);
        returns (p, T, info)."""
        o = opts if opts is not None else default_opts(**kw)
        no = NewtonOpts(int(max_newton), float(tol_f), float(tol_dx), float(rtol), int(maxit),
                        int(restart), int(bool(reuse)), int(bool(line_search)))
        if out is None:
            if _is_torch(p_n):
                import torch
                out = (torch.empty_like(p_n), torch.empty_like(p_n))
            else:
                out = (np.empty(self.N), np.empty(self.N))
        info = NewtonInfo()
        p, d, keep = _args(p_n, T_n, out[0], out[1])
        st = self._lib.tp_newton_step(self._h, p[0], p[1], float(dt), p[2], p[3], C.byref(o),
                                      C.byref(no), C.byref(info), d)
        _check(st, "tp_newton_step", warn_ok=True)
        return keep[2], keep[3], info.as_dict()

    def learned_features(self):
        """Features of every cell at the last assemble, float32 [N, 24]."""
        X = np.empty((self.N, 24), np.float32)
        _check(self._lib.tp_learned_features(self._h, C.c_void_p(X.ctypes.data), 0),
               "tp_learned_features")
        return X

    def set_schur_model(self, mlp):
        """Model used by build(schur=1); None detaches."""
        self._model = mlp
        _check(self._lib.tp_set_schur_model(self._h, mlp._h if mlp is not None else None),
               "tp_set_schur_model")

    def learned_status(self):
        rows, glob = C.c_int(), C.c_int()
        _check(self._lib.tp_learned_status(self._h, C.byref(rows), C.byref(glob)),
               "tp_learned_status")
        return rows.value, bool(glob.value)

    def probe_schur_columns(self, cols, rtol=1e-12):
        """Exact Schur columns on the pattern: (entry [n, 7], value [n, 7],
        total FGMRES iterations, status)."""
        cols = np.ascontiguousarray(cols, np.int32)
        entry = np.empty((cols.size, 7), np.int32)
        value = np.empty((cols.size, 7))
        its = C.c_int()
        st = self._lib.tp_probe_schur_columns(self._h, C.c_void_p(cols.ctypes.data), int(cols.size),
                                              float(rtol), C.c_void_p(entry.ctypes.data),
                                              C.c_void_p(value.ctypes.data), C.byref(its))
        _check(st, "tp_probe_schur_columns", warn_ok=True)
        return entry, value, its.value, st

    def probe_enable(self, which):
        """Time every launch of one kernel class (0 finest A_pp sweeps,
        1 finest S~ sweeps or line steps, 2 block SpMV, 3 A_pp level-1
        sweeps, -1 off) during solves; call before build()."""
        _check(self._lib.tp_probe_enable(self._h, int(which)), "tp_probe_enable")

    def probe_read(self, reset=False):
        ms, n, by = C.c_double(), C.c_longlong(), C.c_double()
        _check(self._lib.tp_probe_read(self._h, C.byref(ms), C.byref(n), C.byref(by), int(reset)),
               "tp_probe_read")
        return dict(ms=ms.value, launches=n.value, bytes=by.value)

    def spmv(self, x_p, x_T):
        y = (np.empty(self.N), np.empty(self.N)) if not _is_torch(x_p) else None
        if y is None:
            import torch
            y = (torch.empty_like(x_p), torch.empty_like(x_p))
        p, d, keep = _args(x_p, x_T, y[0], y[1])
        _check(self._lib.tp_spmv(self._h, *p, d), "tp_spmv")
        return keep[2], keep[3]

    def apply_preconditioner(self, v_p, v_T):
        z = (np.empty(self.N), np.empty(self.N))
        p, d, keep = _args(v_p, v_T, z[0], z[1])
        _check(self._lib.tp_apply_preconditioner(self._h, *p, d), "tp_apply_preconditioner")
        return keep[2], keep[3]

    def export_system(self):
        """Host copies: rowptr, col, val [nnzb, 2, 2], S~ values, scales."""
        rp = np.empty(self.N + 1, np.int32)
        col = np.empty(self.nnzb, np.int32)
        val = np.empty((self.nnzb, 2, 2))
        sv = np.empty(self.nnzb)
        sc = np.empty(2)
        _check(self._lib.tp_export_system(self._h, rp.ctypes.data_as(_ip), col.ctypes.data_as(_ip),
                                          val.ctypes.data_as(_dp), sv.ctypes.data_as(_dp),
                                          sc.ctypes.data_as(_dp)), "tp_export_system")
        return rp, col, val, sv, sc

    def setup_timings(self, which):
        ms = np.empty(5)
        _check(self._lib.tp_setup_timings(self._h, which, ms.ctypes.data_as(_dp)), "tp_setup_timings")
        return dict(zip(("pmis", "interp", "transpose", "galerkin", "finish"), ms.tolist()))

    def hierarchy_info(self, which):
        nl = C.c_int()
        n = np.zeros(64, np.int32)
        nnz = np.zeros(64, np.int32)
        _check(self._lib.tp_hierarchy_info(self._h, which, C.byref(nl), n.ctypes.data_as(_ip),
                                           nnz.ctypes.data_as(_ip), 64), "tp_hierarchy_info")
        return n[:nl.value].copy(), nnz[:nl.value].copy()

    def vcycle_measure(self, which, reps=20):
        """Mean time (ms) of one V-cycle of hierarchy `which` (0 A_pp, 1
        Schur) replayed as a graph, its algorithmic bytes and the operator
        complexity."""
        ms, by, opc = C.c_double(), C.c_double(), C.c_double()
        _check(self._lib.tp_vcycle_measure(self._h, which, reps, C.byref(ms), C.byref(by),
                                           C.byref(opc)), "tp_vcycle_measure")
        return {"ms": ms.value, "bytes": by.value, "opc": opc.value,
                "gbs": by.value / (ms.value * 1e-3) / 1e9 if ms.value > 0 else None}

    def level_storage(self, which, level):
        """(format, stored entries) of a level's operator: format 0 CSR,
        1 ELL, 2 sliced ELL, 3 ELL by grid direction (no column indices)."""
        f, e = C.c_int(), C.c_longlong()
        _check(self._lib.tp_level_storage(self._h, which, level, C.byref(f), C.byref(e)),
               "tp_level_storage")
        return f.value, e.value

    def export_level(self, which, level):
        n, nnz = self.hierarchy_info(which)
        return _export_level(lambda *a: self._lib.tp_export_level(self._h, which, level, *a),
                             int(n[level]), int(nnz[level]))


def _export_level(fn, n, nnz):
    rp = np.empty(n + 1, np.int32)
    col = np.empty(nnz, np.int32)
    val = np.empty(nnz)
    cf = np.empty(n, np.int8)
    strong = np.empty(nnz, np.int8)
    pnnz = C.c_int()
    _check(fn(rp.ctypes.data_as(_ip), col.ctypes.data_as(_ip), val.ctypes.data_as(_dp),
              cf.ctypes.data_as(_sp), strong.ctypes.data_as(_sp), C.byref(pnnz), None, None, None),
           "export_level")
    P = None
    if pnnz.value > 0:
        prp = np.empty(n + 1, np.int32)
        pc = np.empty(pnnz.value, np.int32)
        pv = np.empty(pnnz.value)
        _check(fn(None, None, None, None, None, C.byref(pnnz), prp.ctypes.data_as(_ip),
                  pc.ctypes.data_as(_ip), pv.ctypes.data_as(_dp)), "export_level")
        P = (prp, pc, pv)
    return dict(A=(rp, col, val), cf=cf, strong=strong.astype(bool), P=P)


NPARAM = 6280


class MLP:
    """The per-cell Schur-correction network on the GPU (BF16 tensor cores,
    FP32 master weights, Adam)."""

    def __init__(self, params):
        lib = load()
        self._lib = lib
        self._h = C.c_void_p()
        p = np.ascontiguousarray(params, np.float64)
        if p.size != NPARAM:
            raise ValueError(f"expected {NPARAM} parameters")
        _check(lib.tp_mlp_create(C.byref(self._h), C.c_void_p(p.ctypes.data), None),
               "tp_mlp_create")

    def close(self):
        if self._h:
            self._lib.tp_mlp_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self):
        out = np.empty(NPARAM)
        _check(self._lib.tp_mlp_get_params(self._h, C.c_void_p(out.ctypes.data)), "tp_mlp_get_params")
        return out

    def set_params(self, params):
        p = np.ascontiguousarray(params, np.float64)
        _check(self._lib.tp_mlp_set_params(self._h, C.c_void_p(p.ctypes.data)), "tp_mlp_set_params")

    def forward(self, X):
        X = np.ascontiguousarray(X, np.float32)
        O = np.empty((X.shape[0], 8), np.float32)
        _check(self._lib.tp_mlp_forward(self._h, X.shape[0], C.c_void_p(X.ctypes.data),
                                        C.c_void_p(O.ctypes.data), 0), "tp_mlp_forward")
        return O

    @staticmethod
    def _batch(X, slot, St, Sd, target):
        return (np.ascontiguousarray(X, np.float32), np.ascontiguousarray(slot, np.int32),
                np.ascontiguousarray(St, np.float64), np.ascontiguousarray(Sd, np.float64),
                np.ascontiguousarray(target, np.float64))

    def gradient(self, X, slot, St, Sd, target):
        b = self._batch(X, slot, St, Sd, target)
        g = np.empty(NPARAM)
        loss = C.c_double()
        _check(self._lib.tp_mlp_gradient(self._h, b[0].shape[0], *[C.c_void_p(a.ctypes.data) for a in b],
                                         C.c_void_p(g.ctypes.data), C.byref(loss), 0),
               "tp_mlp_gradient")
        return loss.value, g

    def train_step(self, X, slot, St, Sd, target, lr=1e-3):
        b = self._batch(X, slot, St, Sd, target)
        loss = C.c_double()
        _check(self._lib.tp_mlp_train_step(self._h, b[0].shape[0], *[C.c_void_p(a.ctypes.data) for a in b],
                                           float(lr), C.byref(loss), 0), "tp_mlp_train_step")
        return loss.value


class AMG:
    """Standalone AMG hierarchy of a CSR matrix (structurally symmetric)."""

    def __init__(self, rowptr, col, val, opts=None, **kw):
        lib = load()
        self._lib = lib
        self._h = C.c_void_p()
        rp = np.ascontiguousarray(rowptr, np.int32)
        cc = np.ascontiguousarray(col, np.int32)
        vv = np.ascontiguousarray(val, np.float64)
        self.n = rp.size - 1
        o = opts if opts is not None else default_opts(**kw)
        _check(lib.tp_amg_create(C.byref(self._h), self.n, int(cc.size), C.c_void_p(rp.ctypes.data),
                                 C.c_void_p(cc.ctypes.data), C.c_void_p(vv.ctypes.data), C.byref(o),
                                 None, 0), "tp_amg_create")

    def close(self):
        if self._h:
            self._lib.tp_amg_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def vcycle(self, b):
        x = np.empty(self.n)
        p, d, keep = _args(b, x)
        _check(self._lib.tp_amg_vcycle(self._h, p[0], p[1], d), "tp_amg_vcycle")
        return keep[1]

    def info(self):
        nl = C.c_int()
        n = np.zeros(64, np.int32)
        nnz = np.zeros(64, np.int32)
        _check(self._lib.tp_amg_info(self._h, C.byref(nl), n.ctypes.data_as(_ip),
                                     nnz.ctypes.data_as(_ip), 64), "tp_amg_info")
        return n[:nl.value].copy(), nnz[:nl.value].copy()

    def level_storage(self, level):
        """(format, stored entries) of a level's operator: format 0 CSR,
        1 ELL, 2 sliced ELL, 3 ELL by grid direction (no column indices)."""
        f, e = C.c_int(), C.c_longlong()
        _check(self._lib.tp_amg_level_storage(self._h, level, C.byref(f), C.byref(e)),
               "tp_amg_level_storage")
        return f.value, e.value

    def export_level(self, level):
        n, nnz = self.info()
        return _export_level(lambda *a: self._lib.tp_amg_export_level(self._h, level, *a),
                             int(n[level]), int(nnz[level]))
