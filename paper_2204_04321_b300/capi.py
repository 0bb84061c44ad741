"""Thin ctypes binding of libbp (include/bp.h): the same entry points, argument marshalling only.

Device buffers are torch CUDA tensors (PyTorch supplies device memory and streams); every
computation runs in libbp's kernels.  There is no CPU fallback: if libbp.so is missing or
cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libbp.so")

BP_OK, BP_EINVAL, BP_EMESH, BP_ENOMEM, BP_ECUDA, BP_ENAN, BP_ENOCONV, BP_EUNSUP, BP_ESIZE, BP_EIO = range(10)
BP_NOALLOC_MAX_NDOF = 1048576
BP_F64, BP_F32, BP_F64X2, BP_F32_ALL, BP_F32_DS, BP_F64X2_DS = 0, 1, 2, 3, 4, 5
BP_SCATTER_AUTO, BP_SCATTER_ATOMIC, BP_SCATTER_COLOR = 0, 1, 2
BP_JAC_AUTO, BP_JAC_DUAL, BP_JAC_FACTORED = 0, 1, 2
BP_GUESS_ZERO, BP_GUESS_SIA = 0, 1
BP_KRYLOV_CG, BP_KRYLOV_GMRES = 0, 1
BP_PREC_COLUMN, BP_PREC_MDSC, BP_PREC_MDSC_AMG = 0, 1, 2
BP_JUDGE_RESIDUAL, BP_JUDGE_ENERGY, BP_JUDGE_NONE = 0, 1, 2
BP_LS_OFF, BP_LS_HALVING, BP_LS_QUADRATIC = 0, 1, 2
BP_MARGIN_FREE, BP_MARGIN_OCEAN = 0, 1
BP_MLP_IN, BP_MLP_HIDDEN, BP_MLP_OUT, BP_MLP_OUT_USED, BP_MLP_LEVELS = 16, 128, 32, 22, 11


class BPError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {bp_strerror(status)} (status {status})")
        self.status = status


class bp_params(ctypes.Structure):
    _fields_ = [("n", ctypes.c_double), ("A", ctypes.c_double), ("rho", ctypes.c_double),
                ("g", ctypes.c_double), ("delta", ctypes.c_double), ("rho_w", ctypes.c_double),
                ("margin", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class bp_mesh_desc(ctypes.Structure):
    _fields_ = [("nv", ctypes.c_int32), ("ntri", ctypes.c_int32), ("nlayers", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("xy", ctypes.c_void_p), ("tri", ctypes.c_void_p),
                ("bed", ctypes.c_void_p), ("thick", ctypes.c_void_p), ("beta", ctypes.c_void_p),
                ("sigma", ctypes.c_void_p), ("params", bp_params)]


class bp_mesh_info_t(ctypes.Structure):
    _fields_ = [("ndof", ctypes.c_int64), ("nnz", ctypes.c_int64), ("nwedges", ctypes.c_int64),
                ("nv", ctypes.c_int32), ("ntri", ctypes.c_int32), ("nlayers", ctypes.c_int32),
                ("ncolors", ctypes.c_int32), ("device_bytes", ctypes.c_int64)]


class bp_solve_opts(ctypes.Structure):
    _fields_ = [("rtol", ctypes.c_double), ("max_newton", ctypes.c_int), ("max_krylov", ctypes.c_int),
                ("eta_max", ctypes.c_double), ("precision", ctypes.c_int), ("krylov", ctypes.c_int),
                ("line_search", ctypes.c_int), ("check_every", ctypes.c_int), ("picard_rtol", ctypes.c_double),
                ("value32_rtol", ctypes.c_double), ("device_loop", ctypes.c_int), ("preconditioner", ctypes.c_int),
                ("gmres_restart", ctypes.c_int)]


class bp_solve_report(ctypes.Structure):
    _fields_ = [("newton_iters", ctypes.c_int), ("krylov_iters", ctypes.c_int), ("converged", ctypes.c_int),
                ("value32_steps", ctypes.c_int), ("fnorm_ref", ctypes.c_double), ("fnorm_initial", ctypes.c_double),
                ("fnorm_final", ctypes.c_double), ("history", ctypes.c_double * 65),
                ("krylov_per_newton", ctypes.c_int * 64), ("alpha", ctypes.c_double * 64),
                ("t_total", ctypes.c_double), ("t_assemble", ctypes.c_double), ("t_precond", ctypes.c_double),
                ("t_krylov", ctypes.c_double), ("t_linesearch", ctypes.c_double)]

    def as_dict(self) -> dict:
        k = self.newton_iters
        return {"newton_iters": k, "krylov_iters": self.krylov_iters, "converged": bool(self.converged),
                "value32_steps": self.value32_steps,
                "fnorm_ref": self.fnorm_ref, "fnorm_initial": self.fnorm_initial, "fnorm_final": self.fnorm_final,
                "history": list(self.history[:k + 1]), "krylov_per_newton": list(self.krylov_per_newton[:k]),
                "alpha": list(self.alpha[:k]), "t_total": self.t_total, "t_assemble": self.t_assemble,
                "t_precond": self.t_precond, "t_krylov": self.t_krylov, "t_linesearch": self.t_linesearch}


# (name, restype, argtypes) of every exported entry point
_P = ctypes.c_void_p
_I = ctypes.c_int
SIGNATURES = {
    "bp_version": (ctypes.c_char_p, []),
    "bp_strerror": (ctypes.c_char_p, [_I]),
    "bp_mesh_upload": (_I, [_P, _P, _P]),
    "bp_mesh_free": (None, [_P]),
    "bp_mesh_info": (_I, [_P, _P]),
    "bp_csr_pattern": (_I, [_P, _P, _P]),
    "bp_assemble_residual": (_I, [_P, _P, _P, _P]),
    "bp_assemble_jacobian": (_I, [_P, _P, _P, _P, _I, _I, _I, _P]),
    "bp_assemble_jacobian_noalloc": (_I, [_P, _P, _P, _I, _I, _I, _P]),
    "bp_spmv": (_I, [_P, _P, _I, _P, _P, _P]),
    "bp_spmv_f32": (_I, [_P, _P, _P, _P, _P]),
    "bp_colprec_setup": (_I, [_P, _P, _I, _P]),
    "bp_colprec_apply": (_I, [_P, _P, _P, _P]),
    "bp_mdsc_setup": (_I, [_P, _P, _I, _P]),
    "bp_mdsc_apply": (_I, [_P, _P, _P, _P, _P]),
    "bp_energy": (_I, [_P, _P, _P, _P]),
    "bp_energy_change": (_I, [_P, _P, _P, ctypes.c_double, _P, _P]),
    "bp_energy_change_ex": (_I, [_P, _P, _P, ctypes.c_double, ctypes.c_int, _P, _P]),
    "bp_initial_guess": (_I, [_P, _I, _P, _P]),
    "bp_solve_opts_default": (None, [_P]),
    "bp_newton_solve": (_I, [_P, _P, _P, _P, _P]),
    "bp_ensemble_create": (_I, [_P, _I, _P, _P, _P, _I, _P, _P]),
    "bp_ensemble_tune": (_I, [_P, _I, _P, _P, _P]),
    "bp_ensemble_select": (_I, [_P, _I, _I, _P]),
    "bp_ensemble_assemble": (_I, [_P, _P]),
    "bp_ensemble_free": (None, [_P]),
    "bp_mlp_param_count": (ctypes.c_int64, []),
    "bp_mlp_create": (_I, [ctypes.c_uint64, _P]),
    "bp_mlp_free": (None, [_P]),
    "bp_mlp_get_params": (_I, [_P, _P, ctypes.c_int64, _P]),
    "bp_mlp_set_params": (_I, [_P, _P, ctypes.c_int64, _P]),
    "bp_mlp_forward": (_I, [_P, _P, ctypes.c_int64, _P, _P]),
    "bp_mlp_gradient": (_I, [_P, _P, _P, ctypes.c_int64, _P, _P, _P]),
    "bp_mlp_train_step": (_I, [_P, _P, _P, ctypes.c_int64, ctypes.c_float, _P]),
    "bp_mlp_features": (_I, [_P, _P, _P]),
    "bp_mesh_set_beta": (_I, [_P, _P, _P]),
    "bp_initial_guess_learned": (_I, [_P, _P, _P, _I, _P, _P]),
    "bp_learned_decode": (_I, [_P, _P, _P, _P]),
    "bp_learned_targets": (_I, [_P, _P, ctypes.c_double, _P, _P]),
    "bp_mlp_save": (_I, [_P, ctypes.c_char_p]),
    "bp_measure_fma_peak": (_I, [_I, _P, _P]),
    "bp_mdsc_amg_setup": (_I, [_P, _P, _I, _P]),
    "bp_mdsc_amg_apply": (_I, [_P, _P, _P, _P, _P]),
    "bp_mdsc_amg_levels": (_I, [_P, _P, _I, _P]),
    "bp_mdsc_amg_aggregates": (_I, [_P, _I, _P]),
    "bp_mlp_load": (_I, [_P, ctypes.c_char_p]),
    "bp_mesh_set_rate_factor": (_I, [_P, _P, _P]),
}

_lock = threading.Lock()
_lib = None


def lib():
    """Load libbp.so (raises if it is missing: there is no fallback path)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"libbp.so not built ({LIB_PATH}); run paper_2204_04321_b300/build.py")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _check(status: int, what: str):
    if status != BP_OK:
        raise BPError(status, what)


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dptr(t):
    return ctypes.c_void_p(t.data_ptr())


def bp_version() -> str:
    return lib().bp_version().decode()


def bp_strerror(status: int) -> str:
    return lib().bp_strerror(status).decode()


def make_desc(mesh):
    """bp_mesh_desc for a `synth.Mesh`; returns (desc, keepalive arrays)."""
    keep = [np.ascontiguousarray(mesh.xy, dtype=np.float64),
            np.ascontiguousarray(mesh.tri, dtype=np.int32),
            np.ascontiguousarray(mesh.bed, dtype=np.float64),
            np.ascontiguousarray(mesh.thick, dtype=np.float64),
            np.ascontiguousarray(mesh.beta, dtype=np.float64),
            np.ascontiguousarray(mesh.sigma, dtype=np.float64)]
    p = mesh.params
    desc = bp_mesh_desc(mesh.nv, mesh.ntri, mesh.nlayers, 0,
                        *[a.ctypes.data for a in keep],
                        bp_params(p.n, p.A, p.rho, p.g, p.delta, p.rho_w, p.margin, 0))
    return desc, keep


def bp_mesh_upload(mesh, stream=None) -> ctypes.c_void_p:
    desc, keep = make_desc(mesh)
    out = ctypes.c_void_p()
    _check(lib().bp_mesh_upload(ctypes.byref(desc), _stream_ptr(stream), ctypes.byref(out)),
           "bp_mesh_upload")
    del keep
    return out


def bp_mesh_free(handle) -> None:
    lib().bp_mesh_free(handle)


def bp_mesh_info(handle) -> dict:
    info = bp_mesh_info_t()
    _check(lib().bp_mesh_info(handle, ctypes.byref(info)), "bp_mesh_info")
    return {f: getattr(info, f) for f, _ in bp_mesh_info_t._fields_}


def bp_csr_pattern(handle):
    """(rowptr_dev, colidx_dev) raw device pointers (borrowed)."""
    rp, ci = ctypes.c_void_p(), ctypes.c_void_p()
    _check(lib().bp_csr_pattern(handle, ctypes.byref(rp), ctypes.byref(ci)), "bp_csr_pattern")
    return rp.value, ci.value


def bp_assemble_residual(handle, U, R, stream=None) -> None:
    _check(lib().bp_assemble_residual(handle, _dptr(U), _dptr(R), _stream_ptr(stream)),
           "bp_assemble_residual")


def bp_assemble_jacobian(handle, U, R, J, precision=BP_F64, scatter=BP_SCATTER_AUTO,
                         method=BP_JAC_AUTO, stream=None) -> None:
    _check(lib().bp_assemble_jacobian(handle, _dptr(U), None if R is None else _dptr(R), _dptr(J),
                                      precision, scatter, method, _stream_ptr(stream)),
           "bp_assemble_jacobian")


def bp_assemble_jacobian_noalloc(handle, U, J, precision=BP_F64, scatter=BP_SCATTER_AUTO,
                                 method=BP_JAC_AUTO, stream=None) -> None:
    _check(lib().bp_assemble_jacobian_noalloc(handle, _dptr(U), _dptr(J), precision, scatter, method,
                                              _stream_ptr(stream)),
           "bp_assemble_jacobian_noalloc")


def bp_spmv(handle, J, x, y, precision=BP_F64, stream=None) -> None:
    _check(lib().bp_spmv(handle, _dptr(J), precision, _dptr(x), _dptr(y), _stream_ptr(stream)), "bp_spmv")


def bp_spmv_f32(handle, J, x, y, stream=None) -> None:
    _check(lib().bp_spmv_f32(handle, _dptr(J), _dptr(x), _dptr(y), _stream_ptr(stream)), "bp_spmv_f32")


def bp_colprec_setup(handle, J, precision=BP_F64, stream=None) -> None:
    _check(lib().bp_colprec_setup(handle, _dptr(J), precision, _stream_ptr(stream)), "bp_colprec_setup")


def bp_colprec_apply(handle, r, z, stream=None) -> None:
    _check(lib().bp_colprec_apply(handle, _dptr(r), _dptr(z), _stream_ptr(stream)), "bp_colprec_apply")


def bp_mdsc_setup(handle, J, precision=BP_F64, stream=None) -> None:
    _check(lib().bp_mdsc_setup(handle, _dptr(J), precision, _stream_ptr(stream)), "bp_mdsc_setup")


def bp_mdsc_apply(handle, J, r, z, stream=None) -> None:
    _check(lib().bp_mdsc_apply(handle, _dptr(J), _dptr(r), _dptr(z), _stream_ptr(stream)), "bp_mdsc_apply")


def bp_mdsc_amg_setup(handle, J, precision=BP_F64, stream=None) -> None:
    _check(lib().bp_mdsc_amg_setup(handle, _dptr(J), precision, _stream_ptr(stream)), "bp_mdsc_amg_setup")


def bp_mdsc_amg_apply(handle, J, r, z, stream=None) -> None:
    _check(lib().bp_mdsc_amg_apply(handle, _dptr(J), _dptr(r), _dptr(z), _stream_ptr(stream)), "bp_mdsc_amg_apply")


def bp_mdsc_amg_levels(handle):
    """Vertex counts of the SA-AMG plane levels (after bp_mdsc_amg_setup)."""
    n = ctypes.c_int()
    sizes = np.zeros(16, dtype=np.int32)
    _check(lib().bp_mdsc_amg_levels(handle, sizes.ctypes.data_as(ctypes.c_void_p), 16, ctypes.byref(n)),
           "bp_mdsc_amg_levels")
    return [int(x) for x in sizes[:n.value]]


def bp_mdsc_amg_aggregates(handle, level, n):
    """Aggregate index of each of the n vertices of plane level `level`."""
    out = np.empty(n, dtype=np.int32)
    _check(lib().bp_mdsc_amg_aggregates(handle, level, out.ctypes.data_as(ctypes.c_void_p)),
           "bp_mdsc_amg_aggregates")
    return out


def bp_energy(handle, U, stream=None) -> float:
    out = ctypes.c_double()
    _check(lib().bp_energy(handle, _dptr(U), ctypes.byref(out), _stream_ptr(stream)), "bp_energy")
    return out.value


def bp_energy_change(handle, U, D, alpha, stream=None) -> float:
    out = ctypes.c_double()
    _check(lib().bp_energy_change(handle, _dptr(U), _dptr(D), alpha, ctypes.byref(out), _stream_ptr(stream)),
           "bp_energy_change")
    return out.value


def bp_energy_change_ex(handle, U, D, alpha, precision, stream=None) -> float:
    out = ctypes.c_double()
    _check(lib().bp_energy_change_ex(handle, _dptr(U), _dptr(D), alpha, precision, ctypes.byref(out),
                                     _stream_ptr(stream)), "bp_energy_change_ex")
    return out.value


def bp_initial_guess(handle, kind, U, stream=None) -> None:
    _check(lib().bp_initial_guess(handle, kind, _dptr(U), _stream_ptr(stream)), "bp_initial_guess")


def bp_solve_opts_default() -> bp_solve_opts:
    o = bp_solve_opts()
    lib().bp_solve_opts_default(ctypes.byref(o))
    return o


def bp_newton_solve(handle, U, opts=None, stream=None, **kw):
    """Runs the Newton solve in place on U; returns (status, report dict).  BP_ENOCONV is returned,
    not raised, so the caller can read the report."""
    o = opts if opts is not None else bp_solve_opts_default()
    for k, v in kw.items():
        setattr(o, k, v)
    rep = bp_solve_report()
    rc = lib().bp_newton_solve(handle, _dptr(U), ctypes.byref(o), ctypes.byref(rep), _stream_ptr(stream))
    if rc not in (BP_OK, BP_ENOCONV):
        raise BPError(rc, "bp_newton_solve")
    return rc, rep.as_dict()


class Ensemble:
    """Many uploaded meshes with their buffers, assembled together (bp_ensemble_*)."""

    CANDIDATES = [(cpb, sc) for cpb in (32, 64, 128, 256) for sc in (BP_SCATTER_ATOMIC, BP_SCATTER_COLOR)]

    def __init__(self, meshes, U_list, precision=BP_F64, stream=None):
        import torch
        self.dms = [m if isinstance(m, DeviceMesh) else DeviceMesh(m) for m in meshes]
        self.U = [u.contiguous() for u in U_list]
        self.R = [torch.empty(d.ndof, dtype=torch.float64, device=d.device) for d in self.dms]
        jt = torch.float64 if precision == BP_F64 else torch.float32
        self.J = [torch.empty(d.nnz, dtype=jt, device=d.device) for d in self.dms]
        n = len(self.dms)
        arr = lambda xs: (ctypes.c_void_p * n)(*[ctypes.c_void_p(x) for x in xs])
        out = ctypes.c_void_p()
        _check(lib().bp_ensemble_create(arr([d.handle.value for d in self.dms]), n,
                                        arr([u.data_ptr() for u in self.U]), arr([r.data_ptr() for r in self.R]),
                                        arr([j.data_ptr() for j in self.J]), precision, _stream_ptr(stream),
                                        ctypes.byref(out)), "bp_ensemble_create")
        self.handle = out

    def tune(self, reps=3, stream=None):
        times = (ctypes.c_double * 8)()
        chosen = (ctypes.c_int * 2)()
        _check(lib().bp_ensemble_tune(self.handle, reps, _stream_ptr(stream), times, chosen), "bp_ensemble_tune")
        return {f"cpb{c}-{'color' if sc == BP_SCATTER_COLOR else 'atomic'}": times[i]
                for i, (c, sc) in enumerate(self.CANDIDATES)}, (chosen[0], chosen[1])

    def select(self, cpb, scatter, stream=None):
        _check(lib().bp_ensemble_select(self.handle, cpb, scatter, _stream_ptr(stream)), "bp_ensemble_select")

    def assemble(self, stream=None):
        _check(lib().bp_ensemble_assemble(self.handle, _stream_ptr(stream)), "bp_ensemble_assemble")

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            lib().bp_ensemble_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Mlp:
    """Per-column warm-start MLP (bp_mlp_*); X is a torch.bfloat16 [n, 16] CUDA tensor."""

    def __init__(self, seed=0):
        out = ctypes.c_void_p()
        _check(lib().bp_mlp_create(ctypes.c_uint64(seed), ctypes.byref(out)), "bp_mlp_create")
        self.handle = out
        self.nparam = lib().bp_mlp_param_count()

    def get_params(self):
        p = np.empty(self.nparam, dtype=np.float32)
        _check(lib().bp_mlp_get_params(self.handle, p.ctypes.data_as(ctypes.c_void_p), self.nparam, None),
               "bp_mlp_get_params")
        return p

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        _check(lib().bp_mlp_set_params(self.handle, p.ctypes.data_as(ctypes.c_void_p), self.nparam, None),
               "bp_mlp_set_params")

    def forward(self, X, Y=None, stream=None):
        import torch
        if Y is None:
            Y = torch.empty(X.shape[0], 32, dtype=torch.float32, device=X.device)
        _check(lib().bp_mlp_forward(self.handle, _dptr(X), X.shape[0], _dptr(Y), _stream_ptr(stream)),
               "bp_mlp_forward")
        return Y

    def gradient(self, X, T, stream=None):
        import torch
        g = torch.empty(self.nparam, dtype=torch.float32, device=X.device)
        loss = ctypes.c_double()
        _check(lib().bp_mlp_gradient(self.handle, _dptr(X), _dptr(T), X.shape[0], _dptr(g), ctypes.byref(loss),
                                     _stream_ptr(stream)), "bp_mlp_gradient")
        return loss.value, g

    def train_step(self, X, T, lr, stream=None):
        _check(lib().bp_mlp_train_step(self.handle, _dptr(X), _dptr(T), X.shape[0], ctypes.c_float(lr),
                                       _stream_ptr(stream)), "bp_mlp_train_step")

    def save(self, path):
        """Writes the parameters as a .npy file (bp_mlp_save)."""
        _check(lib().bp_mlp_save(self.handle, os.fsencode(path)), "bp_mlp_save")

    def load(self, path):
        """Reads parameters written by save() or numpy.save (bp_mlp_load)."""
        _check(lib().bp_mlp_load(self.handle, os.fsencode(path)), "bp_mlp_load")

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            lib().bp_mlp_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def bp_mlp_features(handle, X, stream=None) -> None:
    _check(lib().bp_mlp_features(handle, _dptr(X), _stream_ptr(stream)), "bp_mlp_features")


def bp_mesh_set_rate_factor(handle, A, stream=None) -> None:
    """Nodal rate factor A [nv * (L + 1)] (host array, node order a (L + 1) + l), or None for the
    uniform A of the upload."""
    if A is None:
        _check(lib().bp_mesh_set_rate_factor(handle, None, _stream_ptr(stream)), "bp_mesh_set_rate_factor")
        return
    a = np.ascontiguousarray(A, dtype=np.float64)
    _check(lib().bp_mesh_set_rate_factor(handle, a.ctypes.data_as(ctypes.c_void_p), _stream_ptr(stream)),
           "bp_mesh_set_rate_factor")


def bp_mesh_set_beta(handle, beta, stream=None) -> None:
    b = np.ascontiguousarray(beta, dtype=np.float64)
    _check(lib().bp_mesh_set_beta(handle, b.ctypes.data_as(ctypes.c_void_p), _stream_ptr(stream)),
           "bp_mesh_set_beta")


def bp_measure_fma_peak(precision, stream=None) -> float:
    """Measured FP64 (BP_F64) or FP32 (BP_F32) FMA throughput of the current device, TFLOP/s."""
    out = ctypes.c_double()
    _check(lib().bp_measure_fma_peak(precision, ctypes.byref(out), _stream_ptr(stream)), "bp_measure_fma_peak")
    return out.value


def bp_learned_decode(handle, Y, U, stream=None) -> None:
    """U = structured decoder of the network outputs Y [nv, 32] (float32) on the shallow-ice guess."""
    _check(lib().bp_learned_decode(handle, _dptr(Y), _dptr(U), _stream_ptr(stream)), "bp_learned_decode")


def bp_learned_targets(handle, U, reg, T, stream=None) -> None:
    """T [nv, 32] (float32) = the decoder's training targets (per-column profile scales) of U."""
    _check(lib().bp_learned_targets(handle, _dptr(U), float(reg), _dptr(T), _stream_ptr(stream)),
           "bp_learned_targets")


def bp_initial_guess_learned(handle, mlp, U, judge=None, stream=None) -> bool:
    used = ctypes.c_int()
    judge = BP_JUDGE_RESIDUAL if judge is None else judge
    _check(lib().bp_initial_guess_learned(handle, mlp.handle, _dptr(U), judge, ctypes.byref(used),
                                          _stream_ptr(stream)), "bp_initial_guess_learned")
    return bool(used.value)


class DeviceMesh:
    """Convenience owner of an uploaded mesh (frees it on close / garbage collection)."""

    def __init__(self, mesh, stream=None):
        import torch
        self.mesh = mesh
        self.handle = bp_mesh_upload(mesh, stream)
        if getattr(mesh, "rate_factor", None) is not None:
            bp_mesh_set_rate_factor(self.handle, mesh.rate_factor, stream)
        self.info = bp_mesh_info(self.handle)
        self.ndof = self.info["ndof"]
        self.nnz = self.info["nnz"]
        self.device = torch.device("cuda", torch.cuda.current_device())

    def pattern(self):
        """rowptr, colidx as torch tensors (copies of the library-owned arrays)."""
        rp, ci = bp_csr_pattern(self.handle)
        return (_borrow(rp, self.ndof + 1, "<i8").clone(), _borrow(ci, self.nnz, "<i4").clone())

    def residual(self, U, R=None, stream=None):
        import torch
        if R is None:
            R = torch.empty(self.ndof, dtype=torch.float64, device=self.device)
        bp_assemble_residual(self.handle, U, R, stream)
        return R

    def jacobian(self, U, precision=BP_F64, scatter=BP_SCATTER_AUTO, method=BP_JAC_AUTO,
                 R=None, J=None, want_residual=True, stream=None):
        import torch
        if J is None:
            J = torch.empty(self.nnz, dtype=torch.float32 if precision in (BP_F32, BP_F32_ALL, BP_F32_DS) else torch.float64,
                            device=self.device)
        if R is None and want_residual:
            R = torch.empty(self.ndof, dtype=torch.float64, device=self.device)
        bp_assemble_jacobian(self.handle, U, R, J, precision, scatter, method, stream)
        return J, R

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            bp_mesh_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _DevArray:
    """Minimal __cuda_array_interface__ wrapper of a borrowed device pointer."""

    def __init__(self, ptr: int, n: int, typestr: str):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr, "data": (ptr, False),
                                         "version": 3, "strides": None}


def _borrow(ptr: int, n: int, typestr: str):
    import torch
    return torch.as_tensor(_DevArray(ptr, n, typestr), device="cuda")
