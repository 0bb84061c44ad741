"""CPU oracle (TEST INFRASTRUCTURE ONLY).

Plain, slow FP64 statement of the first-order Stokes assembly (paper Sec. 2 and Sec. 3):
the C++ element loop in `bp_oracle.cpp` (residual, dual-number Jacobian, energy, pattern,
shallow-ice guess) plus a plain Newton solver in `newton.py`.  Only `tests/`, the smoke
check and the benchmark's CPU-baseline leg may import this package; the product library
never does.  It shares no code with the CUDA path -- both read the seeded inputs of
`paper_2204_04321_b300.synth` and nothing else.

Parity status of every function is recorded in the module that defines it; all functions
here are pinned by `tests/test_oracle_pins.py` (closed forms, invariants, finite
differences, a closed-form slab profile).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bp_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with plain g++ -O2 (no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-pthread", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


class _OMesh(ctypes.Structure):
    _fields_ = [("nv", ctypes.c_int32), ("ntri", ctypes.c_int32), ("nlayers", ctypes.c_int32),
                ("pad", ctypes.c_int32),
                ("xy", ctypes.c_void_p), ("tri", ctypes.c_void_p), ("bed", ctypes.c_void_p),
                ("thick", ctypes.c_void_p), ("beta", ctypes.c_void_p), ("sigma", ctypes.c_void_p),
                ("n", ctypes.c_double), ("A", ctypes.c_double), ("rho", ctypes.c_double),
                ("g", ctypes.c_double), ("delta", ctypes.c_double), ("rho_w", ctypes.c_double),
                ("margin", ctypes.c_int32), ("pad2", ctypes.c_int32), ("Anode", ctypes.c_void_p)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            P = ctypes.c_void_p
            L.oracle_residual.argtypes = [P, P, P, P]
            L.oracle_jacobian.argtypes = [P, P, P, P, P, P, P]
            L.oracle_jacobian_colored.argtypes = [P, P, P, P, P, P, ctypes.c_int]
            L.oracle_pattern_nnz.argtypes = [P, P]
            L.oracle_pattern.argtypes = [P, P, P]
            L.oracle_energy.argtypes = [P, P]
            L.oracle_energy.restype = ctypes.c_double
            L.oracle_element.argtypes = [P, P, ctypes.c_int, ctypes.c_int, P, P]
            L.oracle_qp_state.argtypes = [P, P, ctypes.c_int, ctypes.c_int, ctypes.c_int, P]
            L.oracle_basis_at.argtypes = [P, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                          P, P, P]
            L.oracle_qp.argtypes = [ctypes.c_int, P, P, P, P]
            L.oracle_sia.argtypes = [P, P]
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


class OracleMesh:
    """Holds contiguous copies of a `synth.Mesh` and the C descriptor pointing at them."""

    def __init__(self, mesh):
        self.mesh = mesh
        self.xy = np.ascontiguousarray(mesh.xy, dtype=np.float64)
        self.tri = np.ascontiguousarray(mesh.tri, dtype=np.int32)
        self.bed = np.ascontiguousarray(mesh.bed, dtype=np.float64)
        self.thick = np.ascontiguousarray(mesh.thick, dtype=np.float64)
        self.beta = np.ascontiguousarray(mesh.beta, dtype=np.float64)
        self.sigma = np.ascontiguousarray(mesh.sigma, dtype=np.float64)
        rf = getattr(mesh, "rate_factor", None)
        self.Anode = None if rf is None else np.ascontiguousarray(rf, dtype=np.float64)
        p = mesh.params
        self.desc = _OMesh(mesh.nv, mesh.ntri, mesh.nlayers, 0, _ptr(self.xy).value,
                           _ptr(self.tri).value, _ptr(self.bed).value, _ptr(self.thick).value,
                           _ptr(self.beta).value, _ptr(self.sigma).value,
                           p.n, p.A, p.rho, p.g, p.delta, p.rho_w, p.margin, 0,
                           None if self.Anode is None else _ptr(self.Anode).value)
        self.ndof = mesh.ndof
        self._pattern = None

    @property
    def dptr(self):
        return ctypes.cast(ctypes.pointer(self.desc), ctypes.c_void_p)

    def residual(self, U: np.ndarray, tri_mask: np.ndarray | None = None) -> np.ndarray:
        U = np.ascontiguousarray(U, dtype=np.float64)
        R = np.empty(self.ndof)
        m = None if tri_mask is None else np.ascontiguousarray(tri_mask, dtype=np.uint8)
        rc = lib().oracle_residual(self.dptr, _ptr(U), None if m is None else _ptr(m), _ptr(R))
        if rc:
            raise RuntimeError(f"oracle_residual failed ({rc})")
        return R

    def pattern(self):
        if self._pattern is None:
            nnz = np.zeros(1, dtype=np.int64)
            if lib().oracle_pattern_nnz(self.dptr, _ptr(nnz)):
                raise RuntimeError("oracle_pattern_nnz failed")
            rowptr = np.empty(self.ndof + 1, dtype=np.int64)
            colidx = np.empty(int(nnz[0]), dtype=np.int32)
            if lib().oracle_pattern(self.dptr, _ptr(rowptr), _ptr(colidx)):
                raise RuntimeError("oracle_pattern failed")
            self._pattern = (rowptr, colidx)
        return self._pattern

    def jacobian(self, U: np.ndarray, tri_mask: np.ndarray | None = None):
        """Returns (rowptr, colidx, vals, R) on the oracle's own (brute-force) pattern."""
        rowptr, colidx = self.pattern()
        U = np.ascontiguousarray(U, dtype=np.float64)
        vals = np.empty(colidx.shape[0])
        R = np.empty(self.ndof)
        m = None if tri_mask is None else np.ascontiguousarray(tri_mask, dtype=np.uint8)
        rc = lib().oracle_jacobian(self.dptr, _ptr(U), None if m is None else _ptr(m),
                                   _ptr(rowptr), _ptr(colidx), _ptr(vals), _ptr(R))
        if rc:
            raise RuntimeError(f"oracle_jacobian failed ({rc})")
        return rowptr, colidx, vals, R

    def jacobian_colored(self, U: np.ndarray, nthreads: int = 1):
        """The same Jacobian and residual, columns taken colour by colour and each colour's columns
        split among `nthreads` threads: bitwise the same for every thread count."""
        rowptr, colidx = self.pattern()
        U = np.ascontiguousarray(U, dtype=np.float64)
        vals = np.empty(colidx.shape[0])
        R = np.empty(self.ndof)
        rc = lib().oracle_jacobian_colored(self.dptr, _ptr(U), _ptr(rowptr), _ptr(colidx), _ptr(vals), _ptr(R),
                                           int(nthreads))
        if rc:
            raise RuntimeError(f"oracle_jacobian_colored failed ({rc})")
        return rowptr, colidx, vals, R

    def jacobian_scipy(self, U: np.ndarray):
        import scipy.sparse as sp
        rowptr, colidx, vals, R = self.jacobian(U)
        return sp.csr_matrix((vals, colidx, rowptr), shape=(self.ndof, self.ndof)), R

    def energy(self, U: np.ndarray) -> float:
        U = np.ascontiguousarray(U, dtype=np.float64)
        return float(lib().oracle_energy(self.dptr, _ptr(U)))

    def element(self, U: np.ndarray, t: int, l: int):
        U = np.ascontiguousarray(U, dtype=np.float64)
        Re = np.empty(12)
        Ke = np.empty(144)
        if lib().oracle_element(self.dptr, _ptr(U), t, l, _ptr(Re), _ptr(Ke)):
            raise RuntimeError("oracle_element failed")
        return Re, Ke.reshape(12, 12)

    def qp_state(self, U: np.ndarray, t: int, l: int, q: int) -> dict:
        U = np.ascontiguousarray(U, dtype=np.float64)
        out = np.empty(11)
        if lib().oracle_qp_state(self.dptr, _ptr(U), t, l, q, _ptr(out)):
            raise RuntimeError("oracle_qp_state failed")
        return {"grad_u": out[0:3].copy(), "grad_v": out[3:6].copy(), "eps2": out[6],
                "mu": out[7], "wdetJ": out[8], "grad_s": out[9:11].copy()}

    def sia(self) -> np.ndarray:
        U = np.empty(self.ndof)
        if lib().oracle_sia(self.dptr, _ptr(U)):
            raise RuntimeError("oracle_sia failed")
        return U


def basis_at(X: np.ndarray, xi: float, eta: float, zeta: float):
    """N[6], grad N [6, 3] and det J at reference point (xi, eta, zeta) of wedge X [6, 3]."""
    X = np.ascontiguousarray(X, dtype=np.float64).reshape(18)
    N = np.empty(6)
    gN = np.empty(18)
    det = np.empty(1)
    lib().oracle_basis_at(_ptr(X), xi, eta, zeta, _ptr(N), _ptr(gN), _ptr(det))
    return N, gN.reshape(6, 3), float(det[0])


def quadrature_point(q: int):
    out = np.empty(4)
    lib().oracle_qp(q, _ptr(out[0:1]), _ptr(out[1:2]), _ptr(out[2:3]), _ptr(out[3:4]))
    return tuple(float(v) for v in out)
