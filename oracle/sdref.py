"""ctypes binding of the plain FP64 CPU oracle (``sdref.c``).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU-baseline leg
of the benchmark call it; the product path never does.  States are numpy
float64 arrays of shape (9, n_elements, N**3) in the variable order
(rho, rho u, rho v, rho w, E, Bx, By, Bz, psi).
"""
import ctypes as C
import os
from dataclasses import dataclass, field
from typing import Optional, Sequence

import numpy as np

from . import build as _build

_lib = None

BC_PERIODIC, BC_WALL_CONDUCTING, BC_WALL_RADIAL, BC_FARFIELD = 0, 1, 2, 3
INIT_UNIFORM, INIT_ALFVEN, INIT_SHELL_POLYTROPE, INIT_DIVB_PULSE, INIT_SINB, INIT_SHELL_FLUX_BALANCED = 0, 1, 2, 3, 4, 5


class _Phys(C.Structure):
    _fields_ = [("gamma", C.c_double), ("GM", C.c_double), ("omega", C.c_double),
                ("glm_alpha", C.c_double), ("c_h", C.c_double), ("powell", C.c_int32),
                ("gravity", C.c_int32), ("coriolis", C.c_int32), ("pad_", C.c_int32),
                ("farfield", C.c_double * 9), ("mu", C.c_double), ("eta", C.c_double), ("kappa", C.c_double),
                ("kappa_r", C.c_double), ("R_gas", C.c_double), ("viscous", C.c_int32), ("pad2_", C.c_int32),
                ("q_bottom", C.c_double), ("T_top", C.c_double), ("visc_walls", C.c_int32), ("pad3_", C.c_int32),
                ("kappa_r1", C.c_double), ("kappa_r2", C.c_double)]


class _Diag(C.Structure):
    _fields_ = [(k, C.c_double) for k in
                ("ke", "eb", "max_divb", "mass", "energy", "lambda_max", "min_rho", "min_p", "volume")]


@dataclass
class Phys:
    gamma: float = 5.0 / 3.0
    GM: float = 0.0
    omega: float = 0.0
    glm_alpha: float = 0.0
    c_h: float = 0.0
    powell: int = 1
    gravity: int = 0
    coriolis: int = 0
    farfield: Sequence[float] = field(default_factory=lambda: [0.0] * 9)
    # viscous, resistive and thermal fluxes (off unless viscous=1)
    mu: float = 0.0
    eta: float = 0.0
    kappa: float = 0.0
    kappa_r: float = 0.0
    R_gas: float = 1.0
    viscous: int = 0
    # walls of the viscous path: stress-free, heat flux through the inner sphere, temperature on the outer
    q_bottom: float = 0.0
    T_top: float = 1.0
    visc_walls: int = 0
    # radiative diffusivity kappa_r(r) = kappa_r + kappa_r1 r + kappa_r2 r^2
    kappa_r1: float = 0.0
    kappa_r2: float = 0.0

    def _c(self) -> _Phys:
        p = _Phys()
        p.gamma, p.GM, p.omega, p.glm_alpha, p.c_h = self.gamma, self.GM, self.omega, self.glm_alpha, self.c_h
        p.powell, p.gravity, p.coriolis = int(self.powell), int(self.gravity), int(self.coriolis)
        for i in range(9):
            p.farfield[i] = float(self.farfield[i])
        p.mu, p.eta, p.kappa, p.kappa_r, p.R_gas = self.mu, self.eta, self.kappa, self.kappa_r, self.R_gas
        p.viscous = int(self.viscous)
        p.q_bottom, p.T_top, p.visc_walls = self.q_bottom, self.T_top, int(self.visc_walls)
        p.kappa_r1, p.kappa_r2 = self.kappa_r1, self.kappa_r2
        return p


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        dp, ip = C.POINTER(C.c_double), C.POINTER(C.c_int64)
        L.sdref_last_error.restype = C.c_char_p
        L.sdref_nodes.argtypes = [C.c_int, dp, dp, dp, dp, dp]
        L.sdref_mesh_create.restype = C.c_void_p
        L.sdref_mesh_create.argtypes = [C.c_int, C.c_int64, dp, C.c_int64, ip, dp, C.c_int, C.c_double,
                                        C.c_double, C.c_int, C.c_int]
        L.sdref_mesh_destroy.argtypes = [C.c_void_p]
        L.sdref_mesh_info.argtypes = [C.c_void_p, ip, ip, dp]
        L.sdref_mesh_faces.argtypes = [C.c_void_p, C.c_int64, ip, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                       C.POINTER(C.c_int32)]
        L.sdref_geometry.argtypes = [C.c_void_p, C.c_int64, dp, dp, dp, dp]
        L.sdref_residual.argtypes = [C.c_void_p, C.POINTER(_Phys), dp, dp, dp, dp]
        L.sdref_residual_elements.argtypes = [C.c_void_p, C.POINTER(_Phys), dp, C.c_int64, ip, dp, dp]
        L.sdref_gradients.argtypes = [C.c_void_p, C.POINTER(_Phys), dp, dp]
        L.sdref_spherical_averages.argtypes = [C.c_void_p, dp, C.c_int, C.c_int, dp]
        L.sdref_flux_balanced.argtypes = [dp, C.c_double, C.c_double, C.c_int, C.c_int, dp, dp, dp]
        L.sdref_rk_stage.argtypes = [C.c_void_p, C.POINTER(_Phys), C.c_int, C.c_double, dp, dp, dp]
        L.sdref_rk53_step.argtypes = [C.c_void_p, C.POINTER(_Phys), C.c_double, dp, dp]
        L.sdref_diagnostics.argtypes = [C.c_void_p, C.POINTER(_Phys), dp, C.POINTER(_Diag)]
        L.sdref_state_init.argtypes = [C.c_void_p, C.POINTER(_Phys), C.c_int, dp, C.c_uint64, dp, dp]
        L.sdref_polytrope.argtypes = [C.c_double] * 8 + [dp, dp, dp]
        L.sdref_uniform.restype = C.c_double
        L.sdref_uniform.argtypes = [C.c_uint64, C.c_uint64]
        L.sdref_splitmix64.restype = C.c_uint64
        L.sdref_splitmix64.argtypes = [C.c_uint64, C.c_uint64]
        L.sdref_flux.argtypes = [dp, dp, C.c_double, C.c_double, dp]
        L.sdref_fast_speed.restype = C.c_double
        L.sdref_fast_speed.argtypes = [dp, dp, C.c_double]
        L.sdref_rusanov.argtypes = [dp, dp, dp, C.c_double, C.c_double, dp]
        L.sdref_set_threads.argtypes = [C.c_int]
        L.sdref_get_threads.restype = C.c_int
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _check(rc: int):
    if rc != 0:
        raise RuntimeError("oracle: " + lib().sdref_last_error().decode())


def set_threads(n: int):
    lib().sdref_set_threads(int(n))


def get_threads() -> int:
    return int(lib().sdref_get_threads())


def flux_balanced(params, r, gamma=5.0 / 3.0, GM=1.0, n_nodes=4096):
    """almost flux-balanced profile rho(r), p(r) (Sec. Initial Conditions); params as for
    INIT_SHELL_FLUX_BALANCED: N_rho, r_b, r_t, rho_b, R, noise, dipole, L, kappa, kappa_r[, kappa_r1,
    kappa_r2]"""
    P = _f64(np.asarray(list(params) + [0.0] * (16 - len(params))))
    r = _f64(np.atleast_1d(r))
    rho, p = np.zeros_like(r), np.zeros_like(r)
    _check(lib().sdref_flux_balanced(_dp(P), float(gamma), float(GM), int(n_nodes), r.size, _dp(r), _dp(rho), _dp(p)))
    return rho, p


def nodes(N: int):
    xs, xf = np.zeros(N), np.zeros(N + 1)
    E, D, w = np.zeros((N + 1, N)), np.zeros((N, N + 1)), np.zeros(N)
    _check(lib().sdref_nodes(N, _dp(xs), _dp(xf), _dp(E), _dp(D), _dp(w)))
    return xs, xf, E, D, w


def splitmix64(seed: int, index: int) -> int:
    return int(lib().sdref_splitmix64(seed, index))


def uniform(seed: int, index: int) -> float:
    return float(lib().sdref_uniform(seed, index))


def polytrope(r, N_rho, r_b, r_t, rho_b, R_gas, gamma, GM):
    rho, p, T = C.c_double(), C.c_double(), C.c_double()
    lib().sdref_polytrope(r, N_rho, r_b, r_t, rho_b, R_gas, gamma, GM, C.byref(rho), C.byref(p), C.byref(T))
    return rho.value, p.value, T.value


def flux(q, n, gamma, c_h):
    q, n, F = _f64(q), _f64(n), np.zeros(9)
    lib().sdref_flux(_dp(q), _dp(n), gamma, c_h, _dp(F))
    return F


def fast_speed(q, n, gamma):
    q, n = _f64(q), _f64(n)
    return float(lib().sdref_fast_speed(_dp(q), _dp(n), gamma))


def rusanov(qL, qR, n, gamma, c_h):
    qL, qR, n, F = _f64(qL), _f64(qR), _f64(n), np.zeros(9)
    lib().sdref_rusanov(_dp(qL), _dp(qR), _dp(n), gamma, c_h, _dp(F))
    return F


class Mesh:
    """Oracle mesh over the same (vertices, hexahedra) input the CUDA library takes."""

    def __init__(self, N: int, vertices, hexes, periodic: Optional[Sequence[float]] = None, geom: int = 0,
                 r_in: float = 0.0, r_out: float = 0.0, bc_in: int = BC_WALL_CONDUCTING,
                 bc_out: int = BC_WALL_RADIAL):
        self.N = int(N)
        self.p = self.N // 2
        self._v = _f64(vertices).reshape(-1, 3)
        self._h = np.ascontiguousarray(hexes, dtype=np.int64).reshape(-1, 8)
        self.n_e = self._h.shape[0]
        per = None if periodic is None else _f64(periodic)
        self._per = per
        h = lib().sdref_mesh_create(self.N, self._v.shape[0], _dp(self._v), self.n_e,
                                    self._h.ctypes.data_as(C.POINTER(C.c_int64)),
                                    None if per is None else _dp(per), int(geom), float(r_in), float(r_out),
                                    int(bc_in), int(bc_out))
        if not h:
            raise RuntimeError("oracle: " + lib().sdref_last_error().decode())
        self._h_ptr = h

    def __del__(self):
        if getattr(self, "_h_ptr", None):
            lib().sdref_mesh_destroy(self._h_ptr)
            self._h_ptr = None

    @property
    def N3(self):
        return self.N ** 3

    def info(self):
        nb, ni, hm = C.c_int64(), C.c_int64(), C.c_double()
        lib().sdref_mesh_info(self._h_ptr, C.byref(nb), C.byref(ni), C.byref(hm))
        return {"n_boundary_faces": nb.value, "n_interior_faces": ni.value, "h_min": hm.value}

    def faces(self, e: int):
        nb = np.zeros(6, np.int64)
        nf, ow, cd = (np.zeros(6, np.int32) for _ in range(3))
        i32 = C.POINTER(C.c_int32)
        _check(lib().sdref_mesh_faces(self._h_ptr, e, nb.ctypes.data_as(C.POINTER(C.c_int64)),
                                      nf.ctypes.data_as(i32), ow.ctypes.data_as(i32), cd.ctypes.data_as(i32)))
        return nb, nf, ow, cd

    def geometry(self, e: int):
        N, p1 = self.N, self.p + 1
        S = np.zeros((3, N, N, N + 1, 3))  # [d][b][a][f][c]
        J = np.zeros(N ** 3)
        X = np.zeros((N ** 3, 3))
        Xp = np.zeros((p1 ** 3, 3))
        _check(lib().sdref_geometry(self._h_ptr, e, _dp(S), _dp(J), _dp(X), _dp(Xp)))
        return S, J, X, Xp

    def _q(self, q):
        q = _f64(q)
        assert q.shape == (9, self.n_e, self.N3), q.shape
        return q

    def residual(self, phys: Phys, q, want_divb: bool = False):
        q = self._q(q)
        out = np.zeros_like(q)
        divb = np.zeros((self.n_e, self.N3)) if want_divb else None
        scale = np.zeros(9)
        ph = phys._c()
        _check(lib().sdref_residual(self._h_ptr, C.byref(ph), _dp(q), _dp(out),
                                    None if divb is None else _dp(divb), _dp(scale)))
        return (out, scale, divb) if want_divb else (out, scale)

    def residual_elements(self, phys: Phys, q, elems):
        q = self._q(q)
        el = np.ascontiguousarray(elems, dtype=np.int64)
        out = np.zeros((el.size, 9, self.N3))
        scale = np.zeros(9)
        ph = phys._c()
        _check(lib().sdref_residual_elements(self._h_ptr, C.byref(ph), _dp(q), el.size,
                                             el.ctypes.data_as(C.POINTER(C.c_int64)), _dp(out), _dp(scale)))
        return out, scale

    def spherical_sums(self, q, n_r: int, n_theta: int):
        """[n_r, n_theta, 8] volume sums (volume, V_r, V_theta, V_phi, E_pol, E_tor, rho, KE) per bin"""
        q = self._q(q)
        out = np.zeros((n_r, n_theta, 8))
        _check(lib().sdref_spherical_averages(self._h_ptr, _dp(q), int(n_r), int(n_theta), _dp(out)))
        return out

    def gradients(self, phys: Phys, q):
        """gradients of (u, v, w, T, S, Bx, By, Bz) at the solution points: [n_e, 8, 3, N^3]"""
        q = self._q(q)
        out = np.zeros((self.n_e, 8, 3, self.N3))
        ph = phys._c()
        _check(lib().sdref_gradients(self._h_ptr, C.byref(ph), _dp(q), _dp(out)))
        return out

    def rk_stage(self, phys: Phys, stage: int, dt: float, q_n, q_in):
        q_in = self._q(q_in)
        q_n = self._q(q_n) if q_n is not None else q_in
        out = np.zeros_like(q_in)
        ph = phys._c()
        _check(lib().sdref_rk_stage(self._h_ptr, C.byref(ph), stage, dt, _dp(q_n), _dp(q_in), _dp(out)))
        return out

    def rk_step(self, phys: Phys, dt: float, q):
        q1 = self.rk_stage(phys, 0, dt, q, q)
        q2 = self.rk_stage(phys, 1, dt, q, q1)
        return self.rk_stage(phys, 2, dt, q, q2)

    def rk53_step(self, phys: Phys, dt: float, q):
        """one step of the five-stage third-order SSP method (SSPRK(5,3))"""
        q = self._q(q)
        out = np.zeros_like(q)
        ph = phys._c()
        _check(lib().sdref_rk53_step(self._h_ptr, C.byref(ph), dt, _dp(q), _dp(out)))
        return out

    def diagnostics(self, phys: Phys, q) -> dict:
        q = self._q(q)
        d = _Diag()
        ph = phys._c()
        _check(lib().sdref_diagnostics(self._h_ptr, C.byref(ph), _dp(q), C.byref(d)))
        return {k: getattr(d, k) for k, _ in _Diag._fields_}

    def state_init(self, phys: Phys, kind: int, params: Sequence[float], seed: int = 0, background: bool = False):
        q = np.zeros((9, self.n_e, self.N3))
        qb = np.zeros_like(q) if background else None
        P = np.zeros(16)
        P[:len(params)] = params
        ph = phys._c()
        _check(lib().sdref_state_init(self._h_ptr, C.byref(ph), kind, _dp(P), seed, _dp(q),
                                      None if qb is None else _dp(qb)))
        return (q, qb) if background else q
