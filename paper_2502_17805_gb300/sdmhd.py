"""Python binding of the C ABI in ``include/sdmhd.h`` (``libsdmhd.so``).

Argument marshalling only: every step of the computation runs in the CUDA
kernels of the library.  Device buffers are torch tensors (float64, CUDA,
shape ``(9, n_elements, elem_stride)``), passed by pointer with torch's
current stream.  There is no CPU fallback: if the library is missing or no
CUDA device is present, the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass, field
from typing import Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsdmhd.so")

SD_FP64, SD_FP32_MIXED = 0, 1
# time integrators of sd_step / sd_advance (sd_phys.rk_scheme)
RK_SSP33, RK_SSP53 = 0, 1
BC_PERIODIC, BC_WALL_CONDUCTING, BC_WALL_RADIAL, BC_FARFIELD = 0, 1, 2, 3
INIT_UNIFORM, INIT_ALFVEN, INIT_SHELL_POLYTROPE, INIT_DIVB_PULSE, INIT_SHELL_FLUX_BALANCED = 0, 1, 2, 3, 4
STATUS = {0: "SD_OK", 1: "SD_ERR_INVALID_ARGUMENT", 2: "SD_ERR_UNSUPPORTED", 3: "SD_ERR_MESH_TOPOLOGY",
          4: "SD_ERR_MESH_GEOMETRY", 5: "SD_ERR_OUT_OF_MEMORY", 6: "SD_ERR_CUDA", 7: "SD_ERR_NONPHYSICAL",
          8: "SD_ERR_TIMEOUT"}

# every symbol include/sdmhd.h declares
EXPORTS = ["sd_last_error", "sd_mesh_create", "sd_mesh_destroy", "sd_mesh_query", "sd_state_init",
           "sd_background_create", "sd_background_destroy", "sd_residual", "sd_rk_stage", "sd_step", "sd_advance",
           "sd_diagnostics", "sd_spherical_sums", "sd_profile_enable", "sd_profile_read", "sd_residual_noalloc",
           "sd_packer_create", "sd_packer_destroy", "sd_step_packed", "sd_mesh_set_wait_limit",
           "sd_memory_pool_keep"]


class SDError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("%s: %s" % (STATUS.get(code, str(code)), msg))
        self.code = code


class MeshDesc(C.Structure):
    _fields_ = [("order", C.c_int32), ("geom", C.c_int32), ("n_vertices", C.c_int64),
                ("vertices", C.POINTER(C.c_double)), ("n_elements", C.c_int64), ("hex", C.POINTER(C.c_int64)),
                ("periodic_lengths", C.POINTER(C.c_double)), ("r_inner", C.c_double), ("r_outer", C.c_double),
                ("bc_inner", C.c_int32), ("bc_outer", C.c_int32)]


class PhysC(C.Structure):
    _fields_ = [("gamma", C.c_double), ("GM", C.c_double), ("omega", C.c_double), ("glm_alpha", C.c_double),
                ("c_h", C.c_double), ("powell", C.c_int32), ("gravity", C.c_int32), ("coriolis", C.c_int32),
                ("rk_scheme", C.c_int32), ("farfield", C.c_double * 9), ("mu", C.c_double), ("eta", C.c_double),
                ("kappa", C.c_double), ("kappa_r", C.c_double), ("R_gas", C.c_double), ("viscous", C.c_int32),
                ("pad2_", C.c_int32), ("q_bottom", C.c_double), ("T_top", C.c_double), ("visc_walls", C.c_int32),
                ("pad3_", C.c_int32), ("kappa_r1", C.c_double), ("kappa_r2", C.c_double), ("visc_cfl", C.c_double)]


class InitC(C.Structure):
    _fields_ = [("kind", C.c_int32), ("pad_", C.c_int32), ("params", C.c_double * 16), ("seed", C.c_uint64)]


class DiagC(C.Structure):
    _fields_ = [(k, C.c_double) for k in
                ("ke", "eb", "max_divb", "mass", "energy", "lambda_max", "min_rho", "min_p", "volume")]


class ProfileC(C.Structure):
    _fields_ = [("stage_launches", C.c_int64), ("stage_ms", C.c_double), ("trace_launches", C.c_int64),
                ("trace_ms", C.c_double), ("other_launches", C.c_int64), ("other_ms", C.c_double)]


class MeshInfoC(C.Structure):
    _fields_ = [("order", C.c_int32), ("p_map", C.c_int32), ("n_elements", C.c_int64), ("n_points", C.c_int64),
                ("elem_stride", C.c_int64), ("state_bytes", C.c_int64), ("n_boundary_faces", C.c_int64),
                ("n_interior_faces", C.c_int64), ("h_min", C.c_double), ("device_bytes", C.c_int64),
                ("trace_bytes", C.c_int64)]


class StepReqC(C.Structure):
    _fields_ = [("mesh", C.c_void_p), ("phys", PhysC), ("bg", C.c_void_p), ("q", C.c_void_p), ("work", C.c_void_p),
                ("traces", C.c_void_p), ("dyn", C.c_void_p), ("cfl", C.c_double), ("flags", C.c_int32),
                ("pad_", C.c_int32)]


# sd_step_req.flags
REQ_KEEP_TRACES = 1
REQ_TRACES_READY = 2


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
    # viscous, resistive and thermal fluxes (FP64 path; off unless viscous=1)
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
    # time integrator of step / advance: RK_SSP33 (three-stage SSP-RK3) or RK_SSP53 (SSPRK(5,3))
    rk_scheme: int = RK_SSP33
    # diffusive limit of the step with the viscous terms: dt <= visc_cfl dx_min^2 / nu_max (0 = off)
    visc_cfl: float = 0.0

    def c(self) -> PhysC:
        p = PhysC()
        p.gamma, p.GM, p.omega, p.glm_alpha, p.c_h = self.gamma, self.GM, self.omega, self.glm_alpha, self.c_h
        p.powell, p.gravity, p.coriolis = int(self.powell), int(self.gravity), int(self.coriolis)
        for i in range(9):
            p.farfield[i] = float(self.farfield[i])
        p.mu, p.eta, p.kappa, p.kappa_r, p.R_gas = self.mu, self.eta, self.kappa, self.kappa_r, self.R_gas
        p.viscous = int(self.viscous)
        p.q_bottom, p.T_top, p.visc_walls = self.q_bottom, self.T_top, int(self.visc_walls)
        p.kappa_r1, p.kappa_r2 = self.kappa_r1, self.kappa_r2
        p.rk_scheme = int(self.rk_scheme)
        p.visc_cfl = float(self.visc_cfl)
        return p


_lib = None


def lib():
    """Load libsdmhd.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libsdmhd.so is not built; run __graft_entry__.build() or "
                               "python paper_2502_17805_gb300/build.py")
        L = C.CDLL(LIB_PATH)
        vp, dp = C.c_void_p, C.POINTER(C.c_double)
        L.sd_last_error.restype = C.c_char_p
        L.sd_mesh_create.argtypes = [C.POINTER(MeshDesc), vp, C.POINTER(vp)]
        L.sd_mesh_destroy.argtypes = [vp]
        L.sd_mesh_query.argtypes = [vp, C.POINTER(MeshInfoC)]
        L.sd_state_init.argtypes = [vp, C.POINTER(PhysC), C.POINTER(InitC), vp, vp, vp]
        L.sd_background_create.argtypes = [vp, C.POINTER(PhysC), vp, vp, C.POINTER(vp)]
        L.sd_background_destroy.argtypes = [vp]
        L.sd_residual.argtypes = [vp, C.POINTER(PhysC), C.c_int, vp, vp, vp, vp]
        L.sd_rk_stage.argtypes = [vp, C.POINTER(PhysC), C.c_int, C.c_int32, C.c_double, vp, vp, vp, vp, vp]
        L.sd_step.argtypes = [vp, C.POINTER(PhysC), C.c_int, C.c_double, vp, vp, vp, vp, vp]
        L.sd_advance.argtypes = [vp, C.POINTER(PhysC), C.c_int, C.c_double, C.c_int32, vp, vp, vp, vp, vp]
        L.sd_spherical_sums.argtypes = [vp, vp, C.c_double, C.c_double, C.c_int32, C.c_int32, vp, vp]
        L.sd_diagnostics.argtypes = [vp, C.POINTER(PhysC), vp, C.POINTER(DiagC), vp]
        L.sd_profile_enable.argtypes = [vp, C.c_int32]
        L.sd_mesh_set_wait_limit.argtypes = [vp, C.c_int32]
        L.sd_memory_pool_keep.argtypes = [C.c_int64]
        L.sd_profile_read.argtypes = [vp, C.POINTER(ProfileC)]
        L.sd_residual_noalloc.argtypes = [vp, C.POINTER(PhysC), vp, vp, vp]
        L.sd_packer_create.argtypes = [C.c_int32, C.POINTER(vp)]
        L.sd_packer_destroy.argtypes = [vp]
        L.sd_step_packed.argtypes = [vp, C.c_int32, C.POINTER(StepReqC), vp]
        for name in EXPORTS:
            getattr(L, name).restype = C.c_int if name != "sd_last_error" else C.c_char_p
        _lib = L
    return _lib


def _check(rc: int):
    if rc != 0:
        raise SDError(rc, lib().sd_last_error().decode())


def _stream(stream=None) -> int:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _ptr(t) -> Optional[int]:
    if t is None:
        return None
    return t.data_ptr()


class Background:
    def __init__(self, mesh: "Mesh", handle):
        self.mesh = mesh
        self._h = handle

    def __del__(self):
        if getattr(self, "_h", None):
            lib().sd_background_destroy(self._h)
            self._h = None


class Mesh:
    """A device mesh: geometry and face tables live on the current CUDA device."""

    def __init__(self, N: int, vertices, hexes, periodic: Optional[Sequence[float]] = None, geom: int = 0,
                 r_in: float = 0.0, r_out: float = 0.0, bc_in: int = BC_WALL_CONDUCTING,
                 bc_out: int = BC_WALL_RADIAL, stream=None):
        v = np.ascontiguousarray(vertices, dtype=np.float64).reshape(-1, 3)
        h = np.ascontiguousarray(hexes, dtype=np.int64).reshape(-1, 8)
        per = None if periodic is None else np.ascontiguousarray(periodic, dtype=np.float64)
        d = MeshDesc()
        d.order, d.geom = int(N), int(geom)
        d.n_vertices, d.vertices = v.shape[0], v.ctypes.data_as(C.POINTER(C.c_double))
        d.n_elements, d.hex = h.shape[0], h.ctypes.data_as(C.POINTER(C.c_int64))
        d.periodic_lengths = per.ctypes.data_as(C.POINTER(C.c_double)) if per is not None else None
        d.r_inner, d.r_outer, d.bc_inner, d.bc_outer = float(r_in), float(r_out), int(bc_in), int(bc_out)
        out = C.c_void_p()
        self._h = None
        _check(lib().sd_mesh_create(C.byref(d), _stream(stream), C.byref(out)))
        self._h = out
        info = MeshInfoC()
        _check(lib().sd_mesh_query(self._h, C.byref(info)))
        self.info = {k: getattr(info, k) for k, _ in MeshInfoC._fields_}
        self.N = int(N)
        self.n_e = h.shape[0]
        self.stride = int(info.elem_stride)

    def __del__(self):
        if getattr(self, "_h", None):
            lib().sd_mesh_destroy(self._h)
            self._h = None

    # ---- buffers
    def empty_state(self):
        import torch
        return torch.zeros((9, self.n_e, self.stride), dtype=torch.float64, device="cuda")

    def to_device(self, q_dense: np.ndarray):
        """Copy a dense host state (9, n_e, N^3) into a padded device state."""
        import torch
        q = self.empty_state()
        q[:, :, : self.N ** 3] = torch.from_numpy(np.ascontiguousarray(q_dense, dtype=np.float64)).to("cuda")
        return q

    def to_host(self, q) -> np.ndarray:
        return q[:, :, : self.N ** 3].cpu().numpy()

    # ---- the C ABI
    def state_init(self, phys: Phys, kind: int, params: Sequence[float], seed: int = 0, q=None, background=None,
                   stream=None):
        q = self.empty_state() if q is None else q
        ini = InitC()
        ini.kind, ini.seed = int(kind), int(seed)
        for i, x in enumerate(params):
            ini.params[i] = float(x)
        ph = phys.c()
        _check(lib().sd_state_init(self._h, C.byref(ph), C.byref(ini), _ptr(q), _ptr(background), _stream(stream)))
        return q

    def background(self, phys: Phys, q_background, stream=None) -> Background:
        out = C.c_void_p()
        ph = phys.c()
        _check(lib().sd_background_create(self._h, C.byref(ph), _ptr(q_background), _stream(stream), C.byref(out)))
        return Background(self, out)

    def residual(self, phys: Phys, q, dqdt=None, prec: int = SD_FP64, bg: Optional[Background] = None, stream=None):
        dqdt = self.empty_state() if dqdt is None else dqdt
        ph = phys.c()
        _check(lib().sd_residual(self._h, C.byref(ph), int(prec), _ptr(q), bg._h if bg else None, _ptr(dqdt),
                                 _stream(stream)))
        return dqdt

    def residual_noalloc(self, phys: Phys, q, dqdt, stream=None):
        """FP64 residual through sd_residual_noalloc: no allocation; scratch in the library's fixed array."""
        ph = phys.c()
        _check(lib().sd_residual_noalloc(self._h, C.byref(ph), _ptr(q), _ptr(dqdt), _stream(stream)))
        return dqdt

    def rk_stage(self, phys: Phys, stage: int, dt: float, q_n, q_in, q_out, prec: int = SD_FP64,
                 bg: Optional[Background] = None, stream=None):
        ph = phys.c()
        _check(lib().sd_rk_stage(self._h, C.byref(ph), int(prec), int(stage), float(dt), _ptr(q_n), _ptr(q_in),
                                 _ptr(q_out), bg._h if bg else None, _stream(stream)))
        return q_out

    def rk_step(self, phys: Phys, dt: float, q, work, prec: int = SD_FP64, bg: Optional[Background] = None,
                stream=None):
        """Three explicit stages with a fixed dt; the result is written into q."""
        self.rk_stage(phys, 0, dt, q, q, work, prec, bg, stream)
        self.rk_stage(phys, 1, dt, q, work, work, prec, bg, stream)
        self.rk_stage(phys, 2, dt, q, work, q, prec, bg, stream)
        return q

    def step(self, phys: Phys, cfl: float, q, work, prec: int = SD_FP64, bg: Optional[Background] = None,
             dt_out=None, stream=None):
        ph = phys.c()
        _check(lib().sd_step(self._h, C.byref(ph), int(prec), float(cfl), _ptr(q), _ptr(work),
                             bg._h if bg else None, _ptr(dt_out), _stream(stream)))
        return q

    def advance(self, phys: Phys, cfl: float, n_steps: int, q, work, prec: int = SD_FP64,
                bg: Optional[Background] = None, dt_out=None, stream=None):
        """n_steps calls of step() in one (same results); dt_out: device float64[2 * n_steps] or None."""
        ph = phys.c()
        _check(lib().sd_advance(self._h, C.byref(ph), int(prec), float(cfl), int(n_steps), _ptr(q), _ptr(work),
                                bg._h if bg else None, _ptr(dt_out), _stream(stream)))
        return q

    def spherical_sums(self, q, r_min: float, r_max: float, n_r: int, n_theta: int, out=None, stream=None):
        """device float64 [n_r, n_theta, 8]: w|J|-weighted sums of (1, V_r, V_theta, V_phi, E_pol, E_tor, rho,
        KE) per bin of radius x colatitude (divide by [..., 0] for the means)"""
        import torch
        out = torch.empty((n_r, n_theta, 8), dtype=torch.float64, device="cuda") if out is None else out
        _check(lib().sd_spherical_sums(self._h, _ptr(q), float(r_min), float(r_max), int(n_r), int(n_theta),
                                       _ptr(out), _stream(stream)))
        return out

    def set_wait_limit(self, spins: int = -1):
        """Polls of a stage kernel's bounded waits before a time-out (failure-detection test
        hook); -1 restores the default."""
        _check(lib().sd_mesh_set_wait_limit(self._h, int(spins)))

    def profile(self, enable: bool = True):
        """Start (or stop) CUDA-event timing of every kernel the library launches for this mesh."""
        _check(lib().sd_profile_enable(self._h, 1 if enable else 0))

    def profile_read(self) -> dict:
        p = ProfileC()
        _check(lib().sd_profile_read(self._h, C.byref(p)))
        return {k: getattr(p, k) for k, _ in ProfileC._fields_}

    def diagnostics(self, phys: Phys, q, stream=None, check: bool = True) -> dict:
        d = DiagC()
        ph = phys.c()
        rc = lib().sd_diagnostics(self._h, C.byref(ph), _ptr(q), C.byref(d), _stream(stream))
        out = {k: getattr(d, k) for k, _ in DiagC._fields_}
        if rc != 0 and (check or rc != 7):
            _check(rc)
        out["status"] = rc
        return out


def memory_pool_keep(n_bytes: int):
    """Keep up to n_bytes of freed stream-ordered memory in the current device's default pool
    (sd_memory_pool_keep; negative: all of it)."""
    _check(lib().sd_memory_pool_keep(int(n_bytes)))


class Packer:
    """Packed SSP-RK3 steps of many independent solves (sd_step_packed, FP32-mixed path)."""

    def __init__(self, max_requests: int):
        out = C.c_void_p()
        self._h = None
        _check(lib().sd_packer_create(int(max_requests), C.byref(out)))
        self._h = out
        self.cap = int(max_requests)

    def __del__(self):
        if getattr(self, "_h", None):
            lib().sd_packer_destroy(self._h)
            self._h = None

    @staticmethod
    def request(mesh, phys, bg, q, work, traces, dyn, cfl, flags=0) -> StepReqC:
        """The C record of one request (the caller keeps the tensors alive while it is used)."""
        r = StepReqC()
        r.mesh, r.phys, r.bg = mesh._h, phys.c(), bg._h
        r.q, r.work, r.traces, r.dyn = _ptr(q), _ptr(work), _ptr(traces), _ptr(dyn)
        r.cfl = float(cfl)
        r.flags = int(flags)
        return r

    def step(self, reqs, stream=None):
        """reqs: sequence of (mesh, phys, background, q, work, traces, dyn, cfl[, flags])."""
        self.step_records([self.request(*req) for req in reqs], stream)

    def step_records(self, recs, stream=None):
        """recs: sequence of StepReqC records (see request())."""
        arr = (StepReqC * max(len(recs), 1))(*recs)
        _check(lib().sd_step_packed(self._h, len(recs), arr, _stream(stream)))
