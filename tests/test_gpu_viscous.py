"""Parity of the viscous, resistive and thermal fluxes (FP64 path, BR1 gradients) of the CUDA path
with the FP64 oracle; tolerances as in test_gpu_parity (|g - o| <= 1e-12 (|o| + s_v) per residual
entry, s_v the oracle's un-cancelled magnitude, which includes the viscous terms)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import sdref  # noqa: E402
from paper_2502_17805_gb300 import inputs, sdmhd  # noqa: E402

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
VISC = dict(viscous=1, mu=0.03, eta=0.02, kappa=0.01, kappa_r=0.015, R_gas=0.9)


@pytest.fixture(scope="module", autouse=True)
def _device():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_17805_gb300 import build
    build.build()
    torch.cuda.set_device(0)


def _pair(N, v, h, **kw):
    return sdmhd.Mesh(N, v, h, **kw), sdref.Mesh(N, v, h, **kw)


def _phys(**kw):
    return sdmhd.Phys(**kw), sdref.Phys(**kw)


def _c19(g, o, s):
    return float((np.abs(g - o) / (np.abs(o) + s[:, None, None])).max())


@pytest.mark.parametrize("N", [2, 3, 4, 5, 6, 7, 8])
def test_viscous_residual_jittered_periodic_box(N):
    v, h, per = inputs.box_mesh(3, jitter=0.15, seed=N)
    gm, om = _pair(N, v, h, periodic=per, geom=0)
    gph, oph = _phys(powell=1, c_h=0.7, glm_alpha=0.3, **VISC)
    q0 = inputs.random_state(gm.n_e, N, seed=20 + N)
    R = gm.to_host(gm.residual(gph, gm.to_device(q0)))
    Ro, s = om.residual(oph, q0)
    # the viscous part is a sizeable share of this residual
    R0, _ = om.residual(sdref.Phys(powell=1, c_h=0.7, glm_alpha=0.3), q0)
    assert np.abs(Ro - R0).max() > 1e-2 * np.abs(R0).max()
    assert _c19(R, Ro, s) < TOL64


@pytest.mark.parametrize("N", [4, 6])
def test_viscous_residual_shell_with_walls_and_sources(N):
    """Curved shell: BR1 averages against the wall ghost states, a wall's own viscous flux, every
    source on."""
    v, h = inputs.shell_mesh(2, 2)
    h = inputs.reorient(h, seed=4)
    gm, om = _pair(N, v, h, geom=1, r_in=0.7, r_out=0.98, bc_in=sdref.BC_WALL_CONDUCTING,
                   bc_out=sdref.BC_WALL_RADIAL)
    gph, oph = _phys(powell=1, c_h=0.8, glm_alpha=0.5, gravity=1, GM=1.0, coriolis=1, omega=1.0, **VISC)
    q0 = inputs.random_state(gm.n_e, N, seed=31)
    R = gm.to_host(gm.residual(gph, gm.to_device(q0)))
    Ro, s = om.residual(oph, q0)
    assert _c19(R, Ro, s) < TOL64


@pytest.mark.parametrize("N", [3, 5])
def test_viscous_residual_shell_far_field(N):
    """Far-field faces: the BR1 average against the far-field state, this side's viscous flux alone."""
    v, h = inputs.shell_mesh(2, 2)
    gm, om = _pair(N, v, inputs.reorient(h, seed=N), geom=1, r_in=0.7, r_out=0.98, bc_in=sdref.BC_FARFIELD,
                   bc_out=sdref.BC_FARFIELD)
    gph, oph = _phys(powell=1, c_h=0.8, glm_alpha=0.5, **VISC)
    q0 = inputs.random_state(gm.n_e, N, seed=40 + N)
    gph.farfield = oph.farfield = list(q0[:, 0, 0])
    R = gm.to_host(gm.residual(gph, gm.to_device(q0)))
    Ro, s = om.residual(oph, q0)
    assert _c19(R, Ro, s) < TOL64


def test_viscous_steps_follow_the_oracle():
    """Three SSP-RK3 steps through sd_step (device dt, c_h) against the oracle given them."""
    N = 4
    v, h, per = inputs.box_mesh(3, jitter=0.1, seed=6)
    gm, om = _pair(N, v, h, periodic=per, geom=0)
    gph, oph = _phys(powell=1, c_h=0.0, glm_alpha=0.3, **VISC)
    q0 = inputs.random_state(gm.n_e, N, seed=8)
    q, work = gm.to_device(q0), gm.empty_state()
    dts = torch.zeros(2, dtype=torch.float64, device="cuda")
    qo = q0
    for _ in range(3):
        gm.step(gph, 0.1, q, work, dt_out=dts)
        dt, ch = dts.cpu().numpy()
        oph.c_h = float(ch)
        qo = om.rk_step(oph, float(dt), qo)
    change = np.abs(qo - q0).max(axis=(1, 2))
    err = np.abs(gm.to_host(q) - qo).max(axis=(1, 2))
    scale = np.abs(q0).max(axis=(1, 2))
    assert np.all(err <= 1e-12 * scale + 1e-9 * change), (err, change)


def test_viscous_advance_equals_repeated_steps():
    N = 5
    v, h, per = inputs.box_mesh(3, jitter=0.1, seed=7)
    gm = sdmhd.Mesh(N, v, h, periodic=per, geom=0)
    gph = sdmhd.Phys(powell=1, c_h=0.0, glm_alpha=0.3, **VISC)
    q0 = inputs.random_state(gm.n_e, N, seed=9)
    qa, wa = gm.to_device(q0), gm.empty_state()
    for _ in range(3):
        gm.step(gph, 0.1, qa, wa)
    qb, wb = gm.to_device(q0), gm.empty_state()
    gm.advance(gph, 0.1, 3, qb, wb)
    torch.cuda.synchronize()
    assert torch.equal(qa, qb)


def test_viscous_fluxes_are_rejected_where_unsupported():
    N = 4
    v, h = inputs.shell_mesh(2, 1)
    gm = sdmhd.Mesh(N, v, h, geom=1, r_in=0.7, r_out=0.98)
    gph = sdmhd.Phys(gravity=1, GM=1.0, **VISC)
    qb = gm.empty_state()
    q = gm.state_init(gph, sdmhd.INIT_SHELL_POLYTROPE, [1.5, 0.7, 0.98, 1.0, 1.0, 1e-4, 0.0], seed=0, background=qb)
    # the mixed path takes viscous fluxes only about a background built with them
    bg = gm.background(sdmhd.Phys(gravity=1, GM=1.0), qb)
    with pytest.raises(sdmhd.SDError, match="background built with them"):
        gm.residual(gph, q, prec=sdmhd.SD_FP32_MIXED, bg=bg)
    walls = sdmhd.Phys(gravity=1, GM=1.0, visc_walls=1, q_bottom=0.05, T_top=0.6, **VISC)
    with pytest.raises(sdmhd.SDError, match="FP64"):
        gm.background(walls, qb)
    with pytest.raises(sdmhd.SDError, match="sd_residual"):
        gm.residual_noalloc(gph, q, gm.empty_state())
    bad = sdmhd.Phys(gravity=1, GM=1.0, **dict(VISC, mu=-1.0))
    with pytest.raises(sdmhd.SDError, match="non-negative"):
        gm.residual(bad, q)


@pytest.mark.parametrize("N", [2, 3, 4, 5, 6, 7, 8])
def test_viscous_walls_residual(N):
    """Stress-free walls, heat flux through the inner sphere, temperature held on the outer sphere."""
    v, h = inputs.shell_mesh(2, 2)
    h = inputs.reorient(h, seed=6)
    gm, om = _pair(N, v, h, geom=1, r_in=0.7, r_out=0.98, bc_in=sdref.BC_WALL_CONDUCTING,
                   bc_out=sdref.BC_WALL_RADIAL)
    walls = dict(VISC, visc_walls=1, q_bottom=0.05, T_top=0.6)
    gph, oph = _phys(powell=1, c_h=0.8, glm_alpha=0.5, gravity=1, GM=1.0, coriolis=1, omega=1.0, **walls)
    q0 = inputs.random_state(gm.n_e, N, seed=41)
    R = gm.to_host(gm.residual(gph, gm.to_device(q0)))
    Ro, s = om.residual(oph, q0)
    assert _c19(R, Ro, s) < TOL64
    # and the walls change the residual of the wall elements
    R_own, _ = om.residual(sdref.Phys(**dict(vars(oph), visc_walls=0)), q0)
    assert np.abs(Ro - R_own).max() > 1e-3 * np.abs(Ro).max()


VISC_R = dict(VISC, kappa_r=0.004, kappa_r1=0.012, kappa_r2=0.006)


@pytest.mark.parametrize("N", [3, 4, 6])
def test_radius_dependent_kappa_r_box(N):
    """kappa_r(r) = kappa_r + kappa_r1 r + kappa_r2 r^2 at every flux, face and wall point (reading V7)."""
    v, h, per = inputs.box_mesh(3, jitter=0.15, seed=N)
    gm, om = _pair(N, v, h, periodic=per, geom=0)
    gph, oph = _phys(powell=1, c_h=0.7, glm_alpha=0.3, **VISC_R)
    q0 = inputs.random_state(gm.n_e, N, seed=60 + N)
    R = gm.to_host(gm.residual(gph, gm.to_device(q0)))
    Ro, s = om.residual(oph, q0)
    # the radius dependence is a visible part of this residual
    R1, _ = om.residual(sdref.Phys(**dict(vars(oph), kappa_r1=0.0, kappa_r2=0.0)), q0)
    assert np.abs(Ro - R1).max() > 1e-4 * np.abs(Ro).max()
    assert _c19(R, Ro, s) < TOL64


@pytest.mark.parametrize("N", [4, 5])
def test_radius_dependent_kappa_r_shell_walls(N):
    v, h = inputs.shell_mesh(2, 2)
    h = inputs.reorient(h, seed=7)
    gm, om = _pair(N, v, h, geom=1, r_in=0.7, r_out=0.98, bc_in=sdref.BC_WALL_CONDUCTING,
                   bc_out=sdref.BC_WALL_RADIAL)
    walls = dict(VISC_R, visc_walls=1, q_bottom=0.05, T_top=0.6)
    gph, oph = _phys(powell=1, c_h=0.8, glm_alpha=0.5, gravity=1, GM=1.0, coriolis=1, omega=1.0, **walls)
    q0 = inputs.random_state(gm.n_e, N, seed=71)
    R = gm.to_host(gm.residual(gph, gm.to_device(q0)))
    Ro, s = om.residual(oph, q0)
    assert _c19(R, Ro, s) < TOL64


def _nu_max(q0, ph, xyz=None):
    """max over the solution points of (4/3 mu / rho, eta, kappa, gamma kappa_r(r))"""
    nu = max(4.0 / 3.0 * ph.mu / q0[0].min(), ph.eta, ph.kappa, ph.gamma * ph.kappa_r)
    if xyz is not None:
        r = np.sqrt((xyz ** 2).sum(axis=-1))
        nu = max(nu, float((ph.gamma * (ph.kappa_r + ph.kappa_r1 * r + ph.kappa_r2 * r * r)).max()))
    return nu


@pytest.mark.parametrize("radial", [False, True])
def test_visc_cfl_limits_the_step(radial):
    """With visc_cfl set, dt = min(cfl dx_min / lambda_max, visc_cfl dx_min^2 / nu_max), nu_max the
    largest diffusivity of the step's start state (with kappa_r(r), at the points' radii)."""
    N = 4
    v, h = inputs.shell_mesh(2, 2)
    kw = dict(geom=1, r_in=0.7, r_out=0.98, bc_in=sdref.BC_WALL_CONDUCTING, bc_out=sdref.BC_WALL_RADIAL)
    gm, om = _pair(N, v, inputs.reorient(h, seed=9), **kw)
    coef = dict(VISC_R, mu=1e-3) if radial else dict(VISC)  # radial: gamma kappa_r(r) the largest
    base = dict(powell=1, c_h=0.0, glm_alpha=0.5, **coef)
    q0 = inputs.random_state(gm.n_e, N, seed=77)
    xyz = np.stack([om.geometry(e)[2] for e in range(gm.n_e)]) if radial else None
    ph0 = sdmhd.Phys(**base)
    nu = _nu_max(q0, ph0, xyz)
    if radial:
        assert nu > 1.5 * max(4.0 / 3.0 * ph0.mu / q0[0].min(), ph0.eta, ph0.kappa)
    xs = sdref.nodes(N)[0]
    dx_min = gm.info["h_min"] * (xs[1] - xs[0])

    def dt_of(ph, prec=sdmhd.SD_FP64):
        q, work = gm.to_device(q0), gm.empty_state()
        dts = torch.zeros(2, dtype=torch.float64, device="cuda")
        gm.step(ph, 0.2, q, work, dt_out=dts)
        return float(dts[0])

    dt_adv = dt_of(ph0)
    c = 0.25 * dt_adv * nu / dx_min ** 2  # the diffusive limit at a quarter of the advective step
    dt_v = dt_of(sdmhd.Phys(visc_cfl=c, **base))
    assert abs(dt_v - c * dx_min ** 2 / nu) <= 1e-12 * dt_v, (dt_v, c * dx_min ** 2 / nu)
    assert abs(dt_v / dt_adv - 0.25) < 1e-9
    # a loose diffusive limit leaves the advective step; the five-stage method takes the same limit
    assert dt_of(sdmhd.Phys(visc_cfl=100 * c, **base)) == dt_adv
    dt53 = dt_of(sdmhd.Phys(visc_cfl=c, rk_scheme=sdmhd.RK_SSP53, **base))
    assert abs(dt53 - dt_v) <= 1e-12 * dt_v


def test_visc_cfl_refused_when_negative():
    N = 3
    v, h = inputs.shell_mesh(2, 1)
    gm = sdmhd.Mesh(N, v, h, geom=1, r_in=0.7, r_out=0.98)
    q = gm.to_device(inputs.random_state(gm.n_e, N, seed=3))
    with pytest.raises(sdmhd.SDError, match="visc_cfl"):
        gm.step(sdmhd.Phys(visc_cfl=-1.0, **VISC), 0.2, q, gm.empty_state())

