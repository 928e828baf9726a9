"""The viscous, resistive and thermal fluxes on the FP32-mixed path (perturbation gradients of
(U, T', S', B) in FP32 about the background, the background's own viscous residual in FP64) against
the FP64 oracle's full-state residual and steps: every variable within 1e-5 of its largest value."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import sdref  # noqa: E402
from paper_2502_17805_gb300 import inputs, sdmhd  # noqa: E402

pytestmark = pytest.mark.gpu

VISC = dict(viscous=1, mu=0.03, eta=0.02, kappa=0.01, kappa_r=0.015, R_gas=0.9)
VARS = ("rho", "mx", "my", "mz", "E", "Bx", "By", "Bz", "psi")


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


def _strict(g, o, label):
    err = np.abs(g - o).reshape(9, -1).max(axis=1)
    ref = 1e-5 * np.abs(o).reshape(9, -1).max(axis=1)
    print("mixed viscous %s: max|g-o|/(1e-5 max|o|) = %s" % (
        label, " ".join("%s %.2e" % (n, r) for n, r in zip(VARS, err / np.maximum(ref, 1e-300)))))
    return bool(np.all(err <= ref)), err, ref


def _box(N, seed):
    v, h, per = inputs.box_mesh(3, jitter=0.15, seed=seed)
    gm, om = _pair(N, v, inputs.reorient(h, seed=seed), periodic=per, geom=0)
    q0 = inputs.random_state(gm.n_e, N, seed=50 + seed)
    src = inputs.random_state(gm.n_e, N, seed=90 + seed)
    qb = np.zeros_like(q0)
    qb[0] = src[0]        # rho0 in [0.8, 1.2]
    qb[4] = 0.8 * src[4]  # E0 = p0 / (gamma - 1)
    return gm, om, q0, qb


@pytest.mark.parametrize("N", [2, 3, 4, 5, 6, 7, 8])
def test_mixed_viscous_residual_periodic_box(N):
    """A non-uniform background (its heat flux does not vanish) and a random state on a jittered,
    reoriented periodic box."""
    gm, om, q0, qb = _box(N, N)
    gph, oph = _phys(powell=1, c_h=0.7, glm_alpha=0.3, **VISC)
    bg = gm.background(gph, gm.to_device(qb))
    R = gm.to_host(gm.residual(gph, gm.to_device(q0), prec=sdmhd.SD_FP32_MIXED, bg=bg))
    Ro, _ = om.residual(oph, q0)
    # the viscous part is a sizeable share of this residual
    Ri, _ = om.residual(sdref.Phys(powell=1, c_h=0.7, glm_alpha=0.3), q0)
    assert np.abs(Ro - Ri).max() > 1e-2 * np.abs(Ri).max()
    ok, err, ref = _strict(R, Ro, "residual box N=%d" % N)
    assert ok, (err, ref)


@pytest.mark.parametrize("N", [3, 4, 6])
def test_mixed_viscous_residual_stratified_shell_with_walls(N):
    """The stratified shell (conducting inner, radial outer wall, each passing its own viscous flux),
    gravity, Coriolis, Powell, GLM, with a seeded flow."""
    v, h = inputs.shell_mesh(3, 2)
    gm, om = _pair(N, v, inputs.reorient(h, seed=3), geom=1, r_in=0.7, r_out=0.98,
                   bc_in=sdref.BC_WALL_CONDUCTING, bc_out=sdref.BC_WALL_RADIAL)
    gph, oph = _phys(powell=1, c_h=1.0, glm_alpha=0.5, gravity=1, GM=1.0, coriolis=1, omega=1.0, **VISC)
    prm = [2.5, 0.7, 0.98, 1.0, 0.9, 1e-4, 1e-3]
    q0, qb = om.state_init(oph, sdref.INIT_SHELL_POLYTROPE, prm, seed=4, background=True)
    rng = np.random.default_rng(N)
    mom = rng.uniform(-1e-2, 1e-2, size=q0[1:4].shape) * q0[0]
    q0[1:4] += mom
    q0[4] += 0.5 * (mom ** 2).sum(axis=0) / q0[0]
    bg = gm.background(gph, gm.to_device(qb))
    R = gm.to_host(gm.residual(gph, gm.to_device(q0), prec=sdmhd.SD_FP32_MIXED, bg=bg))
    Ro, _ = om.residual(oph, q0)
    ok, err, ref = _strict(R, Ro, "residual shell N=%d" % N)
    assert ok, (err, ref)


@pytest.mark.parametrize("N", [4, 6])
def test_mixed_viscous_steps_follow_the_oracle(N):
    """Three FP32-mixed sd_step steps (increment form: the viscous kernels read q' + D) against the
    oracle given each step's dt and c_h; every variable's change within 1e-5 of its largest value."""
    gm, om, q0, qb = _box(N, 10 + N)
    gph, oph = _phys(powell=1, c_h=0.0, glm_alpha=0.3, **VISC)
    bg = gm.background(gph, gm.to_device(qb))
    q, work = gm.to_device(q0), gm.empty_state()
    dts = torch.zeros(2, dtype=torch.float64, device="cuda")
    qo = q0
    for _ in range(3):
        gm.step(gph, 0.1, q, work, prec=sdmhd.SD_FP32_MIXED, bg=bg, dt_out=dts)
        dt, ch = dts.cpu().numpy()
        oph.c_h = float(ch)
        qo = om.rk_step(oph, float(dt), qo)
    ok, err, ref = _strict(gm.to_host(q) - q0, qo - q0, "sd_step x3 N=%d" % N)
    assert ok, (err, ref)


def test_mixed_viscous_rk_stage_and_advance():
    """sd_rk_stage on the mixed path (the q^n form, FP64 stage states) against the oracle's step, and
    sd_advance bitwise equal to repeated sd_step."""
    N = 5
    gm, om, q0, qb = _box(N, 21)
    gph, oph = _phys(powell=1, c_h=0.6, glm_alpha=0.3, **VISC)
    bg = gm.background(gph, gm.to_device(qb))
    dt = 2e-3
    q, work = gm.to_device(q0), gm.empty_state()
    gm.rk_step(gph, dt, q, work, prec=sdmhd.SD_FP32_MIXED, bg=bg)
    qo = om.rk_step(oph, dt, q0)
    ok, err, ref = _strict(gm.to_host(q) - q0, qo - q0, "rk_stage step")
    assert ok, (err, ref)
    gph.c_h = 0.0
    K = 3
    qa, wa = gm.to_device(q0), gm.empty_state()
    da = torch.zeros(2 * K, dtype=torch.float64, device="cuda")
    for k in range(K):
        gm.step(gph, 0.1, qa, wa, prec=sdmhd.SD_FP32_MIXED, bg=bg, dt_out=da[2 * k: 2 * k + 2])
    qb_, wb = gm.to_device(q0), gm.empty_state()
    db = torch.zeros(2 * K, dtype=torch.float64, device="cuda")
    gm.advance(gph, 0.1, K, qb_, wb, prec=sdmhd.SD_FP32_MIXED, bg=bg, dt_out=db)
    torch.cuda.synchronize()
    assert torch.equal(da, db) and torch.equal(qa, qb_)


def test_mixed_viscous_refusals():
    N = 3
    gm, om, q0, qb = _box(N, 2)
    visc = sdmhd.Phys(powell=1, c_h=0.7, **VISC)
    plain_bg = gm.background(sdmhd.Phys(powell=1, c_h=0.7), gm.to_device(qb))
    q = gm.to_device(q0)
    with pytest.raises(sdmhd.SDError, match="background built with them"):
        gm.residual(visc, q, prec=sdmhd.SD_FP32_MIXED, bg=plain_bg)
    bg = gm.background(visc, gm.to_device(qb))
    other = sdmhd.Phys(powell=1, c_h=0.7, **dict(VISC, mu=0.05))
    with pytest.raises(sdmhd.SDError, match="other viscous coefficients"):
        gm.residual(other, q, prec=sdmhd.SD_FP32_MIXED, bg=bg)
    walls = sdmhd.Phys(powell=1, c_h=0.7, visc_walls=1, q_bottom=0.0, T_top=1.0, **VISC)
    with pytest.raises(sdmhd.SDError) as exc:
        gm.residual(walls, q, prec=sdmhd.SD_FP32_MIXED, bg=bg)
    assert exc.value.code in (1, 2)
    v, h = inputs.shell_mesh(2, 1)
    ff = sdmhd.Mesh(N, v, h, geom=1, r_in=0.7, r_out=0.98, bc_in=sdmhd.BC_FARFIELD, bc_out=sdmhd.BC_FARFIELD)
    with pytest.raises(sdmhd.SDError) as exc:
        ff.background(visc, ff.empty_state())
    assert exc.value.code == 2


VISC_R = dict(VISC, kappa_r=0.004, kappa_r1=0.012, kappa_r2=0.006)


@pytest.mark.parametrize("N", [3, 6])
def test_mixed_viscous_radius_dependent_kappa_r(N):
    """kappa_r(r) = kappa_r + kappa_r1 r + kappa_r2 r^2 (reading V7) on the mixed path: the viscous
    kernel's instance that extrapolates the coordinates to every flux point, on the stratified shell
    with walls (the background's own viscous residual taken with the same kappa_r(r))."""
    v, h = inputs.shell_mesh(3, 2)
    gm, om = _pair(N, v, inputs.reorient(h, seed=5), geom=1, r_in=0.7, r_out=0.98,
                   bc_in=sdref.BC_WALL_CONDUCTING, bc_out=sdref.BC_WALL_RADIAL)
    gph, oph = _phys(powell=1, c_h=1.0, glm_alpha=0.5, gravity=1, GM=1.0, coriolis=1, omega=1.0, **VISC_R)
    prm = [2.5, 0.7, 0.98, 1.0, 0.9, 1e-4, 1e-3]
    q0, qb = om.state_init(oph, sdref.INIT_SHELL_POLYTROPE, prm, seed=6, background=True)
    rng = np.random.default_rng(20 + N)
    mom = rng.uniform(-1e-2, 1e-2, size=q0[1:4].shape) * q0[0]
    q0[1:4] += mom
    q0[4] += 0.5 * (mom ** 2).sum(axis=0) / q0[0]
    bg = gm.background(gph, gm.to_device(qb))
    R = gm.to_host(gm.residual(gph, gm.to_device(q0), prec=sdmhd.SD_FP32_MIXED, bg=bg))
    Ro, _ = om.residual(oph, q0)
    # the radius dependence is a visible part of this residual (0.7% of it at N = 6, 9% at N = 3),
    # far above the 1e-5 tolerance
    R1, _ = om.residual(sdref.Phys(**dict(vars(oph), kappa_r1=0.0, kappa_r2=0.0)), q0)
    assert np.abs(Ro - R1).max() > 1e-3 * np.abs(Ro).max()
    ok, err, ref = _strict(R, Ro, "kappa_r(r) shell N=%d" % N)
    assert ok, (err, ref)


@pytest.mark.parametrize("N", [3, 5])
def test_mixed_viscous_radius_dependent_kappa_r_periodic_box(N):
    """kappa_r(r) on the jittered periodic box, whose periodic faces join points at different radii:
    both sides take the owner's face point (reading V7), so the face flux is one value."""
    gm, om, q0, qb = _box(N, 30 + N)
    gph, oph = _phys(powell=1, c_h=0.7, glm_alpha=0.3, **VISC_R)
    bg = gm.background(gph, gm.to_device(qb))
    R = gm.to_host(gm.residual(gph, gm.to_device(q0), prec=sdmhd.SD_FP32_MIXED, bg=bg))
    Ro, _ = om.residual(oph, q0)
    R1, _ = om.residual(sdref.Phys(**dict(vars(oph), kappa_r1=0.0, kappa_r2=0.0)), q0)
    assert np.abs(Ro - R1).max() > 1e-3 * np.abs(Ro).max()
    ok, err, ref = _strict(R, Ro, "kappa_r(r) periodic box N=%d" % N)
    assert ok, (err, ref)


def test_mixed_visc_cfl_limits_the_step():
    """sd_phys.visc_cfl on the mixed path: dt = min(cfl dx_min / lambda_max, visc_cfl dx_min^2 /
    nu_max), nu_max from the step's FP64 start state, as on the FP64 path."""
    N = 4
    gm, om, q0, qb = _box(N, 41)
    base = dict(powell=1, c_h=0.0, glm_alpha=0.3, **VISC)
    bg = gm.background(sdmhd.Phys(**base), gm.to_device(qb))
    nu = max(4.0 / 3.0 * VISC["mu"] / q0[0].min(), VISC["eta"], VISC["kappa"], 5.0 / 3.0 * VISC["kappa_r"])
    xs = sdref.nodes(N)[0]
    dx_min = gm.info["h_min"] * (xs[1] - xs[0])

    def dt_of(ph):
        q, work = gm.to_device(q0), gm.empty_state()
        dts = torch.zeros(2, dtype=torch.float64, device="cuda")
        gm.step(ph, 0.2, q, work, prec=sdmhd.SD_FP32_MIXED, bg=bg, dt_out=dts)
        return float(dts[0])

    dt_adv = dt_of(sdmhd.Phys(**base))
    c = 0.5 * dt_adv * nu / dx_min ** 2
    dt_v = dt_of(sdmhd.Phys(visc_cfl=c, **base))
    assert abs(dt_v - c * dx_min ** 2 / nu) <= 1e-12 * dt_v, (dt_v, c * dx_min ** 2 / nu)
    assert abs(dt_v / dt_adv - 0.5) < 1e-9

