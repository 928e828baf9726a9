"""Parity at full size: the 6th-order shells of 41,472 elements (the benchmark
workload) and 221,184 elements, checked on sampled elements that the oracle
computes one by one.  The GPU runs the same kernels, grid and block shape as
the benchmark (trace kernel + fused stage kernel over every element)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import sdref  # noqa: E402
from paper_2502_17805_gb300 import inputs, sdmhd  # noqa: E402

pytestmark = pytest.mark.gpu

TOL64 = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _device():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_17805_gb300 import build
    build.build()
    torch.cuda.set_device(0)


def _shell(nz, nr, N=6):
    v, h = inputs.shell_mesh(nz, nr)
    kw = dict(geom=1, r_in=0.70, r_out=0.98, bc_in=sdref.BC_WALL_CONDUCTING, bc_out=sdref.BC_WALL_RADIAL)
    return sdmhd.Mesh(N, v, h, **kw), sdref.Mesh(N, v, h, **kw)


def _sample(n_e, k=48, seed=0):
    rng = np.random.default_rng(seed)
    return np.unique(np.concatenate([[0, n_e - 1], rng.choice(n_e, size=k, replace=False)]))


def _phys(ch=0.8):
    kw = dict(gamma=5.0 / 3.0, GM=1.0, omega=1.0, glm_alpha=1.0, c_h=ch, powell=1, gravity=1, coriolis=1)
    return sdmhd.Phys(**kw), sdref.Phys(**kw)


VARS = ("rho", "mx", "my", "mz", "E", "Bx", "By", "Bz", "psi")


def _mixed_bound(g, o, s, scale=1.0, floor=(4,), label="", var_axis=0):
    """max|g - o| <= 1e-5 max|o| per variable; the variables in `floor` (default: the energy, whose
    residual for a fluid at rest is the dissipation of discretisation-level face jumps, below FP32
    resolution of its terms) may add 4 eps32 scale s_v.  g, o: variables along `var_axis`."""
    g9 = np.moveaxis(g, var_axis, 0).reshape(9, -1)
    o9 = np.moveaxis(o, var_axis, 0).reshape(9, -1)
    err = np.abs(g9 - o9).max(axis=1)
    strict = 1e-5 * np.abs(o9).max(axis=1)
    fl = np.zeros(9)
    if floor:
        fl[list(floor)] = 4 * 2.0 ** -24 * scale * np.asarray(s).reshape(9)[list(floor)]
    ratio = err / np.maximum(strict, 1e-300)
    print("mixed %s: max|g-o|/(1e-5 max|o|) = %s" % (label, " ".join("%s %.2e" % (n, r) for n, r in zip(VARS, ratio))))
    return bool(np.all(err <= strict + fl)), err, strict + fl


def _gather(gm, q_dev, elems):
    """device state rows of the sampled elements -> (len, 9, N^3) on the host"""
    idx = torch.as_tensor(elems, device="cuda")
    return q_dev[:, idx, : gm.N ** 3].permute(1, 0, 2).cpu().numpy()


def test_shell41k_fp64_residual_and_stage_sampled():
    gm, om = _shell(24, 12)
    gph, oph = _phys()
    q0 = om.state_init(oph, sdref.INIT_SHELL_POLYTROPE, [3.0, 0.70, 0.98, 1.0, 1.0, 1e-4, 1e-6], seed=0)
    q = gm.to_device(q0)
    elems = _sample(gm.n_e)
    Ro, s = om.residual_elements(oph, q0, elems)
    R = _gather(gm, gm.residual(gph, q), elems)
    err = (np.abs(R - Ro) / (np.abs(Ro) + s[None, :, None])).max()
    assert err < TOL64, err
    # stage 0 of an SSP-RK3 step: q1 = q + dt R(q)
    dt = 1e-4
    q1 = gm.empty_state()
    gm.rk_stage(gph, 0, dt, q, q, q1)
    g1 = _gather(gm, q1, elems)
    qs = q0[:, elems].transpose(1, 0, 2)
    o1 = qs + dt * Ro
    # per-entry floor: the magnitudes that sum to q1 (the momentum of this state starts at zero)
    floor = np.abs(qs) + dt * (np.abs(Ro) + s[None, :, None])
    assert (np.abs(g1 - o1) / floor).max() < TOL64


def test_shell41k_mixed_residual_sampled():
    gm, om = _shell(24, 12)
    gph, oph = _phys()
    prm = [3.0, 0.70, 0.98, 1.0, 1.0, 1e-4, 1e-6]
    q0, qb = om.state_init(oph, sdref.INIT_SHELL_POLYTROPE, prm, seed=0, background=True)
    bg = gm.background(gph, gm.to_device(qb))
    elems = _sample(gm.n_e, seed=1)
    Ro, s = om.residual_elements(oph, q0, elems)
    R = _gather(gm, gm.residual(gph, gm.to_device(q0), prec=sdmhd.SD_FP32_MIXED, bg=bg), elems)
    ok, err, bound = _mixed_bound(R, Ro, s, label="41k residual at rest", var_axis=1)
    assert ok, (err, bound)


def test_shell221k_fp64_residual_sampled():
    gm, om = _shell(48, 16)
    gph, oph = _phys(ch=1.1)
    q0 = inputs.random_state(gm.n_e, 6, seed=3)
    elems = _sample(gm.n_e, k=32, seed=2)
    Ro, s = om.residual_elements(oph, q0, elems)
    q = gm.to_device(q0)
    del q0
    R = _gather(gm, gm.residual(gph, q), elems)
    err = (np.abs(R - Ro) / (np.abs(Ro) + s[None, :, None])).max()
    assert err < TOL64, err


def test_shell1536_hundred_fp64_steps():
    """The 1,536-element N=6 shell (N_rho = 1, GM = 1, Omega = 1, noise 1e-4 seed 0, dipole 1e-6):
    100 SSP-RK3 steps through sd_step (device dt and c_h) against the oracle stepping with its own
    lambda_max each step."""
    gm, om = _shell(8, 4)
    gph, oph = _phys(ch=0.0)
    prm = [1.0, 0.70, 0.98, 1.0, 1.0, 1e-4, 1e-6]
    q0 = om.state_init(oph, sdref.INIT_SHELL_POLYTROPE, prm, seed=0)
    q, work = gm.to_device(q0), gm.empty_state()
    xs = sdref.nodes(6)[0]
    dx = om.info()["h_min"] * (xs[1] - xs[0])
    dts = torch.zeros(2, dtype=torch.float64, device="cuda")
    qo, dt_err, t_run = q0, 0.0, 0.0
    for _ in range(100):
        gm.step(gph, 0.2, q, work, dt_out=dts)
        lam = om.diagnostics(oph, qo)["lambda_max"]
        oph.c_h = lam
        qo = om.rk_step(oph, 0.2 * dx / lam, qo)
        dt_err = max(dt_err, abs(float(dts[0]) / (0.2 * dx / lam) - 1.0))
        t_run += 0.2 * dx / lam
    change = np.abs(qo - q0).max(axis=(1, 2))
    err = np.abs(gm.to_host(q) - qo).max(axis=(1, 2))
    # The momentum is a small difference of pressure and gravity terms: the two FP64 runs part at
    # the round-off of those un-cancelled magnitudes (s_v per unit time) accumulated over the run,
    # on top of 1e-9 of the change.
    _, s = om.residual(oph, q0)
    bound = 1e-9 * change + 1e-12 * t_run * s
    assert dt_err < 1e-11 and np.all(err <= bound), (dt_err, err, bound)


def test_shell41k_mixed_advance_matches_the_oracle():
    """The benchmark's launch configuration: two FP32-mixed steps of sd_advance on the 41,472-element
    shell (fused stages, the second step taking its traces and lambda_max from the first step's last
    stage) against two oracle steps with the same dt and c_h, on every element."""
    gm, om = _shell(24, 12)
    gph, oph = _phys(ch=0.0)
    prm = [3.0, 0.70, 0.98, 1.0, 1.0, 1e-4, 1e-6]
    q0, qb = om.state_init(oph, sdref.INIT_SHELL_POLYTROPE, prm, seed=0, background=True)
    bg = gm.background(gph, gm.to_device(qb))
    del qb
    q, work = gm.to_device(q0), gm.empty_state()
    dts = torch.zeros(4, dtype=torch.float64, device="cuda")
    gm.advance(gph, 0.2, 2, q, work, prec=sdmhd.SD_FP32_MIXED, bg=bg, dt_out=dts)
    d = dts.cpu().numpy()
    qo = q0
    for k in range(2):
        oph.c_h = float(d[2 * k + 1])
        qo = om.rk_step(oph, float(d[2 * k]), qo)
    _, s = om.residual(oph, q0)
    g = gm.to_host(q)
    ok, err, bound = _mixed_bound(g - q0, qo - q0, s, floor=(), label="41k advance x2 at rest")
    assert ok, (err, bound)


def test_shell41k_mixed_advance_developed_flow():
    """As above from the same shell with a seeded flow (U ~ 1e-2 U[-1, 1]): every variable's change,
    the energy's too, within 1e-5 of its largest value."""
    gm, om = _shell(24, 12)
    gph, oph = _phys(ch=0.0)
    prm = [3.0, 0.70, 0.98, 1.0, 1.0, 1e-4, 1e-6]
    q0, qb = om.state_init(oph, sdref.INIT_SHELL_POLYTROPE, prm, seed=0, background=True)
    rng = np.random.default_rng(41)
    mom = rng.uniform(-1e-2, 1e-2, size=q0[1:4].shape) * q0[0]
    q0[1:4] += mom
    q0[4] += 0.5 * (mom ** 2).sum(axis=0) / q0[0]
    del mom
    bg = gm.background(gph, gm.to_device(qb))
    del qb
    q, work = gm.to_device(q0), gm.empty_state()
    dts = torch.zeros(4, dtype=torch.float64, device="cuda")
    gm.advance(gph, 0.2, 2, q, work, prec=sdmhd.SD_FP32_MIXED, bg=bg, dt_out=dts)
    d = dts.cpu().numpy()
    qo = q0
    for k in range(2):
        oph.c_h = float(d[2 * k + 1])
        qo = om.rk_step(oph, float(d[2 * k]), qo)
    ok, err, bound = _mixed_bound(gm.to_host(q) - q0, qo - q0, None, floor=(), label="41k advance x2 developed")
    assert ok, (err, bound)


def test_shell221k_mixed_residual_sampled():
    gm, om = _shell(48, 16)
    gph, oph = _phys()
    prm = [3.0, 0.70, 0.98, 1.0, 1.0, 1e-4, 1e-6]
    q0, qb = om.state_init(oph, sdref.INIT_SHELL_POLYTROPE, prm, seed=0, background=True)
    bg = gm.background(gph, gm.to_device(qb))
    del qb
    elems = _sample(gm.n_e, k=32, seed=3)
    Ro, s = om.residual_elements(oph, q0, elems)
    R = _gather(gm, gm.residual(gph, gm.to_device(q0), prec=sdmhd.SD_FP32_MIXED, bg=bg), elems)
    ok, err, bound = _mixed_bound(R, Ro, s, label="221k residual at rest", var_axis=1)
    assert ok, (err, bound)


VISC = dict(viscous=1, mu=0.03, eta=0.02, kappa=0.01, kappa_r=0.015, R_gas=0.9)


def _flow(q0, seed):
    """a seeded flow U ~ 1e-2 U[-1, 1] added to a state at rest (in place)"""
    rng = np.random.default_rng(seed)
    mom = rng.uniform(-1e-2, 1e-2, size=q0[1:4].shape) * q0[0]
    q0[1:4] += mom
    q0[4] += 0.5 * (mom ** 2).sum(axis=0) / q0[0]


def test_shell41k_fp64_viscous_residual_sampled():
    """The viscous FP64 residual at full size, in the benchmark's launch configuration (the viscous
    kernel, then the face-flux kernel with the common viscous flux and the element kernel over every
    element), with the viscous wall conditions, kappa_r(r) and every source on."""
    gm, om = _shell(24, 12)
    kw = dict(gamma=5.0 / 3.0, GM=1.0, omega=1.0, glm_alpha=1.0, c_h=0.8, powell=1, gravity=1, coriolis=1,
              visc_walls=1, q_bottom=0.05, T_top=0.6, kappa_r1=0.01, kappa_r2=0.005, **VISC)
    gph, oph = sdmhd.Phys(**kw), sdref.Phys(**kw)
    q0 = om.state_init(oph, sdref.INIT_SHELL_POLYTROPE, [3.0, 0.70, 0.98, 1.0, 1.0, 1e-4, 1e-3], seed=0)
    _flow(q0, 43)
    elems = _sample(gm.n_e, seed=4)
    Ro, s = om.residual_elements(oph, q0, elems)
    R = _gather(gm, gm.residual(gph, gm.to_device(q0)), elems)
    err = (np.abs(R - Ro) / (np.abs(Ro) + s[None, :, None])).max()
    assert err < TOL64, err


def test_shell41k_mixed_viscous_residual_sampled():
    """The viscous FP32-mixed residual at full size (background built with the viscous coefficients)
    with a seeded flow: every variable within 1e-5 of its largest value over the sampled elements."""
    gm, om = _shell(24, 12)
    kw = dict(gamma=5.0 / 3.0, GM=1.0, omega=1.0, glm_alpha=1.0, c_h=0.8, powell=1, gravity=1, coriolis=1,
              **VISC)
    gph, oph = sdmhd.Phys(**kw), sdref.Phys(**kw)
    prm = [3.0, 0.70, 0.98, 1.0, 1.0, 1e-4, 1e-3]
    q0, qb = om.state_init(oph, sdref.INIT_SHELL_POLYTROPE, prm, seed=0, background=True)
    _flow(q0, 44)
    bg = gm.background(gph, gm.to_device(qb))
    del qb
    elems = _sample(gm.n_e, seed=5)
    Ro, _ = om.residual_elements(oph, q0, elems)
    R = _gather(gm, gm.residual(gph, gm.to_device(q0), prec=sdmhd.SD_FP32_MIXED, bg=bg), elems)
    ok, err, bound = _mixed_bound(R, Ro, None, floor=(), label="41k viscous residual developed", var_axis=1)
    assert ok, (err, bound)


_last_dts = []  # (dt, c_h) of each step of the last _advance_vs_oracle call


def _advance_vs_oracle(gm, om, gph, oph, q0, qb, steps, cfl, stepper):
    """sd_advance of `steps` FP32-mixed steps against the oracle's steps (`stepper`) given each
    step's dt and c_h; returns (gpu change, oracle change)"""
    bg = gm.background(gph, gm.to_device(qb))
    q, work = gm.to_device(q0), gm.empty_state()
    dts = torch.zeros(2 * steps, dtype=torch.float64, device="cuda")
    gm.advance(gph, cfl, steps, q, work, prec=sdmhd.SD_FP32_MIXED, bg=bg, dt_out=dts)
    d = dts.cpu().numpy()
    _last_dts[:] = [(float(d[2 * k]), float(d[2 * k + 1])) for k in range(steps)]
    qo = q0
    for k in range(steps):
        oph.c_h = float(d[2 * k + 1])
        qo = stepper(oph, float(d[2 * k]), qo)
    return gm.to_host(q) - q0, qo - q0


def test_shell41k_mixed_ssprk53_advance_developed_flow():
    """The five-stage SSPRK(5,3) through sd_advance at full size and CFL 0.5 (the bench's ssprk53
    leg), from the shell with a seeded flow: every variable's change within 1e-5 of its largest
    value."""
    gm, om = _shell(24, 12)
    kw = dict(gamma=5.0 / 3.0, GM=1.0, omega=1.0, glm_alpha=1.0, c_h=0.0, powell=1, gravity=1, coriolis=1)
    gph, oph = sdmhd.Phys(rk_scheme=sdmhd.RK_SSP53, **kw), sdref.Phys(**kw)
    prm = [3.0, 0.70, 0.98, 1.0, 1.0, 1e-4, 1e-6]
    q0, qb = om.state_init(oph, sdref.INIT_SHELL_POLYTROPE, prm, seed=0, background=True)
    _flow(q0, 45)
    g, o = _advance_vs_oracle(gm, om, gph, oph, q0, qb, 2, 0.5, om.rk53_step)
    ok, err, bound = _mixed_bound(g, o, None, floor=(), label="41k ssprk53 x2 developed")
    assert ok, (err, bound)


def test_shell41k_mixed_viscous_advance_developed_flow():
    """The viscous FP32-mixed path through sd_advance at full size, from the shell with a seeded flow,
    at CFL 0.05 and mu = eta = kappa = kappa_r = 1e-4 (explicitly stable for the grid-scale modes of
    the flow): every variable's change within 1e-5 of its largest value, the viscous terms a visible
    part of it."""
    gm, om = _shell(24, 12)
    kw = dict(gamma=5.0 / 3.0, GM=1.0, omega=1.0, glm_alpha=1.0, c_h=0.0, powell=1, gravity=1, coriolis=1)
    visc = dict(viscous=1, mu=1e-4, eta=1e-4, kappa=1e-4, kappa_r=1e-4, R_gas=1.0)
    gph, oph = sdmhd.Phys(**kw, **visc), sdref.Phys(**kw, **visc)
    prm = [3.0, 0.70, 0.98, 1.0, 1.0, 1e-4, 1e-3]
    q0, qb = om.state_init(oph, sdref.INIT_SHELL_POLYTROPE, prm, seed=0, background=True)
    _flow(q0, 46)
    g, o = _advance_vs_oracle(gm, om, gph, oph, q0, qb, 2, 0.05, om.rk_step)
    ok, err, bound = _mixed_bound(g, o, None, floor=(), label="41k viscous x2 developed")
    assert ok, (err, bound)
    # the same two steps without the viscous terms differ visibly in the momentum
    qi = q0
    for dt, ch in _last_dts:
        qi = om.rk_step(sdref.Phys(**dict(kw, c_h=ch)), dt, qi)
    dm = np.abs(o[1:4] - (qi - q0)[1:4]).max() / np.abs(o[1:4]).max()
    assert dm > 1e-3, dm
