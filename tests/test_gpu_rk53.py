"""The five-stage third-order SSP method (sd_phys.rk_scheme = RK_SSP53; SSPRK(5,3), reading R23)
through sd_step and sd_advance, against the oracle's step (sdref_rk53_step) given each step's dt and
c_h: FP64 within 1e-11 of the state, FP32-mixed within 1e-5 of each variable's change."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import sdref  # noqa: E402
from paper_2502_17805_gb300 import inputs, sdmhd  # noqa: E402

pytestmark = pytest.mark.gpu

ALFVEN = [1.0, 0.1, 1.0, 0.1, 2 * math.pi, 2 * math.pi, 2 * math.pi, 0.0]
VARS = ("rho", "mx", "my", "mz", "E", "Bx", "By", "Bz", "psi")
R_SSP = 2.6506291914393882


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
    return sdmhd.Phys(rk_scheme=sdmhd.RK_SSP53, **kw), sdref.Phys(**kw)


def _strict(g, o, label):
    """every variable within 1e-5 of its largest value in o (the change of the state)"""
    err = np.abs(g - o).reshape(9, -1).max(axis=1)
    ref = 1e-5 * np.abs(o).reshape(9, -1).max(axis=1)
    print("ssp53 %s: max|g-o|/(1e-5 max|o|) = %s" % (
        label, " ".join("%s %.2e" % (n, r) for n, r in zip(VARS, err / np.maximum(ref, 1e-300)))))
    return bool(np.all(err <= ref)), err, ref


def _shell(N, Nrho=2.5, seed=9, flow=True):
    v, h = inputs.shell_mesh(3, 2)
    gm, om = _pair(N, v, inputs.reorient(h, seed=seed), geom=1, r_in=0.7, r_out=0.98,
                   bc_in=sdref.BC_WALL_CONDUCTING, bc_out=sdref.BC_WALL_RADIAL)
    gph, oph = _phys(powell=1, c_h=0.0, glm_alpha=0.5, gravity=1, GM=1.0, coriolis=1, omega=1.0)
    prm = [Nrho, 0.7, 0.98, 1.0, 1.0, 1e-4, 1e-6]
    q0, qb = om.state_init(oph, sdref.INIT_SHELL_POLYTROPE, prm, seed=seed, background=True)
    if flow:  # a seeded flow, so that every component of the change is far above FP32 resolution
        rng = np.random.default_rng(seed)
        mom = rng.uniform(-1e-2, 1e-2, size=q0[1:4].shape) * q0[0]
        q0[1:4] += mom
        q0[4] += 0.5 * (mom ** 2).sum(axis=0) / q0[0]
    return gm, om, gph, oph, q0, qb


def _follow(gm, om, gph, oph, q0, steps, cfl, **kw):
    """sd_step `steps` times; the oracle's step with each step's dt and c_h"""
    q, work = gm.to_device(q0), gm.empty_state()
    dts = torch.zeros(2, dtype=torch.float64, device="cuda")
    qo = q0
    for _ in range(steps):
        gm.step(gph, cfl, q, work, dt_out=dts, **kw)
        dt, ch = dts.cpu().numpy()
        oph.c_h = float(ch)
        qo = om.rk53_step(oph, float(dt), qo)
    return gm.to_host(q), qo


def test_fp64_alfven_box():
    """The periodic Alfven-wave box at N = 6: 8 steps at CFL 0.5 (within r times the three-stage
    method's 0.2), dt and c_h from lambda_max on the device."""
    N, cfl = 6, 0.5
    v, h, per = inputs.box_mesh(4)
    gm, om = _pair(N, v, h, periodic=per, geom=0)
    gph, oph = _phys(powell=1, c_h=0.0, glm_alpha=0.0)
    q0 = om.state_init(oph, sdref.INIT_ALFVEN, ALFVEN)
    g, o = _follow(gm, om, gph, oph, q0, 8, cfl)
    scale = np.abs(o).max(axis=(1, 2))
    scale[8] = np.abs(o[5:8]).max()  # psi stays at the rounding level of the discrete div B
    err = np.abs(g - o).max(axis=(1, 2)) / scale
    print("ssp53 fp64 alfven: state rel err %s" % err)
    assert err.max() < 1e-11, err
    # the wave moved: the step is not a no-op
    assert np.abs(o - q0).max() > 1e-3


@pytest.mark.parametrize("N", [3, 4])
def test_fp64_stratified_shell(N):
    gm, om, gph, oph, q0, _ = _shell(N)
    g, o = _follow(gm, om, gph, oph, q0, 3, 0.5)
    err = np.abs(g - o).reshape(9, -1).max(axis=1) / np.abs(o - q0).reshape(9, -1).max(axis=1)
    print("ssp53 fp64 shell N=%d: max|g-o| / max|change| = %s" % (N, err))
    assert err.max() < 1e-9, err


@pytest.mark.parametrize("N", [2, 3, 4, 5, 6, 7, 8])
def test_mixed_steps_follow_the_oracle(N):
    """Three FP32-mixed steps (increment form; stage 2 leaves W = a61 D2 + a62 D3 in a second FP32
    register, the last stage adds its increment to q^n + W) on the stratified shell with a flow."""
    gm, om, gph, oph, q0, qb = _shell(N)
    bg = gm.background(gph, gm.to_device(qb))
    g, o = _follow(gm, om, gph, oph, q0, 3, 0.5, prec=sdmhd.SD_FP32_MIXED, bg=bg)
    ok, err, ref = _strict(g - q0, o - q0, "mixed x3 N=%d" % N)
    assert ok, (err, ref)


def test_mixed_viscous_steps_follow_the_oracle():
    """The viscous, resistive and thermal fluxes on the mixed path under the five-stage method: the
    gradient and viscous-residual kernels run on each of the five stage states."""
    N = 4
    v, h, per = inputs.box_mesh(3, jitter=0.15, seed=14)
    gm, om = _pair(N, v, inputs.reorient(h, seed=14), periodic=per, geom=0)
    visc = dict(viscous=1, mu=0.03, eta=0.02, kappa=0.01, kappa_r=0.015, R_gas=0.9)
    gph, oph = _phys(powell=1, c_h=0.0, glm_alpha=0.3, **visc)
    q0 = inputs.random_state(gm.n_e, N, seed=64)
    src = inputs.random_state(gm.n_e, N, seed=104)
    qb = np.zeros_like(q0)
    qb[0] = src[0]
    qb[4] = 0.8 * src[4]
    bg = gm.background(gph, gm.to_device(qb))
    g, o = _follow(gm, om, gph, oph, q0, 3, 0.1, prec=sdmhd.SD_FP32_MIXED, bg=bg)
    ok, err, ref = _strict(g - q0, o - q0, "mixed viscous x3")
    assert ok, (err, ref)


@pytest.mark.parametrize("prec,N", [("fp64", 5), ("mixed", 4), ("mixed", 6)])
def test_advance_equals_repeated_steps(prec, N):
    """sd_advance under the five-stage method gives the same bits as sd_step once per step."""
    gm, om, gph, oph, q0, qb = _shell(N, seed=6, flow=False)
    kw = dict(prec=sdmhd.SD_FP32_MIXED, bg=gm.background(gph, gm.to_device(qb))) if prec == "mixed" else {}
    K = 3
    qa, wa = gm.to_device(q0), gm.empty_state()
    da = torch.zeros(2 * K, dtype=torch.float64, device="cuda")
    for k in range(K):
        gm.step(gph, 0.5, qa, wa, dt_out=da[2 * k: 2 * k + 2], **kw)
    qb_, wb = gm.to_device(q0), gm.empty_state()
    db = torch.zeros(2 * K, dtype=torch.float64, device="cuda")
    gm.advance(gph, 0.5, K, qb_, wb, dt_out=db, **kw)
    torch.cuda.synchronize()
    assert torch.equal(da, db) and torch.equal(qa, qb_)
    assert not torch.equal(qa, gm.to_device(q0))


def test_refusals():
    N = 3
    gm, om, gph, oph, q0, qb = _shell(N, flow=False)
    q = gm.to_device(q0)
    with pytest.raises(sdmhd.SDError) as exc:  # sd_rk_stage runs the three-stage stages only
        gm.rk_stage(gph, 0, 1e-3, q, q, gm.empty_state())
    assert exc.value.code == 2
    bad = sdmhd.Phys(**dict(vars(gph), rk_scheme=7))
    with pytest.raises(sdmhd.SDError) as exc:
        gm.step(bad, 0.2, q, gm.empty_state())
    assert exc.value.code == 1


def test_fp64_viscous_walls_steps_follow_the_oracle():
    """The FP64 path with the viscous fluxes and the wall conditions of the viscous path under the
    five-stage method (its stages run with dt / r)."""
    N = 4
    v, h = inputs.shell_mesh(2, 2)
    gm, om = _pair(N, v, inputs.reorient(h, seed=7), geom=1, r_in=0.7, r_out=0.98,
                   bc_in=sdref.BC_WALL_CONDUCTING, bc_out=sdref.BC_WALL_RADIAL)
    walls = dict(viscous=1, mu=0.03, eta=0.02, kappa=0.01, kappa_r=0.015, R_gas=0.9, visc_walls=1,
                 q_bottom=0.05, T_top=0.6)
    gph, oph = _phys(powell=1, c_h=0.0, glm_alpha=0.5, gravity=1, GM=1.0, coriolis=1, omega=1.0, **walls)
    prm = [2.0, 0.7, 0.98, 1.0, 0.9, 1e-4, 1e-3]
    q0 = om.state_init(oph, sdref.INIT_SHELL_POLYTROPE, prm, seed=8)
    g, o = _follow(gm, om, gph, oph, q0, 2, 0.1)
    err = np.abs(g - o).reshape(9, -1).max(axis=1) / np.abs(o - q0).reshape(9, -1).max(axis=1)
    print("ssp53 fp64 viscous walls: max|g-o| / max|change| = %s" % err)
    assert err.max() < 1e-9, err
