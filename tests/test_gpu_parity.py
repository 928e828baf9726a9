"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Inputs come from the oracle or the seeded input generators only.  Tolerances:
  FP64 residual:  |g - o| <= 1e-12 (|o| + s_v) per entry, s_v the oracle's
                  un-cancelled magnitude of variable v (sum |D F| / |J| + |M|);
  FP64 states:    1e-12 of the variable's magnitude after one stage or step;
  FP32-mixed:     max |g - o| <= 1e-5 max |o| per variable (1e-5 relative,
                  normwise per variable).  Only the variables a test names in
                  `floor` may add 4 eps32 s_v (eps32 = 2^-24): components whose
                  residual cancels to below FP32 resolution of their own terms,
                  each named with its reason at the test.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import sdref  # noqa: E402
from paper_2502_17805_gb300 import inputs, sdmhd  # noqa: E402

pytestmark = pytest.mark.gpu

ALFVEN = [1.0, 0.1, 1.0, 0.1, 2 * math.pi, 2 * math.pi, 2 * math.pi, 0.0]
TOL64 = 1e-12


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


EPS32 = 2.0 ** -24


VARS = ("rho", "mx", "my", "mz", "E", "Bx", "By", "Bz", "psi")
# The residual of the energy of a fluid at rest (U = 0): R_E is the Rusanov dissipation of face
# jumps of E that are themselves at the discretisation error (~1e-12 of E); the FP32 split into a
# rounded background and an FP32 perturbation resolves it only to a few eps32 of its terms.  Only
# the residual tests of a state at rest take this floor; every stage, step and advance test holds
# all nine variables to 1e-5 of their change outright.
AT_REST_FLOOR = (4,)


def mixed_ok(g, o, s, scale=1.0, floor=(), label=""):
    """Per-variable FP32-mixed bound max|g - o| <= 1e-5 max|o|; the variables in `floor` may add
    4 eps32 scale s_v.  g, o: (9, ...) arrays; s: (9,) un-cancelled magnitudes.  Prints the plain
    ratio max|g - o| / (1e-5 max|o|) of every variable."""
    err = np.abs(g - o).reshape(9, -1).max(axis=1)
    strict = 1e-5 * np.abs(o).reshape(9, -1).max(axis=1)
    fl = np.zeros(9)
    idx = list(floor)
    fl[idx] = 4 * EPS32 * scale * np.asarray(s, dtype=np.float64).reshape(9)[idx]
    bound = strict + fl
    ratio = err / np.maximum(strict, 1e-300)
    print("mixed %s: max|g-o|/(1e-5 max|o|) = %s; floor on %s" % (
        label, " ".join("%s %.2e" % (n, r) for n, r in zip(VARS, ratio)), [VARS[i] for i in idx]))
    return bool(np.all(err <= bound)), err, bound


def _rel_c19(g, o, s):
    return float((np.abs(g - o) / (np.abs(o) + s[:, None, None])).max())


def _rel_plain(g, o):
    """max |g - o| / max |o| per variable, no cancellation scale"""
    return np.abs(g - o).reshape(9, -1).max(axis=1) / np.maximum(np.abs(o).reshape(9, -1).max(axis=1), 1e-300)


def _residual_parity(gm, om, gph, oph, q0, plain_tol=None):
    R = gm.to_host(gm.residual(gph, gm.to_device(q0)))
    torch.cuda.synchronize()
    Ro, s = om.residual(oph, q0)
    plain = _rel_plain(R, Ro)
    print("fp64 residual: c19 %.2e, plain per variable %s" % (_rel_c19(R, Ro, s), " ".join("%.1e" % x for x in plain)))
    if plain_tol is not None:
        assert plain.max() < plain_tol, plain
    return _rel_c19(R, Ro, s)


@pytest.mark.parametrize("N", [2, 3, 4, 5, 6, 7, 8])
def test_residual_box_alfven_all_orders(N):
    v, h, per = inputs.box_mesh(3, jitter=0.1, seed=N)
    gm, om = _pair(N, v, inputs.reorient(h, seed=N), periodic=per, geom=0)
    gph, oph = _phys(powell=1, c_h=0.8, glm_alpha=0.3)
    q0 = om.state_init(oph, sdref.INIT_ALFVEN, ALFVEN)
    # the wave's rho, E and psi residuals vanish up to the discretisation error (k.U = 0, U.B and
    # |B| uniform): only the c19 measure applies to them, the plain one is printed
    assert _residual_parity(gm, om, gph, oph, q0) < TOL64


def test_residual_random_state_box():
    N = 5
    v, h, per = inputs.box_mesh(4, jitter=0.15, seed=3)
    gm, om = _pair(N, v, inputs.reorient(h, seed=4), periodic=per, geom=0)
    gph, oph = _phys(powell=1, c_h=0.6, glm_alpha=0.4)
    q0 = inputs.random_state(gm.n_e, N, seed=11)
    assert _residual_parity(gm, om, gph, oph, q0, plain_tol=TOL64) < TOL64


@pytest.mark.parametrize("N", [2, 3, 4, 5, 6, 7, 8])
def test_residual_shell_walls_all_sources(N):
    v, h = inputs.shell_mesh(3, 2)
    h = inputs.reorient(h, seed=5)
    gm, om = _pair(N, v, h, geom=1, r_in=0.7, r_out=0.98, bc_in=sdref.BC_WALL_CONDUCTING,
                   bc_out=sdref.BC_WALL_RADIAL)
    gph, oph = _phys(powell=1, c_h=0.9, glm_alpha=0.5, gravity=1, GM=1.0, coriolis=1, omega=1.3)
    q0 = inputs.random_state(gm.n_e, N, seed=6)
    assert _residual_parity(gm, om, gph, oph, q0, plain_tol=TOL64) < TOL64
    q1 = om.state_init(oph, sdref.INIT_SHELL_POLYTROPE, [2.0, 0.7, 0.98, 1.0, 1.0, 1e-4, 1e-3], seed=3)
    assert _residual_parity(gm, om, gph, oph, q1) < TOL64


def test_free_stream_on_shell():
    N = 6
    v, h = inputs.shell_mesh(2, 2)
    h = inputs.reorient(h, seed=8)
    gm, om = _pair(N, v, h, geom=1, r_in=0.7, r_out=0.98, bc_in=sdref.BC_FARFIELD, bc_out=sdref.BC_FARFIELD)
    gph, oph = _phys(powell=1, c_h=0.9)
    q0 = om.state_init(oph, sdref.INIT_UNIFORM, [1.0, 0.3, -0.2, 0.1, 0.5, 0.4, 0.2, -0.3, 0.0])
    gph.farfield = oph.farfield = list(q0[:, 0, 0])
    R = gm.to_host(gm.residual(gph, gm.to_device(q0)))
    _, s = om.residual(oph, q0)
    for var in range(9):
        assert np.abs(R[var]).max() <= 1e-13 * s[var]


def test_mixed_free_stream_on_shell():
    """FP32-mixed path, far-field walls: a uniform flowing, magnetised state about the uniform
    background of its own density and pressure (gravity off) has a residual at FP32 rounding of the
    un-cancelled terms (the background residual vanishes by the metric identity, the perturbation
    flux is uniform, and the far-field ghost is the same state)."""
    N = 6
    v, h = inputs.shell_mesh(2, 2)
    h = inputs.reorient(h, seed=8)
    gm, om = _pair(N, v, h, geom=1, r_in=0.7, r_out=0.98, bc_in=sdref.BC_FARFIELD, bc_out=sdref.BC_FARFIELD)
    gph, oph = _phys(powell=1, c_h=0.9)
    q0 = om.state_init(oph, sdref.INIT_UNIFORM, [1.0, 0.3, -0.2, 0.1, 0.5, 0.4, 0.2, -0.3, 0.0])
    gph.farfield = oph.farfield = list(q0[:, 0, 0])
    qb = np.zeros_like(q0)
    qb[0] = q0[0]
    qb[4] = 0.5 / (5.0 / 3.0 - 1.0)  # p = 0.5 (INIT_UNIFORM parameter 4)
    bg = gm.background(gph, gm.to_device(qb))
    R = gm.to_host(gm.residual(gph, gm.to_device(q0), prec=sdmhd.SD_FP32_MIXED, bg=bg))
    _, s = om.residual(oph, q0)
    ratio = np.abs(R).reshape(9, -1).max(axis=1) / (EPS32 * s)
    assert np.all(ratio <= 8.0), ratio


def test_conservation_is_exact_on_periodic_box():
    N = 5
    v, h, per = inputs.box_mesh(3, jitter=0.15, seed=2)
    gm, om = _pair(N, v, inputs.reorient(h, seed=9), periodic=per, geom=0)
    gph, oph = _phys(powell=0, c_h=0.6)
    q0 = inputs.random_state(gm.n_e, N, seed=5)
    R = gm.to_host(gm.residual(gph, gm.to_device(q0)))
    w = sdref.nodes(N)[4]
    W = np.einsum("i,j,k->kji", w, w, w).ravel()
    J = np.stack([om.geometry(e)[1] for e in range(om.n_e)])
    tot = (R * W * J).sum(axis=(1, 2))
    mag = (np.abs(R) * W * J).sum(axis=(1, 2))
    assert np.all(np.abs(tot) <= 1e-13 * mag), tot / mag


def test_rk_stages_individually():
    N = 4
    v, h, per = inputs.box_mesh(3, jitter=0.1, seed=7)
    gm, om = _pair(N, v, inputs.reorient(h, seed=7), periodic=per, geom=0)
    gph, oph = _phys(powell=1, c_h=0.7, glm_alpha=0.2)
    qn = inputs.random_state(gm.n_e, N, seed=1)
    qi = inputs.random_state(gm.n_e, N, seed=2)
    dt = 2e-3
    for stage in range(3):
        g_out = gm.empty_state()
        gm.rk_stage(gph, stage, dt, gm.to_device(qn), gm.to_device(qi), g_out)
        o_out = om.rk_stage(oph, stage, dt, qn, qi)
        err = np.abs(gm.to_host(g_out) - o_out).max(axis=(1, 2)) / np.abs(o_out).max(axis=(1, 2))
        assert err.max() < TOL64, (stage, err)


def test_alfven_box_twenty_steps_fp64():
    """The periodic Alfven-wave box at N = 6: 20 SSP-RK3 steps at CFL 0.2, dt and c_h from lambda_max."""
    N, cfl = 6, 0.2
    v, h, per = inputs.box_mesh(4)
    gm, om = _pair(N, v, h, periodic=per, geom=0)
    gph, oph = _phys(powell=1, c_h=0.0, glm_alpha=0.0)
    q0 = om.state_init(oph, sdref.INIT_ALFVEN, ALFVEN)
    q, work = gm.to_device(q0), gm.empty_state()
    dts = torch.zeros(2, dtype=torch.float64, device="cuda")
    xs = sdref.nodes(N)[0]
    dx_min = om.info()["h_min"] * (xs[1] - xs[0])
    qo = q0
    dt_err = 0.0
    for _ in range(20):
        gm.step(gph, cfl, q, work, dt_out=dts)
        lam = om.diagnostics(oph, qo)["lambda_max"]
        oph.c_h = lam
        qo = om.rk_step(oph, cfl * dx_min / lam, qo)
        dt_err = max(dt_err, abs(dts.cpu().numpy()[0] / (cfl * dx_min / lam) - 1.0))
    # psi stays at the rounding-driven level of the discrete div B (~1e-6): measure it against |B|
    scale = np.abs(qo).max(axis=(1, 2))
    scale[8] = np.abs(qo[5:8]).max()
    err = np.abs(gm.to_host(q) - qo).max(axis=(1, 2)) / scale
    print("dt rel err %.2e, state rel err %s" % (dt_err, err))
    assert dt_err < 1e-12 and err.max() < 1e-11, (dt_err, err)


def test_state_init_parity():
    N = 5
    v, h = inputs.shell_mesh(3, 2)
    gm, om = _pair(N, v, h, geom=1, r_in=0.7, r_out=0.98)
    gph, oph = _phys(gravity=1, GM=1.0)
    prm = [3.0, 0.7, 0.98, 1.0, 1.0, 1e-4, 1e-6]
    bg = gm.empty_state()
    q = gm.state_init(gph, sdmhd.INIT_SHELL_POLYTROPE, prm, seed=7, background=bg)
    qo, qbo = om.state_init(oph, sdref.INIT_SHELL_POLYTROPE, prm, seed=7, background=True)
    for g, o in ((gm.to_host(q), qo), (gm.to_host(bg), qbo)):
        scale = np.maximum(np.abs(o).max(axis=(1, 2)), 1e-300)
        assert (np.abs(g - o).max(axis=(1, 2)) / scale).max() < TOL64
    v2, h2, per = inputs.box_mesh(3, jitter=0.1, seed=1)
    gm2, om2 = _pair(N, v2, h2, periodic=per, geom=0)
    qa = gm2.to_host(gm2.state_init(gph, sdmhd.INIT_ALFVEN, ALFVEN))
    qao = om2.state_init(oph, sdref.INIT_ALFVEN, ALFVEN)
    assert np.abs(qa - qao).max() < 1e-13


def test_diagnostics_parity():
    N = 5
    v, h = inputs.shell_mesh(3, 2)
    gm, om = _pair(N, v, inputs.reorient(h, seed=2), geom=1, r_in=0.7, r_out=0.98)
    gph, oph = _phys(gravity=1, GM=1.0, powell=1)
    q0 = inputs.random_state(gm.n_e, N, seed=3)
    g = gm.diagnostics(gph, gm.to_device(q0))
    o = om.diagnostics(oph, q0)
    for k in ("ke", "eb", "max_divb", "mass", "energy", "lambda_max", "min_rho", "min_p", "volume"):
        assert abs(g[k] - o[k]) <= 1e-12 * abs(o[k]), (k, g[k], o[k])


def test_diagnostics_flags_nonphysical_state():
    N = 3
    v, h, per = inputs.box_mesh(3)
    gm = sdmhd.Mesh(N, v, h, periodic=per, geom=0)
    q0 = inputs.random_state(gm.n_e, N, seed=3)
    q0[0, 4, 5] = -1.0  # negative density planted on the host
    d = gm.diagnostics(sdmhd.Phys(), gm.to_device(q0), check=False)
    assert d["status"] == 7 and d["min_rho"] == -1.0


def _mixed_case(nz, nr, N, Nrho, seed=0):
    v, h = inputs.shell_mesh(nz, nr)
    gm, om = _pair(N, v, h, geom=1, r_in=0.7, r_out=0.98, bc_in=sdref.BC_WALL_CONDUCTING,
                   bc_out=sdref.BC_WALL_RADIAL)
    gph, oph = _phys(powell=1, c_h=1.0, glm_alpha=0.5, gravity=1, GM=1.0, coriolis=1, omega=1.0)
    prm = [Nrho, 0.7, 0.98, 1.0, 1.0, 1e-4, 1e-6]
    q0, qb = om.state_init(oph, sdref.INIT_SHELL_POLYTROPE, prm, seed=seed, background=True)
    return gm, om, gph, oph, q0, qb


@pytest.mark.parametrize("N", [2, 3, 4, 5, 6, 7, 8])
def test_mixed_residual_stratified_shell(N):
    gm, om, gph, oph, q0, qb = _mixed_case(4 if N <= 6 else 3, 2, N, 3.0)
    bg = gm.background(gph, gm.to_device(qb))
    R = gm.to_host(gm.residual(gph, gm.to_device(q0), prec=sdmhd.SD_FP32_MIXED, bg=bg))
    Ro, s = om.residual(oph, q0)
    ok, err, bound = mixed_ok(R, Ro, s, floor=AT_REST_FLOOR, label="residual at rest N=%d" % N)
    assert ok, (err, bound)


@pytest.mark.parametrize("N", [2, 3, 4, 5, 6, 7, 8])
def test_mixed_residual_random_background_periodic_box(N):
    """FP32-mixed residual about a non-uniform, non-hydrostatic background on a jittered, reoriented
    periodic box: the background jumps across every interior and periodic face (each side's flux is
    taken about its own background), there are no walls, and R0 carries the background's residual."""
    v, h, per = inputs.box_mesh(3, jitter=0.15, seed=N)
    gm, om = _pair(N, v, inputs.reorient(h, seed=N), periodic=per, geom=0)
    gph, oph = _phys(powell=1, c_h=0.7, glm_alpha=0.3)
    q0 = inputs.random_state(gm.n_e, N, seed=40 + N)
    src = inputs.random_state(gm.n_e, N, seed=80 + N)
    qb = np.zeros_like(q0)
    qb[0] = src[0]          # rho0 in [0.8, 1.2]
    qb[4] = 0.8 * src[4]    # E0 = p0 / (gamma - 1) in [1.2, 2.0]
    bg = gm.background(gph, gm.to_device(qb))
    R = gm.to_host(gm.residual(gph, gm.to_device(q0), prec=sdmhd.SD_FP32_MIXED, bg=bg))
    Ro, s = om.residual(oph, q0)
    ok, err, bound = mixed_ok(R, Ro, s, label="residual random background N=%d" % N)
    assert ok, (err, bound)


@pytest.mark.parametrize("N", [3, 6, 8])
def test_mixed_residual_developed_flow_strict(N):
    """With a seeded velocity field on the stratified shell every component of the residual is far
    above FP32 resolution; there the mixed path meets 1e-5 relative per variable outright."""
    gm, om, gph, oph, q0, qb = _mixed_case(4 if N <= 6 else 3, 2, N, 3.0, seed=2)
    rng = np.random.default_rng(17)
    q1 = q0.copy()
    q1[1:4] += rng.uniform(-1e-2, 1e-2, size=q1[1:4].shape) * q1[0]
    bg = gm.background(gph, gm.to_device(qb))
    R = gm.to_host(gm.residual(gph, gm.to_device(q1), prec=sdmhd.SD_FP32_MIXED, bg=bg))
    Ro, _ = om.residual(oph, q1)
    err = np.abs(R - Ro).max(axis=(1, 2)) / np.abs(Ro).max(axis=(1, 2))
    assert err.max() <= 1e-5, err


@pytest.mark.parametrize("N", [2, 3, 4, 5, 6, 7, 8])
def test_mixed_stage_stratified_shell(N):
    """sd_rk_stage on the FP32-mixed path (the q^n form with FP64 stage states, the FP64 state
    loaded and converted in the kernel) against the oracle's RK step."""
    gm, om, gph, oph, q0, qb = _mixed_case(3, 2, N, 2.0, seed=4)
    bg = gm.background(gph, gm.to_device(qb))
    dt = 1e-3
    q, work = gm.to_device(q0), gm.empty_state()
    gm.rk_step(gph, dt, q, work, prec=sdmhd.SD_FP32_MIXED, bg=bg)
    qo = om.rk_step(oph, dt, q0)
    # compare the change over the step, per variable (three stages of dt R)
    _, s = om.residual(oph, q0)
    ok, err, bound = mixed_ok(gm.to_host(q) - q0, qo - q0, s, label="rk_stage step N=%d" % N)
    assert ok, (err, bound)


def test_step_equals_three_stages():
    N = 4
    v, h = inputs.shell_mesh(2, 2)
    gm = sdmhd.Mesh(N, v, h, geom=1, r_in=0.7, r_out=0.98)
    gph = sdmhd.Phys(powell=1, c_h=0.0, glm_alpha=0.5, gravity=1, GM=1.0, coriolis=1, omega=1.0)
    q0 = inputs.random_state(gm.n_e, N, seed=12)
    qa, wa = gm.to_device(q0), gm.empty_state()
    dts = torch.zeros(2, dtype=torch.float64, device="cuda")
    gm.step(gph, 0.3, qa, wa, dt_out=dts)
    dt, ch = dts.cpu().numpy()
    gph.c_h = float(ch)
    qb, wb = gm.to_device(q0), gm.empty_state()
    gm.rk_step(gph, float(dt), qb, wb)
    assert torch.equal(qa, qb)


@pytest.mark.parametrize("N", [2, 3, 4, 5, 6, 7, 8])
def test_mixed_sd_step_low_storage_matches_oracle(N):
    """sd_step on the FP32-mixed path (the stored FP32 q' of q^n and the FP32 difference register
    instead of q^n: bulk-copied for even N, loaded for odd N) follows the FP64 oracle over three
    steps, given each step's dt and c_h."""
    gm, om, gph, oph, q0, qb = _mixed_case(3, 2, N, 2.5, seed=9)
    bg = gm.background(gph, gm.to_device(qb))
    gph.c_h = 0.0  # c_h = lambda_max each step
    q, work = gm.to_device(q0), gm.empty_state()
    dts = torch.zeros(2, dtype=torch.float64, device="cuda")
    qo = q0
    for _ in range(3):
        gm.step(gph, 0.2, q, work, prec=sdmhd.SD_FP32_MIXED, bg=bg, dt_out=dts)
        dt, ch = dts.cpu().numpy()
        oph.c_h = float(ch)
        qo = om.rk_step(oph, float(dt), qo)
    _, s = om.residual(oph, q0)
    ok, err, bound = mixed_ok(gm.to_host(q) - q0, qo - q0, s, label="sd_step x3 N=%d" % N)
    assert ok, (err, bound)


def _developed(q0, seed=17, amp=1e-2):
    """q0 with a seeded velocity field U ~ amp U[-1, 1] per component (momentum rho U): every residual
    component, B and psi included (the induction of the seed field), is far above FP32 resolution"""
    rng = np.random.default_rng(seed)
    q1 = q0.copy()
    mom = rng.uniform(-amp, amp, size=q1[1:4].shape) * q1[0]
    q1[1:4] += mom
    q1[4] += 0.5 * (mom ** 2).sum(axis=0) / q1[0]  # kinetic energy of the added flow, pressure unchanged
    return q1


@pytest.mark.parametrize("N", [2, 3, 4, 5, 6, 7, 8])
def test_mixed_sd_step_developed_flow_strict(N):
    """Three FP32-mixed sd_step steps from the stratified shell with a seeded flow: every variable's
    change over the steps within 1e-5 of its largest value, no floor."""
    gm, om, gph, oph, q0, qb = _mixed_case(3, 2, N, 2.5, seed=9)
    q0 = _developed(q0, seed=N)
    bg = gm.background(gph, gm.to_device(qb))
    gph.c_h = 0.0
    q, work = gm.to_device(q0), gm.empty_state()
    dts = torch.zeros(2, dtype=torch.float64, device="cuda")
    qo = q0
    for _ in range(3):
        gm.step(gph, 0.2, q, work, prec=sdmhd.SD_FP32_MIXED, bg=bg, dt_out=dts)
        dt, ch = dts.cpu().numpy()
        oph.c_h = float(ch)
        qo = om.rk_step(oph, float(dt), qo)
    _, s = om.residual(oph, q0)
    ok, err, bound = mixed_ok(gm.to_host(q) - q0, qo - q0, s, label="sd_step x3 developed N=%d" % N)
    assert ok, (err, bound)


@pytest.mark.parametrize("prec,N", [("fp64", 5), ("fp64", 6)] + [("mixed", n) for n in range(2, 9)])
def test_advance_equals_repeated_steps(prec, N):
    """sd_advance takes the traces and lambda_max of each step's start state from the last stage of
    the step before instead of a trace pass; the states and (dt, c_h) are the same bits as sd_step
    called once per step."""
    gm, om, gph, oph, q0, qb = _mixed_case(3, 2, N, 2.0, seed=6)
    gph.c_h = 0.0
    kw = dict(prec=sdmhd.SD_FP32_MIXED, bg=gm.background(gph, gm.to_device(qb))) if prec == "mixed" else {}
    K = 4
    qa, wa = gm.to_device(q0), gm.empty_state()
    da = torch.zeros(2 * K, dtype=torch.float64, device="cuda")
    for k in range(K):
        gm.step(gph, 0.2, qa, wa, dt_out=da[2 * k: 2 * k + 2], **kw)
    qb_, wb = gm.to_device(q0), gm.empty_state()
    db = torch.zeros(2 * K, dtype=torch.float64, device="cuda")
    gm.advance(gph, 0.2, K, qb_, wb, dt_out=db, **kw)
    torch.cuda.synchronize()
    assert torch.equal(da, db) and torch.equal(qa, qb_)
    assert not torch.equal(qa, gm.to_device(q0))
    # zero steps leave the state alone
    qc = qb_.clone()
    gm.advance(gph, 0.2, 0, qc, wb, **kw)
    assert torch.equal(qc, qb_)


@pytest.mark.parametrize("kr", [(0.01,), (0.004, 0.01, -0.003)])
def test_flux_balanced_state_and_mixed_residual(kr):
    """The almost flux-balanced initial state (host-integrated radial table, interpolated on the
    device) against the oracle's, with a constant or a radius-dependent kappa_r, and the FP32-mixed
    residual around it as background."""
    N = 5
    v, h = inputs.shell_mesh(3, 2)
    gm, om = _pair(N, v, h, geom=1, r_in=0.7, r_out=0.98, bc_in=sdref.BC_WALL_CONDUCTING,
                   bc_out=sdref.BC_WALL_RADIAL)
    gph, oph = _phys(powell=1, c_h=1.0, glm_alpha=0.5, gravity=1, GM=1.0, coriolis=1, omega=1.0)
    prm = [3.0, 0.7, 0.98, 1.0, 1.0, 1e-4, 1e-6, 0.02, 0.05] + list(kr)
    q0, qb = om.state_init(oph, sdref.INIT_SHELL_FLUX_BALANCED, prm, seed=3, background=True)
    gb = gm.empty_state()
    gq = gm.state_init(gph, sdmhd.INIT_SHELL_FLUX_BALANCED, prm, seed=3, background=gb)
    for g, o in ((gm.to_host(gq), q0), (gm.to_host(gb), qb)):
        scale = np.abs(o).reshape(9, -1).max(axis=1)
        err = np.abs(g - o).reshape(9, -1).max(axis=1)
        assert np.all(err <= 1e-12 * np.maximum(scale, 1e-300)), (err, scale)
    bg = gm.background(gph, gm.to_device(qb))
    R = gm.to_host(gm.residual(gph, gm.to_device(q0), prec=sdmhd.SD_FP32_MIXED, bg=bg))
    Ro, s = om.residual(oph, q0)
    ok, err, bound = mixed_ok(R, Ro, s, floor=AT_REST_FLOOR, label="residual flux-balanced")
    assert ok, (err, bound)


def test_flux_balanced_profile_that_turns_negative_is_refused():
    """A radiative diffusivity large enough that the profile's density integrates through zero is an
    invalid argument, not a state with NaNs."""
    N = 4
    v, h = inputs.shell_mesh(2, 1)
    gm = sdmhd.Mesh(N, v, h, geom=1, r_in=0.7, r_out=0.98)
    gph = sdmhd.Phys(gravity=1, GM=1.0)
    prm = [3.0, 0.7, 0.98, 1.0, 1.0, 1e-4, 1e-6, 0.02, 0.05, 0.01, 0.012, -0.004]
    with pytest.raises(sdmhd.SDError, match="positive and finite"):
        gm.state_init(gph, sdmhd.INIT_SHELL_FLUX_BALANCED, prm, seed=0)
