"""Pins of the oracle's fluid-particle forces (CPU only)."""
import math

import numpy as np
import pytest

from paper_1601_03801_gb300.workloads import default_params

RHO = 2500.0


def single(oracle_mod, p, x, v, d=1e-3):
    o = oracle_mod.Oracle(p)
    o.set_particles(np.array([x]), np.array([v]), np.zeros((1, 3)), np.array([d]), np.array([RHO]))
    return o


def free_fall_params(**over):
    p = default_params(lubrication=0, periodic=(1, 1, 1), wall_lo=(0, 0, 0), wall_hi=(0, 0, 0),
                       lo=(0, 0, 0), hi=(0.02, 0.02, 0.02), ncell=(4, 4, 4))
    p.update(over)
    return p


def terminal_velocity(d, rho_p, rho_f, nu, g=9.81):
    """Closed-form settling speed of the drag law at eps_f = 1 (V_r = 1)."""
    K = 4.0 / 3.0 * (rho_p / rho_f - 1.0) * g * d
    a = 4.8 * math.sqrt(nu / d)
    s = (-a + math.sqrt(a * a + 2.52 * math.sqrt(K))) / 1.26
    return s * s


@pytest.mark.parametrize("d", [1e-3, 0.5e-3])
def test_p3_terminal_settling(oracle_mod, d):
    """P3: a sphere released in quiescent water reaches the closed-form terminal
    velocity of the drag law (eps_s = 0, no lubrication)."""
    p = free_fall_params(dt=2e-5)
    o = single(oracle_mod, p, [0.01, 0.01, 0.01], [0, 0, 0], d)
    o.step(20000)
    _, v, _, a = o.get_particles()
    vt = terminal_velocity(d, RHO, 1000.0, 1e-6)
    assert abs(-v[0, 2] / vt - 1) < 1e-4
    assert abs(a[0, 2]) < 1e-3 * 9.81
    if d == 1e-3:
        assert 0.125 < vt < 0.145


def test_p3_added_mass_initial_acceleration(oracle_mod):
    """P3b: from rest, the lagged added-mass force drives the acceleration to the
    fixed point (rho_p - rho_f) g / (rho_p + C_add rho_f)."""
    p = free_fall_params(dt=1e-6)
    o = single(oracle_mod, p, [0.01, 0.01, 0.01], [0, 0, 0])
    o.step(12)
    _, _, _, a = o.get_particles()
    expect = -(RHO - 1000.0) * 9.81 / (RHO + 0.5 * 1000.0)
    assert abs(a[0, 2] / expect - 1) < 1e-4
    o2 = single(oracle_mod, dict(p, added_mass=0), [0.01, 0.01, 0.01], [0, 0, 0])
    o2.step(1)
    _, _, _, a2 = o2.get_particles()
    assert abs(a2[0, 2] / (-(RHO - 1000.0) * 9.81 / RHO) - 1) < 1e-9


def test_p9_drag_identities(oracle_mod):
    """P9: V_r = 1 at eps_f = 1 for every Re; the A2 branches meet at 0.85; at
    eps_f = 1 the drag is (1/2) rho C_d (pi d^2/4) |w| w with the Dalla Valle C_d,
    points along the slip w = U - u, and tends to 0.96 x Stokes at small Re."""
    p = default_params()
    for Re in (0.0, 1e-3, 1.0, 50.0, 1e4):
        assert abs(oracle_mod.vr(1.0, Re) - 1.0) < 1e-12
    assert abs(0.8 * 0.85 ** 1.28 - 0.85 ** 2.65) < 1e-3
    # the two branches bracket the switch: values just below/above 0.85 are close
    assert abs(oracle_mod.vr(0.85, 10.0) - oracle_mod.vr(0.850001, 10.0)) < 1e-3
    d = 1e-3
    for wmag in (1e-4, 0.01, 0.3):
        w = np.array([0.6, -0.8, 0.0]) * wmag
        f, vr, cdw = oracle_mod.drag(p, 0.0, w, d)
        Re = d * wmag / p["nu_f"]
        Cd = (0.63 + 4.8 / math.sqrt(Re)) ** 2
        ref = 0.5 * p["rho_f"] * Cd * math.pi * d * d / 4 * wmag * w
        assert np.allclose(f, ref, rtol=1e-12, atol=0)
        assert abs(vr - 1.0) < 1e-12
    w = np.array([0.0, 0.0, 1e-9])
    f, _, _ = oracle_mod.drag(p, 0.0, w, d)
    stokes = 3 * math.pi * p["rho_f"] * p["nu_f"] * d * w[2]
    assert abs(f[2] / stokes - 23.04 / 24.0) < 1e-3
    # hindered settling: more solids -> smaller V_r -> larger drag at the same slip
    f1, vr1, _ = oracle_mod.drag(p, 0.3, np.array([0.0, 0.0, 0.05]), d)
    f0, vr0, _ = oracle_mod.drag(p, 0.0, np.array([0.0, 0.0, 0.05]), d)
    assert vr1 < vr0 and f1[2] > f0[2] > 0


def test_p10_lubrication_log_law(oracle_mod):
    """P10: lubrication alone slows a sphere approaching a wall as
    v(h) = v0 + (6 pi mu r^2 / m) ln(h0 / h) (v < 0 towards the wall)."""
    d = 1e-3
    r = d / 2
    p = default_params(drag=0, pressure_grad=0, added_mass=0, g=(0, 0, 0), dt=1e-6,
                       wall_hi=(0, 0, 0))
    h0 = 0.099 * d
    v0 = -0.01
    o = single(oracle_mod, p, [0.01, 0.01, r + h0], [0, 0, v0], d)
    m = RHO * math.pi / 6 * d ** 3
    mu = p["rho_f"] * p["nu_f"]
    k = 6 * math.pi * mu * r * r / m
    checked = 0
    steps = 0
    for target in (h0 / 3, h0 / 10):
        while True:
            x, v, _, _ = o.get_particles()
            h = x[0, 2] - r
            if h <= target:
                break
            o.step(10)
            steps += 10
            assert steps < 200000, "the sphere stopped short of the wall"
        o.step(1)
        x2, v2, _, _ = o.get_particles()
        # v is the half-step velocity between the two positions
        hmid = 0.5 * (h + x2[0, 2] - r)
        expect = v0 + k * math.log(h0 / hmid)
        assert abs(v2[0, 2] / expect - 1) < 2e-3
        checked += 1
    assert checked == 2


def test_trilinear_interpolation_of_linear_field(oracle_mod):
    """Cell-centred trilinear interpolation reproduces a linear field exactly in the
    interior, clamps below the first cell centre at a wall and wraps periodically."""
    p = default_params(drag=0, added_mass=0, lubrication=0)
    nx, ny, nz = p["ncell"]
    hx = (p["hi"][0] - p["lo"][0]) / nx
    hz = (p["hi"][2] - p["lo"][2]) / nz
    zc = (np.arange(nz) + 0.5) * hz
    xc = (np.arange(nx) + 0.5) * hx
    gp = np.zeros((nz, ny, nx, 3))
    gp[..., 2] = 100.0 + 5e4 * zc[:, None, None]
    gp[..., 0] = 7.0 + 3e4 * xc[None, None, :]
    d = 1e-3
    Vp = math.pi / 6 * d ** 3
    pts = [[0.0101, 0.0123, 0.0177], [0.0005, 0.01, 0.0004], [0.0195, 0.005, 0.03]]
    o = oracle_mod.Oracle(p)
    o.set_particles(np.array(pts), np.zeros((3, 3)), np.zeros((3, 3)), np.full(3, d),
                    np.full(3, RHO))
    o.set_fluid(grad_p=gp.reshape(-1, 3))
    f = o.forces()["fluid"]
    # interior point: exact linear values
    assert abs(-f[0, 2] / Vp - (100.0 + 5e4 * pts[0][2])) < 1e-9
    assert abs(-f[0, 0] / Vp - (7.0 + 3e4 * pts[0][0])) < 1e-9
    # below the first z centre: clamped to the first centre value
    assert abs(-f[1, 2] / Vp - (100.0 + 5e4 * zc[0])) < 1e-9
    # x below the first centre wraps between the last and first cell
    s = pts[1][0] / hx - 0.5 + nx
    fr = s - math.floor(s)
    expect = (1 - fr) * (7.0 + 3e4 * xc[-1]) + fr * (7.0 + 3e4 * xc[0])
    assert abs(-f[1, 0] / Vp - expect) < 1e-9
    # x above the last centre wraps too
    s = pts[2][0] / hx - 0.5
    fr = s - math.floor(s)
    expect = (1 - fr) * (7.0 + 3e4 * xc[-1]) + fr * (7.0 + 3e4 * xc[0])
    assert abs(-f[2, 0] / Vp - expect) < 1e-9
