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


# Eq. 6 limits at eps_f < 1, computed by hand (30-digit arithmetic) from the printed
# exponents: A1 = eps_f^4.14; A2 = 0.8 eps_f^1.28 for eps_f <= 0.85, else eps_f^2.65.
VR_LIMITS = {  # eps_f: (A1, A2)
    0.4: (0.022517924781948604002, 0.24758639476830814702),
    0.7: (0.22840514666231898778, 0.50677534527606156953),
    0.85: (0.51026332237862154106, 0.64974988589687697339),
    0.9: (0.64649324148994868621, 0.7563845512207213536),
}


@pytest.mark.parametrize("eps_f", sorted(VR_LIMITS))
def test_p9b_vr_limits_below_unit_fluid_fraction(oracle_mod, eps_f):
    """P9b (Sec. 2.3, Eq. 6): the terminal-velocity ratio V_r tends to A1 = eps_f^4.14 as
    Re -> 0 and to A2 as Re -> infinity (the square root grows like 0.06 Re + 2 A2 - A1),
    on both sides of the switch of A2 at eps_f = 0.85; in between it is monotone.  The
    Re -> infinity side is taken at Re = 1e8, where the O(1/Re) remainder (~4e-8) and the
    FP64 cancellation of 0.06 Re against the square root (~1e-9) both stay below 2e-7."""
    A1, A2 = VR_LIMITS[eps_f]
    assert abs(oracle_mod.vr(eps_f, 1e-14) - A1) < 1e-10 * A1
    assert abs(oracle_mod.vr(eps_f, 1e8) - A2) < 2e-7 * A2
    vals = [oracle_mod.vr(eps_f, Re) for Re in np.logspace(-6, 8, 57)]
    assert np.all(np.diff(vals) > 0) and A1 < vals[0] < vals[-1] < A2


def test_p9c_hindered_stokes_limit(oracle_mod):
    """P9c: at a small slip in a suspension of solid fraction eps_s, C_d -> 23.04 V_r / Re
    and the drag tends to (23.04 / 24) x Stokes / eps_f^4.14 (Eq. 3-6 combined)."""
    p = default_params()
    d, wz = 1e-3, 1e-12
    stokes = 3 * math.pi * p["rho_f"] * p["nu_f"] * d * wz
    for eps_s, (eps_f, A1) in ((0.3, (0.7, VR_LIMITS[0.7][0])), (0.6, (0.4, VR_LIMITS[0.4][0]))):
        f, vr, _ = oracle_mod.drag(p, eps_s, np.array([0.0, 0.0, wz]), d)
        assert abs(vr / A1 - 1) < 1e-6
        assert abs(f[2] / stokes / (0.96 / A1) - 1) < 1e-4


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


def cell_centres(p):
    n = p["ncell"]
    c = [p["lo"][a] + (np.arange(n[a]) + 0.5) * (p["hi"][a] - p["lo"][a]) / n[a] for a in range(3)]
    Z, Y, X = np.meshgrid(c[2], c[1], c[0], indexing="ij")
    return X.ravel(), Y.ravel(), Z.ravel()


def test_p15_vorticity_closed_forms(oracle_mod):
    """P15: the cell vorticity is exact for linear fields (central and one-sided
    differences alike): simple shear U = (G z, 0, 0) gives omega = (0, G, 0) in every
    cell, rigid rotation U = W x (x - x0) gives 2 W; a periodic sine U_x = sin(k z)
    gives the central-difference closed form k cos(k z) sin(k h) / (k h)."""
    p = default_params(periodic=(0, 0, 0), wall_lo=(1, 1, 1), wall_hi=(1, 1, 1), ncell=(5, 4, 6))
    X, Y, Z = cell_centres(p)
    G = 37.0
    U = np.stack([G * Z, 0 * Z, 0 * Z], 1)
    om = oracle_mod.curl(p, U)
    np.testing.assert_allclose(om, np.tile([0.0, G, 0.0], (len(X), 1)), rtol=0, atol=1e-10 * G)
    W = np.array([3.0, -2.0, 5.0])
    r = np.stack([X - 0.004, Y - 0.013, Z + 0.002], 1)
    U = np.cross(W, r)
    om = oracle_mod.curl(p, U)
    np.testing.assert_allclose(om, np.tile(2 * W, (len(X), 1)), rtol=0, atol=1e-10)
    q = default_params(periodic=(1, 1, 1), wall_lo=(0, 0, 0), wall_hi=(0, 0, 0), ncell=(3, 2, 16))
    X, Y, Z = cell_centres(q)
    L = q["hi"][2] - q["lo"][2]
    h = L / q["ncell"][2]
    k = 2 * np.pi / L
    U = np.stack([np.sin(k * Z), 0 * Z, 0 * Z], 1)
    om = oracle_mod.curl(q, U)
    expect = k * np.cos(k * Z) * np.sin(k * h) / (k * h)
    np.testing.assert_allclose(om[:, 1], expect, rtol=0, atol=1e-12 * k)
    assert np.abs(om[:, [0, 2]]).max() < 1e-12 * k


def test_p16_saffman_lift_in_simple_shear(oracle_mod):
    """P16: a sphere at rest in the simple shear U = (G z, 0, 0) feels Saffman's lift
    C_l rho_f nu^0.5 d^2 G^0.5 U_x towards the faster fluid (+z); a sphere leading
    the flow is pushed down; one moving with the fluid feels none; the force is
    perpendicular to the slip and to the vorticity."""
    d, G = 0.5e-3, 40.0
    p = default_params(drag=0, pressure_grad=0, added_mass=0, lubrication=0, lift=1,
                       periodic=(1, 1, 0), ncell=(4, 4, 8))
    X, Y, Z = cell_centres(p)
    o = oracle_mod.Oracle(p)
    z0 = 0.0137
    Ux = G * z0
    for vx, sign in ((0.0, 1.0), (2 * Ux, -1.0), (Ux, 0.0)):
        o.set_particles(np.array([[0.011, 0.009, z0]]), np.array([[vx, 0.0, 0.0]]),
                        np.zeros((1, 3)), np.array([d]), np.array([RHO]))
        o.set_fluid(U=np.stack([G * Z, 0 * Z, 0 * Z], 1))
        f = o.forces()["fluid"][0]
        expect = p["c_lift"] * p["rho_f"] * math.sqrt(p["nu_f"]) * d * d * math.sqrt(G) * abs(Ux - vx)
        assert abs(f[2] - sign * expect) <= 1e-9 * max(expect, 1e-30) + 1e-30
        assert abs(f[0]) <= 1e-12 * expect + 1e-30 and abs(f[1]) <= 1e-12 * expect + 1e-30
    # general orientation: perpendicular to w and omega, magnitude |w x omega| / |omega|^0.5 scale
    rng = np.random.default_rng(4)
    for _ in range(5):
        w, om = rng.normal(size=3), rng.normal(size=3) * 20
        f = oracle_mod.lift(p, w, om, d)
        assert abs(f @ w) < 1e-12 * np.linalg.norm(f) * np.linalg.norm(w)
        assert abs(f @ om) < 1e-12 * np.linalg.norm(f) * np.linalg.norm(om)
        mag = p["c_lift"] * p["rho_f"] * math.sqrt(p["nu_f"]) * d * d * np.linalg.norm(np.cross(w, om))
        assert abs(np.linalg.norm(f) - mag / math.sqrt(np.linalg.norm(om))) < 1e-12 * mag
    assert np.all(oracle_mod.lift(p, [0.1, 0, 0], [0, 0, 0], d) == 0)


def test_p17_tangential_lubrication_limits(oracle_mod):
    """P17: the shear lubrication term has the published leading terms: equal
    spheres 6 pi mu a (1/6) ln(a/h) (Jeffrey & Onishi), sphere-wall
    6 pi mu a (8/15) ln(a/h) (Goldman, Cox & Brenner); its prefactor tends to the
    wall's as one sphere grows; the pair is antisymmetric, conserves angular
    momentum, and a sphere rolling without slip on a wall feels none of it."""
    p = default_params(lub_tangential=1)
    mu = p["rho_f"] * p["nu_f"]
    a = 0.5e-3
    h = 0.02 * a
    v = np.array([0.0, 0.013, 0.0])
    z = np.zeros(3)
    F, Ta, Tb = oracle_mod.lub_pair(p, [2 * a + h, 0, 0], a, a, v, z, z, z)
    expect = -np.pi * mu * a * math.log(a / h) * v
    np.testing.assert_allclose(F, expect, rtol=1e-12, atol=0)
    n = np.array([0.0, 0.0, -1.0])
    Fw, Tw = oracle_mod.lub_wall(p, n, a + h, a, v, z)
    np.testing.assert_allclose(Fw, -6 * np.pi * mu * a * (8 / 15) * math.log(a / h) * v, rtol=1e-12)
    np.testing.assert_allclose(Tw, np.cross((a + h / 2) * n, Fw), rtol=1e-12)
    # prefactor -> the wall's as r_b grows (the logarithm is the pair's own)
    for beta in (1e3, 1e5):
        rb = beta * a
        # h_in scales with the pair-mean diameter: keep it below h
        F, _, _ = oracle_mod.lub_pair(dict(p, lub_h_in_frac=1e-12), [a + rb + h, 0, 0], a, rb,
                                      v, z, z, z)
        pref = -F[1] / (v[1] * math.log((a + rb) / (2 * h)))
        assert abs(pref / (6 * np.pi * mu * a * 8 / 15) - 1) < 3 / beta
    # antisymmetry and angular momentum for an unequal pair with spins
    rng = np.random.default_rng(2)
    ra, rb = 0.3e-3, 0.45e-3
    e = rng.normal(size=3)
    e /= np.linalg.norm(e)
    dx = (ra + rb + 0.03e-3) * e
    va, vb, wa, wb = (rng.normal(size=3) * s for s in (0.01, 0.01, 30, 30))
    F, Ta, Tb = oracle_mod.lub_pair(p, dx, ra, rb, va, vb, wa, wb)
    G, Ua, Ub = oracle_mod.lub_pair(p, -dx, rb, ra, vb, va, wb, wa)
    np.testing.assert_allclose(G, -F, rtol=1e-12, atol=1e-24)
    np.testing.assert_allclose(Ua, Tb, rtol=1e-12, atol=1e-28)
    np.testing.assert_allclose(Ub, Ta, rtol=1e-12, atol=1e-28)
    L = Ta + Tb - np.cross(dx, F)
    assert np.abs(L).max() <= 1e-12 * np.abs(Ta).max()
    # rolling without slip: surface velocity at the gap midpoint is zero
    w = np.array([0.0, 80.0, 0.0])
    l = a + h / 2
    vroll = -np.cross(l * w, n)
    Fr, Tr = oracle_mod.lub_wall(p, n, a + h, a, vroll, w)
    assert np.abs(Fr).max() <= 1e-12 * 6 * np.pi * mu * a * np.abs(vroll).max()
    # switched off: the normal squeeze alone, no torque
    F0, Ta0, _ = oracle_mod.lub_pair(dict(p, lub_tangential=0), dx, ra, rb, va, vb, wa, wb)
    assert np.all(Ta0 == 0) and abs(F0 @ np.cross(e, [1.0, 0, 0])) <= 1e-12 * np.linalg.norm(F0)


def test_p17_sliding_sphere_spins_up_above_wall(oracle_mod):
    """P17 through the stepping oracle: a sphere sliding parallel to a wall at a
    lubrication gap starts to spin in the rolling sense (w_y > 0 for v_x > 0 above
    a floor) and slows; without the tangential term neither happens."""
    d = 1e-3
    r = d / 2
    out = []
    for lt in (1, 0):
        p = default_params(drag=0, pressure_grad=0, added_mass=0, g=(0, 0, 0), wall_hi=(0, 0, 0),
                           lub_tangential=lt)
        o = single(oracle_mod, p, [0.01, 0.01, r + 0.01 * d], [0.02, 0, 0], d)
        o.step(50)
        x, v, w, _ = o.get_particles()
        out.append((v[0], w[0]))
    (v1, w1), (v0, w0) = out
    assert w1[1] > 0 and v1[0] < 0.02 and abs(w1[0]) < 1e-12 * abs(w1[1]) + 1e-30
    assert np.all(w0 == 0) and v0[0] == 0.02
