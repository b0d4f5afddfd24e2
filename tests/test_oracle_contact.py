"""Pins of the oracle's contact law and time integration (CPU only).

Each pin compares the oracle with a closed form or an independent integration, so
that a dropped term, a wrong sign or a wrong lever arm fails at least one.
"""
import math

import numpy as np
import pytest

from paper_1601_03801_gb300.workloads import default_params

RHO = 2500.0
D = 1e-3


def dry(**over):
    """No fluid, no gravity, no lubrication; a large periodic box."""
    p = default_params(drag=0, pressure_grad=0, added_mass=0, lubrication=0, g=(0.0, 0.0, 0.0),
                       lo=(0.0, 0.0, 0.0), hi=(0.02, 0.02, 0.02), periodic=(1, 1, 1),
                       wall_lo=(0, 0, 0), wall_hi=(0, 0, 0), ncell=(4, 4, 4))
    p.update(over)
    return p


def mass(d=D, rho=RHO):
    return rho * math.pi / 6 * d ** 3


def e_star(p):
    return p["E"] / (2 * (1 - p["poisson"] ** 2))


def hertz_tc(p, vrel, d=D):
    """Hertz elastic contact duration of two equal spheres (Johnson 1985)."""
    ms = mass(d) / 2
    Rs = d / 4
    dmax = (15 * ms * vrel ** 2 / (16 * e_star(p) * math.sqrt(Rs))) ** 0.4
    beta_int = 0.4 * math.gamma(0.4) * math.gamma(0.5) / math.gamma(0.9)  # int_0^1 (1-x^2.5)^-1/2
    return 2 * beta_int * dmax / vrel, dmax


def head_on(oracle_mod, p, vrel, nsteps, d=D):
    o = oracle_mod.Oracle(p)
    gap = 1e-9
    x = np.array([[0.01 - d / 2 - gap, 0.01, 0.01], [0.01 + d / 2 + gap, 0.01, 0.01]])
    v = np.array([[vrel / 2, 0, 0], [-vrel / 2, 0, 0]])
    o.set_particles(x, v, np.zeros((2, 3)), np.full(2, d), np.full(2, RHO))
    deltas, vs = [], []
    for _ in range(nsteps):
        xx, vv, _, _ = o.get_particles()
        deltas.append(d - (xx[1, 0] - xx[0, 0]))
        vs.append(vv[0, 0] - vv[1, 0])
        o.step(1)
    return np.array(deltas), np.array(vs)


def crossing_times(delta, dt):
    """Linear-interpolated times where the overlap becomes positive / non-positive."""
    pos = delta > 0
    k0 = int(np.argmax(pos))
    k1 = k0 + int(np.argmax(~pos[k0:]))
    t0 = (k0 - 1 + (-delta[k0 - 1]) / (delta[k0] - delta[k0 - 1])) * dt
    t1 = (k1 - 1 + delta[k1 - 1] / (delta[k1 - 1] - delta[k1])) * dt
    return t0, t1, k1


@pytest.mark.parametrize("vrel", [0.1, 1.0])
def test_p1_hertz_contact_time(oracle_mod, vrel):
    """P1: elastic (e = 1) head-on contact lasts 2.9432 delta_max / v0; the DEM
    converges to it at second order in dt and conserves the approach speed."""
    tc, dmax = hertz_tc(dry(), vrel)
    errs = []
    for nper in (200, 400):
        dt = tc / nper
        p = dry(restitution=1.0, dt=dt)
        delta, vrel_hist = head_on(oracle_mod, p, vrel, int(1.3 * nper))
        t0, t1, k1 = crossing_times(delta, dt)
        errs.append(abs((t1 - t0) - tc) / tc)
        assert abs(delta.max() - dmax) / dmax < 2e-3
        assert abs(-vrel_hist[k1 + 2] / vrel - 1.0) < 1e-3
    assert errs[1] < 2e-4
    assert errs[1] < errs[0]


def restitution_ode(p, v0, d=D, nper=20000):
    """Independent RK4 integration of the normal Hertz + Tsuji-damping ODE."""
    ms = mass(d) / 2
    Rs = d / 4
    Es = e_star(p)
    lne = math.log(p["restitution"])
    beta = lne / math.sqrt(lne ** 2 + math.pi ** 2)
    kn = 4.0 / 3.0 * Es * math.sqrt(Rs)

    def acc(x, u):
        if x <= 0:
            return 0.0
        sn = 2 * Es * math.sqrt(Rs * x)
        c = -2 * math.sqrt(5 / 6) * beta * math.sqrt(sn * ms)
        return (-kn * x ** 1.5 - c * u) / ms

    tc, _ = hertz_tc(p, v0, d)
    h = tc / nper
    x, u = 0.0, v0
    for _ in range(4 * nper):
        k1x, k1u = u, acc(x, u)
        k2x, k2u = u + 0.5 * h * k1u, acc(x + 0.5 * h * k1x, u + 0.5 * h * k1u)
        k3x, k3u = u + 0.5 * h * k2u, acc(x + 0.5 * h * k2x, u + 0.5 * h * k2u)
        k4x, k4u = u + h * k3u, acc(x + h * k3x, u + h * k3u)
        xn = x + h / 6 * (k1x + 2 * k2x + 2 * k3x + k4x)
        u = u + h / 6 * (k1u + 2 * k2u + 2 * k3u + k4u)
        if xn <= 0 and x > 0:
            return -u / v0
        x = xn
    raise AssertionError("ODE contact did not end")


def test_p2_restitution_matches_ode(oracle_mod):
    """P2: the damping gives a velocity-independent restitution equal to that of
    the 1-D normal ODE, which reproduces the nominal e to 1e-3."""
    p = dry(restitution=0.9)
    e_ode = [restitution_ode(p, v) for v in (0.1, 1.0)]
    assert abs(e_ode[0] - e_ode[1]) < 1e-4
    assert abs(e_ode[0] - p["restitution"]) < 1e-3
    for vrel in (0.1, 1.0):
        tc, _ = hertz_tc(p, vrel)
        dt = tc / 1000
        delta, vh = head_on(oracle_mod, dict(p, dt=dt), vrel, 1300)
        _, _, k1 = crossing_times(delta, dt)
        e_dem = -vh[k1 + 2] / vrel
        assert abs(e_dem - e_ode[0]) < 2e-3


@pytest.mark.parametrize("lub_t", [0, 1])
def test_p4_momentum_and_angular_momentum(oracle_mod, lub_t):
    """P4: pair forces cancel (sum F = 0) and, with lever arms r - delta/2 (r + h/2
    across a lubrication gap), the pair torques close the angular-momentum balance
    sum(x x F + T) = 0, with and without the tangential lubrication terms."""
    rng = np.random.default_rng(4)
    n = 60
    p = dry(lubrication=1, periodic=(0, 0, 0), hi=(0.05, 0.05, 0.05), ncell=(4, 4, 4),
            lub_tangential=lub_t)
    x = 0.025 + rng.uniform(-1.6e-3, 1.6e-3, (n, 3))
    d = rng.uniform(0.8e-3, 1.2e-3, n)
    v = rng.normal(0, 0.2, (n, 3))
    w = rng.normal(0, 200.0, (n, 3))
    o = oracle_mod.Oracle(p)
    o.set_particles(x, v, w, d, np.full(n, RHO))
    o.step(3)  # build some tangential history
    xx, _, _, _ = o.get_particles()
    f = o.forces()
    F = f["contact"] + f["lub"]
    scale = np.abs(F).sum()
    assert scale > 0
    assert np.abs(F.sum(0)).max() <= 64 * n * np.finfo(float).eps * scale
    L = np.cross(xx - 0.025, F).sum(0) + f["torque"].sum(0)
    assert np.abs(L).max() <= 64 * n * np.finfo(float).eps * scale * 2e-3
    assert np.abs(f["torque"]).max() > 0


def resting_case(p, vx0):
    m = mass()
    Es = e_star(p)
    r = D / 2
    dstat = (m * 9.81 / (4.0 / 3.0 * Es * math.sqrt(r))) ** (2.0 / 3.0)
    x = np.array([[0.01, 0.01, r - dstat]])
    v = np.array([[vx0, 0.0, 0.0]])
    return x, v, dstat


def wall_params(**over):
    p = dry(g=(0.0, 0.0, -9.81), periodic=(1, 1, 0), wall_lo=(0, 0, 1), wall_hi=(0, 0, 0),
            hi=(0.02, 0.02, 0.02))
    p.update(over)
    return p


def test_p13_sliding_sphere_rolls_at_five_sevenths(oracle_mod):
    """P13: a sphere sliding on a wall under Coulomb friction ends rolling with
    v = v0 / (1 + I/(m l^2)) = 5/7 v0 (l -> r) and l*omega = v; while it slides it
    decelerates at mu g."""
    p = wall_params(dt=2e-6)
    v0 = 0.05
    x, v, dstat = resting_case(p, v0)
    o = oracle_mod.Oracle(p)
    o.set_particles(x, v, np.zeros((1, 3)), np.array([D]), np.array([RHO]))
    o.step(500)
    _, v1, _, _ = o.get_particles()
    o.step(500)
    _, v2, _, _ = o.get_particles()
    decel = (v1[0, 0] - v2[0, 0]) / (500 * p["dt"])
    assert abs(decel / (p["friction"] * 9.81) - 1) < 2e-2
    o.step(6000)
    xx, vv, ww, _ = o.get_particles()
    r = D / 2
    l = r - 0.5 * dstat
    expect = v0 / (1 + 0.4 * r * r / (l * l))
    assert abs(vv[0, 0] / expect - 1) < 2e-4
    assert abs(vv[0, 0] - 5.0 / 7.0 * v0) / v0 < 1e-3
    assert abs(ww[0, 1] * l - vv[0, 0]) / vv[0, 0] < 1e-3


def test_p14_static_overlap_on_wall(oracle_mod):
    """P14: a sphere at rest on the wall settles at the Hertz overlap
    delta = (m g / ((4/3) E* sqrt(r)))^(2/3)."""
    p = wall_params(dt=2e-6, restitution=0.3)
    x, v, dstat = resting_case(p, 0.0)
    x[0, 2] += 0.3 * dstat
    o = oracle_mod.Oracle(p)
    o.set_particles(x, v, np.zeros((1, 3)), np.array([D]), np.array([RHO]))
    o.step(20000)
    xx, vv, _, _ = o.get_particles()
    assert abs((D / 2 - xx[0, 2]) / dstat - 1) < 1e-4
    assert abs(vv[0, 2]) < 1e-6


def test_timestep_rule_config_small():
    """P12: for the small bed at the settling speed 0.134 m/s the Hertz contact time
    is ~1.5e-4 s, so dt = 1e-6 s resolves it with far more than 50 steps."""
    p = default_params()
    tc, _ = hertz_tc(p, 0.134)
    assert 1.2e-4 < tc < 1.8e-4
    assert p["dt"] <= tc / 50


def linear_closed_form(p, d=D):
    """Damped linear oscillator of the relative normal motion (equal spheres):
    omega_0 = sqrt(k_n / m*), zeta = -ln e / sqrt(pi^2 + ln^2 e); contact ends at zero
    overlap after half a damped period, with exactly the speed ratio e."""
    ms = mass(d) / 2
    w0 = math.sqrt(p["kn_linear"] / ms)
    le = math.log(p["restitution"])
    zeta = -le / math.sqrt(math.pi ** 2 + le * le)
    return math.pi / (w0 * math.sqrt(1 - zeta * zeta)), w0


@pytest.mark.parametrize("e,vrel", [(0.97, 0.1), (0.97, 1.0), (0.5, 0.1)])
def test_linear_spring_dashpot_restitution_and_duration(oracle_mod, e, vrel):
    """Linear spring-dashpot of Sec. 2.5 / Table 1 (k_n = 800 N/m): the head-on
    collision lasts pi / omega_d whatever the impact speed, rebounds with exactly
    the restitution coefficient e, and reaches the undamped peak overlap
    v0 / omega_0 when e = 1; the DEM converges to these at first order or better."""
    p0 = dry(contact_law=1, restitution=e)
    tc, w0 = linear_closed_form(p0)
    errs = []
    for nper in (400, 800):
        dt = tc / nper
        p = dry(contact_law=1, restitution=e, dt=dt)
        delta, vh = head_on(oracle_mod, p, vrel, int(1.3 * nper))
        t0, t1, k1 = crossing_times(delta, dt)
        e_dem = -vh[k1 + 2] / vh[0]
        errs.append((abs((t1 - t0) - tc) / tc, abs(e_dem - e)))
    # errors fall with dt and are small at the finer step
    assert errs[1][0] < 2e-3 and errs[1][1] < 2e-3, errs
    assert errs[1][0] <= errs[0][0] + 1e-12 and errs[1][1] <= errs[0][1] + 1e-12, errs
    # elastic case: peak overlap of the undamped oscillator
    pe = dry(contact_law=1, restitution=1.0, dt=tc / 800)
    delta, _ = head_on(oracle_mod, pe, vrel, 1100)
    assert abs(delta.max() - vrel / w0) / (vrel / w0) < 2e-3


def test_linear_law_differs_from_hertz_at_same_state(oracle_mod):
    """The law switch changes the force (guards against the flag being ignored)."""
    x = np.array([[0.01 - 0.4999e-3, 0.01, 0.01], [0.01 + 0.4999e-3, 0.01, 0.01]])
    f = []
    for law in (0, 1):
        o = oracle_mod.Oracle(dry(contact_law=law))
        o.set_particles(x, np.zeros((2, 3)), np.zeros((2, 3)), np.full(2, D), np.full(2, RHO))
        f.append(o.forces()["contact"][0, 0])
    delta = D - 2 * 0.4999e-3
    assert abs(f[1] + 800.0 * delta) < 1e-12 * 800.0 * D  # F = -k_n delta on the left sphere
    assert abs(f[0] - f[1]) > 1e-3 * abs(f[1])


def test_case1_bounce_effective_restitution(oracle_mod):
    """Case 1 (Sec. 4.1) on the oracle: with lubrication and added mass the effective
    restitution e_water / e_air falls with the Stokes number (small at St ~ 25, near 1
    at St ~ 5000); without them the sphere keeps nearly its dry coefficient."""
    from paper_1601_03801_gb300 import diagnostics as dg
    from paper_1601_03801_gb300.workloads import bounce_case
    d, rho = 6e-3, 7800.0
    dt = dg.linear_contact_time(800.0, rho * math.pi / 6 * d ** 3, 0.97) / 50
    e_lub, e_dry, st = [], [], []
    for nu in (1e-6, 1e-5, 1e-4):
        for on, out in ((1, e_lub), (0, e_dry)):
            prm, parts = bounce_case(rho, nu, dt, d=d, lubrication=on, added_mass=on)
            o = oracle_mod.Oracle(prm)
            o.set_particles(parts["x"], parts["v"], parts["w"], parts["d"], parts["rho"])
            v_in, v_out, _ = dg.bounce_velocities(o, chunk=10)
            out.append(v_out / abs(v_in) / 0.97)
            if on:
                st.append(dg.stokes_number(rho, d, v_in, nu, 1000.0))
    assert st[0] > st[1] > st[2] and st[2] < 40 and st[0] > 3000
    assert e_lub[0] > e_lub[1] > e_lub[2] and e_lub[2] < 0.2 and e_lub[0] > 0.85
    assert all(e > 0.95 for e in e_dry) and all(a < b for a, b in zip(e_lub, e_dry))


def _rot_z(th, v):
    c, s = math.cos(th), math.sin(th)
    return np.array([c * v[0] - s * v[1], s * v[0] + c * v[1], v[2]])


def _rigid_rotation(oracle_mod, xi0, steps, omega=100.0, p=None):
    """Two touching spheres turning rigidly about their common centre (axis z, rate
    omega) with no surface slip: positions, velocities and spins prescribed in closed
    form, the spring fed from one substep to the next through the contact law."""
    p = p or dry(friction=10.0)
    dt = p["dt"]
    m = mass()
    delta = 2e-6
    dist = D - delta
    xi = np.array(xi0, float)
    W = np.array([0.0, 0.0, omega])
    forces = []
    for k in range(steps + 1):
        th = omega * dt * k
        n = _rot_z(th, [1.0, 0.0, 0.0])
        xa, xb = -0.5 * dist * n, 0.5 * dist * n
        act, F, _, _, xi_new = oracle_mod.hm_pair(p, xb - xa, D / 2, D / 2, m, m, np.cross(W, xa),
                                                  np.cross(W, xb), W, W, xi)
        assert act
        forces.append((th, F))
        xi = xi_new  # tangent to n of substep k
    return xi, forces, p


def test_p19_spring_turns_with_rigidly_rotating_contact(oracle_mod):
    """P19 (Sec. 2.5, endured contacts): a contact that turns rigidly carries its
    tangential spring with it.  Relative surface velocity is zero, so each substep only
    rotates the spring onto the new tangent plane and restores its length: a spring in
    the plane of rotation after angle theta is R(theta) xi0 (exact up to rounding), the
    contact force is constant in the co-rotating frame, and a spring with a component
    along the axis keeps its length and converges to R(theta) xi0 at first order in the
    step angle."""
    xi0 = np.array([0.0, 2e-7, 0.0])  # tangent at n = x, in the plane of rotation
    steps = 10000                      # 1 rad at 100 rad/s and dt = 1e-6 s
    xi, forces, p = _rigid_rotation(oracle_mod, xi0, steps)
    th = 100.0 * p["dt"] * steps
    assert np.abs(xi - _rot_z(th, xi0)).max() < 1e-12 * np.linalg.norm(xi0)
    # force in the co-rotating frame (n, t, z): constant along the whole rotation
    fr = np.array([[F @ _rot_z(t, [1, 0, 0]), F @ _rot_z(t, [0, 1, 0]), F[2]] for t, F in forces[1:]])
    assert np.abs(fr - fr[0]).max() < 1e-10 * np.abs(fr[0]).max()
    assert fr[0][1] < 0 and abs(fr[0][2]) < 1e-12 * abs(fr[0][1])  # F_t = -S_t xi, along -t
    # with a component along the rotation axis: length kept, first-order convergence
    xi0 = np.array([0.0, 2e-7, 1e-7])
    errs = []
    for steps in (2500, 5000):
        p2 = dry(friction=10.0, dt=1e-6 * 10000 / steps)
        xi, _, _ = _rigid_rotation(oracle_mod, xi0, steps, p=p2)
        assert abs(np.linalg.norm(xi) / np.linalg.norm(xi0) - 1) < 1e-12
        errs.append(np.abs(xi - _rot_z(1.0, xi0)).max())
    assert 1.8 < errs[0] / errs[1] < 2.2 and errs[1] < 1e-3 * np.linalg.norm(xi0)
