"""Diagnostics of Case 1 (Sec. 4.1): the particle Stokes number, the time-step rule
of Sec. 2.5 for the linear contact law, and the impact and rebound speeds of a
sphere bouncing on a wall, from which the effective restitution coefficient
e = e_water / e_air of the particle-wall collision test is formed.

These are post-processing helpers: they drive a simulation object through its
public calls (``step`` and ``get_particles``) and hold none of the method's force
or update arithmetic.
"""
from __future__ import annotations

import math


def stokes_number(rho_p, d, u, nu_f, rho_f):
    """St = rho_p d u / (9 nu_f rho_f) (Sec. 4.1, Eq. 11)."""
    return rho_p * d * abs(u) / (9.0 * nu_f * rho_f)


def linear_contact_time(kn, m_eff, e):
    """Duration of one collision under the linear spring-dashpot (Sec. 2.5): half a
    damped period pi / (omega_0 sqrt(1 - zeta^2)), omega_0 = sqrt(k_n / m*),
    zeta = -ln e / sqrt(pi^2 + ln^2 e).  Sec. 2.5 takes dt = t_c / 50."""
    le = math.log(e)
    zeta = -le / math.sqrt(math.pi ** 2 + le * le)
    return math.pi / (math.sqrt(kn / m_eff) * math.sqrt(1.0 - zeta * zeta))


def bounce_velocities(sim, chunk=10, max_steps=60000):
    """Impact and rebound speeds of particle 0 falling onto a floor (z is up).

    Steps ``sim`` in chunks of substeps and samples the vertical velocity: the impact
    speed is the largest downward speed before the velocity turns upward, the
    rebound speed the largest upward speed after it (0 when the sphere comes to rest
    on the wall without leaving it).  Returns (v_in, v_out, substeps) with
    v_in < 0 <= v_out."""
    v_in, v_out, falling, steps = 0.0, 0.0, True, 0
    while steps < max_steps:
        sim.step(chunk)
        steps += chunk
        vz = float(sim.get_particles()[1][0, 2])
        if falling:
            v_in = min(v_in, vz)
            if v_in < 0.0 and vz > 0.0:
                falling, v_out = False, vz
            elif v_in < 0.0 and abs(vz) < 1e-4 * abs(v_in):
                break  # at rest on the wall: no rebound
        elif vz > v_out:
            v_out = vz
        else:
            break  # past the rebound peak
    return v_in, v_out, steps
