"""GPU parity: the CUDA library (through its C ABI) against the FP64 oracle.

Tolerances:
  FP64 form   forces 1e-12 of the largest force of each kind (measured ~1e-15);
              positions 1e-10 d
  split form  forces 1e-5 of the largest force of each kind; 200-step positions 1e-4 d
  plain form  same physics, loose (FP32 absolute positions): forces 5e-3
  neighbour lists, fixed-point deposition of eps and eps*U: bit-exact
"""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from oracle import oracle as orc  # noqa: E402
from paper_1601_03801_gb300 import sedi  # noqa: E402
from paper_1601_03801_gb300.workloads import (bed_case, default_params, small_case,  # noqa: E402
                                              storage_round)

FORCE_TOL = {"fp64": 1e-12, "split": 1e-5, "plain": 5e-3}


def make_pair(prm, parts, form, threads=1, **extra):
    """The library and the oracle at the same state: the oracle gets the value the
    library stores for each input (storage_round, computed on the host)."""
    g = sedi.Sedi(dict(prm, precision_form=form, **extra))
    g.set_particles(parts["x"], parts["v"], parts["w"], parts["d"], parts["rho"])
    o = orc.Oracle(prm, threads=threads)
    o.set_particles(*(storage_round(parts[k], form) for k in ("x", "v", "w")), parts["d"],
                    parts["rho"])
    return g, o


@pytest.mark.parametrize("form", ["fp64", "split", "plain"])
def test_inputs_stored_as_the_host_rounding_says(small, form):
    """What the library holds right after sedi_set_particles is storage_round of the
    inputs, bit for bit (so the oracle is given exactly the library's state)."""
    prm, parts = small
    g = sedi.Sedi(dict(prm, precision_form=form))
    g.set_particles(parts["x"], parts["v"], parts["w"], parts["d"], parts["rho"])
    x, v, w, _ = g.get_particles()
    for got, k in ((x, "x"), (v, "v"), (w, "w")):
        assert np.array_equal(got, storage_round(parts[k], form)), k


def min_image(dx, prm):
    L = np.array(prm["hi"]) - np.array(prm["lo"])
    return dx - L * np.round(dx / L) * np.array(prm["periodic"])


def rel_err(a, b):
    scale = np.abs(b).max()
    return np.abs(a - b).max() / scale if scale > 0 else np.abs(a).max()


SPRING_TOL = {"fp64": 1e-10, "split": 1e-5}


def compare_springs(g, o, prm, parts, form):
    """Springs of the pairs in contact agree to SPRING_TOL of the largest spring; the
    contact sets are equal except for pairs whose overlap is within rounding of zero
    (|delta| <= 1e-9 d at the oracle's positions), which may be in contact on one side.
    A spring that slid is reset from the capped force, -(F_t + c_t v_t) / S_t: in the
    split form that force is FP32, and as a contact ends its elastic and damping normal
    parts cancel while S_t -> 0, so the spring of a separating pair carries FP32
    rounding amplified without bound (its forces stay within 1e-7).  Pairs whose final
    overlap is <= 0 (separating: the spring is dropped at the next substep) are held to
    1e-3 of the largest spring only."""
    ijg, xig = g.contacts()
    ijo, xio = o.contacts()
    assert len(ijo) > 10
    kg = {tuple(p): k for k, p in enumerate(ijg)}
    ko = {tuple(p): k for k, p in enumerate(ijo)}
    xo = o.get_particles()[0]

    def overlap(pairs):
        ij = np.array(pairs).reshape(-1, 2)
        dx = min_image(xo[ij[:, 1]] - xo[ij[:, 0]], prm)
        return 0.5 * (parts["d"][ij[:, 0]] + parts["d"][ij[:, 1]]) - np.sqrt((dx * dx).sum(1))

    diff = sorted(set(kg) ^ set(ko))
    if diff:
        delta = overlap(diff)
        d_i = parts["d"][np.array(diff)[:, 0]]
        assert np.all(np.abs(delta) <= 1e-9 * d_i), (form, diff, delta)
    common = sorted(set(kg) & set(ko))
    a = np.array([xig[kg[c]] for c in common]); b = np.array([xio[ko[c]] for c in common])
    scale = np.abs(b).max()
    err = np.abs(a - b).max(axis=1) / scale
    held = overlap(common) > 0
    assert err[held].max() <= SPRING_TOL[form], (form, err[held].max())
    assert err.max() <= max(SPRING_TOL[form], 1e-3 if form == "split" else 0.0), (form, err.max())
    return len(common)


@pytest.fixture(scope="module")
def small():
    return small_case(parity_addon=True)


@pytest.mark.parametrize("form", ["fp64", "split", "plain"])
def test_neighbor_lists_bit_exact(small, form):
    prm, parts = small
    g, o = make_pair(prm, parts, form)
    off_g, ids_g = g.neighbors()
    off_o, ids_o = o.neighbors(prm["skin"], brute=True)
    assert np.array_equal(off_g, off_o)
    assert np.array_equal(ids_g, ids_o)
    assert len(ids_o) > len(parts["x"]) // 10


@pytest.mark.parametrize("form", ["fp64", "split", "plain"])
def test_forces_identical_state(small, form):
    prm, parts = small
    g, o = make_pair(prm, parts, form)
    rng = np.random.default_rng(3)
    C = int(np.prod(prm["ncell"]))
    eps = rng.uniform(0.0, 0.4, C)
    U = rng.normal(0, 0.05, (C, 3))
    DU = rng.normal(0, 0.5, (C, 3))
    for h in (g, o):
        h.set_fluid(U=U, DUDt=DU)
        h.set_eps(eps)
    fg, fo = g.compute_forces(), o.forces()
    for k in ("contact", "lub", "fluid", "torque"):
        assert np.abs(fo[k]).max() > 0, k
        err = rel_err(fg[k], fo[k])
        assert err <= FORCE_TOL[form], f"{form} {k}: {err:.3e}"


@pytest.mark.parametrize("form", ["fp64", "split"])
def test_forces_bed_moving_as_a_whole(small, form):
    # every sphere carries the same 2.4 m/s drift plus relative velocities four thousand
    # times smaller: the pair forces depend on the relative velocity only, so its
    # digits must survive the drift (the split form forms it from both words)
    prm, parts = small
    rng = np.random.default_rng(5)
    n = len(parts["x"])
    moving = dict(parts, v=np.array([2.0, -1.2, 0.4]) + rng.normal(0, 5e-4, (n, 3)),
                  w=rng.normal(0, 1.0, (n, 3)))
    g, o = make_pair(prm, moving, form)
    fg, fo = g.compute_forces(), o.forces()
    for k in ("contact", "lub", "torque"):
        assert np.abs(fo[k]).max() > 0, k
        err = rel_err(fg[k], fo[k])
        assert err <= FORCE_TOL[form], f"{form} {k}: {err:.3e}"


# the paper's own contact law (Sec. 2.5, Table 1): linear spring-dashpot, k_n = 800 N/m,
# e = 0.97, mu = 0.1
LINEAR = dict(contact_law=1, kn_linear=800.0, kt_ratio=2.0 / 7.0, restitution=0.97, friction=0.1)


@pytest.mark.parametrize("form", ["fp64", "split"])
def test_linear_law_forces_and_trajectory(small, form):
    prm, parts = small
    prm = dict(prm, **LINEAR)
    g, o = make_pair(prm, parts, form)
    fg, fo = g.compute_forces(), o.forces()
    for k in ("contact", "torque"):
        assert np.abs(fo[k]).max() > 0, k
        err = rel_err(fg[k], fo[k])
        assert err <= FORCE_TOL[form], f"{form} {k}: {err:.3e}"
    g.step(100)
    o.step(100)
    xg, _, _, _ = g.get_particles()
    xo, _, _, _ = o.get_particles()
    err = np.abs(min_image(xg - xo, prm)).max(axis=1) / parts["d"]
    assert err.max() <= (1e-10 if form == "fp64" else 1e-4), f"{form}: {err.max():.3e}"
    # the softer spring leaves fewer pairs touching than the Hertz law; the run still
    # carries tangential springs through the 100 steps
    ij, xi = o.contacts()
    assert len(ij) >= 4 and np.abs(xi).max() > 0


def shear_flow(prm, seed, G=5.0, noise=0.02):
    """Shear U_x = G z plus a random perturbation: vorticity of every orientation."""
    n = prm["ncell"]
    hz = (prm["hi"][2] - prm["lo"][2]) / n[2]
    zc = prm["lo"][2] + (np.arange(n[2]) + 0.5) * hz
    rng = np.random.default_rng(seed)
    C = int(np.prod(n))
    U = rng.normal(0, noise, (C, 3))
    U[:, 0] += G * np.repeat(zc, n[0] * n[1])
    return U, rng.uniform(0.0, 0.4, C)


@pytest.mark.parametrize("form", ["fp64", "split"])
def test_lift_and_tangential_lubrication(small, form):
    # Saffman lift (Sec. 2.3, Eq. 7) and the shear lubrication terms with their
    # torques (Sec. 2.5), against the oracle at the same state, then 100 steps
    prm, parts = small
    prm = dict(prm, lift=1, lub_tangential=1)
    g, o = make_pair(prm, parts, form)
    U, eps = shear_flow(prm, 12)
    for h in (g, o):
        h.set_fluid(U=U)
        h.set_eps(eps)
    fg, fo = g.compute_forces(), o.forces()
    for k in ("contact", "lub", "fluid", "torque"):
        err = rel_err(fg[k], fo[k])
        assert err <= FORCE_TOL[form], f"{form} {k}: {err:.3e}"
    # the lift is part of f_fp, so the fluid receives it through the deposition
    _, _, Fg = g.average()
    _, _, Fo = o.average()
    assert rel_err(Fg, Fo) <= 1e-4
    # the terms are there: the same state without them differs well beyond tolerance
    o0 = orc.Oracle(dict(prm, lift=0, lub_tangential=0))
    o0.set_particles(*(storage_round(parts[k], form) for k in ("x", "v", "w")), parts["d"],
                     parts["rho"])
    o0.set_fluid(U=U)
    o0.set_eps(eps)
    f0 = o0.forces()
    assert rel_err(f0["fluid"], fo["fluid"]) > 1e-3
    assert rel_err(f0["lub"], fo["lub"]) > 1e-3
    assert rel_err(f0["torque"], fo["torque"]) > 1e-6
    g.step(100)
    o.step(100)
    xg, _, wg, _ = g.get_particles()
    xo, _, wo, _ = o.get_particles()
    err = np.abs(min_image(xg - xo, prm)).max(axis=1) / parts["d"]
    assert err.max() <= (1e-10 if form == "fp64" else 1e-4), f"{form}: {err.max():.3e}"
    assert rel_err(wg, wo) <= (1e-8 if form == "fp64" else 1e-3)


@pytest.mark.parametrize("form", ["fp64", "split"])
def test_graded_mesh_matches_oracle(small, form):
    # graded z mesh (Sec. 4.2: refined towards the floor, top cell 4x the bottom one):
    # deposition cells and volumes, smoothing with both schemes, interpolation of the
    # fluid fields, vorticity for the lift, averaging, 100 steps
    prm, parts = small
    prm = dict(prm, z_grading=4.0, lift=1)
    g, o = make_pair(prm, parts, form)
    qg, qo = g.deposit(), o.deposit()
    assert np.array_equal(qg[:4], qo[:4])
    C = int(np.prod(prm["ncell"]))
    nxy = prm["ncell"][0] * prm["ncell"][1]
    w = np.repeat(np.diff(orc.z_faces(prm)), nxy)
    rng = np.random.default_rng(21)
    phi = rng.random((3, C)) * (rng.random((3, C)) < 0.5)
    for scheme in (0, 1):
        gs = sedi.Sedi(dict(prm, precision_form=form, tau_scheme=scheme))
        sg, itg = gs.smooth(phi)
        so, _ = orc.Oracle(dict(prm, tau_scheme=scheme)).smooth(phi)
        assert np.all(itg > 0)
        for f in range(3):
            assert np.abs(sg[f] - so[f]).max() <= 1e-7 * np.abs(phi[f]).max(), (scheme, f)
            assert abs((w * sg[f]).sum() / (w * phi[f]).sum() - 1) <= 1e-9
    U, eps = shear_flow(prm, 22)
    for h in (g, o):
        h.set_fluid(U=U)
        h.set_eps(eps)
    fg, fo = g.compute_forces(), o.forces()
    for k in ("contact", "lub", "fluid", "torque"):
        err = rel_err(fg[k], fo[k])
        assert err <= FORCE_TOL[form], f"{form} {k}: {err:.3e}"
    eg, _, Fg = g.average()
    eo, _, Fo = o.average()
    assert np.abs(eg - eo).max() <= 1e-7 * np.abs(eo).max()
    assert rel_err(Fg, Fo) <= 1e-4
    g.step(100)
    o.step(100)
    xg, _, _, _ = g.get_particles()
    xo, _, _, _ = o.get_particles()
    err = np.abs(min_image(xg - xo, prm)).max(axis=1) / parts["d"]
    assert err.max() <= (1e-10 if form == "fp64" else 1e-4), f"{form}: {err.max():.3e}"


def test_graded_mesh_grid_solver():
    # a graded mesh whose planes are too large for the cluster solver (grid solver);
    # a graded z axis cannot be periodic
    prm = default_params(hi=(96e-3, 96e-3, 24e-3), ncell=(96, 96, 24), wall_hi=(0, 0, 1),
                         bandwidth=(2e-3, 2e-3, 1.5e-3), z_grading=3.0)
    g = sedi.Sedi(dict(prm, precision_form="split"))
    o = orc.Oracle(prm)
    rng = np.random.default_rng(23)
    C = int(np.prod(prm["ncell"]))
    phi = rng.random((2, C)) * (rng.random((2, C)) < 0.3)
    sg, _ = g.smooth(phi)
    so, _ = o.smooth(phi)
    assert np.abs(sg - so).max() <= 1e-7 * np.abs(phi).max()
    with pytest.raises(sedi.SediError):
        sedi.Sedi(dict(prm, periodic=(1, 1, 1), wall_lo=(0, 0, 0), wall_hi=(0, 0, 0)))


@pytest.mark.parametrize("form", ["fp64", "split"])
def test_case1_bounce_matches_oracle(form):
    # Case 1 (Sec. 4.1): a 6 mm steel sphere falls onto the floor under the paper's
    # linear contact, with lubrication and added mass; impact and rebound speeds of
    # the library against the oracle sampled every 10 substeps
    import math
    from paper_1601_03801_gb300 import diagnostics as dg
    from paper_1601_03801_gb300.workloads import bounce_case
    d, rho = 6e-3, 7800.0
    dt = dg.linear_contact_time(800.0, rho * math.pi / 6 * d ** 3, 0.97) / 50
    for nu in (1e-5, 1e-4):
        prm, parts = bounce_case(rho, nu, dt, d=d)
        g = sedi.Sedi(dict(prm, precision_form=form))
        g.set_particles(parts["x"], parts["v"], parts["w"], parts["d"], parts["rho"])
        o = orc.Oracle(prm)
        o.set_particles(parts["x"], parts["v"], parts["w"], parts["d"], parts["rho"])
        vg, vo = dg.bounce_velocities(g, chunk=10), dg.bounce_velocities(o, chunk=10)
        assert vg[2] == vo[2], (vg, vo)
        tol = 1e-9 if form == "fp64" else 2e-4
        assert abs(vg[0] - vo[0]) <= tol * abs(vo[0]) and abs(vg[1] - vo[1]) <= tol * abs(vo[0]), (vg, vo)
        assert vo[1] > 0.0


@pytest.mark.parametrize("form,steps,tol", [("fp64", 200, 1e-10), ("split", 200, 1e-4)])
def test_trajectory_200_steps(small, form, steps, tol):
    prm, parts = small
    g, o = make_pair(prm, parts, form, use_graphs=1)
    g.step(20)
    o.step(20)
    compare_springs(g, o, prm, parts, form)
    g.step(steps - 20)
    o.step(steps - 20)
    xg, vg, wg, _ = g.get_particles()
    xo, vo, wo, _ = o.get_particles()
    err = np.abs(min_image(xg - xo, prm)).max(axis=1) / parts["d"]
    assert err.max() <= tol, f"{form}: {err.max():.3e}"


def test_graphs_equal_plain_launches(small):
    prm, parts = small
    out = []
    for graphs in (0, 1):
        g = sedi.Sedi(dict(prm, precision_form="split", use_graphs=graphs))
        g.set_particles(parts["x"], parts["v"], parts["w"], parts["d"], parts["rho"])
        for _ in range(3):
            g.step(20)
            g.average()
        out.append(g.get_particles()[0])
    assert np.array_equal(out[0], out[1])


def test_deterministic_runs(small):
    prm, parts = small
    res = []
    for _ in range(2):
        g = sedi.Sedi(dict(prm, precision_form="split"))
        g.set_particles(parts["x"], parts["v"], parts["w"], parts["d"], parts["rho"])
        g.step(60)
        eps, Us, F = g.average()
        res.append((g.get_particles(), eps, Us, F))
    for a, b in zip(res[0][0], res[1][0]):
        assert np.array_equal(a, b)
    for k in (1, 2, 3):
        assert np.array_equal(res[0][k], res[1][k])


@pytest.mark.parametrize("form", ["split", "plain"])
def test_substep_variants_bit_identical(small, form):
    """Every launch variant of the substep kernel gives the same bits in the split
    form: each particle's arithmetic does not depend on the block it runs in, and
    the warp-cooperative pair phase adds the same terms in the same order as the
    per-particle loop (variant 5).  The plain FP32 form agrees to FP32 rounding."""
    prm, parts = small
    ref = None
    for variant in range(10):
        g = sedi.Sedi(dict(prm, precision_form=form, substep_variant=variant))
        g.set_particles(parts["x"], parts["v"], parts["w"], parts["d"], parts["rho"])
        g.step(40)
        eps, _, F = g.average()
        st = g.stats()
        assert st["substep_variant"] == variant
        assert st["substep_block"] == {0: 128, 1: 64, 2: 256, 3: 128, 4: 128, 5: 128, 6: 128,
                                       7: 64, 8: 128, 9: 128}[variant]
        got = (*g.get_particles(), eps, F)
        if ref is None:
            ref = got
        elif form == "split":
            for a, b in zip(ref, got):
                assert np.array_equal(a, b), variant
        else:
            # plain FP32: positions and velocities identical; the stored acceleration
            # may differ in its last bits between launch shapes
            for a, b in zip(ref[:3], got[:3]):
                assert np.array_equal(a, b), variant
            for a, b in zip(ref[3:], got[3:]):
                assert np.abs(a - b).max() <= 1e-5 * max(np.abs(a).max(), 1e-30), variant


@pytest.mark.parametrize("variant", [5, 8, 9])
def test_bins_per_cutoff_change_no_result(small, variant):
    """Bins of one list cutoff (27-bin stencil) or of half a cutoff (125 bins), stored x
    fastest or z fastest: every list holds its partners in caller-index order, so lists,
    springs, trajectory and averaging are the same bits."""
    prm, parts = small
    out = []
    for R, order in ((1, 0), (2, 0), (1, 1), (2, 1)):
        g = sedi.Sedi(dict(prm, precision_form="split", substep_variant=variant, bins_per_cutoff=R,
                           bin_order=order))
        g.set_particles(parts["x"], parts["v"], parts["w"], parts["d"], parts["rho"])
        g.step(60)
        eps, _, F = g.average()
        st = g.stats()
        assert st["bins_per_cutoff"] == R and st["bin_order"] == order
        out.append((*g.get_particles(), eps, F, *g.neighbors(), *g.contacts()))
    assert len(out[0][-2]) > 10
    for other in out[1:]:
        for a, b in zip(out[0], other):
            assert np.array_equal(a, b)


def test_pair_list_contacts_match_loop(small):
    # the pair list keeps each spring in the first particle's slot; the contact
    # export copies it to the partner's slot first, so both runs export the same
    prm, parts = small
    out = []
    for v in (5, 8, 9):
        g = sedi.Sedi(dict(prm, precision_form="split", substep_variant=v))
        g.set_particles(parts["x"], parts["v"], parts["w"], parts["d"], parts["rho"])
        g.step(60)
        out.append((g.contacts(), g.get_particles()))
    (c5, p5) = out[0]
    assert len(c5[0]) > 10
    for c8, p8 in out[1:]:
        assert np.array_equal(c5[0], c8[0]) and np.array_equal(c5[1], c8[1])
        for a, b in zip(p5, p8):
            assert np.array_equal(a, b)


def test_autotuner_chooses_and_caches(small, tmp_path, monkeypatch):
    prm, parts = small
    cache = tmp_path / "tune.jsonl"
    monkeypatch.setenv("SEDI_AUTOTUNE_CACHE", str(cache))
    # a particle count no other test uses, so the in-process cache is cold
    n = len(parts["x"]) - 3
    sub = {k: parts[k][:n] for k in ("x", "v", "w", "d", "rho")}
    g = sedi.Sedi(dict(prm, precision_form="split"))
    g.set_particles(sub["x"], sub["v"], sub["w"], sub["d"], sub["rho"])
    assert g.stats()["substep_variant"] == -1
    # the launch shapes are compared once springs have formed (200 substeps)
    g.step(200)
    assert g.stats()["substep_variant"] == -1
    g.step(10)
    st = g.stats()
    assert 0 <= st["substep_variant"] < 10 and st["substep_block"] in (64, 128, 256)
    assert st["bins_per_cutoff"] in (1, 2) and st["bin_order"] in (0, 1)
    lines = cache.read_text().splitlines()
    assert len(lines) == 1 and f"N={n}|" in lines[0] and '"median_us"' in lines[0]
    assert f'"bins_per_cutoff": {st["bins_per_cutoff"]}' in lines[0] and '"R2z"' in lines[0]
    assert '"bin_order": "%s"' % "xz"[st["bin_order"]] in lines[0]
    # a second handle on the same workload takes the cached choice without re-timing
    h = sedi.Sedi(dict(prm, precision_form="split"))
    h.set_particles(sub["x"], sub["v"], sub["w"], sub["d"], sub["rho"])
    h.step(200)
    h.step(10)
    assert h.stats()["substep_variant"] == st["substep_variant"]
    assert h.stats()["bins_per_cutoff"] == st["bins_per_cutoff"]
    assert h.stats()["bin_order"] == st["bin_order"]
    assert len(cache.read_text().splitlines()) == 1
    # the tuned run is the same trajectory as a fixed variant on bins of one cutoff
    f = sedi.Sedi(dict(prm, precision_form="split", substep_variant=0, bins_per_cutoff=1, bin_order=0))
    f.set_particles(sub["x"], sub["v"], sub["w"], sub["d"], sub["rho"])
    f.step(200)
    f.step(10)
    for a, b in zip(h.get_particles(), f.get_particles()):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("form", ["fp64", "split"])
def test_deposition_bit_exact(small, form):
    prm, parts = small
    g, o = make_pair(prm, parts, form)
    rng = np.random.default_rng(4)
    C = int(np.prod(prm["ncell"]))
    U, DU = rng.normal(0, 0.05, (C, 3)), rng.normal(0, 0.5, (C, 3))
    for h in (g, o):
        h.set_fluid(U=U, DUDt=DU)
    qg, qo = g.deposit(), o.deposit()
    assert np.array_equal(qg[:4], qo[:4])
    Sf = prm["shift_force"]
    Fg = np.ldexp(qg[4:].astype(float), -Sf)
    Fo = np.ldexp(qo[4:].astype(float), -Sf)
    assert rel_err(Fg, Fo) < FORCE_TOL[form] * 10 + 2.0 ** -Sf / max(np.abs(Fo).max(), 1e-300)


@pytest.mark.parametrize("form", ["fp64", "split"])
def test_smoothing_matches_oracle(small, form):
    prm, _ = small
    g = sedi.Sedi(dict(prm, precision_form=form))
    o = orc.Oracle(prm)
    rng = np.random.default_rng(5)
    C = int(np.prod(prm["ncell"]))
    phi = rng.random((7, C))
    phi[rng.random((7, C)) < 0.6] = 0.0
    sg, itg = g.smooth(phi)
    so, ito = o.smooth(phi)
    # Chebyshev iterations on the GPU, CG in the oracle: same system, same tolerance
    assert np.all(itg > 0)
    assert np.all(itg <= 2 * ito + 4 * prm["n_tau"])
    for f in range(7):
        assert np.abs(sg[f] - so[f]).max() <= 1e-7 * np.abs(phi[f]).max()
        assert abs(sg[f].sum() - phi[f].sum()) <= 1e-9 * phi[f].sum()


@pytest.mark.parametrize("form", ["fp64", "split"])
def test_bdf2_smoothing_matches_oracle(small, form):
    # BDF2 pseudo-time (second-order implicit scheme of Sec. 2.4): operator
    # I - (2/3) dtau D L after a backward-Euler first step, right-hand side
    # (4/3) phi^m - (1/3) phi^{m-1}
    prm, _ = small
    prm = dict(prm, tau_scheme=1)
    g = sedi.Sedi(dict(prm, precision_form=form))
    o = orc.Oracle(prm)
    rng = np.random.default_rng(6)
    C = int(np.prod(prm["ncell"]))
    phi = rng.random((7, C))
    phi[rng.random((7, C)) < 0.6] = 0.0
    sg, itg = g.smooth(phi)
    so, _ = o.smooth(phi)
    se, _ = orc.Oracle(dict(prm, tau_scheme=0)).smooth(phi)
    assert np.all(itg > 0)
    for f in range(7):
        scale = np.abs(phi[f]).max()
        assert np.abs(sg[f] - so[f]).max() <= 1e-7 * scale
        assert abs(sg[f].sum() - phi[f].sum()) <= 1e-9 * phi[f].sum()
        # a different scheme: the result moves well beyond the tolerance
        assert np.abs(so[f] - se[f]).max() > 1e-4 * scale


def test_bdf2_grid_solver_mesh():
    # 96 x 96 planes hold more cells than one CTA of the cluster solver, so this mesh
    # takes the grid solver in the split form
    prm = default_params(hi=(96e-3, 96e-3, 24e-3), ncell=(96, 96, 24), wall_hi=(0, 0, 0),
                         bandwidth=(2e-3, 2e-3, 1.5e-3), tau_scheme=1)
    g = sedi.Sedi(dict(prm, precision_form="split"))
    o = orc.Oracle(prm)
    rng = np.random.default_rng(9)
    C = int(np.prod(prm["ncell"]))
    phi = rng.random((2, C)) * (rng.random((2, C)) < 0.3)
    sg, _ = g.smooth(phi)
    so, _ = o.smooth(phi)
    assert np.abs(sg - so).max() <= 1e-7 * np.abs(phi).max()


def test_anisotropic_bandwidth_matches_oracle():
    # Case-3 bandwidths of Sec. 4.3: 4 d horizontally, 2 d vertically (d = 0.5 mm), on
    # the benchmark's 64 x 32 x 64 mesh of 1 mm cells
    d = 0.5e-3
    prm = default_params(hi=(64e-3, 32e-3, 64e-3), ncell=(64, 32, 64), wall_hi=(0, 0, 0),
                         bandwidth=(4 * d, 4 * d, 2 * d))
    g = sedi.Sedi(dict(prm, precision_form="split"))
    o = orc.Oracle(prm)
    rng = np.random.default_rng(10)
    C = int(np.prod(prm["ncell"]))
    phi = rng.random((3, C)) * (rng.random((3, C)) < 0.3)
    sg, _ = g.smooth(phi)
    so, _ = o.smooth(phi)
    si, _ = orc.Oracle(dict(prm, bandwidth=(4 * d,) * 3)).smooth(phi)
    scale = np.abs(phi).max()
    assert np.abs(sg - so).max() <= 1e-7 * scale
    assert np.abs(so - si).max() > 1e-3 * scale


def test_bdf2_rejects_learned_guess(small):
    prm, _ = small
    with pytest.raises(sedi.SediError):
        sedi.Sedi(dict(prm, tau_scheme=1, use_cnn_guess=1))
    with pytest.raises(sedi.SediError):
        sedi.Sedi(dict(prm, tau_scheme=2))


def test_smoothing_guess_and_large_mesh():
    prm = default_params(hi=(64e-3, 32e-3, 64e-3), ncell=(64, 32, 64), wall_hi=(0, 0, 0),
                         bandwidth=(1.5e-3,) * 3)
    g = sedi.Sedi(dict(prm, precision_form="split"))
    o = orc.Oracle(prm)
    rng = np.random.default_rng(8)
    C = int(np.prod(prm["ncell"]))
    phi = rng.random((2, C)) * (rng.random((2, C)) < 0.3)
    guess = phi * 0.5 + 0.01
    sg, _ = g.smooth(phi, guess=guess)
    so, _ = o.smooth(phi, guess=guess)
    assert np.abs(sg - so).max() <= 1e-7 * np.abs(phi).max()


@pytest.mark.parametrize("form", ["fp64", "split"])
def test_average_matches_oracle(small, form):
    prm, parts = small
    g, o = make_pair(prm, parts, form)
    eg, ug, Fg = g.average()
    eo, uo, Fo = o.average()
    assert np.abs(eg - eo).max() <= 1e-7 * np.abs(eo).max()
    mask = eo > 1e-3 * eo.max()
    assert np.abs(ug[mask] - uo[mask]).max() <= 1e-5 * np.abs(uo[mask]).max()
    assert rel_err(Fg, Fo) <= 1e-4
    # conservation of solid volume: sum(eps) V_c = sum(V_p)
    vc = np.prod((np.array(prm["hi"]) - np.array(prm["lo"])) / np.array(prm["ncell"]))
    vp = (np.pi / 6 * parts["d"] ** 3).sum()
    assert abs(eg.sum() * vc - vp) <= 1e-9 * vp


def test_momentum_conserved_on_gpu(small):
    prm0, parts = small
    prm = dict(prm0, periodic=(1, 1, 1), wall_lo=(0, 0, 0), wall_hi=(0, 0, 0), g=(0, 0, 0),
               drag=0, pressure_grad=0, added_mass=0)
    g = sedi.Sedi(dict(prm, precision_form="split"))
    g.set_particles(parts["x"], parts["v"], parts["w"], parts["d"], parts["rho"])
    g.step(50)
    f = g.compute_forces()
    F = f["contact"] + f["lub"]
    assert np.abs(F).sum() > 0
    assert np.abs(F.sum(0)).max() <= 1e-6 * np.abs(F).sum()


@pytest.mark.parametrize("variant,resume_variant", [(-1, -1), (8, 8), (8, 5), (9, 8)])
def test_checkpoint_resume_bit_identical(small, tmp_path, variant, resume_variant):
    # variant 8 keeps a pair list (rebuilt from the loaded neighbour lists) and each
    # pair's spring in one slot; the checkpoint holds both copies, so another
    # variant resumes the same trajectory
    prm, parts = small
    g = sedi.Sedi(dict(prm, precision_form="split", substep_variant=variant))
    g.set_particles(parts["x"], parts["v"], parts["w"], parts["d"], parts["rho"])
    g.step(25)
    g.average()
    path = tmp_path / "ck.bin"
    g.save_state(path)
    g.step(40)
    ref = g.get_particles()
    h = sedi.Sedi(dict(prm, precision_form="split", substep_variant=resume_variant))
    h.load_state(path)
    h.n = len(parts["x"])
    h.step(40)
    got = h.get_particles()
    for a, b in zip(ref, got):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("bins,order", [(2, 1), (1, 1), (2, 0)])
def test_checkpoint_keeps_its_bins(small, tmp_path, bins, order):
    """A checkpoint stores its particles in the order of its bins (size and storage
    order); a handle whose own bins differ loads it on the stored bins and resumes the
    same trajectory."""
    prm, parts = small
    g = sedi.Sedi(dict(prm, precision_form="split", substep_variant=8, bins_per_cutoff=bins,
                       bin_order=order))
    g.set_particles(parts["x"], parts["v"], parts["w"], parts["d"], parts["rho"])
    g.step(30)
    path = tmp_path / "ck.bin"
    g.save_state(path)
    g.step(30)
    ref = g.get_particles()
    h = sedi.Sedi(dict(prm, precision_form="split", substep_variant=8))
    h.load_state(path)
    h.n = len(parts["x"])
    st = h.stats()
    assert st["bins_per_cutoff"] == bins and st["bin_order"] == order
    h.step(30)
    for a, b in zip(ref, h.get_particles()):
        assert np.array_equal(a, b)


def test_single_particle_and_boundaries():
    prm = default_params()
    hi = np.array(prm["hi"])
    x = np.array([[0.0, hi[1] * (1 - 1e-16), 0.5e-3], [hi[0] - 1e-12, 0.0, 20e-3]])
    for n in (1, 2):
        parts = dict(x=x[:n], v=np.zeros((n, 3)), w=np.zeros((n, 3)), d=np.full(n, 1e-3),
                     rho=np.full(n, 2500.0))
        g, o = make_pair(prm, parts, "split")
        g.step(50)
        o.step(50)
        # the same periodic point may be reported as hi or lo
        assert np.abs(min_image(g.get_particles()[0] - o.get_particles()[0], prm)).max() < 1e-9


def test_pair_list_without_pairs():
    """Spheres too far apart to be listed together: the pair list is empty, every
    block of the ordered pair schedule finds its first claim past the end (and the last
    resets the counter for the next launch); both pair-list variants give the bits of
    the per-particle loop, and the oracle's trajectory."""
    prm = default_params()
    g1 = np.stack(np.meshgrid([5e-3, 15e-3], [5e-3, 15e-3], [10e-3, 20e-3], indexing="ij"), -1).reshape(-1, 3)
    n = len(g1)
    parts = dict(x=g1, v=np.zeros((n, 3)), w=np.zeros((n, 3)), d=np.full(n, 1e-3), rho=np.full(n, 2500.0))
    out = []
    for v in (5, 8, 9):
        g = sedi.Sedi(dict(prm, precision_form="split", substep_variant=v))
        g.set_particles(parts["x"], parts["v"], parts["w"], parts["d"], parts["rho"])
        for _ in range(3):
            g.step(20)
        assert g.contacts()[0].shape[0] == 0
        out.append(g.get_particles())
    for other in out[1:]:
        for a, b in zip(out[0], other):
            assert np.array_equal(a, b)
    o = orc.Oracle(prm, threads=1)
    o.set_particles(*(storage_round(parts[k], "split") for k in ("x", "v", "w")), parts["d"], parts["rho"])
    o.step(60)
    assert np.abs(min_image(out[0][0] - o.get_particles()[0], prm)).max() <= 1e-4 * 1e-3


def test_profile_timings_in_graphs(small):
    prm, parts = small
    g = sedi.Sedi(dict(prm, precision_form="split", profile=1))
    g.set_particles(parts["x"], parts["v"], parts["w"], parts["d"], parts["rho"])
    for _ in range(3):
        g.step(20)
        g.average_inplace()
    t = g.timings()
    assert t["substep_n"] == 60 and t["rebuild_n"] == 60
    assert t["deposit_n"] == 3 and t["smooth_n"] == 3
    assert t["substep_ms"] > 0 and t["smooth_ms"] > 0


def test_errors_are_reported(small):
    prm, parts = small
    with pytest.raises(sedi.SediError):
        sedi.Sedi(dict(prm, restitution=0.0))
    with pytest.raises(sedi.SediError):
        sedi.Sedi(dict(prm, substep_variant=10))
    g = sedi.Sedi(dict(prm, precision_form="split", nbr_capacity=2))
    with pytest.raises(sedi.SediError) as e:
        g.set_particles(parts["x"], parts["v"], parts["w"], parts["d"], parts["rho"])
    assert e.value.code == -4
    g = sedi.Sedi(dict(prm, precision_form="split"))
    with pytest.raises(sedi.SediError) as e:
        g.step(1)
    assert e.value.code == -9
    bad = dict(parts, d=-parts["d"])
    with pytest.raises(sedi.SediError):
        g.set_particles(bad["x"], bad["v"], bad["w"], bad["d"], bad["rho"])
    g = sedi.Sedi(dict(prm, precision_form="split", cg_max_iter=1))
    g.set_particles(parts["x"], parts["v"], parts["w"], parts["d"], parts["rho"])
    with pytest.raises(sedi.SediError) as e:
        g.average()
    assert e.value.code == -6
    # the handle stays usable after the reported error
    g.step(3)
    g.sync()


def test_device_pointers_and_stream(small):
    prm, parts = small
    s = torch.cuda.Stream()
    g = sedi.Sedi(dict(prm, precision_form="split"), stream=s)
    dev = {k: torch.as_tensor(v, device="cuda") for k, v in parts.items()}
    g.set_particles(dev["x"], dev["v"], dev["w"], dev["d"], dev["rho"])
    g.step(10)
    out = torch.zeros((len(parts["x"]), 3), dtype=torch.float64, device="cuda")
    g.get_positions(out)
    torch.cuda.synchronize()
    h = sedi.Sedi(dict(prm, precision_form="split"))
    h.set_particles(parts["x"], parts["v"], parts["w"], parts["d"], parts["rho"])
    h.step(10)
    assert np.array_equal(out.cpu().numpy(), h.get_particles()[0])


@pytest.mark.skipif(os.environ.get("SEDI_SKIP_LARGE") == "1", reason="large case disabled")
def test_full_size_bed_forces_springs_and_lists():
    """The 200k-sphere settled bed at full size, in the launch configuration the
    benchmark uses (split form, CUDA graphs, the pair-list launch variant): lists
    bit-exact at the start, then both sides run 20 substeps from the same inputs, so
    the comparison carries tangential history -- springs (SPRING_TOL), positions
    (1e-4 d) and the forces at the reached state (1e-5 of the largest force of each
    kind, springs included), and the same 20 substeps of the per-particle loop and of
    the ordered pair schedule give the same bits as the pair list."""
    prm, parts, fl = bed_case()
    rng = np.random.default_rng(17)
    n = len(parts["x"])
    parts = dict(parts, v=rng.normal(0, 0.01, (n, 3)), w=rng.normal(0, 20.0, (n, 3)))
    C = int(np.prod(prm["ncell"]))
    eps = rng.uniform(0.0, 0.6, C)
    g, o = make_pair(prm, parts, "split", threads=os.cpu_count() or 1, use_graphs=1,
                     substep_variant=8)
    for h in (g, o):
        h.set_fluid(U=fl["U"])
        h.set_eps(eps)
    off_g, ids_g = g.neighbors()
    off_o, ids_o = o.neighbors(prm["skin"], brute=False)
    assert np.array_equal(off_g, off_o) and np.array_equal(ids_g, ids_o)
    g.step(20)
    o.step(20)
    assert compare_springs(g, o, prm, parts, "split") > n  # more than one spring per two spheres
    xg, xo = g.get_particles()[0], o.get_particles()[0]
    assert (np.abs(min_image(xg - xo, prm)).max(axis=1) / parts["d"]).max() <= 1e-4
    fg, fo = g.compute_forces(), o.forces()
    for k in ("contact", "lub", "fluid", "torque"):
        assert rel_err(fg[k], fo[k]) <= 1e-5, (k, rel_err(fg[k], fo[k]))
    # the per-particle loop and the ordered pair schedule: the same bits
    for v in (5, 9):
        loop = sedi.Sedi(dict(prm, precision_form="split", use_graphs=1, substep_variant=v))
        loop.set_particles(parts["x"], parts["v"], parts["w"], parts["d"], parts["rho"])
        loop.set_fluid(U=fl["U"])
        loop.set_eps(eps)
        loop.step(20)
        for a, b in zip(loop.get_particles(), g.get_particles()):
            assert np.array_equal(a, b), v


@pytest.mark.skipif(os.environ.get("SEDI_SKIP_LARGE") == "1", reason="large case disabled")
def test_large_bed_window_forces_and_lists():
    """The 10M-sphere bed at full size, sampled: forces and lists come from the full
    10M launch; the oracle gets a mesh-aligned window of the same state.  Spheres
    deeper inside the window than the list cut-off (plus two cells) have all their
    partners and interpolation cells inside it, so their forces (split form, 1e-5 of
    the largest force of each kind) and lists (bit-exact) must agree."""
    from paper_1601_03801_gb300.workloads import large_case

    prm, parts, fl = large_case()
    rng = np.random.default_rng(19)
    n = len(parts["x"])
    v = rng.normal(0, 0.01, (n, 3))
    w = rng.normal(0, 20.0, (n, 3))
    eps = rng.uniform(0.0, 0.6, int(np.prod(prm["ncell"])))
    full = sedi.Sedi(dict(prm, precision_form="split"))
    full.set_particles(parts["x"], v, w, parts["d"], parts["rho"])
    full.set_fluid(U=fl["U"], DUDt=fl["DUDt"])
    full.set_eps(eps)
    fg = full.compute_forces()
    # the oracle's window gets the library's storage of the same inputs
    x, v, w = (storage_round(a, "split") for a in (parts["x"], v, w))
    nc = np.array(prm["ncell"])
    h = (np.array(prm["hi"]) - np.array(prm["lo"])) / nc
    c0 = np.array([120, 60, 0]); c1 = np.array([136, 76, nc[2]])  # window in cells
    lo = c0 * h; hi = c1 * h
    idx = np.nonzero(np.all((x >= lo) & (x < hi), axis=1))[0]
    wprm = dict(prm, lo=tuple(lo), hi=tuple(hi), ncell=tuple(c1 - c0), periodic=(0, 0, 0),
                wall_lo=(0, 0, 1), wall_hi=(0, 0, 0))

    def sub(f, k):
        return f.reshape(nc[2], nc[1], nc[0], k)[c0[2]:c1[2], c0[1]:c1[1], c0[0]:c1[0]].reshape(-1, k)

    o = orc.Oracle(wprm)
    o.set_particles(x[idx], v[idx], w[idx], parts["d"][idx], parts["rho"][idx])
    o.set_fluid(U=sub(fl["U"], 3), DUDt=sub(fl["DUDt"], 3))
    o.set_eps(sub(eps.reshape(-1, 1), 1)[:, 0])
    fo = o.forces()
    cut = 2 * parts["d"].max() * (1 + prm["lub_h_out_frac"]) + prm["skin"] + 2 * h.max()
    xi = x[idx]
    deep = np.all((xi[:, :2] >= lo[:2] + cut) & (xi[:, :2] < hi[:2] - cut), axis=1)
    assert deep.sum() > 1000
    for k in ("contact", "lub", "fluid", "torque"):
        assert rel_err(fg[k][idx[deep]], fo[k][deep]) <= 1e-5, k
    off_g, ids_g = full.neighbors()
    off_o, ids_o = o.neighbors(prm["skin"], brute=False)
    for li in np.nonzero(deep)[0][:3000]:
        gi = idx[li]
        want = np.sort(idx[ids_o[off_o[li]:off_o[li + 1]]])
        assert np.array_equal(ids_g[off_g[gi]:off_g[gi + 1]], want)
