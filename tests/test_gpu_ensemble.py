"""Ensembles of independent beds (n_beds > 1): one launch per phase over all beds
must give every bed exactly the bits it gets when run alone in a single-bed
handle, and an ensemble bed matches the FP64 oracle directly (forces, springs,
100-step trajectory, averaging)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from oracle import oracle as orc  # noqa: E402
from paper_1601_03801_gb300 import sedi  # noqa: E402
from paper_1601_03801_gb300.workloads import ensemble_case, storage_round  # noqa: E402


@pytest.fixture(scope="module")
def ens():
    # five beds of 300..3000 spheres on 16..48 mm meshes; a tight jittered lattice
    # so pairs are in contact from the first substep
    prm, beds = ensemble_case(n_beds=5, seed=77, n_min=300, n_max=3000, spacing=1.002, jitter=0.02)
    rng = np.random.default_rng(5)
    for bd in beds:
        bd["parts"]["v"] = rng.normal(0.0, 0.05, bd["parts"]["x"].shape)
    return prm, beds


def make_ensemble(prm, beds, **extra):
    g = sedi.Sedi(dict(prm, n_beds=len(beds), precision_form="split", **extra))
    for b, bd in enumerate(beds):
        g.set_bed(b, bd["lo"], bd["hi"], bd["ncell"])
        p = bd["parts"]
        g.set_particles(p["x"], p["v"], p["w"], p["d"], p["rho"], bed=b)
        g.set_fluid(U=bd["U"], bed=b)
    return g


def make_single(prm, bd, **extra):
    g = sedi.Sedi(dict(prm, lo=bd["lo"], hi=bd["hi"], ncell=bd["ncell"], precision_form="split", **extra))
    p = bd["parts"]
    g.set_particles(p["x"], p["v"], p["w"], p["d"], p["rho"])
    g.set_fluid(U=bd["U"])
    return g


def run(g, beds_idx, single):
    g.average_inplace()
    for _ in range(3):
        g.step(20)
        g.average_inplace()
    g.step(20)
    out = []
    for b in beds_idx:
        kw = {} if single else {"bed": b}
        x, v, w, a = g.get_particles(**kw)
        eps, Us, F = g.average(**kw)
        out.append((x, v, w, a, eps, Us, F))
    return out


@pytest.mark.parametrize("extra", [{}, {"lift": 1, "lub_tangential": 1}, {"z_grading": 3.0}])
def test_ensemble_bit_identical_to_single_beds(ens, extra):
    prm, beds = ens
    prm = dict(prm, **extra)
    E = make_ensemble(prm, beds)
    got = run(E, range(len(beds)), single=False)
    st = E.stats()
    assert st["substeps"] == 80 and st["averages"] >= 4 and st["cg_iterations"] > 0
    contacts = 0
    for b, bd in enumerate(beds):
        S = make_single(prm, bd)
        want = run(S, [0], single=True)[0]
        for k, (p, q) in enumerate(zip(got[b], want)):
            assert np.array_equal(p, q), (b, k)
        contacts += len(E.contacts(bed=b)[0])
    assert contacts > 0


def test_ensemble_bdf2_bit_identical_to_single_beds(ens):
    # the BDF2 pseudo-time scheme through the batched smoothing launch
    prm, beds = ens
    prm = dict(prm, tau_scheme=1)
    E = make_ensemble(prm, beds[:3])
    got = run(E, range(3), single=False)
    for b, bd in enumerate(beds[:3]):
        want = run(make_single(prm, bd), [0], single=True)[0]
        for k, (p, q) in enumerate(zip(got[b], want)):
            assert np.array_equal(p, q), (b, k)


def test_ensemble_graphs_equal_plain_launches(ens):
    prm, beds = ens
    res = []
    for graphs in (1, 0):
        E = make_ensemble(prm, beds, use_graphs=graphs)
        res.append(run(E, range(len(beds)), single=False))
    for a, b in zip(res[0], res[1]):
        for p, q in zip(a, b):
            assert np.array_equal(p, q)


def test_ensemble_checkpoint_resume(ens, tmp_path):
    prm, beds = ens
    E = make_ensemble(prm, beds)
    E.average_inplace()
    E.step(30)
    E.save_state(tmp_path / "ens.ck")
    E.step(25)
    want = [E.get_particles(bed=b) for b in range(len(beds))]
    R = make_ensemble(prm, beds)
    R.load_state(tmp_path / "ens.ck")
    R.step(25)
    for b in range(len(beds)):
        for p, q in zip(want[b], R.get_particles(bed=b)):
            assert np.array_equal(p, q), b


def test_ensemble_errors(ens):
    prm, beds = ens
    E = sedi.Sedi(dict(prm, n_beds=3, precision_form="split"))
    p = beds[0]["parts"]
    E.set_bed(0, beds[0]["lo"], beds[0]["hi"], beds[0]["ncell"])
    E.set_particles(p["x"], p["v"], p["w"], p["d"], p["rho"], bed=0)
    with pytest.raises(sedi.SediError) as e:
        E.step(1)  # beds 1 and 2 have no particles
    assert e.value.code == -9
    with pytest.raises(sedi.SediError) as e:
        E.set_particles(p["x"], p["v"], p["w"], p["d"], p["rho"], bed=3)
    assert e.value.code == -1
    single = sedi.Sedi(dict(prm, precision_form="split"))
    with pytest.raises(sedi.SediError):
        single.set_bed(0, beds[0]["lo"], beds[0]["hi"], beds[0]["ncell"])
    with pytest.raises(sedi.SediError):
        sedi.Sedi(dict(prm, n_beds=2000))


@pytest.mark.parametrize("b", [0, 4])
def test_ensemble_beds_match_oracle(ens, b):
    """One bed of the batched launches against the FP64 oracle on the same inputs:
    forces at the start (1e-5 of the largest force of each kind), springs after 20
    substeps (1e-5 of the largest spring), positions after 100 substeps (1e-4 d) and
    the averaged solid fraction (1e-6 of its maximum)."""
    prm, beds = ens
    E = make_ensemble(prm, beds)
    bd = beds[b]
    p = bd["parts"]
    o = orc.Oracle(dict(prm, lo=bd["lo"], hi=bd["hi"], ncell=bd["ncell"]))
    o.set_particles(*(storage_round(p[k], "split") for k in ("x", "v", "w")), p["d"], p["rho"])
    o.set_fluid(U=bd["U"])
    fg, fo = E.compute_forces(bed=b), o.forces()
    for k in ("contact", "lub", "fluid", "torque"):
        ref = np.abs(fo[k]).max()
        assert ref > 0 and np.abs(fg[k] - fo[k]).max() <= 1e-5 * ref, k
    E.step(20)
    o.step(20)
    ijg, xig = E.contacts(bed=b)
    ijo, xio = o.contacts()
    assert len(ijo) > 10 and np.array_equal(ijg, ijo)
    assert np.abs(xig - xio).max() <= 1e-5 * np.abs(xio).max()
    E.step(80)
    o.step(80)
    L = np.array(bd["hi"]) - np.array(bd["lo"])
    dx = E.get_particles(bed=b)[0] - o.get_particles()[0]
    dx -= L * np.round(dx / L) * np.array(prm["periodic"])
    assert (np.abs(dx).max(axis=1) / p["d"]).max() <= 1e-4
    eg = E.average(bed=b)[0]
    eo = o.average()[0]
    assert np.abs(eg - eo).max() <= 1e-6 * np.abs(eo).max()


def test_tuned_ensemble_keeps_each_bed_bits(ens):
    """After 200 substeps the ensemble times its launch shapes and bin sizes (every bed
    on the same choice) and keeps the cheapest; every bed still gets the bits it gets
    alone on a fixed shape and bins of one cutoff."""
    prm, beds = ens
    idx = [0, 1, 2]
    g = make_ensemble(prm, [beds[b] for b in idx])
    g.step(200)
    assert g.stats()["bins_per_cutoff"] == 1
    g.step(20)
    st = g.stats()
    assert st["substep_variant"] in (5, 7, 6, 0) and st["bins_per_cutoff"] in (1, 2)
    assert st["bin_order"] in (0, 1)
    got = [g.get_particles(bed=b) for b in range(len(idx))]
    for k, b in enumerate(idx):
        s = make_single(prm, beds[b], substep_variant=5, bins_per_cutoff=1, bin_order=0)
        s.step(200)
        s.step(20)
        for a, c in zip(got[k], s.get_particles()):
            assert np.array_equal(a, c), b


@pytest.mark.parametrize("variant", [5, 0])
def test_persistent_ensemble_launch_gives_the_graph_bits(ens, variant):
    """The substeps of a step in one persistent cooperative launch (grid barrier between
    substeps; a substep that leaves a bed needing a list rebuild ends the launch and the
    next one resumes after the rebuild) against the CUDA graph of batched launches: the
    same bits.  The beds move fast enough (0.5 m/s) to rebuild their lists mid-step."""
    prm, beds = ens
    rng = np.random.default_rng(21)
    fast = []
    for bd in beds[:3]:
        b = dict(bd, parts=dict(bd["parts"]))
        b["parts"]["v"] = rng.normal(0.0, 0.5, bd["parts"]["x"].shape)
        fast.append(b)
    out = []
    for persistent in (0, 1):
        g = make_ensemble(prm, fast, substep_variant=variant, ens_persistent=persistent)
        res = run(g, range(len(fast)), single=False)
        out.append((res, g.stats()))
    (r0, s0), (r1, s1) = out
    assert s1["rebuilds"] == s0["rebuilds"] and s1["rebuilds"] > 2 * len(fast)
    for a, b in zip(r0, r1):
        for x, y in zip(a, b):
            assert np.array_equal(x, y)


def test_persistent_ensemble_barrier_timeout_is_reported(ens, monkeypatch):
    """With the grid-barrier poll limit at 1 the first wait of the persistent launch runs
    out: every block returns and the step reports SEDI_ETIMEOUT; the device stays usable."""
    prm, beds = ens
    monkeypatch.setenv("SEDI_BARRIER_SPIN_LIMIT", "1")
    g = make_ensemble(prm, beds[:2], substep_variant=5, ens_persistent=1)
    monkeypatch.delenv("SEDI_BARRIER_SPIN_LIMIT")
    with pytest.raises(sedi.SediError) as e:
        g.step(20)
    assert e.value.code == -8
    h = make_ensemble(prm, beds[:2], substep_variant=5, ens_persistent=1)
    h.step(20)
    h.sync()

