"""Slab decomposition with the CUDA library as the per-rank engine, on one GPU: the
ranks live in this process and take turns (LocalComm), so no kernel waits on another.

Two ranks must give the bits of one rank run through the same driver (each rank orders
its spheres by global id, so lists, pair orientation and sums follow the global order),
and agree with the undivided library run at the split-form trajectory tolerance (the
driver rebuilds the lists every substep, the undivided run between rebuilds, so their
partner slots -- and the FP32 summation order -- may differ)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1601_03801_gb300 import sedi, slab  # noqa: E402
from test_slab import case  # noqa: E402


def run_slabs(prm, parts, U, world, n_sub, form):
    def make(p):
        return sedi.Sedi(dict(p, precision_form=form, use_graphs=0))

    ranks = [slab.SlabRank(prm, parts, r, world, make, fluid=lambda e: e.set_fluid(U=U)) for r in range(world)]
    comm = slab.LocalComm(world)
    slab.substeps(ranks, comm, n_sub)
    avg = slab.average(ranks, comm)[0]
    st = slab.gather_state(ranks, comm, len(parts["x"]))[0]
    springs = {}
    for r in ranks:
        springs.update(r.springs)
    return st, springs, avg


@pytest.mark.parametrize("form", ["split", "fp64"])
def test_library_slabs_match_one_rank_and_the_undivided_run(form):
    prm, parts, U = case(2)
    one, sp1, avg1 = run_slabs(prm, parts, U, 1, 20, form)
    two, sp2, avg2 = run_slabs(prm, parts, U, 2, 20, form)
    for k in ("x", "v", "w", "a"):
        assert np.array_equal(one[k], two[k]), k
    assert sp1.keys() == sp2.keys() and len(sp1) > 20
    for key in sp1:
        assert np.array_equal(sp1[key], sp2[key]), key
    for a, b in zip(avg1, avg2):
        assert np.array_equal(a, b)
    g = sedi.Sedi(dict(prm, precision_form=form))
    g.set_particles(parts["x"], parts["v"], parts["w"], parts["d"], parts["rho"])
    g.set_fluid(U=U)
    g.step(20)
    eps, _, F = g.average()
    x = g.get_particles()[0]
    L = np.array(prm["hi"]) - np.array(prm["lo"])
    dx = two["x"] - x
    dx -= L * np.round(dx / L) * np.array(prm["periodic"])
    tol = 1e-10 if form == "fp64" else 1e-4
    assert (np.abs(dx).max(axis=1) / parts["d"]).max() <= tol
    assert np.abs(avg2[0] - eps).max() <= 1e-6 * np.abs(eps).max()
