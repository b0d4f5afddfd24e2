"""The oracle's multi-threaded particle loops give the same bits as its serial pair
loop (CPU only): forces, trajectories with springs, neighbour lists and averaging,
on the brute-force (1,000 spheres) and link-cell (6,000 spheres) pair searches."""
import numpy as np
import pytest

from paper_1601_03801_gb300.workloads import default_params, lattice_bed, small_case


def _cases():
    prm, parts = small_case(parity_addon=True)
    yield "small", prm, parts
    rng = np.random.default_rng(5)
    n, L, d = 6000, 8e-3, 0.5e-3
    x = lattice_bed(n, L, d, seed=6, jitter=0.02, spacing=1.002)
    prm = default_params(hi=(L, L, 8e-3), ncell=(8, 8, 8), wall_hi=(0, 0, 0), bandwidth=(1.5e-3,) * 3)
    parts = dict(x=x, v=rng.normal(0, 0.05, (n, 3)), w=rng.normal(0, 20.0, (n, 3)), d=np.full(n, d),
                 rho=np.full(n, 2500.0))
    yield "lattice", prm, parts


@pytest.mark.parametrize("case", ["small", "lattice"])
def test_threads_give_identical_bits(oracle_mod, case):
    name, prm, parts = next(c for c in _cases() if c[0] == case)
    C = int(np.prod(prm["ncell"]))
    U = np.random.default_rng(9).normal(0, 0.05, (C, 3))
    runs = []
    for threads in (1, 4):
        o = oracle_mod.Oracle(prm, threads=threads)
        o.set_particles(parts["x"], parts["v"], parts["w"], parts["d"], parts["rho"])
        o.set_fluid(U=U)
        f0 = o.forces()
        o.step(15)
        eps, Us, F = o.average()
        o.step(5)
        off, ids = o.neighbors(prm["skin"], brute=False)
        runs.append((f0, o.get_particles(), o.contacts(), o.wall_history(), (eps, Us, F), (off, ids)))
    (f1, p1, c1, w1, a1, n1), (f4, p4, c4, w4, a4, n4) = runs
    for k in f1:
        assert np.array_equal(f1[k], f4[k]), k
    for a, b in zip(p1 + c1 + a1 + n1, p4 + c4 + a4 + n4):
        assert np.array_equal(a, b)
    assert np.array_equal(w1, w4)
    assert len(c1[0]) > 20  # springs were carried through the steps
