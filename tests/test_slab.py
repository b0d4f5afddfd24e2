"""Slab decomposition of one bed over ranks (paper_1601_03801_gb300.slab), CPU only.

The per-rank engine here is the FP64 oracle behind the engine methods the driver calls.
Because every rank orders its spheres by global id and the ghost layer covers the
interaction range, the decomposed run must give the undivided oracle run's bits:
positions, velocities, spins, lagged accelerations, springs and the averaged fields.
Two and three ranks in one process (LocalComm), and two gloo processes
(ProcessGroupComm)."""
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_1601_03801_gb300 import slab
from paper_1601_03801_gb300.workloads import small_case

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


class OracleEngine:
    """The oracle behind the engine methods of the slab driver."""

    def __init__(self, prm, fluid):
        from oracle import oracle as orc
        self.o = orc.Oracle(prm)
        self.fluid = fluid

    def set_particles(self, x, v, w, d, rho):
        self.o.set_particles(x, v, w, d, rho)
        self.o.set_fluid(U=self.fluid["U"], DUDt=self.fluid.get("DUDt"))
        if self.fluid.get("eps") is not None:
            self.o.set_eps(self.fluid["eps"])

    def set_accel(self, a):
        self.o.set_accel(a)

    def set_wall_springs(self, xw):
        self.o.set_wall_history(xw)

    def set_contacts(self, ij, xi):
        self.o.set_contacts(ij, xi)

    def step(self, n):
        self.o.step(n)

    def get_particles(self):
        return self.o.get_particles()

    def wall_springs(self):
        return self.o.wall_history()

    def contacts(self):
        return self.o.contacts()

    def deposit(self):
        return self.o.deposit()

    def average_deposit(self, q):
        out = self.o.average_fixed(q)
        self.fluid["eps"] = out[0]  # the drag sees the smoothed solid fraction
        return out


def case(world=2):
    """The 1,000-sphere box with moving, touching spheres, plus two spheres placed at
    every slab face of `world` slabs (the periodic face x = 0 / 20 mm included), one
    moving across it each way."""
    prm, parts = small_case(parity_addon=True)
    parts = {k: np.array(v, copy=True) for k, v in parts.items()}
    rng = np.random.default_rng(11)
    faces = slab.slab_bounds(prm, world)[1:]
    movers = rng.choice(len(parts["x"]), 2 * len(faces), replace=False)
    for k, i in enumerate(movers):
        face = faces[k // 2]
        sign = 1.0 if k % 2 == 0 else -1.0
        parts["x"][i, 0] = (face - sign * 2e-7) % 20e-3
        parts["x"][i, 2] = 2e-3 + 3e-3 * k
        parts["v"][i] = [sign * 0.2, 0.0, 0.0]
    C = int(np.prod(prm["ncell"]))
    U = np.random.default_rng(12).normal(0, 0.05, (C, 3))
    return prm, parts, U


def undivided(prm, parts, U, n_sub, n_avg):
    from oracle import oracle as orc
    o = orc.Oracle(prm)
    o.set_particles(parts["x"], parts["v"], parts["w"], parts["d"], parts["rho"])
    o.set_fluid(U=U)
    avg = None
    for _ in range(n_avg):
        o.step(n_sub)
        avg = o.average()
    x, v, w, a = o.get_particles()
    return dict(x=x, v=v, w=w, a=a), o.contacts(), avg


def decomposed(prm, parts, U, n_sub, n_avg, world):
    fluid = {"U": U}
    ranks = [slab.SlabRank(prm, parts, r, world, lambda p: OracleEngine(p, dict(fluid))) for r in range(world)]
    comm = slab.LocalComm(world)
    avg = None
    for _ in range(n_avg):
        slab.substeps(ranks, comm, n_sub)
        avg = slab.average(ranks, comm)[0]
    state = slab.gather_state(ranks, comm, len(parts["x"]))[0]
    springs = {}
    for r in ranks:
        springs.update(r.springs)
    return state, springs, avg, ranks


@pytest.mark.parametrize("world", [2, 3])
def test_decomposed_run_gives_the_undivided_bits(world):
    prm, parts, U = case(world)
    want, (ij, xi), want_avg = undivided(prm, parts, U, 15, 2)
    got, springs, got_avg, ranks = decomposed(prm, parts, U, 15, 2, world)
    for k in ("x", "v", "w", "a"):
        assert np.array_equal(got[k], want[k]), k
    assert len(ij) > 20 and len(springs) == len(ij)
    for (i, j), s in zip(ij, xi):
        assert np.array_equal(springs[(int(i), int(j))], s)
    for g, w in zip(got_avg, want_avg):
        assert np.array_equal(g, w)
    # the face spheres crossed into the neighbouring slabs: ownership changed
    counts = [len(r.gid) for r in ranks]
    assert sum(counts) == len(parts["x"]) and min(counts) > 0
    start = [set(np.nonzero(r._inside(parts["x"][:, 0]))[0].tolist()) for r in ranks]
    moved = sum(len(s0 - set(r.gid.tolist())) for s0, r in zip(start, ranks))
    assert moved >= world, moved


def test_gloo_ranks_give_the_undivided_bits(tmp_path):
    """Two processes over gloo (127.0.0.1): rank 0 writes the gathered state."""
    prm, parts, U = case()
    want, _, want_avg = undivided(prm, parts, U, 10, 1)
    script = tmp_path / "run.py"
    script.write_text(f"""
import os, sys
sys.path.insert(0, {ROOT!r}); sys.path.insert(0, {os.path.dirname(os.path.abspath(__file__))!r})
import numpy as np, torch.distributed as dist
from paper_1601_03801_gb300 import slab
import test_slab as t
dist.init_process_group("gloo")
prm, parts, U = t.case()
fluid = {{"U": U}}
r = slab.SlabRank(prm, parts, dist.get_rank(), dist.get_world_size(), lambda p: t.OracleEngine(p, dict(fluid)))
comm = slab.ProcessGroupComm()
slab.substeps([r], comm, 10)
avg = slab.average([r], comm)[0]
st = slab.gather_state([r], comm, len(parts["x"]))[0]
if dist.get_rank() == 0:
    np.savez({str(tmp_path / "out.npz")!r}, eps=avg[0], F=avg[2], **st)
dist.barrier()
dist.destroy_process_group()
""")
    env = dict(os.environ, MASTER_ADDR="127.0.0.1", PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
                        "--master-addr=127.0.0.1", "--master-port=29561", str(script)],
                       capture_output=True, text=True, env=env, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    got = np.load(tmp_path / "out.npz")
    for k in ("x", "v", "w", "a"):
        assert np.array_equal(got[k], want[k]), k
    assert np.array_equal(got["eps"], want_avg[0]) and np.array_equal(got["F"], want_avg[2])
