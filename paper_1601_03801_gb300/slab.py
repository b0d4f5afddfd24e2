"""Slab decomposition of one bed over several ranks (the parallel coupling of Sec. 3,
"consistent subdomains": particles and mesh split the same way along x).

The box is cut into x-slabs on cell faces, one per rank; rank r owns the spheres whose
centre lies in its slab.  Every substep each rank
  1. receives copies of the spheres that other ranks own within `margin` of its slab
     (ghosts; x is periodic, so the first and last slabs are neighbours), with their
     lagged accelerations and wall springs and the springs of their pairs;
  2. loads owned + ghost spheres into its engine in ascending global id, so that the
     engine's caller-index order is the global order: the canonical orientation of every
     pair, the order of the partners in a list and the order of the force sums are those
     of the undivided bed;
  3. advances one substep and keeps its owned spheres' new state and the springs of
     every pair with an owned sphere (a pair that straddles two slabs is evaluated on
     both ranks from the same inputs, so both keep the same spring);
  4. hands the spheres that left its slab, with their springs, to the rank whose slab
     they entered.
At an averaging every rank deposits its owned spheres (PCM, 64-bit fixed point), the
depositions are summed over the ranks -- exact, so the sum is the undivided bed's
deposition bit for bit -- and every rank smooths the sum (the mesh is replicated: each
engine keeps the global box and mesh and only a local set of spheres).

The engine is the CUDA library (sedi.Sedi) or, in the CPU tests, the FP64 oracle behind
the same methods.  This module only moves data between ranks; every step of the method
runs in the engine.  Exchanges go through `comm`: ProcessGroupComm (one rank per
process, torch.distributed, gloo or NCCL) or LocalComm (every rank in this process, for
tests on one device: the ranks take turns, no kernel waits on another).
"""
from __future__ import annotations

import numpy as np

FIELDS = ("x", "v", "w", "a", "d", "rho")


class LocalComm:
    """Every rank in this process: the collectives see the contributions of all ranks."""

    def __init__(self, world):
        self.world = world

    def allgather(self, per_rank):
        return [list(per_rank) for _ in per_rank]

    def allreduce_sum(self, per_rank):
        total = np.sum(np.stack(per_rank), axis=0)
        return [total.copy() for _ in per_rank]


class ProcessGroupComm:
    """One rank per process over torch.distributed (the default process group)."""

    def __init__(self):
        import torch.distributed as dist
        self.dist = dist
        self.world = dist.get_world_size()

    def allgather(self, per_rank):
        (mine,) = per_rank
        out = [None] * self.world
        self.dist.all_gather_object(out, mine)
        return [out]

    def allreduce_sum(self, per_rank):
        import torch
        (mine,) = per_rank
        t = torch.from_numpy(np.ascontiguousarray(mine, dtype=np.int64).copy())
        if self.dist.get_backend() == "nccl":
            t = t.cuda()
        self.dist.all_reduce(t, op=self.dist.ReduceOp.SUM)
        return [t.cpu().numpy()]


def slab_bounds(prm, world):
    """x-bounds of the slabs on cell faces: rank r spans cells [c_r, c_{r+1})."""
    nx = prm["ncell"][0]
    lo, hi = prm["lo"][0], prm["hi"][0]
    cuts = [(r * nx) // world for r in range(world + 1)]
    h = (hi - lo) / nx
    edges = [lo + c * h for c in cuts]
    edges[-1] = hi
    return edges


def interaction_margin(prm, d_max):
    """Width of the ghost layer: the lubrication reach of the largest pair plus the skin."""
    return d_max * (1.0 + prm["lub_h_out_frac"]) + prm["skin"]


class SlabRank:
    """The owned spheres of one rank and its engine.

    parts: the whole bed (x, v, w, d, rho; optional a) in global-id order; the rank
    keeps the spheres of its slab.  make_engine(prm) returns a fresh engine with the
    global box and mesh; fluid(engine) sets its prescribed fluid fields."""

    def __init__(self, prm, parts, rank, world, make_engine, fluid=None):
        self.prm = dict(prm)
        self.rank, self.world = rank, world
        self.edges = slab_bounds(prm, world)
        self.L = prm["hi"][0] - prm["lo"][0]
        self.lo_x, self.hi_x = self.edges[rank], self.edges[rank + 1]
        d = np.asarray(parts["d"], float)
        self.margin = interaction_margin(prm, float(d.max()))
        n = len(d)
        gid = np.arange(n, dtype=np.int64)
        mine = self._inside(np.asarray(parts["x"])[:, 0])
        self.gid = gid[mine]
        self.s = {}
        for k in FIELDS:
            if k == "a":
                a = parts.get("a")
                self.s[k] = np.zeros((mine.sum(), 3)) if a is None else np.asarray(a, float)[mine].copy()
            else:
                self.s[k] = np.asarray(parts[k], float)[mine].copy()
        self.wall = np.zeros((len(self.gid), 6, 3))
        self.springs = {}  # (gi, gj), gi < gj -> spring as seen from gi
        self.engine = make_engine(self.prm)
        if fluid is not None:
            fluid(self.engine)

    def _inside(self, x):
        return (x >= self.lo_x) & (x < self.hi_x)

    def _near(self, x):
        """Within `margin` of this slab along x, on the periodic axis."""
        c = 0.5 * (self.lo_x + self.hi_x)
        half = 0.5 * (self.hi_x - self.lo_x) + self.margin
        dx = x - c
        dx -= self.L * np.round(dx / self.L)
        return np.abs(dx) < half

    def _payload(self, sel):
        gid = self.gid[sel]
        ids = set(gid.tolist())
        sp = {k: v for k, v in self.springs.items() if k[0] in ids or k[1] in ids}
        return {"gid": gid, **{k: self.s[k][sel] for k in FIELDS}, "wall": self.wall[sel], "springs": sp}

    def boundary(self):
        """Owned spheres that some other slab may need as ghosts (within `margin` of
        this slab's faces)."""
        x = self.s["x"][:, 0]
        dl = (x - self.lo_x) % self.L
        dr = (self.hi_x - x) % self.L
        return self._payload((dl < self.margin) | (dr < self.margin))

    def substep(self, gathered):
        """One substep of owned + ghost spheres; keeps the owned results."""
        ghosts = [p for r, p in enumerate(gathered) if r != self.rank]
        g_gid = [p["gid"] for p in ghosts]
        keep = [self._near(p["x"][:, 0]) for p in ghosts]
        gid = np.concatenate([self.gid] + [g[k] for g, k in zip(g_gid, keep)])
        cat = {k: np.concatenate([self.s[k]] + [p[k][m] for p, m in zip(ghosts, keep)])
               for k in FIELDS}
        wall = np.concatenate([self.wall] + [p["wall"][m] for p, m in zip(ghosts, keep)])
        order = np.argsort(gid, kind="stable")
        gid, wall = gid[order], wall[order]
        cat = {k: v[order] for k, v in cat.items()}
        local = {g: i for i, g in enumerate(gid.tolist())}
        springs = dict(self.springs)
        for p in ghosts:
            for key, xi in p["springs"].items():
                springs.setdefault(key, xi)
        pairs = [(local[a], local[b], xi) for (a, b), xi in springs.items() if a in local and b in local]
        e = self.engine
        e.set_particles(cat["x"], cat["v"], cat["w"], cat["d"], cat["rho"])
        e.set_accel(cat["a"])
        e.set_wall_springs(wall)
        if pairs:
            e.set_contacts(np.array([(i, j) for i, j, _ in pairs], dtype=np.int64),
                           np.array([xi for _, _, xi in pairs], dtype=float))
        else:
            e.set_contacts(np.zeros((0, 2), dtype=np.int64), np.zeros((0, 3)))
        e.step(1)
        x, v, w, a = e.get_particles()
        own = np.isin(gid, self.gid)
        self.gid = gid[own]
        for k, val in (("x", x), ("v", v), ("w", w), ("a", a)):
            self.s[k] = val[own]
        for k in ("d", "rho"):
            self.s[k] = cat[k][own]
        self.wall = e.wall_springs()[own]
        ij, xi = e.contacts()
        gi, gj = gid[ij[:, 0]], gid[ij[:, 1]]
        mine = set(self.gid.tolist())
        self.springs = {(int(a), int(b)): xi[k] for k, (a, b) in enumerate(zip(gi, gj))
                        if int(a) in mine or int(b) in mine}

    def leavers(self):
        """Owned spheres that left this slab (removed here, with their springs)."""
        gone = ~self._inside(self.s["x"][:, 0])
        out = self._payload(gone)
        keep = ~gone
        self.gid = self.gid[keep]
        self.s = {k: v[keep] for k, v in self.s.items()}
        self.wall = self.wall[keep]
        mine = set(self.gid.tolist())
        self.springs = {k: v for k, v in self.springs.items() if k[0] in mine or k[1] in mine}
        return out

    def adopt(self, gathered):
        """Take the spheres that entered this slab from the other ranks' leavers."""
        for r, p in enumerate(gathered):
            if r == self.rank or len(p["gid"]) == 0:
                continue
            m = self._inside(p["x"][:, 0])
            if not m.any():
                continue
            self.gid = np.concatenate([self.gid, p["gid"][m]])
            for k in FIELDS:
                self.s[k] = np.concatenate([self.s[k], p[k][m]])
            self.wall = np.concatenate([self.wall, p["wall"][m]])
            new = set(p["gid"][m].tolist())
            for key, xi in p["springs"].items():
                if key[0] in new or key[1] in new:
                    self.springs[key] = xi
        order = np.argsort(self.gid, kind="stable")
        self.gid = self.gid[order]
        self.s = {k: v[order] for k, v in self.s.items()}
        self.wall = self.wall[order]

    def deposit(self):
        """PCM deposition of the owned spheres into the global mesh (int64 [7][C])."""
        e = self.engine
        e.set_particles(self.s["x"], self.s["v"], self.s["w"], self.s["d"], self.s["rho"])
        e.set_accel(self.s["a"])
        return e.deposit()

    def average(self, q_total):
        """Smoothing of the summed deposition (every rank the same global fields)."""
        return self.engine.average_deposit(q_total)


def substeps(ranks, comm, n):
    """n substeps of the ranks held in this process (all of them with LocalComm, this
    process's rank with ProcessGroupComm)."""
    for _ in range(n):
        per = comm.allgather([r.boundary() for r in ranks])
        for r, gathered in zip(ranks, per):
            r.substep(gathered)
        per = comm.allgather([r.leavers() for r in ranks])
        for r, gathered in zip(ranks, per):
            r.adopt(gathered)


def average(ranks, comm):
    """The averaging of the whole bed from the ranks' depositions; returns, per rank
    held here, (eps_s, U_s, F_fp) of the global mesh."""
    q = comm.allreduce_sum([r.deposit() for r in ranks])
    return [r.average(qt) for r, qt in zip(ranks, q)]


def gather_state(ranks, comm, n_total):
    """The whole bed's state (x, v, w, a in global-id order) on every rank held here."""
    per = comm.allgather([{"gid": r.gid, **{k: r.s[k] for k in ("x", "v", "w", "a")}} for r in ranks])
    out = []
    for gathered in per:
        st = {k: np.zeros((n_total, 3)) for k in ("x", "v", "w", "a")}
        for p in gathered:
            for k in st:
                st[k][p["gid"]] = p[k]
        out.append(st)
    return out
