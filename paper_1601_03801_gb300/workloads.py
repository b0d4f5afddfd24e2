"""Seeded synthetic inputs for the particle-side hot path.

This module only draws particles, diameters, velocities and prescribed fluid
fields; it holds none of the method's arithmetic (no contact law, drag,
deposition or smoothing).  The CUDA library and the FP64 oracle both consume
what it returns.

Workloads (the paper's Case 1 and Case 3 / sediment-transport scaling shapes,
Sec. 4.1, 4.3 and 5.2, Table 1; every one is synthetic):

* ``small``  : 1,000 glass spheres, d = 1 mm, in a 20 x 20 x 40 mm box, periodic
  in x and y, walls at z = 0 and z = 40 mm, quiescent water, 10 x 10 x 20 mesh.
* ``bed``    : 200,000 lognormal spheres (median 0.5 mm, sigma_ln = 0.1, cut at
  +-3 sigma) packed into a bed in a periodic 64 x 32 x 64 mm channel with a wall
  at z = 0, log-law flow u* = 0.02 m/s, 64 x 32 x 64 mesh.
* ``large``  : 10,000,000 spheres, d ~ U[0.4, 0.6] mm, 400 x 200 x 100 mm,
  256 x 128 x 64 mesh, mean flow 0.3 m/s plus filtered noise of rms 0.03 m/s.
* ``bounce`` : Case 1, one 6 mm sphere (sand or steel) released above the floor
  of a 100 x 100 x H mm box of quiescent fluid, the paper's linear contact
  (k_n = 800 N/m, e = 0.97, mu = 0.1); the viscosity sets the Stokes number.

Beds are made without the method (no contact law of the paper, no time
integration of it, no GPU): a small periodic block is seeded on an FCC lattice
near the final density and relaxed under gravity by FIRE energy minimisation of
a harmonic overlap energy (_fire_block), which gives the structure of a settled
bed (about five contacts per sphere at a packing fraction ~0.6); the block is
tiled over the channel.  The same inputs feed the CUDA library and the oracle.
"""
from __future__ import annotations

import os

import numpy as np

G = 9.81


def default_params(**over) -> dict:
    """Physical inputs shared by the CUDA library binding and the oracle."""
    p = dict(
        contact_law=0, E=1.0e7, poisson=0.3, restitution=0.9, friction=0.3,
        kn_linear=800.0, kt_ratio=2.0 / 7.0,
        rho_f=1000.0, nu_f=1.0e-6, g=(0.0, 0.0, -G),
        lo=(0.0, 0.0, 0.0), hi=(20e-3, 20e-3, 40e-3),
        periodic=(1, 1, 0), wall_lo=(0, 0, 1), wall_hi=(0, 0, 1),
        dt=1.0e-6,
        lubrication=1, drag=1, pressure_grad=1, added_mass=1,
        lub_h_in_frac=1.0e-3, lub_h_out_frac=0.1, c_add=0.5, eps_max=0.9,
        lift=0, c_lift=1.6, lub_tangential=0, z_grading=1.0,
        ncell=(10, 10, 20),
        bandwidth=(3e-3, 3e-3, 3e-3), n_tau=4, tau_scheme=0, cg_rtol=1e-8, cg_max_iter=500,
        shift_eps=40, shift_mom=40, shift_force=32,
        skin=0.05e-3,
    )
    for k, v in over.items():
        if k not in p:
            raise KeyError(k)
        p[k] = v
    return p


def _rng(seed):
    return np.random.default_rng(seed)


def rsa_spheres(n, d, lo, hi, periodic, seed, zmargin=True, max_tries=2_000_000):
    """Random sequential addition of n non-overlapping spheres of diameters d."""
    rng = _rng(seed)
    lo = np.asarray(lo, float); hi = np.asarray(hi, float); L = hi - lo
    d = np.broadcast_to(np.asarray(d, float), (n,)).copy()
    x = np.zeros((n, 3))
    placed = 0
    tries = 0
    while placed < n:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("rsa_spheres: box too full")
        r = 0.5 * d[placed]
        c = lo + rng.random(3) * L
        for a in range(3):
            if not periodic[a] and zmargin:
                c[a] = lo[a] + r + rng.random() * (L[a] - 2 * r)
        if placed:
            dx = x[:placed] - c
            for a in range(3):
                if periodic[a]:
                    dx[:, a] -= L[a] * np.round(dx[:, a] / L[a])
            dist2 = np.einsum("ij,ij->i", dx, dx)
            if np.any(dist2 < (0.5 * (d[:placed] + d[placed])) ** 2):
                continue
        x[placed] = c
        placed += 1
    return x, d


def small_case(seed=1601038011, parity_addon=False):
    """1,000 monodisperse glass spheres in quiescent water (Case-1-like box)."""
    prm = default_params()
    n = 1000
    x, d = rsa_spheres(n, 1e-3, prm["lo"], prm["hi"], prm["periodic"], seed)
    v = np.zeros((n, 3)); w = np.zeros((n, 3))
    rho = np.full(n, 2500.0)
    if parity_addon:
        rng = _rng(seed + 7)
        v = rng.normal(0.0, 0.1, (n, 3))
        # 5% of the spheres are moved to touch a partner with a small overlap
        k = n // 20
        movers = rng.choice(n, size=2 * k, replace=False)
        L = np.asarray(prm["hi"]) - np.asarray(prm["lo"])
        for a_i, b_i in movers.reshape(-1, 2):
            u = rng.normal(size=3); u /= np.linalg.norm(u)
            dist = 0.5 * (d[a_i] + d[b_i]) - 2e-6
            c = x[a_i] + dist * u
            c[2] = np.clip(c[2], prm["lo"][2] + 0.5 * d[b_i], prm["hi"][2] - 0.5 * d[b_i])
            for a in range(2):
                c[a] = prm["lo"][a] + np.mod(c[a] - prm["lo"][a], L[a])
            x[b_i] = c
            w[a_i] = rng.normal(0.0, 50.0, 3)
    return prm, dict(x=x, v=v, w=w, d=d, rho=rho)


def _fcc_block(n, d_all, Lx, Ly, spacing, seed):
    """First n sites of an FCC lattice filled from the floor up (periodic x, y)."""
    rng = _rng(seed)
    a = np.sqrt(2.0) * spacing
    nx = max(1, int(round(Lx / a))); ny = max(1, int(round(Ly / a)))
    ax = Lx / nx; ay = Ly / ny; az = a
    basis = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
    per_layer = nx * ny * 4
    nz = n // per_layer + 2
    ii, jj, kk = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    cells = np.stack([ii.ravel(), jj.ravel(), kk.ravel()], 1)
    sites = (cells[:, None, :] + basis[None, :, :]).reshape(-1, 3) * np.array([ax, ay, az])
    sites[:, 2] += 0.5 * d_all.max()
    order = np.lexsort((rng.random(len(sites)), sites[:, 2]))
    sites = sites[order[:n]]
    sites += rng.normal(0.0, 0.02 * spacing, sites.shape)
    sites[:, 0] %= Lx; sites[:, 1] %= Ly
    return sites


def _fire_block(d, Lx, Ly, seed, k=40.0, rho=2500.0, rho_f=1000.0, iters=6000):
    """A load-bearing packing of spheres of diameters d in a periodic Lx x Ly column
    standing on a floor at z = 0, made without the method's contact law or time
    integration: from a jittered FCC start near the final density (packing fraction
    ~0.56), the energy sum_pairs k/2 overlap^2 + sum_i buoyant weight_i z_i (a wall
    spring of 2k keeps the spheres above the floor) is lowered by FIRE (Bitzek,
    Koskinen, Gaehler, Moseler & Gumbsch, PRL 97, 170201, 2006) for a fixed number
    of iterations.  The spheres sink until the weight rests on a network of small
    overlaps (k = 40 N/m gives overlaps of ~1e-7 m under the weight of the bed, the
    order of a Hertz contact under the same load): about five contacts per sphere at
    a packing fraction ~0.6, the structure of a settled sediment bed.  The run is
    not converged to force balance; the method's own dynamics finish the settling.
    Pairs are kept in canonical (i, j) order so the sums run in a fixed order."""
    from scipy.sparse import csr_matrix
    from scipy.spatial import cKDTree

    n = len(d)
    r = 0.5 * d
    m = rho * np.pi / 6 * d ** 3
    g = G * (1.0 - rho_f / rho)
    a = (0.74 * np.mean(d ** 3) / 0.56) ** (1.0 / 3.0)  # FCC spacing for phi ~ 0.56
    x = _fcc_block(n, d, Lx, Ly, a, seed)
    v = np.zeros_like(x)
    skin = 0.2 * d.max()
    cut = d.max() + skin
    dt0 = 0.05 * np.sqrt(m.min() / k)
    dt, dt_max, alpha, n_pos = dt0, 10.0 * dt0, 0.1, 0
    per = np.array([Lx, Ly, 1.0])
    wrap = np.array([1.0, 1.0, 0.0])

    def pairs():
        xx = x.copy()
        xx[:, 0] %= Lx
        xx[:, 1] %= Ly
        p = cKDTree(xx, boxsize=(Lx, Ly, 1e9)).query_pairs(cut, output_type="ndarray")
        p = p[np.lexsort((p[:, 1], p[:, 0]))]
        i, j = p[:, 0], p[:, 1]
        q = np.arange(len(i))
        B = csr_matrix((np.concatenate([-np.ones(len(i)), np.ones(len(i))]),
                        (np.concatenate([i, j]), np.concatenate([q, q]))), shape=(n, len(i)))
        return i, j, r[i] + r[j], B

    i, j, s, B = pairs()
    x_ref = x.copy()
    weight = m[:, None] * np.array([0.0, 0.0, -g])
    inv_m = 1.0 / m[:, None]

    def force():
        dx = x[j] - x[i]
        dx -= wrap * per * np.round(dx / per)
        dist = np.sqrt(np.einsum("ij,ij->i", dx, dx))
        ov = np.maximum(s - dist, 0.0)
        F = weight + B @ ((k * ov / dist)[:, None] * dx)
        below = r - x[:, 2]
        F[:, 2] += np.where(below > 0, 2.0 * k * below, 0.0)
        return F

    F = force()
    for _ in range(iters):
        P = float(np.vdot(F, v))
        if P > 0:
            vn = np.sqrt(np.vdot(v, v))
            fn = np.sqrt(np.vdot(F, F))
            v = (1.0 - alpha) * v + (alpha * vn / max(fn, 1e-300)) * F
            n_pos += 1
            if n_pos > 5:
                dt = min(1.1 * dt, dt_max)
                alpha *= 0.99
        else:
            n_pos, dt, alpha = 0, 0.5 * dt, 0.1
            v[:] = 0.0
        v += dt * F * inv_m
        x += dt * v
        if np.abs(x - x_ref).max() > 0.5 * skin:
            i, j, s, B = pairs()
            x_ref = x.copy()
        F = force()
    x[:, 0] %= Lx
    x[:, 1] %= Ly
    x[:, 0] = np.where(x[:, 0] >= Lx, x[:, 0] - Lx, x[:, 0])
    x[:, 1] = np.where(x[:, 1] >= Ly, x[:, 1] - Ly, x[:, 1])
    return x


def _cache_path(tag):
    root = os.environ.get("SEDI_CACHE", "/tmp/sedi_workloads")
    os.makedirs(root, exist_ok=True)
    return os.path.join(root, tag + ".npz")


def settled_bed(n_total, tiles, block_xy, dsample, seed, iters=6000):
    """n_total spheres: one settled periodic block of n_total / prod(tiles) spheres
    (_fire_block) repeated tiles[0] x tiles[1] times over the floor.  Cached on disk
    (SEDI_CACHE, default /tmp/sedi_workloads) by its parameters."""
    tag = (f"fire1_{n_total}_{tiles[0]}x{tiles[1]}_{block_xy[0]:.4g}_{block_xy[1]:.4g}_{seed}_{iters}")
    path = _cache_path(tag)
    if os.path.exists(path):
        z = np.load(path)
        return z["x"], z["d"]
    nb = n_total // (tiles[0] * tiles[1])
    d = dsample(_rng(seed), nb)
    x = _fire_block(d, block_xy[0], block_xy[1], seed + 1, iters=iters)
    off = np.stack(np.meshgrid(np.arange(tiles[0]) * block_xy[0], np.arange(tiles[1]) * block_xy[1],
                               indexing="ij"), -1).reshape(-1, 2)
    X = np.repeat(x[None], len(off), 0)
    X[:, :, :2] += off[:, None, :]
    X = X.reshape(-1, 3)
    D = np.tile(d, len(off))
    # the offsets can round a coordinate up to the periodic bound: keep [0, L)
    for a in range(2):
        L = tiles[a] * block_xy[a]
        X[:, a] = np.where(X[:, a] >= L, X[:, a] - L, X[:, a])
        X[:, a] = np.minimum(X[:, a], np.nextafter(L, 0.0))
    np.savez(path, x=X, d=D)
    return X, D


def storage_round(a, form):
    """The value the CUDA library holds for an FP64 input in each arithmetic form: one
    FP32 word (plain), a pair of FP32 words hi + lo with hi = fl32(a) and
    lo = fl32(a - hi) (split: 48-bit significand), or the input itself (fp64).  Tests
    give the oracle these values, so both sides start from the same state without
    reading anything back from the CUDA path."""
    a = np.asarray(a, dtype=np.float64)
    if form == "fp64":
        return a.copy()
    hi = a.astype(np.float32).astype(np.float64)
    if form == "plain":
        return hi
    lo = (a - hi).astype(np.float32).astype(np.float64)
    return hi + lo


def lognormal_d(d50, sigma):
    def draw(rng, n):
        z = rng.normal(size=n)
        bad = np.abs(z) > 3
        while np.any(bad):
            z[bad] = rng.normal(size=int(bad.sum()))
            bad = np.abs(z) > 3
        return d50 * np.exp(sigma * z)
    return draw


def uniform_d(a, b):
    def draw(rng, n):
        return rng.uniform(a, b, n)
    return draw


def log_law(ncell, lo, hi, z_bed, u_star, z0):
    """Cell-centred log-law velocity u_x(z) = u*/0.41 ln(z'/z0), z' = z - z_bed."""
    nx, ny, nz = ncell
    dz = (hi[2] - lo[2]) / nz
    zc = lo[2] + (np.arange(nz) + 0.5) * dz
    zp = zc - z_bed
    ux = np.where(zp > z0, u_star / 0.41 * np.log(np.maximum(zp, z0) / z0), 0.0)
    U = np.zeros((nz, ny, nx, 3))
    U[..., 0] = ux[:, None, None]
    return U.reshape(-1, 3)


def bed_case(seed=1601038012, n=200_000):
    """Sheared sediment bed: 200,000 lognormal spheres (median 0.5 mm, sigma_ln 0.1,
    cut at +-3 sigma) settled into a bed (settled_bed: an 8 x 4 mm block of 3,125
    spheres tiled 8 x 8) in a periodic 64 x 32 x 64 mm channel, wall at z = 0, under
    the log-law flow u* = 0.02 m/s that starts at the bed top; 64 x 32 x 64 mesh."""
    Lx, Ly, Lz = 64e-3, 32e-3, 64e-3
    d50 = 0.5e-3
    tiles = (8, 8)
    x, d = settled_bed(n, tiles, (Lx / tiles[0], Ly / tiles[1]), lognormal_d(d50, 0.1), seed)
    prm = default_params(hi=(Lx, Ly, Lz), ncell=(64, 32, 64), wall_hi=(0, 0, 0),
                         bandwidth=(3 * d50,) * 3)
    nn = len(x)
    parts = dict(x=x, v=np.zeros((nn, 3)), w=np.zeros((nn, 3)), d=d, rho=np.full(nn, 2500.0))
    z_bed = float(np.quantile(x[:, 2] + 0.5 * d, 0.99))
    U = log_law(prm["ncell"], prm["lo"], prm["hi"], z_bed, 0.02, d50 / 30.0)
    return prm, parts, dict(U=U, z_bed=z_bed)


def lattice_bed(n, L, d, seed, jitter=0.01, spacing=1.05):
    """n spheres of diameter d on a square lattice filling a periodic L x L footprint
    layer by layer from the wall z = 0 (spacing >= `spacing` d in every direction),
    each moved by a uniform jitter of at most `jitter` d per axis (no overlaps while
    spacing - 2 sqrt(3) jitter > 1)."""
    rng = _rng(seed)
    m = int(np.floor(L / (spacing * d)))
    a = L / m                    # in-plane spacing (>= 1.05 d, periodic-consistent)
    per_layer = m * m
    k = np.arange(n)
    layer, r = k // per_layer, k % per_layer
    ix, iy = r % m, r // m
    x = np.stack([(ix + 0.5) * a, (iy + 0.5) * a, 0.5 * d + 0.05 * d + layer * spacing * d], axis=1)
    x += rng.uniform(-jitter * d, jitter * d, size=x.shape)
    x[:, 0] = np.mod(x[:, 0], L)
    x[:, 1] = np.mod(x[:, 1], L)
    x[:, :2] = np.where(x[:, :2] >= L, x[:, :2] - L, x[:, :2])
    return x


def ensemble_case(n_beds=256, seed=1601038014, n_min=2000, n_max=50000, d=0.5e-3, spacing=1.05,
                  jitter=0.01):
    """Ensemble of independent beds of uneven size: N_b = round(exp(U[ln n_min,
    ln n_max])), monodisperse d, a cubic periodic-x/y, wall-z box of n_b mm with an
    n_b^3 mesh (1 mm cells), n_b = 16 + round(32 (ln N_b - ln n_min) / (ln n_max -
    ln n_min)); the bed is a jittered lattice from the wall (height proportional
    to N_b / n_b^2) under the log-law flow of the 200k bed (u* = 0.02 m/s).
    Returns the shared parameters and a list of beds (box, mesh, parts, U)."""
    rng = _rng(seed)
    lnmin, lnmax = np.log(n_min), np.log(n_max)
    prm = default_params(wall_hi=(0, 0, 0), bandwidth=(3 * d,) * 3)
    beds = []
    for b in range(n_beds):
        t = rng.uniform(lnmin, lnmax)
        nb = int(round(np.exp(t)))
        side = 16 + int(round(32 * (t - lnmin) / (lnmax - lnmin)))
        L = side * 1e-3
        x = lattice_bed(nb, L, d, seed + 1 + b, jitter=jitter, spacing=spacing)
        lo, hi = (0.0, 0.0, 0.0), (L, L, L)
        ncell = (side, side, side)
        z_bed = float(x[:, 2].max() + 0.5 * d)
        U = log_law(ncell, lo, hi, z_bed, 0.02, d / 30.0)
        parts = dict(x=x, v=np.zeros((nb, 3)), w=np.zeros((nb, 3)), d=np.full(nb, d),
                     rho=np.full(nb, 2500.0))
        beds.append(dict(lo=lo, hi=hi, ncell=ncell, parts=parts, U=U, z_bed=z_bed))
    return prm, beds


def _gauss_filter_periodic(f, sigma_cells):
    """Gaussian filter with periodic wrap on every axis (FFT), noise preparation only."""
    out = f
    for ax in range(f.ndim):
        n = f.shape[ax]
        k = np.fft.fftfreq(n)
        g = np.exp(-2.0 * (np.pi * k * sigma_cells) ** 2)
        shape = [1] * f.ndim; shape[ax] = n
        out = np.real(np.fft.ifft(np.fft.fft(out, axis=ax) * g.reshape(shape), axis=ax))
    return out


def turbulent_like(ncell, lo, hi, mean=(0.3, 0.0, 0.0), rms=0.03, sigma_cells=2.0, seed=0):
    """Mean flow plus Gaussian-filtered white noise; DU/Dt = U . grad U (central)."""
    rng = _rng(seed)
    nx, ny, nz = ncell
    U = np.zeros((nz, ny, nx, 3))
    for c in range(3):
        f = _gauss_filter_periodic(rng.normal(size=(nz, ny, nx)), sigma_cells)
        f *= rms / f.std()
        U[..., c] = mean[c] + f
    h = [(hi[a] - lo[a]) / ncell[a] for a in range(3)]
    grads = []
    for ax_arr, hh in ((2, h[0]), (1, h[1]), (0, h[2])):
        grads.append((np.roll(U, -1, axis=ax_arr) - np.roll(U, 1, axis=ax_arr)) / (2 * hh))
    DU = U[..., 0:1] * grads[0] + U[..., 1:2] * grads[1] + U[..., 2:3] * grads[2]
    return U.reshape(-1, 3), DU.reshape(-1, 3)


def large_case(seed=1601038013, n=10_000_000):
    """10M spheres, d ~ U[0.4, 0.6] mm, settled into a bed (settled_bed: a 4 x 4 mm
    block of 2,000 spheres tiled 100 x 50, ~14 mm high at a packing fraction ~0.6) in
    a periodic 400 x 200 x 100 mm box with a wall at z = 0; mean flow 0.3 m/s plus
    Gaussian-filtered noise of rms 0.03 m/s on a 256 x 128 x 64 mesh."""
    Lx, Ly, Lz = 400e-3, 200e-3, 100e-3
    tiles = (100, 50)
    x, d = settled_bed(n, tiles, (Lx / tiles[0], Ly / tiles[1]), uniform_d(0.4e-3, 0.6e-3), seed)
    prm = default_params(hi=(Lx, Ly, Lz), ncell=(256, 128, 64), wall_hi=(0, 0, 0),
                         bandwidth=(1.5e-3,) * 3)
    U, DU = turbulent_like(prm["ncell"], prm["lo"], prm["hi"], seed=seed + 5)
    nn = len(x)
    parts = dict(x=x, v=np.zeros((nn, 3)), w=np.zeros((nn, 3)), d=d, rho=np.full(nn, 2500.0))
    return prm, parts, dict(U=U, DUDt=DU)


def large_patch(prm, parts, fl, cells=(64, 64)):
    """A bounded sample of the large bed: the spheres and mesh cells of the corner
    patch [0, cells[0] h) x [0, cells[1] h) (h = 1.5625 mm, so the default patch is
    100 x 100 mm: 1/8 of the bed), periodic at the patch edges.  The bed repeats every
    4 mm, so the patch is the same bed; the fluid fields are the patch's cells of the
    full fields (they do not wrap smoothly at the patch edges, which changes no cost)."""
    nc = prm["ncell"]
    h = [(prm["hi"][a] - prm["lo"][a]) / nc[a] for a in range(3)]
    hi = (cells[0] * h[0], cells[1] * h[1], prm["hi"][2])
    x = parts["x"]
    keep = (x[:, 0] < hi[0]) & (x[:, 1] < hi[1])
    sub = {k: parts[k][keep] for k in ("x", "v", "w", "d", "rho")}
    pprm = dict(prm, hi=hi, ncell=(cells[0], cells[1], nc[2]))

    def cut(f):
        return f.reshape(nc[2], nc[1], nc[0], 3)[:, :cells[1], :cells[0]].reshape(-1, 3)

    return pprm, sub, dict(U=cut(fl["U"]), DUDt=cut(fl["DUDt"]))


def random_fields(ncell, nf, seed, scale=1.0):
    """Non-negative random cell fields [nf, C] (deposition-like sparsity)."""
    rng = _rng(seed)
    C = int(np.prod(ncell))
    f = rng.random((nf, C)) * scale
    f[rng.random((nf, C)) < 0.5] = 0.0
    return f


def bounce_case(rho_p, nu_f, dt, d=6e-3, height=0.5, drop=0.45, lubrication=1, added_mass=1):
    """Case 1 of Sec. 4.1 (Table 1): one sphere of diameter d and density rho_p
    released at rest at z = drop in quiescent fluid (rho_f = 1000, viscosity nu_f)
    in a 100 x 100 x height mm box, periodic in x and y, floor and lid walls, 10 x
    10 x (height / 10 mm) mesh; the paper's linear spring-dashpot contact
    (k_n = 800 N/m, e = 0.97, mu = 0.1).  The box is taller than the paper's 200 mm
    so the sphere nears its settling speed before the impact."""
    prm = default_params(
        contact_law=1, kn_linear=800.0, kt_ratio=2.0 / 7.0, restitution=0.97, friction=0.1,
        rho_f=1000.0, nu_f=nu_f, lo=(0.0, 0.0, 0.0), hi=(0.1, 0.1, height),
        periodic=(1, 1, 0), wall_lo=(0, 0, 1), wall_hi=(0, 0, 1), dt=dt, skin=1e-3,
        lubrication=lubrication, added_mass=added_mass, drag=1, pressure_grad=1,
        ncell=(10, 10, int(round(height / 0.01))), bandwidth=(0.0, 0.0, 0.0))
    parts = dict(x=np.array([[0.05, 0.05, drop]]), v=np.zeros((1, 3)), w=np.zeros((1, 3)),
                 d=np.array([d]), rho=np.array([rho_p]))
    return prm, parts

