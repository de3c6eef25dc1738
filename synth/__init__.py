"""Seeded synthetic models standing in for the paper's hydrodynamics snapshots.

This module only builds inputs: point clouds, neighbour lists (the mesh
pre-processing that the paper delegates to Gmsh / Delaunay / the octree), the
physical fields on the points, and the random sample that the ray set draws.
It contains none of the method's own arithmetic and is used by both the CUDA
path's tests/benchmark and the oracle, so neither depends on the other.

A model is a dict with keys
  pos [n,3] f64, vel [n,3] f64 (km/s), nbr_off [n+1] i64, nbr_idx [E] i32,
  nu0 [L] f64 (Hz), chi0 [n,L], eta0 [n,L], dvw [n] (km/s), chi_c [n], eta_c [n],
  n_freq, x_span, l_min, l_max, sample [n_sample] i32, rho [n], T [n], name.
"""
from __future__ import annotations

import numpy as np

K_B = 1.380649e-23  # J/K
AMU = 1.66053906660e-27  # kg
NU_CO10 = 115.2712018e9  # Hz, CO J=1-0 (any line works: only ratios enter)


def doppler_width(T, mass_amu=28.0):
    """Thermal Doppler width sqrt(2kT/m) in km/s."""
    return np.sqrt(2.0 * K_B * np.asarray(T, np.float64) / (mass_amu * AMU)) / 1e3


def sample_indices(n: int, n_sample: int = 10000, seed: int = 0) -> np.ndarray:
    """Uniform sample of point indices without replacement (all points if n <= n_sample)."""
    if n <= n_sample:
        return np.arange(n, dtype=np.int32)
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0x5A]))
    return np.sort(rng.choice(n, size=n_sample, replace=False)).astype(np.int32)


def csr_from_pairs(n: int, a: np.ndarray, b: np.ndarray):
    """Symmetric CSR (rows sorted ascending, no duplicates, no self loops)."""
    a = np.asarray(a, np.int64)
    b = np.asarray(b, np.int64)
    src = np.concatenate([a, b])
    dst = np.concatenate([b, a])
    keep = src != dst
    src, dst = src[keep], dst[keep]
    key = np.unique(src * n + dst)
    src, dst = key // n, key % n
    off = np.zeros(n + 1, np.int64)
    np.add.at(off, src + 1, 1)
    off = np.cumsum(off)
    return off, dst.astype(np.int32)


def delaunay_csr(pos: np.ndarray):
    """Neighbour CSR from the edges of the 3-D Delaunay tetrahedralisation."""
    from scipy.spatial import Delaunay

    tri = Delaunay(pos)
    s = tri.simplices.astype(np.int64)
    pairs = [(s[:, i], s[:, j]) for i in range(4) for j in range(i + 1, 4)]
    a = np.concatenate([p[0] for p in pairs])
    b = np.concatenate([p[1] for p in pairs])
    return csr_from_pairs(len(pos), a, b)


def grid_csr(m: int):
    """26-neighbour CSR of an m^3 Cartesian grid, point id = (i*m + j)*m + k."""
    idx = np.arange(m ** 3).reshape(m, m, m)
    a_list, b_list = [], []
    for di in (-1, 0, 1):
        for dj in (-1, 0, 1):
            for dk in (-1, 0, 1):
                if di == dj == dk == 0:
                    continue
                src = idx[max(0, -di):m - max(0, di), max(0, -dj):m - max(0, dj),
                          max(0, -dk):m - max(0, dk)].ravel()
                a_list.append(src)
                b_list.append(src + (di * m + dj) * m + dk)
    return csr_from_pairs(m ** 3, np.concatenate(a_list), np.concatenate(b_list))


def grid_model(m: int = 16, chi_line: float = 5.0, n_freq: int = 31, x_span: float = 4.0,
               level: int = 0, floor: float = 1e-10):
    """Homogeneous static cube: m^3 grid points x = i/(m-1), 26 neighbours, one line of
    width 1 km/s, line-centre optical depth chi_line across the unit cube, S = 1
    everywhere (the continuum floor has S = 1 too), no velocity."""
    g = np.arange(m, dtype=np.float64) / (m - 1)
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    pos = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    n = len(pos)
    off, nbr = grid_csr(m)
    chi0 = np.full((n, 1), chi_line)
    return dict(
        name=f"grid{m}", pos=pos, vel=np.zeros((n, 3)), nbr_off=off, nbr_idx=nbr,
        nu0=np.array([NU_CO10]), chi0=chi0, eta0=chi0.copy(), dvw=np.ones(n),
        chi_c=np.full(n, floor * chi_line), eta_c=np.full(n, floor * chi_line),
        n_freq=n_freq, x_span=x_span, l_min=level, l_max=level,
        sample=sample_indices(n), rho=np.ones(n), T=np.full(n, 2000.0))


def wind_model(n: int = 50000, seed: int = 2, n_freq: int = 50, x_span: float = 4.0,
               level: int = 2, l_min: int | None = None, tau_radial: float = 10.0,
               v_inf: float = 15.0, cont_frac: float = 1e-4, n_sample: int = 10000):
    """Spherical stellar wind, r in [1, 100] stellar radii log-uniform (so the point
    density falls as r^-3 and the element size grows as r), isotropic directions.
    Density ~ r^-2, beta-law radial velocity v = v_inf (1 - 1/r)^0.5, temperature
    T = 2000 K r^-0.7, CO-like thermal width, line-centre opacity ~ density scaled
    to a radial line-centre optical depth tau_radial (static), line source function
    S = T / 2000 K, weak continuum with the same source function."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0x57]))
    r = np.exp(rng.uniform(0.0, np.log(100.0), n))
    mu = rng.uniform(-1.0, 1.0, n)
    ph = rng.uniform(0.0, 2.0 * np.pi, n)
    st = np.sqrt(1.0 - mu * mu)
    rhat = np.stack([st * np.cos(ph), st * np.sin(ph), mu], axis=1)
    pos = rhat * r[:, None]
    off, nbr = delaunay_csr(pos)
    vel = rhat * (v_inf * np.sqrt(1.0 - 1.0 / r))[:, None]
    T = 2000.0 * r ** -0.7
    rho = r ** -2.0
    k = tau_radial / (1.0 - 1.0 / 100.0)
    chi0 = (k * rho)[:, None]
    S = T / 2000.0
    eta0 = chi0 * S[:, None]
    chi_c = cont_frac * chi0[:, 0]
    return dict(
        name=f"wind{n}", pos=pos, vel=vel, nbr_off=off, nbr_idx=nbr,
        nu0=np.array([NU_CO10]), chi0=chi0, eta0=eta0, dvw=doppler_width(T),
        chi_c=chi_c, eta_c=chi_c * S, n_freq=n_freq, x_span=x_span,
        l_min=level if l_min is None else l_min, l_max=level,
        sample=sample_indices(n, n_sample, seed), rho=rho, T=T)


def random_cloud(n: int = 40, seed: int = 0, n_lines: int = 1, n_freq: int = 7,
                 x_span: float = 3.0, l_min: int = 0, l_max: int = 0, v_rms: float = 2.0):
    """Small random point cloud in the unit cube with Delaunay neighbours and random
    smooth-ish fields; for brute-force checks."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0xC1]))
    pos = rng.uniform(0.0, 1.0, (n, 3))
    off, nbr = delaunay_csr(pos)
    vel = rng.normal(0.0, v_rms, (n, 3))
    T = rng.uniform(500.0, 3000.0, n)
    nu0 = NU_CO10 * (1.0 + np.arange(n_lines) * 3e-4)
    chi0 = rng.uniform(0.5, 8.0, (n, n_lines))
    S = rng.uniform(0.2, 1.5, (n, n_lines))
    chi_c = rng.uniform(0.01, 0.1, n)
    return dict(
        name=f"cloud{n}", pos=pos, vel=vel, nbr_off=off, nbr_idx=nbr, nu0=nu0, chi0=chi0,
        eta0=chi0 * S, dvw=doppler_width(T), chi_c=chi_c, eta_c=chi_c * S[:, 0],
        n_freq=n_freq, x_span=x_span, l_min=l_min, l_max=l_max,
        sample=sample_indices(n), rho=rng.uniform(0.1, 1.0, n), T=T)


def spiral_density(x: np.ndarray, r_in: float = 10.0, arm_spacing: float = 50.0, contrast: float = 10.0) -> np.ndarray:
    """Analytic tracer of the binary-wind spiral (the density of spiral_model):
    (max(r, r_in)/r_in)^-2 (1 + (contrast - 1) g), g the Gaussian arm profile
    about r = r_in + arm_spacing phi / 2 pi (half-width 8 AU, scale height 30 AU)."""
    x = np.asarray(x, np.float64)
    r = np.sqrt((x ** 2).sum(-1))
    rc = np.sqrt(x[..., 0] ** 2 + x[..., 1] ** 2)
    ph = np.arctan2(x[..., 1], x[..., 0]) % (2 * np.pi)
    r0 = r_in + arm_spacing * ph / (2 * np.pi)
    d = np.abs(((rc - r0 + 0.5 * arm_spacing) % arm_spacing) - 0.5 * arm_spacing)
    g = np.exp(-(d / 8.0) ** 2) * np.exp(-(x[..., 2] / 30.0) ** 2)
    return (np.maximum(r, r_in) / r_in) ** -2.0 * (1 + (contrast - 1) * g)


def spiral_model(n: int = 1_000_000, seed: int = 4, n_freq: int = 100, x_span: float = 4.0, level: int = 2,
                 l_min: int | None = None, box: float = 1200.0, arm_spacing: float = 50.0,
                 contrast: float = 10.0, tau_radial: float = 10.0, cont_frac: float = 1e-4):
    """Binary-wind Archimedean spiral as an SPH-like particle cloud: density
    rho ~ r^-2 (1 + (contrast - 1) g), g a Gaussian arm profile around the
    spiral r = r0 + arm_spacing phi / 2 pi in the orbital plane (arm half-width
    8 AU, scale height 30 AU), in a box of `box` AU; equal-mass particles
    (positions drawn with probability ~ rho), Delaunay neighbours, a 15 km/s
    radial wind plus a smooth random field of 64 Fourier modes (1 km/s rms per
    component), T = 2000 K (r / 10 AU)^-0.7."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0x5B]))
    r_in, r_out = 10.0, box / 2.0

    def arm(x):
        r = np.sqrt(x[:, 0] ** 2 + x[:, 1] ** 2)
        ph = np.arctan2(x[:, 1], x[:, 0]) % (2 * np.pi)
        r0 = r_in + arm_spacing * ph / (2 * np.pi)
        d = np.abs(((r - r0 + 0.5 * arm_spacing) % arm_spacing) - 0.5 * arm_spacing)
        return np.exp(-(d / 8.0) ** 2) * np.exp(-(x[:, 2] / 30.0) ** 2)

    pts = []
    need = n
    while need > 0:
        m = int(need * 2.5) + 1000
        r = rng.uniform(r_in, r_out, m)  # mass ~ rho r^2 dr is uniform in r for rho ~ r^-2
        mu = rng.uniform(-1.0, 1.0, m)
        ph = rng.uniform(0.0, 2 * np.pi, m)
        st = np.sqrt(1 - mu * mu)
        x = np.stack([st * np.cos(ph), st * np.sin(ph), mu], 1) * r[:, None]
        acc = rng.uniform(0.0, 1.0, m) < (1 + (contrast - 1) * arm(x)) / contrast
        pts.append(x[acc][:need])
        need -= len(pts[-1])
    pos = np.concatenate(pts)[:n]
    off, nbr = delaunay_csr(pos)
    r = np.sqrt((pos ** 2).sum(1))
    rhat = pos / r[:, None]
    vel = 15.0 * rhat + _fourier_velocity(pos, rng, 64, 1.0, box)
    rho = (r / r_in) ** -2.0 * (1 + (contrast - 1) * arm(pos))
    T = 2000.0 * (r / r_in) ** -0.7
    k = tau_radial / (r_in * (1 - r_in / r_out))  # radial line-centre depth of the smooth r^-2 part
    chi0 = (k * rho)[:, None]
    S = T / 2000.0
    chi_c = cont_frac * chi0[:, 0]
    return dict(
        name=f"spiral{n}", pos=pos, vel=vel, nbr_off=off, nbr_idx=nbr, nu0=np.array([NU_CO10]), chi0=chi0,
        eta0=chi0 * S[:, None], dvw=doppler_width(T), chi_c=chi_c, eta_c=chi_c * S, n_freq=n_freq, x_span=x_span,
        l_min=level if l_min is None else l_min, l_max=level, sample=sample_indices(n, 10000, seed), rho=rho, T=T)


def _clump_params(rng, n_clumps: int, box: float):
    centres = rng.uniform(-0.3 * box, 0.3 * box, (n_clumps, 3))
    sigmas = rng.uniform(30.0, 80.0, n_clumps)
    return centres, sigmas


def _clump_density(x, centres, sigmas, contrast):
    rho = np.ones(len(x))
    for c, s in zip(centres, sigmas):
        rho += (contrast - 1.0) * np.exp(-((x - c) ** 2).sum(1) / (2 * s * s))
    return rho


def _refine(box, lo_level, hi_level, centres, sigmas, contrast, thr, q):
    """Leaves (level, i, j, k) of an octree over [-box/2, box/2]^3: every cell
    down to lo_level, then a cell of level l is split while the largest density
    inside it (the clump profiles evaluated at each clump's nearest point of the
    cell) exceeds thr * q^(l - lo_level)."""
    n0 = 2 ** lo_level
    ijk = np.stack(np.meshgrid(*([np.arange(n0)] * 3), indexing="ij"), -1).reshape(-1, 3)
    leaves = []
    for l in range(lo_level, hi_level + 1):
        h = box / 2 ** l
        lo = -box / 2 + ijk * h
        rho_max = np.ones(len(ijk))
        for c, s in zip(centres, sigmas):
            near = np.clip(c, lo, lo + h)
            rho_max += (contrast - 1.0) * np.exp(-((near - c) ** 2).sum(1) / (2 * s * s))
        split = rho_max > thr * q ** (l - lo_level) if l < hi_level else np.zeros(len(ijk), bool)
        leaves.append(np.concatenate([np.full((int((~split).sum()), 1), l), ijk[~split]], 1))
        kids = ijk[split]
        d = np.stack(np.meshgrid([0, 1], [0, 1], [0, 1], indexing="ij"), -1).reshape(-1, 3)
        ijk = (2 * kids[:, None, :] + d[None]).reshape(-1, 3)
    return np.concatenate(leaves)


def octree_leaf_csr(leaves: np.ndarray, hi_level: int):
    """Neighbour CSR of octree leaves: two leaves are neighbours when their closed
    cubes touch (share a face, an edge or a corner). Every leaf is rasterised
    on the finest grid; two leaves touch iff two of their fine voxels are
    26-adjacent."""
    g = 2 ** hi_level
    grid = np.empty((g, g, g), np.int32)
    for l in np.unique(leaves[:, 0]):
        sel = np.where(leaves[:, 0] == l)[0]
        s = 2 ** (hi_level - l)
        v = grid.reshape(g // s, s, g // s, s, g // s, s)
        i, j, k = leaves[sel, 1], leaves[sel, 2], leaves[sel, 3]
        v[i, :, j, :, k, :] = sel.astype(np.int32)[:, None, None, None]
    a_all, b_all = [], []
    offs = [(dx, dy, dz) for dx in (-1, 0, 1) for dy in (-1, 0, 1) for dz in (-1, 0, 1) if (dx, dy, dz) > (0, 0, 0)]
    for dx, dy, dz in offs:
        sa = tuple(slice(max(0, -d), g - max(0, d)) for d in (dx, dy, dz))
        sb = tuple(slice(max(0, d), g - max(0, -d)) for d in (dx, dy, dz))
        A, B = grid[sa].ravel(), grid[sb].ravel()
        diff = A != B
        key = np.unique(np.minimum(A[diff], B[diff]).astype(np.int64) * len(leaves) + np.maximum(A[diff], B[diff]))
        a_all.append(key // len(leaves))
        b_all.append(key % len(leaves))
    return csr_from_pairs(len(leaves), np.concatenate(a_all), np.concatenate(b_all))


def _fourier_velocity(pos, rng, n_modes: int, rms: float, box: float):
    """Smooth random velocity field: a sum of n_modes seeded Fourier modes with
    wavelengths between box/8 and box, each component scaled to the given rms
    over the points."""
    kdir = rng.normal(size=(n_modes, 3))
    kdir /= np.linalg.norm(kdir, axis=1, keepdims=True)
    lam = box * np.exp(rng.uniform(np.log(1 / 8), 0.0, n_modes))
    kvec = kdir * (2 * np.pi / lam)[:, None]
    amp = rng.normal(size=(n_modes, 3)) * (lam / box)[:, None]
    phase = rng.uniform(0.0, 2 * np.pi, n_modes)
    v = np.cos(pos @ kvec.T + phase) @ amp
    v -= v.mean(0)
    return v * (rms / v.std(0))


def multi_line(nu0: float, n_lines: int, spacing: float = 1e-3):
    """Line centres spaced by `spacing` in relative frequency (300 km/s for 1e-3),
    several hundred thermal widths apart."""
    return nu0 * (1.0 + spacing * np.arange(n_lines))


def octree_model(n_leaves: int = 300_000, seed: int = 3, n_lines: int = 2, n_freq: int = 64, x_span: float = 4.0,
                 l_min: int = 0, l_max: int = 3, box: float = 1000.0, lo_level: int = 3, hi_level: int = 8,
                 contrast: float = 1e3, v_rms: float = 2.0, n_modes: int = 64, tau_box: float = 1.0,
                 line_ratio: float = 0.1, cont_frac: float = 1e-4, velocity: str = "fourier"):
    """Octree AMR-like mesh of leaf-cell centres: a box of `box` AU refined from
    lo_level to hi_level around three seeded Gaussian clumps (sigma 30-80 AU,
    peak/background density contrast `contrast`), with the split threshold tuned
    by bisection so that the leaf count is close to n_leaves. Neighbours are the
    leaves whose closed cubes touch. Velocity: a smooth field of n_modes Fourier
    modes (or i.i.d. Gaussian per leaf with velocity='iid'), v_rms per component.
    n_lines lines with line-centre opacity ratio 1 : line_ratio : line_ratio^2 ...,
    opacity ~ density with a line-centre optical depth tau_box across the box
    at background density, T = 1000 K rho^-0.2, S = T / 1000 K."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0x0C]))
    centres, sigmas = _clump_params(rng, 3, box)
    lo, hi = 1.0, contrast
    best = None
    for _ in range(40):  # bisection on log threshold; leaf count decreases with it
        thr = np.sqrt(lo * hi)
        leaves = _refine(box, lo_level, hi_level, centres, sigmas, contrast, thr, 2.0)
        if best is None or abs(len(leaves) - n_leaves) < abs(len(best) - n_leaves):
            best = leaves
        if len(leaves) > n_leaves:
            lo = thr
        else:
            hi = thr
        if hi / lo < 1.0 + 1e-4 or abs(len(leaves) - n_leaves) <= 0.01 * n_leaves:
            break
    leaves = best
    n = len(leaves)
    h = box / 2.0 ** leaves[:, 0]
    pos = -box / 2 + (leaves[:, 1:] + 0.5) * h[:, None]
    off, nbr = octree_leaf_csr(leaves, hi_level)
    if velocity == "iid":
        vel = rng.normal(0.0, v_rms, (n, 3))
    else:
        vel = _fourier_velocity(pos, rng, n_modes, v_rms, box)
    rho = _clump_density(pos, centres, sigmas, contrast)
    T = 1000.0 * rho ** -0.2
    S = T / 1000.0
    chi0 = (tau_box / box) * rho[:, None] * line_ratio ** np.arange(n_lines)[None, :]
    chi_c = cont_frac * chi0[:, 0]
    return dict(
        name=f"octree{n}", pos=pos, vel=vel, nbr_off=off, nbr_idx=nbr, nu0=multi_line(NU_CO10, n_lines), chi0=chi0,
        eta0=chi0 * S[:, None], dvw=doppler_width(T), chi_c=chi_c, eta_c=chi_c * S, n_freq=n_freq, x_span=x_span,
        l_min=l_min, l_max=l_max, sample=sample_indices(n, 10000, seed), rho=rho, T=T, level=leaves[:, 0])


def with_lines(m: dict, n_lines: int, n_freq: int, line_ratio: float = 0.5) -> dict:
    """The model with its first line's opacity and source function repeated over
    n_lines separated lines (opacity ratio 1 : line_ratio : ...)."""
    out = dict(m)
    S = m["eta0"][:, :1] / m["chi0"][:, :1]
    chi0 = m["chi0"][:, :1] * line_ratio ** np.arange(n_lines)[None, :]
    out.update(nu0=multi_line(m["nu0"][0], n_lines), chi0=chi0, eta0=chi0 * S, n_freq=n_freq)
    return out


def batch_models(n_models: int = 64, seed: int = 5, n_min: int = 10_000, n_max: int = 200_000, n_lines: int = 4,
                 n_freq: int = 100, l_min: int = 0, l_max: int = 3, only=None):
    """Independent models with seeded sizes log-uniform in [n_min, n_max], the
    generators taken in turn (Cartesian grid, stellar wind, clump octree), each
    with n_lines separated lines of n_freq bins and adaptive rays l_min..l_max.
    `only` (indices) builds just those members of the same draw."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0xBA]))
    sizes = np.exp(rng.uniform(np.log(n_min), np.log(n_max), n_models)).astype(np.int64)
    out = []
    for k, n in enumerate(sizes):
        if only is not None and k not in only:
            continue
        s = seed * 1000 + k
        kind = k % 3
        if kind == 0:
            m = grid_model(max(3, int(round(n ** (1 / 3)))), n_freq=n_freq)
            m = with_lines(m, n_lines, n_freq)
        elif kind == 1:
            m = with_lines(wind_model(int(n), seed=s, n_freq=n_freq), n_lines, n_freq)
        else:
            m = octree_model(int(n), seed=s, n_lines=n_lines, n_freq=n_freq, hi_level=max(5, min(8, int(np.log2(n) / 3) + 3)))
        m.update(l_min=l_min, l_max=l_max, name=f"{m['name']}_b{k}")
        out.append(m)
    return out
