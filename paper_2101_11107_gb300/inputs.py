"""Seeded synthetic inputs: voxelised vessels, wall fractions, inflow waveforms, initial fields.

This module holds geometry and random draws only -- none of the lattice Boltzmann arithmetic.
It feeds both the CUDA library and the CPU oracle, so that both see identical inputs.

The paper's own geometries (a CAD sidewall aneurysm, a segmented patient ICA aneurysm, Sec. 2.2)
are not available; the generators below stand in for them with the shapes and parameter ranges
the paper reports: a bent parent vessel with a spherical sac fused at the outer bend, Reynolds
numbers of a few hundred, relaxation times near 0.506 (Sec. 2.2.3), and a pulsatile inflow curve.

Conventions (shared with the C-ABI):
  * a mask has shape (nz, ny, nx), x fastest in memory; 0 solid, 1 fluid, 2 inlet, 3 outlet;
  * cell (x, y, z) has its centre at (x + 1/2, y + 1/2, z + 1/2);
  * directions are numbered i = (cx+1) + 3 (cy+1) + 9 (cz+1);
  * a wall link is (box index of fluid cell, beta, q): the neighbour x + c_beta is not fluid
    and the wall surface cuts the segment from x to x + c_beta at fraction q in (0, 1]
    (the paper's q = |x_f - x_s| / |c|, Sec. 2.1.4).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

C27 = np.array([[(i % 3) - 1, ((i // 3) % 3) - 1, (i // 9) - 1] for i in range(27)], dtype=np.int64)


@dataclasses.dataclass
class Geometry:
    """A voxelised case: mask, wall links, inlet description and physical parameters."""

    mask: np.ndarray                       # uint8 (nz, ny, nx)
    periodic: tuple = (0, 0, 0)
    links: tuple | None = None             # (cell int64, beta uint8, q float64)
    inlet_center: tuple = (0.0, 0.0, 0.0)
    inlet_radius: float = 1.0
    tau: float = 0.6
    g0: tuple = (0.0, 0.0, 0.0)
    gamp: tuple = (0.0, 0.0, 0.0)
    gomega: float = 0.0
    wave: tuple | None = None              # (a[0..n], b[1..n], period_steps, u_peak)
    tau_cell: np.ndarray | None = None     # optional relaxation time per cell (nz, ny, nx)
    info: dict = dataclasses.field(default_factory=dict)

    @property
    def shape(self):
        return self.mask.shape

    @property
    def nfluid(self) -> int:
        return int(np.count_nonzero(self.mask))

    def n_links(self) -> int:
        return 0 if self.links is None else int(len(self.links[0]))


# --------------------------------------------------------------------------------- pipes
def pipe(nx: int, ny: int, nz: int, radius: float, center=None, tau=0.6, g0=(0, 0, 0),
         gamp=(0, 0, 0), gomega=0.0, bouzidi=False) -> Geometry:
    """Straight circular pipe along z, periodic in z; fluid iff the cell centre is inside."""
    if center is None:
        center = (nx / 2.0, ny / 2.0)
    cx, cy = center
    x = np.arange(nx) + 0.5
    y = np.arange(ny) + 0.5
    r2 = (x[None, :] - cx) ** 2 + (y[:, None] - cy) ** 2
    inside = r2 < radius * radius
    mask = np.broadcast_to(inside[None, :, :], (nz, ny, nx)).astype(np.uint8).copy()
    links = None
    if bouzidi:
        def sdf(p):
            return np.sqrt((p[..., 0] - cx) ** 2 + (p[..., 1] - cy) ** 2) - radius
        links = wall_links(mask, sdf, periodic=(0, 0, 1))
    return Geometry(mask=mask, periodic=(0, 0, 1), links=links, tau=tau, g0=tuple(g0),
                    gamp=tuple(gamp), gomega=gomega,
                    info=dict(kind="pipe", radius=radius, center=(cx, cy)))


def poiseuille_pipe_32() -> Geometry:
    """Body-force pipe flow: radius 12 in a 32x32x64 box periodic along z, tau 0.6,
    g = 1e-6 along z, halfway bounce-back walls."""
    return pipe(32, 32, 64, 12.0, center=(16.0, 16.0), tau=0.6, g0=(0.0, 0.0, 1e-6))


def womersley_pipe(nz=256, radius=28.0, box=64, womersley=4.0, tau=0.55, amp=1e-5) -> Geometry:
    """Pulsatile pipe flow driven by g_z(n) = amp cos(omega n), omega = Wo^2 nu / R^2."""
    nu = (tau - 0.5) / 3.0
    omega = womersley ** 2 * nu / radius ** 2
    g = pipe(box, box, nz, radius, center=(box / 2.0, box / 2.0), tau=tau, gamp=(0.0, 0.0, amp),
             gomega=omega)
    g.info.update(kind="womersley", womersley=womersley, nu=nu, omega=omega,
                  period_steps=2 * math.pi / omega)
    return g


def plane_channel(ny: int, y_lo: float, y_hi: float, nx: int = 4, nz: int = 4, tau=0.8,
                  g=1e-6, bouzidi=True) -> Geometry:
    """Force-driven flow between flat plates y = y_lo and y = y_hi (box coordinates), periodic
    in x and z.  With bouzidi the wall links carry the exact q of the planes."""
    y = np.arange(ny) + 0.5
    fluid = (y > y_lo) & (y < y_hi)
    mask = np.broadcast_to(fluid[None, :, None], (nz, ny, nx)).astype(np.uint8).copy()
    links = None
    if bouzidi:
        def sdf(p):
            return np.maximum(y_lo - p[..., 1], p[..., 1] - y_hi)
        links = wall_links(mask, sdf, periodic=(1, 0, 1))
    return Geometry(mask=mask, periodic=(1, 0, 1), links=links, tau=tau, g0=(g, 0.0, 0.0),
                    info=dict(kind="channel", y_lo=y_lo, y_hi=y_hi))


def inlet_pipe(nx: int, ny: int, nz: int, radius: float, u_peak=0.02, tau=0.8,
               bouzidi=False) -> Geometry:
    """Circular pipe along x (centre (ny/2, nz/2)) with a velocity inlet on face x = 0 and a
    density outlet on face x = nx - 1; the inlet profile is 2 U (1 - r^2/R^2), U = u_peak."""
    cy, cz = ny / 2.0, nz / 2.0
    y = np.arange(ny) + 0.5
    z = np.arange(nz) + 0.5
    r2 = (y[None, :] - cy) ** 2 + (z[:, None] - cz) ** 2
    inside = r2 < radius * radius
    mask = np.broadcast_to(inside[:, :, None], (nz, ny, nx)).astype(np.uint8).copy()
    mask[:, :, 0][mask[:, :, 0] == 1] = 2
    mask[:, :, nx - 1][mask[:, :, nx - 1] == 1] = 3
    links = None
    if bouzidi:
        def sdf(p):
            return np.sqrt((p[..., 1] - cy) ** 2 + (p[..., 2] - cz) ** 2) - radius
        links = wall_links(mask, sdf)
    return Geometry(mask=mask, periodic=(0, 0, 0), links=links, inlet_center=(0.0, cy, cz),
                    inlet_radius=radius, tau=tau, wave=(np.array([1.0]), np.zeros(0), 1.0, u_peak),
                    info=dict(kind="inlet_pipe", radius=radius))


# --------------------------------------------------------------------------------- walls
def wall_links(mask: np.ndarray, sdf, periodic=(0, 0, 0), iters: int = 60):
    """Wall links of every plain fluid cell (mask == 1) whose neighbour x + c_beta is not
    fluid; q found by bisection of the signed distance sdf (negative inside the fluid) along
    the link.  Returns (cell, beta, q) sorted by cell then beta."""
    nz, ny, nx = mask.shape
    fluid = mask != 0
    cells_all = []
    beta_all = []
    q_all = []
    zz, yy, xx = np.nonzero(mask == 1)
    base = np.stack([xx, yy, zz], axis=1)
    dims = np.array([nx, ny, nz])
    for beta in range(27):
        if beta == 13:
            continue
        c = C27[beta]
        p = base + c
        inside = np.ones(len(p), bool)
        for d in range(3):
            if periodic[d]:
                p[:, d] %= dims[d]
            else:
                inside &= (p[:, d] >= 0) & (p[:, d] < dims[d])
        nb_fluid = np.zeros(len(p), bool)
        pi = p[inside]
        nb_fluid[inside] = fluid[pi[:, 2], pi[:, 1], pi[:, 0]]
        sel = ~nb_fluid
        if not np.any(sel):
            continue
        x0 = base[sel].astype(np.float64) + 0.5
        cf = c.astype(np.float64)
        lo = np.zeros(len(x0))
        hi = np.ones(len(x0))
        f_hi = sdf(x0 + cf)
        # neighbours that are solid only because they are outside a face get q = 1 if the
        # surface is not crossed on the link
        crossed = f_hi >= 0
        for _ in range(iters):
            mid = 0.5 * (lo + hi)
            v = sdf(x0 + mid[:, None] * cf)
            pos = v >= 0
            hi = np.where(pos, mid, hi)
            lo = np.where(pos, lo, mid)
        q = np.where(crossed, hi, 1.0)
        q = np.clip(q, 1e-6, 1.0)
        cell = base[sel, 0] + nx * (base[sel, 1] + ny * base[sel, 2])
        cells_all.append(cell.astype(np.int64))
        beta_all.append(np.full(len(cell), beta, np.uint8))
        q_all.append(q)
    if not cells_all:
        return (np.zeros(0, np.int64), np.zeros(0, np.uint8), np.zeros(0))
    cell = np.concatenate(cells_all)
    beta = np.concatenate(beta_all)
    q = np.concatenate(q_all)
    order = np.lexsort((beta, cell))
    return cell[order], beta[order], q[order]


# --------------------------------------------------------------------------------- waveform
def cardiac_waveform(seed: int, n_harm: int = 5, period: float = 4000.0, u_peak: float = 0.025):
    """Seeded Fourier inflow curve s(t) = a0 + sum_k a_k cos + b_k sin (2 pi k t / P) with
    coefficients decaying like 1/k^2; redrawn until min s >= 0.15 max s (no backflow).
    Returns (a[0..n], b[1..n], period, u_peak): U(t) = u_peak s(t) / max s."""
    rng = np.random.default_rng(1_000_003 + seed)
    t = np.arange(int(period))
    while True:
        a = np.empty(n_harm + 1)
        b = np.empty(n_harm)
        a[0] = 1.0
        k = np.arange(1, n_harm + 1)
        a[1:] = rng.normal(0.0, 0.35, n_harm) / k ** 2
        b[:] = rng.normal(0.0, 0.35, n_harm) / k ** 2
        ph = 2 * np.pi * np.outer(k, t) / period
        s = a[0] + (a[1:, None] * np.cos(ph) + b[:, None] * np.sin(ph)).sum(0)
        if s.min() >= 0.15 * s.max():
            return a, b, float(period), float(u_peak)


# --------------------------------------------------------------------------------- aneurysm
def _dist_segment(p, a, b):
    ab = b - a
    t = np.clip(((p - a) @ ab) / (ab @ ab), 0.0, 1.0)
    q = a + t[..., None] * ab
    return np.linalg.norm(p - q, axis=-1)


def aneurysm_params(seed: int, edge: int = 256):
    """Seeded parameters of the synthetic sidewall aneurysm scaled to a box of `edge`^3."""
    rng = np.random.default_rng(seed)
    s = edge / 256.0
    r_v = rng.uniform(10.0, 14.0) * s
    r_s = rng.uniform(20.0, 35.0) * s
    return dict(edge=edge, scale=s, r_vessel=r_v, r_sac=r_s, arc_center=(40.0 * s, 40.0 * s, 128.0 * s),
                arc_radius=80.0 * s)


def aneurysm_sdf(par):
    """Signed distance (negative inside) of the vessel: inlet segment along +y from face y = 0,
    a quarter-arc centreline (radius 80, centre (40, 40, 128), all x edge/256), an outlet
    segment along -x to face x = 0, and a sphere fused at the outer 45-degree bend."""
    C = np.array(par["arc_center"])
    R = par["arc_radius"]
    r_v = par["r_vessel"]
    r_s = par["r_sac"]
    e = par["edge"]
    a_in = np.array([C[0] + R, -0.1 * e, C[2]])
    b_in = np.array([C[0] + R, C[1], C[2]])
    a_out = np.array([C[0], C[1] + R, C[2]])
    b_out = np.array([-0.1 * e, C[1] + R, C[2]])
    dirn = np.array([math.sqrt(0.5), math.sqrt(0.5), 0.0])
    sac = C + (R + r_v + 0.4 * r_s) * dirn

    def sdf(p):
        p = np.asarray(p, dtype=np.float64)
        d1 = _dist_segment(p, a_in, b_in)
        d2 = _dist_segment(p, a_out, b_out)
        rel = p - C
        rho = np.hypot(rel[..., 0], rel[..., 1])
        ang = np.arctan2(rel[..., 1], rel[..., 0])
        on = (ang >= 0.0) & (ang <= 0.5 * math.pi)
        d_arc = np.where(on, np.hypot(rho - R, rel[..., 2]), np.inf)
        d_tube = np.minimum(np.minimum(d1, d2), d_arc) - r_v
        d_sac = np.linalg.norm(p - sac, axis=-1) - r_s
        return np.minimum(d_tube, d_sac)

    return sdf


def outlet_sponge(mask: np.ndarray, tau: float, length: float, tau_max: float) -> np.ndarray:
    """Relaxation-time field with an absorbing layer before the outlets: cells within `length`
    of a box face that holds outlet cells (cells lying on that face only; distance along the
    face normal, d = 0 on the face) get tau + (tau_max - tau) (1 - d/length)^2; tau elsewhere."""
    nz, ny, nx = mask.shape
    dims = (nx, ny, nz)
    zz, yy, xx = np.nonzero(mask == 3)
    pos = (xx, yy, zz)
    on = []
    for axis in range(3):
        for side in (0, 1):
            v = 0 if side == 0 else dims[axis] - 1
            on.append(pos[axis] == v)
    n_faces = np.sum(on, axis=0) if on else np.zeros(0)
    field = np.full(mask.shape, float(tau))
    for f, hit in enumerate(on):
        axis, side = divmod(f, 2)
        if not np.any(hit & (n_faces == 1)):
            continue
        idx = np.arange(dims[axis], dtype=np.float64)
        d = idx if side == 0 else dims[axis] - 1 - idx
        ramp = np.where(d < length, (1.0 - d / length) ** 2, 0.0)
        shape = [1, 1, 1]
        shape[2 - axis] = dims[axis]
        field = np.maximum(field, tau + (tau_max - tau) * ramp.reshape(shape))
    return field


def aneurysm(seed: int, edge: int = 256, reynolds: float = 300.0, u_peak: float = 0.025,
             period: float = 4000.0, bouzidi: bool = True, wave_seed: int | None = None,
             sponge: bool = True) -> Geometry:
    """Seeded synthetic aneurysm in an edge^3 box: velocity inlet on face y = 0, density
    outlet on face x = 0, Bouzidi wall links from the analytic surface, tau from
    Re = u_peak 2 r_v / nu (u_peak the peak mean inflow velocity).  With `sponge`, an absorbing
    layer of edge/8 cells before the outlet raises tau smoothly by 0.1 at the outlet face: the
    outlet segment is short, and without it outgoing vortices destabilise the density outlet
    at tau ~ 0.503-0.507 (Re >= 150)."""
    par = aneurysm_params(seed, edge)
    sdf = aneurysm_sdf(par)
    n = edge
    mask = np.zeros((n, n, n), np.uint8)
    x = np.arange(n) + 0.5
    X, Y = np.meshgrid(x, x, indexing="xy")      # (ny, nx)
    for z in range(n):
        pts = np.stack([X, Y, np.full_like(X, z + 0.5)], axis=-1)
        mask[z] = sdf(pts) < 0
    mask[:, 0, :][mask[:, 0, :] == 1] = 2         # inlet face y = 0
    mask[:, :, 0][mask[:, :, 0] == 1] = 3         # outlet face x = 0
    links = wall_links(mask, sdf) if bouzidi else None
    nu = u_peak * 2.0 * par["r_vessel"] / reynolds
    tau = 0.5 + 3.0 * nu
    wave = cardiac_waveform(seed if wave_seed is None else wave_seed, period=period, u_peak=u_peak)
    C = par["arc_center"]
    g = Geometry(mask=mask, periodic=(0, 0, 0), links=links,
                 inlet_center=(C[0] + par["arc_radius"], 0.0, C[2]), inlet_radius=par["r_vessel"],
                 tau=tau, wave=wave, info=dict(kind="aneurysm", seed=seed, **par, nu=nu,
                                               reynolds=reynolds))
    g.info["fluid_fraction"] = g.nfluid / float(n ** 3)
    if sponge:
        g.tau_cell = outlet_sponge(mask, tau, edge / 8.0, tau + 0.1)
        g.info["sponge"] = dict(length=edge / 8.0, tau_max=tau + 0.1)
    return g


# --------------------------------------------------------------------------------- fields
def taylor_green(nx: int, ny: int, nz: int, u0: float = 0.01):
    """Initial density and velocity of the 2-D Taylor-Green vortex (z-invariant), on cell
    centres: u = -u0 cos(kx x) sin(ky y), v = u0 sin(kx x) cos(ky y), rho = 1."""
    kx = 2 * math.pi / nx
    ky = 2 * math.pi / ny
    x = np.arange(nx) + 0.5
    y = np.arange(ny) + 0.5
    X, Y = np.meshgrid(x, y, indexing="xy")
    ux = -u0 * np.cos(kx * X) * np.sin(ky * Y)
    uy = u0 * np.sin(kx * X) * np.cos(ky * Y)
    rho = np.ones((nz, ny, nx))
    u = np.zeros((3, nz, ny, nx))
    u[0] = ux[None]
    u[1] = uy[None]
    return rho, u


# --------------------------------------------------------------------------------- corrector
def corrector_init_params(seed: int):
    """Seeded initial parameters of the 3-layer corrector network: weights (27, 16, 16) per
    layer, He-normal with fan-in 27 x 16 (the last layer scaled by 0.1), biases zero; rounded
    to FP32.  Returned as [W1, b1, W2, b2, W3, b3]."""
    rng = np.random.default_rng(7_000_001 + seed)
    std = np.sqrt(2.0 / (27 * 16))
    ws = [rng.normal(0.0, std, (27, 16, 16)), rng.normal(0.0, std, (27, 16, 16)),
          rng.normal(0.0, 0.1 * std, (27, 16, 16))]
    out = []
    for w in ws:
        out += [w.astype(np.float32).astype(np.float64), np.zeros(16)]
    return out
