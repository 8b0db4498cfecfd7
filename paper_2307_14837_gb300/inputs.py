"""Seeded synthetic inputs for the DNN-MG patch-correction path.

This module produces *inputs only*: coarse hexahedral meshes with boundary
markers, coarse velocity/pressure fields, fine-level right-hand sides and
network weights.  It contains none of the method's arithmetic (no refinement,
prolongation, residual, gather, network evaluation or scatter), so both the
CPU oracle tests and the CUDA path can draw from it without sharing any of the
computation they are compared on.

Random numbers come from one counter-based generator, SplitMix64 (Steele,
Lea & Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014):
value i of stream s is mix64(s + (i + 1) * 0x9E3779B97F4A7C15), mapped to
[0, 1) with its top 53 bits.

Mesh conventions (shared by every consumer):
  * vertices ``xyz`` float64 [n_vertices, 3];
  * cells ``cells`` int32 [n_cells, 8]; local vertex k sits at reference
    corner (k & 1, (k >> 1) & 1, (k >> 2) & 1) of the trilinear map;
  * ``vertex_bc`` int32 [n_vertices]: 0 interior, 1 no-slip wall,
    2 driven Dirichlet (lid or inflow), 3 do-nothing outflow.  Where two
    kinds meet at a vertex, 2 wins over 1 and 1 over 3.
  * ``patch_groups``: True when the cells come in consecutive groups of 8
    that are the lexicographic children (i + 2 j + 4 k) of a parent hex;
    this is the patch structure the two-level local projection needs on the
    coarse level.

Workloads (Sec. 6.2 of the paper describes the benchmark channel; the paper's
own meshes, data and weights are not available, so these seeded families stand
in for them):
  * ``cavity_mesh``: unit cube, lid z = 1 moving with u = (1, 0, 0);
  * ``channel_mesh``: channel [0, 2.5] x [0, 0.41] x [0, 0.41] with a
    cylinder along z whose diameter and centre are drawn from the seed,
    parabolic inflow at x = 0, do-nothing outflow at x = 2.5.
"""
from __future__ import annotations

import math

import numpy as np

CHANNEL_LENGTH = 2.5
CHANNEL_HEIGHT = 0.41

# Sec. 6.4, table of training-data statistics: mean and standard
# deviation of v_x, v_y, v_z and p.  Used only to shape synthetic fields.
PAPER_FIELD_MEAN = (0.978, 0.0005974, 0.0, 0.2389)
PAPER_FIELD_STD = (0.7074, 0.2583, 0.1705, 0.5443)

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix64(z: np.ndarray) -> np.ndarray:
    z = z.copy()
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def splitmix_uniform(stream: int, n: int) -> np.ndarray:
    """n uniform doubles in [0, 1) from SplitMix64 stream ``stream``."""
    i = np.arange(1, n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(stream & 0xFFFFFFFFFFFFFFFF) + i * _GOLDEN
    return (_mix64(z) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def splitmix_normal(stream: int, n: int) -> np.ndarray:
    """n standard normal doubles (Box-Muller on two SplitMix64 draws)."""
    u = splitmix_uniform(stream, 2 * n)
    u1 = 1.0 - u[0::2]          # (0, 1]
    u2 = u[1::2]
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def _stream(seed: int, tag: int) -> int:
    """Derive an independent stream id from (seed, tag)."""
    z = np.array([(seed * 0x10001 + tag) & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64)
    return int(_mix64(z)[0])


# --------------------------------------------------------------------------
# meshes
# --------------------------------------------------------------------------

class Mesh(dict):
    """dict with keys xyz, cells, vertex_bc, patch_groups, meta."""

    @property
    def n_vertices(self) -> int:
        return int(self["xyz"].shape[0])

    @property
    def n_cells(self) -> int:
        return int(self["cells"].shape[0])


def first_level(idx: np.ndarray, n_fine: int, levels: int) -> np.ndarray:
    """Level (0 = coarsest of levels + 1) at which grid line idx of a grid of
    n_fine intervals refined `levels` times from n_fine / 2^levels appears."""
    lev = np.full(idx.shape, levels, dtype=np.int64)
    for s in range(levels - 1, -1, -1):
        step = 1 << (levels - s)
        lev = np.where(idx % step == 0, s, lev)
    return lev


def nested_order(i, j, k, flip, nbi, nbj, levels: int) -> np.ndarray:
    """Order of cells (i, j, k) (indices at the finest level, `levels`
    refinements of a base grid) such that every 8 consecutive cells are the
    children of one parent, child (a, b, c) at offset a + 2 b + 4 c in the
    parent's local frame, recursively: cells sorted by base cell, then by
    child index at each level from the coarsest down.  flip marks cells whose
    local xi axis runs against i.  nbi, nbj: base cells along i and j (the
    base index is ib + nbi (jb + nbj kb))."""
    i, j, k = (np.asarray(a, dtype=np.int64) for a in (i, j, k))
    flip = np.asarray(flip, dtype=bool)
    key = (i >> levels) + nbi * ((j >> levels) + nbj * (k >> levels))
    for s in range(levels - 1, -1, -1):
        a = (i >> s) & 1
        a = np.where(flip, 1 - a, a)
        key = key * 8 + a + 2 * ((j >> s) & 1) + 4 * ((k >> s) & 1)
    return np.argsort(key, kind="stable")


def cavity_mesh(n: int, jitter: float = 0.0, seed: int = 0, grouped: bool = True,
                levels: int | None = None) -> Mesh:
    """Unit cube split into n^3 hexahedra (n even when ``grouped``).

    With ``grouped`` the cells are ordered parent by parent: the 8 children of
    parent (I, J, K) of the n/2 grid are consecutive, child (i, j, k) at
    offset i + 2 j + 4 k.  ``levels`` = k >= 1 nests this k times (n a
    multiple of 2^k): see ``nested_order``; the mesh is then the k-th uniform
    refinement of the (n / 2^k)^3 grid with its vertices numbered coarsest
    level first.  ``jitter`` moves interior vertices by up to jitter * h in
    each coordinate (seeded), which makes the cells non-affine.
    """
    if levels is not None and levels >= 1:
        if n % (1 << levels):
            raise ValueError("nested cavity mesh needs n divisible by 2^levels")
        grouped = True
    if grouped and n % 2:
        raise ValueError("grouped cavity mesh needs an even n")
    m = n + 1
    g = np.arange(m, dtype=np.float64) / n
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    # vertex id = i + m j + m^2 k
    xyz = np.stack([X.transpose(2, 1, 0).ravel(), Y.transpose(2, 1, 0).ravel(),
                    Z.transpose(2, 1, 0).ravel()], axis=1)
    ii, jj, kk = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    ii, jj, kk = (a.transpose(2, 1, 0).ravel() for a in (ii, jj, kk))
    corners = []
    for c in range(8):
        di, dj, dk = c & 1, (c >> 1) & 1, (c >> 2) & 1
        corners.append((ii + di) + m * (jj + dj) + m * m * (kk + dk))
    cells = np.stack(corners, axis=1).astype(np.int32)
    k_lev = levels if (levels is not None and levels >= 1) else (1 if grouped else 0)
    if k_lev >= 1:
        order = nested_order(ii, jj, kk, np.zeros_like(ii, dtype=bool), n >> k_lev, n >> k_lev, k_lev)
        cells = cells[order]
    if levels is not None and levels >= 1:
        vi = np.arange(m)
        lev1 = first_level(vi, n, levels)
        vl = np.maximum(np.maximum(lev1[:, None, None], lev1[None, :, None]), lev1[None, None, :])
        vlev = vl.transpose(2, 1, 0).ravel()          # vertex id = i + m j + m^2 k
        perm = np.argsort(vlev, kind="stable")        # new id -> old id
        inv = np.empty_like(perm)
        inv[perm] = np.arange(perm.size)
        xyz = xyz[perm]
        cells = inv[cells].astype(np.int32)
    on_b = np.any((xyz == 0.0) | (xyz == 1.0), axis=1)
    bc = np.where(on_b, 1, 0).astype(np.int32)
    bc[xyz[:, 2] == 1.0] = 2
    if jitter > 0.0:
        u = splitmix_uniform(_stream(seed, 11), xyz.size).reshape(xyz.shape)
        d = (2.0 * u - 1.0) * jitter / n
        d[on_b] = 0.0
        xyz = xyz + d
    return Mesh(xyz=np.ascontiguousarray(xyz), cells=np.ascontiguousarray(cells),
                vertex_bc=bc, patch_groups=bool(grouped),
                meta=dict(kind="cavity", n=n, jitter=jitter, seed=seed,
                          mg_levels=int(levels) if (levels is not None and levels >= 1) else 0))


def channel_geometry(seed: int):
    """Cylinder diameter D ~ U[0.08, 0.12] and centre near (0.5, 0.2)."""
    u = splitmix_uniform(_stream(seed, 21), 3)
    D = 0.08 + 0.04 * u[0]
    cx = 0.5 + 0.1 * (u[1] - 0.5)
    cy = 0.2 + 0.04 * (u[2] - 0.5)
    return D, cx, cy


def channel_mesh(nz: int, seed: int = 0, box_half: float = 0.15, levels: int = 0) -> Mesh:
    """Hexahedral mesh of the channel with a cylindrical obstacle.

    The x-y cross-section is a 3 x 3 block layout: an O-grid of four blocks
    between the circle and a square of half-size ``box_half`` around the
    cylinder, and eight rectangular blocks filling the rest of the channel.
    The 2D mesh has cell size about H / nz and is extruded into nz layers in z.
    Cell counts: about 6.3 nz^3 (nz = 19 gives ~43k cells, nz = 37 ~318k).

    ``levels`` = k >= 1 builds the k-th uniform refinement of the mesh with
    nz / 2^k layers (nz a multiple of 2^k): every block keeps 2^k times the
    base block's cells per direction, points on the circle stay on it, the
    cells are ordered by ``nested_order`` (8 consecutive cells are the
    children of one parent, recursively) and vertices are numbered by the
    level on which they first appear, so the first vertices of the mesh are
    those of each coarser level.  Base points are reproduced bit for bit.
    """
    H, Lx = CHANNEL_HEIGHT, CHANNEL_LENGTH
    D, cx, cy = channel_geometry(seed)
    R, b = 0.5 * D, box_half
    if levels < 0 or nz % (1 << levels):
        raise ValueError("nz must be a multiple of 2^levels")
    nzb = nz >> levels
    h = H / nzb
    nx1 = max(1, round((cx - b) / h))
    nx3 = max(1, round((Lx - cx - b) / h))
    nth = max(2, round(2 * b / h))
    ny1 = max(1, round((cy - b) / h))
    ny3 = max(1, round((H - cy - b) / h))
    nr = max(2, round((b - R) / h))
    f = 1 << levels
    xs = [0.0, cx - b, cx + b, Lx]
    ys = [0.0, cy - b, cy + b, H]
    ncx = [nx1, nth, nx3]
    ncy = [ny1, nth, ny3]

    pts: dict = {}
    plist: list = []
    flags: list = []
    plev: list = []       # level on which a point first appears

    def lev_of(i, j):
        for s_ in range(levels + 1):
            step = 1 << (levels - s_)
            if i % step == 0 and j % step == 0:
                return s_
        return levels

    def pid(x, y, lev, on_circle=False):
        key = (round(x * 1e9), round(y * 1e9))
        k = pts.get(key)
        if k is None:
            k = len(plist)
            pts[key] = k
            plist.append((x, y))
            flags.append(on_circle)
            plev.append(lev)
        else:
            if on_circle:
                flags[k] = True
            plev[k] = min(plev[k], lev)
        return k

    quads = []
    qidx = []             # (block, i, j) of each quad at the finest level

    def add_block(P, blk):   # P: [nu+1][nv+1] point ids, structured
        nu, nv = len(P) - 1, len(P[0]) - 1
        for i in range(nu):
            for j in range(nv):
                quads.append((P[i][j], P[i + 1][j], P[i][j + 1], P[i + 1][j + 1]))
                qidx.append((blk, i, j))

    blocks = []           # base cells of each block along i and j
    for bx in range(3):
        for by in range(3):
            if bx == 1 and by == 1:
                continue
            x0, x1, y0, y1 = xs[bx], xs[bx + 1], ys[by], ys[by + 1]
            nu, nv = ncx[bx] * f, ncy[by] * f
            P = [[pid(x0 + (x1 - x0) * i / nu, y0 + (y1 - y0) * j / nv, lev_of(i, j)) for j in range(nv + 1)]
                 for i in range(nu + 1)]
            add_block(P, len(blocks))
            blocks.append((ncx[bx], ncy[by]))

    # O-grid: side s of the square, parameter i along the side (nth cells),
    # radial index j from the circle (j = 0) to the square (j = nr).
    sides = [  # (square start, square end, angle start, angle end)
        ((cx - b, cy - b), (cx + b, cy - b), 1.25 * math.pi, 1.75 * math.pi),   # bottom
        ((cx + b, cy - b), (cx + b, cy + b), -0.25 * math.pi, 0.25 * math.pi),  # right
        ((cx + b, cy + b), (cx - b, cy + b), 0.25 * math.pi, 0.75 * math.pi),   # top
        ((cx - b, cy + b), (cx - b, cy - b), 0.75 * math.pi, 1.25 * math.pi),   # left
    ]
    nthf, nrf = nth * f, nr * f
    for (s0, s1, a0, a1) in sides:
        P = []
        for i in range(nthf + 1):
            t = i / nthf
            sq = (s0[0] + (s1[0] - s0[0]) * t, s0[1] + (s1[1] - s0[1]) * t)
            a = a0 + (a1 - a0) * t
            ci = (cx + R * math.cos(a), cy + R * math.sin(a))
            col = []
            for j in range(nrf + 1):
                w = j / nrf
                x = (1 - w) * ci[0] + w * sq[0]
                y = (1 - w) * ci[1] + w * sq[1]
                col.append(pid(x, y, lev_of(i, j), on_circle=(j == 0)))
            P.append(col)
        add_block(P, len(blocks))
        blocks.append((nth, nr))

    p2 = np.array(plist, dtype=np.float64)
    on_circle = np.array(flags, dtype=bool)
    q = np.array(quads, dtype=np.int64)
    # orient every quad counter-clockwise in the (u, v) = (0..1, 0..1) order
    a, bq, c = p2[q[:, 0]], p2[q[:, 1]], p2[q[:, 2]]
    cross = (bq[:, 0] - a[:, 0]) * (c[:, 1] - a[:, 1]) - (bq[:, 1] - a[:, 1]) * (c[:, 0] - a[:, 0])
    flip = cross < 0
    q[flip] = q[flip][:, [1, 0, 3, 2]]

    n2 = p2.shape[0]
    zs = np.arange(nz + 1, dtype=np.float64) * (H / nz)
    zs[-1] = H
    xyz = np.empty(((nz + 1) * n2, 3))
    for k in range(nz + 1):
        xyz[k * n2:(k + 1) * n2, 0:2] = p2
        xyz[k * n2:(k + 1) * n2, 2] = zs[k]
    nq = q.shape[0]
    cells = np.empty((nz * nq, 8), dtype=np.int64)
    for k in range(nz):
        sl = slice(k * nq, (k + 1) * nq)
        cells[sl, 0:4] = q + k * n2
        cells[sl, 4:8] = q + (k + 1) * n2
    if levels >= 1:
        qi = np.array(qidx, dtype=np.int64)
        # one base grid per block: base cell index = block offset + (ib + nbi jb) + n_base2d * kb
        off = np.cumsum([0] + [bi * bj for bi, bj in blocks])
        nb2 = int(off[-1])
        kk = np.repeat(np.arange(nz), nq)
        ii = np.tile(qi[:, 1], nz)
        jj = np.tile(qi[:, 2], nz)
        blk = np.tile(qi[:, 0], nz)
        fl = np.tile(flip, nz)
        nbi = np.array([bi for bi, _ in blocks])[blk]
        base = off[blk] + (ii >> levels) + nbi * (jj >> levels) + nb2 * (kk >> levels)
        key = base
        for s_ in range(levels - 1, -1, -1):
            a_ = (ii >> s_) & 1
            a_ = np.where(fl, 1 - a_, a_)
            key = key * 8 + a_ + 2 * ((jj >> s_) & 1) + 4 * ((kk >> s_) & 1)
        cells = cells[np.argsort(key, kind="stable")]
        zlev = first_level(np.arange(nz + 1), nz, levels)
        vlev = np.maximum(np.tile(np.array(plev, dtype=np.int64), nz + 1), np.repeat(zlev, n2))
        perm = np.argsort(vlev, kind="stable")
        inv = np.empty_like(perm)
        inv[perm] = np.arange(perm.size)
        xyz = xyz[perm]
        on_circle = np.tile(on_circle, nz + 1)[perm]
        cells = inv[cells]
    else:
        on_circle = np.tile(on_circle, nz + 1)
    eps = 1e-12
    x, y, z = xyz[:, 0], xyz[:, 1], xyz[:, 2]
    wall = (np.abs(y) < eps) | (np.abs(y - H) < eps) | (np.abs(z) < eps) | (np.abs(z - H) < eps)
    wall |= on_circle
    bc = np.zeros(xyz.shape[0], dtype=np.int32)
    bc[np.abs(x - Lx) < eps] = 3
    bc[wall] = 1
    bc[np.abs(x) < eps] = 2
    return Mesh(xyz=xyz, cells=cells.astype(np.int32), vertex_bc=bc, patch_groups=levels >= 1,
                meta=dict(kind="channel", nz=nz, seed=seed, D=D, cx=cx, cy=cy,
                          nu_re200=D / 200.0, mg_levels=int(levels)))


# --------------------------------------------------------------------------
# boundary data (problem definition, Sec. 6.2 and the cavity configuration)
# --------------------------------------------------------------------------

def inflow_ramp(t: float) -> float:
    """Start-up factor omega(t) of the inflow (Sec. 6.2, Eq. (18))."""
    return 0.5 - 0.5 * math.cos(5.0 * math.pi * t) if t <= 0.2 else 1.0


def inflow_profile(y, z, t: float, mean: float = 1.0):
    """x-velocity at x = 0 with mean ``mean``: 36 y (H-y) z (H-z) / H^4.

    The printed formula is garbled; this reading vanishes on all four walls
    and has mean value ``mean`` over the inflow square.
    """
    H = CHANNEL_HEIGHT
    return inflow_ramp(t) * mean * 36.0 * y * (H - y) * z * (H - z) / H ** 4


def dirichlet_values(mesh: Mesh, xyz: np.ndarray, kind: np.ndarray, t: float = 1.0) -> np.ndarray:
    """Velocity [n, 3] prescribed at points with boundary kind 1 or 2."""
    v = np.zeros((xyz.shape[0], 3))
    drv = kind == 2
    if mesh["meta"]["kind"] == "cavity":
        v[drv, 0] = 1.0
    else:
        v[drv, 0] = inflow_profile(xyz[drv, 1], xyz[drv, 2], t)
    return v


# --------------------------------------------------------------------------
# fields and weights
# --------------------------------------------------------------------------

def smooth_field(xyz: np.ndarray, seed: int, n_modes: int = 8, kmax: int = 4,
                 mean=PAPER_FIELD_MEAN, std=PAPER_FIELD_STD) -> np.ndarray:
    """Smooth random (u, v, w, p) at the points ``xyz`` [n, 3].

    Each component is a sum of ``n_modes`` products of cosines with integer
    wave numbers 1..kmax per axis (relative to the bounding box) and random
    phases, then shifted and scaled to the given mean and standard deviation
    (default: the paper's training-data statistics).
    """
    lo, hi = xyz.min(axis=0), xyz.max(axis=0)
    ext = np.where(hi > lo, hi - lo, 1.0)
    s = (xyz - lo) / ext
    out = np.empty((xyz.shape[0], 4))
    for comp in range(4):
        r = splitmix_uniform(_stream(seed, 100 + comp), n_modes * 7)
        f = np.zeros(xyz.shape[0])
        for m in range(n_modes):
            k = 1 + np.floor(r[7 * m:7 * m + 3] * kmax)
            ph = 2 * np.pi * r[7 * m + 3:7 * m + 6]
            amp = 2.0 * r[7 * m + 6] - 1.0
            f += amp * np.cos(np.pi * k[0] * s[:, 0] + ph[0]) * np.cos(np.pi * k[1] * s[:, 1] + ph[1]) \
                * np.cos(np.pi * k[2] * s[:, 2] + ph[2])
        sd = f.std()
        f = (f - f.mean()) / (sd if sd > 0 else 1.0)
        out[:, comp] = mean[comp] + std[comp] * f
    return out


def coarse_state(mesh: Mesh, seed: int, t: float = 1.0) -> np.ndarray:
    """Coarse-level x^L [n_vertices, 4] = (u, v, w, p): a smooth field with the
    paper's statistics whose velocity obeys the Dirichlet data."""
    x = smooth_field(mesh["xyz"], seed)
    bc = mesh["vertex_bc"]
    dv = dirichlet_values(mesh, mesh["xyz"], bc, t)
    d = (bc == 1) | (bc == 2)
    x[d, 0:3] = dv[d]
    return x


def fine_rhs(n_fine: int, seed: int, scale: float = 1e-3) -> np.ndarray:
    """A right-hand side F [n_fine, 4] with iid normal entries times ``scale``
    (stands in for the previous step's b^{L+1} at the first step)."""
    return scale * splitmix_normal(_stream(seed, 200), 4 * n_fine).reshape(n_fine, 4)


def network_weights(widths, seed: int = 0, scale_shift: bool = False):
    """Weights W_i [widths[i+1], widths[i]] drawn U(-1/sqrt(fan_in), 1/sqrt(fan_in)).

    Returns (Ws, scales, shifts).  Without ``scale_shift`` every layer gets
    scale 1 and shift 0 (batch normalisation at its initial state).  With it,
    hidden layers get seeded scale in [0.5, 1.5] and shift in [-0.1, 0.1],
    standing in for folded batch-normalisation parameters.  The last layer
    always has scale 1 and shift 0 (no bias, as the paper's parameter counts
    imply).
    """
    Ws, ss, ts = [], [], []
    L = len(widths) - 1
    for i in range(L):
        fin, fout = widths[i], widths[i + 1]
        u = splitmix_uniform(_stream(seed, 1000 + i), fin * fout)
        Ws.append(((2.0 * u - 1.0) / math.sqrt(fin)).reshape(fout, fin))
        if scale_shift and i < L - 1:
            v = splitmix_uniform(_stream(seed, 2000 + i), 2 * fout)
            ss.append(0.5 + v[:fout])
            ts.append(0.2 * v[fout:] - 0.1)
        else:
            ss.append(np.ones(fout))
            ts.append(np.zeros(fout))
    return Ws, ss, ts


# The configurations the path is measured and tested on.
CFG_CAVITY = dict(name="cavity-8^3->16^3 Re100 BE fp64 MLP 228-256-256-81",
                  mesh=dict(kind="cavity", n=8), nu=0.01, dt=0.01, theta=1.0,
                  widths=(228, 256, 256, 81))
CFG_CHANNEL = dict(name="channel ~43k->~340k hex Re200 CN fp32 MLP 228-512x3-81",
                   mesh=dict(kind="channel", nz=19), dt=0.005, theta=0.5,
                   widths=(228, 512, 512, 512, 81))
CFG_CHANNEL_BF16 = dict(name="channel ~318k->~2.5M hex Re200 CN bf16 MLP 228-1024x4-81",
                        mesh=dict(kind="channel", nz=37), dt=0.005, theta=0.5,
                        widths=(228, 1024, 1024, 1024, 1024, 81))


def make_mesh(spec: dict, seed: int = 0) -> Mesh:
    if spec["kind"] == "cavity":
        return cavity_mesh(spec["n"], jitter=spec.get("jitter", 0.0), seed=seed)
    return channel_mesh(spec["nz"], seed=seed)
