"""Seeded synthetic spin systems: lattice generation and CSR neighbour lists.

This module builds the *inputs* of the Heun-LLG step -- site positions, per-site moments
and anisotropies, and the exchange neighbour list in CSR form -- following the system
generation scheme of arXiv:1310.6143 (Appendix B: replicate a unit cell, cut the shape,
assign materials, build the nearest-neighbour interaction list from per-cell offsets).
It contains no part of the integrator, field or reduction arithmetic, and is used by
both the CUDA path and the CPU oracle's tests.

Conventions
-----------
* SI units: moments in J/T, energies in J, fields in T, lengths in m.
* CSR rows list every neighbour j of site i (both directions of every bond), no self
  bonds; ``row_ptr`` is int64, ``col`` int32, ``J`` float64.
* Simple-cubic index ``i = z + nz * (x + nx * y)`` (z fastest): for a thin film the
  short axis is contiguous, so the six neighbours of a site are within +-nz*nx sites.
* FCC: four sites per cubic cell at (0,0,0), (1/2,1/2,0), (1/2,0,1/2), (0,1/2,1/2);
  index ``i = b + 4 * (cz + nz * (cx + nx * cy))``.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

MU_B = 9.2740e-24  # Bohr magneton, J/T (Table I of the paper)
KB = 1.3807e-23    # Boltzmann constant, J/K (Table I)


@dataclass
class SpinLattice:
    """A spin system as plain arrays (the argument set of ``spin_system_create``)."""

    row_ptr: np.ndarray            # int64 [n+1]
    col: np.ndarray                # int32 [nnz]
    J: np.ndarray                  # float64 [nnz], J/link
    mu_s: np.ndarray               # float64 [n], J/T
    k_u: np.ndarray                # float64 [n], J/atom
    easy_axis: np.ndarray          # float64 [n, 3]
    K_neel: np.ndarray | None = None   # float64 [n, 6] (xx, yy, zz, xy, xz, yz) or None
    pos: np.ndarray | None = None      # float64 [n, 3], m
    meta: dict = field(default_factory=dict)
    J_tensor: np.ndarray | None = None  # float64 [nnz, 3, 3] exchange tensors (J then unused), or None
    k_c: np.ndarray | None = None       # float64 [n] cubic anisotropy, J/atom, or None

    @property
    def n(self) -> int:
        return int(self.row_ptr.size - 1)

    @property
    def nnz(self) -> int:
        return int(self.col.size)


def _csr_from_targets(targets: np.ndarray, jvals: np.ndarray | float):
    """targets: (n, z) int64 neighbour ids, -1 where absent; rows keep column order."""
    valid = targets >= 0
    counts = valid.sum(axis=1)
    row_ptr = np.zeros(targets.shape[0] + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    col = targets[valid].astype(np.int32)
    if np.isscalar(jvals):
        J = np.full(col.size, float(jvals))
    else:
        J = np.asarray(jvals, dtype=np.float64)[valid]
    return row_ptr, col, J


def _homogeneous(n, mu_s, k_u, easy_axis):
    ax = np.asarray(easy_axis, dtype=np.float64)
    ax = ax / np.linalg.norm(ax)
    return (np.full(n, float(mu_s)), np.full(n, float(k_u)), np.ascontiguousarray(np.broadcast_to(ax, (n, 3))))


def simple_cubic(nx: int, ny: int, nz: int, periodic=(True, True, True), J=6.0e-21,
                 mu_s=1.5 * MU_B, k_u=1.0e-24, easy_axis=(0.0, 0.0, 1.0), a=3.0e-10,
                 with_pos: bool = False) -> SpinLattice:
    """Simple-cubic lattice with nearest-neighbour exchange (z = 6 in the bulk).

    Each row lists neighbours in the order -z, +z, -x, +x, -y, +y (absent ones skipped at
    free surfaces).  A periodic axis needs at least 3 sites, so that no bond is a self
    bond or a duplicate.
    """
    for L, p in zip((nx, ny, nz), periodic):
        if L < 1 or (p and L < 3):
            raise ValueError("each axis needs >= 1 site, periodic axes >= 3 sites")
    n = nx * ny * nz
    idx = np.arange(n, dtype=np.int64)
    z = idx % nz
    x = (idx // nz) % nx
    y = idx // (nz * nx)

    def site(xx, yy, zz):
        return zz + nz * (xx + nx * yy)

    targets = np.full((n, 6), -1, dtype=np.int64)
    for d, (axis, step) in enumerate((("z", -1), ("z", 1), ("x", -1), ("x", 1), ("y", -1), ("y", 1))):
        L, p = {"x": (nx, periodic[0]), "y": (ny, periodic[1]), "z": (nz, periodic[2])}[axis]
        coord = {"x": x, "y": y, "z": z}[axis]
        c2 = coord + step
        ok = (c2 >= 0) & (c2 < L)
        if p:
            c2 = c2 % L
            ok = np.ones(n, dtype=bool)
        xx = c2 if axis == "x" else x
        yy = c2 if axis == "y" else y
        zz = c2 if axis == "z" else z
        t = site(xx % nx, yy % ny, zz % nz)
        targets[:, d] = np.where(ok, t, -1)
    row_ptr, col, Jv = _csr_from_targets(targets, J)
    mu, ku, ax = _homogeneous(n, mu_s, k_u, easy_axis)
    pos = np.stack([x, y, z], axis=1).astype(np.float64) * a if with_pos else None
    return SpinLattice(row_ptr, col, Jv, mu, ku, ax, None, pos,
                       meta={"kind": "sc", "dims": (nx, ny, nz), "periodic": tuple(periodic), "a": a})


_FCC_BASIS = np.array([[0, 0, 0], [1, 1, 0], [1, 0, 1], [0, 1, 1]], dtype=np.int64)  # doubled units
_FCC_NN = np.array([[sx, sy, 0] for sx in (-1, 1) for sy in (-1, 1)]
                   + [[sx, 0, sz] for sx in (-1, 1) for sz in (-1, 1)]
                   + [[0, sy, sz] for sy in (-1, 1) for sz in (-1, 1)], dtype=np.int64)


def _fcc_sites(nx, ny, nz):
    """Doubled integer coordinates of all fcc sites in nx*ny*nz cells, in index order."""
    ncell = nx * ny * nz
    c = np.arange(ncell, dtype=np.int64)
    cz = c % nz
    cx = (c // nz) % nx
    cy = c // (nz * nx)
    cell = np.stack([cx, cy, cz], axis=1) * 2
    X = (cell[:, None, :] + _FCC_BASIS[None, :, :]).reshape(-1, 3)
    return X


def _fcc_index(X, nx, ny, nz):
    """Inverse of _fcc_sites for doubled coordinates already wrapped into the box."""
    cx, cy, cz = X[:, 0] // 2, X[:, 1] // 2, X[:, 2] // 2
    px, py, pz = X[:, 0] % 2, X[:, 1] % 2, X[:, 2] % 2
    b = np.where((px == 0) & (py == 0), 0, np.where(pz == 0, 1, np.where(py == 0, 2, 3)))
    return b + 4 * (cz + nz * (cx + nx * cy))


def fcc(nx: int, ny: int, nz: int, periodic=(True, True, True), J=11.2e-21, mu_s=1.72 * MU_B,
        k_u=6.69e-24, easy_axis=(0.0, 0.0, 1.0), a=3.524e-10, with_pos: bool = False) -> SpinLattice:
    """Face-centred-cubic lattice of nx*ny*nz cubic cells, 12 nearest neighbours at a/sqrt(2)."""
    for L, p in zip((nx, ny, nz), periodic):
        if L < 1 or (p and L < 2):
            raise ValueError("fcc: each axis needs >= 1 cell, periodic axes >= 2 cells")
    X = _fcc_sites(nx, ny, nz)
    n = X.shape[0]
    dims = np.array([2 * nx, 2 * ny, 2 * nz])
    targets = np.full((n, 12), -1, dtype=np.int64)
    for d in range(12):
        Y = X + _FCC_NN[d]
        ok = np.ones(n, dtype=bool)
        for ax in range(3):
            if periodic[ax]:
                Y[:, ax] %= dims[ax]
            else:
                ok &= (Y[:, ax] >= 0) & (Y[:, ax] < dims[ax])
        Yc = np.where(ok[:, None], Y, 0)
        targets[:, d] = np.where(ok, _fcc_index(Yc, nx, ny, nz), -1)
    row_ptr, col, Jv = _csr_from_targets(targets, J)
    mu, ku, ax_ = _homogeneous(n, mu_s, k_u, easy_axis)
    pos = X.astype(np.float64) * (a / 2) if with_pos else None
    return SpinLattice(row_ptr, col, Jv, mu, ku, ax_, None, pos,
                       meta={"kind": "fcc", "cells": (nx, ny, nz), "periodic": tuple(periodic), "a": a,
                             "box": tuple(np.array([nx, ny, nz], dtype=np.float64) * a * np.array(periodic)
                                          + np.array([0 if p else np.inf for p in periodic]))})


def fcc_stencil(r_cut: float):
    """The fcc lattice vectors within r_cut (in units of the cubic lattice constant a), as
    doubled integer coordinates (x + y + z even), sorted by length then lexicographically."""
    m = int(np.floor(2 * r_cut + 1e-9))
    g = np.stack(np.meshgrid(*[np.arange(-m, m + 1, dtype=np.int64)] * 3, indexing="ij"), -1).reshape(-1, 3)
    n2 = (g * g).sum(axis=1)
    g = g[(g.sum(axis=1) % 2 == 0) & (n2 > 0) & (n2 <= int(np.floor((2 * r_cut) ** 2 + 1e-9)))]
    order = np.lexsort((g[:, 2], g[:, 1], g[:, 0], (g * g).sum(axis=1)))
    return g[order]


def fcc_long_range(nx: int, ny: int, nz: int, r_cut=4.0, decay=0.5, J_total=12 * 11.2e-21, periodic=(True, True, True),
                   mu_s=1.72 * MU_B, k_u=6.69e-24, easy_axis=(0.0, 0.0, 1.0), a=3.524e-10,
                   with_pos: bool = False) -> SpinLattice:
    """FCC with isotropic exchange to every site within r_cut * a (1,060 neighbours for r_cut = 4,
    30 distance shells): J(r) = J_nn exp(-(r - r_nn) / (decay * a)), r_nn = a / sqrt(2), with J_nn
    set so that the bonds of a bulk site sum to J_total (12 x 11.2e-21 J by default, the total of
    the nearest-neighbour fcc system).  A synthetic stand-in for the long-ranged ab initio
    exchange of the paper's additional scaling tests (over 1,000 neighbours per atom), whose
    parameters are not used here.  Rows list the neighbours in stencil order (by distance);
    periodic axes need more than 2 r_cut cells so that every neighbour is a distinct site."""
    for L, p in zip((nx, ny, nz), periodic):
        if L < 1:
            raise ValueError("fcc_long_range: each axis needs >= 1 cell")
        if p and L <= 2 * r_cut:
            raise ValueError("fcc_long_range: periodic axes need more than 2 * r_cut cells")
    st = fcc_stencil(r_cut)
    r = np.sqrt((st * st).sum(axis=1)) * 0.5  # in units of a
    shape = np.exp(-(r - 1 / np.sqrt(2)) / decay)
    Jd = J_total / shape.sum() * shape
    n = 4 * nx * ny * nz
    z = st.shape[0]
    # site i = b + 4 (cz + nz (cx + nx cy)): targets per (basis, stencil vector) over the cell grid
    targets = np.empty((4, z, ny, nx, nz), dtype=np.int32)  # filled contiguously, transposed below
    ncell = (nx, ny, nz)

    def axis_map(ax, o):
        """Cell index along axis ax after a shift by o cells (-1 outside a free axis)."""
        c = np.arange(ncell[ax], dtype=np.int64) + o
        if periodic[ax]:
            return c % ncell[ax]
        return np.where((c >= 0) & (c < ncell[ax]), c, -1)

    for b in range(4):
        w = _FCC_BASIS[b] + st                      # doubled coordinates of the targets
        o, par = w // 2, w % 2                     # cell offsets and parities
        bt = _fcc_index(par, 1, 1, 1)              # target basis index from the parities
        for d in range(z):
            mx, my, mz = axis_map(0, o[d, 0]), axis_map(1, o[d, 1]), axis_map(2, o[d, 2])
            t = bt[d] + 4 * (mz[None, None, :] + nz * (mx[None, :, None] + nx * my[:, None, None]))
            bad = (mz[None, None, :] < 0) | (mx[None, :, None] < 0) | (my[:, None, None] < 0)
            targets[b, d] = np.where(bad, -1, t)
    targets = np.ascontiguousarray(targets.transpose(2, 3, 4, 0, 1)).reshape(n, z)
    if all(periodic):
        row_ptr = np.arange(n + 1, dtype=np.int64) * z
        col = targets.reshape(-1)
        J = np.tile(Jd, n)
    else:
        valid = targets >= 0
        row_ptr = np.zeros(n + 1, dtype=np.int64)
        np.cumsum(valid.sum(axis=1), out=row_ptr[1:])
        col = targets[valid]
        J = np.broadcast_to(Jd, (n, z))[valid]
    mu, ku, ax_ = _homogeneous(n, mu_s, k_u, easy_axis)
    pos = _fcc_sites(nx, ny, nz).astype(np.float64) * (a / 2) if with_pos else None
    return SpinLattice(row_ptr, col, J, mu, ku, ax_, None, pos,
                       meta={"kind": "fcc_long_range", "cells": (nx, ny, nz), "periodic": tuple(periodic), "a": a,
                             "r_cut": r_cut, "shells": int(np.unique((st * st).sum(axis=1)).size),
                             "J_shells": np.unique(Jd)[::-1]})


def film(nx=1024, ny=1024, nz=16, J=6.0e-21, mu_s=1.5 * MU_B, k_u=1.0e-24) -> SpinLattice:
    """Thin simple-cubic film, periodic in-plane, free surfaces in z."""
    lat = simple_cubic(nx, ny, nz, periodic=(True, True, False), J=J, mu_s=mu_s, k_u=k_u)
    lat.meta["kind"] = "film"
    return lat


def neel_tensors(pos: np.ndarray, row_ptr: np.ndarray, col: np.ndarray, k_s: float,
                 mask: np.ndarray) -> np.ndarray:
    """Neel pair surface-anisotropy tensors K_i = (k_s/2) sum_j e_ij e_ij^T on masked sites.

    e_ij is the unit bond vector to neighbour j.  The energy of site i is -S_i^T K_i S_i.
    Returns (n, 6) in the order xx, yy, zz, xy, xz, yz (zero rows where mask is False).
    """
    n = row_ptr.size - 1
    rows = np.repeat(np.arange(n), np.diff(row_ptr))
    d = pos[col] - pos[rows]
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    comps = np.stack([d[:, 0] * d[:, 0], d[:, 1] * d[:, 1], d[:, 2] * d[:, 2],
                      d[:, 0] * d[:, 1], d[:, 0] * d[:, 2], d[:, 1] * d[:, 2]], axis=1)
    K = np.zeros((n, 6))
    np.add.at(K, rows, comps)
    K *= 0.5 * k_s
    K[~mask] = 0.0
    return K


def subset(lat: SpinLattice, sites: np.ndarray) -> SpinLattice:
    """The lattice induced on `sites` (sorted site ids): their per-site arrays and the bonds
    between them, renumbered 0..len(sites)-1 in the given order."""
    sites = np.asarray(sites, dtype=np.int64)
    new_id = np.full(lat.n, -1, dtype=np.int64)
    new_id[sites] = np.arange(sites.size)
    rows = np.repeat(np.arange(lat.n), np.diff(lat.row_ptr))
    keep = (new_id[rows] >= 0) & (new_id[lat.col] >= 0)
    r, c, j = new_id[rows[keep]], new_id[lat.col[keep]], lat.J[keep]
    order = np.lexsort((np.arange(r.size), r))  # rows in order, bonds in their CSR order
    row_ptr = np.zeros(sites.size + 1, dtype=np.int64)
    np.cumsum(np.bincount(r, minlength=sites.size), out=row_ptr[1:])
    return SpinLattice(row_ptr, c[order].astype(np.int32), j[order], lat.mu_s[sites], lat.k_u[sites],
                       lat.easy_axis[sites], None if lat.K_neel is None else lat.K_neel[sites],
                       None if lat.pos is None else lat.pos[sites], meta=dict(lat.meta, subset=True),
                       J_tensor=None if lat.J_tensor is None else lat.J_tensor[keep][order],
                       k_c=None if lat.k_c is None else lat.k_c[sites])


def prolate_ellipsoid(diameter=10e-9, height=20e-9, a=3.54e-10, mu_s=1.5 * MU_B, H_a=1.0, J=11.2e-21) -> SpinLattice:
    """The demagnetising-field test particle of the paper's prolate-ellipsoid section: an fcc
    crystal (lattice constant a, moment mu_s, uniaxial anisotropy field H_a = 2 k_u / mu_s along
    the long axis z) cut to an ellipsoid `diameter` across and `height` long, with positions.
    The paper gives no exchange constant for it; J is the fcc value used elsewhere here."""
    nxy = int(np.ceil(diameter / a)) + 1
    nz = int(np.ceil(height / a)) + 1
    big = fcc(nxy, nxy, nz, periodic=(False, False, False), J=J, mu_s=mu_s, k_u=0.5 * mu_s * H_a, a=a,
              with_pos=True)
    c = big.pos - np.array([nxy, nxy, nz]) * a / 2
    keep = (c[:, 0] / (diameter / 2)) ** 2 + (c[:, 1] / (diameter / 2)) ** 2 + (c[:, 2] / (height / 2)) ** 2 <= 1.0
    lat = subset(big, np.nonzero(keep)[0])
    lat.meta.update(kind="prolate_ellipsoid", atom_volume=a ** 3 / 4, a=a)
    return lat


def with_dm(lat: SpinLattice, D: float, normal=(0.0, 0.0, 1.0)) -> SpinLattice:
    """Exchange tensors J_ij I + [D_ij]x with an interface-type Dzyaloshinskii-Moriya vector
    D_ij = D (r_ij x n) / |r_ij| (r_ij from site i to its neighbour j, n the interface normal),
    so that the energy gains D_ij . (S_i x S_j) (Eqs. HJijM, HJijSMS); the reverse bond carries
    the transpose (D_ji = -D_ij).  Needs positions; periodic neighbours take the shortest image
    of the lattice box (meta "box")."""
    if lat.pos is None:
        raise ValueError("with_dm needs positions")
    rows = np.repeat(np.arange(lat.n), np.diff(lat.row_ptr))
    r = lat.pos[lat.col] - lat.pos[rows]
    box = lat.meta.get("box")
    if box is not None:
        box = np.asarray(box, dtype=np.float64)
        r -= box * np.round(r / box)
    u = r / np.linalg.norm(r, axis=1, keepdims=True)
    Dv = D * np.cross(u, np.asarray(normal, dtype=np.float64))
    Jt = lat.J[:, None, None] * np.eye(3)[None].repeat(lat.nnz, 0)
    # [d]x with [d]x v = d x v, so that S_i . [d]x S_j = d . (S_j x S_i) and -S_i.[d]x S_j = d . (S_i x S_j)
    Jt[:, 0, 1] -= Dv[:, 2]
    Jt[:, 0, 2] += Dv[:, 1]
    Jt[:, 1, 0] += Dv[:, 2]
    Jt[:, 1, 2] -= Dv[:, 0]
    Jt[:, 2, 0] -= Dv[:, 1]
    Jt[:, 2, 1] += Dv[:, 0]
    lat.J_tensor = Jt
    return lat


def core_shell_sphere(diameter=20e-9, a=3.524e-10, r_core=8e-9, J_core=11.2e-21, J_shell=-5.0e-21,
                      J_int=2.0e-21, mu_s=1.72 * MU_B, k_s=5.0e-23, z_full=12) -> SpinLattice:
    """FCC sphere cut from a crystal: ferromagnetic core, antiferromagnetic shell.

    Bonds are core-core J_core, shell-shell J_shell and core-shell J_int.  Sites with
    fewer than ``z_full`` neighbours (the surface) carry a Neel pair anisotropy tensor of
    strength k_s.  No uniaxial anisotropy (k_u = 0, easy axis +z).
    """
    R = diameter / 2
    cells = int(np.ceil(diameter / a)) + 1
    X = _fcc_sites(cells, cells, cells)
    centre = np.full(3, cells * a / 2)
    P = X.astype(np.float64) * (a / 2) - centre
    keep = np.einsum("ij,ij->i", P, P) <= R * R
    new_id = np.full(X.shape[0], -1, dtype=np.int64)
    new_id[keep] = np.arange(int(keep.sum()))
    Xk = X[keep]
    Pk = P[keep]
    n = Xk.shape[0]
    dims = np.array([2 * cells] * 3)
    core = np.einsum("ij,ij->i", Pk, Pk) < r_core * r_core
    targets = np.full((n, 12), -1, dtype=np.int64)
    jv = np.zeros((n, 12))
    for d in range(12):
        Y = Xk + _FCC_NN[d]
        ok = np.all((Y >= 0) & (Y < dims), axis=1)
        Yc = np.where(ok[:, None], Y, 0)
        t = new_id[_fcc_index(Yc, cells, cells, cells)]
        t = np.where(ok, t, -1)
        targets[:, d] = t
        tc = np.where(t >= 0, core[np.maximum(t, 0)], False)
        jv[:, d] = np.where(core & tc, J_core, np.where(~core & ~tc, J_shell, J_int))
    row_ptr, col, Jv = _csr_from_targets(targets, jv)
    mu, ku, ax = _homogeneous(n, mu_s, 0.0, (0, 0, 1))
    coord = np.diff(row_ptr)
    K = neel_tensors(Pk, row_ptr, col, k_s, coord < z_full)
    return SpinLattice(row_ptr, col, Jv, mu, ku, ax, K, Pk,
                       meta={"kind": "core_shell", "diameter": diameter, "r_core": r_core,
                             "n_core": int(core.sum()), "n_surface": int((coord < z_full).sum())})


def _grain_shape(rng, target_columns, n_nbr=7):
    """Columns (x, y) of one Voronoi-like cell: the points nearer the origin than any of
    n_nbr seeded neighbour seeds, with the seed distance scaled so the cell holds
    about target_columns lattice columns."""
    ang = (np.linspace(0, 2 * np.pi, n_nbr, endpoint=False) + rng.uniform(-0.3, 0.3, n_nbr)
           + rng.uniform(0, 2 * np.pi))
    rad = rng.uniform(0.8, 1.2, n_nbr)
    q = np.stack([np.cos(ang) * rad, np.sin(ang) * rad], axis=1)

    def columns(D):
        ext = int(np.ceil(D * 1.3)) + 2
        g = np.arange(-ext, ext + 1)
        gx, gy = np.meshgrid(g, g, indexing="ij")
        p = np.stack([gx.ravel(), gy.ravel()], axis=1).astype(np.float64)
        qq = q * D
        inside = np.all(p @ qq.T < 0.5 * np.einsum("ij,ij->i", qq, qq)[None, :], axis=1)
        return p[inside].astype(np.int64)

    lo, hi = 1.0, 2.0
    while columns(hi).shape[0] < target_columns:
        hi *= 2
    for _ in range(40):
        mid = 0.5 * (lo + hi)
        if columns(mid).shape[0] < target_columns:
            lo = mid
        else:
            hi = mid
    return columns(hi)


def grain(columns: np.ndarray, layers: int, J=6.0e-21, mu_s=1.5 * MU_B, k_u=1.0e-23,
          easy_axis=(0, 0, 1)) -> SpinLattice:
    """A columnar grain: the given (x, y) columns extruded over ``layers`` simple-cubic
    layers, free surfaces everywhere, sites ordered by column then layer."""
    cols = columns - columns.min(axis=0)
    W = int(cols[:, 0].max()) + 1
    H = int(cols[:, 1].max()) + 1
    order = np.lexsort((cols[:, 0], cols[:, 1]))
    cols = cols[order]
    ncol = cols.shape[0]
    colid = np.full((W + 2, H + 2), -1, dtype=np.int64)
    colid[cols[:, 0] + 1, cols[:, 1] + 1] = np.arange(ncol)
    n = ncol * layers
    idx = np.arange(n)
    z = idx % layers
    c = idx // layers
    cx, cy = cols[c, 0] + 1, cols[c, 1] + 1
    targets = np.full((n, 6), -1, dtype=np.int64)
    targets[:, 0] = np.where(z > 0, idx - 1, -1)
    targets[:, 1] = np.where(z < layers - 1, idx + 1, -1)
    for d, (dx, dy) in enumerate(((-1, 0), (1, 0), (0, -1), (0, 1))):
        nb = colid[cx + dx, cy + dy]
        targets[:, 2 + d] = np.where(nb >= 0, nb * layers + z, -1)
    row_ptr, col, Jv = _csr_from_targets(targets, J)
    mu, ku, ax = _homogeneous(n, mu_s, k_u, easy_axis)
    return SpinLattice(row_ptr, col, Jv, mu, ku, ax, None, None,
                       meta={"kind": "grain", "columns": ncol, "layers": layers})


def grain_ensemble(count=256, n_min=2000, n_max=40000, layers=10, seed=12345, J=6.0e-21,
                   mu_s=1.5 * MU_B, ku_mean=1.0e-23, ku_lnsigma=0.3, cap_deg=5.0, T_max=800.0):
    """Independent columnar Voronoi-like grains (the granular-medium picture of Appendix B).

    Grain sizes are uniform in [n_min, n_max] spins; k_u is log-normal with arithmetic mean
    ku_mean and log-sigma ku_lnsigma; easy axes are uniform on the spherical cap within
    cap_deg of +z; temperatures are uniform in [0, T_max].  Returns (grains, temperatures).
    """
    rng = np.random.default_rng(seed)
    sizes = rng.integers(n_min, n_max + 1, size=count)
    mu_ln = np.log(ku_mean) - 0.5 * ku_lnsigma ** 2
    kus = np.exp(rng.normal(mu_ln, ku_lnsigma, size=count))
    cos_cap = np.cos(np.deg2rad(cap_deg))
    ct = rng.uniform(cos_cap, 1.0, size=count)
    ph = rng.uniform(0, 2 * np.pi, size=count)
    st = np.sqrt(1 - ct * ct)
    axes = np.stack([st * np.cos(ph), st * np.sin(ph), ct], axis=1)
    temps = rng.uniform(0.0, T_max, size=count)
    grains = []
    for g in range(count):
        cols = _grain_shape(rng, max(1, int(round(sizes[g] / layers))))
        gr = grain(cols, layers, J=J, mu_s=mu_s, k_u=float(kus[g]), easy_axis=axes[g])
        gr.meta.update({"grain": g, "T": float(temps[g])})
        grains.append(gr)
    return grains, temps


def single_spin(mu_s=1.5 * MU_B, k_u=0.0, easy_axis=(0, 0, 1)) -> SpinLattice:
    """One isolated spin (empty neighbour list)."""
    mu, ku, ax = _homogeneous(1, mu_s, k_u, easy_axis)
    return SpinLattice(np.zeros(2, dtype=np.int64), np.zeros(0, dtype=np.int32), np.zeros(0), mu, ku, ax,
                       meta={"kind": "single"})


def dimer(J=6.0e-21, mu_s=1.5 * MU_B, k_u=0.0) -> SpinLattice:
    """Two spins joined by one bond."""
    mu, ku, ax = _homogeneous(2, mu_s, k_u, (0, 0, 1))
    return SpinLattice(np.array([0, 1, 2], dtype=np.int64), np.array([1, 0], dtype=np.int32),
                       np.array([J, J]), mu, ku, ax, meta={"kind": "dimer"})


def uniform_state(n: int, direction=(0.0, 0.0, 1.0)) -> np.ndarray:
    d = np.asarray(direction, dtype=np.float64)
    return np.ascontiguousarray(np.broadcast_to(d / np.linalg.norm(d), (n, 3)))


def random_state(n: int, seed: int) -> np.ndarray:
    """Seeded random unit vectors (numpy generator; input data, not the method's stream)."""
    rng = np.random.default_rng(seed)
    v = rng.normal(size=(n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)
