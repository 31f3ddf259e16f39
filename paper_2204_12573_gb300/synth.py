"""Seeded synthetic inputs: H2/Pt(111) slabs, Maxwell velocities and model matrices.

This module holds none of the force-field arithmetic.  It only builds the
inputs that both the CUDA path and the FP64 oracle consume, so that the two
can be compared on identical data.

Geometry follows the paper's simulated system (Sec. VI-A: H2 gas over a
Pt(111) slab, Nose-Hoover MD at 450 K) with the sizes of the benchmark
workloads:

* Pt is FCC with a = 3.92 A; the (111) surface is a hexagonal net with
  in-plane spacing a/sqrt(2) and ABC stacking at interlayer spacing a/sqrt(3).
* H2 has a 0.74 A bond and a uniformly random orientation.
* x/y are periodic, z is open (vacuum above and below the slab).

Species codes: 0 = Pt, 1 = H.  Positions are returned in float64 and are
rounded to float32 by :func:`as_f32_positions` before use, so that both
implementations see bit-identical coordinates.

The model matrices beta_s (mean) and Sigma_s (variance) of the mapped sparse
GP (Eq. 1 and Eq. 2) are not published; they are drawn here as seeded random
symmetric matrices: beta_s = Q diag(lambda) Q^T with lambda ~ U[-1, 1] scaled
so that ||beta_s||_2 = 1 eV, and Sigma_s = Q' diag(mu) Q'^T with mu
log-uniform in [1e-4, 1] (positive definite).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

A_PT = 3.92                       # FCC lattice constant of Pt (A)
D_NN = A_PT / math.sqrt(2.0)      # in-plane nearest-neighbour spacing (A)
DZ_111 = A_PT / math.sqrt(3.0)    # (111) interlayer spacing (A)
H2_BOND = 0.74                    # H-H bond length (A)
KB_EV = 8.617333262e-5            # Boltzmann constant (eV/K)
FTM2V = 1.0 / 1.0364269e-4        # (eV/A)/amu -> A/ps^2
MASS = {0: 195.084, 1: 1.008}     # amu
PT, H = 0, 1


@dataclasses.dataclass
class Structure:
    """A periodic-in-plane atomic structure (float64 master copy)."""
    pos: np.ndarray        # [n, 3] float64, A
    species: np.ndarray    # [n] int32
    cell: np.ndarray       # [3, 3] float64, rows are lattice vectors
    pbc: tuple             # (1, 1, 0)
    name: str = ""

    @property
    def n_atoms(self) -> int:
        return int(self.pos.shape[0])


def as_f32_positions(pos: np.ndarray) -> np.ndarray:
    """Round positions to float32 and return them as an [n, 4] float32 array
    (x, y, z, 0); the float64 values of this array are what the oracle sees."""
    out = np.zeros((pos.shape[0], 4), dtype=np.float32)
    out[:, :3] = pos.astype(np.float32)
    return out


def f32_exact_f64(pos4: np.ndarray) -> np.ndarray:
    """The float64 view of float32 positions (exact conversion)."""
    return pos4[:, :3].astype(np.float64)


def _random_unit(rng: np.random.Generator, n: int) -> np.ndarray:
    v = rng.normal(size=(n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def _layer_offset(layer: int) -> np.ndarray:
    # ABC stacking: successive layers sit over the hollow sites, shifted by
    # (u1 + u2) / 3 with u1 = (d, 0), u2 = (d/2, d*sqrt(3)/2).
    k = layer % 3
    return k * np.array([D_NN / 2.0, D_NN * math.sqrt(3.0) / 6.0, 0.0])


def pt111_hex_slab(n1: int, n2: int, n_layers: int, vacuum: float = 15.0):
    """n1 x n2 hexagonal Pt(111) cell (cell vectors n1*u1, n2*u2), n_layers deep.
    Returns (pos, cell, z_top)."""
    u1 = np.array([D_NN, 0.0, 0.0])
    u2 = np.array([D_NN / 2.0, D_NN * math.sqrt(3.0) / 2.0, 0.0])
    pts = []
    for layer in range(n_layers):
        off = _layer_offset(layer) + np.array([0.0, 0.0, layer * DZ_111])
        for i in range(n1):
            for j in range(n2):
                pts.append(i * u1 + j * u2 + off)
    pos = np.asarray(pts, dtype=np.float64)
    z_top = (n_layers - 1) * DZ_111
    cell = np.array([n1 * u1, n2 * u2, [0.0, 0.0, z_top + vacuum]])
    # wrap the in-plane fractional coordinates into [0, 1)
    frac = pos @ np.linalg.inv(cell)
    frac[:, :2] -= np.floor(frac[:, :2])
    pos = frac @ cell
    return pos, cell, z_top


def pt111_ortho_slab(nx: int, n_rows: int, n_layers: int, vacuum: float = 15.0):
    """Orthogonal Pt(111) supercell: nx atoms per row along x, n_rows rows
    (n_rows even) spaced d*sqrt(3)/2 along y, alternate rows shifted by d/2."""
    assert n_rows % 2 == 0
    dy = D_NN * math.sqrt(3.0) / 2.0
    ix = np.arange(nx, dtype=np.float64)
    iy = np.arange(n_rows, dtype=np.float64)
    X, Y = np.meshgrid(ix, iy, indexing="xy")          # [rows, nx]
    X = (X + 0.5 * (Y % 2)) * D_NN
    Y = Y * dy
    base = np.stack([X.ravel(), Y.ravel(), np.zeros(X.size)], axis=1)
    layers = []
    for layer in range(n_layers):
        off = _layer_offset(layer) + np.array([0.0, 0.0, layer * DZ_111])
        layers.append(base + off)
    pos = np.concatenate(layers, axis=0)
    z_top = (n_layers - 1) * DZ_111
    cell = np.diag([nx * D_NN, n_rows * dy, z_top + vacuum])
    pos[:, 0] %= cell[0, 0]
    pos[:, 1] %= cell[1, 1]
    return pos, cell, z_top


def _min_image_dist(a: np.ndarray, b: np.ndarray, cell: np.ndarray, pbc) -> np.ndarray:
    """Distances |a_i - b_j| over in-plane images (-1, 0, 1); small inputs only."""
    best = None
    for s1 in (-1, 0, 1) if pbc[0] else (0,):
        for s2 in (-1, 0, 1) if pbc[1] else (0,):
            t = s1 * cell[0] + s2 * cell[1]
            d = np.linalg.norm(a[:, None, :] - (b[None, :, :] + t), axis=2)
            best = d if best is None else np.minimum(best, d)
    return best


def tiny_system(seed: int = 0, sigma_disp: float = 0.05) -> Structure:
    """3x3 hexagonal Pt(111) x 4 layers (36 Pt) + 4 H2 molecules 1.5-3 A above
    the top layer, random orientations, Gaussian displacements; 44 atoms."""
    rng = np.random.default_rng(seed)
    pos, cell, z_top = pt111_hex_slab(3, 3, 4, vacuum=15.0)
    pos = pos + rng.normal(scale=sigma_disp, size=pos.shape)
    species = [PT] * len(pos)
    h_atoms = np.zeros((0, 3))
    placed = 0
    while placed < 4:
        f = rng.uniform(size=2)
        c = f[0] * cell[0] + f[1] * cell[1]
        c[2] = z_top + rng.uniform(1.5, 3.0)
        u = _random_unit(rng, 1)[0]
        mol = np.stack([c + 0.5 * H2_BOND * u, c - 0.5 * H2_BOND * u])
        mol = mol + rng.normal(scale=sigma_disp, size=mol.shape)
        others = np.concatenate([pos, h_atoms], axis=0)
        if _min_image_dist(mol, others, cell, (1, 1, 0)).min() < 1.5:
            continue
        h_atoms = np.concatenate([h_atoms, mol], axis=0)
        placed += 1
    pos = np.concatenate([pos, h_atoms], axis=0)
    species = np.asarray(species + [H] * len(h_atoms), dtype=np.int32)
    pos = _wrap(pos, cell, (1, 1, 0))
    return Structure(pos, species, cell, (1, 1, 0), "tiny-pt111-h2-44")


def _wrap(pos, cell, pbc):
    frac = pos @ np.linalg.inv(cell)
    for d in range(3):
        if pbc[d]:
            frac[:, d] -= np.floor(frac[:, d])
    return frac @ cell


def big_slab(seed: int = 1, nx: int = 256, n_rows: int = 256, n_layers: int = 32,
             n_h2: int = 16384, gas_lo: float = 3.0, gas_hi: float = 33.0,
             sigma_disp: float = 0.05, vacuum: float = 40.0) -> Structure:
    """The 2.1M-atom MD workload: 256 x 256 atoms per layer x 32 layers of
    Pt(111) (2,097,152 Pt) plus n_h2 H2 molecules in the gas above it.

    H2 centres are placed by stratified jitter: the gas box (full x/y extent,
    z from gas_lo to gas_hi above the top layer) is cut into n_h2 equal cells
    and each cell receives one molecule whose centre is uniform inside the
    cell shrunk by 0.75 A + half a bond on every face, so any two atoms of
    different molecules are at least 1.5 A apart.  Orientations are uniform.
    """
    rng = np.random.default_rng(seed)
    pos, cell, z_top = pt111_ortho_slab(nx, n_rows, n_layers, vacuum=vacuum)
    pos = pos + rng.normal(scale=sigma_disp, size=pos.shape)
    # grid of gas cells: choose (gx, gy, gz) with gx*gy*gz == n_h2
    gz = 4
    while n_h2 % gz:
        gz -= 1
    rest = n_h2 // gz
    gx = int(round(math.sqrt(rest * cell[0, 0] / cell[1, 1])))
    while rest % gx:
        gx -= 1
    gy = rest // gx
    lx, ly, lz = cell[0, 0] / gx, cell[1, 1] / gy, (gas_hi - gas_lo) / gz
    margin = 0.75 + 0.5 * H2_BOND
    assert min(lx, ly, lz) > 2 * margin
    ix, iy, iz = np.meshgrid(np.arange(gx), np.arange(gy), np.arange(gz), indexing="ij")
    lo = np.stack([ix.ravel() * lx, iy.ravel() * ly, z_top + gas_lo + iz.ravel() * lz], axis=1)
    span = np.array([lx, ly, lz]) - 2 * margin
    centres = lo + margin + rng.uniform(size=lo.shape) * span
    u = _random_unit(rng, len(centres))
    h = np.empty((2 * len(centres), 3))
    h[0::2] = centres + 0.5 * H2_BOND * u
    h[1::2] = centres - 0.5 * H2_BOND * u
    pos = np.concatenate([pos, h], axis=0)
    species = np.concatenate([np.zeros(len(pos) - len(h), np.int32), np.ones(len(h), np.int32)])
    pos = _wrap(pos, cell, (1, 1, 0))
    return Structure(pos, species, cell, (1, 1, 0),
                     f"pt111-{nx}x{n_rows}x{n_layers}+{n_h2}h2")


def slab_with_adsorbed_h(rng: np.random.Generator, n: int, n_layers: int, coverage: float,
                         sigma_disp: float = 0.1, vacuum: float = 15.0) -> Structure:
    """n x n hexagonal Pt(111) slab with H at a random `coverage` fraction of
    the fcc-hollow sites, 0.9 A above the top layer; Gaussian displacements."""
    pos, cell, z_top = pt111_hex_slab(n, n, n_layers, vacuum=vacuum)
    # fcc hollow sites of the top layer sit over the third layer below, i.e.
    # at the stacking offset of layer (n_layers) in the ABC sequence
    u1 = np.array([D_NN, 0.0, 0.0])
    u2 = np.array([D_NN / 2.0, D_NN * math.sqrt(3.0) / 2.0, 0.0])
    off = _layer_offset(n_layers) + np.array([0.0, 0.0, z_top + 0.9])
    sites = np.array([i * u1 + j * u2 + off for i in range(n) for j in range(n)])
    n_h = int(round(coverage * n * n))
    pick = rng.choice(len(sites), size=n_h, replace=False) if n_h else np.zeros(0, int)
    h = sites[np.sort(pick)]
    allpos = np.concatenate([pos, h], axis=0)
    allpos = allpos + rng.normal(scale=sigma_disp, size=allpos.shape)
    species = np.concatenate([np.zeros(len(pos), np.int32), np.ones(len(h), np.int32)])
    allpos = _wrap(allpos, cell, (1, 1, 0))
    return Structure(allpos, species, cell, (1, 1, 0), f"pt111-{n}x{n}x{n_layers}+{n_h}h")


def slab_batch(seed: int = 3, n_slabs: int = 256, lo: int = 200, hi: int = 600):
    """Batch of periodic Pt(111)+H slabs with 200-600 atoms each: layers
    uniform in 3..6, lateral n x n with n in 5..10 chosen so the total falls
    in [lo, hi], H coverage uniform in [0, 1] ML, displacements 0.1 A."""
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < n_slabs:
        layers = int(rng.integers(3, 7))
        cov = float(rng.uniform(0.0, 1.0))
        ok = [n for n in range(5, 11) if lo <= n * n * layers + round(cov * n * n) <= hi]
        if not ok:
            continue
        n = int(rng.choice(ok))
        out.append(slab_with_adsorbed_h(rng, n, layers, cov))
    return out


def serving_structure(rng: np.random.Generator, n_target: int) -> Structure:
    """A Pt(111)+H2 structure of roughly n_target atoms (at least 32): an
    orthogonal slab of 4-8 layers plus about 1.5 % of the atoms as H2 gas."""
    n_layers = int(rng.integers(4, 9))
    per_layer = max(8, int(round(n_target * 0.985 / n_layers)))
    n_rows = max(4, 2 * int(round(math.sqrt(per_layer / 2.0 / 1.15))))
    nx = max(4, int(round(per_layer / n_rows)))
    n_pt = nx * n_rows * n_layers
    n_h2 = max(1, int(round((n_target - n_pt) / 2)))
    pos, cell, z_top = pt111_ortho_slab(nx, n_rows, n_layers, vacuum=25.0)
    pos = pos + rng.normal(scale=0.05, size=pos.shape)
    # H2 in the gas layer 3-13 A above the top layer by rejection (small counts)
    area = cell[0, 0] * cell[1, 1]
    h = np.zeros((0, 3))
    tries = 0
    while len(h) < 2 * n_h2 and tries < 50 * n_h2:
        tries += 1
        c = np.array([rng.uniform(0, cell[0, 0]), rng.uniform(0, cell[1, 1]),
                      z_top + rng.uniform(3.0, 3.0 + max(10.0, 2 * n_h2 * 30.0 / area))])
        u = _random_unit(rng, 1)[0]
        mol = np.stack([c + 0.5 * H2_BOND * u, c - 0.5 * H2_BOND * u])
        if len(h):
            dd = mol[:, None, :2] - h[None, :, :2]
            dd[..., 0] -= np.round(dd[..., 0] / cell[0, 0]) * cell[0, 0]
            dd[..., 1] -= np.round(dd[..., 1] / cell[1, 1]) * cell[1, 1]
            dist = np.sqrt((dd ** 2).sum(-1) + (mol[:, None, 2] - h[None, :, 2]) ** 2)
            if dist.min() < 1.5:
                continue
        h = np.concatenate([h, mol], axis=0)
    pos = np.concatenate([pos, h], axis=0)
    species = np.concatenate([np.zeros(n_pt, np.int32), np.ones(len(h), np.int32)])
    pos = _wrap(pos, cell, (1, 1, 0))
    return Structure(pos, species, cell, (1, 1, 0), f"serve-{len(pos)}")


def maxwell_velocities(species: np.ndarray, temperature: float, seed: int) -> np.ndarray:
    """Maxwell-Boltzmann velocities (A/ps) at `temperature` K with the
    centre-of-mass momentum removed.  Returns [n, 4] float32 (vx, vy, vz, 0)."""
    rng = np.random.default_rng(seed)
    m = np.array([MASS[int(s)] for s in range(2)])[species]
    scale = np.sqrt(KB_EV * temperature / m * FTM2V)
    v = rng.normal(size=(len(species), 3)) * scale[:, None]
    p = (v * m[:, None]).sum(0)
    v -= p / m.sum()
    out = np.zeros((len(species), 4), np.float32)
    out[:, :3] = v
    return out


def descriptor_dims(n_species: int, n_max: int, l_max: int):
    """(full, single-species) B2 descriptor dimensions: a <= b over the
    S*N radial channels, times (l_max + 1)."""
    c = n_species * n_max
    return c * (c + 1) // 2 * (l_max + 1), n_max * (n_max + 1) // 2 * (l_max + 1)


def random_symmetric(d: int, seed: int, kind: str, sigma_log10_min: float = -4.0) -> np.ndarray:
    """Seeded random symmetric d x d matrix (float64).

    kind == "beta":  eigenvalues U[-1, 1], rescaled so the spectral norm is 1.
    kind == "sigma": eigenvalues log-uniform in [10^sigma_log10_min, 1]
                     (positive definite; the default range is [1e-4, 1]).
    """
    rng = np.random.default_rng(seed)
    g = rng.normal(size=(d, d))
    q, r = np.linalg.qr(g)
    q = q * np.sign(np.diag(r))[None, :]          # Haar-distributed orthogonal
    if kind == "beta":
        lam = rng.uniform(-1.0, 1.0, size=d)
        lam = lam / np.abs(lam).max()
    elif kind == "sigma":
        lam = 10.0 ** rng.uniform(sigma_log10_min, 0.0, size=d)
    else:
        raise ValueError(kind)
    m = (q * lam[None, :]) @ q.T
    return 0.5 * (m + m.T)


def random_model(n_species: int = 2, n_max: int = 8, l_max: int = 3,
                 beta_seed: int = 1001, sigma_seed: int = 2001, sigma_log10_min: float = -4.0):
    """beta[s], Sigma[s] for each species s (float64, [S, d, d]); seeds are
    beta_seed + s and sigma_seed + s; Sigma's eigenvalues are log-uniform in
    [10^sigma_log10_min, 1]."""
    d, _ = descriptor_dims(n_species, n_max, l_max)
    beta = np.stack([random_symmetric(d, beta_seed + s, "beta") for s in range(n_species)])
    sigma = np.stack([random_symmetric(d, sigma_seed + s, "sigma", sigma_log10_min) for s in range(n_species)])
    return beta, sigma
