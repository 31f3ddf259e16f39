"""The seeded synthetic inputs against the recipe they stand for: H2 gas over
a Pt(111) slab (Sec. VI-A) at the benchmark sizes, Maxwell velocities, and
model matrices with the stated spectra.  Each check compares the generated
data with a fact of the recipe (counts, lattice, bond length, heights,
separations, temperature, eigenvalues), not with the generator's code."""
import math

import numpy as np
import pytest

from paper_2204_12573_gb300 import synth

D_NN = 3.92 / math.sqrt(2.0)        # Pt(111) in-plane spacing (A)
DZ = 3.92 / math.sqrt(3.0)          # (111) interlayer spacing (A)
KB = 8.617333262e-5                  # eV/K
AMU_A2_PS2_IN_EV = 1.0364269e-4      # 1 amu A^2/ps^2 in eV


@pytest.fixture(scope="module")
def slab():
    return synth.big_slab(seed=1)


def _min_image(d, cell):
    """Minimum-image difference vectors for an orthogonal cell periodic in x, y."""
    d = d.copy()
    for k in range(2):
        d[:, k] -= np.round(d[:, k] / cell[k, k]) * cell[k, k]
    return d


def test_benchmark_slab_counts_cell_and_periodicity(slab):
    assert slab.n_atoms == 2_129_920
    assert int((slab.species == 0).sum()) == 256 * 256 * 32
    assert int((slab.species == 1).sum()) == 2 * 16384
    assert tuple(slab.pbc) == (1, 1, 0)
    cell = slab.cell
    assert np.count_nonzero(cell - np.diag(np.diag(cell))) == 0        # orthogonal
    assert cell[0, 0] == pytest.approx(256 * D_NN, rel=1e-12)           # 709.6 A
    assert cell[1, 1] == pytest.approx(256 * D_NN * math.sqrt(3) / 2, rel=1e-12)   # 614.6 A
    xy = slab.pos[:, :2]
    assert (xy >= 0).all() and (xy[:, 0] < cell[0, 0]).all() and (xy[:, 1] < cell[1, 1]).all()


def test_benchmark_slab_layers_and_nearest_neighbours(slab):
    pt = slab.pos[slab.species == 0]
    # 32 layers of 65,536 atoms, (111) spacing apart (displacements sigma = 0.05 A)
    layer = np.round((pt[:, 2] - pt[:, 2].min()) / DZ).astype(int)
    counts = np.bincount(layer)
    assert len(counts) == 32 and (counts == 256 * 256).all()
    dz = pt[:, 2] - (pt[:, 2].min() + layer * DZ)
    assert abs(dz.std() - 0.05) < 0.002
    # nearest neighbours inside a layer: the hexagonal spacing a / sqrt(2)
    rng = np.random.default_rng(0)
    top = pt[layer == 31]
    pick = top[rng.choice(len(top), 50, replace=False)]
    for p in pick:
        d = np.linalg.norm(_min_image(top - p, slab.cell)[:, :2], axis=1)
        d = np.sort(d)[1:7]                                  # six in-plane neighbours
        assert np.abs(d - D_NN).max() < 0.35


def test_benchmark_h2_gas(slab):
    h = slab.pos[slab.species == 1]
    a, b = h[0::2], h[1::2]
    bond = np.linalg.norm(_min_image(a - b, slab.cell), axis=1)
    assert np.abs(bond - 0.74).max() < 1e-9
    pt_z = slab.pos[slab.species == 0, 2]
    z_top = pt_z.min() + 31 * DZ
    centre_z = 0.5 * (a[:, 2] + b[:, 2])
    assert centre_z.min() >= z_top + 3.0 - 1e-9 and centre_z.max() <= z_top + 33.0 + 1e-9
    # atoms of different molecules at least 1.5 A apart (periodic in x and y)
    scipy_spatial = pytest.importorskip("scipy.spatial")
    box = np.array([slab.cell[0, 0], slab.cell[1, 1], 1e6])
    pts = h.copy()
    pts[:, 2] -= pts[:, 2].min()
    tree = scipy_spatial.cKDTree(pts, boxsize=box)
    pairs = tree.query_pairs(1.5, output_type="ndarray")
    assert all(i // 2 == j // 2 for i, j in pairs)            # only the two atoms of a molecule


def test_benchmark_velocities_are_maxwell_at_300_k(slab):
    v = synth.maxwell_velocities(slab.species, 300.0, seed=1)[:, :3].astype(np.float64)
    m = np.where(slab.species == 0, 195.084, 1.008)
    p = (m[:, None] * v).sum(0)
    assert np.abs(p).max() < 1e-6 * (m[:, None] * np.abs(v)).sum()
    ke = 0.5 * (m[:, None] * v * v).sum() * AMU_A2_PS2_IN_EV          # eV
    t = 2.0 * ke / (3.0 * len(m) * KB)
    assert abs(t - 300.0) < 1.5                                    # 2.1 M atoms: statistical spread ~0.3 K


def test_generators_are_seeded():
    a = synth.big_slab(seed=7, nx=16, n_rows=16, n_layers=4, n_h2=64)
    b = synth.big_slab(seed=7, nx=16, n_rows=16, n_layers=4, n_h2=64)
    c = synth.big_slab(seed=8, nx=16, n_rows=16, n_layers=4, n_h2=64)
    assert np.array_equal(a.pos, b.pos) and np.array_equal(a.species, b.species)
    assert not np.array_equal(a.pos, c.pos)


def test_float32_positions_are_what_both_sides_see():
    s = synth.tiny_system(0)
    p4 = synth.as_f32_positions(s.pos)
    assert p4.dtype == np.float32 and p4.shape == (s.n_atoms, 4)
    assert np.array_equal(synth.f32_exact_f64(p4), s.pos.astype(np.float32).astype(np.float64))


def test_tiny_system():
    s = synth.tiny_system(0)
    assert s.n_atoms == 44 and int((s.species == 0).sum()) == 36 and int((s.species == 1).sum()) == 8
    assert np.allclose(s.cell[0], [3 * D_NN, 0, 0]) and np.allclose(s.cell[1], [1.5 * D_NN, 1.5 * math.sqrt(3) * D_NN, 0])
    pt_z = s.pos[s.species == 0, 2]
    h = s.pos[s.species == 1]
    z_top = 3 * DZ
    assert ((h[:, 2] > z_top + 1.5 - 0.6) & (h[:, 2] < z_top + 3.0 + 0.6)).all()   # centres 1.5-3 A up, bond, jitter
    assert pt_z.max() < z_top + 0.3


def test_slab_batch_sizes_and_coverage():
    """3-6 layers of an n x n net (n = 5..10), 200-600 atoms, H coverage at
    most one per fcc-hollow site of the top layer (<= 1 ML)."""
    batch = synth.slab_batch(seed=3)
    assert len(batch) == 256
    for s in batch:
        n_pt, n_h = int((s.species == 0).sum()), int((s.species == 1).sum())
        assert 200 <= s.n_atoms <= 600
        nets = [(n, k) for n in range(5, 11) for k in range(3, 7) if n * n * k == n_pt]
        assert nets, n_pt
        assert any(n_h <= n * n for n, _ in nets)
        assert s.cell[0, 0] == pytest.approx(nets[0][0] * D_NN) or len(nets) > 1


@pytest.mark.parametrize("species", [0, 1])
def test_model_spectra(species):
    beta, sigma = synth.random_model()
    assert beta.shape == (2, 544, 544) and sigma.shape == (2, 544, 544)
    b, g = beta[species], sigma[species]
    assert np.array_equal(b, b.T) and np.array_equal(g, g.T)
    eb = np.linalg.eigvalsh(b)
    assert np.abs(eb).max() == pytest.approx(1.0, rel=1e-10)    # ||beta||_2 = 1 eV
    assert eb.min() < -0.5 and eb.max() > 0.5                    # indefinite, U[-1, 1] spectrum
    eg = np.linalg.eigvalsh(g)
    assert eg.min() > 1e-4 * (1 - 1e-8) and eg.max() <= 1.0 + 1e-10   # log-uniform in [1e-4, 1]
    # log-uniform: about a quarter of the 544 eigenvalues per decade
    per_decade = np.histogram(np.log10(eg), bins=[-4, -3, -2, -1, 0])[0]
    assert (np.abs(per_decade - 136) < 40).all()


def test_serving_sizes_are_log_uniform():
    from paper_2204_12573_gb300 import serving
    k = 4096
    n = serving.log_uniform_sizes(k)
    assert n.min() >= 32 and n.max() <= 200_000
    mean = (200_000 - 32) / math.log(200_000 / 32)               # mean of the log-uniform law, ~22.9k
    assert abs(n.mean() - mean) / mean < 0.01
    assert abs(np.median(n) - math.sqrt(32 * 200_000)) / math.sqrt(32 * 200_000) < 0.01
    lat = np.random.default_rng(0).exponential(2e6, size=1000)
    assert serving.percentile_ms(lat, 99) == pytest.approx(np.percentile(lat, 99) / 1e6)
    assert serving.percentile_ms([], 50) is None
