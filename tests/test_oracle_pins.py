"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these re-types the oracle's formulas: each compares it with a closed
form, a library routine, an invariance, brute force, or a finite difference.
"""
import math

import numpy as np
import pytest

import oracle as O
from oracle import sgp
from paper_2204_12573_gb300 import synth

H8 = O.Hyper(n_species=2, n_max=8, l_max=3, r_cut=4.5)


def _tiny():
    s = synth.tiny_system(0)
    pos = synth.f32_exact_f64(synth.as_f32_positions(s.pos))
    return s, pos


def _model(h=H8):
    return synth.random_model(h.n_species, h.n_max, h.l_max)


def _cluster(seed=5, n=14, species=None):
    """An isolated cluster (no periodicity) of n atoms with separations > 1.8 A."""
    rng = np.random.default_rng(seed)
    pts = []
    while len(pts) < n:
        p = rng.uniform(-3.5, 3.5, size=3)
        if all(np.linalg.norm(p - q) > 1.8 for q in pts):
            pts.append(p)
    pos = np.array(pts)
    sp = rng.integers(0, 2, size=n).astype(np.int32) if species is None else species
    cell = np.diag([30.0, 30.0, 30.0])
    return pos, sp, cell, (0, 0, 0)


# ---------------------------------------------------------------- Y_lm pins

def _legendre(l, x):
    c = np.zeros(l + 1)
    c[l] = 1.0
    return np.polynomial.legendre.legval(x, c)


def test_ylm_addition_theorem():
    """sum_m Y_lm(u) Y_lm(v) = (2l+1)/(4 pi) P_l(u.v)  (closed form)."""
    rng = np.random.default_rng(0)
    for _ in range(50):
        u, v = rng.normal(size=(2, 3))
        u /= np.linalg.norm(u)
        v /= np.linalg.norm(v)
        Yu, Yv = O.ylm(3, u), O.ylm(3, v)
        for l in range(4):
            sl = slice(l * l, (l + 1) ** 2)
            lhs = float(Yu[sl] @ Yv[sl])
            rhs = (2 * l + 1) / (4 * math.pi) * _legendre(l, float(u @ v))
            assert abs(lhs - rhs) < 1e-14


def test_ylm_orthonormal_by_quadrature():
    """Gauss-Legendre in cos(theta) x uniform phi integrates degree <= 6 exactly."""
    xg, wg = np.polynomial.legendre.leggauss(8)
    nphi = 16
    phis = 2 * math.pi * np.arange(nphi) / nphi
    G = np.zeros((16, 16))
    for x, w in zip(xg, wg):
        st = math.sqrt(1 - x * x)
        for ph in phis:
            Y = O.ylm(3, np.array([st * math.cos(ph), st * math.sin(ph), x]))
            G += w * (2 * math.pi / nphi) * np.outer(Y, Y)
    assert np.abs(G - np.eye(16)).max() < 1e-13


def test_ylm_matches_scipy_real_form():
    """Real harmonics built from scipy's complex Y_l^m, up to one sign per (l, m)."""
    sp = pytest.importorskip("scipy.special")
    if not hasattr(sp, "sph_harm_y"):
        pytest.skip("scipy without sph_harm_y")
    rng = np.random.default_rng(1)
    pts = rng.normal(size=(20, 3))
    pts /= np.linalg.norm(pts, axis=1, keepdims=True)
    ours = np.array([O.ylm(3, p) for p in pts])
    theta = np.arccos(pts[:, 2])
    phi = np.arctan2(pts[:, 1], pts[:, 0])
    for l in range(4):
        for m in range(-l, l + 1):
            c = sp.sph_harm_y(l, abs(m), theta, phi)
            if m > 0:
                ref = math.sqrt(2) * c.real
            elif m < 0:
                ref = math.sqrt(2) * c.imag
            else:
                ref = c.real
            col = ours[:, l * l + m + l]
            sgn = np.sign(col @ ref)
            assert np.abs(col - sgn * ref).max() < 1e-13, (l, m)


# ---------------------------------------------------------------- basis pins

def test_basis_gradient_matches_central_difference():
    """Complex-step gradients of the basis vs FP64 central differences."""
    rng = np.random.default_rng(2)
    for _ in range(10):
        r = rng.normal(size=3)
        r *= rng.uniform(1.0, 4.3) / np.linalg.norm(r)
        _, dphi = O.basis_point(H8, r)
        h = 1e-6
        for c in range(3):
            e = np.zeros(3)
            e[c] = h
            fd = (O.basis_point(H8, r + e)[0] - O.basis_point(H8, r - e)[0]) / (2 * h)
            assert np.abs(fd - dphi[:, :, c]).max() < 1e-7


def test_basis_vanishes_with_zero_slope_at_cutoff():
    r = np.array([0.3, -0.2, 1.0])
    r = r / np.linalg.norm(r) * (H8.r_cut - 1e-7)
    phi, dphi = O.basis_point(H8, r)
    assert np.abs(phi).max() < 1e-12 and np.abs(dphi).max() < 1e-5
    phi, dphi = O.basis_point(H8, r / np.linalg.norm(r) * (H8.r_cut + 1e-3))
    assert not phi.any() and not dphi.any()


# ---------------------------------------------------------------- neighbours

def _numpy_brute_pairs(pos, cell, pbc, rc):
    n = len(pos)
    K = [3 if p else 0 for p in pbc]
    rows = []
    for sx in range(-K[0], K[0] + 1):
        for sy in range(-K[1], K[1] + 1):
            for sz in range(-K[2], K[2] + 1):
                t = np.array([sx, sy, sz]) @ cell
                d = pos[None, :, :] + t - pos[:, None, :]
                r2 = (d ** 2).sum(-1)
                ii, jj = np.nonzero(r2 < rc * rc)
                for i, j in zip(ii, jj):
                    if i == j and sx == sy == sz == 0:
                        continue
                    rows.append((i, j, sx, sy, sz))
    rows.sort()
    return np.array(rows, np.int32).reshape(-1, 5)


@pytest.mark.parametrize("rc", [4.5, 5.0])
def test_neighbors_three_ways_agree(rc):
    s, pos = _tiny()
    ref = _numpy_brute_pairs(pos, s.cell, s.pbc, rc)
    assert np.array_equal(O.neighbors(pos, s.cell, s.pbc, rc, method="brute"), ref)
    assert np.array_equal(O.neighbors(pos, s.cell, s.pbc, rc, method="cells"), ref)


def test_neighbors_cells_on_slab_batch_member():
    s = synth.slab_batch(seed=3, n_slabs=2)[1]
    pos = synth.f32_exact_f64(synth.as_f32_positions(s.pos))
    a = O.neighbors(pos, s.cell, s.pbc, 5.0, method="brute")
    b = O.neighbors(pos, s.cell, s.pbc, 5.0, method="cells")
    assert np.array_equal(a, b)


@pytest.mark.parametrize("rc,count", [(4.5, 18), (5.0, 42)])
def test_fcc_bulk_neighbor_counts(rc, count):
    """Perfect FCC Pt: 12 + 6 neighbours within 4.5 A, +24 more within 5.0 A."""
    a = synth.A_PT
    basis = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]]) * a
    g = np.array([[i, j, k] for i in range(3) for j in range(3) for k in range(3)]) * a
    pos = (g[:, None, :] + basis[None, :, :]).reshape(-1, 3)
    cell = np.eye(3) * 3 * a
    pairs = O.neighbors(pos, cell, (1, 1, 1), rc, method="cells")
    cnt = np.bincount(pairs[:, 0], minlength=len(pos))
    assert (cnt == count).all()


# ---------------------------------------------------------------- descriptor

def test_descriptor_dimension_matches_paper():
    """Sec. V-B: 420 components for the two-species model, 112 when only one
    species is present; with a <= b over S*N channels times (L+1) this holds
    for N = 7, L = 3."""
    d_full, d_single = synth.descriptor_dims(2, 7, 3)
    golden = dict(line.split("=") for line in open(
        __file__.replace("test_oracle_pins.py", "golden/descriptor_dims.txt")).read().split()
        if "=" in line)
    assert d_full == int(golden["full"]) and d_single == int(golden["single"])
    assert O.Hyper(2, 7, 3).d == d_full


def _b2_closed_form(h, rvecs, sps):
    """B_{ab,l} = (2l+1)/(4 pi) sum_{j,k} g_a(r_j) g_b(r_k) P_l(rhat_j . rhat_k),
    g_a(r) = [s = s_a] T_n(2r/rc - 1)(rc - r)^2; bypasses Y_lm entirely."""
    C = h.n_channels
    r = np.linalg.norm(rvecs, axis=1)
    keep = r < h.r_cut
    rvecs, r, sps = rvecs[keep], r[keep], sps[keep]
    x = 2 * r / h.r_cut - 1
    T = np.polynomial.chebyshev.chebvander(x, h.n_max - 1)         # [m, N]
    g = np.zeros((len(r), C))
    for s in range(h.n_species):
        g[sps == s, s * h.n_max:(s + 1) * h.n_max] = (T * ((h.r_cut - r) ** 2)[:, None])[sps == s]
    u = rvecs / r[:, None]
    cosm = np.clip(u @ u.T, -1, 1)
    out = []
    for a in range(C):
        for b in range(a, C):
            for l in range(h.l_max + 1):
                out.append((2 * l + 1) / (4 * math.pi) * g[:, a] @ _legendre(l, cosm) @ g[:, b])
    return np.array(out)


def test_b2_matches_closed_form():
    s, pos = _tiny()
    beta, sigma = _model()
    pairs = O.neighbors(pos, s.cell, s.pbc, 5.0)
    o = O.evaluate(H8, pos, s.species, s.cell, pairs, beta, sigma, want_forces=False)
    for i in [0, 17, 35, 36, 43]:
        sel = pairs[:, 0] == i
        rv = o["rij"][sel]
        ref = _b2_closed_form(H8, rv, s.species[pairs[sel, 1]])
        assert np.abs(o["B"][i] - ref).max() <= 1e-12 * np.abs(ref).max()
        assert abs(o["norm"][i] - np.linalg.norm(ref)) <= 1e-12 * np.linalg.norm(ref)


def test_single_neighbor_on_z_axis():
    """One neighbour at distance r on the z axis: B_{ab,l} = g_a g_b (2l+1)/(4 pi)."""
    h = H8
    r = 2.7
    pos = np.array([[0.0, 0.0, 0.0], [0.0, 0.0, r]])
    sp = np.array([0, 1], np.int32)
    cell = np.diag([20.0, 20.0, 20.0])
    beta, sigma = _model()
    pairs = O.neighbors(pos, cell, (0, 0, 0), 5.0)
    o = O.evaluate(h, pos, sp, cell, pairs, beta, sigma, want_forces=False)
    x = 2 * r / h.r_cut - 1
    T = np.polynomial.chebyshev.chebvander(np.array([x]), h.n_max - 1)[0] * (h.r_cut - r) ** 2
    g = np.zeros(h.n_channels)
    g[h.n_max:] = T                       # the neighbour of atom 0 is H (species 1)
    C = h.n_channels
    ref = [g[a] * g[b] * (2 * l + 1) / (4 * math.pi)
           for a in range(C) for b in range(a, C) for l in range(h.l_max + 1)]
    assert np.abs(o["B"][0] - np.array(ref)).max() < 1e-12 * np.abs(ref).max()


def _rotation(seed):
    rng = np.random.default_rng(seed)
    q, r = np.linalg.qr(rng.normal(size=(3, 3)))
    q = q * np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def test_invariance_rotation_translation_permutation():
    pos, sp, cell, pbc = _cluster()
    beta, sigma = _model()
    ref = O.energy_forces(H8, pos, sp, cell, pbc, beta, sigma)
    R = _rotation(7)
    rot = O.energy_forces(H8, pos @ R.T, sp, cell, pbc, beta, sigma)
    assert np.abs(rot["dhat"] - ref["dhat"]).max() < 1e-12
    assert np.abs(rot["E"] - ref["E"]).max() < 1e-12
    assert np.abs(rot["V"] - ref["V"]).max() < 1e-12
    assert np.abs(rot["F"] - ref["F"] @ R.T).max() < 1e-11      # forces rotate
    tr = O.energy_forces(H8, pos + np.array([0.7, -1.3, 2.1]), sp, cell, pbc, beta, sigma)
    assert np.abs(tr["E"] - ref["E"]).max() < 1e-12
    assert np.abs(tr["F"] - ref["F"]).max() < 1e-11
    perm = np.random.default_rng(3).permutation(len(pos))
    pm = O.energy_forces(H8, pos[perm], sp[perm], cell, pbc, beta, sigma)
    assert np.abs(pm["E"] - ref["E"][perm]).max() < 1e-12
    assert np.abs(pm["F"] - ref["F"][perm]).max() < 1e-11


def test_periodic_translation_with_wrapping():
    s, pos = _tiny()
    beta, sigma = _model()
    ref = O.energy_forces(H8, pos, s.species, s.cell, s.pbc, beta, sigma, skin=0.5)
    moved = synth._wrap(pos + np.array([1.9, -3.3, 0.4]), s.cell, s.pbc)
    mv = O.energy_forces(H8, moved, s.species, s.cell, s.pbc, beta, sigma, skin=0.5)
    assert np.abs(mv["E"] - ref["E"]).max() < 1e-12
    assert np.abs(mv["F"] - ref["F"]).max() < 1e-11
    assert np.abs(mv["W"] - ref["W"]).max() < 1e-11


# ---------------------------------------------------------------- quadratic forms

def test_identity_beta_gives_constant_energy_and_zero_force():
    s, pos = _tiny()
    d = H8.d
    beta = np.stack([2.5 * np.eye(d)] * 2)
    sigma = np.stack([np.eye(d)] * 2)
    o = O.energy_forces(H8, pos, s.species, s.cell, s.pbc, beta, sigma)
    assert np.abs(o["E"] - 2.5).max() < 1e-13
    assert np.abs(o["V"] - 1.0).max() < 1e-13
    assert np.abs(o["F"]).max() < 1e-12


def test_rank_one_sigma():
    s, pos = _tiny()
    beta, _ = _model()
    u = np.random.default_rng(9).normal(size=H8.d)
    sigma = np.stack([np.outer(u, u)] * 2)
    o = O.energy_forces(H8, pos, s.species, s.cell, s.pbc, beta, sigma)
    assert np.abs(o["V"] - (o["dhat"] @ u) ** 2).max() < 1e-12


def test_energy_linear_in_beta():
    """E is linear in beta: E(beta + eps D) - E(beta) = eps d^T D d per atom."""
    s, pos = _tiny()
    beta, sigma = _model()
    D = synth.random_symmetric(H8.d, 77, "beta")
    o0 = O.energy_forces(H8, pos, s.species, s.cell, s.pbc, beta, sigma)
    b1 = beta.copy()
    b1[0] += 0.3 * D
    o1 = O.energy_forces(H8, pos, s.species, s.cell, s.pbc, b1, sigma)
    dh = o0["dhat"]
    pred = np.where(s.species == 0, 0.3 * np.einsum("ij,jk,ik->i", dh, D, dh), 0.0)
    assert np.abs(o1["E"] - o0["E"] - pred).max() < 1e-13


def test_mapping_is_lossless():
    """Eq. 1 / Eq. 2 summed over a sparse set equal the mapped quadratic forms."""
    s, pos = _tiny()
    rng = np.random.default_rng(11)
    o = O.energy_forces(H8, pos, s.species, s.cell, s.pbc, *_model())
    D_S = o["dhat"][rng.choice(len(pos), 12, replace=False)]
    D_S = D_S + 0.05 * rng.normal(size=D_S.shape)
    D_S /= np.linalg.norm(D_S, axis=1, keepdims=True)
    alpha = rng.normal(size=len(D_S))
    sig2 = 1.7
    K_SS = D_S @ D_S.T + 1e-3 * np.eye(len(D_S))
    beta = sgp.mapped_beta(D_S, alpha, sig2)
    gamma = sgp.mapped_gamma(D_S, K_SS, sig2)
    d = o["dhat"]
    assert np.abs(sgp.quad(d, beta) - sgp.sgp_mean(d, D_S, alpha, sig2)).max() < 1e-10
    assert np.abs(sgp.quad(d, gamma) - sgp.sgp_variance(d, D_S, K_SS, sig2)).max() < 1e-10
    # and the oracle's own quadratic forms agree with the unmapped sums
    om = O.energy_forces(H8, pos, s.species, s.cell, s.pbc, np.stack([beta] * 2),
                         np.stack([gamma] * 2))
    assert np.abs(om["E"] - sgp.sgp_mean(d, D_S, alpha, sig2)).max() < 1e-10
    assert np.abs(om["V"] - sgp.sgp_variance(d, D_S, K_SS, sig2)).max() < 1e-10


# ---------------------------------------------------------------- forces & virial

def test_forces_equal_minus_central_difference():
    """F = -(E_tot(x + h) - E_tot(x - h)) / 2h with h = 1e-3 A, FP64 (error O(h^2))."""
    s, pos = _tiny()
    beta, sigma = _model()
    o = O.energy_forces(H8, pos, s.species, s.cell, s.pbc, beta, sigma)
    h = 1e-3
    rng = np.random.default_rng(4)
    for k in list(rng.choice(36, 4, replace=False)) + [36, 40, 43]:
        for c in range(3):
            p1, p2 = pos.copy(), pos.copy()
            p1[k, c] += h
            p2[k, c] -= h
            e1 = O.energy_forces(H8, p1, s.species, s.cell, s.pbc, beta, sigma)["E_tot"]
            e2 = O.energy_forces(H8, p2, s.species, s.cell, s.pbc, beta, sigma)["E_tot"]
            assert abs(-(e1 - e2) / (2 * h) - o["F"][k, c]) < 2e-6


def test_net_force_zero():
    s, pos = _tiny()
    o = O.energy_forces(H8, pos, s.species, s.cell, s.pbc, *_model())
    assert np.abs(o["F"].sum(0)).max() < 1e-12


def test_virial_equals_strain_derivative():
    """W_ab = -dE/d eps_ba for a homogeneous strain of cell and positions."""
    s, pos = _tiny()
    beta, sigma = _model()
    o = O.energy_forces(H8, pos, s.species, s.cell, s.pbc, beta, sigma)
    h = 1e-5
    for a in range(3):
        for b in range(3):
            vals = []
            for sgn in (1, -1):
                eps = np.eye(3)
                eps[b, a] += sgn * h
                p = pos @ eps.T
                cl = s.cell @ eps.T
                vals.append(O.energy_forces(H8, p, s.species, cl, s.pbc, beta, sigma)["E_tot"])
            assert abs(-(vals[0] - vals[1]) / (2 * h) - o["W"][a, b]) < 1e-7
    assert np.abs(o["W"] - o["W"].T).max() < 1e-12


def test_forces_subset_matches_full():
    s = synth.slab_batch(seed=3, n_slabs=1)[0]
    pos = synth.f32_exact_f64(synth.as_f32_positions(s.pos))
    beta, sigma = _model()
    full = O.energy_forces(H8, pos, s.species, s.cell, s.pbc, beta, sigma, skin=0.5)
    atoms = np.array([0, 5, len(pos) - 1])
    sub = O.forces_subset(H8, pos, s.species, s.cell, s.pbc, beta, sigma, atoms, skin=0.5)
    assert np.abs(sub["F"] - full["F"][atoms]).max() < 1e-12
    assert np.abs(sub["E"] - full["E"][atoms]).max() < 1e-14


def test_single_species_environment_has_zero_cross_blocks():
    """Sec. V-B compaction premise: with neighbours of one species only, every
    descriptor component that involves the other species' channels is zero."""
    s, pos = _tiny()
    o = O.energy_forces(H8, pos, s.species, s.cell, s.pbc, *_model())
    pairs = O.neighbors(pos, s.cell, s.pbc, H8.r_cut)
    C, N, L1 = H8.n_channels, H8.n_max, H8.l_max + 1
    idx = [(a, b) for a in range(C) for b in range(a, C)]
    for i in range(len(pos)):
        nb_sp = set(s.species[pairs[pairs[:, 0] == i, 1]].tolist())
        if len(nb_sp) != 1:
            continue
        t = nb_sp.pop()
        for k, (a, b) in enumerate(idx):
            inside = (a // N == t) and (b // N == t)
            if not inside:
                assert not o["B"][i, k * L1:(k + 1) * L1].any()


def test_isolated_atom_reads_as_zero():
    pos = np.array([[0.0, 0.0, 0.0], [0.0, 0.0, 10.0], [0.0, 1.5, 10.0]])
    sp = np.array([0, 0, 1], np.int32)
    cell = np.diag([30.0, 30.0, 30.0])
    o = O.energy_forces(H8, pos, sp, cell, (0, 0, 0), *_model())
    assert o["norm"][0] == 0 and o["E"][0] == 0 and o["V"][0] == 0
    assert not o["F"][0].any()
