"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances: the plain FP32 path must give bit-exact neighbour sets, per-atom
energy error <= 1e-5 * max(|E_i|, ||beta_s||_2), force error <= 1e-4 eV/A
and variance relative error <= 1e-4; the TF32 and 3xBF16 tensor-core paths
must give forces within 1e-3 eV/A.
"""
import numpy as np
import pytest

from paper_2204_12573_gb300 import synth

from gpu_common import (F_TOL_MIXED, compare_efv, compare_mixed, decode_entries, gpu_run, oracle_run)
import oracle as O

pytestmark = pytest.mark.gpu

BETA, SIGMA = synth.random_model()


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2204_12573_gb300 import build
    build.build()


def _tiny():
    return synth.tiny_system(0)


def _slabs(k=3):
    return synth.slab_batch(seed=3, n_slabs=k)


# ------------------------------------------------------------ neighbours

def _ortho(n=3000, seed=21):
    """An orthogonal-cell Pt(111)+H2 slab (the bin stencil is pruned by box distance there)."""
    return synth.serving_structure(np.random.default_rng(seed), n)


@pytest.mark.parametrize("which", ["tiny", "slab0", "slab1", "slab2", "ortho", "ortho_small"])
def test_neighbor_sets_bit_exact(which):
    if which == "tiny":
        s = _tiny()
    elif which == "ortho":
        s = _ortho()
    elif which == "ortho_small":
        s = _ortho(200, 22)
    else:
        s = _slabs()[int(which[-1])]
    g, *_ = gpu_run(s, BETA, SIGMA, max_nbr=96)
    pos = synth.f32_exact_f64(synth.as_f32_positions(s.pos))
    ref = O.neighbors(pos, s.cell, s.pbc, 5.0, method="brute" if s.n_atoms < 100 else "cells")
    got = decode_entries(g["entries"], g["count"])
    assert got.shape == ref.shape
    assert np.array_equal(got, ref.astype(np.int64))
    # every entry carries its neighbour's species in bit 7
    e = g["entries"].cpu().numpy()
    c = g["count"].cpu().numpy()
    for i in range(len(c)):
        v = e[i, :c[i]].astype(np.int64)
        assert np.array_equal((v >> 7) & 1, s.species[v >> 8])


def _boundary_cluster():
    """A 13-atom Pt cuboctahedron (nearest neighbours 2.77 A) and an H2
    molecule, centred on a corner of a 2000 A triclinic cell periodic in x
    and y and wrapped into it: most pairs cross the periodic boundary, with
    coordinates near 0 and near 2000 A.  Forming r_j - r_i + S.cell plainly
    in FP32 loses about 6e-5 A there, far outside the descriptor tolerance."""
    a = 3.92
    pts = [np.zeros(3)]
    for i, j in ((0, 1), (0, 2), (1, 2)):
        for si in (-1, 1):
            for sj in (-1, 1):
                v = np.zeros(3)
                v[i], v[j] = si * a / 2, sj * a / 2
                pts.append(v)
    pt = np.array(pts)
    h2 = np.array([[0.37, 0.0, 4.6], [-0.37, 0.0, 4.6]])
    cell = np.array([[2000.0, 0.0, 0.0], [1000.0, 1732.0508075688772, 0.0], [0.0, 0.0, 60.0]])
    pos = np.concatenate([pt, h2]) + np.array([0.35, 0.2, 25.0])
    pos = synth._wrap(pos, cell, (1, 1, 0))
    sp = np.array([0] * 13 + [1, 1], np.int32)
    return synth.Structure(pos, sp, cell, (1, 1, 0), "boundary-cluster")


def test_large_cell_boundary_pairs():
    s = _boundary_cluster()
    assert s.pos[:, 0].max() > 1990.0          # wrapped to the far side of the cell
    g, *_ = gpu_run(s, BETA, SIGMA, want_desc=True)
    pos = synth.f32_exact_f64(synth.as_f32_positions(s.pos))
    ref = O.neighbors(pos, s.cell, s.pbc, 5.0, method="brute")
    assert np.array_equal(decode_entries(g["entries"], g["count"]), ref.astype(np.int64))
    o = oracle_run(s, BETA, SIGMA)
    assert np.abs(g["dhat"] - o["dhat"]).max() <= 2e-6
    compare_efv(g, o)


def test_rows_are_deterministic():
    s = _slabs()[0]
    g1, *_ = gpu_run(s, BETA, SIGMA)
    g2, *_ = gpu_run(s, BETA, SIGMA)
    assert np.array_equal(g1["entries"].cpu().numpy(), g2["entries"].cpu().numpy())


# ------------------------------------------------------------ descriptors

def test_descriptors_match_oracle():
    s = _tiny()
    g, *_ = gpu_run(s, BETA, SIGMA, want_desc=True)
    o = oracle_run(s, BETA, SIGMA)
    assert np.abs(g["norm"] - o["norm"]).max() <= 1e-5 * o["norm"].max()
    assert np.abs(g["dhat"] - o["dhat"]).max() <= 2e-6


def test_descriptors_compaction_zero_blocks():
    s = _slabs()[1]
    g, *_ = gpu_run(s, BETA, SIGMA, want_desc=True)
    o = oracle_run(s, BETA, SIGMA)
    assert np.abs(g["dhat"] - o["dhat"]).max() <= 2e-6


# ------------------------------------------------------------ energy / forces / variance

def test_fp32_tiny_matches_oracle():
    s = _tiny()
    g, *_ = gpu_run(s, BETA, SIGMA, precision="fp32")
    o = oracle_run(s, BETA, SIGMA)
    compare_efv(g, o)
    assert abs(g["totals"][0] - o["E_tot"]) <= 1e-5 * max(1.0, abs(o["E_tot"]))
    W = g["totals"][1:10].reshape(3, 3)
    assert np.abs(W - o["W"]).max() <= 1e-4 * max(1.0, np.abs(o["W"]).max())
    assert abs(g["totals"][10] - np.sqrt(o["V"]).max()) <= 1e-5


@pytest.mark.parametrize("k", [0, 1, 2])
def test_fp32_slabs_match_oracle(k):
    s = _slabs()[k]
    g, *_ = gpu_run(s, BETA, SIGMA, precision="fp32")
    o = oracle_run(s, BETA, SIGMA)
    compare_efv(g, o)


@pytest.mark.parametrize("precision,fused", [("tf32", None), ("bf16x3", True), ("bf16x3", False)])
def test_mixed_precision_matches_oracle(precision, fused):
    """Forces within 1e-3 eV/A; every atom's energy and variance within the
    bounds derived from the split-precision products (gpu_common).  3xBF16
    runs with the one-species atoms in the fused descriptor + tensor-core
    kernel and with separate kernels; the fused kernel must have run."""
    for s in [_tiny()] + _slabs(3):
        g, *_ = gpu_run(s, BETA, SIGMA, precision=precision, fused=fused, profile=True)
        o = oracle_run(s, BETA, SIGMA)
        compare_mixed(g, o, precision, s.species, BETA, SIGMA)
        assert (g["profile"]["fused"][1] > 0) == bool(fused)


def test_fused_and_separate_kernels_agree():
    """The fused one-species path and the separate kernels compute the same
    forms; their 3xBF16 results differ only by the epilogue's hi + lo
    descriptor (relative 2^-16) against the FP32 row."""
    s = _slabs(3)[2]
    a, *_ = gpu_run(s, BETA, SIGMA, precision="bf16x3", fused=True)
    b, *_ = gpu_run(s, BETA, SIGMA, precision="bf16x3", fused=False)
    assert np.array_equal(a["group"].cpu().numpy(), b["group"].cpu().numpy())
    assert np.abs(a["energy"] - b["energy"]).max() <= 1e-4
    assert np.abs(a["forces"] - b["forces"]).max() <= 2e-4
    assert (np.abs(a["variance"] - b["variance"]) <= 1e-4 * np.abs(b["variance"]) + 1e-5).all()


@pytest.mark.parametrize("precision", ["fp32", "bf16x3"])
def test_virial_and_total_energy_match_oracle(precision):
    """The FP64 totals against the oracle: the virial W_ab = -sum over pairs of
    (r_ij)_a (dE_i/dr_ij)_b (the stress the model predicts, Sec. V-B) and the
    total energy.  Each is a sum whose terms carry a relative error of at most
    eps, so the bound is eps times the sum of the terms' absolute values:
    eps = 1e-5 in FP32 (the per-atom energy bound), 1e-4 with the 3xBF16
    quadratic forms.  The single-system path sums the pair terms directly; the
    per-structure path of batches (compared with it in test_gpu_batch.py) sums
    per-atom virials."""
    s = _slabs(3)[1]
    g, *_ = gpu_run(s, BETA, SIGMA, precision=precision)
    o = oracle_run(s, BETA, SIGMA)
    eps = 1e-5 if precision == "fp32" else 1e-4
    abs_w = np.einsum("pa,pb->ab", np.abs(o["rij"]), np.abs(o["fpair"]))
    w = g["totals"][1:10].reshape(3, 3)
    assert np.abs(o["W"]).max() > 1e-3                       # a non-trivial virial
    assert (np.abs(w - o["W"]) <= eps * abs_w + 1e-9).all()
    assert abs(g["totals"][0] - o["E_tot"]) <= eps * np.abs(o["E"]).sum()


def test_two_species_overlap_is_bitwise_serial():
    """The one-species quadratic-form kernel launched as a programmatic
    dependent of the two-species one (the default) and launched after it give
    bitwise the same outputs: each tile is computed by one CTA either way,
    whichever CTA claims it.  Over MD steps too, with the rebuilds in between."""
    import torch
    from paper_2204_12573_gb300 import flare as F
    s = _slabs(3)[2]
    a, *_ = gpu_run(s, BETA, SIGMA, precision="bf16x3", overlap=True)
    b, *_ = gpu_run(s, BETA, SIGMA, precision="bf16x3", overlap=False)
    groups = b["group"]
    assert (groups % 3 == 0).sum() > 0 and (groups % 3 != 0).sum() > 0   # both compaction classes present
    for k in ("energy", "forces", "variance", "sigma"):
        assert np.array_equal(a[k], b[k]), k
    runs = []
    for ovl in (True, False):
        ff = F.FlareGB(precision="bf16x3")
        ff.set_model(BETA, SIGMA)
        ff.set_overlap(ovl)
        sysg = F.System.from_numpy(synth.as_f32_positions(s.pos), s.species, s.cell, s.pbc)
        vel = torch.as_tensor(synth.maxwell_velocities(s.species, 300.0, 5), device="cuda")
        nl = ff.nbrlist(s.n_atoms)
        F.build_neighbors(ff, sysg, nl)
        st = F.MDState(sysg, vel, dt=0.0005, rebuild_every=3)
        out = F.make_outputs(s.n_atoms)
        F.md_step(ff, st, nl, 8, out)
        ff.sync()
        runs.append((sysg.pos.cpu().numpy().copy(), st.vel.cpu().numpy().copy(), out["forces"].cpu().numpy().copy()))
    for x, y in zip(runs[0], runs[1]):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("precision", ["tf32", "bf16x3"])
def test_mixed_precision_other_models(precision):
    """The same bounds for other seeded models and for |beta|_2 = 2 eV (forces
    scale with beta, so this doubles the force error of the products): the
    1e-3 eV/A force bound must hold with margin, not by luck of one model."""
    s = _slabs(4)[3]
    for scale, bseed, sseed in ((1.0, 3001, 4001), (2.0, 1001, 2001), (2.0, 5001, 6001)):
        b, sg = synth.random_model(beta_seed=bseed, sigma_seed=sseed)
        b = scale * b
        g, *_ = gpu_run(s, b, sg, precision=precision)
        o = oracle_run(s, b, sg)
        compare_mixed(g, o, precision, s.species, b, sg, beta_norm=scale)


def test_compaction_on_off_agree():
    s = _slabs()[2]
    a, *_ = gpu_run(s, BETA, SIGMA, compaction=True)
    b, *_ = gpu_run(s, BETA, SIGMA, compaction=False)
    assert np.abs(a["energy"] - b["energy"]).max() <= 2e-6
    assert np.abs(a["forces"] - b["forces"]).max() <= 2e-5
    assert (b["group"].cpu().numpy() % 3 == 0).all()


def test_forces_bitwise_reproducible():
    s = _slabs()[0]
    a, *_ = gpu_run(s, BETA, SIGMA, precision="bf16x3")
    b, *_ = gpu_run(s, BETA, SIGMA, precision="bf16x3")
    assert np.array_equal(a["forces"], b["forces"])
    assert np.array_equal(a["energy"], b["energy"])


def test_net_force_zero():
    s = _slabs()[1]
    g, *_ = gpu_run(s, BETA, SIGMA)
    assert np.abs(g["forces"].astype(np.float64).sum(0)).max() <= 1e-4


def test_paper_dimensions_n7():
    """n_max = 7 reproduces the paper's 420 / 112 descriptor sizes on the GPU path."""
    s = _tiny()
    b7, s7 = synth.random_model(n_max=7)
    g, ff, *_ = gpu_run(s, b7, s7, n_max=7)
    assert (ff.d_full, ff.d_single) == (420, 112)
    o = oracle_run(s, b7, s7, n_max=7)
    compare_efv(g, o)
    # the fused one-species kernel at N = 7 (K = 112, one MMA column half of 112)
    gb, *_ = gpu_run(s, b7, s7, n_max=7, precision="bf16x3", fused=True, profile=True)
    assert gb["profile"]["fused"][1] > 0
    compare_mixed(gb, o, "bf16x3", s.species, b7, s7, d_full=420, d_single=112)


# ------------------------------------------------------------ edge cases

def test_isolated_and_empty():
    import torch
    from paper_2204_12573_gb300 import flare as F
    ff = F.FlareGB(precision="fp32")
    ff.set_model(BETA, SIGMA)
    pos = np.array([[0, 0, 0, 0], [0, 0, 10, 0], [0, 1.5, 10, 0]], np.float32)
    sp = np.array([0, 0, 1], np.int32)
    sysg = F.System.from_numpy(pos, sp, np.diag([30.0, 30.0, 30.0]), (0, 0, 0))
    nl = ff.nbrlist(3)
    F.build_neighbors(ff, sysg, nl)
    out = F.energy_forces_uncertainty(ff, sysg, nl)
    ff.sync()
    o = O.energy_forces(O.Hyper(), pos[:, :3].astype(np.float64), sp, np.diag([30.0] * 3), (0, 0, 0), BETA, SIGMA)
    assert out["energy"][0].item() == 0.0 and out["variance"][0].item() == 0.0
    assert out["totals"][11].item() == 1.0
    assert np.abs(out["forces"].cpu().numpy() - o["F"]).max() <= 1e-4
    # an empty system is accepted and leaves zero totals
    sys0 = F.System.from_numpy(np.zeros((0, 4), np.float32), np.zeros(0, np.int32), np.eye(3) * 10, (0, 0, 0))
    nl0 = ff.nbrlist(0)
    F.build_neighbors(ff, sys0, nl0)
    out0 = F.energy_forces_uncertainty(ff, sys0, nl0)
    ff.sync()
    assert out0["totals"].abs().sum().item() == 0.0
    torch.cuda.synchronize()


def test_overflow_is_reported():
    from paper_2204_12573_gb300 import flare as F
    from paper_2204_12573_gb300 import _native as N
    s = _slabs()[0]
    ff = F.FlareGB(max_nbr=32, precision="fp32")
    ff.set_model(BETA, SIGMA)
    sysg = F.System.from_numpy(synth.as_f32_positions(s.pos), s.species, s.cell, s.pbc)
    nl = ff.nbrlist(s.n_atoms)
    with pytest.raises(N.FlareError) as e:
        F.build_neighbors(ff, sysg, nl)
    assert e.value.code == N.FLR_ENBR_OVERFLOW


def test_model_required():
    from paper_2204_12573_gb300 import flare as F
    from paper_2204_12573_gb300 import _native as N
    s = _tiny()
    ff = F.FlareGB()
    sysg = F.System.from_numpy(synth.as_f32_positions(s.pos), s.species, s.cell, s.pbc)
    nl = ff.nbrlist(s.n_atoms)
    F.build_neighbors(ff, sysg, nl)
    with pytest.raises(N.FlareError) as e:
        F.energy_forces_uncertainty(ff, sysg, nl)
    assert e.value.code == N.FLR_ENOMODEL
