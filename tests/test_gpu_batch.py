"""Batched evaluation of many structures (flr_build_neighbors_batch,
flr_energy_forces_uncertainty_batch) through the C ABI.

Each structure's neighbours, descriptors and per-atom outputs depend only on
that structure (Eq. 1 sums over the atom's own environment), so the batch
must give every atom exactly the bits it gets when its structure is
evaluated alone; per-structure totals are sums in another order and agree
to rounding.  The whole 256-slab batch (200-600 atoms per slab) is checked
against the FP64 oracle with the FP32 tolerances.
"""
import dataclasses

import numpy as np
import pytest

from paper_2204_12573_gb300 import synth

from gpu_common import F_TOL_MIXED, compare_efv, decode_entries, oracle_run
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


def _mixed_structs():
    """Slabs of different sizes and cells, the 44-atom system, a cluster with
    no periodic direction and a bulk-like block periodic in all three."""
    slabs = synth.slab_batch(seed=5, n_slabs=5)
    tiny = synth.tiny_system(0)
    cluster = dataclasses.replace(tiny, pbc=(0, 0, 0), name="cluster")
    pos, cell, _ = synth.pt111_hex_slab(4, 4, 6, vacuum=synth.DZ_111)
    rng = np.random.default_rng(9)
    bulk = synth.Structure(pos + rng.normal(scale=0.05, size=pos.shape), np.zeros(len(pos), np.int32), cell,
                           (1, 1, 1), "bulk")
    bulk = dataclasses.replace(bulk, pos=synth._wrap(bulk.pos, cell, (1, 1, 1)))
    return [slabs[0], tiny, cluster, slabs[1], bulk, slabs[2], slabs[3], slabs[4]]


def _run_batch(ff, structs):
    import torch
    from paper_2204_12573_gb300 import flare as F
    b = F.Batch.from_structures(structs)
    nl = ff.nbrlist(b.n_atoms)
    F.build_neighbors_batch(ff, b, nl)
    out = F.energy_forces_uncertainty_batch(ff, b, nl)
    torch.cuda.synchronize()
    res = {k: v.cpu().numpy() for k, v in out.items()}
    res["entries"], res["count"], _ = nl.view(b.n_atoms)
    return res, b


def _run_single(ff, s):
    import torch
    from paper_2204_12573_gb300 import flare as F
    sysg = F.System.from_numpy(synth.as_f32_positions(s.pos), s.species, s.cell, s.pbc)
    nl = ff.nbrlist(s.n_atoms)
    F.build_neighbors(ff, sysg, nl)
    out = F.energy_forces_uncertainty(ff, sysg, nl)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


@pytest.mark.parametrize("precision", ["fp32", "bf16x3", "tf32"])
def test_batch_equals_each_structure_alone(precision):
    from paper_2204_12573_gb300 import flare as F
    structs = _mixed_structs()
    ff = F.FlareGB(precision=precision, max_nbr=96)
    ff.set_model(BETA, SIGMA)
    g, b = _run_batch(ff, structs)
    assert g["totals"].shape == (len(structs), 24)
    for k, s in enumerate(structs):
        lo, hi = int(b.offsets[k]), int(b.offsets[k + 1])
        a = _run_single(ff, s)
        for key in ("energy", "forces", "variance", "sigma"):
            assert np.array_equal(g[key][lo:hi], a[key]), (s.name, key)
        t, ta = g["totals"][k], a["totals"]
        assert abs(t[0] - ta[0]) <= 1e-9 * max(1.0, abs(ta[0])) + 1e-6
        assert np.abs(t[1:10] - ta[1:10]).max() <= 1e-5 * max(1.0, np.abs(ta[1:10]).max())
        assert t[10] == ta[10]
        assert t[11] == ta[11]


def test_batch_neighbors_bit_exact_per_structure():
    from paper_2204_12573_gb300 import flare as F
    structs = _mixed_structs()
    ff = F.FlareGB(precision="fp32", max_nbr=96)
    ff.set_model(BETA, SIGMA)
    g, b = _run_batch(ff, structs)
    got = decode_entries(g["entries"], g["count"])
    for k, s in enumerate(structs):
        lo, hi = int(b.offsets[k]), int(b.offsets[k + 1])
        mine = got[(got[:, 0] >= lo) & (got[:, 0] < hi)].copy()
        assert ((mine[:, 1] >= lo) & (mine[:, 1] < hi)).all(), "pair crosses a structure boundary"
        mine[:, :2] -= lo
        pos = synth.f32_exact_f64(synth.as_f32_positions(s.pos))
        ref = O.neighbors(pos, s.cell, s.pbc, 5.0, method="brute")
        assert np.array_equal(mine, ref.astype(np.int64)), s.name


@pytest.mark.slow
def test_slab_batch_256_matches_oracle():
    """All 256 slabs of 200-600 atoms in one batch, FP32, against the oracle."""
    from paper_2204_12573_gb300 import flare as F
    structs = synth.slab_batch(seed=3, n_slabs=256)
    ff = F.FlareGB(precision="fp32")
    ff.set_model(BETA, SIGMA)
    g, b = _run_batch(ff, structs)
    for k, s in enumerate(structs):
        lo, hi = int(b.offsets[k]), int(b.offsets[k + 1])
        o = oracle_run(s, BETA, SIGMA)
        compare_efv({key: g[key][lo:hi] for key in ("energy", "forces", "variance")}, o)
        assert abs(g["totals"][k, 0] - o["E_tot"]) <= 1e-5 * max(1.0, abs(o["E_tot"]))
        W = g["totals"][k, 1:10].reshape(3, 3)
        assert np.abs(W - o["W"]).max() <= 1e-4 * max(1.0, np.abs(o["W"]).max())


def test_slab_batch_mixed_precision_forces():
    from paper_2204_12573_gb300 import flare as F
    structs = synth.slab_batch(seed=3, n_slabs=24)
    ff = F.FlareGB(precision="bf16x3")
    ff.set_model(BETA, SIGMA)
    g, b = _run_batch(ff, structs)
    for k, s in enumerate(structs):
        lo, hi = int(b.offsets[k]), int(b.offsets[k + 1])
        o = oracle_run(s, BETA, SIGMA)
        assert np.abs(g["forces"][lo:hi] - o["F"]).max() <= F_TOL_MIXED


def test_batch_of_empty_and_single_atom_structures():
    import torch
    from paper_2204_12573_gb300 import flare as F
    tiny = synth.tiny_system(0)
    empty = synth.Structure(np.zeros((0, 3)), np.zeros(0, np.int32), tiny.cell, tiny.pbc, "empty")
    lone = synth.Structure(np.array([[1.0, 1.0, 5.0]]), np.array([1], np.int32), tiny.cell, (0, 0, 0), "lone")
    structs = [empty, tiny, lone, empty]
    ff = F.FlareGB(precision="fp32")
    ff.set_model(BETA, SIGMA)
    g, b = _run_batch(ff, structs)
    o = oracle_run(tiny, BETA, SIGMA)
    compare_efv({key: g[key][0:44] for key in ("energy", "forces", "variance")}, o)
    assert g["energy"][44] == 0.0 and np.all(g["forces"][44] == 0.0)
    assert g["totals"][0, 0] == 0.0 and g["totals"][3, 0] == 0.0
    assert g["totals"][2, 11] == 1.0
    torch.cuda.synchronize()
