"""Variance quadratic form (Eq. 2) when Sigma is ill-conditioned.

Sigma is built with eigenvalue 1e-6 on the span of the system's own
descriptors and eigenvalues in [0.1, 1] elsewhere, so every atom's variance
is about 1e-6 while the terms d_k (Sigma d)_k are of order 1e-1: the FP32
sum cancels.  The default mode (FLR_VAR_AUTO) must detect those atoms and
re-evaluate them in FP64 (relative error <= 1e-4 against the FP64 oracle);
the plain FP32 form ("direct") cannot; the factored form V = |L^T d|^2 avoids
the final cancellation.  Energies and forces do not depend on the mode.
"""
import numpy as np
import pytest

from paper_2204_12573_gb300 import synth

from gpu_common import gpu_run, oracle_run
import oracle as O

pytestmark = pytest.mark.gpu

BETA, SIGMA = synth.random_model()
SMALL = 1e-6


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2204_12573_gb300 import build
    build.build()


def _aligned_sigma(struct, seed=5):
    """Per species: eigenvalue SMALL on the span of that species' descriptors
    (from the oracle), log-uniform [0.1, 1] on the orthogonal complement."""
    o = oracle_run(struct, BETA, SIGMA)
    d = o["dhat"].shape[1]
    rng = np.random.default_rng(seed)
    out = []
    for sp in range(2):
        D = o["dhat"][(struct.species == sp) & (o["norm"] > 0)]
        _, s, vt = np.linalg.svd(D, full_matrices=True)
        rank = int((s > 1e-9 * s.max()).sum())
        basis = vt[:rank].T                                  # d x rank, the descriptors' span
        comp = rng.normal(size=(d, d - rank))
        comp -= basis @ (basis.T @ comp)
        comp, _ = np.linalg.qr(comp)
        Q = np.concatenate([basis, comp], axis=1)
        lam = np.concatenate([np.full(rank, SMALL), 10.0 ** rng.uniform(-1.0, 0.0, d - rank)])
        S = (Q * lam) @ Q.T
        out.append(0.5 * (S + S.T))
    return np.stack(out)


def _run(struct, sigma, precision, mode):
    import torch
    from paper_2204_12573_gb300 import flare as F
    ff = F.FlareGB(precision=precision)
    ff.set_variance_mode(mode)
    ff.set_model(BETA, sigma)
    sysg = F.System.from_numpy(synth.as_f32_positions(struct.pos), struct.species, struct.cell, struct.pbc)
    nl = ff.nbrlist(struct.n_atoms)
    F.build_neighbors(ff, sysg, nl)
    out = F.energy_forces_uncertainty(ff, sysg, nl)
    ff.sync()
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def _vrel(g, o):
    ok = o["norm"] > 0
    return float((np.abs(g["variance"][ok] - o["V"][ok]) / o["V"][ok]).max())


@pytest.mark.parametrize("precision", ["fp32", "bf16x3"])
def test_ill_conditioned_variance_fp64_path(precision):
    s = synth.tiny_system(0)
    sig = _aligned_sigma(s)
    pos = synth.f32_exact_f64(synth.as_f32_positions(s.pos))
    o = O.energy_forces(O.Hyper(), pos, s.species, s.cell, s.pbc, BETA, sig, skin=0.5)
    ok = o["norm"] > 0
    assert o["V"][ok].max() < 10 * SMALL            # the construction makes every variance tiny
    auto = _run(s, sig, precision, "auto")
    direct = _run(s, sig, precision, "direct")
    assert _vrel(auto, o) <= 1e-4
    assert auto["totals"][14] == ok.sum()           # every atom was re-evaluated in FP64
    assert direct["totals"][14] == 0
    assert _vrel(direct, o) > 1e-2                   # FP32 alone loses the variance here
    sig_ref = np.sqrt(o["V"][ok])
    assert np.abs(auto["sigma"][ok] - sig_ref).max() <= 1e-4 * sig_ref.max()
    # the mode touches only V and sigma
    assert np.array_equal(auto["energy"], direct["energy"])
    assert np.array_equal(auto["forces"], direct["forces"])


def test_factored_variance_avoids_the_final_cancellation():
    s = synth.tiny_system(0)
    sig = _aligned_sigma(s)
    pos = synth.f32_exact_f64(synth.as_f32_positions(s.pos))
    o = O.energy_forces(O.Hyper(), pos, s.species, s.cell, s.pbc, BETA, sig, skin=0.5)
    fac = _run(s, sig, "fp32", "factored")
    direct = _run(s, sig, "fp32", "direct")
    assert np.isfinite(fac["variance"]).all() and (fac["variance"] >= 0).all()
    assert _vrel(fac, o) < _vrel(direct, o)


@pytest.mark.parametrize("precision", ["fp32", "bf16x3"])
def test_well_conditioned_sigma_rarely_needs_fp64(precision):
    """Sigma with eigenvalues in [1e-4, 1]: few atoms (if any) take the FP64
    path, and where they do their variance changes only in its last digits."""
    s = synth.slab_batch(seed=3, n_slabs=1)[0]
    auto = _run(s, SIGMA, precision, "auto")
    direct = _run(s, SIGMA, precision, "direct")
    assert auto["totals"][14] <= 0.01 * s.n_atoms
    for key in ("energy", "forces"):
        assert np.array_equal(auto[key], direct[key])
    ok = direct["variance"] > 0
    assert (np.abs(auto["variance"][ok] - direct["variance"][ok]) / direct["variance"][ok]).max() <= 1e-4


def test_indefinite_sigma_is_rejected():
    from paper_2204_12573_gb300 import flare as F
    from paper_2204_12573_gb300 import _native as N
    bad = SIGMA.copy()
    bad[0] -= 2.0 * np.eye(bad.shape[1])           # eigenvalues down to -2
    ff = F.FlareGB(precision="fp32")
    with pytest.raises(N.FlareError) as e:
        ff.set_model(BETA, bad)
    assert e.value.code == N.FLR_EINVAL
    ff.set_variance_mode("direct")                  # the direct form does not need a factorization
    ff.set_model(BETA, bad)
