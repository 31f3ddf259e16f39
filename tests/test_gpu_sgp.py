"""Sparse-GP mapping on the device (flr_map_sgp, Sec. V-B "Mapped Sparse GP"):
beta = sig2 D_S^T diag(alpha) D_S and Sigma = sig2 I - sig2^2 D_S^T K_SS^{-1} D_S
against the FP64 oracle's mapping, and the mapped model's energies and
variances on other environments against Eq. 1 and Eq. 2 summed over the
sparse set (the mapping is lossless)."""
import numpy as np
import pytest

from paper_2204_12573_gb300 import synth

from gpu_common import E_TOL_FP32, V_TOL_FP32, gpu_run, oracle_run
from oracle import sgp

pytestmark = pytest.mark.gpu

BETA, SIGMA = synth.random_model()
SIG2 = 0.7
JITTER = 1e-3


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2204_12573_gb300 import build
    build.build()


@pytest.fixture(scope="module")
def sparse_sets():
    """Per central species: descriptor rows of real environments (the
    oracle's FP64 d-hat of two slabs), random mean weights, and
    K_SS = sig2 D_S D_S^T + jitter I (the xi = 1 kernel, positive definite)."""
    rng = np.random.default_rng(11)
    rows = {0: [], 1: []}
    for s in synth.slab_batch(seed=11, n_slabs=2):
        o = oracle_run(s, BETA, SIGMA)
        ok = o["norm"] > 0
        for sp in (0, 1):
            rows[sp].append(o["dhat"][ok & (s.species == sp)])
    out = {}
    for sp in (0, 1):
        D = np.concatenate(rows[sp])
        n_s = min(120, len(D))
        D_S = D[rng.choice(len(D), n_s, replace=False)]
        alpha = rng.normal(size=n_s)
        K = SIG2 * (D_S @ D_S.T) + JITTER * np.eye(n_s)
        out[sp] = (D_S, alpha, K)
    return out


def _ff(sets, precision="fp32"):
    import torch
    from paper_2204_12573_gb300 import flare as F
    ff = F.FlareGB(precision=precision)
    mats = {}
    for sp in (0, 1):
        D_S, alpha, K = sets[sp]
        b, g = ff.map_sgp(sp, torch.as_tensor(D_S), torch.as_tensor(alpha), torch.as_tensor(K), SIG2)
        mats[sp] = (b.cpu().numpy(), g.cpu().numpy())
    return ff, mats


def test_mapped_matrices_match_oracle(sparse_sets):
    _, mats = _ff(sparse_sets)
    for sp in (0, 1):
        D_S, alpha, K = sparse_sets[sp]
        b_ref = sgp.mapped_beta(D_S, alpha, SIG2)
        g_ref = sgp.mapped_gamma(D_S, K, SIG2)
        b, g = mats[sp]
        assert np.abs(b - b_ref).max() <= 1e-11 * max(1.0, np.abs(b_ref).max())
        assert np.abs(g - g_ref).max() <= 1e-9 * max(1.0, np.abs(g_ref).max())


def test_mapping_is_lossless_on_the_gpu_path(sparse_sets):
    """E_i and V_i of the FP32 path with the mapped model equal Eq. 1 and
    Eq. 2 evaluated over the sparse set, on environments not in it."""
    import torch
    from paper_2204_12573_gb300 import flare as F
    ff, mats = _ff(sparse_sets)
    s = synth.tiny_system(3)
    sysg = F.System.from_numpy(synth.as_f32_positions(s.pos), s.species, s.cell, s.pbc)
    nl = ff.nbrlist(s.n_atoms)
    F.build_neighbors(ff, sysg, nl)
    r = F.energy_forces_uncertainty(ff, sysg, nl)
    ff.sync()
    E = r["energy"].cpu().numpy()
    V = r["variance"].cpu().numpy()
    beta = np.stack([mats[0][0], mats[1][0]])
    gam = np.stack([mats[0][1], mats[1][1]])
    o = oracle_run(s, beta, gam)
    for sp in (0, 1):
        D_S, alpha, K = sparse_sets[sp]
        sel = (s.species == sp) & (o["norm"] > 0)
        d = o["dhat"][sel]
        e_ref = sgp.sgp_mean(d, D_S, alpha, SIG2)
        v_ref = sgp.sgp_variance(d, D_S, K, SIG2)
        # the oracle's quadratic forms with the mapped matrices reach the same values
        assert np.abs(o["E"][sel] - e_ref).max() <= 1e-9 * max(1.0, np.abs(e_ref).max())
        assert np.abs(o["V"][sel] - v_ref).max() <= 1e-9 * max(1.0, np.abs(v_ref).max())
        bn = np.linalg.norm(beta[sp], 2)
        assert (np.abs(E[sel] - e_ref) <= E_TOL_FP32 * np.maximum(np.abs(e_ref), bn)).all()
        assert (np.abs(V[sel] - v_ref) <= V_TOL_FP32 * np.maximum(v_ref, 1e-6)).all()
    torch.cuda.synchronize()


def test_not_positive_definite_is_rejected(sparse_sets):
    import torch
    from paper_2204_12573_gb300 import flare as F
    from paper_2204_12573_gb300 import _native as N
    D_S, alpha, K = sparse_sets[0]
    bad = K.copy()
    bad[0, 0] = -1.0
    ff = F.FlareGB(precision="fp32")
    with pytest.raises(N.FlareError) as e:
        ff.map_sgp(0, torch.as_tensor(D_S), torch.as_tensor(alpha), torch.as_tensor(bad), SIG2)
    assert e.value.code == N.FLR_EINVAL


@pytest.mark.parametrize("n_s", [1, 33, 300])
def test_mapping_sizes_against_oracle(n_s):
    """A single sparse point, one past a 32-column Cholesky panel, and many
    panels: random unit descriptor rows, K_SS = sig2 D D^T + jitter I."""
    import torch
    from paper_2204_12573_gb300 import flare as F
    rng = np.random.default_rng(100 + n_s)
    ff = F.FlareGB(precision="fp32")
    d = ff.d_full
    D = rng.normal(size=(n_s, d))
    D /= np.linalg.norm(D, axis=1, keepdims=True)
    alpha = rng.normal(size=n_s)
    K = SIG2 * (D @ D.T) + JITTER * np.eye(n_s)
    b, g = ff.map_sgp(1, torch.as_tensor(D), torch.as_tensor(alpha), torch.as_tensor(K), SIG2)
    b, g = b.cpu().numpy(), g.cpu().numpy()
    b_ref = sgp.mapped_beta(D, alpha, SIG2)
    g_ref = sgp.mapped_gamma(D, K, SIG2)
    assert np.abs(b - b_ref).max() <= 1e-11 * max(1.0, np.abs(b_ref).max())
    assert np.abs(g - g_ref).max() <= 1e-9 * max(1.0, np.abs(g_ref).max())

