"""The hand-written backward (flr_energy_backward) and the autograd wrapper.

For L = sum_i u_i E_i (E_i = d_i^T beta_s d_i, Eq. 1-2 with the mapped beta of
Sec. II-C):
  dL/dr_k   = -(forces of L): the oracle's per-pair dE_i/dr_ij scaled by u_i
              and assembled like forces; also central differences of the
              oracle energy with h = 1e-3 A;
  dL/dbeta_s = sum_{i of species s} u_i d_i d_i^T, from the oracle's d_i.
L is linear in beta, so a finite step of beta must change the GPU's L by
exactly <dL/dbeta, step> up to FP32 rounding.
"""
import numpy as np
import pytest

from paper_2204_12573_gb300 import synth

from gpu_common import F_TOL_FP32, F_TOL_MIXED
import oracle as O

pytestmark = pytest.mark.gpu

BETA, SIGMA = synth.random_model()
H = O.Hyper(2, 8, 3, 4.5)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2204_12573_gb300 import build
    build.build()


def _oracle_grads(s, u):
    """(dL/dpos [n, 3], dL/dbeta [2, d, d]) of L = sum u_i E_i from the oracle."""
    pos = synth.f32_exact_f64(synth.as_f32_positions(s.pos))
    pairs = O.neighbors(pos, s.cell, s.pbc, H.r_cut)
    o = O.evaluate(H, pos, s.species, s.cell, pairs, BETA, SIGMA)
    fw = o["fpair"] * u[pairs[:, 0]][:, None]
    Fw, _ = O.assemble(len(pos), pairs, o["rij"], fw)
    gb = np.zeros((2, H.d, H.d))
    for sp in range(2):
        m = s.species == sp
        gb[sp] = (o["dhat"][m] * u[m][:, None]).T @ o["dhat"][m]
    return -Fw, gb, o


def _weights(n, seed):
    return np.random.default_rng(seed).uniform(-1.0, 1.0, n)


def _batch_model(structs, precision):
    from paper_2204_12573_gb300 import flare as F
    from paper_2204_12573_gb300.autograd import BatchModel
    ff = F.FlareGB(precision=precision, max_nbr=96)
    return BatchModel.from_structures(ff, SIGMA, structs)


def _autograd(structs, u, precision, want_beta=True):
    import torch
    from paper_2204_12573_gb300.autograd import energies
    model = _batch_model(structs, precision)
    pos = torch.tensor(np.concatenate([synth.f32_exact_f64(synth.as_f32_positions(s.pos)) for s in structs]),
                       dtype=torch.float32, device="cuda", requires_grad=True)
    beta = torch.tensor(BETA, dtype=torch.float64, requires_grad=want_beta)
    E, Fo, sig = energies(pos, beta, model)
    L = (torch.as_tensor(u, dtype=torch.float32, device="cuda") * E).sum()
    L.backward()
    torch.cuda.synchronize()
    return (pos.grad.cpu().numpy().astype(np.float64),
            None if beta.grad is None else beta.grad.numpy(),
            E.detach().cpu().numpy(), Fo.cpu().numpy())


def _split(structs):
    off = np.concatenate([[0], np.cumsum([s.n_atoms for s in structs])])
    return [(int(off[k]), int(off[k + 1])) for k in range(len(structs))]


@pytest.mark.parametrize("which", ["tiny", "slabs"])
def test_grad_pos_and_beta_match_oracle_fp32(which):
    structs = [synth.tiny_system(0)] if which == "tiny" else synth.slab_batch(seed=3, n_slabs=6)
    n = sum(s.n_atoms for s in structs)
    u = _weights(n, 17)
    gpos, gbeta, E, _ = _autograd(structs, u, "fp32")
    gb_ref = np.zeros_like(gbeta)
    for (lo, hi), s in zip(_split(structs), structs):
        gp, gb, o = _oracle_grads(s, u[lo:hi])
        assert np.abs(gpos[lo:hi] - gp).max() <= F_TOL_FP32, s.name
        assert np.abs(E[lo:hi] - o["E"]).max() <= 1e-5 * max(1.0, np.abs(o["E"]).max())
        gb_ref += gb
    # |d_i| = 1 and each FP32 descriptor component is within 2e-6 of the oracle's
    assert np.abs(gbeta - gb_ref).max() <= 4e-6 * np.abs(u).sum()


def test_grad_pos_matches_finite_differences():
    """Central differences of the FP64 oracle energy, h = 1e-3 A."""
    s = synth.slab_batch(seed=3, n_slabs=1)[0]
    u = _weights(s.n_atoms, 23)
    gpos, _, _, _ = _autograd([s], u, "fp32", want_beta=False)
    pos0 = synth.f32_exact_f64(synth.as_f32_positions(s.pos))
    rng = np.random.default_rng(5)
    top = np.argsort(pos0[:, 2])[-20:]
    atoms = np.concatenate([rng.choice(top, 3, replace=False), rng.choice(s.n_atoms, 3, replace=False)])
    h = 1e-3

    def L(p):
        pairs = O.neighbors(p, s.cell, s.pbc, H.r_cut)
        return float(u @ O.evaluate(H, p, s.species, s.cell, pairs, BETA, SIGMA, want_forces=False)["E"])

    for a in atoms:
        for c in range(3):
            pp, pm = pos0.copy(), pos0.copy()
            pp[a, c] += h
            pm[a, c] -= h
            fd = (L(pp) - L(pm)) / (2 * h)
            assert abs(gpos[a, c] - fd) <= F_TOL_MIXED, (a, c, gpos[a, c], fd)


def test_grad_beta_is_exact_for_linear_energy():
    """L is linear in beta: L(beta + t*D) - L(beta) = t * <dL/dbeta, D>."""
    import torch
    from paper_2204_12573_gb300.autograd import energies
    structs = synth.slab_batch(seed=3, n_slabs=4)
    n = sum(s.n_atoms for s in structs)
    u = _weights(n, 29)
    model = _batch_model(structs, "fp32")
    pos = torch.tensor(np.concatenate([synth.as_f32_positions(s.pos)[:, :3] for s in structs]), device="cuda")
    beta = torch.tensor(BETA, dtype=torch.float64, requires_grad=True)
    ut = torch.as_tensor(u, dtype=torch.float32, device="cuda")
    E0 = energies(pos, beta, model)[0]
    (ut * E0).sum().backward()
    L0 = float((ut.double() * E0.detach().double()).sum())
    D = torch.tensor(synth.random_model(beta_seed=77, sigma_seed=78)[0], dtype=torch.float64)
    t = 0.5
    L1 = float((ut.double() * energies(pos, beta.detach() + t * D, model)[0].double()).sum())
    pred = t * float((beta.grad * D).sum())
    assert abs((L1 - L0) - pred) <= 1e-5 * max(1.0, abs(pred)) + 1e-6 * np.abs(u).sum()


@pytest.mark.parametrize("precision", ["bf16x3", "tf32"])
def test_grad_pos_mixed_precision(precision):
    structs = synth.slab_batch(seed=3, n_slabs=4)
    n = sum(s.n_atoms for s in structs)
    u = _weights(n, 31)
    gpos, _, _, _ = _autograd(structs, u, precision, want_beta=False)
    for (lo, hi), s in zip(_split(structs), structs):
        gp, _, _ = _oracle_grads(s, u[lo:hi])
        assert np.abs(gpos[lo:hi] - gp).max() <= F_TOL_MIXED


def test_unit_weights_give_minus_forces():
    """u = 1: dL/dpos is exactly -F of the forward call (same kernels)."""
    structs = synth.slab_batch(seed=3, n_slabs=3)
    n = sum(s.n_atoms for s in structs)
    gpos, _, _, Fo = _autograd(structs, np.ones(n), "bf16x3", want_beta=False)
    assert np.array_equal(gpos.astype(np.float32), -Fo)


@pytest.mark.slow
def test_slab_batch_256_backward():
    """Both gradients over the whole batch of 256 slabs (200-600 atoms)."""
    structs = synth.slab_batch(seed=3, n_slabs=256)
    n = sum(s.n_atoms for s in structs)
    u = _weights(n, 41)
    gpos, gbeta, _, _ = _autograd(structs, u, "fp32")
    gb_ref = np.zeros_like(gbeta)
    for (lo, hi), s in zip(_split(structs), structs):
        gp, gb, _ = _oracle_grads(s, u[lo:hi])
        assert np.abs(gpos[lo:hi] - gp).max() <= F_TOL_FP32, s.name
        gb_ref += gb
    assert np.abs(gbeta - gb_ref).max() <= 4e-6 * np.abs(u).sum()
