"""Parity at the full benchmark size, in the configuration bench.py times:
the 2,129,920-atom H2/Pt(111) slab, max_nbr 64, velocity-Verlet steps with
on-device rebuild decisions.  The oracle evaluates sampled atoms one by one
(forces need each sampled atom's neighbours as centres), at the positions the
GPU holds after the steps.  Properties that hold at any size are checked on
all atoms: zero net force, bitwise-reproducible forces, the totals against
sums of the per-atom outputs."""
import numpy as np
import pytest

from paper_2204_12573_gb300 import synth

from gpu_common import E_TOL_FP32, F_TOL_FP32, F_TOL_MIXED, V_TOL_FP32, mixed_bounds
import oracle as O

pytestmark = pytest.mark.gpu

BETA, SIGMA = synth.random_model()


@pytest.fixture(scope="module")
def slab():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2204_12573_gb300 import build
    build.build()
    return synth.big_slab(seed=1)


def _sample(groups, rng, n_mixed=64, n_rest=192):
    mixed = np.nonzero(groups % 3 == 0)[0]
    rest = np.nonzero(groups % 3 != 0)[0]
    return np.sort(np.concatenate([rng.choice(mixed, min(n_mixed, len(mixed)), replace=False),
                                   rng.choice(rest, n_rest, replace=False)]))


@pytest.mark.parametrize("precision", ["fp32", "tf32", "bf16x3"])
def test_full_size_md_then_sampled_parity(slab, precision):
    import torch
    from paper_2204_12573_gb300 import flare as F
    s = slab
    n = s.n_atoms
    ff = F.FlareGB(precision=precision, max_nbr=64)
    ff.set_model(BETA, SIGMA)
    sysg = F.System.from_numpy(synth.as_f32_positions(s.pos), s.species, s.cell, s.pbc)
    vel = torch.as_tensor(synth.maxwell_velocities(s.species, 300.0, seed=1), device="cuda")
    nl = ff.nbrlist(n)
    F.build_neighbors(ff, sysg, nl)
    st = F.MDState(sysg, vel)
    out = F.make_outputs(n)
    F.md_step(ff, st, nl, 12, out)          # crosses the rebuild cadence
    ff.sync()
    assert st.step == 12
    assert out["totals"][13].item() >= 1    # at least one rebuild happened in the steps
    # one more evaluation at the current positions, against the oracle on sampled atoms
    F.build_neighbors(ff, sysg, nl)
    r = F.energy_forces_uncertainty(ff, sysg, nl, F.make_outputs(n))
    ff.sync()
    _, _, groups = nl.view(n)
    idx = _sample(groups.cpu().numpy(), np.random.default_rng(7))
    pos = sysg.pos[:, :3].double().cpu().numpy()
    o = O.forces_subset(O.Hyper(), pos, s.species, s.cell, s.pbc, BETA, SIGMA, idx, skin=0.5)
    E = r["energy"].cpu().numpy()[idx]
    Fg = r["forces"].cpu().numpy()[idx]
    V = r["variance"].cpu().numpy()[idx]
    f_tol = F_TOL_FP32 if precision == "fp32" else F_TOL_MIXED
    assert np.abs(Fg - o["F"]).max() <= f_tol
    if precision == "fp32":
        assert (np.abs(E - o["E"]) <= E_TOL_FP32 * np.maximum(np.abs(o["E"]), 1.0)).all()
        ok = o["V"] > 0
        assert (np.abs(V[ok] - o["V"][ok]) / o["V"][ok] <= V_TOL_FP32).all()
    else:
        g_idx = groups.cpu().numpy()[idx]
        bE, bV = mixed_bounds(precision, o["dhat"], s.species[idx], g_idx, BETA, SIGMA, o["E"], o["V"])
        assert (np.abs(E - o["E"]) <= bE).all(), float((np.abs(E - o["E"]) / bE).max())
        assert (np.abs(V - o["V"]) <= bV).all(), float((np.abs(V - o["V"]) / bV).max())
    # properties over all atoms
    Fall = r["forces"].double()
    assert Fall.sum(0).abs().max().item() <= 1e-3          # fixed-point scatter: F_i + F_j = 0 per pair
    Etot = r["energy"].double().sum().item()
    assert abs(r["totals"][0].item() - Etot) <= 1e-9 * max(1.0, abs(Etot)) + 1e-6
    r2 = F.energy_forces_uncertainty(ff, sysg, nl, F.make_outputs(n))
    ff.sync()
    assert torch.equal(r["forces"], r2["forces"])
