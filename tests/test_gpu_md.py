"""Velocity-Verlet MD (flr_md_step): one step against the integrator written
out on the host with the library's own forces, and energy conservation in
NVE, whose error must shrink like dt^2 (the method is symplectic and second
order; the forces are conservative by construction, Sec. V-B)."""
import numpy as np
import pytest

from paper_2204_12573_gb300 import synth

pytestmark = pytest.mark.gpu

BETA, SIGMA = synth.random_model()


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2204_12573_gb300 import build
    build.build()


def _pt_slab(seed=0):
    """4x4 hexagonal Pt(111) cell, 4 layers (64 Pt), displacements 0.05 A."""
    rng = np.random.default_rng(seed)
    pos, cell, _ = synth.pt111_hex_slab(4, 4, 4, vacuum=15.0)
    pos = pos + rng.normal(scale=0.05, size=pos.shape)
    return synth.Structure(synth._wrap(pos, cell, (1, 1, 0)), np.zeros(len(pos), np.int32), cell, (1, 1, 0), "pt64")


def _setup(s, dt, precision="fp32", seed=1):
    import torch
    from paper_2204_12573_gb300 import flare as F
    ff = F.FlareGB(precision=precision)
    ff.set_model(BETA, SIGMA)
    sysg = F.System.from_numpy(synth.as_f32_positions(s.pos), s.species, s.cell, s.pbc)
    vel = torch.as_tensor(synth.maxwell_velocities(s.species, 300.0, seed), device="cuda")
    nl = ff.nbrlist(s.n_atoms)
    F.build_neighbors(ff, sysg, nl)
    st = F.MDState(sysg, vel, dt=dt, rebuild_every=10)
    return ff, sysg, vel, nl, st


def test_one_step_is_velocity_verlet():
    from paper_2204_12573_gb300 import flare as F
    s = _pt_slab()
    dt = 0.001
    ff, sysg, vel, nl, st = _setup(s, dt)
    x0 = sysg.pos[:, :3].double().cpu().numpy()
    v0 = vel[:, :3].double().cpu().numpy()
    f0 = F.energy_forces_uncertainty(ff, sysg, nl)["forces"].double().cpu().numpy()
    out = F.make_outputs(s.n_atoms)
    F.md_step(ff, st, nl, 1, out)
    ff.sync()
    x1 = sysg.pos[:, :3].double().cpu().numpy()
    v1 = vel[:, :3].double().cpu().numpy()
    f1 = out["forces"].double().cpu().numpy()
    m = np.array([synth.MASS[int(k)] for k in s.species])[:, None]
    a0 = f0 * synth.FTM2V / m
    a1 = f1 * synth.FTM2V / m
    assert np.abs(x1 - (x0 + dt * v0 + 0.5 * dt * dt * a0)).max() <= 2e-5
    assert np.abs(v1 - (v0 + 0.5 * dt * (a0 + a1))).max() <= 1e-4 * max(1.0, np.abs(v1).max())
    # kinetic energy reported in the totals
    ke = 0.5 * (m[:, 0] * (v1 ** 2).sum(1)).sum() / synth.FTM2V
    assert abs(float(out["totals"][12]) - ke) <= 1e-5 * ke
    assert st.step == 1


def _energy_trace(s, dt, steps):
    from paper_2204_12573_gb300 import flare as F
    ff, sysg, vel, nl, st = _setup(s, dt)
    out = F.make_outputs(s.n_atoms)
    e = []
    for _ in range(steps):
        F.md_step(ff, st, nl, 1, out)
        t = out["totals"].cpu().numpy()
        e.append(t[0] + t[12])
    ff.sync()
    return np.array(e)


def test_nve_energy_error_scales_as_dt_squared():
    """Same 200 fs trajectory at dt = 2 fs and 1 fs: the total-energy
    excursion must be small against the kinetic energy and shrink ~4x."""
    s = _pt_slab()
    e2 = _energy_trace(s, 0.002, 100)
    e1 = _energy_trace(s, 0.001, 200)
    d2 = np.abs(e2 - e2[0]).max()
    d1 = np.abs(e1 - e1[0]).max()
    ke = 1.5 * s.n_atoms * synth.KB_EV * 300.0
    assert d2 < 0.05 * ke, (d2, ke)
    assert 2.5 <= d2 / d1 <= 6.5, (d2, d1)
