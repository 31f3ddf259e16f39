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


def _temperature(ke, n):
    return 2.0 * ke / (3.0 * n * synth.KB_EV)


def test_nose_hoover_reaches_and_holds_the_target_temperature():
    """NVT at 450 K from 300 K Maxwell velocities (64 Pt atoms, dt = 1 fs,
    tau = 50 fs): the mean temperature of the second half of 1200 steps is
    within 8 % of the target, and E_pot + KE + thermostat energy is conserved."""
    from paper_2204_12573_gb300 import flare as F
    s = _pt_slab()
    ff, sysg, vel, nl, _ = _setup(s, 0.001)
    st = F.MDState(sysg, vel, dt=0.001, rebuild_every=10, temperature=450.0, tau=0.05)
    out = F.make_outputs(s.n_atoms)
    temps, cons = [], []
    for _ in range(120):
        F.md_step(ff, st, nl, 10, out)
        t = out["totals"].cpu().numpy()
        temps.append(_temperature(t[12], s.n_atoms))
        cons.append(t[0] + t[12] + t[17])
    ff.sync()
    assert st.step == 1200
    t_mean = float(np.mean(temps[60:]))
    assert abs(t_mean - 450.0) <= 0.08 * 450.0, t_mean
    ke_scale = 1.5 * s.n_atoms * synth.KB_EV * 450.0
    assert abs(cons[-1] - cons[0]) <= 0.02 * ke_scale, (cons[0], cons[-1])
    assert st.xi != 0.0


def test_uncertainty_stop():
    """sigma_stop below the largest sigma halts after the first step; above it
    every step runs."""
    from paper_2204_12573_gb300 import flare as F
    s = synth.tiny_system(0)
    ff, sysg, vel, nl, _ = _setup(s, 0.0005)
    sig = F.energy_forces_uncertainty(ff, sysg, nl)["sigma"].cpu().numpy()
    st = F.MDState(sysg, vel, dt=0.0005, sigma_stop=0.5 * float(sig.max()))
    out = F.make_outputs(s.n_atoms)
    F.md_step(ff, st, nl, 5, out)
    assert st.halted and st.step == 1
    assert out["totals"][15].item() >= 1
    st2 = F.MDState(sysg, vel, dt=0.0005, sigma_stop=10.0 * float(sig.max()))
    F.md_step(ff, st2, nl, 5, out)
    assert not st2.halted and st2.step == 5
    assert out["totals"][15].item() == 0


def test_coordination_count_of_h2():
    """Same-species coordination of H within 1 A counts the atoms of intact H2
    molecules, checked against a minimum-image count on the host."""
    from paper_2204_12573_gb300 import flare as F
    s = synth.tiny_system(0)
    ff, sysg, vel, nl, _ = _setup(s, 0.0005)
    for cut in (1.0, 0.5):
        st = F.MDState(sysg, vel, dt=0.0005, cn_species=1, cn_cutoff=cut)
        out = F.make_outputs(s.n_atoms)
        F.md_step(ff, st, nl, 2, out)
        ff.sync()
        p = sysg.pos[:, :3].double().cpu().numpy()
        h = np.nonzero(s.species == 1)[0]
        inv = np.linalg.inv(s.cell)
        cnt = 0
        for a in h:
            dr = p[h] - p[a]
            f = dr @ inv
            f[:, :2] -= np.round(f[:, :2])
            dist = np.linalg.norm(f @ s.cell, axis=1)
            dist[h == a] = 1e9
            cnt += int((dist < cut).any())
        assert out["totals"][16].item() == cnt
    assert cnt == 0                      # no H pair closer than 0.5 A
