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


def test_one_nvt_step_matches_the_fp64_oracle_step():
    """One Nose-Hoover velocity-Verlet step at the paper's protocol (450 K,
    dt = 0.1 fs) of the 44-atom H2/Pt(111) system, against the FP64 oracle's
    step (oracle/md.py) driven by the oracle's own forces: positions,
    velocities and the thermostat variables xi and eta."""
    import oracle as O
    from oracle import md as OM
    from paper_2204_12573_gb300 import flare as F
    s = synth.tiny_system(0)
    dt, T, tau = 1e-4, 450.0, 0.01
    ff, sysg, vel, nl, _ = _setup(s, dt)
    x0 = sysg.pos[:, :3].double().cpu().numpy()
    v0 = vel[:, :3].double().cpu().numpy()
    st = F.MDState(sysg, vel, dt=dt, rebuild_every=10, temperature=T, tau=tau)
    out = F.make_outputs(s.n_atoms)
    F.md_step(ff, st, nl, 1, out)
    ff.sync()
    x1 = sysg.pos[:, :3].double().cpu().numpy()
    v1 = vel[:, :3].double().cpu().numpy()

    def force(x):
        return O.energy_forces(O.Hyper(), x, s.species, s.cell, s.pbc, BETA, SIGMA, skin=0.5)["F"]

    m = np.array([synth.MASS[int(k)] for k in s.species])
    xr, vr, xir, etar, _ = OM.nvt_step(x0, v0, m, force, dt, T, tau, 0.0, 0.0)
    # FP32 positions (|x| < 30 A) and the FP32 force tolerance (1e-4 eV/A over dt on 1 amu)
    assert np.abs(x1 - xr).max() <= 1e-5
    assert np.abs(v1 - vr).max() <= 5e-4
    assert abs(st.xi - xir) <= 1e-5 * abs(xir) and xir < 0.0     # heating from 300 K: xi < 0
    assert abs(st.eta - etar) <= 1e-5 * abs(etar)


def test_nvt_paper_protocol_450K_0p1fs():
    """The production protocol of Sec. VI-A: Nose-Hoover NVT at 450 K with a
    0.1 fs step, on a Pt(111) slab with adsorbed H (225 atoms) started
    from 300 K: after 60 thermostat periods the mean temperature is within
    5 % of 450 K, and E_pot + KE + thermostat energy stays within 1 % of the
    kinetic energy.  (Without the thermostat's energy term it would move by
    the heat put in, about two thirds of the kinetic energy; the remaining
    fluctuation is velocity Verlet's on the light H atoms in the stiff model
    potential.)"""
    from paper_2204_12573_gb300 import flare as F
    s = synth.slab_batch(seed=3, n_slabs=1)[0]
    dt, T, tau = 1e-4, 450.0, 0.01
    ff, sysg, vel, nl, _ = _setup(s, dt)
    st = F.MDState(sysg, vel, dt=dt, rebuild_every=10, temperature=T, tau=tau)
    out = F.make_outputs(s.n_atoms)
    temps, cons = [], []
    for _ in range(120):
        F.md_step(ff, st, nl, 50, out)
        t = out["totals"].cpu().numpy()
        temps.append(_temperature(t[12], s.n_atoms))
        cons.append(t[0] + t[12] + t[17])
    ff.sync()
    assert st.step == 6000
    t_mean = float(np.mean(temps[60:]))
    assert abs(t_mean - T) <= 0.05 * T, t_mean
    ke_scale = 1.5 * s.n_atoms * synth.KB_EV * T
    assert np.abs(np.array(cons) - cons[0]).max() <= 1e-2 * ke_scale, (cons[0], max(cons), min(cons))


def test_uncertainty_stop():
    """sigma_stop below the largest sigma halts after the first step; above it
    every step runs.  The count of uncertain atoms is integer work: it must
    equal, exactly, the number of atoms whose returned sigma at the halting
    step exceeds sigma_stop (the FP32 comparison the device makes)."""
    from paper_2204_12573_gb300 import flare as F
    s = synth.tiny_system(0)
    ff, sysg, vel, nl, _ = _setup(s, 0.0005)
    sig = F.energy_forces_uncertainty(ff, sysg, nl)["sigma"].cpu().numpy()
    for frac in (0.5, 0.9, 0.999):
        thr = frac * float(sig.max())
        st = F.MDState(sysg, vel, dt=0.0005, sigma_stop=thr)
        out = F.make_outputs(s.n_atoms)
        F.md_step(ff, st, nl, 5, out)
        ff.sync()
        assert st.halted and st.step == 1
        sig_step = out["sigma"].cpu().numpy()
        n_above = int((sig_step > np.float32(thr)).sum())
        assert n_above >= 1
        assert out["totals"][15].item() == n_above
    st2 = F.MDState(sysg, vel, dt=0.0005, sigma_stop=10.0 * float(sig.max()))
    out = F.make_outputs(s.n_atoms)
    F.md_step(ff, st2, nl, 5, out)
    assert not st2.halted and st2.step == 5
    assert out["totals"][15].item() == 0


def test_uncertainty_count_on_a_large_slab():
    """The same exact count on a 130k-atom slab with a threshold inside the
    sigma distribution (thousands of atoms above it)."""
    from paper_2204_12573_gb300 import flare as F
    s = synth.big_slab(seed=1, nx=64, n_rows=64, n_layers=32, n_h2=1024)
    ff, sysg, vel, nl, _ = _setup(s, 0.0005, precision="bf16x3")
    sig = F.energy_forces_uncertainty(ff, sysg, nl)["sigma"].cpu().numpy()
    thr = float(np.quantile(sig, 0.97))
    st = F.MDState(sysg, vel, dt=0.0005, sigma_stop=thr)
    out = F.make_outputs(s.n_atoms)
    F.md_step(ff, st, nl, 3, out)
    ff.sync()
    assert st.halted and st.step == 1
    n_above = int((out["sigma"].cpu().numpy() > np.float32(thr)).sum())
    assert n_above > 1000
    assert out["totals"][15].item() == n_above


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


def test_rebuild_steps_match_a_fresh_build():
    """MD steps run the list rebuild as a conditional graph (the sequence runs
    only when the rebuild flag is set).  With a rebuild due every step, the
    list after the last step must equal, entry for entry, a fresh build at the
    final (wrapped) positions; with rebuilds every 4 steps over 6 steps,
    exactly one rebuild is counted unless the displacement trigger fired."""
    from paper_2204_12573_gb300 import flare as F
    s = _pt_slab(3)
    ff, sysg, vel, nl, st = _setup(s, 0.002)
    st.c.rebuild_every = 1
    out = F.make_outputs(s.n_atoms)
    F.md_step(ff, st, nl, 3, out)
    ff.sync()
    assert int(out["totals"][13].item()) == 3
    e1, c1, g1 = (t.cpu().numpy() for t in nl.view(s.n_atoms))
    nl2 = ff.nbrlist(s.n_atoms)
    F.build_neighbors(ff, sysg, nl2)
    e2, c2, g2 = (t.cpu().numpy() for t in nl2.view(s.n_atoms))
    assert np.array_equal(c1, c2) and np.array_equal(g1, g2)
    for i in range(s.n_atoms):
        assert np.array_equal(np.sort(e1[i, :c1[i]]), np.sort(e2[i, :c2[i]]))
    # a cadence of 4: steps 4 and (if the trigger fires) others rebuild; step 1-3 and 5-6 skip the body
    ff3, sysg3, vel3, nl3, st3 = _setup(s, 0.0005)
    st3.c.rebuild_every = 4
    out3 = F.make_outputs(s.n_atoms)
    F.md_step(ff3, st3, nl3, 6, out3)
    ff3.sync()
    assert 1 <= int(out3["totals"][13].item()) <= 6


def _host_vs_device(s, n_calls, steps_per_call, temperature=0.0, halve_vel_after=None):
    """The same MD run through flr_md_step (state on the device) and through
    flr_md_step_host (state in pinned host x, y, z rows, uploaded before and
    downloaded after every step).  The unpack and pack are copies of x, y, z,
    so every result must agree bit for bit."""
    import torch
    from paper_2204_12573_gb300 import flare as F
    ffa, sysa, vela, nla, sta = _setup(s, 0.002)
    ffb, sysb, velb, nlb, stb = _setup(s, 0.002)
    for st in (sta, stb):
        st.c.rebuild_every = 3
        st.c.temperature = temperature
    outa, outb = F.make_outputs(s.n_atoms), F.make_outputs(s.n_atoms)
    host = F.HostState(sysb.pos.cpu(), velb.cpu(), results=("energy", "forces", "variance", "sigma", "totals"))
    # the working copies start from something else: the host rows are the state
    sysb.pos.zero_()
    velb.zero_()
    for k in range(n_calls):
        F.md_step(ffa, sta, nla, steps_per_call, outa)
        F.md_step_host(ffb, stb, nlb, steps_per_call, outb, host)
        if halve_vel_after is not None and k == halve_vel_after:
            ffa.sync()
            ffb.sync()              # the host rows may be changed once the copies have landed
            vela[:, :3] *= 0.5
            host.vel.mul_(0.5)
    ffa.sync()
    ffb.sync()
    torch.cuda.synchronize()
    assert np.array_equal(host.pos.numpy(), sysa.pos[:, :3].cpu().numpy())
    assert np.array_equal(host.vel.numpy(), vela[:, :3].cpu().numpy())
    for key in ("energy", "forces", "variance", "sigma"):
        assert np.array_equal(host[key].numpy(), outa[key].cpu().numpy()), key
    # the virial's FP32 partial sums follow the force kernel's dynamic
    # atom-to-warp assignment, so it agrees to rounding; every other total
    # (fixed-order reductions and counts) bit for bit
    ta, tb = outa["totals"].cpu().numpy(), host["totals"].numpy()
    vir = slice(1, 10)
    assert np.abs(ta[vir] - tb[vir]).max() <= 1e-6 * max(1.0, np.abs(ta[vir]).max())
    assert np.array_equal(np.delete(ta, np.r_[vir]), np.delete(tb, np.r_[vir]))
    assert sta.step == stb.step == n_calls * steps_per_call
    # the device working copies hold the same state as the host rows
    assert np.array_equal(sysb.pos[:, :3].cpu().numpy(), host.pos.numpy())
    return ta


def test_host_state_md_matches_device_md():
    s = _pt_slab(5)
    # cadence 3: the list is rebuilt at steps 3 and 6 of the 7
    _host_vs_device(s, n_calls=7, steps_per_call=1, halve_vel_after=3)
    _host_vs_device(s, n_calls=2, steps_per_call=3)
    _host_vs_device(s, n_calls=3, steps_per_call=1, temperature=450.0)


def test_host_state_requires_pos_and_vel():
    import ctypes
    from paper_2204_12573_gb300 import _native as N, flare as F
    s = _pt_slab(6)
    ff, sysg, vel, nl, st = _setup(s, 0.001)
    out = F.make_outputs(s.n_atoms)
    host = N.HostState()
    rc = ff.lib.flr_md_step_host(ff.handle, ctypes.byref(st.c), nl.handle, 1, ctypes.byref(F._outputs_struct(out)),
                                 ctypes.byref(host), F._stream(None))
    assert rc != 0
    assert st.step == 0


def test_host_state_uncertainty_stop():
    """The uncertainty stop through flr_md_step_host: the call ends after the
    halting step, and the host rows hold that step's state and results, the
    same bits as the device-state call."""
    import torch
    from paper_2204_12573_gb300 import flare as F
    s = synth.tiny_system(0)
    ffa, sysa, vela, nla, _ = _setup(s, 0.0005)
    ffb, sysb, velb, nlb, _ = _setup(s, 0.0005)
    sig = F.energy_forces_uncertainty(ffa, sysa, nla)["sigma"].cpu().numpy()
    thr = 0.9 * float(sig.max())
    sta = F.MDState(sysa, vela, dt=0.0005, sigma_stop=thr)
    stb = F.MDState(sysb, velb, dt=0.0005, sigma_stop=thr)
    outa, outb = F.make_outputs(s.n_atoms), F.make_outputs(s.n_atoms)
    host = F.HostState(sysb.pos.cpu(), velb.cpu(), results=("energy", "forces", "sigma", "totals"))
    F.md_step(ffa, sta, nla, 5, outa)
    F.md_step_host(ffb, stb, nlb, 5, outb, host)
    ffa.sync()
    ffb.sync()
    torch.cuda.synchronize()
    assert sta.halted and stb.halted and sta.step == stb.step == 1
    assert np.array_equal(host.pos.numpy(), sysa.pos[:, :3].cpu().numpy())
    assert np.array_equal(host.vel.numpy(), vela[:, :3].cpu().numpy())
    for key in ("energy", "forces", "sigma"):
        assert np.array_equal(host[key].numpy(), outa[key].cpu().numpy()), key
    assert host["totals"][15].item() == outa["totals"][15].item() >= 1
