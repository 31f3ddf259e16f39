"""Shared helpers of the GPU parity tests: run the CUDA path and the FP64
oracle on the same seeded inputs."""
import numpy as np

import oracle as O
from paper_2204_12573_gb300 import synth

HYPER = dict(n_species=2, n_max=8, l_max=3, r_cut=4.5, skin=0.5)

# Tolerances of the plain FP32 path (stated for the method; see the tests):
#   energy:   |dE_i| <= 1e-5 * max(|E_i|, ||beta_s||_2)   (||beta_s||_2 = 1 eV)
#   forces:   |dF| <= 1e-4 eV/A per component
#   variance: |dV_i| <= 1e-4 * V_i
# Mixed-precision paths (TF32, 3xBF16): forces <= 1e-3 eV/A.
E_TOL_FP32 = 1e-5
F_TOL_FP32 = 1e-4
V_TOL_FP32 = 1e-4
F_TOL_MIXED = 1e-3


def decode_entries(entries, count):
    """Library ELL rows -> sorted [m, 5] (i, j, sx, sy, sz) like the oracle."""
    e = entries.cpu().numpy()
    c = count.cpu().numpy()
    rows = []
    for i in range(len(c)):
        v = e[i, :c[i]].astype(np.int64)
        j = v >> 8
        code = v & 127
        sx = code // 25 - 2
        sy = (code // 5) % 5 - 2
        sz = code % 5 - 2
        rows.append(np.stack([np.full_like(j, i), j, sx, sy, sz], axis=1))
    if not rows:
        return np.zeros((0, 5), np.int64)
    out = np.concatenate(rows, axis=0)
    order = np.lexsort((out[:, 4], out[:, 3], out[:, 2], out[:, 1], out[:, 0]))
    return out[order]


def gpu_run(struct, beta, sigma, precision="fp32", compaction=True, max_nbr=64, n_max=8, want_desc=False):
    import torch
    from paper_2204_12573_gb300 import flare as F
    ff = F.FlareGB(n_max=n_max, precision=precision, compaction=compaction, max_nbr=max_nbr)
    ff.set_model(beta, sigma)
    pos4 = synth.as_f32_positions(struct.pos)
    sysg = F.System.from_numpy(pos4, struct.species, struct.cell, struct.pbc)
    nl = ff.nbrlist(struct.n_atoms)
    F.build_neighbors(ff, sysg, nl)
    out = F.energy_forces_uncertainty(ff, sysg, nl)
    res = {k: v.detach().cpu().numpy() for k, v in out.items()}
    if want_desc:
        d, norm = F.compute_descriptors(ff, sysg, nl)
        res["dhat"] = d.cpu().numpy()
        res["norm"] = norm.cpu().numpy()
    ff.sync()
    res["entries"], res["count"], res["group"] = nl.view(struct.n_atoms)
    torch.cuda.synchronize()
    return res, ff, nl, sysg


def oracle_run(struct, beta, sigma, n_max=8, skin=0.5):
    h = O.Hyper(2, n_max, 3, 4.5)
    pos = synth.f32_exact_f64(synth.as_f32_positions(struct.pos))
    return O.energy_forces(h, pos, struct.species, struct.cell, struct.pbc, beta, sigma, skin=skin)


def compare_efv(g, o, beta_norm=1.0, e_tol=E_TOL_FP32, f_tol=F_TOL_FP32, v_tol=V_TOL_FP32):
    dE = np.abs(g["energy"] - o["E"])
    assert (dE <= e_tol * np.maximum(np.abs(o["E"]), beta_norm)).all(), dE.max()
    dF = np.abs(g["forces"] - o["F"]).max()
    assert dF <= f_tol, dF
    if v_tol is not None:
        ok = o["V"] > 0
        dV = np.abs(g["variance"][ok] - o["V"][ok]) / o["V"][ok]
        assert (dV <= v_tol).all(), dV.max()
    return dict(dE=float(dE.max()), dF=float(dF))
