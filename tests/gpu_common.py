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

# Energy and variance bounds of the mixed-precision paths, from the error of
# the split-precision products (not fitted to any output).  The GEMM forms
# p_j = sum_k d_k w_jk with w a row of beta or Sigma:
#   3xBF16: x = h + l + e with h = RN_bf16(x), l = RN_bf16(x - h), |e| <= u_b^2 |x|,
#           |l| <= u_b (1 + u_b) |x| (u_b = 2^-8); the kernel adds h_d h_w + h_d l_w
#           + l_d h_w (each exact in FP32) and drops l_d l_w, so one product is off
#           by at most (2 u_b^2 + u_b^4 + u_b^2 (1 + u_b)^2) |d_k w_jk| < 3.1 u_b^2 |d_k w_jk|;
#   TF32:   both operands rounded to nearest TF32 (u_t = 2^-11), products exact in
#           FP32: at most (2 u_t + u_t^2) |d_k w_jk|;
# and the FP32 accumulation of n products adds at most n u_a sum_k |d_k w_jk|
# (u_a = 2^-23, one ulp per addition, whether the adder rounds or truncates;
# n = 3K for the three 3xBF16 passes, K for TF32).  The epilogue's FP32 dot
# product d . p adds K u_a more.  With |d|^T |W| |d| = sum_jk |d_j| |w_jk| |d_k|:
#   |dE_i| <= E_TOL_FP32 max(|E_i|, ||beta||_2) + c |d_i|^T |beta_s| |d_i|
#   |dV_i| <= V_TOL_FP32 V_i                    + c |d_i|^T |Sigma_s| |d_i|
# where the first terms are the FP32 path's own tolerances (FP32 descriptor)
# and c = (product bound) + (n + K) u_a for the atom's class dimension K.
U_BF16 = 2.0 ** -8
U_TF32 = 2.0 ** -11
U_ACC = 2.0 ** -23


def mixed_coefficient(precision, K):
    if precision == "bf16x3":
        return 3.1 * U_BF16 ** 2 + (3 * K + K) * U_ACC
    if precision == "tf32":
        return 2 * U_TF32 + U_TF32 ** 2 + (K + K) * U_ACC
    raise ValueError(precision)


def mixed_bounds(precision, dhat, species, groups, beta, sigma, E, V, d_full=544, d_single=144, beta_norm=1.0):
    """Per-atom bounds on |dE| and |dV| of a mixed-precision path (see above).
    dhat: the oracle's FP64 descriptors (full layout), groups: the GPU's
    compaction groups (group % 3 == 0: two-species class of dimension d_full)."""
    d = np.abs(np.asarray(dhat, np.float64))
    aE = np.zeros(len(d))
    aV = np.zeros(len(d))
    for sp in np.unique(species):
        m = species == sp
        aE[m] = np.einsum("ij,jk,ik->i", d[m], np.abs(beta[sp]), d[m])
        aV[m] = np.einsum("ij,jk,ik->i", d[m], np.abs(sigma[sp]), d[m])
    K = np.where(np.asarray(groups) % 3 == 0, d_full, d_single)
    c = np.array([mixed_coefficient(precision, int(k)) for k in K])
    bE = E_TOL_FP32 * np.maximum(np.abs(E), beta_norm) + c * aE
    bV = V_TOL_FP32 * np.abs(V) + c * aV
    return bE, bV


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


def gpu_run(struct, beta, sigma, precision="fp32", compaction=True, max_nbr=64, n_max=8, want_desc=False,
            fused=None, profile=False, overlap=None):
    import torch
    from paper_2204_12573_gb300 import flare as F
    ff = F.FlareGB(n_max=n_max, precision=precision, compaction=compaction, max_nbr=max_nbr)
    ff.set_model(beta, sigma)
    if fused is not None:
        ff.set_fused(fused)
    if overlap is not None:
        ff.set_overlap(overlap)
    if profile:
        ff.profile(True)
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
    if profile:
        res["profile"] = ff.profile_read()
    torch.cuda.synchronize()
    return res, ff, nl, sysg


def oracle_run(struct, beta, sigma, n_max=8, skin=0.5):
    h = O.Hyper(2, n_max, 3, 4.5)
    pos = synth.f32_exact_f64(synth.as_f32_positions(struct.pos))
    return O.energy_forces(h, pos, struct.species, struct.cell, struct.pbc, beta, sigma, skin=skin)


def compare_mixed(g, o, precision, species, beta, sigma, beta_norm=1.0, f_tol=F_TOL_MIXED, d_full=544,
                  d_single=144):
    """Mixed-precision results against the oracle: forces within f_tol
    (eV/A), energy and variance within the per-atom bounds above."""
    groups = g["group"].cpu().numpy() if hasattr(g["group"], "cpu") else np.asarray(g["group"])
    bE, bV = mixed_bounds(precision, o["dhat"], np.asarray(species), groups, beta, sigma, o["E"], o["V"],
                          d_full=d_full, d_single=d_single, beta_norm=beta_norm)
    dE = np.abs(g["energy"] - o["E"])
    dV = np.abs(g["variance"] - o["V"])
    dF = np.abs(g["forces"] - o["F"]).max()
    assert (dE <= bE).all(), (precision, float((dE / bE).max()))
    assert (dV <= bV).all(), (precision, float((dV / bV).max()))
    assert dF <= f_tol, (precision, float(dF))
    return dict(dE=float(dE.max()), dV=float(dV.max()), dF=float(dF), E_use=float((dE / bE).max()),
                V_use=float((dV / bV).max()))


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
