"""FP64 CPU oracle for the FLARE energy / force / uncertainty path.

TEST INFRASTRUCTURE ONLY: the tests, the package smoke check and the
benchmark's CPU-baseline leg may import this package; the product path
(`paper_2204_12573_gb300`) never does, and this package never imports it.

The arithmetic lives in `flare_oracle.c` (plain double-precision C, OpenMP
over centre atoms) and `sgp.py` (the unmapped sparse-GP sums of Eq. 1 and
Eq. 2, numpy).  This module compiles the C file with gcc on first use and
wraps it with ctypes.

Each function is pinned by the `-m "not gpu"` tests in tests/test_oracle_*.py.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "flare_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, -O2, OpenMP, no FMA contraction)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
           "-std=c11", "-D_GNU_SOURCE", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            lib.orc_neighbors_brute.restype = ctypes.c_long
            lib.orc_neighbors_brute.argtypes = [ctypes.c_int, P, P, P, ctypes.c_double, ctypes.c_long, P]
            lib.orc_neighbors_cells.restype = ctypes.c_long
            lib.orc_neighbors_cells.argtypes = [ctypes.c_int, P, P, P, ctypes.c_double,
                                                ctypes.c_int, P, ctypes.c_long, P]
            lib.orc_evaluate.restype = ctypes.c_int
            lib.orc_evaluate.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                         ctypes.c_int, P, P, P, ctypes.c_long, P, P, P, P,
                                         ctypes.c_int, P, P, P, P, P, P, P, P]
            lib.orc_assemble.restype = None
            lib.orc_assemble.argtypes = [ctypes.c_int, ctypes.c_long, P, P, P, P, P, P]
            lib.orc_basis_point.restype = None
            lib.orc_basis_point.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, P, P, P]
            lib.orc_ylm_point.restype = None
            lib.orc_ylm_point.argtypes = [ctypes.c_int, P, P]
            lib.orc_max_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def max_threads() -> int:
    return int(_load().orc_max_threads())


def neighbors(pos, cell, pbc, rc, centers=None, method="cells"):
    """Neighbour pairs [m, 5] int32 rows (i, j, sx, sy, sz), sorted, with
    |r_j + S.cell - r_i| < rc.  method: "brute" (O(N^2) over images) or
    "cells" (cell list; periodic coordinates must lie inside the cell)."""
    lib = _load()
    pos = _c(pos, np.float64)
    cell = _c(cell, np.float64)
    pbc_a = _c(pbc, np.int32)
    n = pos.shape[0]
    cap = max(1024, 64 * (n if centers is None else len(centers)))
    while True:
        out = np.empty((cap, 5), np.int32)
        if method == "brute":
            assert centers is None
            cnt = lib.orc_neighbors_brute(n, _p(pos), _p(cell), _p(pbc_a), rc, cap, _p(out))
        else:
            cen = None if centers is None else _c(centers, np.int32)
            cnt = lib.orc_neighbors_cells(n, _p(pos), _p(cell), _p(pbc_a), rc,
                                          0 if cen is None else len(cen), _p(cen), cap, _p(out))
        if cnt <= cap:
            return out[:cnt].copy()
        cap = int(cnt) + 16


class Hyper:
    """Descriptor hyperparameters: species count S, radial functions N,
    maximum angular momentum L, cutoff r_cut (A)."""

    def __init__(self, n_species=2, n_max=8, l_max=3, r_cut=4.5):
        self.n_species, self.n_max, self.l_max, self.r_cut = n_species, n_max, l_max, r_cut

    @property
    def n_channels(self):
        return self.n_species * self.n_max

    @property
    def d(self):
        c = self.n_channels
        return c * (c + 1) // 2 * (self.l_max + 1)

    @property
    def n_a(self):
        return self.n_channels * (self.l_max + 1) ** 2


def evaluate(h: Hyper, pos, species, cell, pairs, beta, sigma, flag=None, n_threads=0,
             want_forces=True):
    """Evaluate centres (all, or those with flag != 0).  Returns a dict with
    A, B, dhat, norm, E, V (per atom; rows of skipped centres are zero),
    fpair (dE_i/dr_ij per pair) and rij (per pair)."""
    lib = _load()
    pos = _c(pos, np.float64)
    species = _c(species, np.int32)
    cell = _c(cell, np.float64)
    pairs = _c(pairs, np.int32)
    beta = _c(beta, np.float64)
    sigma = _c(sigma, np.float64)
    n = pos.shape[0]
    m = pairs.shape[0]
    fl = None if flag is None else _c(flag, np.int32)
    out = dict(A=np.zeros((n, h.n_a)), B=np.zeros((n, h.d)), dhat=np.zeros((n, h.d)),
               norm=np.zeros(n), E=np.zeros(n), V=np.zeros(n),
               fpair=np.zeros((m, 3)) if want_forces else None, rij=np.zeros((m, 3)))
    st = lib.orc_evaluate(h.n_species, h.n_max, h.l_max, h.r_cut, n, _p(pos), _p(species), _p(cell),
                          m, _p(pairs), _p(beta), _p(sigma), _p(fl), int(n_threads),
                          _p(out["A"]), _p(out["B"]), _p(out["dhat"]), _p(out["norm"]),
                          _p(out["E"]), _p(out["V"]), _p(out["fpair"]), _p(out["rij"]))
    if st != 0:
        raise RuntimeError(f"orc_evaluate failed with status {st}")
    return out


def assemble(n, pairs, rij, fpair, flag=None):
    """Forces F [n, 3] and virial W [3, 3] from per-pair dE_i/dr_ij."""
    lib = _load()
    pairs = _c(pairs, np.int32)
    rij = _c(rij, np.float64)
    fpair = _c(fpair, np.float64)
    fl = None if flag is None else _c(flag, np.int32)
    F = np.zeros((n, 3))
    W = np.zeros(9)
    lib.orc_assemble(n, pairs.shape[0], _p(pairs), _p(rij), _p(fpair), _p(fl), _p(F), _p(W))
    return F, W.reshape(3, 3)


def energy_forces(h: Hyper, pos, species, cell, pbc, beta, sigma, skin=0.0, method="cells",
                  n_threads=0):
    """Whole-system oracle: neighbours, per-atom E, V, sigma, forces, virial.
    Returns a dict (E, V, sigma, F, W, E_tot, dhat, norm, pairs)."""
    pairs = neighbors(pos, cell, pbc, h.r_cut + skin, method=method)
    o = evaluate(h, pos, species, cell, pairs, beta, sigma, n_threads=n_threads)
    F, W = assemble(len(pos), pairs, o["rij"], o["fpair"])
    o.update(F=F, W=W, E_tot=float(o["E"].sum()), sigma=np.sqrt(np.maximum(o["V"], 0.0)),
             pairs=pairs)
    return o


def forces_subset(h: Hyper, pos, species, cell, pbc, beta, sigma, atoms, skin=0.0, n_threads=0):
    """Per-atom E, V and full forces for the listed atoms of a large system.

    F_k needs dE_i/dr_k from k itself and from every neighbour i of k, so the
    oracle evaluates k and its neighbours (within r_cut) as centres.  Returns
    dict(atoms, E, V, F, dhat, norm) for the listed atoms only."""
    atoms = np.asarray(atoms, np.int64)
    rc = h.r_cut + skin
    first = neighbors(pos, cell, pbc, rc, centers=atoms)
    centres = np.unique(np.concatenate([atoms, first[:, 1]]))
    pairs = neighbors(pos, cell, pbc, rc, centers=centres)
    flag = np.zeros(len(pos), np.int32)
    flag[centres] = 1
    o = evaluate(h, pos, species, cell, pairs, beta, sigma, flag=flag, n_threads=n_threads)
    F, W = assemble(len(pos), pairs, o["rij"], o["fpair"], flag=flag)
    return dict(atoms=atoms, E=o["E"][atoms], V=o["V"][atoms], F=F[atoms],
                dhat=o["dhat"][atoms], norm=o["norm"][atoms], A=o["A"][atoms])


def basis_point(h: Hyper, r):
    """phi[n, lm] and dphi[n, lm, 3] for one neighbour vector r (complex step)."""
    lib = _load()
    r = _c(r, np.float64)
    nlm = (h.l_max + 1) ** 2
    phi = np.zeros(h.n_max * nlm)
    dphi = np.zeros(h.n_max * nlm * 3)
    lib.orc_basis_point(h.n_max, h.l_max, h.r_cut, _p(r), _p(phi), _p(dphi))
    return phi.reshape(h.n_max, nlm), dphi.reshape(h.n_max, nlm, 3)


def ylm(l_max, u):
    """Real orthonormal Y_lm (index l*l + m + l) of a real unit vector u."""
    lib = _load()
    u = _c(u, np.float64)
    Y = np.zeros((l_max + 1) ** 2)
    lib.orc_ylm_point(l_max, _p(u), _p(Y))
    return Y
