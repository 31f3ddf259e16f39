"""Python binding of libflare_gb: the calls of include/flare_gb.h with the
same names, on torch CUDA tensors.

PyTorch supplies device memory and streams; every step of the force field
runs in the library's CUDA kernels.  On a machine without the built library
or without a GPU these calls raise instead of falling back to anything.
"""
from __future__ import annotations

import ctypes
import dataclasses

import numpy as np
import torch

from . import _native as N


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


@dataclasses.dataclass
class System:
    """One structure on the device: pos [n, 4] float32 (x, y, z, unused),
    species [n] int32, cell (3, 3) rows = lattice vectors, pbc (3,)."""
    pos: torch.Tensor
    species: torch.Tensor
    cell: np.ndarray
    pbc: tuple = (1, 1, 0)

    @property
    def n_atoms(self):
        return int(self.pos.shape[0])

    def c_struct(self):
        s = N.System()
        s.n_atoms = self.n_atoms
        s.pos = _ptr(self.pos)
        s.species = _ptr(self.species)
        s.cell = (ctypes.c_double * 9)(*np.asarray(self.cell, np.float64).ravel().tolist())
        s.pbc = (ctypes.c_int32 * 3)(*[int(bool(p)) for p in self.pbc])
        return s

    @staticmethod
    def from_numpy(pos4, species, cell, pbc=(1, 1, 0), device="cuda"):
        return System(torch.as_tensor(pos4, dtype=torch.float32, device=device).contiguous(),
                      torch.as_tensor(species, dtype=torch.int32, device=device).contiguous(),
                      np.asarray(cell, np.float64), tuple(pbc))


class FlareGB:
    """A context: hyperparameters, the mapped model (beta, Sigma per species)
    and the device workspace."""

    def __init__(self, n_species=2, n_max=8, l_max=3, r_cut=4.5, skin=0.5, max_nbr=64,
                 precision="bf16x3", compaction=True, device=None):
        self.lib = N.lib()
        if device is None:
            device = torch.cuda.current_device()
        self.device = int(device)
        p = N.Params(n_species, n_max, l_max, max_nbr, r_cut, skin, N.PREC[precision], int(bool(compaction)))
        h = ctypes.c_void_p()
        N.check(self.lib.flr_create(ctypes.byref(p), self.device, ctypes.byref(h)))
        self.handle = h
        self.params = p
        self.r_cut, self.skin, self.max_nbr = r_cut, skin, max_nbr
        self.n_species, self.n_max, self.l_max = n_species, n_max, l_max
        df, ds = ctypes.c_int32(), ctypes.c_int32()
        N.check(self.lib.flr_descriptor_dims(h, ctypes.byref(df), ctypes.byref(ds)))
        self.d_full, self.d_single = df.value, ds.value
        self.precision = precision

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            try:
                self.lib.flr_destroy(h)
            except Exception:
                pass
            self.handle = None

    def set_precision(self, precision: str):
        N.check(self.lib.flr_set_precision(self.handle, N.PREC[precision]))
        self.precision = precision

    def set_fused(self, on: bool):
        """FLR_OPT_FUSED_ONE_SPECIES: one-species atoms in the fused descriptor +
        tensor-core kernel (3xBF16 with compaction), or separate kernels."""
        N.check(self.lib.flr_set_option(self.handle, N.OPT_FUSED_ONE_SPECIES, 1 if on else 0))

    def set_overlap(self, on: bool):
        """FLR_OPT_OVERLAP_TWO_SPECIES: the one-species quadratic-form kernel
        starts beside the two-species one as a programmatic dependent (3xBF16
        with compaction; default on), or after it."""
        N.check(self.lib.flr_set_option(self.handle, N.OPT_OVERLAP_TWO_SPECIES, 1 if on else 0))

    def set_variance_mode(self, mode: str):
        """"auto" (FP32 quadratic form, FP64 re-evaluation of cancelled
        variances), "direct" (FP32 only) or "factored" (V = |L^T d|^2)."""
        N.check(self.lib.flr_set_variance_mode(self.handle, N.VAR_MODE[mode]))

    def set_model(self, beta, sigma):
        """beta, sigma: [n_species, d_full, d_full] float64 (host)."""
        beta = np.ascontiguousarray(beta, np.float64)
        sigma = np.ascontiguousarray(sigma, np.float64)
        for s in range(self.n_species):
            N.check(self.lib.flr_set_model(self.handle, s, beta[s].ctypes.data_as(ctypes.c_void_p),
                                           sigma[s].ctypes.data_as(ctypes.c_void_p)))

    def map_sgp(self, species, d_sparse, alpha, k_ss, sig2, stream=None):
        """Install the mapped sparse GP of one central species (Sec. V-B,
        Eq. 1 and Eq. 2): d_sparse [n_S, d_full], alpha [n_S], k_ss [n_S, n_S],
        float64 CUDA tensors.  Returns the mapped (beta, Sigma) as float64
        CUDA tensors [d_full, d_full]."""
        import torch
        d_sparse = d_sparse.to(device="cuda", dtype=torch.float64).contiguous()
        alpha = alpha.to(device="cuda", dtype=torch.float64).contiguous()
        k_ss = k_ss.to(device="cuda", dtype=torch.float64).contiguous()
        n_s = int(d_sparse.shape[0])
        if d_sparse.shape != (n_s, self.d_full) or alpha.shape != (n_s,) or k_ss.shape != (n_s, n_s):
            raise ValueError("map_sgp: shapes must be d_sparse [n_S, d_full], alpha [n_S], k_ss [n_S, n_S]")
        beta = torch.empty((self.d_full, self.d_full), dtype=torch.float64, device="cuda")
        sigma = torch.empty_like(beta)
        N.check(self.lib.flr_map_sgp(self.handle, int(species), n_s, _ptr(d_sparse), _ptr(alpha), _ptr(k_ss),
                                     float(sig2), _ptr(beta), _ptr(sigma), _stream(stream)))
        return beta, sigma

    def nbrlist(self, n_atoms):
        return NbrList(self, n_atoms)

    def launch_count(self):
        return int(self.lib.flr_launch_count(self.handle))

    def sync(self, stream=None):
        N.check(self.lib.flr_sync(self.handle, _stream(stream)))

    def profile(self, on: bool):
        """Per-kernel CUDA-event timing on the launching stream (clears totals when turned on)."""
        N.check(self.lib.flr_profile_enable(self.handle, int(bool(on))))

    def profile_read(self):
        """{kernel class: (total ms, launches)} accumulated since profiling was enabled."""
        out = {}
        for k, name in enumerate(N.KERNEL_CLASSES):
            ms, cnt = ctypes.c_double(), ctypes.c_int64()
            N.check(self.lib.flr_profile_read(self.handle, k, ctypes.byref(ms), ctypes.byref(cnt)))
            out[name] = (ms.value, cnt.value)
        return out


class NbrList:
    def __init__(self, ff: FlareGB, n_atoms: int):
        self.ff = ff
        h = ctypes.c_void_p()
        N.check(ff.lib.flr_nbrlist_create(ff.handle, int(n_atoms), ctypes.byref(h)))
        self.handle = h
        self.n_cap = int(n_atoms)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            try:
                self.ff.lib.flr_nbrlist_destroy(h)
            except Exception:
                pass
            self.handle = None

    def view(self, n_atoms):
        """(entries [n, max_nbr], count [n], group [n]) as int32 torch tensors
        (copies, made after synchronizing the current stream)."""
        e, c, g = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
        m = ctypes.c_int32()
        N.check(self.ff.lib.flr_nbrlist_view(self.handle, ctypes.byref(e), ctypes.byref(c), ctypes.byref(g),
                                             ctypes.byref(m)))
        torch.cuda.current_stream().synchronize()
        return tuple(_device_view(ptr.value, shape).clone()
                     for ptr, shape in ((e, (n_atoms, m.value)), (c, (n_atoms,)), (g, (n_atoms,))))


class _CudaArray:
    """Minimal __cuda_array_interface__ wrapper of library-owned int32 memory."""

    def __init__(self, ptr, shape):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": "<i4", "data": (int(ptr), False),
                                         "version": 2, "strides": None}


def _device_view(ptr, shape):
    if int(np.prod(shape)) == 0:
        return torch.empty(shape, dtype=torch.int32, device="cuda")
    return torch.as_tensor(_CudaArray(ptr, shape), device="cuda")


def build_neighbors(ff: FlareGB, system: System, nl: NbrList, stream=None):
    """Cell-list neighbour search and compaction classification (synchronizes)."""
    s = system.c_struct()
    N.check(ff.lib.flr_build_neighbors(ff.handle, ctypes.byref(s), nl.handle, _stream(stream)))


def build_neighbors_noalloc(system: System, r_list: float, max_nbr: int, entries, count, stream=None):
    """Neighbour list into caller-provided int32 tensors (entries [n, max_nbr],
    count [n]) without any device allocation by the library; synchronizes.
    Meant for callers that cannot allocate device memory (see include/flare_gb.h
    for the size limits and the shared-scratch caveat)."""
    s = system.c_struct()
    N.check(N.lib().flr_build_neighbors_noalloc(ctypes.byref(s), float(r_list), int(max_nbr), _ptr(entries),
                                                _ptr(count), _stream(stream)))


def compute_descriptors(ff: FlareGB, system: System, nl: NbrList, stream=None):
    """Normalized B2 descriptors [n, d_full] (float32) and norms ||B|| [n]."""
    n = system.n_atoms
    d = torch.empty((n, ff.d_full), dtype=torch.float32, device="cuda")
    norm = torch.empty((n,), dtype=torch.float32, device="cuda")
    s = system.c_struct()
    N.check(ff.lib.flr_compute_descriptors(ff.handle, ctypes.byref(s), nl.handle, _ptr(d), _ptr(norm),
                                           _stream(stream)))
    return d, norm


def make_outputs(n, device="cuda"):
    return dict(energy=torch.empty(n, dtype=torch.float32, device=device),
                forces=torch.empty((n, 3), dtype=torch.float32, device=device),
                variance=torch.empty(n, dtype=torch.float32, device=device),
                sigma=torch.empty(n, dtype=torch.float32, device=device),
                totals=torch.zeros(N.NTOTALS, dtype=torch.float64, device=device))


def _outputs_struct(out):
    o = N.Outputs()
    o.energy = _ptr(out["energy"])
    o.forces = _ptr(out["forces"])
    o.variance = _ptr(out.get("variance"))
    o.sigma = _ptr(out.get("sigma"))
    o.totals = _ptr(out.get("totals"))
    return o


def energy_forces_uncertainty(ff: FlareGB, system: System, nl: NbrList, out=None, stream=None):
    """Per-atom energy, forces, variance, sigma and FP64 totals (asynchronous)."""
    if out is None:
        out = make_outputs(system.n_atoms)
    s = system.c_struct()
    o = _outputs_struct(out)
    N.check(ff.lib.flr_energy_forces_uncertainty(ff.handle, ctypes.byref(s), nl.handle, ctypes.byref(o),
                                                 _stream(stream)))
    return out


class MDState:
    """Velocity-Verlet state: pos, vel [n, 4] float32 device tensors updated in place."""

    def __init__(self, system: System, vel: torch.Tensor, masses=(195.084, 1.008), dt=0.0005,
                 rebuild_every=10, temperature=0.0, tau=0.1, sigma_stop=0.0, cn_species=-1, cn_cutoff=1.0):
        """temperature > 0: Nose-Hoover NVT with period tau (ps); sigma_stop > 0:
        stop after the first step with an atom's sigma above it; cn_species >= 0:
        count atoms of that species with a same-species neighbour within
        cn_cutoff (A) after every step."""
        self.system = system
        self.vel = vel
        self.c = N.MDState()
        c = self.c
        c.n_atoms = system.n_atoms
        c.pos = _ptr(system.pos)
        c.vel = _ptr(vel)
        c.species = _ptr(system.species)
        c.cell = (ctypes.c_double * 9)(*np.asarray(system.cell, np.float64).ravel().tolist())
        c.pbc = (ctypes.c_int32 * 3)(*[int(bool(p)) for p in system.pbc])
        m = list(masses) + [1.0] * (8 - len(masses))
        c.masses = (ctypes.c_double * 8)(*m)
        c.dt = dt
        c.rebuild_every = rebuild_every
        c.forces_valid = 0
        c.step = 0
        c.temperature = temperature
        c.tau = tau
        c.xi = 0.0
        c.eta = 0.0
        c.sigma_stop = sigma_stop
        c.halted = 0
        c.cn_species = cn_species
        c.cn_cutoff = cn_cutoff

    @property
    def step(self):
        return int(self.c.step)

    @property
    def halted(self):
        return bool(self.c.halted)

    @property
    def xi(self):
        return float(self.c.xi)

    @property
    def eta(self):
        return float(self.c.eta)


def md_step(ff: FlareGB, state: MDState, nl: NbrList, n_steps: int, out, stream=None):
    """n_steps of velocity Verlet with on-device rebuild decisions (asynchronous)."""
    o = _outputs_struct(out)
    N.check(ff.lib.flr_md_step(ff.handle, ctypes.byref(state.c), nl.handle, int(n_steps), ctypes.byref(o),
                               _stream(stream)))
    return out


class HostState:
    """MD state and results in page-locked host memory for md_step_host:
    pos, vel [n, 3] float32 (read before and written after every step) and
    the last step's energy [n], forces [n, 3], variance [n], sigma [n] and
    totals [FLR_NTOTALS] (float64); `results` names the ones to read back."""

    def __init__(self, pos, vel, results=("energy", "forces", "sigma")):
        n = int(pos.shape[0])
        self.pos = torch.empty((n, 3), dtype=torch.float32).pin_memory()
        self.vel = torch.empty((n, 3), dtype=torch.float32).pin_memory()
        self.pos.copy_(torch.as_tensor(pos, dtype=torch.float32)[:, :3])
        self.vel.copy_(torch.as_tensor(vel, dtype=torch.float32)[:, :3])
        shapes = {"energy": (n,), "forces": (n, 3), "variance": (n,), "sigma": (n,), "totals": (N.NTOTALS,)}
        self.results = {}
        for k in results:
            dt = torch.float64 if k == "totals" else torch.float32
            self.results[k] = torch.zeros(shapes[k], dtype=dt).pin_memory()
        c = N.HostState()
        c.pos = self.pos.data_ptr()
        c.vel = self.vel.data_ptr()
        for k, v in self.results.items():
            setattr(c, k, v.data_ptr())
        self.c = c

    def __getitem__(self, k):
        return self.results[k]


def md_step_host(ff: FlareGB, state: MDState, nl: NbrList, n_steps: int, out, host: HostState, stream=None):
    """n_steps of velocity Verlet with the state in host memory: each step
    uploads host.pos / host.vel, steps on the device (state.system.pos and
    state.vel are the working copies) and downloads the new state; the last
    step's results follow.  Asynchronous: read `host` after ff.sync() or
    host_join + a synchronize."""
    o = _outputs_struct(out)
    N.check(ff.lib.flr_md_step_host(ff.handle, ctypes.byref(state.c), nl.handle, int(n_steps), ctypes.byref(o),
                                    ctypes.byref(host.c), _stream(stream)))
    return out


def host_join(ff: FlareGB, stream=None):
    """Make `stream` wait for every copy md_step_host has enqueued."""
    N.check(ff.lib.flr_host_join(ff.handle, _stream(stream)))


def sync(ff: FlareGB, stream=None):
    ff.sync(stream)


class Batch:
    """Several structures of different sizes and cells evaluated together.

    Atoms are concatenated on the device (pos [n, 4] float32, species [n]
    int32); offsets, cells and pbc stay on the host (they describe the batch
    to the library, which copies what the kernels need)."""

    def __init__(self, pos, species, offsets, cells, pbc):
        self.pos = pos
        self.species = species
        self.offsets = np.ascontiguousarray(offsets, np.int32)
        self.cells = np.ascontiguousarray(np.asarray(cells, np.float64).reshape(-1, 9))
        self.pbc = np.ascontiguousarray(np.asarray(pbc, np.int32).reshape(-1, 3))

    @property
    def n_atoms(self):
        return int(self.pos.shape[0])

    @property
    def n_structs(self):
        return int(len(self.offsets) - 1)

    @staticmethod
    def from_structures(structs, device="cuda"):
        """structs: objects with .pos (float64 [n, 3]), .species, .cell, .pbc."""
        from .synth import as_f32_positions
        pos = np.concatenate([as_f32_positions(s.pos) for s in structs], axis=0)
        sp = np.concatenate([np.asarray(s.species, np.int32) for s in structs])
        offsets = np.concatenate([[0], np.cumsum([len(s.species) for s in structs])]).astype(np.int32)
        return Batch(torch.as_tensor(pos, device=device), torch.as_tensor(sp, device=device), offsets,
                     np.stack([np.asarray(s.cell, np.float64).ravel() for s in structs]),
                     np.stack([np.asarray(s.pbc, np.int32) for s in structs]))

    def c_struct(self):
        b = N.Batch()
        b.n_structs = self.n_structs
        b.n_atoms = self.n_atoms
        b.pos = _ptr(self.pos)
        b.species = _ptr(self.species)
        b.offsets = self.offsets.ctypes.data_as(ctypes.c_void_p)
        b.cells = self.cells.ctypes.data_as(ctypes.c_void_p)
        b.pbc = self.pbc.ctypes.data_as(ctypes.c_void_p)
        return b


def build_neighbors_batch(ff: FlareGB, batch: Batch, nl: NbrList, stream=None):
    """Neighbour lists of every structure of a batch (synchronizes once)."""
    b = batch.c_struct()
    N.check(ff.lib.flr_build_neighbors_batch(ff.handle, ctypes.byref(b), nl.handle, _stream(stream)))


def energy_forces_uncertainty_batch(ff: FlareGB, batch: Batch, nl: NbrList, out=None, stream=None):
    """Per-atom outputs over the whole batch; out["totals"] is [n_structs, NTOTALS]."""
    if out is None:
        out = make_outputs(batch.n_atoms)
        out["totals"] = torch.zeros((batch.n_structs, N.NTOTALS), dtype=torch.float64, device="cuda")
    b = batch.c_struct()
    o = _outputs_struct(out)
    N.check(ff.lib.flr_energy_forces_uncertainty_batch(ff.handle, ctypes.byref(b), nl.handle, ctypes.byref(o),
                                                       _stream(stream)))
    return out


def energy_backward(ff: FlareGB, batch: Batch, nl: NbrList, grad_energy, want_beta=True, stream=None):
    """(dL/dpos [n, 3], dL/dbeta [S, d, d] or None) for L = sum_i grad_energy[i] * E_i."""
    n = batch.n_atoms
    gpos = torch.empty((n, 3), dtype=torch.float32, device="cuda")
    gbeta = (torch.empty((ff.n_species, ff.d_full, ff.d_full), dtype=torch.float32, device="cuda")
             if want_beta else None)
    u = grad_energy.detach().to(device="cuda", dtype=torch.float32).contiguous()
    b = batch.c_struct()
    N.check(ff.lib.flr_energy_backward(ff.handle, ctypes.byref(b), nl.handle, _ptr(u), _ptr(gpos), _ptr(gbeta),
                                       _stream(stream)))
    return gpos, gbeta


def fp32_fma_peak(device=0, launches=10):
    """Measured FP32 FMA rate of a device (flr_fp32_fma_peak): best and
    median TFLOP/s over `launches` timed launches, and the SM count."""
    best, med, sms = ctypes.c_double(), ctypes.c_double(), ctypes.c_int32()
    N.check(N.lib().flr_fp32_fma_peak(int(device), int(launches), ctypes.byref(best), ctypes.byref(med),
                                      ctypes.byref(sms)))
    return {"tflops_best": best.value, "tflops_median": med.value, "num_sms": sms.value}
