#!/usr/bin/env python
"""Benchmark: velocity-Verlet MD with the FLARE force field on one GB300.

Workload: a 2,129,920-atom H2/Pt(111) slab (256 x 256 atoms per layer x 32
layers of Pt plus 16,384 H2 molecules in the gas above), 300 K Maxwell
velocities, dt = 0.5 fs, neighbour list rebuilt every 10 steps (skin 0.5 A,
plus a device-side displacement trigger).  One step = half kick + drift +
(conditional) rebuild + energy / forces / uncertainty + half kick.

Headline `value`: M atom-steps/s with the quadratic forms on the tensor
cores in 3xBF16 (FP32 accumulate); `plain_fp32` gives the same run with the
FP32 SIMT quadratic forms, `compaction_off` the 3xBF16 run with every atom
at the two-species descriptor size (no species-block compaction), and
`force_err_ev_per_A` the force error of each precision against the FP64
oracle on sampled atoms.  Inputs are larger than L2 (the
neighbour list alone is 545 MB), so no L2 flush is needed between steps.

`--impl reference` times the FP64 CPU oracle on bounded samples of the same
workload instead (the reference arm).  Under torchrun every rank runs an
independent replica (the path has no data exchange on one GPU per replica).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("M atom-steps/s (E+F+σ) mixed vs plain FP32 at ≤1e-3 eV/Å force err; p50/p99 ms")
UNIT = "M atom-steps/s"


def _env_rank():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def max_over_ranks(ms, dist=None, device="cuda"):
    """The slowest rank's time, which is the job's time (identity for one process)."""
    if dist is None:
        return float(ms)
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, atoms_per_rank, steps, ms):
    """Whole-job M atom-steps/s: every replica's atom-steps over the slowest replica's time."""
    return world * atoms_per_rank * steps / (ms / 1e3) / 1e6


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0}, "fallback"


class Clocks:
    """nvidia-smi clock / throttle sampling during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        # raw samples; the summary goes into the JSON line
        self.path = os.path.join(os.environ.get("BENCH_CLOCKS_DIR", tempfile.gettempdir()),
                                 f"flare_gb_clocks_{os.getpid()}.csv")

    def __enter__(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                try:
                    rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
                except ValueError:
                    pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for _, _, r in rows for k in range(4) if r[k].lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def _source_hash(files):
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _traffic_per_atom(kernel):
    """DRAM bytes per atom of `kernel` from the committed ncu summary, if it was
    taken on the current source of that kernel (else None)."""
    p = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(p):
        return None
    for line in open(p):
        if line.startswith("#") or "=" not in line:
            continue
        kv = dict(x.split("=", 1) for x in line.split())
        if kv.get("kernel") == kernel:
            srcs = kv.get("sources", "").split(",")
            try:
                if _source_hash(srcs) != kv.get("hash"):
                    return None
            except OSError:
                return None
            return float(kv["bytes_per_atom"])
    return None


# Algorithmic work of one launch, from the method (not from what the kernels
# execute).  N = 8 radial functions, 16 real harmonics (l <= 3); p = pairs
# inside r_cut per atom; C_g = radial channels of the atom's class (16 for a
# two-species environment, 8 for a one-species one); K = descriptor length
# of the class (544 or 144).
#   descriptor, per pair: A_{n,lm} += R_n Y_lm            2 N 16 flop
#                         geometry, R_n f_c, Y_lm           70 flop
#               per atom: B2 = sum_m A A (C_g(C_g+1)/2 channel pairs x 16 m
#                         products) 32 C_g(C_g+1)/2 flop, norm and scaling 3 K flop
#   quadratic forms, per atom: P = d [beta | Sigma]        2 K (2K) flop
#   force, per pair: c_lm, c'_lm = sum_n w (R_n, R'_n)     4 N 16 flop
#                    geometry, radial with derivatives, Y_lm and grad P_lm,
#                    the three l-weighted sums, f_ij        325 flop
#          per atom: w = G~ A                               2 C_g^2 16 flop
DESC_PAIR = 2 * 8 * 16 + 70
FORCE_PAIR = 4 * 8 * 16 + 325


def _class_counts(groups):
    g = np.bincount(groups + 1, minlength=7)[1:]   # counts of the 6 compaction groups
    return int(g[0] + g[3]), int(g[1] + g[2] + g[4] + g[5])


def _algorithmic(kernel, groups, n_atoms, d_full, d_single, pairs_per_atom):
    """Algorithmic FLOPs of one launch of `kernel` (see the table above)."""
    n_full, n_single = _class_counts(groups)
    if kernel == "qform":
        return 2.0 * (n_full * d_full * 2 * d_full + n_single * d_single * 2 * d_single)
    if kernel == "force":
        return float(n_atoms * pairs_per_atom * FORCE_PAIR + n_full * 2 * 16 * 16 * 16 + n_single * 2 * 8 * 8 * 16)
    if kernel == "descriptor":
        # 32 flop per channel pair and d = 4 x channel pairs: 8 d + 3 d per atom
        return float(n_atoms * pairs_per_atom * DESC_PAIR + n_full * 11 * d_full + n_single * 11 * d_single)
    return None


def _pairs_within_cutoff(nl, sysg, n, r_cut):
    """Number of list entries with |r_ij| < r_cut (the pairs the descriptor
    and force kernels evaluate), counted with torch from the list view."""
    import torch
    entries, count, _ = nl.view(n)
    pos = sysg.pos[:, :3]
    cell = torch.as_tensor(np.asarray(sysg.cell), dtype=torch.float64, device="cuda")
    total = 0
    for a in range(0, n, 1 << 18):
        b = min(n, a + (1 << 18))
        e = entries[a:b].long()
        valid = torch.arange(e.shape[1], device="cuda")[None, :] < count[a:b, None]
        j = e >> 8               # entry = (j << 8) | (s_j << 7) | image code
        code = e & 127
        s = torch.stack([code // 25 - 2, (code // 5) % 5 - 2, code % 5 - 2], -1).double()
        r = (pos[j.clamp(0, n - 1)].double() + s @ cell - pos[a:b, None, :].double())
        d2 = (r * r).sum(-1)
        total += int(((d2 < r_cut * r_cut) & valid).sum().item())
    return total


def measure_fp32_peak(device):
    """FP32 FMA peak measured on this device (flr_fp32_fma_peak: all SMs, 8
    independent register-resident FMA chains per thread, best of 20 timed
    launches), with the SM clock sampled while it runs."""
    from paper_2204_12573_gb300 import flare as F
    clocks = Clocks(device)
    with clocks:
        r = F.fp32_fma_peak(device, 20)
    r["clocks"] = clocks.summary()
    r["nominal_tflops"] = r["num_sms"] * 128 * 2 * (r["clocks"].get("sm_max_mhz") or 2070.0) * 1e6 / 1e12
    r["note"] = ("flr_fp32_fma_peak: every SM at its occupancy limit, 8 independent FMA chains per thread, "
                 "best of 20 launches timed with CUDA events; nominal = SMs x 128 lanes x 2 x max SM clock")
    return r


class OracleSample:
    """The FP64 oracle (cell-list neighbours + E/F/sigma) timed on a compact
    column of the slab, sized from a pilot run to take about target_s."""

    def __init__(self, struct, beta, sigma):
        import oracle as O
        from paper_2204_12573_gb300 import synth
        self.O = O
        self.struct, self.beta, self.sigma = struct, beta, sigma
        self.pos = synth.f32_exact_f64(synth.as_f32_positions(struct.pos))
        self.h = O.Hyper()
        self.cores = O.max_threads()   # all host cores (OpenMP default), before any 1-thread run
        # two pilots give the fixed cost (neighbour search over the whole slab) and the cost per atom
        self.t_fixed, self.t_atom = 0.0, 1e-3
        pts = []
        for side in (10.0, 25.0):
            blk = self._block(side)
            t0 = time.time()
            self._run(blk)
            pts.append((len(blk), time.time() - t0))
        (n1, t1), (n2, t2) = pts
        self.t_atom = max((t2 - t1) / max(n2 - n1, 1), 1e-7)
        self.t_fixed = max(t1 - self.t_atom * n1, 0.0)

    def _block(self, side):
        return np.nonzero((self.pos[:, 0] < side) & (self.pos[:, 1] < side))[0]

    def _run(self, atoms, n_threads=0):
        s = self.struct
        self.O.forces_subset(self.h, self.pos, s.species, s.cell, s.pbc, self.beta, self.sigma, atoms, skin=0.5,
                             n_threads=n_threads or self.cores)

    def step(self, target_s):
        n25 = len(self._block(25.0))
        want = max(target_s - self.t_fixed, 0.1 * target_s) / self.t_atom
        side = float(np.clip(25.0 * np.sqrt(want / max(n25, 1)), 10.0, 300.0))
        blk = self._block(side)
        t0 = time.time()
        self._run(blk)
        dt = time.time() - t0
        return {"value": len(blk) / dt / 1e6, "unit": UNIT, "cores": self.cores, "kind": "oracle",
                "seconds": round(dt, 2),
                "sample": f"{len(blk)} atoms (x,y < {side:.1f} A column of the slab, Pt and H): cell-list "
                          f"neighbours over all atoms + FP64 E/F/sigma of the column, one step"}


    def one_core(self, target_s):
        """The same kind of step on one thread, on a column sized for about target_s."""
        n25 = len(self._block(25.0))
        want = target_s / (self.t_atom * self.cores)
        side = float(np.clip(25.0 * np.sqrt(want / max(n25, 1)), 10.0, 300.0))
        blk = self._block(side)
        t0 = time.time()
        self._run(blk, n_threads=1)
        dt = time.time() - t0
        return len(blk) / dt / 1e6, f"{len(blk)} atoms (x,y < {side:.1f} A column), 1 thread, {dt:.2f} s"


def cpu_baseline_sample(struct, beta, sigma, target_s=12.0):
    samp = OracleSample(struct, beta, sigma)
    r = samp.step(target_s)
    v1, s1 = samp.one_core(4.0)
    r["value_1core"] = v1
    r["sample_1core"] = s1
    return r


def run_reference(args):
    rank, world, _ = _env_rank()
    if rank != 0:
        return
    from paper_2204_12573_gb300 import synth
    struct = synth.big_slab(seed=1)
    beta, sigma = synth.random_model()
    samp = OracleSample(struct, beta, sigma)          # pilot run doubles as warm-up
    per_step = float(np.clip(150.0 / max(args.steps + args.warmup, 1), 1.0, args.ref_seconds))
    for _ in range(args.warmup):
        samp.step(0.25 * per_step)
    vals = []
    cb = None
    for k in range(max(args.steps, 1)):
        cb = samp.step(per_step)
        vals.append(cb["value"])
    v = statistics.median(vals)
    cb["value"] = v
    cb["sample"] += f"; median of {len(vals)} steps"
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": None, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": _config(struct.n_atoms, "f64 oracle"), "cpu_baseline": cb,
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _config(n_atoms, precision):
    return {"workload": f"H2/Pt(111) slab 256x256 atoms/layer x 32 layers + 16384 H2 = {n_atoms} atoms; "
                        "velocity Verlet dt=0.5 fs, 300 K, rebuild every 10 steps, skin 0.5 A, r_cut 4.5 A, "
                        "n_max 8, l_max 3 (d=544/144)",
            "n_atoms": n_atoms, "precision": precision, "l2": "inputs larger than L2 (no flush)",
            "parallelism": "replicas"}


def run_ours(args):
    import torch
    rank, world, local = _env_rank()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2204_12573_gb300 import build
    build.build()
    import oracle as O
    from paper_2204_12573_gb300 import flare as F
    from paper_2204_12573_gb300 import synth
    from paper_2204_12573_gb300 import _native as N

    if args.small:
        struct = synth.big_slab(seed=1, nx=64, n_rows=64, n_layers=32, n_h2=1024)
    else:
        struct = synth.big_slab(seed=1)
    n = struct.n_atoms
    beta, sigma = synth.random_model()
    pos0 = synth.as_f32_positions(struct.pos)
    vel0 = synth.maxwell_velocities(struct.species, 300.0, seed=1)
    ff = F.FlareGB(precision="bf16x3", max_nbr=64)
    ff.set_model(beta, sigma)
    sysg = F.System.from_numpy(pos0, struct.species, struct.cell, struct.pbc)
    vel = torch.as_tensor(vel0, device="cuda")
    nl = ff.nbrlist(n)
    out = F.make_outputs(n)
    stream = torch.cuda.current_stream()

    def reset():
        sysg.pos.copy_(torch.as_tensor(pos0, device="cuda"))
        vel.copy_(torch.as_tensor(vel0, device="cuda"))
        F.build_neighbors(ff, sysg, nl)
        return F.MDState(sysg, vel)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    rebuild_count = {}

    def timed(precision, profile=False, clocks=None):
        ff.set_precision(precision)
        st = reset()
        F.md_step(ff, st, nl, args.warmup, out)
        ff.sync()
        if profile:
            ff.profile(True)
        l0 = ff.launch_count()
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if clocks:
            clocks.__enter__()
        e0.record(stream)
        F.md_step(ff, st, nl, args.steps, out)
        e1.record(stream)
        barrier()
        if clocks:
            clocks.__exit__()
        ms = e0.elapsed_time(e1)
        rebuild_count[precision] = int(out["totals"][13].item())
        # host-counted launches, plus the rebuild kernels the conditional graph ran on rebuild steps
        launches = ff.launch_count() - l0 + rebuild_count[precision] * N.REBUILD_KERNELS
        prof = None
        if profile:
            prof = ff.profile_read()
            ff.profile(False)
        ff.sync()
        ms = max_over_ranks(ms, dist)
        return ms, launches, prof, st

    if args.profile_run:
        # the mixed-precision timed region only (for launch lists and ncu captures)
        ff.set_fused(args.fused)
        ms, launches, _, _ = timed(args.precision)
        if rank == 0:
            print(json.dumps({"profile_run": True, "n_atoms": n, "precision": args.precision,
                              "ms_per_step": ms / args.steps, "launches": launches}), flush=True)
        return
    clocks = Clocks(torch.cuda.current_device())
    ms_mix, launches, _, st_mix = timed("bf16x3", clocks=clocks)
    clk = clocks.summary()
    _, _, prof_mix, _ = timed("bf16x3", profile=True)
    ms_fp32, _, _, _ = timed("fp32", profile=False)
    _, _, prof_fp32, _ = timed("fp32", profile=True)

    value = job_throughput(world, n, args.steps, ms_mix)
    value_fp32 = job_throughput(world, n, args.steps, ms_fp32)

    # compaction off: every atom takes the two-species (d = 544) descriptor,
    # the paper's method without its species-block compaction (own context)
    def timed_no_compaction(steps):
        ffn = F.FlareGB(precision="bf16x3", max_nbr=64, compaction=False)
        ffn.set_model(beta, sigma)
        nln = ffn.nbrlist(n)
        res = []
        for profile in (False, True):
            sysg.pos.copy_(torch.as_tensor(pos0, device="cuda"))
            vel.copy_(torch.as_tensor(vel0, device="cuda"))
            F.build_neighbors(ffn, sysg, nln)
            stn = F.MDState(sysg, vel)
            F.md_step(ffn, stn, nln, args.warmup, out)
            ffn.sync()
            if profile:
                ffn.profile(True)
            barrier()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            F.md_step(ffn, stn, nln, steps, out)
            e1.record(stream)
            barrier()
            res.append(max_over_ranks(e0.elapsed_time(e1), dist))
            if profile:
                res.append(ffn.profile_read())
                ffn.profile(False)
            ffn.sync()
        _, _, groups_nc = nln.view(n)
        groups_nc = groups_nc.cpu().numpy()
        del nln, ffn
        torch.cuda.synchronize()
        return res[0], res[2], groups_nc

    nc_steps = max(1, min(args.steps, 10))
    ms_nc, prof_nc, groups_nc = timed_no_compaction(nc_steps)
    value_nc = job_throughput(world, n, nc_steps, ms_nc)

    # sparse-GP -> (beta, Sigma) mapping on the device (once per model, not per step)
    def timed_sgp_mapping(n_s=2048, reps=3):
        ffm = F.FlareGB(precision="fp32")
        g = torch.Generator(device="cuda").manual_seed(5)
        D = torch.randn((n_s, ffm.d_full), dtype=torch.float64, device="cuda", generator=g)
        D /= D.norm(dim=1, keepdim=True)
        alpha = torch.randn(n_s, dtype=torch.float64, device="cuda", generator=g)
        K = 0.7 * D @ D.T + 1e-3 * torch.eye(n_s, dtype=torch.float64, device="cuda")
        ffm.map_sgp(0, D, alpha, K, 0.7)          # warm-up
        times = []
        for _ in range(reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ffm.map_sgp(0, D, alpha, K, 0.7)
            times.append((time.perf_counter() - t0) * 1e3)
        d_full = ffm.d_full
        del ffm
        return {"n_sparse": n_s, "d": d_full, "ms": round(float(np.median(times)), 2),
                "note": "flr_map_sgp: FP64 Cholesky of K_SS, X = L^-1 D_S, beta and Sigma products, "
                        "copy to host and model upload; wall clock, median of 3"}
    sgp_map = timed_sgp_mapping() if rank == 0 else None

    # force error of each precision against the FP64 oracle on sampled atoms (same positions)
    ff.set_precision("bf16x3")
    F.build_neighbors(ff, sysg, nl)
    _, _, groups = nl.view(n)
    groups = groups.cpu().numpy()
    rng = np.random.default_rng(2)
    # 4,096 atoms drawn with seed 2, at least a quarter of them from the mixed (two-species) class
    mixed = np.nonzero(groups % 3 == 0)[0]
    rest = np.nonzero(groups % 3 != 0)[0]
    n_mixed = min(args.err_atoms // 4, len(mixed))
    sample = np.sort(np.concatenate([rng.choice(mixed, n_mixed, replace=False),
                                     rng.choice(rest, args.err_atoms - n_mixed, replace=False)]))
    pos_now = sysg.pos.detach().cpu().numpy()
    o = O.forces_subset(O.Hyper(), pos_now[:, :3].astype(np.float64), struct.species, struct.cell,
                        struct.pbc, beta, sigma, sample, skin=0.5)
    ferr, errs = {}, {}
    for prec in ("bf16x3", "tf32", "fp32"):
        ff.set_precision(prec)
        r = F.energy_forces_uncertainty(ff, sysg, nl, F.make_outputs(n))
        ff.sync()
        r = {k: v.cpu().numpy() for k, v in r.items()}
        ferr[prec] = float(np.abs(r["forces"][sample] - o["F"]).max())
        okv = o["V"] > 0
        errs[prec] = {
            "variance_fp64_atoms": int(r["totals"][14]),
            "force_max_ev_per_A": ferr[prec],
            "energy_max_rel": float((np.abs(r["energy"][sample] - o["E"]) / np.maximum(np.abs(o["E"]), 1.0)).max()),
            "variance_max_rel": float((np.abs(r["variance"][sample][okv] - o["V"][okv]) / o["V"][okv]).max()),
            "sigma_max_rel": float((np.abs(r["sigma"][sample][okv] - np.sqrt(o["V"][okv])) / np.sqrt(o["V"][okv])).max()),
        }
    ff.set_precision("bf16x3")
    err_sample = f"{len(sample)} atoms (seed 2; {n_mixed} mixed-class), FP64 oracle at the same positions"


    # rooflines: every kernel of each run against its own peak
    peaks, peak_kind = _peaks()
    fma = measure_fp32_peak(torch.cuda.current_device())
    fp32_peak = fma["tflops_best"]
    bf16_sus = peaks.get("bf16_tflops_sustained", 1700.0)
    per_step = {k: v[0] / max(args.steps, 1) for k, v in prof_mix.items()}
    dom = max(("descriptor", "qform", "force"), key=lambda k: prof_mix[k][0])
    cnt = out["energy"].numel()
    pairs_per_atom = _pairs_within_cutoff(nl, sysg, n, ff.r_cut) / n

    def kernel_rooflines(prof, grp, precision):
        res = {}
        for k in ("descriptor", "qform", "force"):
            amt = _algorithmic(k, grp, n, ff.d_full, ff.d_single, pairs_per_atom)
            avg = prof[k][0] / max(prof[k][1], 1)
            ach = amt / (avg / 1e3) / 1e12
            if k == "qform" and precision == "bf16x3":
                pk, bound, src = bf16_sus, "tensor", f"BF16 dense sustained ({peak_kind})"
            elif k == "qform" and precision == "tf32":
                pk, bound, src = bf16_sus / 2, "tensor", f"TF32 = BF16 dense sustained ({peak_kind}) x 1/2 (nominal ratio)"
            else:
                pk, bound, src = fp32_peak, "alu", "FP32 FMA, measured (flr_fp32_fma_peak)"
            r = {"ms_per_launch": round(avg, 4), "algorithmic_tflop": round(amt / 1e12, 4), "achieved": round(ach, 3),
                 "peak": round(pk, 1), "unit": "TFLOP/s", "bound": bound, "frac": round(ach / pk, 4),
                 "peak_source": src}
            if k == "qform" and precision == "bf16x3":
                r["frac_executed"] = round(3 * ach / pk, 4)   # the split issues 3 BF16 products per FP32 product
            res[k] = r
        return res

    rooflines = {"bf16x3": kernel_rooflines(prof_mix, groups, "bf16x3"),
                 "fp32": kernel_rooflines(prof_fp32, groups, "fp32"),
                 "compaction_off_bf16x3": kernel_rooflines(prof_nc, groups_nc, "bf16x3")}
    # whole step against the sum of per-kernel bounds (kernels run one after another)
    step_bound = {}
    n_full, n_single = _class_counts(groups)
    for k in ("descriptor", "qform", "force"):
        amt = _algorithmic(k, groups, n, ff.d_full, ff.d_single, pairs_per_atom)
        pk = bf16_sus if k == "qform" else fp32_peak
        step_bound[k + "_ms"] = round(amt / (pk * 1e12) * 1e3, 4)
    # HBM: positions, the list read twice, forces and E/V/sigma written (the unavoidable bytes)
    hbm_bytes = n * (16 + 2 * 64 * 4 + 12 + 12)
    step_bound["hbm_ms"] = round(hbm_bytes / (peaks.get("hbm_gbs", 6800.0) * 1e9) * 1e3, 4)
    step_bound["sum_ms"] = round(sum(step_bound[k + "_ms"] for k in ("descriptor", "qform", "force")) +
                                 step_bound["hbm_ms"], 4)
    step_bound["measured_ms"] = round(ms_mix / args.steps, 4)
    step_bound["frac"] = round(step_bound["sum_ms"] / step_bound["measured_ms"], 4)
    step_bound["atoms_mixed_class"] = n_full
    step_bound["atoms_one_species_class"] = n_single
    step_bound["pairs_per_atom"] = round(pairs_per_atom, 3)
    step_bound["note"] = ("algorithmic FLOPs of each kernel over its peak (measured FP32 FMA for the descriptor and "
                          "force kernels, BF16 dense sustained for the quadratic forms, whose 3xBF16 split executes "
                          "3x these FLOPs) plus the step's unavoidable HBM bytes; frac = bound / measured")
    dr = rooflines["bf16x3"][dom]
    tpa = _traffic_per_atom(dom)
    roofline = {"kernel": dom, "bound": dr["bound"], "achieved": dr["achieved"], "peak": dr["peak"],
                "unit": "TFLOP/s", "frac": dr["frac"], "peak_source": dr["peak_source"] + ", measured",
                "traffic": None if tpa is None else tpa * cnt, "avg_launch_ms": dr["ms_per_launch"],
                "algorithmic_per_launch": dr["algorithmic_tflop"] * 1e12,
                "per_unit": {"descriptor_flop_per_pair": DESC_PAIR, "force_flop_per_pair": FORCE_PAIR,
                             "pairs_per_atom": round(pairs_per_atom, 3)}}

    # end to end through the C ABI with host buffers: flr_md_step_host, one
    # call per step, uploads the step's positions and velocities from pinned
    # host memory (x, y, z rows), steps on the device, downloads the new state
    # and then reads back the step's energies, forces and sigma (asynchronous;
    # the library moves the positions while the step's kernels run, overlaps
    # one call's read-back with the next call's kernels and each chunk's
    # upload with the previous download)
    e2e = None
    if not args.no_e2e:
        ff.set_precision("bf16x3")
        st = reset()
        host = F.HostState(sysg.pos.cpu(), vel.cpu(), results=("energy", "forces", "sigma"))
        for _ in range(2):   # the first call creates the copy streams and staging rows
            F.md_step_host(ff, st, nl, 1, out, host, stream)
        ff.sync()
        barrier()
        t0 = time.perf_counter()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            F.md_step_host(ff, st, nl, 1, out, host, stream)
        F.host_join(ff, stream)
        e1.record(stream)
        ff.sync()
        barrier()
        wall = time.perf_counter() - t0
        ms_e2e = max(e0.elapsed_time(e1), wall * 1e3)
        bi = 2 * n * 12
        bo = 2 * n * 12 + sum(v.numel() * v.element_size() for v in host.results.values())
        ms_e2e = max_over_ranks(ms_e2e, dist)
        e2e = {"value": job_throughput(world, n, args.steps, ms_e2e), "unit": UNIT,
               "h2d_bytes_per_step": bi, "d2h_bytes_per_step": bo,
               "note": "per step one flr_md_step_host call: H2D pos+vel (pinned x, y, z rows), md step, D2H pos+vel, "
                       "then D2H energy, forces, sigma; copies in 8 chunks on two copy streams, the positions "
                       "downloaded (and the next step's uploaded) while the step's kernels run, the read-back "
                       "overlapping the next call's kernels"}

    serving = None
    if args.serving_seconds > 0:
        serving = run_serving(args, beta, sigma)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_sample(struct, beta, sigma, target_s=args.ref_seconds)

    if rank == 0:
        line = {"metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": round(ms_mix / args.steps, 4), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32+bf16x3", "data": "synthetic",
                "config": _config(n, "3xBF16 tcgen05 quadratic forms, FP32 elsewhere, FP64 totals"),
                "plain_fp32": {"value": round(value_fp32, 3), "ms_per_step": round(ms_fp32 / args.steps, 4)},
                "compaction_off": {"value": round(value_nc, 3), "ms_per_step": round(ms_nc / nc_steps, 4),
                                   "steps": nc_steps, "note": "3xBF16, every atom at d = 544"},
                "sgp_mapping": sgp_map,
                "step_bound": step_bound,
                "force_err_ev_per_A": ferr,
                "errors_vs_oracle": {"sample": err_sample, **errs},
                "rebuilds_in_timed_steps": rebuild_count,
                "kernels_ms_per_step": {k: round(v, 4) for k, v in per_step.items()},
                "kernels_ms_per_step_fp32": {k: round(v[0] / max(args.steps, 1), 4) for k, v in prof_fp32.items()},
                "kernels_ms_per_step_compaction_off": {k: round(v[0] / nc_steps, 4) for k, v in prof_nc.items()},
                "kernel_rooflines": rooflines, "fp32_fma_peak": fma,
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
                "clocks": clk, "serving": serving}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


SERVING_RATES = (50, 150, 500, 1500, 5000)


def run_serving(args, beta, sigma):
    """Open-loop serving: Poisson arrivals at each rate, requests drawn from
    a pool of 64 Pt(111)+H2 structures whose sizes are the midpoints of 64
    equal-probability strata of log-uniform[32, 200000] atoms (mean 22.9k);
    3xBF16; 150 GB admission budget.  Latency = output written - scheduled
    arrival (host pinned staging, H2D, neighbour build, evaluation, D2H)."""
    from paper_2204_12573_gb300 import flare as F
    from paper_2204_12573_gb300 import synth
    from paper_2204_12573_gb300.serving import Server, log_uniform_sizes, open_loop
    rng = np.random.default_rng(4)
    pool = []
    for n in log_uniform_sizes(64):
        s = synth.serving_structure(rng, int(n))
        pool.append((synth.as_f32_positions(s.pos), s.species, s.cell, s.pbc))
    ff = F.FlareGB(precision="bf16x3", max_nbr=64)
    ff.set_model(beta, sigma)
    res = []
    # batches are capped at 4M atoms (about 20 ms of device work), and device
    # and pinned memory for such a batch is reserved up front
    with Server(ff, budget_bytes=150e9, max_batch_atoms=4_000_000, reserve_atoms=4_000_000,
                reserve_structs=4096) as srv:
        open_loop(srv, pool, rate=5000, seconds=0.5, seed=99)   # warm-up
        for rate in SERVING_RATES:
            r = open_loop(srv, pool, rate=rate, seconds=args.serving_seconds, seed=4)
            res.append({k: (round(v, 4) if isinstance(v, float) else v) for k, v in r.items()})
        st = srv.stats()
    mean_atoms = float(np.mean([len(p[1]) for p in pool]))
    return {"rates": res, "budget_gb": 150, "seconds_per_rate": args.serving_seconds,
            "pool": f"64 structures, {min(len(p[1]) for p in pool)}-{max(len(p[1]) for p in pool)} atoms, "
                    f"mean {mean_atoms:.0f}", "precision": "bf16x3",
            "bytes_per_atom": st["bytes_per_atom"], "reserved_gb": round(st["reserved_bytes"] / 1e9, 2),
            "max_batch_atoms": st["max_batch_atoms_seen"], "batch_cap_atoms": 4_000_000,
            "batches_overlapped": st["batches_overlapped"], "grow_events": st["grow_events"]}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--ref-seconds", type=float, default=12.0)
    ap.add_argument("--profile-run", action="store_true",
                    help="time only the MD steps at --precision (for ncu launch lists)")
    ap.add_argument("--precision", default="bf16x3", choices=["fp32", "tf32", "bf16x3"])
    ap.add_argument("--fused", action="store_true",
                    help="with --profile-run: one-species atoms in the fused descriptor + tensor-core kernel")
    ap.add_argument("--err-atoms", type=int, default=4096,
                    help="atoms sampled for the error report against the FP64 oracle")
    ap.add_argument("--serving-seconds", type=float, default=3.0,
                    help="open-loop serving run per arrival rate (0: skip)")
    ap.add_argument("--serving-only", action="store_true",
                    help="run only the open-loop serving sweep and print its JSON line")
    ap.add_argument("--small", action="store_true",
                    help="64x64x32 slab + 1024 H2 (132k atoms) instead of the 2.1M-atom slab")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.serving_only:
        import torch
        from paper_2204_12573_gb300 import build
        from paper_2204_12573_gb300 import synth
        build.build()
        torch.cuda.set_device(_env_rank()[2])
        beta, sigma = synth.random_model()
        print(json.dumps({"serving": run_serving(args, beta, sigma)}), flush=True)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
