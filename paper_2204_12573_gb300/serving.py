"""Continuous-batching evaluation service (flr_server_* in the C ABI) and an
open-loop load generator that measures its latency.

    srv = Server(ff, budget_bytes=150e9)
    tag = srv.submit(pos4, species, cell, pbc)
    done = srv.poll(wait=0.1)          # [(tag, result dict, completion dict)]

The worker loop, admission control, packing and all GPU work are native;
this module marshals arguments and keeps each request's host output arrays
alive until its completion is polled.
"""
from __future__ import annotations

import ctypes
import gc
import itertools
import threading
import time

import numpy as np

from . import _native as N

FIELDS = ("energy", "forces", "variance", "sigma", "totals")


class Server:
    def __init__(self, ff, budget_bytes=150e9, max_batch_structs=0, max_batch_atoms=0, reserve_atoms=0,
                 reserve_structs=0):
        self.ff = ff
        self.lib = ff.lib
        p = N.ServerParams(int(budget_bytes), int(max_batch_structs), int(max_batch_atoms), int(reserve_atoms),
                           int(reserve_structs))
        h = ctypes.c_void_p()
        N.check(self.lib.flr_server_create(ff.handle, ctypes.byref(p), ctypes.byref(h)))
        self.handle = h
        self._pending = {}
        self._lock = threading.Lock()
        self._tags = itertools.count(1)
        self._buf = (N.Completion * 4096)()

    @staticmethod
    def bytes_per_atom(ff):
        b = ctypes.c_int64()
        N.check(ff.lib.flr_bytes_per_atom(ff.handle, ctypes.byref(b)))
        return int(b.value)

    def submit(self, pos4, species, cell, pbc=(1, 1, 0), fields=FIELDS, tag=None):
        """Queue one structure (host arrays: pos4 float32 [n, 4], species
        int32 [n]).  Returns the request's tag."""
        pos4 = np.ascontiguousarray(pos4, np.float32)
        species = np.ascontiguousarray(species, np.int32)
        n = int(pos4.shape[0])
        out = {}
        if "energy" in fields:
            out["energy"] = np.empty(n, np.float32)
        if "forces" in fields:
            out["forces"] = np.empty((n, 3), np.float32)
        if "variance" in fields:
            out["variance"] = np.empty(n, np.float32)
        if "sigma" in fields:
            out["sigma"] = np.empty(n, np.float32)
        if "totals" in fields:
            out["totals"] = np.empty(N.NTOTALS, np.float64)
        if tag is None:
            tag = next(self._tags)
        r = N.Request()
        r.n_atoms = n
        r.pos = pos4.ctypes.data_as(ctypes.c_void_p)
        r.species = species.ctypes.data_as(ctypes.c_void_p)
        r.cell = (ctypes.c_double * 9)(*np.asarray(cell, np.float64).ravel().tolist())
        r.pbc = (ctypes.c_int32 * 3)(*[int(bool(v)) for v in pbc])
        for k in ("energy", "forces", "variance", "sigma", "totals"):
            setattr(r, k, out[k].ctypes.data_as(ctypes.c_void_p) if k in out else None)
        r.tag = tag
        with self._lock:
            self._pending[tag] = out
        code = self.lib.flr_server_submit(self.handle, ctypes.byref(r))
        if code != N.FLR_OK:
            with self._lock:
                self._pending.pop(tag, None)
            N.check(code)
        return tag

    def poll(self, wait=0.0, max_items=4096):
        """Finished requests: a list of (tag, outputs, completion dict)."""
        n = ctypes.c_int32()
        N.check(self.lib.flr_server_poll(self.handle, self._buf, min(max_items, len(self._buf)), ctypes.byref(n),
                                         float(wait)))
        res = []
        for k in range(n.value):
            c = self._buf[k]
            with self._lock:
                out = self._pending.pop(c.tag)
            res.append((c.tag, out, dict(status=c.status, batch_structs=c.batch_structs,
                                         batch_atoms=c.batch_atoms, t_submit_ns=c.t_submit_ns,
                                         t_start_ns=c.t_start_ns, t_done_ns=c.t_done_ns, slot=c.slot,
                                         gpu_start_ms=c.gpu_start_ms, gpu_built_ms=c.gpu_built_ms,
                                         gpu_eval_start_ms=c.gpu_eval_start_ms,
                                         gpu_eval_end_ms=c.gpu_eval_end_ms, gpu_done_ms=c.gpu_done_ms)))
        return res

    def wait_all(self, tags, timeout=120.0):
        """Poll until every tag in `tags` has completed; returns {tag: (outputs, completion)}."""
        want = set(tags)
        got = {}
        t_end = time.monotonic() + timeout
        while want - set(got):
            if time.monotonic() > t_end:
                raise TimeoutError(f"{len(want - set(got))} requests still pending")
            for tag, out, c in self.poll(wait=0.05):
                got[tag] = (out, c)
        return got

    def stats(self):
        s = N.ServerStats()
        N.check(self.lib.flr_server_stats_read(self.handle, ctypes.byref(s)))
        return dict(requests=s.requests, batches=s.batches, atoms=s.atoms,
                    max_batch_atoms_seen=s.max_batch_atoms_seen, queued=s.queued,
                    reserved_bytes=s.reserved_bytes, bytes_per_atom=s.bytes_per_atom,
                    last_error=s.last_error.decode(), batches_overlapped=s.batches_overlapped,
                    grow_events=s.grow_events, grow_ms=s.grow_ms, pack_ms=s.pack_ms,
                    enqueue_ms=s.enqueue_ms, finish_ms=s.finish_ms)

    def close(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            self.lib.flr_server_destroy(h)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def log_uniform_sizes(k, lo=32, hi=200_000):
    """k sizes at the midpoints of k equal-probability strata of the
    log-uniform distribution on [lo, hi]."""
    q = (np.arange(k) + 0.5) / k
    return np.exp(np.log(lo) + q * (np.log(hi) - np.log(lo))).round().astype(int)


def percentile_ms(lat_ns, q):
    return float(np.percentile(np.asarray(lat_ns, np.float64), q) / 1e6) if len(lat_ns) else None


def open_loop(server, pool, rate, seconds, seed=4, drain_timeout=120.0):
    """Poisson arrivals at `rate` requests/s for `seconds`; each request is a
    structure drawn uniformly from `pool` (list of (pos4, species, cell,
    pbc)).  Latency is measured from the scheduled arrival time to the moment
    the request's outputs were written.  Returns a summary dict."""
    rng = np.random.default_rng(seed)
    n_req = max(1, int(rng.poisson(rate * seconds)))
    arrivals = np.sort(rng.uniform(0.0, seconds, n_req))
    picks = rng.integers(0, len(pool), n_req)
    sched = {}
    lat = []
    atoms_done = [0]
    batch_sizes = []
    batches = {}                 # (slot, gpu_start_ms) -> (built, eval start, eval end, done)
    errors = [0]
    st0 = server.stats()
    finished = threading.Event()

    def collect():
        while not finished.is_set() or len(lat) + errors[0] < len(sched):
            for tag, out, c in server.poll(wait=0.02):
                if c["status"] != N.FLR_OK:
                    errors[0] += 1
                    continue
                lat.append(c["t_done_ns"] - sched[tag][0])
                atoms_done[0] += sched[tag][1]
                batch_sizes.append(c["batch_structs"])
                batches[(c["slot"], c["gpu_start_ms"])] = (c["gpu_built_ms"], c["gpu_eval_start_ms"],
                                                           c["gpu_eval_end_ms"], c["gpu_done_ms"])
            if finished.is_set() and time.monotonic() > t_drain_end[0]:
                break

    # host-side stalls of the load generator, reported with the result:
    # garbage-collector pauses (timed by a gc callback), the longest submit
    # call and the longest oversleep
    gc_pause = []
    gc_t = [0]

    def on_gc(phase, info):
        if phase == "start":
            gc_t[0] = time.monotonic_ns()
        else:
            gc_pause.append(time.monotonic_ns() - gc_t[0])

    # objects alive before the run (the pool, the server, the interpreter's
    # own) are frozen out of the collector's full passes
    gc.collect()
    gc.freeze()
    gc.callbacks.append(on_gc)
    t_drain_end = [float("inf")]
    th = threading.Thread(target=collect, daemon=True)
    t0 = time.monotonic_ns()
    th.start()
    late = 0
    max_submit = 0
    max_oversleep = 0
    try:
        for k in range(n_req):
            t_arr = t0 + int(arrivals[k] * 1e9)
            dt = (t_arr - time.monotonic_ns()) / 1e9
            if dt > 0:
                time.sleep(dt)
                max_oversleep = max(max_oversleep, time.monotonic_ns() - t_arr)
            elif dt < -1e-3:
                late += 1
            pos4, species, cell, pbc = pool[picks[k]]
            tag = k + 1
            sched[tag] = (t_arr, len(species))
            ts = time.monotonic_ns()
            server.submit(pos4, species, cell, pbc, fields=("energy", "forces", "sigma"), tag=tag)
            max_submit = max(max_submit, time.monotonic_ns() - ts)
        t_drain_end[0] = time.monotonic() + drain_timeout
        finished.set()
        th.join()
    finally:
        gc.callbacks.remove(on_gc)
        gc.unfreeze()
    t_last = time.monotonic_ns()
    wall = (t_last - t0) / 1e9
    st1 = server.stats()
    # device overlap: batches whose copies or neighbour build ran while the
    # previous batch (other slot) was still being evaluated or copied back
    ivals = sorted((k[1], v) for k, v in batches.items())   # (copies started, (built, eval0, eval1, done))
    overlap = sum(1 for (_, prev), (s1, cur) in zip(ivals, ivals[1:]) if s1 < prev[2] and cur[0] > prev[1])
    return dict(rate=rate, seconds=seconds, requests=n_req, completed=len(lat), errors=errors[0],
                p50_ms=percentile_ms(lat, 50), p99_ms=percentile_ms(lat, 99), mean_ms=(
                    float(np.mean(lat) / 1e6) if lat else None),
                atoms_per_s=atoms_done[0] / wall, offered_atoms_per_s=float(
                    sum(len(pool[p][1]) for p in picks) / seconds),
                mean_batch_structs=float(np.mean(batch_sizes)) if batch_sizes else 0.0,
                late_submits=late, max_submit_ms=max_submit / 1e6, max_oversleep_ms=max_oversleep / 1e6,
                gc_pauses=len(gc_pause), gc_max_ms=(max(gc_pause) / 1e6 if gc_pause else 0.0),
                max_batch_gpu_ms=max((v[3] - k0 for k0, v in ivals), default=0.0),
                batches=len(ivals), batches_overlapping_previous=overlap,
                grow_events=st1["grow_events"] - st0["grow_events"],
                worker_ms={k: round(st1[k] - st0[k], 2) for k in ("grow_ms", "pack_ms", "enqueue_ms", "finish_ms")})
