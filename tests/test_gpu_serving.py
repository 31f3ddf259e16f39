"""The continuous-batching server (flr_server_*): each request's results are
the same bits whether it is served alone or inside a mixed batch, equal the
direct batch API's, match the oracle, and the memory-budget admission holds.
"""
import dataclasses

import numpy as np
import pytest

from paper_2204_12573_gb300 import synth

from gpu_common import compare_efv, oracle_run

pytestmark = pytest.mark.gpu

BETA, SIGMA = synth.random_model()


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2204_12573_gb300 import build
    build.build()


def _ff(precision="bf16x3"):
    from paper_2204_12573_gb300 import flare as F
    ff = F.FlareGB(precision=precision, max_nbr=96)
    ff.set_model(BETA, SIGMA)
    return ff


def _mix():
    rng = np.random.default_rng(12)
    out = [synth.tiny_system(0), dataclasses.replace(synth.tiny_system(1), pbc=(0, 0, 0))]
    out += synth.slab_batch(seed=7, n_slabs=6)
    out += [synth.serving_structure(rng, n) for n in (40, 900, 5000)]
    return out


def _submit(srv, s, tag=None):
    return srv.submit(synth.as_f32_positions(s.pos), s.species, s.cell, s.pbc, tag=tag)


@pytest.mark.parametrize("precision", ["bf16x3", "fp32"])
def test_same_alone_and_in_the_mix(precision):
    from paper_2204_12573_gb300.serving import Server
    structs = _mix()
    ff = _ff(precision)
    with Server(ff, budget_bytes=8e9) as srv:
        alone = []
        for s in structs:
            t = _submit(srv, s)
            alone.append(srv.wait_all([t])[t])
            assert alone[-1][1]["batch_structs"] == 1
        # all at once, twice in a different order: they share batches
        tags = [_submit(srv, s) for s in structs] + [_submit(srv, s) for s in reversed(structs)]
        got = srv.wait_all(tags)
        shared = max(got[t][1]["batch_structs"] for t in tags)
        assert shared > 1
        for k, s in enumerate(structs):
            for t in (tags[k], tags[2 * len(structs) - 1 - k]):
                out, c = got[t]
                assert c["status"] == 0
                for key in ("energy", "forces", "variance", "sigma", "totals"):
                    assert np.array_equal(out[key], alone[k][0][key]), (s.name, key)


def test_server_matches_batch_api_and_oracle():
    import torch
    from paper_2204_12573_gb300 import flare as F
    from paper_2204_12573_gb300.serving import Server
    structs = _mix()[:8]
    ff = _ff("fp32")
    b = F.Batch.from_structures(structs)
    nl = ff.nbrlist(b.n_atoms)
    F.build_neighbors_batch(ff, b, nl)
    ref = {k: v.cpu().numpy() for k, v in F.energy_forces_uncertainty_batch(ff, b, nl).items()}
    torch.cuda.synchronize()
    del nl
    with Server(ff, budget_bytes=4e9) as srv:
        tags = [_submit(srv, s) for s in structs]
        got = srv.wait_all(tags)
    for k, s in enumerate(structs):
        lo, hi = int(b.offsets[k]), int(b.offsets[k + 1])
        out = got[tags[k]][0]
        for key in ("energy", "forces", "variance", "sigma"):
            assert np.array_equal(out[key], ref[key][lo:hi]), (s.name, key)
        if k < 3:
            compare_efv(out, oracle_run(s, BETA, SIGMA))


def test_budget_admission():
    from paper_2204_12573_gb300 import _native as N
    from paper_2204_12573_gb300.serving import Server
    ff = _ff()
    bpa = Server.bytes_per_atom(ff)
    slabs = synth.slab_batch(seed=3, n_slabs=12)
    budget = bpa * 1300 + 10**6
    with Server(ff, budget_bytes=budget) as srv:
        tags = [_submit(srv, s) for s in slabs]
        got = srv.wait_all(tags)
        for t in tags:
            c = got[t][1]
            assert c["status"] == 0
            assert c["batch_atoms"] * bpa <= budget
        st = srv.stats()
        assert st["requests"] == len(slabs) and st["batches"] >= 4
        assert st["reserved_bytes"] <= budget
        big = synth.serving_structure(np.random.default_rng(0), 2000)
        with pytest.raises(N.FlareError) as e:
            _submit(srv, big)
        assert e.value.code == N.FLR_EBUDGET


def test_max_batch_structs_and_empty_request():
    from paper_2204_12573_gb300.serving import Server
    ff = _ff()
    tiny = synth.tiny_system(0)
    with Server(ff, budget_bytes=2e9, max_batch_structs=1) as srv:
        tags = [_submit(srv, tiny) for _ in range(5)]
        t_empty = srv.submit(np.zeros((0, 4), np.float32), np.zeros(0, np.int32), tiny.cell, tiny.pbc)
        got = srv.wait_all(tags + [t_empty])
        assert all(got[t][1]["batch_structs"] == 1 for t in tags)
        assert got[t_empty][1]["status"] == 0
        assert got[t_empty][0]["totals"][0] == 0.0
        e0 = got[tags[0]][0]["energy"]
        assert all(np.array_equal(got[t][0]["energy"], e0) for t in tags)


def test_open_loop_reports_latency():
    from paper_2204_12573_gb300.serving import Server, log_uniform_sizes, open_loop
    ff = _ff()
    rng = np.random.default_rng(4)
    pool = []
    for n in log_uniform_sizes(8, 32, 20000):
        s = synth.serving_structure(rng, int(n))
        pool.append((synth.as_f32_positions(s.pos), s.species, s.cell, s.pbc))
    with Server(ff, budget_bytes=20e9) as srv:
        r = open_loop(srv, pool, rate=200, seconds=1.0, seed=4)
    assert r["errors"] == 0 and r["completed"] == r["requests"]
    assert 0 < r["p50_ms"] <= r["p99_ms"]


def test_batches_overlap_on_the_device():
    """The two slots' batches overlap on the device: while one batch is being
    evaluated, the next batch's copies and neighbour build run (device
    timestamps of the completions).  Results stay the same bits as alone,
    and with the memory reserved up front nothing grows under load.  FP32
    quadratic forms give each batch more device time than the worker's host
    copies take, so the worker can run ahead of the device (with 3xBF16 the
    two are close on a GB300 and the overlap comes and goes)."""
    from paper_2204_12573_gb300.serving import Server
    ff = _ff("fp32")
    rng = np.random.default_rng(5)
    big = [synth.serving_structure(rng, 150000) for _ in range(3)]
    with Server(ff, budget_bytes=60e9, max_batch_structs=2, reserve_atoms=300000, reserve_structs=4) as srv:
        alone = {}
        for k, s in enumerate(big):
            t = _submit(srv, s)
            alone[k] = srv.wait_all([t])[t][0]
        order = [k % 3 for k in range(12)]
        tags = [_submit(srv, big[k]) for k in order]
        got = srv.wait_all(tags)
        st = srv.stats()
    for t, k in zip(tags, order):
        out, c = got[t]
        assert c["status"] == 0
        for key in ("energy", "forces", "variance", "sigma"):
            assert np.array_equal(out[key], alone[k][key]), key
    batches = {}
    for t in tags:
        c = got[t][1]
        batches[c["gpu_start_ms"]] = (c["slot"], c["gpu_built_ms"], c["gpu_eval_start_ms"], c["gpu_eval_end_ms"],
                                      c["gpu_done_ms"])
    iv = sorted(batches.items())
    assert len(iv) >= 6      # at most 2 structures per batch (fewer when requests trickle in)
    for start, (_, built, e0, e1, done) in iv:
        assert start <= built <= e0 <= e1 <= done
    # evaluations run one at a time, in order
    for (_, a), (_, b) in zip(iv, iv[1:]):
        assert b[2] >= a[3]
    overlapped = sum(1 for (_, a), (s1, b) in zip(iv, iv[1:]) if s1 < a[3] and b[1] > a[2] and b[0] != a[0])
    assert overlapped >= 1, iv
    assert st["grow_events"] == 0 and st["batches_overlapped"] >= 1
