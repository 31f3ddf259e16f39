"""flr_build_neighbors_noalloc: the neighbour build for callers that cannot
allocate device memory (its scratch is a fixed array inside the library).

Checked through the C ABI against the regular flr_build_neighbors on the same
inputs: the rows must be identical (integer output, so bit-exact), on two
calls in a row, since every call reuses the same scratch array.  Collected
last so that a run stopping at its first failure has run everything else.
"""
import numpy as np
import pytest

from paper_2204_12573_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2204_12573_gb300 import build
    build.build()


def _reference_rows(struct, max_nbr):
    from paper_2204_12573_gb300 import flare as F
    ff = F.FlareGB(max_nbr=max_nbr, precision="fp32")
    sysg = F.System.from_numpy(synth.as_f32_positions(struct.pos), struct.species, struct.cell, struct.pbc)
    nl = ff.nbrlist(struct.n_atoms)
    F.build_neighbors(ff, sysg, nl)
    e, c, _ = nl.view(struct.n_atoms)
    return sysg, e.cpu().numpy(), c.cpu().numpy()


def test_noalloc_matches_regular_build_twice():
    import torch
    from paper_2204_12573_gb300 import flare as F
    structs = [synth.tiny_system(0)] + synth.slab_batch(seed=3, n_slabs=2)
    max_nbr = 96
    for s in structs:
        sysg, e_ref, c_ref = _reference_rows(s, max_nbr)
        for _ in range(2):
            entries = torch.full((s.n_atoms, max_nbr), -7, dtype=torch.int32, device="cuda")
            count = torch.full((s.n_atoms,), -7, dtype=torch.int32, device="cuda")
            F.build_neighbors_noalloc(sysg, 4.5 + 0.5, max_nbr, entries, count)
            c = count.cpu().numpy()
            e = entries.cpu().numpy()
            assert np.array_equal(c, c_ref)
            for i in range(s.n_atoms):
                assert np.array_equal(e[i, :c[i]], e_ref[i, :c_ref[i]])


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    from paper_2204_12573_gb300 import _native as N
    from paper_2204_12573_gb300 import flare as F
    n = (1 << 16) + 1
    sysg = F.System(torch.zeros((n, 4), dtype=torch.float32, device="cuda"),
                    torch.zeros(n, dtype=torch.int32, device="cuda"), np.eye(3) * 100.0, (1, 1, 0))
    entries = torch.empty((n, 32), dtype=torch.int32, device="cuda")
    count = torch.empty(n, dtype=torch.int32, device="cuda")
    with pytest.raises(N.FlareError) as e:
        F.build_neighbors_noalloc(sysg, 5.0, 32, entries, count)
    assert e.value.code == N.FLR_EINVAL and "65536" in str(e.value)
