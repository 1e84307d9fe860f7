"""The seeded input generators (synth/), on the CPU: the counter-based stream against its
published definition (splitmix64 of key + (index + 1) * golden ratio), determinism, the
distinctness and ranges of drawn coordinates (one and several 62-bit key groups), the Zipf
law of the skewed modes, and the fold-in request recipe.  No GPU."""
import math

import numpy as np
import pytest
import torch

import synth


def test_counter_stream_matches_its_definition():
    for seed, stream in ((0, 0), (7, 3), (2**40 + 5, 123)):
        t = synth.bits64(seed, stream, 10, 20)
        for i in range(20):
            ref = synth.bits64_reference(seed, stream, 10 + i)
            assert (int(t[i]) & ((1 << 64) - 1)) == ref


def test_splitmix_finaliser_known_value():
    """splitmix64 of state 0 (one increment of the golden ratio, then the finaliser) is
    0xE220A8397B1DCDAF, the generator's first output for seed 0."""
    z = 0x9E3779B97F4A7C15
    assert synth._mix_int(z) == 0xE220A8397B1DCDAF


def test_uniform_and_normal_moments():
    u = synth.uniform01(3, 9, 0, 200_000)
    assert float(u.min()) >= 0.0 and float(u.max()) < 1.0
    assert abs(float(u.mean()) - 0.5) < 5e-3
    z = synth.normal(3, 9, 0, 200_000, std=2.0)
    assert abs(float(z.mean())) < 2e-2 and abs(float(z.std()) - 2.0) < 2e-2


def test_generators_are_deterministic():
    a = synth.small(11, (50, 40, 30), 3_000, 3, 4)
    b = synth.small(11, (50, 40, 30), 3_000, 3, 4)
    c = synth.small(12, (50, 40, 30), 3_000, 3, 4)
    assert torch.equal(a.coords, b.coords) and torch.equal(a.x, b.x)
    assert not torch.equal(a.coords, c.coords)


@pytest.mark.parametrize("dims,modes", [
    ((60, 50, 40), None),                          # one key group
    ((200, 300, 50), ["zipf", "zipf", "uniform"]),  # skewed modes
    ((10**6,) * 5, None),                          # > 2^62 cells: two key groups
])
def test_distinct_coords_are_distinct_and_in_range(dims, modes):
    nnz = 20_000
    c = synth.distinct_coords(dims, nnz, 5, modes).numpy()
    assert c.shape == (nnz, len(dims)) and c.dtype == np.int32
    for n, d in enumerate(dims):
        assert c[:, n].min() >= 0 and c[:, n].max() < d
    assert len({tuple(r) for r in c}) == nnz


def test_zipf_mode_follows_its_law():
    """Rank frequencies of Zipf(1.1) over 1,000 rows: the most frequent row carries about
    1 / H(1000, 1.1) of the draws, and the row counts fall off as a power of the rank."""
    I, s = 1000, 1.1
    z = synth.Zipf(I, s, 4, 50)
    rows = z.sample(synth.uniform01(4, 51, 0, 400_000)).numpy()
    counts = np.sort(np.bincount(rows, minlength=I))[::-1]
    H = sum(k ** -s for k in range(1, I + 1))
    assert abs(counts[0] / len(rows) - 1 / H) < 0.01
    # slope of log count vs log rank over ranks 2..100
    r = np.arange(2, 101)
    slope = np.polyfit(np.log(r), np.log(counts[1:100]), 1)[0]
    assert abs(slope + s) < 0.1
    # the rank-0 row is not row 0: ranks go through a seeded permutation
    assert int(np.bincount(rows, minlength=I).argmax()) == int(z.perm[0])


def test_foldin_requests_recipe():
    p = synth.small(13, (80, 60, 40), 5_000, 3, 6)
    reqs = synth.foldin_requests(p, 30, 9, m_min=5, m_max=500)
    assert len(reqs) == 30
    for other, x in reqs:
        m = other.shape[0]
        assert 5 <= m <= 500 and x.shape == (m,)
        assert other.shape[1] == 2
        assert other[:, 0].max() < 60 and other[:, 1].max() < 40
        assert len({tuple(r) for r in other}) == m      # distinct entries of the new slice
        assert np.all(np.isfinite(x))


def test_cap_at_half_the_cells():
    p = synth.make_problem((8, 8, 8), 10_000, 2, 4, 1)
    assert p.nnz == 256
