"""The seeded input generators against the recipes they implement (CPU)."""
import numpy as np

from paper_1412_7789_gb300 import workloads


def test_acgt_text_is_uniform_over_four_letters():
    t = workloads.acgt_text(1 << 20, 0)
    vals, counts = np.unique(t, return_counts=True)
    assert bytes(vals) == b"ACGT"
    assert np.all(np.abs(counts / t.size - 0.25) < 0.005)
    assert np.array_equal(t, workloads.acgt_text(1 << 20, 0))  # seeded


def test_zipf_text_follows_the_power_law():
    """Rank r (byte r - 1) has probability proportional to r^-1.1."""
    t = workloads.zipf_text(1 << 22, 1)
    counts = np.bincount(t, minlength=256).astype(np.float64)
    p = counts / counts.sum()
    r = np.arange(1, 257, dtype=np.float64)
    want = r ** -1.1 / np.sum(r ** -1.1)
    assert np.all(np.abs(p[:8] - want[:8]) < 0.01 * want[:8] + 2e-4)
    slope = np.polyfit(np.log(r[:32]), np.log(p[:32]), 1)[0]
    assert abs(slope + 1.1) < 0.03


def test_sweep_keywords_recipe():
    """10,000 keywords of 16-64 bytes; half copied from the first 4 KiB (so
    every prefix of the text of 4 KiB or more holds them), half random ACGT."""
    text, pats = workloads.sweep_acgt(1 << 16, seed=0)
    assert len(pats) == 10_000
    lens = np.array([len(p) for p in pats])
    assert lens.min() >= 16 and lens.max() <= 64
    head = bytes(text[:4096])
    copied = sum(1 for p in pats if p in head)
    assert 4900 <= copied <= 5100
    assert all(set(p) <= set(b"ACGT") for p in pats)
    # the keywords depend only on the first 4 KiB
    assert workloads.sweep_acgt(1 << 14, seed=0)[1] == pats


def test_batch_texts_lengths_and_alphabets():
    texts, kinds = workloads.batch_texts(400, 1024, 4 << 20, seed=0)
    lens = np.array([t.size for t in texts])
    assert lens.min() >= 1024 and lens.max() <= 4 << 20
    med = np.exp(np.median(np.log(lens)))
    assert 0.7 * np.sqrt(1024 * (4 << 20)) < med < 1.4 * np.sqrt(1024 * (4 << 20))  # log-uniform
    for t, k in zip(texts[:40], kinds[:40]):
        if k == 0:
            assert set(np.unique(t)) <= set(b"ACGT")
    assert 0.35 < np.mean(kinds) < 0.65


def test_paper_keywords_are_permutations_not_rotations():
    pats = workloads.paper_keywords(10, seed=0)
    alpha = bytes(range(ord("a"), ord("z") + 1))
    assert pats[0] == alpha and len(set(pats)) == 10
    rotations = {alpha[i:] + alpha[:i] for i in range(26)}
    for p in pats[1:]:
        assert sorted(p) == sorted(alpha) and p not in rotations
    t = workloads.paper_text(100)
    assert bytes(t) == (alpha * 4)[:100]


def test_poisson_arrivals_rate():
    a = workloads.poisson_arrivals(20000, 10000.0, seed=0)
    gaps = np.diff(np.concatenate([[0.0], a]))
    assert np.all(gaps > 0)
    assert abs(np.mean(gaps) - 100.0) < 3.0  # microseconds at 10k/s
