"""Seeded synthetic inputs shaped like the workloads the paper and its follow-on
configurations measure.  Both the library's tests and the CPU oracle consume the
arrays made here; this module holds none of the matching arithmetic.

All randomness comes from numpy's PCG64 generator seeded explicitly; every
function is deterministic in its arguments.

Workloads:

* ``paper_text`` / ``paper_keywords`` -- section III: the English alphabet
  repeated into a text file, and five (later ten, section IV) keywords that are
  permutations of the 26 letters.  Keyword 0 is the example the paper prints
  (a..z); the others are seeded permutations that are not rotations of a..z.
* ``single_text_acgt`` -- 1 MiB i.i.d. uniform ACGT text; 100 keywords of
  length 8-32, half copied from random text offsets, half random ACGT.
* ``sweep_acgt`` -- ACGT text up to 1 GiB whose prefixes form the input-size
  sweep (4 KiB .. 1 GiB, powers of 4); 10,000 keywords of length 16-64, half
  copied from offsets inside the first 4 KiB (so every prefix holds them), half
  random ACGT.
* ``zipf_byte`` -- Zipf(s=1.1) text over all 256 byte values (rank r -> byte
  r-1); 20,000 keywords of length 4-100, 30% copied from text offsets, 70%
  Zipf-random (duplicates kept).
* ``batch_texts`` / ``batch_pattern_sets`` -- many texts of log-uniform length,
  ACGT and Zipf-256 mixed, against several keyword sets.
"""
from __future__ import annotations

import numpy as np

ACGT = np.frombuffer(b"ACGT", dtype=np.uint8)
ALPHABET = np.frombuffer(b"abcdefghijklmnopqrstuvwxyz", dtype=np.uint8)
_CHUNK = 1 << 26
_ZIPF_BITS = 20


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


# ----------------------------------------------------------------------------
# texts
# ----------------------------------------------------------------------------
def acgt_text(n: int, seed: int) -> np.ndarray:
    """n bytes i.i.d. uniform over {A, C, G, T}."""
    g = rng(seed)
    out = np.empty(n, dtype=np.uint8)
    for lo in range(0, n, _CHUNK):
        hi = min(n, lo + _CHUNK)
        out[lo:hi] = ACGT[g.integers(0, 4, size=hi - lo, dtype=np.uint8)]
    return out


def zipf_table(s: float = 1.1, ranks: int = 256, bits: int = _ZIPF_BITS) -> np.ndarray:
    """Inverse-CDF lookup: a uniform ``bits``-bit integer -> byte (rank r -> byte r-1).

    P(rank r) is proportional to r**-s; the table quantises the CDF to
    2**-bits resolution (every rank keeps at least one slot)."""
    r = np.arange(1, ranks + 1, dtype=np.float64)
    p = r ** (-s)
    p /= p.sum()
    cdf = np.cumsum(p)
    u = (np.arange(1 << bits, dtype=np.float64) + 0.5) / float(1 << bits)
    lut = np.searchsorted(cdf, u, side="right").astype(np.int64)
    lut = np.minimum(lut, ranks - 1)
    # keep every rank reachable: the last slots go to the rarest ranks
    missing = np.setdiff1d(np.arange(ranks), np.unique(lut))
    if missing.size:
        lut[-missing.size:] = missing
        lut.sort()
    return lut.astype(np.uint8)


_ZIPF_CACHE: dict = {}


def _zipf_lut(s: float) -> np.ndarray:
    if s not in _ZIPF_CACHE:
        _ZIPF_CACHE[s] = zipf_table(s)
    return _ZIPF_CACHE[s]


def zipf_bytes(g: np.random.Generator, n: int, s: float = 1.1) -> np.ndarray:
    lut = _zipf_lut(s)
    out = np.empty(n, dtype=np.uint8)
    mask = np.uint32((1 << _ZIPF_BITS) - 1)
    for lo in range(0, n, _CHUNK):
        hi = min(n, lo + _CHUNK)
        u = g.integers(0, 1 << 32, size=hi - lo, dtype=np.uint32) & mask
        out[lo:hi] = lut[u]
    return out


def zipf_text(n: int, seed: int, s: float = 1.1) -> np.ndarray:
    """n bytes i.i.d. Zipf(s) over the 256 byte values."""
    return zipf_bytes(rng(seed), n, s)


def paper_text(n: int) -> np.ndarray:
    """The English alphabet a..z repeated and cut to n bytes (section III)."""
    reps = n // 26 + 1
    return np.tile(ALPHABET, reps)[:n].copy()


# ----------------------------------------------------------------------------
# keyword sets
# ----------------------------------------------------------------------------
def _is_rotation_of_alphabet(p: bytes) -> bool:
    a = bytes(ALPHABET)
    return len(p) == 26 and p in (a + a)


def paper_keywords(count: int = 5, seed: int = 0) -> list[bytes]:
    """Keyword 0 = a..z (the paper's example); the rest are distinct seeded
    permutations of the 26 letters that are not rotations of a..z."""
    g = rng(seed)
    out = [bytes(ALPHABET)]
    seen = set(out)
    while len(out) < count:
        p = bytes(ALPHABET[g.permutation(26)])
        if _is_rotation_of_alphabet(p) or p in seen:
            continue
        out.append(p)
        seen.add(p)
    return out


def _copied(g, text: np.ndarray, count: int, lmin: int, lmax: int, window: int) -> list[bytes]:
    window = min(window, text.size)
    out = []
    for _ in range(count):
        L = int(g.integers(lmin, lmax + 1))
        L = min(L, window)
        off = int(g.integers(0, window - L + 1))
        out.append(bytes(text[off:off + L]))
    return out


def _random_acgt(g, count: int, lmin: int, lmax: int) -> list[bytes]:
    out = []
    for _ in range(count):
        L = int(g.integers(lmin, lmax + 1))
        out.append(bytes(ACGT[g.integers(0, 4, size=L)]))
    return out


def _random_zipf(g, count: int, lmin: int, lmax: int, s: float = 1.1) -> list[bytes]:
    out = []
    for _ in range(count):
        L = int(g.integers(lmin, lmax + 1))
        out.append(bytes(zipf_bytes(g, L, s)))
    return out


def _shuffled(g, pats: list[bytes]) -> list[bytes]:
    order = g.permutation(len(pats))
    return [pats[i] for i in order]


def keywords_acgt(text: np.ndarray, count: int, lmin: int, lmax: int, frac_copied: float,
                  seed: int, copy_window: int | None = None) -> list[bytes]:
    """ACGT keywords: a fraction copied from ``text[:copy_window]`` at uniform
    offsets, the rest uniform random ACGT; lengths uniform in [lmin, lmax]."""
    g = rng(seed)
    nc = int(round(count * frac_copied))
    window = text.size if copy_window is None else copy_window
    pats = _copied(g, text, nc, lmin, lmax, window) + _random_acgt(g, count - nc, lmin, lmax)
    return _shuffled(g, pats)


def keywords_zipf(text: np.ndarray, count: int, lmin: int, lmax: int, frac_copied: float,
                  seed: int, s: float = 1.1) -> list[bytes]:
    g = rng(seed)
    nc = int(round(count * frac_copied))
    pats = _copied(g, text, nc, lmin, lmax, text.size) + _random_zipf(g, count - nc, lmin, lmax, s)
    return _shuffled(g, pats)


# ----------------------------------------------------------------------------
# the configurations
# ----------------------------------------------------------------------------
SWEEP_SIZES = [4096 * 4 ** j for j in range(10)]  # 4 KiB .. 1 GiB


def single_text_acgt(seed: int = 0, n: int = 1 << 20):
    text = acgt_text(n, seed)
    pats = keywords_acgt(text, 100, 8, 32, 0.5, seed + 1)
    return text, pats


def sweep_acgt(n: int = 1 << 30, seed: int = 0, n_keywords: int = 10_000):
    """Text of n bytes (prefixes give the sweep) and the sweep's keyword set.
    The keywords depend only on the first 4 KiB, so every prefix of a longer
    text of the same seed shares them."""
    text = acgt_text(n, seed)
    head = text[:4096] if n >= 4096 else acgt_text(4096, seed)[:4096]
    pats = keywords_acgt(head, n_keywords, 16, 64, 0.5, seed + 1, copy_window=4096)
    return text, pats


def zipf_byte(n: int = 1 << 30, seed: int = 0, n_keywords: int = 20_000):
    text = zipf_text(n, seed)
    pats = keywords_zipf(text, n_keywords, 4, 100, 0.3, seed + 1)
    return text, pats


def batch_pattern_sets(seed: int = 0, counts=(1000, 1750, 3000, 5500, 9500, 16500, 29000, 50000),
                       lmin: int = 8, lmax: int = 64):
    """Keyword sets for the batched workload: even sets ACGT, odd sets Zipf-256."""
    sets = []
    for j, c in enumerate(counts):
        g = rng(seed + 1000 + j)
        if j % 2 == 0:
            sets.append(_random_acgt(g, c, lmin, lmax))
        else:
            sets.append(_random_zipf(g, c, lmin, lmax))
    return sets


def batch_texts(count: int, lmin: int, lmax: int, seed: int = 0):
    """``count`` texts with log-uniform lengths in [lmin, lmax]; even-indexed
    draws ACGT, odd Zipf-256 (decided by a seeded coin).  Returns (texts, kinds)
    with kind 0 = ACGT, 1 = Zipf."""
    g = rng(seed + 77)
    lengths = np.exp(g.uniform(np.log(lmin), np.log(lmax), size=count)).astype(np.int64)
    kinds = g.integers(0, 2, size=count)
    texts = []
    for i in range(count):
        sub = int(g.integers(0, 1 << 62))
        if kinds[i] == 0:
            texts.append(acgt_text(int(lengths[i]), sub))
        else:
            texts.append(zipf_text(int(lengths[i]), sub))
    return texts, kinds


def batch_layout(texts, kinds, n_sets: int = 8, seed: int = 0):
    """Pack ``texts`` back to back (no gaps, so most start unaligned) and give
    each a keyword set of its own alphabet, uniformly: sets 0, 2, 4, ... are
    ACGT and 1, 3, 5, ... Zipf-256 (``batch_pattern_sets``).  Returns
    (buffer, offsets, lengths, set index per text); a dense output laid out
    like the buffer uses the same offsets."""
    g = rng(seed + 99)
    lens = np.array([t.size for t in texts], dtype=np.int64)
    offs = np.zeros(len(texts), dtype=np.int64)
    if len(texts) > 1:
        offs[1:] = np.cumsum(lens)[:-1]
    buf = np.concatenate(texts) if len(texts) else np.zeros(0, dtype=np.uint8)
    half = (n_sets + 1) // 2
    pick = g.integers(0, 1 << 30, size=len(texts))
    sets = np.empty(len(texts), dtype=np.int64)
    for i, k in enumerate(kinds):
        if k == 0:
            sets[i] = 2 * (pick[i] % half)
        else:
            sets[i] = 2 * (pick[i] % (n_sets // 2)) + 1
    return buf, offs, lens, sets


def serve_pattern_sets(seed: int = 0, count: int = 16, kmin: int = 1000, kmax: int = 50_000,
                       lmin: int = 4, lmax: int = 100):
    """Keyword sets of the served workload: ``count`` sets with log-uniform
    keyword counts in [kmin, kmax] and lengths uniform in [lmin, lmax]; the
    first half random ACGT, the second half Zipf(1.1)-random bytes."""
    g = rng(seed + 2000)
    ks = np.exp(g.uniform(np.log(kmin), np.log(kmax), size=count)).astype(np.int64)
    sets = []
    for j in range(count):
        sub = rng(seed + 3000 + j)
        if j < count // 2:
            sets.append(_random_acgt(sub, int(ks[j]), lmin, lmax))
        else:
            sets.append(_random_zipf(sub, int(ks[j]), lmin, lmax))
    return sets


def serve_requests(count: int, pool_bytes: int, seed: int = 0, n_sets: int = 16, lmin: int = 256,
                   lmax: int = 64 << 20):
    """Requests of the served workload: (set index, pool offset, length) with
    lengths log-uniform in [lmin, lmax] and the set uniform; the offset is
    uniform in a text pool of ``pool_bytes`` of the set's alphabet (sets
    below n_sets // 2: ACGT, the rest Zipf)."""
    g = rng(seed + 4000)
    lens = np.exp(g.uniform(np.log(lmin), np.log(lmax), size=count)).astype(np.int64)
    lens = np.minimum(lens, pool_bytes)
    sets = g.integers(0, n_sets, size=count)
    offs = (g.random(count) * (pool_bytes - lens + 1)).astype(np.int64)
    return sets, offs, lens


def poisson_arrivals(count: int, rate_per_s: float, seed: int = 0) -> np.ndarray:
    """Arrival times in microseconds of a Poisson process of the given rate."""
    g = rng(seed + 5000)
    return np.cumsum(g.exponential(1e6 / rate_per_s, size=count))
