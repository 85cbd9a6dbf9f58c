"""Seeded synthetic workloads, host side (numpy).

Every value is a pure function of (seed, stream, index): the generator is the
SplitMix64 output function (Steele, Lea & Flood, OOPSLA 2014; constants from
Vigna's public-domain splitmix64.c) applied to a counter, so the device
generator in ``gen/device.cu`` reproduces it bit for bit.  Nothing here
computes any part of the sorting method itself: these are inputs only.

Recipes (the shapes of the paper's workloads, Section III-B and Table VII):

* uniform integers below m: Lemire's multiply-shift on the top bits of a draw;
* "Zipf over 1,024 distinct values": value of rank r is a 32-bit bijective
  hash of r (so the 1,024 values are distinct by construction), ranks are
  drawn by inverse CDF of p_r ~ r^-s over an fp64 CDF table;
* presorted / nearly sorted / reversed arrays (Section III-B edge cases);
* a taxi-timestamp-shaped uint64 ramp with 5% uniform replacements;
* log-uniform segment lengths for batches of many arrays.
"""
from __future__ import annotations

import math

import numpy as np

U64 = np.uint64
GOLDEN = 0x9E3779B97F4A7C15
MIX1 = 0xBF58476D1CE4E5B9
MIX2 = 0x94D049BB133111EB
M64 = (1 << 64) - 1

# P(replace) = 0.05 expressed on the 53-bit integer scale, so host and device
# take the same integer decision: replace iff (draw >> 11) < REPLACE_53.
REPLACE_53 = 450359962737050  # ceil(0.05 * 2**53)


def mix64_int(z: int) -> int:
    """SplitMix64 finaliser on a Python int (mod 2**64)."""
    z &= M64
    z = ((z ^ (z >> 30)) * MIX1) & M64
    z = ((z ^ (z >> 27)) * MIX2) & M64
    return z ^ (z >> 31)


def mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 finaliser on a uint64 array (wrapping arithmetic)."""
    z = z.astype(U64, copy=True)
    z ^= z >> U64(30)
    z *= U64(MIX1)
    z ^= z >> U64(27)
    z *= U64(MIX2)
    z ^= z >> U64(31)
    return z


def stream_key(seed: int, stream: int) -> int:
    """Per-(seed, stream) starting state of the counter generator."""
    return mix64_int((seed * GOLDEN + mix64_int(stream + GOLDEN)) & M64)


def draws(seed: int, stream: int, start: int, count: int) -> np.ndarray:
    """Draws number start .. start+count-1 of stream (seed, stream), as uint64."""
    key = U64(stream_key(seed, stream))
    i = np.arange(start, start + count, dtype=U64)
    with np.errstate(over="ignore"):
        z = key + (i + U64(1)) * U64(GOLDEN)
    return mix64(z)


def draw_int(seed: int, stream: int, i: int) -> int:
    return mix64_int(stream_key(seed, stream) + (i + 1) * GOLDEN)


def below32(r: np.ndarray, m: int) -> np.ndarray:
    """Uniform integer in [0, m) for 1 <= m <= 2**32 from 64-bit draws."""
    assert 1 <= m <= (1 << 32)
    return ((r >> U64(32)) * U64(m)) >> U64(32)


def mulhi64(a: np.ndarray, b: int) -> np.ndarray:
    """High 64 bits of the 128-bit product a*b (a uint64 array, b < 2**64)."""
    mask = U64(0xFFFFFFFF)
    a_lo, a_hi = a & mask, a >> U64(32)
    b_lo, b_hi = U64(b & 0xFFFFFFFF), U64(b >> 32)
    ll = a_lo * b_lo
    lh = a_lo * b_hi
    hl = a_hi * b_lo
    hh = a_hi * b_hi
    mid = (ll >> U64(32)) + (lh & mask) + (hl & mask)
    return hh + (lh >> U64(32)) + (hl >> U64(32)) + (mid >> U64(32))


def below64(r: np.ndarray, m: int) -> np.ndarray:
    """Uniform integer in [0, m) for 1 <= m <= 2**64 (Lemire multiply-shift)."""
    assert 1 <= m <= (1 << 64)
    if m == (1 << 64):
        return r.copy()
    return mulhi64(r, m)


def unit53(r: np.ndarray) -> np.ndarray:
    """fp64 in [0, 1) from the top 53 bits of a draw."""
    return (r >> U64(11)).astype(np.float64) * (2.0 ** -53)


def hash32(x: np.ndarray) -> np.ndarray:
    """A bijection on 32-bit integers (xorshift-multiply, 'lowbias32' by C. Wellons)."""
    x = x.astype(np.uint32, copy=True)
    x ^= x >> np.uint32(16)
    x *= np.uint32(0x7FEB352D)
    x ^= x >> np.uint32(15)
    x *= np.uint32(0x846CA68B)
    x ^= x >> np.uint32(16)
    return x


# ----------------------------------------------------------------------------
# Elementary generators (each mirrored by a kernel in gen/device.cu)
# ----------------------------------------------------------------------------

def uniform_u32(n: int, seed: int, stream: int, m: int, start: int = 0) -> np.ndarray:
    """n keys i.i.d. uniform in [0, m), m <= 2**32."""
    with np.errstate(over="ignore"):
        return below32(draws(seed, stream, start, n), m).astype(np.uint32)


def zipf_cdf(n_values: int, s: float) -> np.ndarray:
    """fp64 CDF of p_r proportional to r**-s over ranks r = 1..n_values.

    Built by sequential summation in rank order; the last entry is set to 1.0
    exactly so every unit draw maps to a valid rank.
    """
    w = np.array([math.pow(r, -s) for r in range(1, n_values + 1)], dtype=np.float64)
    total = 0.0
    for x in w:
        total += x
    cdf = np.empty(n_values, dtype=np.float64)
    acc = 0.0
    for r in range(n_values):
        acc += w[r]
        cdf[r] = acc / total
    cdf[-1] = 1.0
    return cdf


def zipf_values(seed: int, stream: int, n_values: int) -> np.ndarray:
    """The n_values distinct uint32 values of a Zipf workload (value of rank r)."""
    k = draw_int(seed, stream, 0)
    k1 = np.uint32(k & 0xFFFFFFFF)
    k2 = np.uint32(k >> 32)
    r = np.arange(n_values, dtype=np.uint32)
    return hash32(r ^ k1) ^ k2


def zipf_u32(n: int, seed: int, stream_values: int, stream_ranks: int,
             n_values: int = 1024, s: float = 1.1, start: int = 0) -> np.ndarray:
    """n keys drawn Zipf(s) over n_values distinct random uint32 values."""
    values = zipf_values(seed, stream_values, n_values)
    cdf = zipf_cdf(n_values, s)
    u = unit53(draws(seed, stream_ranks, start, n))
    rank = np.searchsorted(cdf, u, side="right")  # first index with cdf > u
    np.minimum(rank, n_values - 1, out=rank)
    return values[rank]


def apply_swaps(a: np.ndarray, n_swaps: int, seed: int, stream: int) -> np.ndarray:
    """Apply n_swaps sequential swaps of index pairs (i, j) drawn uniform in [0, len(a))."""
    n = len(a)
    if n_swaps == 0 or n == 0:
        return a
    r = draws(seed, stream, 0, 2 * n_swaps)
    with np.errstate(over="ignore"):
        idx = below64(r, n).astype(np.int64)
    ii = idx[0::2].tolist()
    jj = idx[1::2].tolist()
    for i, j in zip(ii, jj):
        t = a[i]
        a[i] = a[j]
        a[j] = t
    return a


def ramp_u64(n: int, seed: int, t0: int = 1_700_000_000_000_000_000,
             max_step: int = 1000) -> np.ndarray:
    """Taxi-timestamp-shaped uint64 keys: a ramp with steps uniform in
    [0, max_step], then each key replaced with probability 0.05 by a uniform
    draw over [t_0, t_{n-1}]."""
    if n == 0:
        return np.zeros(0, dtype=np.uint64)
    with np.errstate(over="ignore"):
        steps = below64(draws(seed, 1, 0, n), max_step + 1)
        steps[0] = 0
        t = np.cumsum(steps, dtype=np.uint64) + U64(t0)
        last = int(t[-1])
        rep = (draws(seed, 2, 0, n) >> U64(11)) < U64(REPLACE_53)
        repl = below64(draws(seed, 3, 0, n), last - t0 + 1) + U64(t0)
    t[rep] = repl[rep]
    return t


# ----------------------------------------------------------------------------
# Second workload family (Section III-B, Table VII)
# ----------------------------------------------------------------------------

GAUSS_TERMS = 12          # Irwin-Hall: a sum of 12 uniform 32-bit integers
KMER_LEN = 30             # k-mers of 30 bases, 2 bits each: 60-bit keys, k = 4^30
KMER_BLOCK = 1000         # bases per block of the synthetic genome
KMER_REPEATS = 16         # distinct repeat units the blocks are copied from
KMER_MUT_53 = 90071992547410   # P(point mutation) = 0.01 on the 53-bit integer scale


def gauss_sigma_q16(k: int) -> int:
    """sigma = sqrt(k / 4) = sqrt(k) / 2 in 16.16 fixed point (the one fp64
    step, taken on the host and passed to both generators)."""
    return int(round(math.sqrt(k) / 2.0 * 65536.0))


def gaussian_i32(n: int, seed: int, stream: int, k: int, start: int = 0) -> np.ndarray:
    """n int32 keys shaped like N(0, sigma^2 = k/4) (Section III-B).  Integer
    only, so host and device agree bit for bit: S is the sum of 12 uniform
    32-bit integers (the top and bottom halves of 6 draws per key), whose
    mean 6 (2^32 - 1) and standard deviation ~2^32 make
    Z = (S - mean) / 2^32 close to a standard normal (Irwin-Hall);
    key = floor((S - 6 (2^32 - 1)) * sigma_q16 / 2^48)."""
    sq = gauss_sigma_q16(k)
    d = draws(seed, stream, 6 * start, 6 * n).reshape(n, 6) if n else np.zeros((0, 6), U64)
    hi = (d >> U64(32)).astype(np.int64)
    lo = (d & U64(0xFFFFFFFF)).astype(np.int64)
    S = hi.sum(axis=1) + lo.sum(axis=1)
    dev_ = S - 6 * (2**32 - 1)
    return ((dev_ * sq) >> 48).astype(np.int32)


def kmer_bases(count: int, seed: int, stream: int, start: int = 0) -> np.ndarray:
    """Bases (0..3) of a synthetic repetitive genome at positions
    [start, start + count): position p lies in block p // 1000, a copy of one
    of 16 repeat units (chosen per block), at offset p % 1000 of it; each
    position mutates to a random base with probability 0.01."""
    if count == 0:
        return np.zeros(0, dtype=np.uint64)
    p = np.arange(start, start + count, dtype=np.int64)
    blocks = p // KMER_BLOCK
    b0 = int(blocks[0])
    nb = int(blocks[-1]) - b0 + 1
    with np.errstate(over="ignore"):
        rep = (below64(draws(seed, stream, b0, nb), KMER_REPEATS)).astype(np.int64)
    unit = draws(seed, stream + 1, 0, KMER_REPEATS * KMER_BLOCK) >> U64(62)
    base = unit[rep[blocks - b0] * KMER_BLOCK + (p % KMER_BLOCK)]
    m = draws(seed, stream + 2, start, count)
    mut = (m >> U64(11)) < U64(KMER_MUT_53)
    base = np.where(mut, m & U64(3), base)
    return base.astype(U64)


def kmer_u64(n: int, seed: int, stream: int, start: int = 0) -> np.ndarray:
    """n uint64 k-mer keys: key i packs the 30 bases at positions
    i .. i + 29 of the genome, first base in the high bits (60-bit keys)."""
    b = kmer_bases(n + KMER_LEN - 1, seed, stream, start)
    key = np.zeros(n, dtype=U64)
    for j in range(KMER_LEN):
        key |= b[j:j + n] << U64(2 * (KMER_LEN - 1 - j))
    return key


# ----------------------------------------------------------------------------
# Served requests generated by the library (config 5)
# ----------------------------------------------------------------------------

REPLACE_1PCT_53 = 90071992547410   # P = 0.01 on the 53-bit integer scale
REQ_KINDS = ("a", "b", "c", "e")   # config-4 shapes, as gen_kind 0..3


def replace_u32(a: np.ndarray, seed: int, stream: int, thresh53: int = REPLACE_1PCT_53) -> np.ndarray:
    """Replace each position with probability thresh53 / 2^53 by a uniform
    32-bit draw (position-parallel: a nearly sorted shape without a
    sequential swap chain)."""
    n = len(a)
    if n == 0:
        return a
    d = draws(seed, stream, 0, n)
    rep = (d >> U64(11)) < U64(thresh53)
    v = (draws(seed, stream + 1, 0, n) >> U64(32)).astype(np.uint32)
    a[rep] = v[rep]
    return a


def request_stream(rid: int, part: int) -> int:
    """Stream of part `part` of served request `rid` (keys 0, Zipf values 1, replacement 2)."""
    return (1 << 40) + 4 * rid + part


def request_keys(seed: int, rid: int, kind: int, n: int) -> np.ndarray:
    """The uint32 keys of a library-generated served request (gen_kind 0..3:
    uniform below 4096; Zipf(1.1) over 1,024 distinct values; uniform 32-bit;
    sorted uniform 32-bit with 1% of the positions replaced)."""
    s0 = request_stream(rid, 0)
    if kind == 0:
        return uniform_u32(n, seed, s0, 4096)
    if kind == 1:
        return zipf_u32(n, seed, request_stream(rid, 1), s0)
    if kind == 2:
        return uniform_u32(n, seed, s0, 1 << 32)
    if kind == 3:
        return replace_u32(np.sort(uniform_u32(n, seed, s0, 1 << 32)), seed, request_stream(rid, 2))
    raise ValueError(kind)


# ----------------------------------------------------------------------------
# The workload configurations
# ----------------------------------------------------------------------------

CONFIG2_VARIANTS = ("a", "b", "c", "d", "e", "f")
N_CFG1 = 1 << 20
N_CFG2 = 1 << 28
N_CFG3 = 1 << 27
SEED_CFG1, SEED_CFG2, SEED_CFG3, SEED_CFG4, SEED_CFG5 = 0, 1, 2, 3, 5


def config1(n: int = N_CFG1) -> np.ndarray:
    """Single array, n uint32 uniform in [0, 255] (IoT-reading shape, k=256)."""
    return uniform_u32(n, SEED_CFG1, 0, 256)


def config2(variant: str, n: int = N_CFG2, seed: int = SEED_CFG2) -> np.ndarray:
    """Single uint32 arrays: (a) uniform [0,4095]; (b) Zipf(1.1) over 1,024
    distinct values; (c) uniform [0,2^32); (d) sorted (c); (e) (d) with
    floor(n/100) random swaps; (f) reversed (d)."""
    if variant == "a":
        return uniform_u32(n, seed, 1, 4096)
    if variant == "b":
        return zipf_u32(n, seed, 2, 3)
    if variant == "c":
        return uniform_u32(n, seed, 4, 1 << 32)
    base = np.sort(uniform_u32(n, seed, 4, 1 << 32))
    if variant == "d":
        return base
    if variant == "e":
        return apply_swaps(base, n // 100, seed, 5)
    if variant == "f":
        return base[::-1].copy()
    raise ValueError(variant)


def config3(n: int = N_CFG3, seed: int = SEED_CFG3):
    """Key-value: uint64 timestamp ramp keys, uint32 payload = original index."""
    return ramp_u64(n, seed), np.arange(n, dtype=np.uint32)


# Config 4: a batch of many uneven arrays.
SEG_TYPES = ("a", "b", "c", "e")


def log_uniform_lengths(count: int, seed: int, stream: int, lo: int, hi: int) -> np.ndarray:
    """Lengths floor(exp(ln lo + u (ln hi - ln lo))) clamped to [lo, hi] (host only)."""
    u = unit53(draws(seed, stream, 0, count))
    L = np.floor(np.exp(math.log(lo) + u * (math.log(hi) - math.log(lo)))).astype(np.int64)
    return np.clip(L, lo, hi)


def config4_layout(n_seg: int = 100_000, seed: int = SEED_CFG4,
                   lo: int = 16, hi: int = 1 << 20):
    """Segment lengths, types (index into SEG_TYPES) and offsets of the batch."""
    lengths = log_uniform_lengths(n_seg, seed, 1, lo, hi)
    with np.errstate(over="ignore"):
        types = below32(draws(seed, 2, 0, n_seg), len(SEG_TYPES)).astype(np.int64)
    offsets = np.zeros(n_seg + 1, dtype=np.uint64)
    np.cumsum(lengths, out=offsets[1:])
    return lengths, types, offsets


def segment_stream(seg: int, part: int) -> int:
    """Stream id of part `part` of segment `seg` (keys=0, zipf values=1, swaps=2)."""
    return 16 + 4 * seg + part


def config4_segment(seg: int, length: int, typ: int, seed: int = SEED_CFG4) -> np.ndarray:
    """Keys of one segment of the batch, regenerated from (seed, segment id)."""
    t = SEG_TYPES[typ]
    s_keys = segment_stream(seg, 0)
    if t == "a":
        return uniform_u32(length, seed, s_keys, 4096)
    if t == "b":
        return zipf_u32(length, seed, segment_stream(seg, 1), s_keys)
    if t == "c":
        return uniform_u32(length, seed, s_keys, 1 << 32)
    if t == "e":
        base = np.sort(uniform_u32(length, seed, s_keys, 1 << 32))
        return apply_swaps(base, length // 100, seed, segment_stream(seg, 2))
    raise ValueError(t)
