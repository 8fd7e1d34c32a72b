"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds no arithmetic of the sorting method: it only draws keys.
Every generator is a pure function of its seed (numpy's Philox4x64 bit
generator), so the CUDA path and the CPU oracle read identical buffers.

Distributions:
  * ``uniform``      keys uniform over [0, 2^64)                 (Sec. 7.5 UNIF)
  * ``gauss_mix``    32 Gaussians (sigma = 2^40, means uniform) cast to u64
  * ``zipf``         values drawn from 2^12 distinct keys with Zipf(s=1.2)
  * the six inputs of Sec. 7.5 (UNIF, SKEW1, SKEW2, SKEW3, GAUSS, AllZeros)
  * ``plummer_morton`` 64-bit Morton keys of a Plummer sphere, 21 bits per
    axis, with the particle index as a u32 payload (the N-body workload of
    Sec. 7.4 stands in for the ChaNGa datasets, which are not available)
  * ``batch_jobs``   many int64 jobs with log-uniform sizes
  * ``lognormal_job`` lognormal(0, 2) keys scaled to 2^63
"""
from __future__ import annotations

import math

import numpy as np

_CHUNK = 1 << 24


def rng(seed: int, stream: int = 0) -> np.random.Generator:
    """numpy Philox4x64 generator keyed by (seed, stream)."""
    return np.random.Generator(np.random.Philox(key=[seed & ((1 << 64) - 1), stream & ((1 << 64) - 1)]))


def uniform(N: int, seed: int) -> np.ndarray:
    g = rng(seed, 1)
    out = np.empty(N, dtype=np.uint64)
    for a in range(0, N, _CHUNK):
        b = min(N, a + _CHUNK)
        out[a:b] = g.bit_generator.random_raw(b - a)
    return out


def gauss_mix(N: int, seed: int, ncomp: int = 32, sigma: float = 2.0 ** 40) -> np.ndarray:
    g = rng(seed, 2)
    means = g.bit_generator.random_raw(ncomp).view(np.int64)
    out = np.empty(N, dtype=np.uint64)
    for a in range(0, N, _CHUNK):
        b = min(N, a + _CHUNK)
        comp = g.integers(0, ncomp, size=b - a)
        off = np.rint(g.standard_normal(b - a) * sigma).astype(np.int64)
        with np.errstate(over="ignore"):
            out[a:b] = (means[comp] + off).view(np.uint64)
    return out


def _zipf_table(g: np.random.Generator, distinct: int, s: float):
    values = g.bit_generator.random_raw(distinct)
    while np.unique(values).size != distinct:  # practically never
        values = g.bit_generator.random_raw(distinct)
    w = np.arange(1, distinct + 1, dtype=np.float64) ** (-s)
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    return values, cdf


def zipf(N: int, seed: int, distinct: int = 1 << 12, s: float = 1.2) -> np.ndarray:
    g = rng(seed, 3)
    values, cdf = _zipf_table(g, distinct, s)
    out = np.empty(N, dtype=np.uint64)
    for a in range(0, N, _CHUNK):
        b = min(N, a + _CHUNK)
        idx = np.searchsorted(cdf, g.random(b - a), side="right")
        out[a:b] = values[np.minimum(idx, distinct - 1)]
    return out


# --- the input distributions of Sec. 7.5 -------------------------------------

def skew1(N: int, seed: int) -> np.ndarray:
    """Half uniform over the whole range, half uniform over a range of 1000."""
    g = rng(seed, 4)
    out = g.bit_generator.random_raw(N)
    half = N // 2
    base = int(g.bit_generator.random_raw(1)[0]) % ((1 << 64) - 1000)
    out[:half] = np.uint64(base) + g.integers(0, 1000, size=half).astype(np.uint64)
    g.shuffle(out)
    return out


def skew2(N: int, seed: int) -> np.ndarray:
    """Uniform over [0, 100] (101 distinct values)."""
    return rng(seed, 5).integers(0, 101, size=N).astype(np.uint64)


def skew3(N: int, seed: int) -> np.ndarray:
    """Bitwise AND of two uniform keys."""
    g = rng(seed, 6)
    return g.bit_generator.random_raw(N) & g.bit_generator.random_raw(N)


def gauss(N: int, seed: int) -> np.ndarray:
    """One Gaussian centred in the key range (sigma = 2^58)."""
    g = rng(seed, 7)
    v = np.rint(g.standard_normal(N) * 2.0 ** 58).astype(np.int64)
    with np.errstate(over="ignore"):
        return (v.view(np.uint64) + np.uint64(1 << 63))


def allzeros(N: int, seed: int = 0) -> np.ndarray:
    return np.zeros(N, dtype=np.uint64)


def nested_clusters(N: int, seed: int) -> np.ndarray:
    """A stress input for the radix recursion: a third of the keys uniform
    over 64 bits, a third in a window of width 2^40, and a third in a window
    of width 2^20 nested inside it, drawn from 4096 distinct values (many
    duplicates).  The nested window keeps one digit bin over the on-chip
    capacity for three levels of the most-significant-digit split."""
    g = rng(seed, 9)
    c = np.uint64(0x5A12_3400_0000_0000)
    n0, n1 = N // 3, N // 3
    n2 = N - n0 - n1
    a = g.bit_generator.random_raw(n0).astype(np.uint64)
    b = c + (g.bit_generator.random_raw(n1).astype(np.uint64) >> np.uint64(24))
    d = c + np.uint64(1 << 39) + (g.integers(0, 4096, n2, dtype=np.uint64) << np.uint64(8))
    out = np.concatenate([a, b, d])
    return out[g.permutation(N)]


def duplicate_groups(N: int, seed: int, nvals: int, share: float, adjacent: bool = False) -> np.ndarray:
    """A share of the keys drawn from nvals values (each repeated many
    times), the rest uniform over 64 bits.  With ``adjacent`` the repeated
    values are consecutive integers, so several of them share any coarse
    digit of the key range."""
    g = rng(seed, 10)
    nd = int(N * share)
    if adjacent:
        base = np.uint64(g.bit_generator.random_raw(1)[0] >> np.uint64(1))
        vals = base + np.arange(nvals, dtype=np.uint64)
    else:
        vals = g.bit_generator.random_raw(nvals).astype(np.uint64)
    out = np.concatenate([vals[g.integers(0, nvals, nd)], g.bit_generator.random_raw(N - nd).astype(np.uint64)])
    return out[g.permutation(N)]


PAPER_DISTRIBUTIONS = {
    "UNIF": uniform, "SKEW1": skew1, "SKEW2": skew2, "SKEW3": skew3, "GAUSS": gauss, "AllZeros": allzeros,
}

SCALE_DISTRIBUTIONS = {"uniform": uniform, "gauss_mix": gauss_mix, "zipf": zipf}


# --- N-body workload -----------------------------------------------------------

def _spread3(v: np.ndarray) -> np.ndarray:
    """Insert two zero bits between the 21 low bits of v (Morton interleave)."""
    v = v.astype(np.uint64) & np.uint64(0x1FFFFF)
    v = (v | (v << np.uint64(32))) & np.uint64(0x1F00000000FFFF)
    v = (v | (v << np.uint64(16))) & np.uint64(0x1F0000FF0000FF)
    v = (v | (v << np.uint64(8))) & np.uint64(0x100F00F00F00F00F)
    v = (v | (v << np.uint64(4))) & np.uint64(0x10C30C30C30C30C3)
    v = (v | (v << np.uint64(2))) & np.uint64(0x1249249249249249)
    return v


def _cbrt(x: np.ndarray) -> np.ndarray:
    """Cube root of positive doubles by Newton's method from above, with
    IEEE add, multiply and divide only, so the same bits come out on every
    machine (library sin/cos/pow differ between platforms by an ulp, enough to
    move a quantised coordinate across a cell boundary)."""
    x = np.asarray(x, dtype=np.float64)
    _, e = np.frexp(x)                                  # x = f 2^e, f in [0.5, 1)
    y = np.ldexp(np.ones_like(x), -((-e) // 3))          # 2^ceil(e/3) >= cbrt(x)
    for _ in range(12):                                 # monotone from above; 12 steps reach the ulp
        y = (2.0 * y + x / (y * y)) / 3.0
    return y


def _plummer_radius(m: np.ndarray) -> np.ndarray:
    """r = (m^(-2/3) - 1)^(-1/2) for a mass fraction m in (0, 1)."""
    c = _cbrt(m)
    return np.sqrt((c * c) / (1.0 - c * c))


def _unit_vectors(g: np.random.Generator, n: int) -> np.ndarray:
    """n isotropic unit vectors: points uniform in the cube [-1, 1]^3 kept
    when inside the unit ball (and not at its centre), then normalised."""
    out = np.empty((0, 3), dtype=np.float64)
    while out.shape[0] < n:
        v = 2.0 * g.random((2 * (n - out.shape[0]) + 64, 3)) - 1.0
        s = v[:, 0] * v[:, 0] + v[:, 1] * v[:, 1] + v[:, 2] * v[:, 2]
        keep = (s <= 1.0) & (s > 1e-12)
        v = v[keep] / np.sqrt(s[keep])[:, None]
        out = np.concatenate([out, v])
    return out[:n]


def _plummer_chunk(seed: int, c: int, n: int, bits: int) -> np.ndarray:
    g = rng(seed, (8 << 32) | c)
    r_max = float(_plummer_radius(np.array([0.999]))[0])
    scale = float(1 << bits)
    m = 0.999 * (1.0 - g.random(n))  # (0, 0.999]
    r = _plummer_radius(m)
    d = _unit_vectors(g, n)
    q = [np.clip(np.floor((r * d[:, a] + r_max) / (2.0 * r_max) * scale), 0, scale - 1).astype(np.uint64)
         for a in range(3)]
    return _spread3(q[0]) | (_spread3(q[1]) << np.uint64(1)) | (_spread3(q[2]) << np.uint64(2))


def plummer_morton(N: int, seed: int, bits: int = 21):
    """Morton keys of a Plummer sphere plus the particle index as payload.

    Radius from the Plummer mass profile m(r) = r^3 (1+r^2)^(-3/2): for a mass
    fraction m ~ U(0, 0.999], r = (m^(-2/3) - 1)^(-1/2); isotropic direction
    (rejection from the cube); each axis quantised to ``bits`` bits over
    [-r_max, r_max] with r_max = r(0.999).  Only IEEE add, multiply, divide
    and square root are used, so every machine draws the same keys.  Chunks
    of 2^22 particles draw from their own streams, so the chunks are
    generated on all host cores and the result does not depend on the count.
    """
    from concurrent.futures import ThreadPoolExecutor
    import os

    chunk = 1 << 22
    keys = np.empty(N, dtype=np.uint64)

    def work(c):
        a = c * chunk
        b = min(N, a + chunk)
        keys[a:b] = _plummer_chunk(seed, c, b - a, bits)

    nchunks = (N + chunk - 1) // chunk
    with ThreadPoolExecutor(max_workers=max(1, min(16, os.cpu_count() or 1))) as ex:
        list(ex.map(work, range(nchunks)))
    payload = np.arange(N, dtype=np.uint64).astype(np.uint32)
    return keys, payload


# --- batched and served jobs ---------------------------------------------------

def batch_job_plan(njobs: int, seed: int, lo_log2: int = 10, hi_log2: int = 22):
    """Sizes (log-uniform in [2^lo, 2^hi]) and the uniform-or-Zipf coin of
    every job of a batch."""
    g = rng(seed, 9)
    u = g.random(njobs)
    sizes = np.floor(2.0 ** (lo_log2 + (hi_log2 - lo_log2) * u)).astype(np.int64)
    coin = g.random(njobs) < 0.5
    return sizes, coin


def batch_job(j: int, seed: int, n: int, uniform_coin: bool, zipf_s: float = 1.1,
              zipf_distinct: int = 1 << 16) -> np.ndarray:
    """Keys of job j of a batch (int64): every job draws from its own streams."""
    if uniform_coin:
        return uniform(int(n), seed * 1000003 + j).view(np.int64)
    return zipf(int(n), seed * 1000003 + j, distinct=zipf_distinct, s=zipf_s).view(np.int64)


def batch_jobs(njobs: int, seed: int, lo_log2: int = 10, hi_log2: int = 22, zipf_s: float = 1.1,
               zipf_distinct: int = 1 << 16):
    """Independent int64 jobs with sizes log-uniform in [2^lo, 2^hi]; each is
    uniform or Zipf by a seeded coin.  Returns (list of int64 arrays, kinds)."""
    from concurrent.futures import ThreadPoolExecutor
    import os

    sizes, coin = batch_job_plan(njobs, seed, lo_log2, hi_log2)
    kinds = ["uniform" if coin[j] else "zipf" for j in range(njobs)]

    def one(j):  # generated on all host cores
        return batch_job(j, seed, int(sizes[j]), bool(coin[j]), zipf_s, zipf_distinct)

    with ThreadPoolExecutor(max_workers=max(1, min(16, os.cpu_count() or 1))) as ex:
        jobs = list(ex.map(one, range(njobs)))
    return jobs, kinds


def lognormal_job(n: int, seed: int, sigma: float = 2.0) -> np.ndarray:
    """lognormal(0, sigma) keys on one fixed scale for every job: x / e^(6 sigma)
    (six standard deviations of log x) times 2^63, clipped at 2^63 - 1024.  The
    scale does not depend on the job, so jobs of the same stream share one key
    distribution (the one a learned CDF model is trained on)."""
    x = rng(seed, 11).lognormal(0.0, sigma, size=n)
    u = np.minimum(x / math.exp(6.0 * sigma), 1.0)
    return np.floor(u * float((1 << 63) - 1024)).astype(np.uint64)
