"""Seeded synthetic workloads for batched subsequence DTW (sDTW).

This module only *shapes inputs*: it draws random walks, cuts queries out of a
reference, adds noise, z-normalises and quantises.  It holds none of the
alignment arithmetic (no cost, no recurrence, no minimum), so both the CUDA
library's tests and the CPU oracle's tests can draw their inputs from here
without either side depending on the other.

Workload shapes follow the paper's evaluation: batches of 512 queries of length
2,000 against a reference of 100,000 samples (Section 6, the Table 1 set-up).
The paper drew its series from a cylinder-bell-funnel generator (Section 4);
that generator is not available here, so z-normalised Gaussian random walks
stand in for it, with queries cut from the reference at random offsets plus
N(0, 0.1^2) noise and a share of independent random-walk decoys.

z-normalisation follows Eq. 2, z = (x - mean) / S, with S the population
standard deviation (the variance divides by n, as the paper's statistic code
in Section 5.1 does); a constant series is only centred.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional

import numpy as np

SEED_BASE = 240306931

__all__ = [
    "SEED_BASE", "Workload", "rng_for", "random_walk", "znorm", "quantize_i8",
    "planted_batch", "tiny", "small_fp32", "paper_fp32", "paper_i8",
    "ragged_fp32", "stretched", "grad_subset", "by_name",
]


def rng_for(seed: int) -> np.random.Generator:
    """PCG64 generator for a seed (numpy's published bit generator)."""
    return np.random.Generator(np.random.PCG64(int(seed)))


def random_walk(rng: np.random.Generator, n: int) -> np.ndarray:
    """Gaussian random walk: cumulative sum of n standard normal steps (float64)."""
    return np.cumsum(rng.standard_normal(int(n)))


def random_walks(B: int, n: int, seed: int) -> np.ndarray:
    """B raw (not normalised) float32 random walks of length n: the input of a
    batch z-normalisation."""
    rng = rng_for(SEED_BASE + seed)
    return np.stack([random_walk(rng, n) for _ in range(B)]).astype(np.float32)


def znorm(v: np.ndarray) -> np.ndarray:
    """Eq. 2 standardisation in float64: (v - mean) / S with population S.

    Two-pass (mean first, then the centred second moment).  A series with
    S == 0 is returned centred, divided by 1.
    """
    v = np.asarray(v, dtype=np.float64)
    mu = v.mean()
    c = v - mu
    s = np.sqrt(np.mean(c * c))
    return c / (s if s > 0.0 else 1.0)


def quantize_i8(z: np.ndarray, scale: float = 8.0) -> np.ndarray:
    """Linear int8 code of a z-normalised series: clamp(rint(scale*z), -127, 127).

    rint rounds half to even.  This is the integer workload's input coding,
    not the paper's (unbuilt) codebook scheme.
    """
    q = np.rint(np.asarray(z, dtype=np.float64) * scale)
    return np.clip(q, -127, 127).astype(np.int8)


@dataclass
class Workload:
    """One batch: a reference, queries (uniform or ragged) and how they were made.

    ``queries`` is [B, N] for a uniform batch or the flat concatenation [sum N_q]
    with ``offsets`` [B+1] (int64) for a ragged one.  ``planted`` holds, per
    query, the reference offset the query was cut from, or -1 for a decoy.
    """
    name: str
    ref: np.ndarray
    queries: np.ndarray
    offsets: Optional[np.ndarray]
    lengths: np.ndarray
    planted: np.ndarray
    seed: int
    dtype: str
    recipe: dict = field(default_factory=dict)

    @property
    def B(self) -> int:
        return int(self.lengths.shape[0])

    @property
    def M(self) -> int:
        return int(self.ref.shape[0])

    @property
    def N(self) -> int:
        """Uniform query length, or the longest query of a ragged batch."""
        return int(self.lengths.max())

    @property
    def cells(self) -> int:
        """DP cells of the batch: sum over queries of N_q * M."""
        return int(self.lengths.astype(np.int64).sum()) * self.M

    def query(self, q: int) -> np.ndarray:
        if self.offsets is None:
            return self.queries[q]
        return self.queries[self.offsets[q]:self.offsets[q + 1]]


def planted_batch(rng: np.random.Generator, ref_z: np.ndarray, lengths: np.ndarray,
                  noise: float, decoy_frac: float):
    """Cut queries of the given lengths out of ``ref_z`` at uniform offsets.

    Each query is ref_z[o:o+n] + N(0, noise^2), z-normalised; a ``decoy_frac``
    share of the queries are instead independent z-normalised random walks
    (planted offset -1).  Returns (list of float64 queries, planted offsets).
    """
    M = ref_z.shape[0]
    B = lengths.shape[0]
    n_decoy = int(round(decoy_frac * B))
    decoy = np.zeros(B, dtype=bool)
    if n_decoy:
        decoy[rng.choice(B, size=n_decoy, replace=False)] = True
    out, planted = [], np.full(B, -1, dtype=np.int64)
    for q in range(B):
        n = int(lengths[q])
        if decoy[q]:
            out.append(znorm(random_walk(rng, n)))
            continue
        o = int(rng.integers(0, M - n + 1)) if M >= n else 0
        cut = ref_z[o:o + n]
        if cut.shape[0] < n:  # query longer than the reference: wrap-free pad by repeating
            cut = np.resize(cut, n)
        out.append(znorm(cut + noise * rng.standard_normal(n)))
        planted[q] = o
    return out, planted


def _uniform(name, seed, B, N, M, noise, decoy_frac, dtype="f32") -> Workload:
    rng = rng_for(seed)
    ref = znorm(random_walk(rng, M))
    lengths = np.full(B, N, dtype=np.int64)
    qs, planted = planted_batch(rng, ref, lengths, noise, decoy_frac)
    queries = np.stack(qs) if B else np.zeros((0, N))
    recipe = dict(ref="znorm(cumsum N(0,1))", M=M, B=B, N=N, noise_sigma=noise,
                  decoy_frac=decoy_frac, seed=seed)
    return Workload(name, ref.astype(np.float32), queries.astype(np.float32), None,
                    lengths, planted, seed, dtype, recipe)


def tiny(seed: int = SEED_BASE, B: int = 4, N: int = 16, M: int = 300,
         noise: float = 0.1, decoy_frac: float = 0.25) -> Workload:
    """A small uniform fp32 batch for quick checks (same recipe, any shape)."""
    return _uniform("tiny", seed, B, N, M, noise, decoy_frac)


def small_fp32(seed: int = SEED_BASE + 1) -> Workload:
    """8 queries x 128 samples vs a 4,096-sample reference, fp32, no decoys."""
    return _uniform("sdtw_fp32_8x128_vs_4096", seed, 8, 128, 4096, 0.1, 0.0)


def paper_fp32(seed: int = SEED_BASE + 2, B: int = 512, N: int = 2000,
               M: int = 100_000) -> Workload:
    """The paper's batch: 512 x 2,000 vs 100,000, fp32, 10% random-walk decoys."""
    return _uniform(f"sdtw_fp32_{B}x{N}_vs_{M}", seed, B, N, M, 0.1, 0.1)


def paper_i8(seed: int = SEED_BASE + 3, B: int = 512, N: int = 2000,
             M: int = 100_000) -> Workload:
    """The paper's batch shape quantised to int8 codes (costs accumulate in int32)."""
    w = paper_fp32(seed, B, N, M)
    return Workload(f"sdtw_i8_{B}x{N}_vs_{M}", quantize_i8(w.ref), quantize_i8(w.queries),
                    None, w.lengths, w.planted, seed, "i8",
                    dict(w.recipe, quantize="clamp(rint(8z), -127, 127)"))


def ragged_fp32(seed: int = SEED_BASE + 4, B: int = 2048, n_lo: int = 200,
                n_hi: int = 4000, M: int = 1_000_000) -> Workload:
    """Ragged batch: B queries with lengths uniform in [n_lo, n_hi], planted cuts."""
    rng = rng_for(seed)
    ref = znorm(random_walk(rng, M))
    lengths = rng.integers(n_lo, n_hi + 1, size=B).astype(np.int64)
    qs, planted = planted_batch(rng, ref, lengths, 0.1, 0.0)
    offsets = np.zeros(B + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(lengths)
    flat = np.concatenate(qs) if B else np.zeros(0)
    recipe = dict(ref="znorm(cumsum N(0,1))", M=M, B=B, n_lo=n_lo, n_hi=n_hi,
                  noise_sigma=0.1, decoy_frac=0.0, seed=seed)
    return Workload(f"sdtw_ragged_fp32_{B}xU[{n_lo},{n_hi}]_vs_{M}", ref.astype(np.float32),
                    flat.astype(np.float32), offsets, lengths, planted, seed, "f32", recipe)


def stretched(seed: int = SEED_BASE + 6, B: int = 16, N: int = 400, M: int = 40_000,
              step_lo: int = 4, step_hi: int = 24, noise: float = 0.05, scale: float = 1.0) -> Workload:
    """Queries that are the reference subsampled by an integer step in
    [step_lo, step_hi] (plus noise, z-normalised): each optimal path runs about
    `step` columns per row, long horizontal runs across the reference.  With
    scale != 1 the reference and the queries are multiplied by it afterwards
    (larger costs on a small shape)."""
    rng = rng_for(seed)
    ref = znorm(random_walk(rng, M))
    qs, planted = [], np.zeros(B, dtype=np.int64)
    for q in range(B):
        step = int(rng.integers(step_lo, step_hi + 1))
        span = step * (N - 1) + 1
        o = int(rng.integers(0, max(1, M - span)))
        cut = ref[o:o + span:step][:N]
        if cut.shape[0] < N:
            cut = np.resize(cut, N)
        qs.append(znorm(cut + noise * rng.standard_normal(N)))
        planted[q] = o
    recipe = dict(ref="znorm(cumsum N(0,1))", M=M, B=B, N=N, step=(step_lo, step_hi), noise_sigma=noise, seed=seed,
                  scale=scale)
    return Workload(f"sdtw_stretched_{B}x{N}_vs_{M}", (scale * ref).astype(np.float32),
                    (scale * np.stack(qs)).astype(np.float32),
                    None, np.full(B, N, dtype=np.int64), planted, seed, "f32", recipe)


def grad_subset(seed: int = SEED_BASE + 5) -> Workload:
    """Gradient-check subset: 8 queries x 64 samples vs a 512-sample reference."""
    return _uniform("sdtw_grad_8x64_vs_512", seed, 8, 64, 512, 0.1, 0.1)


def by_name(name: str, **kw) -> Workload:
    table = {"small": small_fp32, "paper": paper_fp32, "paper_i8": paper_i8,
             "ragged": ragged_fp32, "grad": grad_subset, "tiny": tiny, "stretched": stretched}
    return table[name](**kw)
