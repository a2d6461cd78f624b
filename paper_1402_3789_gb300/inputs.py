"""Seeded synthetic inputs for the nearest-neighbour-method (NNM) clustering path.

The paper clusters an unnamed data set of up to 2 million records with up to 25
features (abstract; "Introduction") and ships none, so these Gaussian-mixture
generators stand in for it.  This module only draws random numbers: it holds none
of the method's arithmetic (no distances, no minima, no merges), so both the CUDA
path and the CPU oracle may take their inputs from it.

Draw order for every mixture (NumPy PCG64 via ``default_rng(seed)``):
centres, per-component sigmas, component labels (equal weights), Gaussian
draws, optional noise rows / quantisation / duplicates, then a global row
shuffle so that clusters are not contiguous.  Values are cast to float32 last.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = ["Workload", "WORKLOADS", "mixture", "make", "batched_instances"]


@dataclass(frozen=True)
class Workload:
    """One named synthetic workload: sizes, mixture recipe and restrictions."""

    name: str
    n: int
    d: int
    components: int
    centre_hi: float
    sigma: tuple  # ("fixed", s) | ("per_component", lo, hi) | ("per_axis", lo, hi)
    seed: int
    noise_frac: float = 0.0
    grid: float = 0.0          # quantisation step (0: none)
    dup_frac: float = 0.0      # fraction of rows overwritten by copies of other rows
    restrictions: dict = field(default_factory=dict)


# Restriction keys follow the C ABI's nnm_restrictions fields.
WORKLOADS = {
    "nnm_n4096_d8": Workload(
        "nnm_n4096_d8", 4096, 8, 16, 10.0, ("fixed", 0.5), seed=0),
    "nnm_n262144_d16": Workload(
        "nnm_n262144_d16", 262_144, 16, 64, 20.0, ("per_component", 0.2, 1.0), seed=1,
        restrictions={"max_join_dist": 1.5, "kl1_stop_clusters": 200}),
    "nnm_n2097152_d25": Workload(
        "nnm_n2097152_d25", 2_097_152, 25, 1000, 50.0, ("per_axis", 0.1, 1.5), seed=2,
        noise_frac=0.05,
        restrictions={"max_join_dist": 2.0, "kl4_min_size": 10, "kl3_max_size": 50_000}),
    "nnm_n1048576_d25_ties": Workload(
        "nnm_n1048576_d25_ties", 1_048_576, 25, 256, 10.0, ("fixed", 0.3), seed=4,
        grid=1.0 / 64.0, dup_frac=0.02),
}


def mixture(n: int, d: int, components: int, centre_hi: float, sigma: tuple, seed: int,
            noise_frac: float = 0.0, grid: float = 0.0, dup_frac: float = 0.0) -> np.ndarray:
    """Draw ``n`` rows of a ``d``-dimensional Gaussian mixture as float32 [n, d].

    ``noise_frac`` of the rows (rounded) are uniform over the per-feature bounding
    box of the mixture rows; ``grid`` > 0 rounds every value to a multiple of it;
    ``dup_frac`` of the rows are overwritten by copies of other randomly chosen
    rows (exact duplicates).
    """
    rng = np.random.default_rng(seed)
    n_noise = int(round(noise_frac * n))
    n_mix = n - n_noise
    centres = rng.uniform(0.0, centre_hi, size=(components, d))
    kind = sigma[0]
    if kind == "fixed":
        sig = np.full((components, d), float(sigma[1]))
    elif kind == "per_component":
        sig = np.repeat(rng.uniform(sigma[1], sigma[2], size=(components, 1)), d, axis=1)
    elif kind == "per_axis":
        sig = rng.uniform(sigma[1], sigma[2], size=(components, d))
    else:
        raise ValueError(f"unknown sigma recipe {sigma!r}")
    labels = rng.integers(0, components, size=n_mix)
    x = centres[labels] + sig[labels] * rng.standard_normal(size=(n_mix, d))
    if n_noise:
        lo = x.min(axis=0)
        hi = x.max(axis=0)
        noise = rng.uniform(lo, hi, size=(n_noise, d))
        x = np.concatenate([x, noise], axis=0)
    if grid > 0.0:
        x = np.round(x / grid) * grid
    if dup_frac > 0.0:
        n_dup = int(round(dup_frac * n))
        dst = rng.choice(n, size=n_dup, replace=False)
        src = rng.integers(0, n, size=n_dup)
        x[dst] = x[src]
    x = x[rng.permutation(n)]
    return np.ascontiguousarray(x.astype(np.float32))


def make(name: str, n: int | None = None, seed: int | None = None) -> np.ndarray:
    """Rows of the named workload; ``n``/``seed`` override its size/seed (smaller test cases)."""
    w = WORKLOADS[name]
    return mixture(n if n is not None else w.n, w.d, w.components, w.centre_hi, w.sigma,
                   w.seed if seed is None else seed, w.noise_frac, w.grid, w.dup_frac)


def batched_instances(count: int = 512, seed: int = 3, n_lo: int = 1024, n_hi: int = 65536,
                      d_lo: int = 4, d_hi: int = 25):
    """Many independent mixtures of uneven size: N log-uniform in [n_lo, n_hi],
    d uniform in {d_lo..d_hi}, 8..64 components, sigma 0.5, centres U[0,10]^d."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        d = int(rng.integers(d_lo, d_hi + 1))
        comps = int(rng.integers(8, 65))
        sub_seed = int(rng.integers(0, 2**63 - 1))
        out.append(mixture(n, d, comps, 10.0, ("fixed", 0.5), sub_seed))
    return out
