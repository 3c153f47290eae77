"""Seeded synthetic inputs shared by the CUDA path's tests, the benchmark and the oracle.

This module holds none of the method's arithmetic: only random-number streams,
the named workload configurations and the serving arrival trace.

* ``splitmix64`` is the counter form of Steele, Lea & Flood's SplitMix64
  (OOPSLA 2014; Vigna's public-domain ``splitmix64.c``): output k of the stream
  seeded with ``seed`` is mix(seed + (k+1) * 0x9E3779B97F4A7C15).  The CUDA
  library (``sca_adam_init`` with no start field) and the oracle each implement
  the same published definition; the tests check that all three agree bit for
  bit.
* ``seed_phi`` maps output i to phi0_i = top53(x_i) * 2^-53 - 1/2, the uniform
  [-0.5, 0.5) start of the paper's Adam runs (Sec. II: phi is found by ADAM).
* ``WORKLOADS`` are the lattice/temperature/frequency settings the paper uses
  (L x L square lattice, half filling, t = 1; Figs. 1, 4, 5: L = 20, T = 0.1,
  U = 3..6) scaled to the sizes measured here.
* ``serving_trace`` draws the mixed-size request stream (Poisson arrivals,
  L from {8, 12, 16, 20, 24, 32}, U in [2, 8], Delta in [0, 2], T in
  [0.05, 0.6], n_omega = ceil(20 / (2 pi T))).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_GAMMA = 0x9E3779B97F4A7C15
_M64 = (1 << 64) - 1


def splitmix64(seed: int, k: int) -> int:
    """Output k (k = 0, 1, ...) of the SplitMix64 stream started at ``seed``."""
    z = (seed + (k + 1) * _GAMMA) & _M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return z ^ (z >> 31)


def splitmix64_array(seed: int, n: int) -> np.ndarray:
    """First n outputs as uint64 (vectorised; identical to ``splitmix64``)."""
    with np.errstate(over="ignore"):
        k = np.arange(1, n + 1, dtype=np.uint64)
        z = np.uint64(seed & _M64) + k * np.uint64(_GAMMA)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def seed_phi(seed: int, N: int) -> np.ndarray:
    """phi0 in [-0.5, 0.5): top 53 bits of each output times 2^-53, minus 1/2."""
    x = splitmix64_array(seed, N)
    return (x >> np.uint64(11)).astype(np.float64) * 2.0**-53 - 0.5


def random_phi(seed: int, N: int, scale: float = 1.0) -> np.ndarray:
    """A generic random field for parity tests (numpy PCG64, uniform in [-scale, scale))."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-scale, scale, size=N)


def neel_phi(L: int, amplitude: float) -> np.ndarray:
    """Staggered field phi_i = amplitude * (-1)^(x+y) on site i = x*L + y."""
    x, y = np.meshgrid(np.arange(L), np.arange(L), indexing="ij")
    return amplitude * np.where((x + y) % 2 == 0, 1.0, -1.0).reshape(-1)


@dataclass(frozen=True)
class Workload:
    name: str
    L: int
    U: float
    delta: float
    T: float
    n_omega: int
    t: float = 1.0
    mu: float = 0.0
    lr: float = 0.01
    steps: int = 0
    seed: int = 0
    note: str = ""


# Named workloads (square L x L lattice, t = 1, half filling mu = 0).
WORKLOADS = {
    # 4x4, U=6, Delta=0, T=0.1, 64 positive Matsubara frequencies x 2 spins = 128 blocks of 16x16
    "hubbard_4x4": Workload("hubbard_4x4", 4, 6.0, 0.0, 0.1, 64, steps=2000,
                            note="128 complex 16x16 blocks"),
    # 20x20 ionic, U=6, Delta=0.5, T=0.1, 256 frequencies -> 512 blocks of 400x400
    "ionic_20x20": Workload("ionic_20x20", 20, 6.0, 0.5, 0.1, 256, steps=3000,
                            note="512 complex 400x400 blocks"),
    # 40x40 ionic, U=4, Delta=1, T=0.1, 128 frequencies -> 256 blocks of 1600x1600
    "ionic_40x40": Workload("ionic_40x40", 40, 4.0, 1.0, 0.1, 128,
                            note="256 complex 1600x1600 blocks"),
    # 64x64 ionic, U=6, Delta=0.5, T=0.2, 64 frequencies -> 128 blocks of 4096x4096
    "ionic_64x64": Workload("ionic_64x64", 64, 6.0, 0.5, 0.2, 64,
                            note="128 complex 4096x4096 blocks"),
    # 16x16 rerun of the 64x64 parameters (oracle-sized)
    "ionic_16x16_rerun": Workload("ionic_16x16_rerun", 16, 6.0, 0.5, 0.2, 64),
    # profiling case of the dominant kernels: the 40x40 lattice at T = 1.5 with 8 frequencies
    # -> 16 blocks of 1600x1600 (328 MB, above the L2), all diagonally dominant (w_0 > 4t)
    "ionic_40x40_w8": Workload("ionic_40x40_w8", 40, 4.0, 1.0, 1.5, 8,
                               note="16 complex 1600x1600 blocks, none pivoted"),
    # profiling case of the refinement: the 40x40 workload cut to its 32 lowest frequencies
    # -> 64 blocks (12 pivoted, 52 dominant; 1.3 GB of blocks), the same per-block kernels
    "ionic_40x40_w32": Workload("ionic_40x40_w32", 40, 4.0, 1.0, 0.1, 32,
                                note="64 complex 1600x1600 blocks, 12 pivoted"),
}


@dataclass
class Request:
    index: int
    arrival_s: float
    L: int
    U: float
    delta: float
    T: float
    n_omega: int
    seed: int
    extra: dict = field(default_factory=dict)


def serving_trace(n_requests: int = 512, rate_per_s: float = 20.0, seed: int = 2311,
                  sizes=(8, 12, 16, 20, 24, 32)) -> list[Request]:
    """Poisson arrival trace of SCA solve requests (numpy PCG64 with ``seed``).

    Inter-arrival times are exponential with mean 1/rate; each request draws L
    uniformly from ``sizes``, U ~ U[2, 8], Delta ~ U[0, 2], T ~ U[0.05, 0.6] and
    n_omega = ceil(20 / (2 pi T)); its phi0 seed is its index."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_per_s, size=n_requests)
    t = np.cumsum(gaps) - gaps[0]
    out = []
    for i in range(n_requests):
        L = int(rng.choice(sizes))
        U = float(rng.uniform(2.0, 8.0))
        delta = float(rng.uniform(0.0, 2.0))
        T = float(rng.uniform(0.05, 0.6))
        n_omega = int(math.ceil(20.0 / (2.0 * math.pi * T)))
        out.append(Request(i, float(t[i]), L, U, delta, T, n_omega, seed=i))
    return out
