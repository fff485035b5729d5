"""Seeded synthetic knapsack workloads shared by the GPU library's tests, the oracle's
tests and the benchmark.

This module holds no QIEO arithmetic: it only draws problem instances (item weights,
values, capacity) and batch/serve size manifests. Both the CUDA path and the CPU oracle
receive the arrays it returns; neither side generates its own inputs.

The paper's workloads are synthetic 0/1 knapsack instances on an (Np, Ng) grid whose
generator is not printed (Sec. IV-A, Table II). The recipe used here:

* SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number generators",
  OOPSLA 2014) seeded with the instance seed;
* w_j = 1 + floor(hi32(next) * 10 / 2^32), i.e. uniform on [1, 10];
* v_j = w_j + 5;
* W = floor(sum(w) / 2).

Batch manifests draw Ng = floor(exp(ln 50 + U ln 400)) clamped to [50, 20000]
(log-uniform) and Np uniformly from {32, 64, 128, 256, 512}.
"""
from __future__ import annotations

import dataclasses
import json
import math

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

NP_CHOICES = (32, 64, 128, 256, 512)


def splitmix64(seed: int, n: int, start: int = 0) -> np.ndarray:
    """Outputs number start .. start+n-1 of the SplitMix64 stream seeded with `seed`
    (uint64 array). Output i mixes state seed + (i+1)*gamma."""
    with np.errstate(over="ignore"):
        i = np.arange(start + 1, start + n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


@dataclasses.dataclass
class Problem:
    """One 0/1 knapsack instance: int32 weights and values, int64 capacity W."""
    weights: np.ndarray
    values: np.ndarray
    capacity: int

    @property
    def ng(self) -> int:
        return int(self.weights.shape[0])


def knapsack(ng: int, seed: int) -> Problem:
    """The synthetic instance of `ng` items drawn from SplitMix64(seed)."""
    if ng < 1:
        raise ValueError("ng must be >= 1")
    r = splitmix64(seed, ng)
    w = (np.uint64(1) + (((r >> np.uint64(32)) * np.uint64(10)) >> np.uint64(32))).astype(np.int32)
    v = (w + 5).astype(np.int32)
    cap = int(w.astype(np.int64).sum()) // 2
    return Problem(np.ascontiguousarray(w), np.ascontiguousarray(v), cap)


def custom_problem(weights, values, capacity) -> Problem:
    return Problem(np.ascontiguousarray(weights, dtype=np.int32),
                   np.ascontiguousarray(values, dtype=np.int32), int(capacity))


@dataclasses.dataclass
class SizeSpec:
    """One entry of a batch/serve manifest."""
    index: int
    ng: int
    np_: int
    seed: int          # item seed = Philox seed = instance id


def batch_manifest(count: int, manifest_seed: int = 0x51EB_2609, first_seed: int = 1,
                   ng_lo: int = 50, ng_hi: int = 20000) -> list[SizeSpec]:
    """Sizes of `count` independent instances: Ng log-uniform in [ng_lo, ng_hi], Np uniform
    in NP_CHOICES; instance i gets seed first_seed + i."""
    r = splitmix64(manifest_seed, 2 * count)
    out = []
    ln_lo, ln_span = math.log(ng_lo), math.log(ng_hi / ng_lo)
    for i in range(count):
        u = float(int(r[2 * i]) >> 11) * (1.0 / (1 << 53))
        ng = int(math.floor(math.exp(ln_lo + u * ln_span)))
        ng = min(max(ng, ng_lo), ng_hi)
        pick = (int(r[2 * i + 1]) >> 32) * len(NP_CHOICES) >> 32
        out.append(SizeSpec(i, ng, NP_CHOICES[pick], first_seed + i))
    return out


def poisson_arrivals(count: int, rate_per_s: float, seed: int = 0xA771_0E5) -> np.ndarray:
    """Arrival times (s) of a Poisson stream: exponential gaps from SplitMix64."""
    r = splitmix64(seed, count)
    u = ((r >> np.uint64(11)).astype(np.float64) + 0.5) * (1.0 / (1 << 53))
    gaps = -np.log(u) / rate_per_s
    return np.cumsum(gaps)


def manifest_json(specs: list[SizeSpec]) -> str:
    return json.dumps([dataclasses.asdict(s) for s in specs])


# The named workloads: (Ng, Np, generations, item seed, Philox seed, instance id).
WORKLOADS = {
    "c1": dict(ng=100, np=64, gens=500, item_seed=1, seed=1, inst=0),
    "c2": dict(ng=10_000, np=1_024, gens=1_000, item_seed=1, seed=1, inst=0),
    "c3": dict(ng=100_000, np=4_096, gens=200, item_seed=1, seed=1, inst=0),
}
