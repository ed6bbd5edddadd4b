"""Seeded synthetic inputs for the Ginzburg-Landau Jacobian-solve workloads.

This module only draws random numbers and picks sizes. It holds none of the
method's arithmetic (no operator, no phase, no solver), so both the CPU
oracle's tests and the CUDA path's tests and benchmark may take their inputs
from here.

Every generator uses numpy's PCG64 with an explicit seed, so a given
(size, seed) pair always yields the same array on every machine.

Workloads (the paper's domains are the square and the cube, Section 4; the
sizes below are structured node lattices of those domains):

* ``square64``   2D, 64 x 64 nodes, mu = 1, field along z, psi uniform in the
                 unit disk (seed 1), b complex normal (seed 1).
* ``square1024`` 2D, 1024 x 1024 nodes, mu = 2, psi = (Newton steps from
                 psi = 1, at most five, until ||GL||_R <= 1e-7) + 0.1 * (uniform
                 in the unit disk) (seed 2); the solve is that state's Newton
                 system.
* ``cube128``    3D, 128^3 nodes, mu = 1, field along (1,1,1)/sqrt(3),
                 psi == 1 (the state the paper's Section 4 experiments use) or
                 psi uniform in the unit disk (seed 4); b complex normal (seed 5).
* ``batch64``    64 squares with N_s = round(exp(U(ln 32, ln 512))) (seed 6),
                 mu_s = 2 s / 63, psi_s = 1 + 0.1 * disk noise (seed 7 + s).
* ``cube256``    3D, 256^3 nodes, continuation over mu in [0, 1.5].
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "rng",
    "disk",
    "complex_normal",
    "psi_noisy_one",
    "batch_sizes",
    "warmstart_init",
    "WORKLOADS",
]


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def disk(n: int, seed: int) -> np.ndarray:
    """n complex numbers uniform in the closed unit disk: r = sqrt(U), arg = 2 pi U.

    Radii are drawn first (all n), then arguments (all n).
    """
    g = rng(seed)
    r = np.sqrt(g.random(n))
    a = 2.0 * math.pi * g.random(n)
    return (r * np.cos(a) + 1j * (r * np.sin(a))).astype(np.complex128)


def complex_normal(n: int, seed: int) -> np.ndarray:
    """n draws of CN(0, 1): real and imaginary parts N(0, 1/2), real parts first."""
    g = rng(seed)
    re = g.standard_normal(n)
    im = g.standard_normal(n)
    return ((re + 1j * im) / math.sqrt(2.0)).astype(np.complex128)


def psi_noisy_one(n: int, seed: int, amplitude: float = 0.1) -> np.ndarray:
    """1 + amplitude * (uniform in the unit disk)."""
    return (1.0 + amplitude * disk(n, seed)).astype(np.complex128)


def batch_sizes(count: int = 64, seed: int = 6, lo: int = 32, hi: int = 512) -> list[int]:
    """Log-uniform node counts per side: N_s = round(exp(U(ln lo, ln hi)))."""
    g = rng(seed)
    u = g.random(count)
    return [int(round(math.exp(math.log(lo) + (math.log(hi) - math.log(lo)) * x))) for x in u]


INV_SQRT3 = 1.0 / math.sqrt(3.0)

# name -> (dim, nodes per side, mu, unit field direction)
WORKLOADS = {
    "square64": (2, 64, 1.0, (0.0, 0.0, 1.0)),
    "square1024": (2, 1024, 2.0, (0.0, 0.0, 1.0)),
    "cube128": (3, 128, 1.0, (INV_SQRT3, INV_SQRT3, INV_SQRT3)),
    "cube256": (3, 256, 1.5, (0.0, 0.0, 1.0)),
}


def warmstart_init(seed: int = 11, layers: int = 4, channels: int = 64) -> np.ndarray:
    """Random initial parameters of the warm-start network, one flat float32
    vector: layers matrices of channels x (2 channels) drawn N(0, 2 / fan_in)
    (He initialisation, fan_in = 2 channels), then a 2 x channels head drawn
    N(0, 1 / channels) scaled by 0.1."""
    g = rng(seed)
    cin = 2 * channels
    ws = [g.standard_normal(channels * cin) * math.sqrt(2.0 / cin) for _ in range(layers)]
    head = g.standard_normal(2 * channels) * (0.1 / math.sqrt(channels))
    return np.concatenate(ws + [head]).astype(np.float32)
