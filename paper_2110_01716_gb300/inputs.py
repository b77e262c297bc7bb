"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module holds no arithmetic of the method: it only draws meshes and fields.
Both the CUDA library and the CPU oracle consume its outputs, and neither
imports the other.

* ``box_vertices``: the vertex lattice of an ex*ey*ez box of hexahedra on the
  unit cube, interior vertices moved by independent uniform offsets of at most
  ``jitter`` times the local spacing per coordinate.  The offsets come from the
  counter-based splitmix64 generator (Steele, Lea and Flood, OOPSLA 2014, with
  the published mixing constants), so the CUDA library's own built-in mesh
  generator reproduces the same vertices bit for bit.
* ``random_field``: i.i.d. U(-1, 1) values from numpy's PCG64.
* ``fourier_modes``: the smooth random right-hand side of the Neumann problem
  f(x) = sum_m a_m cos(2 pi k_m . x + phi_m).
* ``batch_instances`` / ``arrival_stream``: sizes, orders and arrival times of
  the batched and served solves.
"""

from __future__ import annotations

import math

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, idx: np.ndarray) -> np.ndarray:
    """Value ``idx`` of the splitmix64 stream ``seed``: mix(seed + (idx+1)*gamma)."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (np.asarray(idx, dtype=np.uint64) + np.uint64(1)) * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def splitmix64_unit(seed: int, idx: np.ndarray) -> np.ndarray:
    """U[0,1) doubles: the top 53 bits of splitmix64 times 2^-53."""
    return (splitmix64(seed, idx) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def box_vertices(ex: int, ey: int, ez: int, jitter: float = 0.1, seed: int = 1) -> np.ndarray:
    """Vertex lattice [(ex+1)(ey+1)(ez+1), 3] of a jittered unit-cube box.

    Vertex (a, b, c) sits at index a + (ex+1)(b + (ey+1)c) and at
    (a/ex, b/ey, c/ez) + (2u-1) * jitter * (1/ex, 1/ey, 1/ez), where
    u = splitmix64_unit(seed, 3*index + coordinate), for vertices strictly
    inside the cube only; boundary vertices stay on the lattice, so the domain
    stays the unit cube.
    """
    a = np.arange(ex + 1, dtype=np.float64)
    b = np.arange(ey + 1, dtype=np.float64)
    c = np.arange(ez + 1, dtype=np.float64)
    C, B, A = np.meshgrid(c, b, a, indexing="ij")
    lattice = np.stack([A.ravel(), B.ravel(), C.ravel()], axis=1)
    counts = np.array([ex, ey, ez], dtype=np.float64)
    nv = lattice.shape[0]
    u = splitmix64_unit(seed, np.arange(3 * nv, dtype=np.uint64)).reshape(nv, 3)
    interior = np.all((lattice > 0) & (lattice < counts), axis=1, keepdims=True)
    off = np.where(interior, (2.0 * u - 1.0) * jitter / counts, 0.0)
    return lattice / counts + off


def random_field(n: int, seed: int) -> np.ndarray:
    """n i.i.d. U(-1, 1) doubles from numpy's PCG64 stream ``seed``."""
    return np.random.Generator(np.random.PCG64(seed)).uniform(-1.0, 1.0, size=n)


def fourier_modes(seed: int, m: int = 8):
    """Coefficients of f(x) = sum_m a_m cos(2 pi k_m . x + phi_m).

    k_m uniform on {0..3}^3 without 0, a_m ~ N(0,1)/|k_m|^2, phi_m ~ U(0, 2 pi).
    Returns (a [m], k [m,3] float, phi [m]).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    ks = []
    while len(ks) < m:
        k = rng.integers(0, 4, size=3)
        if k.any():
            ks.append(k)
    k = np.array(ks, dtype=np.float64)
    a = rng.standard_normal(m) / np.sum(k * k, axis=1)
    phi = rng.uniform(0.0, 2.0 * math.pi, size=m)
    return a, k, phi


def fourier_sequence(seed: int, m: int = 8):
    """A smoothly time-varying right-hand side for successive solves:
    f_n(x) = sum_m a_m cos(2 pi k_m . x + phi_m + omega_m n), with (a, k, phi)
    of fourier_modes(seed, m) and angular steps omega_m ~ U(0.02, 0.1) rad
    per solve (one extra draw after the modes).  Returns (a, k, phi, omega)."""
    a, k, phi = fourier_modes(seed, m)
    rng = np.random.Generator(np.random.PCG64(seed + 0x5EED))
    omega = rng.uniform(0.02, 0.1, size=m)
    return a, k, phi, omega


def near_cube_factors(E: int):
    """ex*ey*ez closest to E with factors differing by at most one."""
    best = None
    for ex in range(1, int(round(E ** (1 / 3))) + 3):
        for ey in (ex, ex + 1):
            for ez in (ey, ey + 1):
                if ez - ex > 1:
                    continue
                err = abs(ex * ey * ez - E)
                if best is None or err < best[0]:
                    best = (err, (ex, ey, ez))
    return best[1]


def batch_instances(seed: int, count: int = 64, e_lo: int = 64, e_hi: int = 8192,
                    orders=(5, 7, 9)):
    """``count`` independent problems: E log-uniform in [e_lo, e_hi] mapped to a
    near-cubic box, N uniform over ``orders``, each with its own mesh seed."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(count):
        E = int(round(math.exp(rng.uniform(math.log(e_lo), math.log(e_hi)))))
        ex, ey, ez = near_cube_factors(E)
        N = int(orders[rng.integers(0, len(orders))])
        out.append({"ex": ex, "ey": ey, "ez": ez, "N": N, "seed": int(seed * 1000 + i)})
    return out


def arrival_stream(seed: int, count: int, rate: float, e_lo: int = 512, e_hi: int = 65536,
                   tols=(1e-6, 1e-8, 1e-10)):
    """Poisson arrivals (exponential gaps at ``rate`` per second) of solves with
    E log-uniform in [e_lo, e_hi], N = 7, tolerance uniform over ``tols``."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    out = []
    for i in range(count):
        t += rng.exponential(1.0 / rate)
        E = int(round(math.exp(rng.uniform(math.log(e_lo), math.log(e_hi)))))
        ex, ey, ez = near_cube_factors(E)
        tol = float(tols[rng.integers(0, len(tols))])
        out.append({"t": t, "ex": ex, "ey": ey, "ez": ez, "N": 7, "tol": tol,
                    "seed": int(seed * 100000 + i)})
    return out
