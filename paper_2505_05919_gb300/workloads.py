"""Seeded synthetic workloads (inputs only -- none of the method's arithmetic).

The paper's workloads are synthetic lattices (Sec. III.C); these recipes give
the state points, sizes, seeds and random configurations that the tests and
the benchmark feed to both the GPU path and the CPU oracle.  State points are
physical (T in K, P in MPa); each side converts them with its own Table 1
units.
"""
from __future__ import annotations

import numpy as np

AMBIENT = (300.0, 0.1)                # K, MPa (the paper's ambient point)
TEMPERATURES_C3 = (270.0, 300.0, 330.0)  # 60 degrees around ambient


def random_words(L: int, q: int, seed: int) -> np.ndarray:
    """A uniformly random configuration (numpy PCG64), for set_state inputs."""
    rng = np.random.default_rng(seed)
    arms = rng.integers(0, q, size=(L * L, 4), dtype=np.uint16)
    w = np.zeros(L * L, np.uint16)
    for a in range(4):
        w |= (arms[:, a] << (4 * a)).astype(np.uint16)
    return w.reshape(L, L)


def c1():
    """L = 64, q = 6, random init seed 1, ambient, 1000 steps."""
    return dict(L=64, q=6, seed=1, T=AMBIENT[0], P=AMBIENT[1], sweeps=1000)


def c2():
    """L = 1024, q = 6, random init seed 2, ambient, 10^4 steps, record every 10."""
    return dict(L=1024, q=6, seed=2, T=AMBIENT[0], P=AMBIENT[1], sweeps=10000, record_every=10)


def c3():
    """L = 4096, q = 6; random (seed 3) and ordered init; 270/300/330 K at
    0.1 MPa; 1000 steps each."""
    return [dict(L=4096, q=6, seed=3, T=T, P=0.1, sweeps=1000, init=init)
            for init in (0, 1) for T in TEMPERATURES_C3]


def c4(n_replicas: int = 256, seed: int = 4, sweeps: int = 5000):
    """256 replicas: L drawn from {32, 64, 128, 256, 512}; (T, P) on a 16 x 16
    grid T_i = 270 + 4 i K, P_j = 0.1 + j 49.9/15 MPa; seeds 1000 + r."""
    rng = np.random.default_rng(seed)
    sizes = rng.choice(np.array([32, 64, 128, 256, 512]), size=n_replicas)
    out = []
    for r in range(n_replicas):
        i, j = (r // 16) % 16, r % 16
        out.append(dict(L=int(sizes[r]), q=6, seed=1000 + r, T=270.0 + 4.0 * i,
                        P=0.1 + j * (49.9 / 15.0), sweeps=sweeps))
    return out


def c5(n_jobs: int = 2000, rate_hz: float = 200.0, seed: int = 5,
       sizes=(64, 128, 256, 512, 1024, 2048), sweeps_range=(1e3, 1e5)):
    """Poisson arrivals (exponential gaps at rate_hz); L uniform over sizes;
    sweeps log-uniform in sweeps_range; (T, P) uniform in 270-330 K x
    0.1-50 MPa; job r has seed 5000 + r."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_hz, size=n_jobs)
    t = np.cumsum(gaps) - gaps[0]
    L = rng.choice(np.array(sizes), size=n_jobs)
    lo, hi = np.log(sweeps_range[0]), np.log(sweeps_range[1])
    sw = np.exp(rng.uniform(lo, hi, size=n_jobs)).astype(np.int64)
    T = rng.uniform(270.0, 330.0, size=n_jobs)
    P = rng.uniform(0.1, 50.0, size=n_jobs)
    return [dict(arrival=float(t[r]), L=int(L[r]), q=6, seed=5000 + r, T=float(T[r]),
                 P=float(P[r]), sweeps=int(sw[r])) for r in range(n_jobs)]
