"""Seeded synthetic inputs for the rIGA quadratic eigenproblem workloads.

This module only draws numbers; it holds none of the method's arithmetic.
Both the CUDA path and the FP64 CPU checker receive their inputs from here:
the per-element damping coefficients sigma_e (element ex + ne*ey) and the
Arnoldi start vector.

The paper's own case studies (a three-layer Earth model and an absorbing
cavity) depend on parameters printed only in figures that are not available;
these synthetic meshes keep the shape of its efficiency study instead
(uniform square meshes, B-spline degrees 2..5, 16 x 16-element macroelements,
Section 5.3) with random per-element damping.
"""
import numpy as np

MASK64 = (1 << 64) - 1

# name -> mesh, shift and solver parameters of each workload
CONFIGS = {
    # 16 x 16 elements, p = 2, C^0 lines every 4 elements, sigma_e ~ U[0.1, 1]
    "tiny": dict(ne=16, p=2, block=4, shift=20.0, neig=10, m=40,
                 sigma_law="uniform", lo=0.1, hi=1.0, seed=20211228),
    # 256 x 256 elements, p = 3, C^0 lines every 16 elements
    "p3_256_b16": dict(ne=256, p=3, block=16, shift=500.0, neig=20, m=60,
                       sigma_law="uniform", lo=0.1, hi=1.0, seed=20211229),
    # the same mesh with maximum continuity (IGA) for comparison
    "p3_256_iga": dict(ne=256, p=3, block=0, shift=500.0, neig=20, m=60,
                       sigma_law="uniform", lo=0.1, hi=1.0, seed=20211229),
    # 512 x 512 elements, p = 4, blocks of 32, lognormal damping
    "p4_512_b32": dict(ne=512, p=4, block=32, shift=2000.0, neig=20, m=60,
                       sigma_law="lognormal", median=0.5, logstd=1.0,
                       seed=20211230),
    # 512 x 512 elements, p = 3, blocks of 16 (sensitivity workload)
    "p3_512_b16": dict(ne=512, p=3, block=16, shift=800.0, neig=20, m=60,
                       sigma_law="uniform", lo=0.1, hi=1.0, seed=20211232),
    # 64 x 64 version of the sensitivity workload (checker-sized)
    "p3_64_b16": dict(ne=64, p=3, block=16, shift=800.0, neig=20, m=60,
                      sigma_law="uniform", lo=0.1, hi=1.0, seed=20211232),
    # 64 x 64 version of the mixed-precision workload (checker-sized)
    "p4_64_b32": dict(ne=64, p=4, block=32, shift=2000.0, neig=20, m=60,
                      sigma_law="lognormal", median=0.5, logstd=1.0, seed=20211230),
}


def sigma_e(cfg):
    """Per-element damping coefficients, element ex + ne*ey, float64."""
    ne = cfg["ne"]
    rng = np.random.default_rng(cfg["seed"])
    if cfg["sigma_law"] == "uniform":
        return rng.uniform(cfg["lo"], cfg["hi"], ne * ne)
    if cfg["sigma_law"] == "lognormal":
        return cfg["median"] * np.exp(cfg["logstd"] * rng.standard_normal(ne * ne))
    if cfg["sigma_law"] == "constant":
        return np.full(ne * ne, float(cfg["value"]))
    raise ValueError(cfg["sigma_law"])


def splitmix64(x):
    """SplitMix64 output function (Steele, Lea and Flood, OOPSLA 2014) for
    the 64-bit counter x; python ints, exact."""
    z = (x + 0x9E3779B97F4A7C15) & MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def start_vector(seed, n):
    """v[i] = u_i - 0.5 with u_i = (splitmix64(seed + i) >> 11) * 2^-53."""
    seed = int(seed) & MASK64
    z = (np.arange(n, dtype=np.uint64) + np.uint64(seed)) + np.uint64(0x9E3779B97F4A7C15)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    z = z ^ (z >> np.uint64(31))
    return (z >> np.uint64(11)).astype(np.float64) * 2.0 ** -53 - 0.5


def batch_problems(seed=20211231, count=64):
    """Independent problems of uneven size: ne in {32, 64, 128, 256},
    p in {2, 3, 4, 5}, block in {8, 16}, sigma_e ~ U[0.05, 2], four shifts
    drawn in [10, 5000], eight eigenpairs per shift."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        ne = int(rng.choice([32, 64, 128, 256]))
        p = int(rng.choice([2, 3, 4, 5]))
        block = int(rng.choice([8, 16]))
        shifts = rng.uniform(10.0, 5000.0, 4)
        sub = int(rng.integers(0, 2 ** 62))
        out.append(dict(ne=ne, p=p, block=block, shifts=shifts.tolist(), neig=8,
                        m=24, sigma_law="uniform", lo=0.05, hi=2.0, seed=sub))
    return out
