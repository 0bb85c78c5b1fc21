"""Seeded synthetic cavity sweeps for the batched form (no arithmetic of the method: only
the draws of grid sizes and of the dimensionless numbers each cavity is built from).

The paper's workload is the differentially heated cubic cavity of Sec. 3 at a few
Rayleigh numbers and Pr = 0.71; a sweep varies the edge length, Ra and Pr over a range
around it and advances all cavities together.
"""
import numpy as np


def cavity_sweep(count=64, seed=1, sizes=(32, 48, 64, 96), Ra_range=(1e3, 1e6),
                 Pr_choices=(0.71, 1.0, 7.0)):
    """`count` cubic cavities: edge length uniform over `sizes`, Ra log-uniform over
    Ra_range, Pr uniform over Pr_choices (numpy PCG64 seeded with `seed`).  Returns a
    list of {"grid": (n, n, n), "Ra": Ra, "Pr": Pr}."""
    rng = np.random.default_rng(seed)
    n = rng.choice(np.asarray(sizes), size=count)
    lo, hi = np.log10(Ra_range[0]), np.log10(Ra_range[1])
    Ra = 10.0 ** rng.uniform(lo, hi, size=count)
    Pr = rng.choice(np.asarray(Pr_choices, dtype=np.float64), size=count)
    return [{"grid": (int(a), int(a), int(a)), "Ra": float(r), "Pr": float(p)}
            for a, r, p in zip(n, Ra, Pr)]
