"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle
checks.  This module holds no operator arithmetic: it draws random numbers and
evaluates closed-form fields at node coordinates that the caller supplies.

Workload recipe (Sec. 4 of the paper: Taylor-Green vortex on the periodic cube
[-pi, pi]^3): random vectors are uniform on [-1, 1] from
``numpy.random.default_rng(seed)`` in FP64, in the library's vector order
[comp][elem][z][y][x]; the Taylor-Green field u = (sin x cos y cos z,
-cos x sin y cos z, 0) is interpolated at the nodal points and perturbed by
``noise`` times uniform[-1, 1] noise.
"""
import numpy as np


def uniform(seed, size):
    """FP64 uniform[-1, 1] vector of `size` entries from `seed`."""
    return np.random.default_rng(seed).uniform(-1.0, 1.0, size)


def node_coordinates(n, lo, hi, nodes_1d):
    """Physical coordinates (3, E, N^3) of the nodal points of a DG space on a
    periodic Cartesian mesh with n = (nx, ny, nz) elements on [lo, hi] whose
    1D reference nodes on [0, 1] are `nodes_1d`."""
    n = [int(v) for v in n]
    nodes_1d = np.asarray(nodes_1d, dtype=np.float64)
    N = len(nodes_1d)
    E = n[0] * n[1] * n[2]
    e = np.arange(E)
    ijk = [e % n[0], (e // n[0]) % n[1], e // (n[0] * n[1])]
    I = np.arange(N ** 3)
    loc = [I % N, (I // N) % N, I // (N * N)]
    X = np.empty((3, E, N ** 3))
    for a in range(3):
        h = (hi[a] - lo[a]) / n[a]
        X[a] = lo[a] + (ijk[a][:, None] + nodes_1d[loc[a]][None, :]) * h
    return X


def taylor_green(n, lo, hi, nodes_1d, noise=0.0, seed=0):
    """Taylor-Green velocity at the nodal points, (3, E, N^3), plus `noise`
    times seeded uniform[-1, 1] noise."""
    X = node_coordinates(n, lo, hi, nodes_1d)
    u = np.stack([np.sin(X[0]) * np.cos(X[1]) * np.cos(X[2]),
                  -np.cos(X[0]) * np.sin(X[1]) * np.cos(X[2]),
                  np.zeros_like(X[0])])
    if noise:
        u = u + noise * uniform(seed, u.size).reshape(u.shape)
    return u
