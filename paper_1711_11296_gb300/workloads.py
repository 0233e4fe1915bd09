"""Seeded synthetic inputs and the workload table.

This module holds no transform arithmetic: it only draws random spectral
coefficients with the amplitude envelope of each workload and names the
grid sizes.  Both the GPU tests and the oracle-side tests take their inputs
from here, so neither side generates data for the other.

Spectra are complex ``[ncoef][F]`` arrays, packed m-major (coefficient (m, n)
at row m (N+1) - m (m-1)/2 + (n - m)), with the imaginary part of every
m = 0 coefficient zero (a real field).

Envelopes (the paper's shallow-water and dynamical-core runs start from
smooth fields whose spectra decay with n; the exact initial conditions are
not reproducible here, so these stand in for them):

* ``"n^-1.5"``: Re and Im independent N(0,1) (n+1)^-1.5.
* ``"energy^-2"``: the degree-n energy E(n) = |a_n^0|^2 + 2 sum_{m>=1} |a_n^m|^2
  has expectation proportional to (n+1)^-2, i.e. Re and Im are
  N(0,1) (n+1)^-1 / sqrt(2 (2n+1)).
* ``"uniform^-1/3"``: Re and Im uniform in [1, 2] times (n+1)^-1/3 (the
  amplitude law of the aliasing experiment, Sec. 4.2).
* ``"flat"``: Re and Im independent N(0,1) at every degree (white noise:
  every zonal wavenumber and parity carries a comparable share, so that a
  per-(m, parity) error check weighs the high wavenumbers as much as the
  low ones).
"""
from dataclasses import dataclass

import numpy as np

SEED_BASE = 171111296


@dataclass(frozen=True)
class Workload:
    name: str
    N: int
    J: int
    I: int
    F: int
    envelope: str
    index: int
    note: str = ""


# The workloads (sizes per the truncations named in the paper's experiments).
WORKLOADS = {
    "T31": Workload("T31", 31, 65, 128, 1, "n^-1.5", 0,
                    "plain FP64 round trip, 1 scalar field"),
    "T159": Workload("T159", 159, 321, 640, 256, "energy^-2", 1,
                     "4 fields x 64 levels"),
    "T319": Workload("T319", 319, 641, 1280, 300, "energy^-2", 2,
                     "3 fields x 100 levels"),
    "T639": Workload("T639", 639, 1281, 2560, 256, "energy^-2", 4,
                     "4 fields x 64 levels"),
}

# The aliasing experiment of Sec. 4.2 at the paper's cubic Clenshaw-Curtis
# resolution Tc479 (N = 479, J = 959; I = 4 (N + 1)), with the amplitude law
# of its step 1; F field-levels per field U, V, W.
ALIAS = Workload("Tc479", 479, 959, 1920, 64, "uniform^-1/3", 5,
                 "quadratic and cubic terms of Sec. 4.2")

# Uneven ensemble: 16 members x 32 levels x 2 fields at each truncation.
ENSEMBLE = [
    Workload("ens-T63", 63, 129, 256, 1024, "energy^-2", 3),
    Workload("ens-T127", 127, 257, 512, 1024, "energy^-2", 3),
    Workload("ens-T255", 255, 513, 1024, 1024, "energy^-2", 3),
    Workload("ens-T511", 511, 1025, 2048, 1024, "energy^-2", 3),
]

# Nested restriction ladder on grids with J = 2N+1 (the nesting of Sec. 3.2
# needs J_f + 1 = 2 (J_c + 1)).
LADDER = [
    Workload("lad-T511", 511, 1023, 2048, 64, "energy^-2", 3),
    Workload("lad-T255", 255, 511, 1024, 64, "energy^-2", 3),
    Workload("lad-T127", 127, 255, 512, 64, "energy^-2", 3),
]


def ncoef(N):
    return (N + 1) * (N + 2) // 2


def degree_of_rows(N):
    """Total wavenumber n of every packed row (m-major)."""
    return np.concatenate([np.arange(m, N + 1) for m in range(N + 1)])


def order_of_rows(N):
    """Zonal wavenumber m of every packed row (m-major)."""
    return np.concatenate([np.full(N - m + 1, m) for m in range(N + 1)])


def random_spectrum(N, F, envelope="n^-1.5", seed=SEED_BASE, field0=0):
    """Seeded complex spectrum [ncoef][F]; column f uses seed + field0 + f."""
    n = degree_of_rows(N).astype(np.float64)
    m = order_of_rows(N)
    if envelope == "n^-1.5":
        amp = (n + 1.0) ** -1.5
    elif envelope == "energy^-2":
        amp = (n + 1.0) ** -1.0 / np.sqrt(2.0 * (2.0 * n + 1.0))
    elif envelope == "uniform^-1/3":
        amp = (n + 1.0) ** (-1.0 / 3.0)
    elif envelope == "flat":
        amp = np.ones_like(n)
    else:
        raise ValueError(envelope)
    out = np.empty((len(n), F), dtype=np.complex128)
    for f in range(F):
        g = np.random.Generator(np.random.PCG64(seed + field0 + f))
        if envelope == "uniform^-1/3":
            re = g.uniform(1.0, 2.0, len(n))
            im = g.uniform(1.0, 2.0, len(n))
        else:
            re = g.standard_normal(len(n))
            im = g.standard_normal(len(n))
        col = (re + 1j * im) * amp
        col[m == 0] = col[m == 0].real
        out[:, f] = col
    return out


def workload_spectrum(w: Workload, F=None, field0=0):
    """The seeded spectrum of a workload (optionally only F columns)."""
    F = w.F if F is None else F
    return random_spectrum(w.N, F, w.envelope,
                           SEED_BASE + 1000 * w.index, field0)


def random_grid(F, J, I, seed=SEED_BASE + 7):
    """Seeded non-band-limited real grid [F][J][I] (for linearity/adjoint
    tests, where any input is valid)."""
    g = np.random.Generator(np.random.PCG64(seed))
    return g.standard_normal((F, J, I))


def random_grid_field(f, J, I, seed=SEED_BASE + 17):
    """Field f of a seeded grid, reproducible one field at a time: [J][I]
    standard normal values from seed + f."""
    g = np.random.Generator(np.random.PCG64(seed + f))
    return g.standard_normal((J, I))
