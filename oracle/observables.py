"""Structural observables of the polyethylene melt, plain FP64 numpy.

Test infrastructure, like the rest of `oracle/`: only the tests, smoke() and
bench.py's CPU-baseline leg use it.  Each function is the textbook
definition of the quantity the paper uses to compare its GPU runs with
GROMACS (Sec. 5): the end-to-end vectors of the chains and their
autocorrelation function (Fig. 8), the radius of gyration, the trans/gauche
state of the backbone dihedrals (Eq. 6 fixes the torsion; trans = 180 deg in
the IUPAC convention), and the radial distribution function of non-bonded
sites.  Positions are (N, 3) in nm with chain c holding sites
c * sites .. c * sites + sites - 1.
"""
from __future__ import annotations

import numpy as np


def _chains(x, sites: int) -> np.ndarray:
    x = np.asarray(x, np.float64)
    return x.reshape(-1, sites, 3)


def end_to_end(x_unwrapped, sites: int) -> np.ndarray:
    """R_c = x_last - x_first of every chain (Sec. 5, Fig. 8), [n_chains, 3];
    the positions must be unwrapped (chains continuous)."""
    p = _chains(x_unwrapped, sites)
    return p[:, -1, :] - p[:, 0, :]


def radius_of_gyration_sq(x_unwrapped, sites: int, masses) -> np.ndarray:
    """Mass-weighted R_g^2 = sum_i m_i |x_i - x_cm|^2 / sum_i m_i of every
    chain, [n_chains]; masses [N] per site."""
    p = _chains(x_unwrapped, sites)
    m = np.asarray(masses, np.float64).reshape(-1, sites)
    cm = (m[:, :, None] * p).sum(axis=1) / m.sum(axis=1)[:, None]
    d = p - cm[:, None, :]
    return (m * (d * d).sum(axis=2)).sum(axis=1) / m.sum(axis=1)


def dihedral_angles(x_unwrapped, sites: int) -> np.ndarray:
    """IUPAC dihedral phi in (-180, 180] degrees of every backbone quadruple
    (i, i+1, i+2, i+3) of every chain, [n_chains, sites - 3]; trans = 180."""
    p = _chains(x_unwrapped, sites)
    b1 = p[:, 1:-2] - p[:, :-3]
    b2 = p[:, 2:-1] - p[:, 1:-2]
    b3 = p[:, 3:] - p[:, 2:-1]
    n1 = np.cross(b1, b2)
    n2 = np.cross(b2, b3)
    y = np.linalg.norm(b2, axis=2) * (b1 * n2).sum(axis=2)
    return np.degrees(np.arctan2(y, (n1 * n2).sum(axis=2)))


def trans_fraction(x_unwrapped, sites: int, boundary_deg: float = 120.0) -> float:
    """Fraction of backbone dihedrals in the trans state, |phi| > boundary
    (the three minima of Eq. 6 with n = 3 sit at 180 and +-60 degrees; the
    states split at +-120)."""
    phi = dihedral_angles(x_unwrapped, sites)
    return float(np.mean(np.abs(phi) > boundary_deg))


def end_to_end_acf(R_series, max_lag: int) -> np.ndarray:
    """C(tau) = <R(t + tau) . R(t)> / <R(t) . R(t)> over all time origins t
    and chains (Fig. 8), for tau = 0 .. max_lag samples; R_series
    [n_samples, n_chains, 3]."""
    R = np.asarray(R_series, np.float64)
    n = R.shape[0]
    norm = np.mean((R * R).sum(axis=2))
    out = np.empty(max_lag + 1)
    for tau in range(max_lag + 1):
        out[tau] = np.mean((R[tau:] * R[:n - tau]).sum(axis=2)) / norm
    return out


def rdf(x, L: float, sites: int, r_max: float, n_bins: int):
    """Radial distribution function of non-bonded site pairs (all pairs but
    1-2 and 1-3 neighbours of a chain, the exclusions of Sec. 3.1), minimum
    image in a cubic box of side L, r_max <= L/2.  Returns (bin centres,
    g(r), pair counts per bin): counts / (n_pairs * shell volume / L^3), with
    n_pairs the number of pairs the definition admits."""
    x = np.asarray(x, np.float64)
    N = len(x)
    edges = np.linspace(0.0, r_max, n_bins + 1)
    counts = np.zeros(n_bins, np.int64)
    chain = np.arange(N) // sites
    site = np.arange(N) % sites
    n_pairs = 0
    for i in range(N - 1):
        d = x[i + 1:] - x[i]
        d -= L * np.round(d / L)
        r = np.sqrt((d * d).sum(axis=1))
        keep = ~((chain[i + 1:] == chain[i]) & (np.abs(site[i + 1:] - site[i]) <= 2))
        n_pairs += int(keep.sum())
        h, _ = np.histogram(r[keep], bins=edges)
        counts += h
    shell = 4.0 / 3.0 * np.pi * (edges[1:] ** 3 - edges[:-1] ** 3)
    g = counts / (n_pairs * shell / L ** 3)
    return 0.5 * (edges[1:] + edges[:-1]), g, counts
