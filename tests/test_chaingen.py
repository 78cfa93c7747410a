"""Input generator: geometry rules, density, determinism across platforms."""
import math
import os
import sys

import numpy as np

import chaingen

sys.path.insert(0, os.path.join(os.path.dirname(__file__), "golden"))
import make_golden  # noqa: E402


def _unwrap_chains(m):
    p = m["pos"].reshape(m["n_chains"], m["sites"], 3)
    d = np.diff(p, axis=1)
    d -= m["L"] * np.round(d / m["L"])
    return d


def test_bond_lengths_angles_and_dihedrals():
    m = chaingen.melt(10, seed=1)
    d = _unwrap_chains(m)
    assert np.abs(np.linalg.norm(d, axis=2) - 0.153).max() < 1e-12
    b1, b2 = d[:, :-1], d[:, 1:]
    cos_t = -(b1 * b2).sum(2) / (np.linalg.norm(b1, axis=2) * np.linalg.norm(b2, axis=2))
    assert np.abs(cos_t + 1.0 / 3.0).max() < 1e-12          # tetrahedral angle 109.47 deg
    u1, u2, u3 = d[:, :-2], d[:, 1:-1], d[:, 2:]
    n1, n2 = np.cross(u1, u2), np.cross(u2, u3)
    phi = np.degrees(np.arctan2(np.linalg.norm(u2, axis=2) * (u1 * n2).sum(2), (n1 * n2).sum(2)))
    near = np.minimum.reduce([np.abs(np.abs(phi) - 180.0), np.abs(phi - 60.0), np.abs(phi + 60.0)])
    assert near.max() < 1e-9
    frac_trans = np.mean(np.abs(np.abs(phi) - 180.0) < 1e-6)
    assert 0.4 < frac_trans < 0.8


def test_density_box_and_velocities():
    m = chaingen.melt(10, seed=1)
    N = 1500
    mass_g = m["masses"].sum() * chaingen.AMU_G
    rho = mass_g / (m["L"] * 1e-7) ** 3
    assert abs(rho - 0.77) < 1e-4
    assert abs(m["L"] - 3.5678) < 1e-3                      # "L about 35.6 A"
    assert np.float32(m["L"]) == m["L"]                      # exactly representable in FP32
    assert np.all((m["pos"] >= 0) & (m["pos"] < m["L"]))
    p = (m["masses"][:, None] * m["vel"]).sum(0)
    assert np.abs(p).max() < 1e-9
    ke = 0.5 * (m["masses"][:, None] * m["vel"] ** 2).sum()
    T = 2 * ke / ((3 * N - 3) * chaingen.KB)
    assert abs(T - 500.0) < 40.0
    assert m["types"][0] == 1 and m["types"][1] == 0 and m["types"][149] == 1


def test_same_bits_on_every_platform():
    want = {}
    for line in open(os.path.join(os.path.dirname(__file__), "golden", "chaingen_digest.txt")):
        if line.startswith("#"):
            continue
        n, s, h = line.split()
        want[(int(n), int(s))] = h
    for (n, s), h in want.items():
        assert make_golden.digest(n, s) == h


def test_replica_recipe():
    counts, temps = chaingen.replica_recipe(64, seed=4)
    assert len(counts) == 64 and min(counts) >= 20 and max(counts) <= 400
    assert all(250.0 <= t <= 500.0 for t in temps)
    # log-uniform: median near sqrt(20*400) ~ 89
    assert 50 < sorted(counts)[32] < 160
    assert abs(chaingen._load().cg_ln_export(10.0) - math.log(10.0)) < 1e-15
    assert abs(chaingen._load().cg_exp_export(2.5) - math.exp(2.5)) < 1e-14


def test_maxwell_resample_temperature_and_momentum():
    """Fresh Maxwell draws: zero total momentum, equipartition temperature
    within 4 standard errors (3N-3 degrees of freedom), distinct streams."""
    masses = np.tile(chaingen.site_masses(150), 200)
    T = 437.0
    v = chaingen.maxwell(masses, T, seed=5, stream=100)
    assert np.abs((masses[:, None] * v).sum(0)).max() < 1e-9
    dof = 3 * len(masses) - 3
    t_meas = (masses[:, None] * v * v).sum() / (dof * chaingen.KB)
    assert abs(t_meas / T - 1.0) < 4.0 * math.sqrt(2.0 / dof)
    w = chaingen.maxwell(masses, T, seed=5, stream=101)
    assert np.abs(v - w).max() > 0.1
    assert np.array_equal(v, chaingen.maxwell(masses, T, seed=5, stream=100))
