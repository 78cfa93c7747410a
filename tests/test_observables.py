"""Pins of the structural observables in oracle/observables.py (CPU): closed
forms, constructed geometries, and an independent pair count."""
import math

import numpy as np
import pytest
from scipy.spatial import cKDTree

import chaingen
from oracle import observables as ob


def test_straight_chain_end_to_end_and_radius_of_gyration():
    # n equal masses spaced b on a line: R_ee = (n - 1) b, R_g^2 = b^2 (n^2 - 1) / 12
    n, b = 11, 0.153
    x = np.zeros((2 * n, 3))
    x[:n, 0] = b * np.arange(n)
    x[n:, 1] = 1.0 + b * np.arange(n)                 # a second chain along y
    R = ob.end_to_end(x, n)
    assert np.allclose(R, [[(n - 1) * b, 0, 0], [0, (n - 1) * b, 0]], atol=1e-15)
    rg2 = ob.radius_of_gyration_sq(x, n, np.full(2 * n, 14.027))
    assert np.allclose(rg2, b * b * (n * n - 1) / 12.0, rtol=1e-12)
    # mass weighting: a heavy end pulls the centre of mass
    m = np.full(n, 1.0); m[-1] = 1e6
    rg2_heavy = ob.radius_of_gyration_sq(x[:n], n, m)
    assert rg2_heavy[0] < 1e-3 * rg2[0]


def _quad(phi_deg):
    """a-b-c-d with bond 0.153 nm, bond angles 109.5 deg, dihedral phi
    measured from cis (phi = 0) around b -> c; trans at 180."""
    phi = math.radians(phi_deg)
    ang = math.radians(70.5)
    b = np.array([2.0, 2.0, 2.0]); c = b + np.array([0.153, 0.0, 0.0])
    a = b + 0.153 * np.array([math.cos(ang), math.sin(ang), 0.0])
    u = np.array([-math.cos(ang), math.sin(ang), 0.0]) * 0.153
    d = c + np.array([u[0], u[1] * math.cos(phi), u[1] * math.sin(phi)])
    return np.array([a, b, c, d])


@pytest.mark.parametrize("phi,trans", [(180.0, True), (179.0, True), (121.0, True), (119.0, False),
                                       (60.0, False), (0.0, False), (-60.0, False), (-121.0, True)])
def test_dihedral_states(phi, trans):
    got = ob.dihedral_angles(_quad(phi), 4)[0, 0]
    assert abs(abs(got) - abs(phi)) < 1e-9
    assert ob.trans_fraction(_quad(phi), 4) == (1.0 if trans else 0.0)


def test_dihedral_sign_is_antisymmetric():
    assert ob.dihedral_angles(_quad(60.0), 4)[0, 0] == pytest.approx(-ob.dihedral_angles(_quad(-60.0), 4)[0, 0])


def test_generator_trans_fraction():
    """The generator draws trans with p = 0.6 and gauche+- with 0.2 each."""
    m = chaingen.melt(20, seed=3)
    f = ob.trans_fraction(chaingen.unwrapped(m), m["sites"])
    assert 0.5 < f < 0.7, f


def test_acf_of_rotating_vectors_is_a_cosine():
    # R(t) = A (cos(w t + p), sin(w t + p), 0): <R(t+tau).R(t)> = A^2 cos(w tau) for every origin
    w, n_t = 0.07, 400
    t = np.arange(n_t)[:, None]
    A = np.array([1.0, 2.5, 0.7])[None, :]
    p = np.array([0.0, 1.0, 2.0])[None, :]
    R = np.stack([A * np.cos(w * t + p), A * np.sin(w * t + p), np.zeros((n_t, 3))], axis=2)
    c = ob.end_to_end_acf(R, 50)
    assert np.allclose(c, np.cos(w * np.arange(51)), atol=1e-12)


def test_rdf_counts_match_an_independent_pair_count_and_normalise():
    rng = np.random.default_rng(1)
    L, sites = 3.0, 5
    x = rng.uniform(0.0, L, size=(400, 3))
    r_c, g, cnt = ob.rdf(x, L, sites, 1.4, 14)
    # independent count with a periodic KD tree, exclusions applied by hand
    tr = cKDTree(x, boxsize=L)
    pairs = tr.query_pairs(1.4, output_type="ndarray")
    d = x[pairs[:, 0]] - x[pairs[:, 1]]
    d -= L * np.round(d / L)
    r = np.linalg.norm(d, axis=1)
    same = (pairs[:, 0] // sites == pairs[:, 1] // sites) & (np.abs(pairs[:, 0] - pairs[:, 1]) <= 2)
    want, _ = np.histogram(r[~same], bins=np.linspace(0.0, 1.4, 15))
    assert np.array_equal(cnt, want)
    # an ideal gas: g = 1 within its counting noise
    sigma = 1.0 / np.sqrt(np.maximum(cnt, 1))
    assert np.all(np.abs(g[4:] - 1.0) < 5 * sigma[4:] + 0.02)
