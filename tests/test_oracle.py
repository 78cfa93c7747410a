"""Pins for the FP64 oracle against what the paper and mathematics fix.

Every check here is independent of the oracle's own formulas: the paper's
worked topology example, finite differences of the energy, closed forms at
special geometries, conservation laws, an independent integrator (Leap-Frog),
time reversibility, and a hand-iterated thermostat recurrence.
"""
import math
import os

import numpy as np
import pytest

import chaingen
import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _read_rows(name):
    rows = {}
    for line in open(os.path.join(GOLD, name)):
        if line.startswith("#") or not line.strip():
            continue
        k, *v = line.split()
        rows[k] = np.array([int(a) for a in v])
    return rows


# ---------------------------------------------------------------- topology

def test_fig5_t_angles_worked_example():
    g = _read_rows("fig5_t_angles.txt")
    t = oracle.chain_topology(7)
    idx, rows = t.home_view(t.angles)
    assert np.array_equal(idx, g["index"])
    assert np.array_equal(rows[:, 0], g["ang_idx"])
    assert np.array_equal(rows[:, 1], g["pos"])
    assert np.array_equal(rows[:, 2] + 1, g["at1"])     # paper ids are 1-based
    assert np.array_equal(rows[:, 3] + 1, g["at2"])


def test_t_bonds_worked_example():
    g = _read_rows("t_bonds_7.txt")
    t = oracle.chain_topology(7)
    idx, bond = t.t_bonds()
    assert np.array_equal(idx, g["index"])
    assert np.array_equal(bond + 1, g["bond"])


def test_exclusions_are_first_and_second_neighbours():
    t = oracle.chain_topology(7)
    ex = [set(t.excl[t.excl_index[a]:t.excl_index[a + 1]]) for a in range(7)]
    for a in range(7):
        want = {b for b in range(7) if 1 <= abs(a - b) <= 2}
        assert ex[a] == want
    # dihedral home view: positions 1..4, four per interior atom
    idx, rows = t.home_view(t.dihedrals)
    assert list(np.diff(idx)) == [1, 2, 3, 4, 3, 2, 1]
    assert set(rows[:, 1]) == {1, 2, 3, 4}


# ---------------------------------------------------------------- helpers

def _fd_check(energy, x, atoms, h=1e-6):
    """central differences of energy vs the analytic force on chosen atoms"""
    out = []
    for i in atoms:
        for a in range(3):
            xp = x.copy(); xp[i, a] += h
            xm = x.copy(); xm[i, a] -= h
            out.append(-(energy(xp) - energy(xm)) / (2 * h))
    return np.array(out)


def _melt(n_chains, L=None, seed=3):
    m = chaingen.melt(n_chains, seed=seed, L=L)
    return m, oracle.System(oracle.chain_topology(150), n_chains, m["L"])


# ---------------------------------------------------------------- LJ, Eq. (2)

@pytest.mark.parametrize("ta,tb", [(0, 0), (0, 1), (1, 1)])
def test_lj_pair_closed_forms(ta, tb):
    p = oracle.default_params()
    eps = math.sqrt(p["eps"][ta] * p["eps"][tb])
    sig = math.sqrt(p["sigma"][ta] * p["sigma"][tb])
    # a 2-atom, bond-free molecule holding the two types
    s = oracle.System(oracle.Topology(2, np.zeros((0, 2), np.int32), np.array([ta, tb], np.int32)), 1, 5.0)
    for r, e_want, f_want in [(2 ** (1 / 6) * sig, -eps, 0.0), (sig, 0.0, 24 * eps / sig)]:
        x = np.array([[1.0, 1.0, 1.0], [1.0 + r, 1.0, 1.0]])
        f, en, _ = s.lj(x)
        assert en[0] == pytest.approx(e_want, abs=1e-12)
        assert -f[0, 0] == pytest.approx(f_want, rel=1e-12, abs=1e-9)  # repulsive pushes 0 to -x
        assert np.allclose(f[0], -f[1], atol=0)


def test_lj_cutoff_truncation_and_shift():
    p = oracle.default_params()
    topo = oracle.Topology(2, np.zeros((0, 2), np.int32), np.array([0, 0], np.int32))
    s = oracle.System(topo, 1, 5.0)
    rc = p["rc"]
    eps, sig = p["eps"][0], p["sigma"][0]
    e_rc = 4 * eps * ((sig / rc) ** 12 - (sig / rc) ** 6)
    for r, inside in [(rc * (1 - 1e-9), True), (rc, False), (rc * 1.01, False)]:
        x = np.array([[1.0, 1.0, 1.0], [1.0, 1.0 + r, 1.0]])
        f, en, _ = s.lj(x)
        if inside:
            assert en[0] == pytest.approx(e_rc, rel=1e-6)
            assert abs(en[1]) < 1e-9
        else:
            assert en[0] == 0.0 and en[1] == 0.0 and not f.any()


def test_lj_minimum_image():
    topo = oracle.Topology(2, np.zeros((0, 2), np.int32), np.array([0, 0], np.int32))
    L = 3.0
    s = oracle.System(topo, 1, L)
    a = np.array([[0.1, 1.0, 1.0], [0.5, 1.0, 1.0]])
    b = np.array([[0.1, 1.0, 1.0], [0.5 - L, 1.0, 1.0]])
    c = np.array([[2.9, 1.0, 1.0], [0.5 + L, 1.0, 1.0]])      # 0.6 apart across the face
    c2 = np.array([[2.9, 1.0, 1.0], [3.5, 1.0, 1.0]])
    fa, ea, _ = s.lj(a); fb, eb, _ = s.lj(b)
    assert np.allclose(fa, fb) and ea[0] == pytest.approx(eb[0])
    fc, ec, _ = s.lj(c); fc2, ec2, _ = s.lj(c2)
    assert ec[0] == pytest.approx(ec2[0]) and ec[0] != 0.0


def test_lj_forces_are_minus_energy_gradient():
    m, s = _melt(2, L=3.3)
    x = m["pos"]
    energy = lambda y: s.lj(y)[1][0]
    f, _, _ = s.lj(x)
    atoms = [0, 7, 149, 151, 222]
    fd = _fd_check(energy, x, atoms)
    an = np.concatenate([f[i] for i in atoms])
    assert np.allclose(fd, an, rtol=2e-6, atol=2e-5 * np.abs(an).max())


def test_lj_newton_third_law_and_virial_symmetry():
    m, s = _melt(2, L=3.3)
    f, en, vir = s.lj(m["pos"])
    assert np.abs(f.sum(0)).max() < 1e-10 * np.abs(f).max() * len(f)
    # virial trace equals sum r_ij.f_ij, computed here from forces: sum x_i . f_i
    # is not translation invariant under PBC, so compare cells vs brute instead
    f2, en2, vir2 = s.lj(m["pos"], method="cells")
    assert np.allclose(vir, vir2, rtol=1e-10, atol=1e-9)


@pytest.mark.parametrize("L", [3.05, 4.1])   # M = 3 and M = 4 cells of side >= r_c
def test_lj_brute_equals_cells(L):
    m, s = _melt(2, L=L, seed=5)
    fb, eb, vb = s.lj(m["pos"], method="brute")
    fc, ec, vc = s.lj(m["pos"], method="cells")
    assert int(L / 1.0) in (3, 4)
    assert np.allclose(fb, fc, rtol=1e-11, atol=1e-9)
    assert eb == pytest.approx(ec, rel=1e-11)


@pytest.mark.parametrize("L", [3.05, 4.1])   # M = 3 and M = 4 cells of side >= r_c
def test_lj_atoms_equals_brute_force_on_every_atom(L):
    """orc_lj_atoms (the checker of the full-size GPU tests) against the
    pinned all-pairs sum orc_lj_brute, element by element, for every atom of
    a tiny box.  The boxes hold intra-chain pairs at |i - j| = 2 (excluded)
    and 3 (counted, Sec. 3.1) inside r_c, and pairs across periodic faces,
    so a dropped exclusion, a missing j == i test or a wrong image fails."""
    m, s = _melt(2, L=L, seed=8)
    x = m["pos"]
    fb, _, _ = s.lj(x, method="brute")
    fa = s.lj_atoms(x, np.arange(len(x)))
    assert np.allclose(fa, fb, rtol=1e-12, atol=1e-12 * np.abs(fb).max())
    # the geometry really holds the cases named above
    n = len(x)
    i, j = np.triu_indices(n, 1)
    d = x[i] - x[j]
    img = np.round(d / L)
    r = np.linalg.norm(d - L * img, axis=1)
    same = (i // 150) == (j // 150)
    assert np.any(same & (np.abs(i - j) == 2) & (r < 1.0))
    assert np.any(same & (np.abs(i - j) == 3) & (r < 1.0))
    assert np.any((np.abs(img).sum(1) > 0) & (r < 1.0))


def test_kinetic_energy_hand_computed():
    """orc_kinetic = sum 1/2 m v^2 over atoms, masses by type (Table I:
    14.027 amu for C_32, 15.035 for the C_33 chain ends).  One 4-site chain
    with velocities chosen so the sum is done by hand:
      1/2 15.035 (1)  + 1/2 14.027 (4) + 1/2 14.027 (9) + 1/2 15.035 (3)
      = 7.5175 + 28.054 + 63.1215 + 22.5525 = 121.2455 kJ/mol."""
    s = oracle.System(oracle.chain_topology(4), 1, 10.0)
    v = np.array([[1.0, 0.0, 0.0], [0.0, 2.0, 0.0], [0.0, 0.0, 3.0], [1.0, 1.0, 1.0]])
    assert s.kinetic(v) == pytest.approx(121.2455, rel=1e-14)
    # two molecules: every atom counted once, with its own mass
    s2 = oracle.System(oracle.chain_topology(4), 2, 10.0)
    assert s2.kinetic(np.vstack([v, 2.0 * v])) == pytest.approx(5.0 * 121.2455, rel=1e-14)


# Cell index of one coordinate by the binning reading (Sec. 3.1): wrap
# s = x - L floor(x/L), then k = floor(s M / L) clamped to M - 1.  The boxes
# are chosen so that M / L is exact in FP64 and every step below is exact,
# so the expected cells follow from the reading by hand.
_BIN_CASES = [
    # (L, M, x, expected cell)
    (3.0, 3, 1.0, 1),                 # exactly on the face k L / M: the upper cell
    (3.0, 3, 2.0, 2),
    (3.0, 3, np.nextafter(1.0, 0.0), 0),   # just below that face
    (3.0, 3, 0.0, 0),
    (3.0, 3, -0.0, 0),                # negative zero wraps to 0
    (3.0, 3, 3.0, 0),                 # x = L wraps to 0
    (3.0, 3, np.nextafter(3.0, 4.0), 0),   # L + ulp wraps to a tiny positive s
    (3.0, 3, -1e-300, 2),             # tiny negative: s rounds to L, clamped to M - 1
    (3.0, 3, -1.0, 2),                # one cell below the box: the top cell
    (3.0, 3, 4.0, 1),                 # one box and one cell above
    (2.5, 5, 0.5, 1),                 # M / L = 2 exactly; faces at multiples of 0.5
    (2.5, 5, 2.0, 4),
    (2.5, 5, np.nextafter(0.5, 0.0), 0),
    (2.5, 5, 2.5, 0),
    (4.0, 4, 3.0, 3),
    (4.0, 4, np.nextafter(4.0, 0.0), 3),
]


@pytest.mark.parametrize("L,M,xv,want", _BIN_CASES)
def test_binning_cell_index_convention(L, M, xv, want):
    # the coordinate under test on each axis in turn, the others at a cell interior
    for axis in range(3):
        x = np.full((1, 3), 0.25 * L / M)
        x[0, axis] = xv
        cell_of, start, perm = oracle.bin_atoms(x, L, M)
        k = [0, 0, 0]
        k[axis] = want
        assert cell_of[0] == (k[2] * M + k[1]) * M + k[0]
        assert start[cell_of[0]] == 0 and start[cell_of[0] + 1] == 1 and perm[0] == 0


def test_lj_exclusions_only_first_and_second_neighbours():
    # a straight 4-atom chain spaced 0.4 nm: pairs (0,3) at 1.2 nm are outside r_c,
    # pairs (0,1),(0,2),(1,3) ... are excluded; use spacing 0.3 so 1-4 = 0.9 nm is inside
    topo = oracle.chain_topology(4)
    s = oracle.System(topo, 1, 10.0)
    x = np.array([[1.0 + 0.3 * k, 2.0, 2.0] for k in range(4)])
    f, en, _ = s.lj(x)
    p = oracle.default_params()
    eps = math.sqrt(p["eps"][1] * p["eps"][1]); sig = p["sigma"][1]   # ends are C_33
    r = 0.9
    want = 4 * eps * ((sig / r) ** 12 - (sig / r) ** 6)
    assert en[0] == pytest.approx(want, rel=1e-12)


# ---------------------------------------------------------------- bonded, Eqs. (4)-(6)

def _only(p, **keep):
    q = dict(p)
    for k in ("kb", "ka", "kphi"):
        if k not in keep:
            q[k] = 0.0
    q.update({k: v for k, v in keep.items()})
    return q


def test_single_bond_closed_form():
    p = oracle.default_params()
    topo = oracle.chain_topology(2)
    s = oracle.System(topo, 1, 10.0, params=_only(p, kb=p["kb"]))
    for r in (0.150, 0.153, 0.158):
        x = np.array([[1.0, 1.0, 1.0], [1.0 + r, 1.0, 1.0]])
        f, en, _ = s.bonded(x)
        assert en[0] == pytest.approx(0.5 * p["kb"] * (r - p["b0"]) ** 2, rel=1e-12, abs=1e-15)
        assert f[1, 0] == pytest.approx(-p["kb"] * (r - p["b0"]), rel=1e-12, abs=1e-9)
        assert f[0, 0] == -f[1, 0]


def _angle_positions(theta, r1=0.153, r2=0.153):
    b = np.array([2.0, 2.0, 2.0])
    a = b + r1 * np.array([1.0, 0.0, 0.0])
    c = b + r2 * np.array([math.cos(theta), math.sin(theta), 0.0])
    return np.array([a, b, c])


def test_angle_zero_force_at_equilibrium_and_energy():
    p = oracle.default_params()
    s = oracle.System(oracle.chain_topology(3), 1, 10.0, params=_only(p, ka=p["ka"]))
    f, en, _ = s.bonded(_angle_positions(p["theta0"]))
    assert np.abs(f).max() < 1e-9
    th = p["theta0"] + 0.2
    f, en, _ = s.bonded(_angle_positions(th))
    assert en[1] == pytest.approx(0.5 * p["ka"] * 0.2 ** 2, rel=1e-10)
    # torque-free and force-free
    assert np.abs(f.sum(0)).max() < 1e-10


def _dihedral_positions(phi):
    """a-b-c-d with tetrahedral-ish angles and IUPAC dihedral phi"""
    b = np.array([2.0, 2.0, 2.0]); c = b + np.array([0.153, 0.0, 0.0])
    a = b + 0.153 * np.array([math.cos(math.radians(70.5)), math.sin(math.radians(70.5)), 0.0])
    # d: rotate the cis position (same side as a) by phi around the b->c axis
    u = np.array([-math.cos(math.radians(70.5)), math.sin(math.radians(70.5)), 0.0]) * 0.153
    rot = np.array([u[0], u[1] * math.cos(phi), u[1] * math.sin(phi)])
    d = c + rot
    return np.array([a, b, c, d])


def test_dihedral_closed_forms():
    p = oracle.default_params()
    s = oracle.System(oracle.chain_topology(4), 1, 10.0, params=_only(p, kphi=p["kphi"]))
    k = p["kphi"]
    for phi_deg, e_want in [(180.0, 0.0), (0.0, 2 * k), (60.0, 0.0), (-60.0, 0.0), (120.0, 2 * k)]:
        f, en, _ = s.bonded(_dihedral_positions(math.radians(phi_deg)))
        assert en[2] == pytest.approx(e_want, abs=1e-9), phi_deg
        if e_want == 0.0:
            assert np.abs(f).max() < 1e-8


@pytest.mark.parametrize("term,phis,n", [("kb", 0.0, 3), ("ka", 0.0, 3), ("kphi", 0.0, 3),
                                         ("kphi", 0.4, 3), ("kphi", 1.1, 1), ("kphi", -0.7, 2)])
def test_bonded_forces_are_minus_energy_gradient(term, phis, n):
    p = oracle.default_params()
    q = _only(p, **{term: p[term]})
    q["phis"], q["n_mult"] = phis, n
    m, _ = _melt(1, L=3.4, seed=9)
    x = m["pos"].copy()
    # perturb away from exact tetrahedral geometry
    rng = np.random.default_rng(0)
    x += rng.normal(scale=0.01, size=x.shape)
    s = oracle.System(oracle.chain_topology(150), 1, m["L"], params=q)
    e_idx = {"kb": 0, "ka": 1, "kphi": 2}[term]
    energy = lambda y: s.bonded(y)[1][e_idx]
    f, _, _ = s.bonded(x)
    atoms = [0, 1, 2, 75, 148, 149]
    fd = _fd_check(energy, x, atoms, h=1e-7)
    an = np.concatenate([f[i] for i in atoms])
    assert np.allclose(fd, an, rtol=1e-5, atol=1e-6 * max(1.0, np.abs(an).max()))


def test_bonded_translation_and_rotation_invariance():
    m, _ = _melt(1, L=30.0, seed=2)         # box large enough that no bond crosses a face
    x = m["pos"] - m["pos"].mean(0) + 15.0
    s = oracle.System(oracle.chain_topology(150), 1, 30.0)
    f, en, _ = s.bonded(x)
    assert np.abs(f.sum(0)).max() < 1e-8 * np.abs(f).max() * 150
    torque = np.cross(x - x.mean(0), f).sum(0)
    assert np.abs(torque).max() < 1e-8 * np.abs(f).max() * 150


# ---------------------------------------------------------------- binning (Sec. 3.1)

def test_binning_is_a_stable_sort_and_atoms_lie_in_their_cells():
    m, _ = _melt(4, seed=11)
    x, L = m["pos"], m["L"]
    M = 3
    cell_of, start, perm = oracle.bin_atoms(x, L, M)
    h = L / M
    c = np.stack([cell_of % M, (cell_of // M) % M, cell_of // (M * M)], 1)
    assert np.all(x >= c * h - 1e-12) and np.all(x <= (c + 1) * h + 1e-12)
    # library stable sort by cell id reproduces the permutation
    assert np.array_equal(perm, np.argsort(cell_of, kind="stable"))
    assert np.array_equal(np.diff(start), np.bincount(cell_of, minlength=M ** 3))
    assert start[0] == 0 and start[-1] == len(x)


# ---------------------------------------------------------------- integration

def _small_system(seed=4):
    m = chaingen.melt(2, seed=seed, L=3.3, T=300.0)
    return m, oracle.System(oracle.chain_topology(150), 2, m["L"])


def test_total_energy_gradient_of_whole_system():
    m, s = _small_system()
    x = m["pos"]
    energy = lambda y: sum(s.forces(y)[1][[0, 2, 3, 4]])
    f, _, _ = s.forces(x)
    atoms = [3, 100, 200]
    fd = _fd_check(energy, x, atoms, h=1e-7)
    an = np.concatenate([f[i] for i in atoms])
    assert np.allclose(fd, an, rtol=1e-5, atol=1e-5 * np.abs(an).max())


def test_leapfrog_gives_the_same_positions():
    m, s = _small_system()
    dt, n = 0.001, 40
    x1, v1, f1, _, _ = s.run(m["pos"], m["vel"], dt, n, sample_every=0)
    # independent Leap-Frog: v(-1/2) = v0 - dt/2 a0, then kick-drift
    mass = np.tile(s.masses_m, 2)[:, None]
    x = m["pos"].copy()
    f, _, _ = s.forces(x)
    v = m["vel"] - 0.5 * dt * f / mass
    for _ in range(n):
        v = v + dt * f / mass
        x = x + dt * v
        f, _, _ = s.forces(x)
    assert np.abs(x - x1).max() < 1e-11


def test_time_reversibility():
    m, s = _small_system()
    dt, n = 0.001, 60
    x1, v1, _, _, _ = s.run(m["pos"], m["vel"], dt, n, sample_every=0)
    x2, v2, _, _, _ = s.run(x1, -v1, dt, n, sample_every=0)
    assert np.abs(x2 - m["pos"]).max() < 1e-9
    assert np.abs(v2 + m["vel"]).max() < 1e-7


def test_nve_energy_error_scales_as_dt_squared():
    m, s = _small_system(seed=6)
    # relax the hot start briefly with the thermostat, then run NVE for 0.1 ps
    x, v, _, _, lam = s.run(m["pos"], m["vel"], 0.0005, 400, thermostat=True, T0=300.0, tau=0.02)
    devs = []
    for dt in (0.001, 0.0005, 0.00025):
        steps = int(round(0.1 / dt))
        _, _, _, smp, _ = s.run(x, v, dt, steps, sample_every=1)
        etot = smp[:, 2] + smp[:, 3] + smp[:, 4] + smp[:, 5] + smp[:, 6]
        devs.append(np.sqrt(np.mean((etot - etot[0]) ** 2)))
    r1, r2 = devs[0] / devs[1], devs[1] / devs[2]
    assert 3.0 < r1 < 5.0 and 3.0 < r2 < 5.0, devs


def test_thermostat_matches_hand_recurrence():
    # with every interaction switched off velocities change only by scaling, so
    # T_{k+1} = lambda_{k-1}^2 T_k with lambda_{k-1} from T_{k-1}
    p = oracle.default_params()
    q = dict(p, kb=0.0, ka=0.0, kphi=0.0, eps=(0.0, 0.0))
    m = chaingen.melt(1, seed=2, L=3.3, T=450.0)
    s = oracle.System(oracle.chain_topology(150), 1, m["L"], params=q)
    dt, tau, T0, n = 0.001, 0.01, 300.0, 30
    _, _, _, smp, lam = s.run(m["pos"], m["vel"], dt, n, thermostat=True, T0=T0, tau=tau)
    T = [smp[0, 7]]
    lam_prev = 1.0
    for k in range(n):
        lam_k = math.sqrt(1 + dt / tau * (T0 / T[k] - 1))
        T.append(T[k] * lam_prev ** 2)
        lam_prev = lam_k
    assert np.allclose(smp[:, 7], T, rtol=1e-12)
    assert lam == pytest.approx(lam_prev, rel=1e-12)


# ---------------------------------------------------------------- trajectory means (gradient checks)

def test_traj_means_dimer_matches_exact_discrete_oscillator():
    """One harmonic dimer (Eq. 4 only, no angles or LJ partners), released
    at rest from b0 + delta along x.  Velocity Verlet on the relative
    coordinate has the exact discrete solution delta cos(k W dt) with
    cos(W dt) = 1 - (omega dt)^2 / 2, omega^2 = k_b / mu."""
    p = oracle.default_params()
    s = oracle.System(oracle.chain_topology(2), 1, 4.0, params=p)
    mu = p["mass"][1] / 2.0                      # both ends are C_33
    dt, K, delta = 0.001, 300, 0.004
    x = np.array([[1.0, 1.5, 1.5], [1.0 + p["b0"] + delta, 1.5, 1.5]])
    W = math.acos(1.0 - 0.5 * (p["kb"] / mu) * dt * dt) / dt
    k = np.arange(K + 1)
    q = delta * np.cos(k * W * dt)
    want_u = np.mean(0.5 * p["kb"] * q * q)
    want_r2 = np.mean((p["b0"] + q) ** 2)
    got = s.traj_means(x, np.zeros_like(x), dt, K)
    assert got[0] == pytest.approx(want_u, rel=1e-9)
    assert got[1] == pytest.approx(want_r2, rel=1e-12)


def test_traj_means_end_to_end_of_all_trans_chains():
    """Planar all-trans zigzag of n bonds (length b, angle theta):
    R^2 = b^2 (n^2 sin^2(theta/2) + (n mod 2) cos^2(theta/2))."""
    p = oracle.default_params()
    b, th, sites = p["b0"], p["theta0"], 150
    k = np.arange(sites - 1)
    bonds = b * np.stack([np.full(sites - 1, math.sin(th / 2)), (-1.0) ** k * math.cos(th / 2),
                          np.zeros(sites - 1)], axis=1)
    chain = np.concatenate([np.zeros((1, 3)), np.cumsum(bonds, axis=0)])
    # two chains 3 nm apart in z, in a box much longer than a chain
    x = np.concatenate([chain + [0.5, 1.0, 1.0], chain + [0.5, 1.0, 4.0]])
    s = oracle.System(oracle.chain_topology(sites), 2, 40.0)
    n = sites - 1
    want = b * b * (n * n * math.sin(th / 2) ** 2 + math.cos(th / 2) ** 2)
    assert s.traj_means(x, np.zeros_like(x), 0.001, 0)[1] == pytest.approx(want, rel=1e-12)


def test_fd_gradient_at_zero_steps_against_closed_forms():
    """With K = 0 the means are U(x0) and R_ee^2(x0).  E_d is linear in
    k_phi (Eq. 6), the LJ energy is homogeneous of degree 1 in (eps_C32,
    eps_C33) under the geometric mean, and R_ee^2 does not depend on any
    parameter."""
    m, s = _small_system()
    x = chaingen.unwrapped(m)
    _, en, _ = s.forces(x)
    g = s.fd_gradient(x, m["vel"], 0.001, 0)
    th = s.theta()
    assert g[0, 4] == pytest.approx(en[4] / th[4], rel=1e-8)
    assert th[0] * g[0, 0] + th[1] * g[0, 1] == pytest.approx(en[1], rel=1e-7)
    assert np.abs(g[1]).max() < 1e-9


def test_fd_gradient_sigma_of_an_isolated_pair():
    """Two bond-free C_33 sites at r < r_c: U = 4 eps [(s/r)^12 - (s/r)^6]
    minus the same at r_c, so dU/dsigma_C33 has a closed form."""
    p = oracle.default_params()
    topo = oracle.Topology(2, np.zeros((0, 2), np.int32), np.array([1, 1], np.int32))
    s = oracle.System(topo, 1, 5.0, params=p)
    r, rc, eps, sig = 0.41, p["rc"], p["eps"][1], p["sigma"][1]
    x = np.array([[1.0, 1.0, 1.0], [1.0 + r, 1.0, 1.0]])
    d = lambda q: 4 * eps * (12 * sig ** 11 / q ** 12 - 6 * sig ** 5 / q ** 6)
    g = s.fd_gradient(x, np.zeros_like(x), 0.001, 0, rel_h=1e-5)
    assert g[0, 3] == pytest.approx(d(r) - d(rc), rel=1e-7)
    assert g[0, 1] == pytest.approx((4 * ((sig / r) ** 12 - (sig / r) ** 6 - (sig / rc) ** 12 + (sig / rc) ** 6)),
                                    rel=1e-7)
    assert abs(g[0, 0]) < 1e-9 and abs(g[0, 2]) < 1e-9


def test_force_shifted_variant_closed_form_and_continuity():
    """lj_form = 1: E_sf(r) = E(r) - E(r_c) - (r - r_c) E'(r_c) with
    E = 4 eps [(s/r)^12 - (s/r)^6]; energy and force both vanish at r_c."""
    p = dict(oracle.default_params(), lj_form=1)
    topo = oracle.Topology(2, np.zeros((0, 2), np.int32), np.array([0, 0], np.int32))
    s = oracle.System(topo, 1, 5.0, params=p)
    eps, sig, rc = p["eps"][0], p["sigma"][0], p["rc"]
    E = lambda r: 4 * eps * ((sig / r) ** 12 - (sig / r) ** 6)
    dE = lambda r: 4 * eps * (-12 * sig ** 12 / r ** 13 + 6 * sig ** 6 / r ** 7)
    for r in (0.35, 0.5, 0.8, rc - 1e-9):
        x = np.array([[1.0, 1.0, 1.0], [1.0 + r, 1.0, 1.0]])
        f, en, _ = s.lj(x)
        assert en[0] == pytest.approx(E(r), rel=1e-12)
        assert en[1] == pytest.approx(E(r) - E(rc) - (r - rc) * dE(rc), rel=1e-9, abs=1e-14)
        assert f[1, 0] == pytest.approx(-(dE(r) - dE(rc)), rel=1e-9, abs=1e-12)
    x = np.array([[1.0, 1.0, 1.0], [1.0 + rc - 1e-9, 1.0, 1.0]])
    f, en, _ = s.lj(x)
    assert abs(en[1]) < 1e-15 and abs(f[1, 0]) < 1e-9


def test_force_shifted_variant_forces_are_minus_energy_gradient():
    m = chaingen.melt(2, seed=4, L=3.3, T=300.0)
    s = oracle.System(oracle.chain_topology(150), 2, m["L"], params=dict(oracle.default_params(), lj_form=1))
    x = m["pos"]
    f, _, _ = s.lj(x)
    atoms = [5, 77, 160, 299]
    fd = _fd_check(lambda y: s.lj(y)[1][1], x, atoms, h=1e-7)
    an = np.concatenate([f[i] for i in atoms])
    assert np.allclose(fd, an, rtol=1e-5, atol=1e-6 * np.abs(an).max())


# ------------------------------------------------------------------ Leap-Frog + Nose-Hoover (Sec. 2, 3.4)
def _nh_system(T=450.0, seed=12):
    m = chaingen.melt(4, seed=seed, L=3.4, T=T)
    return m, oracle.System(oracle.chain_topology(150), 4, m["L"], use_cells=False)


def test_nose_hoover_extended_energy_error_is_second_order():
    """The extended energy K + U + g kB Q xi^2/2 + g kB T0 int(xi) is
    conserved by the continuous equations; the leap-frog scheme keeps it to
    O(dt^2) over a fixed time (a quench from 450 K to 300 K with tau = 0.1
    ps, so xi moves far from 0)."""
    m, s = _nh_system()
    err = []
    for dt, K in ((0.001, 200), (0.0005, 400), (0.00025, 800)):
        _, _, _, smp, _ = s.run_nh(m["pos"], m["vel"], dt, K, T0=300.0, tau=0.1, sample_every=K // 50)
        H = s.nh_extended_energy(smp, 300.0, 0.1)
        err.append(np.abs(H - H[0]).max())
    assert 3.3 < err[0] / err[1] < 4.7 and 3.3 < err[1] / err[2] < 4.7, err


def test_nose_hoover_without_coupling_is_velocity_verlet():
    """Q -> infinity: xi stays 0 and the run is NVE velocity Verlet (the
    centre-of-mass velocity of the generator's input is already zero)."""
    m, s = _nh_system()
    xa, va, _, _, xi = s.run_nh(m["pos"], m["vel"], 0.001, 40, T0=300.0, tau=1e9, sample_every=0)
    xb, vb, _, _, _ = s.run(m["pos"], m["vel"], 0.001, 40, sample_every=0)
    assert abs(xi) < 1e-12
    assert np.abs(xa - xb).max() < 1e-12 and np.abs(va - vb).max() < 1e-9


def test_nose_hoover_removes_centre_of_mass_translation():
    m, s = _nh_system()
    masses = np.asarray(m["masses"])                       # per atom
    v = m["vel"] + np.array([0.3, -0.2, 0.1])              # a drifting input
    _, v1, _, _, _ = s.run_nh(m["pos"], v, 0.001, 1, T0=300.0, tau=0.1, sample_every=0)
    p = (masses[:, None] * v1).sum(0)
    assert np.abs(p).max() < 1e-10 * np.abs(masses[:, None] * v1).sum()


def test_nose_hoover_run_splits_at_any_step():
    """Two runs of 7 and 13 steps, the second from the first's on-step state
    and xi, give the 20-step run bit for bit (what a GPU call boundary must
    reproduce)."""
    m, s = _nh_system()
    x20, v20, _, _, xi20 = s.run_nh(m["pos"], m["vel"], 0.001, 20, T0=300.0, tau=0.1, sample_every=0)
    x7, v7, _, _, xi7 = s.run_nh(m["pos"], m["vel"], 0.001, 7, T0=300.0, tau=0.1, sample_every=0)
    x, v, _, _, xi = s.run_nh(x7, v7, 0.001, 13, T0=300.0, tau=0.1, xi=xi7, sample_every=0)
    assert np.array_equal(x, x20) and np.array_equal(v, v20) and xi == xi20


def test_nose_hoover_cools_a_hot_melt_towards_the_target():
    m, s = _nh_system()
    _, _, _, smp, _ = s.run_nh(m["pos"], m["vel"], 0.001, 400, T0=300.0, tau=0.1, sample_every=100)
    assert smp[0, 7] > 400.0
    assert abs(smp[-1, 7] - 300.0) < 10.0
