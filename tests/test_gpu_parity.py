"""CUDA path vs the FP64 oracle, through the C ABI, on seeded melts.

Tolerances (stated here, derived from the arithmetic):
  * binning: bit-exact (cell ids are FP64 on both sides)
  * neighbour pairs: every pair the oracle finds inside r_c is listed; every
    listed pair lies inside r_c + skin (+1e-5 nm of FP32 rounding)
  * forces: the relative force error ||F_gpu - F_oracle||_2 / ||F_oracle||_2
    over all atoms is <= 1e-5, and every atom obeys
    |F_gpu - F_oracle|_max <= 5e-5 * RMS_i |F_oracle| (FP32 coordinates carry
    ~7e-8 nm and FP32 bond lengths ~1e-8 nm of rounding, which at hot-start
    contacts and stiff bonds gives up to ~1e-5 on single atoms), except atoms
    with a pair within 2e-6 nm of r_c (the FP32 and FP64 cutoff tests may
    disagree there), which get |F(r_c)| per such pair on top
  * energies: 1e-5 relative (FP32 terms summed in FP64)
  * short trajectories: 1e-5 nm after 50 steps
"""
import math

import numpy as np
import pytest
from scipy.spatial import cKDTree

import chaingen
import oracle
import paper_1001_3764_gb300 as md

pytestmark = pytest.mark.gpu

FORCE_TOL = 1e-5       # relative RMS force error
ATOM_TOL = 5e-5        # per-atom max error / RMS force


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    md.load()


def _oracle(melt, params=None):
    n = melt["n_chains"]
    return oracle.System(oracle.chain_topology(melt["sites"]), n, melt["L"], params=params,
                         use_cells=n * melt["sites"] > 3000)


def _uploaded(melt, precision=md.MD_MIXED):
    """The state a system holds right after creation, computed on the host
    from the generator's output (its positions are already in [0, L)): FP64
    as given, or rounded to FP32 (nearest even) for the plain form.  Oracle
    inputs come from here, never from the GPU."""
    x = np.array(melt["pos"], np.float64)
    v = np.array(melt["vel"], np.float64)
    if precision == md.MD_PLAIN_FP32:
        x = x.astype(np.float32).astype(np.float64)
        v = v.astype(np.float32).astype(np.float64)
    return x, v


def _ambiguous_pairs(x, L, rc, tol=2e-6):
    tr = cKDTree(np.mod(x, L), boxsize=L)
    pairs = tr.query_pairs(rc + tol, output_type="ndarray")
    if len(pairs) == 0:
        return np.zeros(len(x), int)
    d = x[pairs[:, 0]] - x[pairs[:, 1]]
    d -= L * np.round(d / L)
    r = np.linalg.norm(d, axis=1)
    amb = pairs[np.abs(r - rc) < tol]
    cnt = np.zeros(len(x), int)
    np.add.at(cnt, amb[:, 0], 1)
    np.add.at(cnt, amb[:, 1], 1)
    return cnt


def check_forces(f_gpu, f_orc, x, L, params=None):
    p = params or oracle.default_params()
    scale = np.sqrt(np.mean(np.sum(f_orc ** 2, axis=1)))
    err = np.abs(f_gpu - f_orc).max(axis=1)
    amb = _ambiguous_pairs(x, L, 1.0)
    sig, eps = max(p["sigma"]), max(p["eps"])
    f_rc = abs(24 * eps * (2 * sig ** 12 - sig ** 6))   # |F(r_c)| bound at r_c = 1 nm
    allowed = ATOM_TOL * scale + amb * 1.01 * f_rc
    bad = np.where(err > allowed)[0]
    assert len(bad) == 0, f"{len(bad)} atoms off; worst rel {err.max() / scale:.3e}"
    clean = amb == 0
    rel = np.sqrt(np.sum((f_gpu - f_orc)[clean] ** 2) / np.sum(f_orc[clean] ** 2))
    assert rel <= FORCE_TOL, f"relative force error {rel:.3e}"
    return rel, err.max() / scale


@pytest.mark.parametrize("precision", [md.MD_MIXED, md.MD_PLAIN_FP32])
@pytest.mark.parametrize("n_chains,L", [(10, None), (1, 3.4), (30, 5.2)])
def test_binning_is_bit_exact(precision, n_chains, L):
    m = chaingen.melt(n_chains, seed=21, L=L)
    s = md.System(m, precision=precision)
    x, _ = _uploaded(m, precision)
    M = s.info["cells_per_side"]
    assert M == int(m["L"] // 1.1)
    co, cs, pm = s.bins()
    oc, ocs, opm = oracle.bin_atoms(x, m["L"], M)
    assert np.array_equal(co, oc)
    assert np.array_equal(cs, ocs)
    assert np.array_equal(pm, opm)
    s.close()


def _ingested(x, L, precision):
    """What md_set_state / md_create store for caller positions x (the rule
    stated in md.h): x - L floor(x / L), with a result that is not below L
    (a tiny negative x) stored as 0; in the plain form then rounded to FP32,
    with a value that rounds to L stored as 0."""
    y = np.array(x, np.float64)
    y = y - L * np.floor(y / L)
    y[~((y < L) & (y >= 0.0))] = 0.0
    if precision == md.MD_PLAIN_FP32:
        y = y.astype(np.float32).astype(np.float64)
        y[y >= np.float32(L)] = 0.0
    return y


@pytest.mark.parametrize("precision", [md.MD_MIXED, md.MD_PLAIN_FP32])
def test_binning_at_cell_faces_is_bit_exact(precision):
    """Coordinates placed exactly on cell faces, on the box faces, at -0.0,
    at a tiny negative value and one ulp beyond L (the cases the oracle's
    binning pins fix), uploaded through md_set_state.  r_c + skin = 1 nm and
    L = 4 nm make M / L = 1 exact, so both sides decide every face alike."""
    m = chaingen.melt(14, seed=23, L=4.0)
    L = m["L"]
    x = np.array(m["pos"], np.float64)
    faces = [1.0, 2.0, 3.0, 0.0, -0.0, 4.0, np.nextafter(4.0, 5.0), -1e-300, np.nextafter(1.0, 0.0),
             np.nextafter(4.0, 0.0), np.nextafter(2.0, 3.0)]
    used = set()
    for axis in range(3):
        for v in faces:
            d = np.abs(((x[:, axis] - v + 0.5 * L) % L) - 0.5 * L)
            d[list(used)] = np.inf
            i = int(np.argmin(d))
            assert d[i] < 0.01
            used.add(i)
            x[i, axis] = v
    s = md.System(m, precision=precision, rc=0.9, skin=0.1)
    s.set_state(x, m["vel"])
    M = s.info["cells_per_side"]
    assert M == 4
    co, cs, pm = s.bins()
    oc, ocs, opm = oracle.bin_atoms(_ingested(x, L, precision), L, M)
    assert np.array_equal(co, oc)
    assert np.array_equal(cs, ocs)
    assert np.array_equal(pm, opm)
    s.close()


@pytest.mark.parametrize("precision", [md.MD_MIXED, md.MD_PLAIN_FP32])
def test_neighbour_pairs(precision):
    m = chaingen.melt(20, seed=5, L=4.6)
    s = md.System(m, precision=precision)
    x, _ = _uploaded(m, precision)
    L = m["L"]
    cnt, ent = s.neighbors()
    listed = set()
    for i in range(len(x)):
        for j in ent[i, :cnt[i]]:
            listed.add((i, int(j)))
    # symmetric full list
    assert all((j, i) in listed for (i, j) in listed)
    tr = cKDTree(np.mod(x, L), boxsize=L)
    pairs = tr.query_pairs(1.1 + 1e-5, output_type="ndarray")
    d = x[pairs[:, 0]] - x[pairs[:, 1]]
    d -= L * np.round(d / L)
    r = np.linalg.norm(d, axis=1)
    same = pairs[:, 0] // 150 == pairs[:, 1] // 150
    excl = same & (np.abs(pairs[:, 0] - pairs[:, 1]) <= 2)
    must = {(int(a), int(b)) for (a, b), rr, e in zip(pairs, r, excl) if rr < 1.1 - 1e-5 and not e}
    may = {(int(a), int(b)) for (a, b), e in zip(pairs, excl) if not e}
    half = {(min(i, j), max(i, j)) for (i, j) in listed}
    assert must <= half
    assert half <= may
    s.close()


@pytest.mark.parametrize("precision", [md.MD_MIXED, md.MD_PLAIN_FP32])
@pytest.mark.parametrize("n_chains,seed,L", [(10, 1, None), (2, 3, 3.4), (40, 9, None)])
def test_forces_match_oracle(precision, n_chains, seed, L):
    m = chaingen.melt(n_chains, seed=seed, L=L)
    s = md.System(m, precision=precision)
    x, _ = _uploaded(m, precision)
    f = s.forces()
    f_orc, _, _ = _oracle(m).forces(x)
    check_forces(f, f_orc, x, m["L"])
    s.close()


@pytest.mark.parametrize("precision", [md.MD_MIXED, md.MD_PLAIN_FP32])
def test_energies_match_oracle(precision):
    m = chaingen.melt(10, seed=4)
    s = md.System(m, precision=precision)
    x, v = _uploaded(m, precision)
    e = s.energy()[0]
    ref = _oracle(m)
    _, en, vir = ref.forces(x)
    ke = ref.kinetic(v)
    for got, want in [(e["lj"], en[0]), (e["lj_shifted"], en[1]), (e["bond"], en[2]), (e["angle"], en[3]),
                      (e["dihedral"], en[4]), (e["kinetic"], ke)]:
        assert got == pytest.approx(want, rel=1e-5, abs=1e-3)
    assert np.allclose(e["virial"], vir, rtol=1e-4, atol=1e-2 * np.abs(vir).max())
    s.close()


@pytest.mark.parametrize("precision,tol", [(md.MD_MIXED, 1e-5), (md.MD_PLAIN_FP32, 2e-4)])
def test_short_trajectory_matches_oracle(precision, tol):
    m = chaingen.melt(4, seed=12, L=3.6, T=300.0)
    s = md.System(m, precision=precision, rebin_every=5)
    x0, v0 = _uploaded(m, precision)
    s.step(50)
    x, v, img = s.state()
    xo, vo, _, _, _ = _oracle(m).run(x0, v0, 0.001, 50, sample_every=0)
    d = x + img * m["L"] - xo
    assert np.abs(d).max() < tol
    s.close()


def test_mixed_form_is_deterministic():
    m = chaingen.melt(12, seed=2)
    runs = []
    for _ in range(2):
        s = md.System(m, precision=md.MD_MIXED, rebin_every=2)
        s.step(100)
        runs.append((s.state(), s.forces()))
        s.close()
    (xa, va, ia), fa = runs[0]
    (xb, vb, ib), fb = runs[1]
    assert np.array_equal(xa, xb) and np.array_equal(va, vb) and np.array_equal(ia, ib)
    assert np.array_equal(fa, fb)


def test_net_force_vanishes():
    """Newton's third law: the LJ kernel evaluates each pair once and adds
    +f to i and -f to j, so the net force is zero up to the roundings the
    sums make.  Bound derived from the arithmetic: FP32 summation (the i side
    sums in list order, the j side per list entry, ~1e-7 relative) plus the
    rounding of each partial sum to the 2^-13 kJ/mol/nm accumulators (about
    40 per atom, each uniform in +-2^-14: 6 standard deviations of their sum)."""
    m = chaingen.melt(10, seed=6)
    s = md.System(m, precision=md.MD_MIXED)
    f = s.forces()
    n = len(f)
    scale = np.sqrt(np.mean(np.sum(f ** 2, axis=1)))
    q = 2.0 ** -13
    bound = 1e-6 * scale * np.sqrt(n) + 6.0 * q * np.sqrt(40.0 * n / 12.0)
    assert np.abs(f.sum(0)).max() < bound
    s.close()


def test_pairwise_exact_lj_forces_sum_to_zero_and_match_oracle():
    """With lj_pair_exact every LJ pair force is converted once and added to
    i and subtracted from j as the same integer, so the LJ forces sum to
    exactly zero over the system (bonded terms switched off so that the
    total force is the LJ force), and they still match the FP64 oracle.
    A relaxed melt: its close 1-4 pairs push forces past 512 kJ/mol/nm, the
    range of a single-FFMA rounding, so the two-part rounding is exercised."""
    m, _ = _oracle_relaxed(12, seed=61)
    p = dict(md.default_params())
    p.update(kb=0.0, ka=0.0, kphi=0.0)
    po = oracle.default_params()
    po.update(kb=0.0, ka=0.0, kphi=0.0)
    s = md.System(m, precision=md.MD_MIXED, params=p, lj_pair_exact=True)
    f = s.forces()
    for a in range(3):
        assert math.fsum(f[:, a]) == 0.0
    x, _ = _uploaded(m)
    f_orc, _, _ = _oracle(m, params=po).forces(x)
    assert np.max(np.abs(f_orc)) > 512.0   # beyond the range of a single FFMA rounding
    check_forces(f, f_orc, x, m["L"])
    # the same system without the option: same forces to FP32 rounding,
    # and the trajectory runs
    q = md.System(m, precision=md.MD_MIXED, params=p)
    g = q.forces()
    assert np.sqrt(np.sum((f - g) ** 2) / np.sum(g ** 2)) < FORCE_TOL
    s.step(20)
    q.close()
    s.close()


def test_thermostat_temperature_series_matches_oracle():
    m = chaingen.melt(4, seed=8, L=3.6, T=450.0)
    s = md.System(m, precision=md.MD_MIXED, thermostat=md.MD_VRESCALE, T_target=300.0, tau_t=0.02)
    x0, v0 = _uploaded(m)
    temps = [s.energy()[0]["temperature"]]
    for _ in range(30):
        s.step(1)
        temps.append(s.energy()[0]["temperature"])
    _, _, _, smp, _ = _oracle(m).run(x0, v0, 0.001, 30, thermostat=True, T0=300.0, tau=0.02)
    assert np.allclose(temps, smp[:, 7], rtol=2e-5)
    assert temps[-1] < temps[0]
    s.close()


def test_replicas_equal_separate_runs_and_oracle():
    melts = [chaingen.melt(c, seed=40 + c) for c in (10, 25, 12)]
    both = md.System(melts, precision=md.MD_MIXED, rebin_every=4)
    fb = both.forces()
    off = 0
    for m in melts:
        alone = md.System(m, precision=md.MD_MIXED)
        fa = alone.forces()
        n = len(m["pos"])
        assert np.array_equal(fb[off:off + n], fa)
        x, _ = _uploaded(m)
        check_forces(fa, _oracle(m).forces(x)[0], x, m["L"])
        alone.close()
        off += n
    both.step(20)
    xb, _, _ = both.state()
    off = 0
    for m in melts:
        alone = md.System(m, precision=md.MD_MIXED, rebin_every=4)
        alone.step(20)
        xa, _, _ = alone.state()
        assert np.array_equal(xb[off:off + len(xa)], xa)
        off += len(xa)
        alone.close()
    both.close()


def test_thermostatted_replicas_equal_separate_runs_including_energies():
    # Each replica's kinetic-energy sum (which sets its rescaling factor) and
    # its energy/virial sums have an order fixed by the replica's own size, so
    # a replica stepped with others gives the same bits as alone.  The
    # 400-chain replica has 11^3 cells: its energy sums take two slices.
    melts = [chaingen.melt(c, seed=70 + c) for c in (10, 400, 25)]
    T0 = [300.0, 450.0, 380.0]
    kw = dict(precision=md.MD_MIXED, thermostat=md.MD_VRESCALE, tau_t=0.05, rebin_every=5)
    both = md.System(melts, T_target=T0, **kw)
    both.step(30)
    xb, vb, _ = both.state()
    eb = both.energy()
    off = 0
    for m, T, e in zip(melts, T0, eb):
        alone = md.System(m, T_target=T, **kw)
        alone.step(30)
        xa, va, _ = alone.state()
        n = len(xa)
        assert np.array_equal(xb[off:off + n], xa) and np.array_equal(vb[off:off + n], va)
        ea = alone.energy()[0]
        for k in ("lj", "lj_shifted", "bond", "angle", "dihedral", "kinetic", "temperature"):
            assert e[k] == ea[k], k
        assert np.array_equal(np.asarray(e["virial"]), np.asarray(ea["virial"]))
        off += n
        alone.close()
    both.close()


def test_energy_call_leaves_forces_and_trajectory_unchanged():
    # md_energy recomputes the forces with the energy-form kernels; they must
    # be the bits the force-only kernels give, or reading energies would
    # perturb the dynamics
    m = chaingen.melt(30, seed=8)
    a = md.System(m, precision=md.MD_MIXED, rebin_every=5)
    b = md.System(m, precision=md.MD_MIXED, rebin_every=5)
    for _ in range(3):
        a.step(7)
        b.step(7)
        f = a.forces()
        a.energy()
        assert np.array_equal(a.forces(), f)
    assert np.array_equal(a.state()[0], b.state()[0]) and np.array_equal(a.state()[1], b.state()[1])
    a.close()
    b.close()


@pytest.mark.parametrize("precision,tol_x,tol_t", [(md.MD_MIXED, 1e-5, 2e-5), (md.MD_PLAIN_FP32, 2e-4, 2e-4)])
def test_nose_hoover_matches_oracle(precision, tol_x, tol_t):
    """The paper's NVT ensemble (Leap-Frog + Nose-Hoover + centre-of-mass
    removal), a 450 K melt coupled to 300 K: temperature and xi after every
    step of 30, and positions after 50 steps, against the oracle's run."""
    m = chaingen.melt(4, seed=12, L=3.6, T=450.0)
    s = md.System(m, precision=precision, thermostat=md.MD_NOSE_HOOVER, T_target=300.0, tau_t=0.1,
                  rebin_every=5)
    x0, v0 = _uploaded(m, precision)
    temps, xis = [s.energy()[0]["temperature"]], [s.thermostat_xi()[0]]
    for _ in range(30):
        s.step(1)
        temps.append(s.energy()[0]["temperature"])
        xis.append(s.thermostat_xi()[0])
    s.step(20)
    x, _, img = s.state()
    ref = _oracle(m)
    _, _, _, smp, _ = ref.run_nh(x0, v0, 0.001, 30, T0=300.0, tau=0.1)
    assert np.allclose(temps, smp[:, 7], rtol=tol_t)
    assert np.allclose(xis, smp[:, 8], rtol=10 * tol_t, atol=10 * tol_t * np.abs(smp[:, 8]).max())
    assert abs(xis[-1]) > 0.1                       # the coupling has acted
    xo, _, _, _, _ = ref.run_nh(x0, v0, 0.001, 50, T0=300.0, tau=0.1, sample_every=0)
    d = x + img * m["L"] - xo
    d -= m["L"] * np.round(d / m["L"])
    assert np.abs(d).max() < tol_x, np.abs(d).max()
    s.close()


def test_nose_hoover_replicas_equal_separate_runs():
    melts = [chaingen.melt(c, seed=80 + c, T=420.0) for c in (10, 15, 12)]
    T0 = [300.0, 500.0, 380.0]
    kw = dict(precision=md.MD_MIXED, thermostat=md.MD_NOSE_HOOVER, tau_t=0.1, rebin_every=5)
    both = md.System(melts, T_target=T0, **kw)
    both.step(23)
    xb, vb, _ = both.state()
    xib = both.thermostat_xi()
    off = 0
    for k, (m, T) in enumerate(zip(melts, T0)):
        alone = md.System(m, T_target=T, **kw)
        alone.step(23)
        xa, va, _ = alone.state()
        n = len(xa)
        assert np.array_equal(xb[off:off + n], xa) and np.array_equal(vb[off:off + n], va)
        assert xib[k] == alone.thermostat_xi()[0]
        off += n
        alone.close()
    both.close()


def test_nose_hoover_removes_centre_of_mass_drift():
    m = chaingen.melt(6, seed=13, L=3.6, T=350.0)
    masses = np.asarray(m["masses"])[:, None]
    s = md.System(m, precision=md.MD_MIXED, thermostat=md.MD_NOSE_HOOVER, T_target=350.0, tau_t=0.2)
    s.set_state(m["pos"], m["vel"] + np.array([0.2, -0.1, 0.3]))
    s.step(2)
    _, v, _ = s.state()
    # left: the net force (zero only to FP32 rounding) over the closing half step
    assert np.abs((masses * v).sum(0)).max() < 1e-7 * np.abs(masses * v).sum()
    s.close()


@pytest.mark.parametrize("sites", [4, 7, 150, 511])
def test_short_chains_and_rebin_every_step(sites):
    n_chains = max(1, 1500 // sites)
    m = chaingen.melt(n_chains, sites=sites, seed=3, L=3.6)
    params = oracle.default_params()
    s = md.System(m, precision=md.MD_MIXED, rebin_every=1)
    x, v = _uploaded(m)
    ref = oracle.System(oracle.chain_topology(sites), n_chains, m["L"], use_cells=False)
    check_forces(s.forces(), ref.forces(x)[0], x, m["L"], params)
    # after 7 steps (a rebin before every step): the forces at the end of the
    # oracle's own 7-step run from the same state
    s.step(7)
    xo, _, fo, _, _ = ref.run(x, v, 0.001, 7, sample_every=0)
    check_forces(s.forces(), fo, xo, m["L"], params)
    s.close()


def _two_chains_from_one_walk(sites, seed, L):
    """Two chains whose ends nearly touch: one walk of 2 * sites + 2 sites
    from the generator, with its two middle sites dropped, so that the last
    site of chain 0 and the first site of chain 1 were 1-4 neighbours of the
    walk (0.25 - 0.39 nm apart, inside r_c) but are not bonded here."""
    w = chaingen.melt(1, sites=2 * sites + 2, seed=seed, L=L)
    keep = np.r_[0:sites, sites + 2:2 * sites + 2]
    return dict(pos=w["pos"][keep], vel=w["vel"][keep], L=w["L"], n_chains=2, sites=sites,
                types=np.tile(chaingen.site_types(sites), 2), masses=np.tile(chaingen.site_masses(sites), 2),
                T=w["T"], seed=seed)


@pytest.mark.parametrize("precision", [md.MD_MIXED, md.MD_PLAIN_FP32])
@pytest.mark.parametrize("sites", [150, 511])
def test_last_site_and_next_chains_first_site_interact(sites, precision):
    """The last site of chain c and the first site of chain c + 1 are not
    bonded, so their LJ pair counts (Sec. 3.1 excludes only 1-2 and 1-3
    pairs).  They are placed inside r_c, and the forces must match the
    oracle's, including for 511-site chains, whose site fields sit closest
    in the packed tags."""
    m = _two_chains_from_one_walk(sites, seed=17, L=4.0 if sites == 150 else 5.0)
    s = md.System(m, precision=precision)
    x, _ = _uploaded(m, precision)
    d = x[sites - 1] - x[sites]
    d -= m["L"] * np.round(d / m["L"])
    r = np.linalg.norm(d)
    assert 0.2 < r < 0.45
    ref = oracle.System(oracle.chain_topology(sites), 2, m["L"], use_cells=False)
    f_orc = ref.forces(x)[0]
    # the pair's own force is far above the per-atom bar, so a false
    # exclusion could not pass the check below
    p = oracle.default_params()
    sig, eps = p["sigma"][1], p["eps"][1]
    f_pair = abs(24 * eps / r * (2 * (sig / r) ** 12 - (sig / r) ** 6))
    assert f_pair > 100 * ATOM_TOL * np.sqrt(np.mean(np.sum(f_orc ** 2, axis=1)))
    check_forces(s.forces(), f_orc, x, m["L"])
    s.close()


def test_displacement_beyond_half_skin_triggers_an_early_rebin():
    """A skin of 0.002 nm with the list rebuilt only every 10 steps: atoms
    move more than skin/2 within a few steps.  The displacement check then
    rebuilds the bins and list before that step's forces (counted by
    md_early_rebins), the run continues, and the forces after 10 and after
    17 steps (a remainder block) match the oracle's own run from the same
    state (mixed form: its trajectory follows the oracle's to ~1e-8 nm)."""
    m = chaingen.melt(10, seed=1, L=3.6)
    s = md.System(m, precision=md.MD_MIXED, skin=0.002, rebin_every=10)
    x, v = _uploaded(m)
    ref = oracle.System(oracle.chain_topology(150), 10, m["L"], use_cells=False)
    s.step(10)
    assert s.early_rebins() > 0
    xo, vo, fo, _, _ = ref.run(x, v, 0.001, 10, sample_every=0)
    check_forces(s.forces(), fo, xo, m["L"])
    s.step(7)
    xo, vo, fo, _, _ = ref.run(xo, vo, 0.001, 7, sample_every=0)
    check_forces(s.forces(), fo, xo, m["L"])
    s.close()


def test_displacement_error_policy_reports_instead():
    """With MD_DISP_ERROR the same run stops with MD_EUNSTABLE (round-trip of
    the policy, and the graphs then hold no conditional node)."""
    m = chaingen.melt(10, seed=1, L=3.6)
    s = md.System(m, precision=md.MD_MIXED, skin=0.002, rebin_every=10, displacement=md.MD_DISP_ERROR)
    with pytest.raises(md.MDError) as e:
        s.step(10)
    assert e.value.code == md.MD_EUNSTABLE
    assert s.early_rebins() == 0
    s.close()


def test_workspace_and_library_allocation_agree():
    m = chaingen.melt(10, seed=13)
    a = md.System(m, use_torch_memory=True, rebin_every=3)
    b = md.System(m, use_torch_memory=False, rebin_every=3)
    a.step(15); b.step(15)
    assert np.array_equal(a.state()[0], b.state()[0])
    a.close(); b.close()


def _check_sampled(f, x, sel, f_orc, L):
    """Sampled atoms against the oracle's all-atom sums, with the same bar as
    check_forces (an atom with a pair within 2e-6 nm of r_c gets |F(r_c)| per
    such pair on top)."""
    scale = np.sqrt(np.mean(np.sum(f ** 2, axis=1)))
    tr = cKDTree(np.mod(x, L), boxsize=L)
    amb = np.zeros(len(sel), int)
    for k, i in enumerate(sel):
        for j in tr.query_ball_point(np.mod(x[i], L), 1.0 + 2e-6):
            d = x[i] - x[j]
            d -= L * np.round(d / L)
            amb[k] += abs(np.linalg.norm(d) - 1.0) < 2e-6
    p = oracle.default_params()
    f_rc = abs(24 * max(p["eps"]) * (2 * max(p["sigma"]) ** 12 - max(p["sigma"]) ** 6))
    err = np.abs(f[sel] - f_orc).max(axis=1)
    assert np.all(err <= ATOM_TOL * scale + amb * 1.01 * f_rc), (err / scale).max()
    clean = amb == 0
    rel = np.sqrt(np.sum((f[sel] - f_orc)[clean] ** 2) / np.sum(f_orc[clean] ** 2))
    assert rel <= FORCE_TOL, rel


@pytest.mark.parametrize("precision", [md.MD_MIXED, md.MD_PLAIN_FP32])
def test_full_size_sampled_forces(precision):
    """1.5M sites (10,000 chains, L = 35.68 nm), as benchmarked: forces of
    sampled atoms against the oracle's all-atom sums."""
    m = chaingen.melt(10000, seed=3)
    s = md.System(m, precision=precision)
    x, _ = _uploaded(m, precision)
    f = s.forces()
    rng = np.random.default_rng(0)
    sel = np.sort(rng.choice(len(x), 48, replace=False))
    ref = _oracle(m)
    f_orc = ref.lj_atoms(x, sel) + ref.bonded(x)[0][sel]
    _check_sampled(f, x, sel, f_orc, m["L"])
    s.close()


def test_batched_replicas_full_size_sampled_forces():
    """64 replicas of 20..400 chains (chain counts log-uniform, seed 4;
    ~1.07M sites) in one system, in the launch configuration the benchmark
    tunes to (skin 0.12 nm, list every 12 steps, 256 threads, grid schedule),
    thermostatted at each replica's T0: sampled forces of every replica against
    the oracle's all-atom sums at the generator's state.  (Straight from the
    generator, atoms at the hottest contacts move more than skin/2 within 12
    steps; the benchmark equilibrates first.)"""
    melts = chaingen.replicas(64, seed=4)
    T0 = [m["T"] for m in melts]
    s = md.System(melts, precision=md.MD_MIXED, thermostat=md.MD_VRESCALE, T_target=T0, tau_t=0.1, skin=0.12,
                  rebin_every=12, lj_block=256, schedule=md.MD_SCHED_GRID)
    rng = np.random.default_rng(4)
    f = s.forces()
    off = 0
    for m in melts:
        n = len(m["pos"])
        xr, _ = _uploaded(m)
        fr = f[off:off + n]
        sel = np.sort(rng.choice(n, 3, replace=False))
        ref = _oracle(m)
        _check_sampled(fr, xr, sel, ref.lj_atoms(xr, sel) + ref.bonded(xr)[0][sel], m["L"])
        off += n
    assert off == len(f)
    s.close()


def test_full_size_persistent_schedule_gives_the_same_bits():
    """1.5M sites as benchmarked: the persistent schedule (a fixed grid whose
    blocks take regions from a device counter) gives the same forces and
    energies, bit for bit, as one block per region."""
    m = chaingen.melt(10000, seed=3)
    out = []
    for sch in (md.MD_SCHED_GRID, md.MD_SCHED_PERSISTENT):
        s = md.System(m, precision=md.MD_MIXED, schedule=sch)
        out.append((s.forces(), s.energy()[0]))
        s.close()
    assert np.array_equal(out[0][0], out[1][0])
    for k in ("lj", "lj_shifted", "bond", "angle", "dihedral"):
        assert out[0][1][k] == out[1][1][k], k
    assert out[0][1]["virial"] == out[1][1]["virial"]


@pytest.mark.parametrize("precision", [md.MD_MIXED, md.MD_PLAIN_FP32])
def test_set_state_round_trip_and_non_finite_input(precision):
    """md_set_state copies the arrays to the GPU as they are and wraps them
    there: positions come back wrapped into [0, L) with image counters 0,
    velocities unchanged; a NaN is reported as MD_EINVAL and a good state
    afterwards works again."""
    m = chaingen.melt(6, seed=31, L=3.6)
    L = m["L"]
    s = md.System(m, precision=precision)
    rng = np.random.default_rng(3)
    x_in = m["pos"] + L * rng.integers(-3, 4, size=m["pos"].shape)     # any image
    v_in = m["vel"] * 0.5
    s.set_state(x_in, v_in)
    x, v, img = s.state()
    want = x_in - L * np.floor(x_in / L)
    tol = 1e-14 * L if precision == md.MD_MIXED else 4e-7 * L    # the GPU may fuse L * floor() into the subtraction
    assert np.abs(x - want).max() <= tol
    assert np.abs(v - v_in).max() <= (0.0 if precision == md.MD_MIXED else 1e-6 * np.abs(v_in).max())
    assert not img.any()
    bad = v_in.copy()
    bad[17, 1] = np.nan
    with pytest.raises(md.MDError) as e:
        s.set_state(x_in, bad)
    assert e.value.code == md.MD_EINVAL
    s.set_state(m["pos"], m["vel"])
    f = s.forces()
    xu, _ = _uploaded(m, precision)
    f_orc, _, _ = _oracle(m).forces(xu)
    check_forces(f, f_orc, xu, L)
    s.close()


def test_first_cycle_after_set_state_skips_the_rebin_with_the_same_bits():
    """After md_set_state the bins, list and forces belong to the current
    positions, so the first cycle runs without its leading rebin; with
    profiling on the full cycle runs.  Both give the same trajectory."""
    m = chaingen.melt(10, seed=33)
    out = []
    for prof in (False, True):
        s = md.System(m, precision=md.MD_MIXED)
        s.set_state(m["pos"], m["vel"])
        md.md_profile_enable(s.h, prof)
        s.step(25)
        out.append(s.state())
        s.close()
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(a, b)


def test_schedules_and_block_shapes_agree():
    """The persistent schedule gives the same bits as one block per region,
    and so does any block size (a cluster's forces do not depend on which warp
    of which block computes them).  Regions of 2 x 2 and 3 x 3 cells stage
    positions in different frames, so those two agree to FP32 rounding."""
    m = chaingen.melt(30, seed=23)
    runs = {}
    cases = ((3, 384, md.MD_SCHED_GRID), (3, 384, md.MD_SCHED_PERSISTENT), (3, 256, md.MD_SCHED_GRID),
             (3, 128, md.MD_SCHED_PERSISTENT), (2, 256, md.MD_SCHED_GRID), (2, 256, md.MD_SCHED_PERSISTENT),
             (2, 128, md.MD_SCHED_GRID))
    f0 = {}
    for reg, blk, sch in cases:
        s = md.System(m, precision=md.MD_MIXED, rebin_every=4, lj_block=blk, schedule=sch, lj_region=reg)
        f0[reg] = s.forces()
        s.step(12)
        runs[(reg, blk, sch)] = (s.forces(), s.state()[0], s.energy()[0])
        s.close()
    for key in cases[1:]:
        ref = runs[(key[0],) + ((384, md.MD_SCHED_GRID) if key[0] == 3 else (256, md.MD_SCHED_GRID))]
        f, x, e = runs[key]
        assert np.array_equal(f, ref[0]) and np.array_equal(x, ref[1]) and e == ref[2], key
    # same state: forces to FP32 rounding (the relative RMS bound of the
    # parity tests); after 12 steps the positions
    rel = np.sqrt(np.sum((f0[3] - f0[2]) ** 2) / np.sum(f0[2] ** 2))
    assert rel <= FORCE_TOL, rel
    x3, x2 = runs[(3, 384, md.MD_SCHED_GRID)][1], runs[(2, 256, md.MD_SCHED_GRID)][1]
    assert np.abs(x3 - x2).max() < 1e-6


@pytest.mark.parametrize("lanes", [16, 32])
def test_lanes_per_cluster_give_the_oracle_forces(lanes):
    """16 or 32 lanes per cluster split a cluster's list into other partial
    sums (FP32 rounding apart from 8 lanes) and reduce them over more levels
    of the lane tree: forces against the oracle, and a 12-step trajectory
    within 1e-6 nm of the 8-lane one."""
    m = chaingen.melt(30, seed=23)
    x, _ = _uploaded(m)
    f_orc = _oracle(m).forces(x)[0]
    s = md.System(m, precision=md.MD_MIXED, rebin_every=4, lj_lanes=lanes)
    r = md.System(m, precision=md.MD_MIXED, rebin_every=4, lj_lanes=8)
    check_forces(s.forces(), f_orc, x, m["L"])
    s.step(12)
    r.step(12)
    assert np.abs(s.state()[0] - r.state()[0]).max() < 1e-6
    s.close()
    r.close()


def test_autotune_picks_a_working_setting_and_caches_it(tmp_path):
    m = chaingen.melt(20, seed=29)
    cache = str(tmp_path / "tune.txt")
    s = md.System(m, precision=md.MD_MIXED, autotune=True, tune_cycles=1, tune_cache=cache)
    t = s.tuning
    assert t["from_cache"] == 0 and t["lj_block"] in (128, 256, 384) and t["schedule"] in (0, 1)
    assert t["lj_region"] in (2, 3) and t["lj_lanes"] in (8, 16, 32)
    assert t["skin"] > 0 and t["rebin_every"] >= 1 and t["us_per_step"] > 0
    s.step(2 * s.rebin_every)
    s.close()
    s2 = md.System(m, precision=md.MD_MIXED, autotune=True, tune_cycles=1, tune_cache=cache)
    assert s2.tuning["from_cache"] == 1 and s2.tuning["skin"] == t["skin"]
    assert s2.tuning["lj_region"] == t["lj_region"] and s2.tuning["lj_block"] == t["lj_block"]
    s2.close()


def _oracle_relaxed(n_chains, seed, L=None, T=500.0, rounds=3, steps=300):
    """Generator melt relaxed by the oracle (thermostat rounds with Maxwell
    redraws), so that long GPU runs start from the same well-behaved state."""
    m = chaingen.melt(n_chains, seed=seed, L=L, T=T)
    s = oracle.System(oracle.chain_topology(m["sites"]), n_chains, m["L"], use_cells=True)
    x, v = chaingen.unwrapped(m), m["vel"]
    for r in range(rounds):
        x, v, _, _, _ = s.run(x, v, 0.001, steps, thermostat=True, T0=T, tau=0.05, sample_every=0)
        v = chaingen.maxwell(m["masses"], T, seed, stream=100 + r)
    x, v, _, _, _ = s.run(x, v, 0.001, steps, thermostat=True, T0=T, tau=0.05, sample_every=0)
    return dict(m, pos=x, vel=v), s


@pytest.mark.parametrize("precision", [md.MD_MIXED, md.MD_PLAIN_FP32])
def test_config1_small_box_1000_nve_steps(precision):
    """Config 1: 10 chains (1,500 sites) in L = 3.568 nm (M = 3: the 27 cells
    are the whole box), 1,000 NVE steps at 500 K.  Trajectories part by chaos
    after a few hundred steps, so the run is compared through what it must
    share with the oracle's: the total energy stays within the oracle's own
    excursion (x3 and a 1 kJ/mol floor; plain FP32 within 10 kJ/mol), and the
    mean potential energy over the run agrees within 2 %."""
    m, ref = _oracle_relaxed(10, seed=41, L=3.568)
    s = md.System(m, precision=precision)
    assert s.info["cells_per_side"] == 3
    e_gpu, u_gpu = [], []
    for k in range(21):
        e = s.energy()[0]
        e_gpu.append(e["total"]); u_gpu.append(e["total"] - e["kinetic"])
        if k < 20:
            s.step(50)
    s.close()
    _, _, _, smp, _ = ref.run(m["pos"], m["vel"], 0.001, 1000, sample_every=50)
    e_orc = smp[:, 2] + smp[:, 3] + smp[:, 4] + smp[:, 5] + smp[:, 6]
    u_orc = e_orc - smp[:, 6]
    assert abs(e_gpu[0] - e_orc[0]) < 1e-4 * abs(e_orc[0]) + 1e-2
    exc_orc = np.abs(e_orc - e_orc[0]).max()
    exc_gpu = np.abs(np.array(e_gpu) - e_gpu[0]).max()
    floor = 1.0 if precision == md.MD_MIXED else 10.0
    assert exc_gpu <= 3.0 * exc_orc + floor, (exc_gpu, exc_orc)
    assert abs(np.mean(u_gpu) - np.mean(u_orc)) <= 0.02 * abs(np.mean(u_orc)) + 5.0


def test_config2_quench_plain_fp32():
    """Config 2: 1,000 chains (150,000 sites, L = 16.56 nm) in plain FP32,
    with the weak-coupling thermostat set to 300 K (the quench): sampled
    forces at the start against the oracle's all-atom sums, and the
    temperature series of the first 30 steps against the oracle's run."""
    m = chaingen.melt(1000, seed=2, T=500.0)
    assert abs(m["L"] - 16.56) < 0.01
    # straight from the generator: its hottest contacts move atoms faster than
    # skin/2 per 10 steps with the default 0.1 nm skin, so a wider skin here
    # (the pair set inside r_c does not depend on it)
    s = md.System(m, precision=md.MD_PLAIN_FP32, thermostat=md.MD_VRESCALE, T_target=300.0, tau_t=0.1,
                  skin=0.25, rebin_every=10)
    x0, v0 = _uploaded(m, md.MD_PLAIN_FP32)
    f = s.forces()
    rng = np.random.default_rng(2)
    sel = np.sort(rng.choice(len(x0), 64, replace=False))
    ref = _oracle(m)
    _check_sampled(f, x0, sel, ref.lj_atoms(x0, sel) + ref.bonded(x0)[0][sel], m["L"])
    temps = [s.energy()[0]["temperature"]]
    for _ in range(3):
        s.step(10)
        temps.append(s.energy()[0]["temperature"])
    s.close()
    _, _, _, smp, _ = ref.run(x0, v0, 0.001, 30, thermostat=True, T0=300.0, tau=0.1, sample_every=10)
    # (from the generator's hot start the contacts heat the melt faster than
    # the 0.1 ps coupling removes it over 30 steps; the oracle does the same)
    assert np.allclose(temps, smp[:, 7], rtol=2e-4), (temps, smp[:, 7])


def test_bounded_device_wait_gives_up_and_reports_timeout():
    """A device wait on an mbarrier that nothing arrives on gives up after its
    round limit and reports MD_ETIMEOUT; the context stays usable."""
    assert md.md_wait_selftest(1000) == md.MD_ETIMEOUT
    assert "gave up" in md.md_last_error(None)
    m = chaingen.melt(2, seed=7, L=3.4)
    s = md.System(m, precision=md.MD_MIXED)
    s.step(10)
    assert np.isfinite(s.forces()).all()
    s.close()


def test_list_capacity_overflow_is_reported():
    """A neighbour list capacity far below the ~184 entries an atom needs is
    reported as MD_EOVERFLOW (list writes stop at the capacity)."""
    m = chaingen.melt(10, seed=34)
    with pytest.raises(md.MDError) as e:
        md.System(m, precision=md.MD_MIXED, nbr_capacity=16)
    assert e.value.code == md.MD_EOVERFLOW


def _with_contact(m, gap):
    """Site 10 of chain 1 placed `gap` nm from site 10 of chain 0 (non-bonded)."""
    x = m["pos"].copy()
    x[150 + 10] = x[10] + np.array([gap, 0.0, 0.0])
    return dict(m, pos=x)


def test_fixed_point_range_is_reported():
    """A force part beyond 2^18 kJ/mol/nm (two sites 0.05 nm apart) cannot be
    held in the 2^-32 fixed point: the mixed form reports MD_EOVERFLOW."""
    m = _with_contact(chaingen.melt(4, seed=35, L=3.6), 0.05)
    with pytest.raises(md.MDError) as e:
        md.System(m, precision=md.MD_MIXED)
    assert e.value.code == md.MD_EOVERFLOW


def test_non_finite_state_is_reported():
    """Two sites on the same spot give a non-finite FP32 pair force: the LJ
    kernel's check of every converted sum reports it (MD_EUNSTABLE) as soon as
    the forces are computed, at creation."""
    m = _with_contact(chaingen.melt(4, seed=36, L=3.6), 0.0)
    with pytest.raises(md.MDError) as e:
        md.System(m, precision=md.MD_PLAIN_FP32)
    assert e.value.code == md.MD_EUNSTABLE


@pytest.mark.parametrize("precision", [md.MD_MIXED, md.MD_PLAIN_FP32])
def test_chain_observables_after_steps_and_rebins(precision):
    """The observables of a stepped system (20 steps, a rebin every 5, atoms
    wrapped across faces on the way) against the oracle's definitions on the
    oracle's own 20-step trajectory from the same state (positions agree to
    ~1e-5 nm after 20 steps)."""
    from oracle import observables as ob
    m = chaingen.melt(12, seed=43, L=3.6)
    s = md.System(m, precision=md.MD_MIXED if precision == md.MD_MIXED else md.MD_PLAIN_FP32, rebin_every=5)
    s.step(20)
    got = s.observables()
    x, v = _uploaded(m, precision)
    ref = oracle.System(oracle.chain_topology(m["sites"]), m["n_chains"], m["L"], use_cells=False)
    xo, _, _, _, _ = ref.run(chaingen.unwrapped(dict(m, pos=x)), v, 0.001, 20, sample_every=0)
    ree = ob.end_to_end(xo, m["sites"])
    rg2 = ob.radius_of_gyration_sq(xo, m["sites"], m["masses"])
    tol = 1e-4 if precision == md.MD_MIXED else 1e-3
    assert np.allclose(got["r_ee"], ree, rtol=tol, atol=tol)
    assert np.allclose(got["rg2"], rg2, rtol=tol)
    phi = ob.dihedral_angles(xo, m["sites"])
    want = np.mean(np.abs(phi) > 120.0)
    near = np.sum(np.abs(np.abs(phi) - 120.0) < 0.05)   # states the two trajectories may split
    assert abs(got["trans_fraction"][0] - want) <= near / phi.size + 1e-15
    s.close()


def test_all_trans_chains_have_trans_fraction_one():
    """Planar zigzag chains (every dihedral at 180 deg, bond 0.153 nm, angle
    109.47 deg) in two replicas: the trans fraction is exactly 1, and R_ee is
    the zigzag's closed form (sites - 1) b sin(theta / 2) along the chain."""
    b, th = 0.153, np.arccos(-1.0 / 3.0)
    sites, n_chains = 7, 3
    melts = []
    for r, L in enumerate((4.0, 4.4)):
        pos = []
        for c in range(n_chains):
            base = np.array([0.5, 0.7 + 1.2 * c, 0.9 + 0.3 * r])
            for k in range(sites):
                pos.append(base + [k * b * np.sin(th / 2), (k % 2) * b * np.cos(th / 2), 0.0])
        pos = np.array(pos)
        rng = np.random.default_rng(r)
        melts.append(dict(pos=pos, vel=0.1 * rng.normal(size=pos.shape), L=L, n_chains=n_chains, sites=sites,
                          types=np.tile(chaingen.site_types(sites), n_chains),
                          masses=np.tile(chaingen.site_masses(sites), n_chains), T=300.0))
    s = md.System(melts, precision=md.MD_MIXED)
    got = s.observables()
    assert list(got["trans_fraction"]) == [1.0, 1.0]
    want = (sites - 1) * b * np.sin(th / 2)
    assert np.allclose(got["r_ee"][:, 0], want, rtol=1e-12)
    s.close()


@pytest.mark.parametrize("precision", [md.MD_MIXED, md.MD_PLAIN_FP32])
def test_chain_observables_match_oracle(precision):
    """End-to-end vectors, radii of gyration and the trans fraction computed
    on the GPU against oracle/observables.py on the same (uploaded) state,
    two replicas; the generator's chains cross the box walls."""
    from oracle import observables as ob
    melts = [chaingen.melt(12, seed=41), chaingen.melt(20, seed=42)]
    s = md.System(melts, precision=precision)
    got = s.observables()
    off = 0
    for r, m in enumerate(melts):
        x, _ = _uploaded(m, precision)
        xu = chaingen.unwrapped(dict(m, pos=x))
        n = m["n_chains"]
        ree, rg2 = ob.end_to_end(xu, m["sites"]), ob.radius_of_gyration_sq(xu, m["sites"], m["masses"])
        tol = 1e-12 if precision == md.MD_MIXED else 1e-9
        assert np.allclose(got["r_ee"][off:off + n], ree, rtol=tol, atol=tol)
        assert np.allclose(got["rg2"][off:off + n], rg2, rtol=tol * 100)
        phi = ob.dihedral_angles(xu, m["sites"])
        want = np.mean(np.abs(phi) > 120.0)
        near = np.sum(np.abs(np.abs(phi) - 120.0) < 1e-6)      # classification ties the precisions may split
        assert abs(got["trans_fraction"][r] - want) <= near / phi.size + 1e-15
        off += n
    s.close()


@pytest.mark.parametrize("precision", [md.MD_MIXED, md.MD_PLAIN_FP32])
def test_rdf_counts_are_bit_exact(precision):
    """RDF of non-bonded pairs on the GPU (md_rdf) against the FP64
    definition of oracle/observables.rdf on the same positions, two
    replicas: the integer pair counts per bin are equal."""
    from oracle import observables as ob
    melts = [chaingen.melt(12, seed=51), chaingen.melt(20, seed=52)]
    s = md.System(melts, precision=precision)
    r_max, n_bins = 1.0, 50
    centres, g, counts = s.rdf(r_max, n_bins)
    for r, m in enumerate(melts):
        x, _ = _uploaded(m, precision)
        c_o, g_o, n_o = ob.rdf(x, m["L"], m["sites"], r_max, n_bins)
        assert np.array_equal(counts[r], n_o)
        assert np.allclose(g[r], g_o, rtol=1e-12)
        assert np.allclose(centres, c_o)
    s.close()


def test_end_to_end_acf_accumulator_matches_oracle():
    """The on-GPU ACF accumulator fed a given series (md_acf_push): two
    replicas, 60 samples of seeded end-to-end vectors (a slow rotation plus
    noise), lags 0..20, against oracle/observables.end_to_end_acf of the same
    series per replica."""
    from oracle import observables as ob
    melts = [chaingen.melt(6, seed=53, L=3.6), chaingen.melt(9, seed=54, L=3.6)]
    s = md.System(melts, precision=md.MD_MIXED)
    n_ch = [m["n_chains"] for m in melts]
    rng = np.random.default_rng(7)
    n_s, lag = 60, 20
    phase = rng.uniform(0, 2 * np.pi, size=sum(n_ch))
    series = []
    for t in range(n_s):
        a = phase + 0.05 * t
        R = np.stack([3.0 * np.cos(a), 3.0 * np.sin(a), rng.normal(size=a.size)], axis=1)
        series.append(R)
    series = np.array(series)
    s.acf_reset(lag)
    for t in range(n_s):
        s.acf_push(series[t])
    C, n = s.acf()
    assert n == n_s
    off = 0
    for r, k in enumerate(n_ch):
        want = ob.end_to_end_acf(series[:, off:off + k], lag)
        assert np.allclose(C[r], want, rtol=1e-12, atol=1e-14)
        off += k
    s.close()


def test_end_to_end_acf_sampled_from_the_state():
    """md_acf_sample takes the same end-to-end vectors as md_observables:
    sampling a stepped system gives the same bits as pushing the vectors
    that md_observables returns at each sample."""
    m = chaingen.melt(8, seed=55)
    a = md.System(m, precision=md.MD_MIXED, rebin_every=5)
    b = md.System(m, precision=md.MD_MIXED, rebin_every=5)
    a.acf_reset(6); b.acf_reset(6)
    for _ in range(12):
        a.step(5); b.step(5)
        a.acf_sample()
        b.acf_push(b.observables()["r_ee"])
    ca, na = a.acf()
    cb, nb = b.acf()
    assert na == nb == 12
    assert np.array_equal(ca, cb)
    a.close(); b.close()


@pytest.mark.parametrize("precision", [md.MD_MIXED, md.MD_PLAIN_FP32])
def test_bin_study_arms_give_the_oracle_bins(precision):
    """md_bin_study runs the on-GPU counting sort and the host-copy (CBIN)
    arm of Sec. 3.1 on the same positions: the host arm's bins (left in
    place) and the GPU arm's bins (md_rebin) both equal the oracle's binning
    of the uploaded positions, and a system that ran the study steps on with
    the same bits as one that did not."""
    m = chaingen.melt(30, seed=61, L=5.2)
    a = md.System(m, precision=precision, rebin_every=5)
    b = md.System(m, precision=precision, rebin_every=5)
    x, _ = _uploaded(m, precision)
    M = a.info["cells_per_side"]
    want = oracle.bin_atoms(x, m["L"], M)
    t = a.bin_study(2)
    assert t["host_total"] > 0 and t["gpu_binning"] > 0
    for got, w in zip(a.bins(), want):
        assert np.array_equal(got, w)
    a.rebin()
    for got, w in zip(a.bins(), want):
        assert np.array_equal(got, w)
    a.step(10); b.step(10)
    xa, va, _ = a.state(); xb, vb, _ = b.state()
    assert np.array_equal(xa, xb) and np.array_equal(va, vb)
    a.close(); b.close()


# ---------------------------------------------------------------- general molecules (Sec. 3.3)

def _branched_topology(mixed_types=False):
    """A 12-atom branched molecule: backbone 0-1-...-7, side atoms 8 on 2, 9 on
    4, and a two-atom branch 10-11 on 6.  Atoms with one bond are C_33, the
    others C_32 (the polyethylene convention); with mixed_types the interior
    atom 3 is C_33 as well."""
    bonds = [(k, k + 1) for k in range(7)] + [(2, 8), (4, 9), (6, 10), (10, 11)]
    deg = np.zeros(12, int)
    for a, b in bonds:
        deg[a] += 1; deg[b] += 1
    types = (deg == 1).astype(np.int32)
    if mixed_types:
        types[3] = 1
    return np.array(bonds, np.int32), types


def _branched_melt(n_mol, L, seed):
    """Molecules placed one by one at random positions and orientations,
    rejected while any site comes within 0.32 nm of a site of another
    molecule (periodic cube of side L).  Backbone: a planar zigzag (bond
    0.153 nm, angle 109.47 deg); side atoms 0.153 nm from their parent,
    normal to the backbone plane (alternating sides), and atom 11 off the
    10 - 6 axis (no straight angle)."""
    b, th = 0.153, np.arccos(-1.0 / 3.0)
    base = [np.array([k * b * np.sin(th / 2), (k % 2) * b * np.cos(th / 2), 0.0]) for k in range(8)]
    base.append(base[2] + [0.0, 0.0, b])
    base.append(base[4] + [0.0, 0.0, -b])
    base.append(base[6] + [0.0, 0.0, b])
    base.append(base[10] + b * np.array([0.5, 0.3, 0.8124]) / np.linalg.norm([0.5, 0.3, 0.8124]))
    base = np.array(base)
    base -= base.mean(0)
    rng = np.random.default_rng(seed)
    placed = []
    while len(placed) < n_mol:
        q = rng.normal(size=4)
        q /= np.linalg.norm(q)
        w, x, y, z = q
        Rm = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                       [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                       [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])
        mol = base @ Rm.T + rng.uniform(0, L, size=3)
        ok = True
        for other in placed:
            d = mol[:, None, :] - other[None, :, :]
            d -= L * np.round(d / L)
            if np.min(np.sum(d * d, axis=2)) < 0.32 ** 2:
                ok = False
                break
        if ok:
            placed.append(mol)
    pos = np.mod(np.concatenate(placed), L)
    vel = 0.3 * rng.normal(size=pos.shape)
    return dict(pos=pos, vel=vel, L=L, n_chains=n_mol, sites=12, T=300.0)


@pytest.mark.parametrize("mixed_types", [False, True])
def test_branched_molecules_match_oracle(mixed_types):
    """A branched, and a mixed-type, molecule given by its bond graph
    (md_desc.topology): exclusions, bonds, angles and dihedrals come from the
    per-type lists of Sec. 3.3 built by the library.  Forces and energies at
    the start, and forces after 20 steps, against the oracle's topology built
    from the same bond graph."""
    bonds, types = _branched_topology(mixed_types)
    m = _branched_melt(70, 4.4, seed=91 + int(mixed_types))
    s = md.System(m, precision=md.MD_MIXED, topology=(bonds, types), rebin_every=5)
    topo = oracle.Topology(12, bonds, types)
    ref = oracle.System(topo, m["n_chains"], m["L"], use_cells=False)
    x = np.array(m["pos"], np.float64)
    f_orc, en, _ = ref.forces(x)
    check_forces(s.forces(), f_orc, x, m["L"])
    e = s.energy()[0]
    for k, idx in (("lj", 0), ("lj_shifted", 1), ("bond", 2), ("angle", 3), ("dihedral", 4)):
        assert abs(e[k] - en[idx]) <= 1e-5 * max(1.0, abs(en[idx])), (k, e[k], en[idx])
    s.step(20)
    xo, _, fo, _, _ = ref.run(x, m["vel"], 0.001, 20, sample_every=0)
    check_forces(s.forces(), fo, xo, m["L"])
    with pytest.raises(md.MDError):
        s.observables()
    s.close()
