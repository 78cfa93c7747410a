"""FP64 CPU oracle for the united-atom polyethylene MD step (test infrastructure).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU-baseline leg are the only callers.  The product path never imports this
package.  It shares no code with the CUDA library; its parameter defaults are
restated here from the paper (Table I and the readings listed below).

Readings of the paper taken here (the paper is garbled or silent):
  * Table I columns are shifted: 14.027/15.035 are the CH2/CH3 masses (amu),
    0.3624/0.3699 nm are sigma for C_32/C_33; epsilon is not printed and is
    taken as 46 K and 98 K times k_B (0.3825 and 0.8148 kJ/mol), a labelled
    assumption that stays a runtime parameter.
  * Mixing of unlike pairs: geometric in both epsilon and sigma.
  * Table I units: k_b = 292880 kJ/mol/nm^2 with the 1/2 of Eq. (4),
    k_a = 418.4 kJ/mol/rad^2 with theta0 = 109.471 deg, k_phi = 4.184 kJ/mol,
    n = 3, phi_s = 0.
  * Cutoff r_c = 1.0 nm, plain truncation (Sec. 3.2 listing).  The reported
    LJ energy is also given with the per-pair shift -E(r_c) ("shifted").
  * Dihedral angle phi in the IUPAC convention (trans = 180 deg).
  * params["lj_form"] = 1 selects a force-shifted LJ, E(r) - E(r_c) -
    (r - r_c) E'(r_c), whose force vanishes at r_c.  It is NOT the paper's
    potential: the gradient checks use it to separate the force jump at r_c
    (which no adjoint of the smooth branch sees) from the adjoint itself.

Parity status: every routine here is pinned by tests in tests/test_oracle.py
(finite differences, closed forms, brute force vs cells, the paper's worked
topology example).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "md_oracle.c")
_LIB = os.path.join(_HERE, "libmd_oracle.so")

KB = 0.0083144626  # kJ/mol/K

_lib = None


class FF(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_double * 2), ("sigma", ctypes.c_double * 2),
                ("mass", ctypes.c_double * 2), ("kb", ctypes.c_double), ("b0", ctypes.c_double),
                ("ka", ctypes.c_double), ("theta0", ctypes.c_double), ("kphi", ctypes.c_double),
                ("phis", ctypes.c_double), ("n_mult", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("rc", ctypes.c_double), ("lj_form", ctypes.c_int32), ("pad2", ctypes.c_int32)]


class Sys(ctypes.Structure):
    _fields_ = [("n_mol", ctypes.c_int64), ("naom", ctypes.c_int32), ("nb", ctypes.c_int32),
                ("na", ctypes.c_int32), ("nd", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("type_m", ctypes.c_void_p), ("excl_index", ctypes.c_void_p), ("excl", ctypes.c_void_p),
                ("bonds", ctypes.c_void_p), ("angles", ctypes.c_void_p), ("dih", ctypes.c_void_p),
                ("L", ctypes.c_double), ("use_cells", ctypes.c_int32), ("nthreads", ctypes.c_int32)]


def default_params() -> dict:
    """Table I with the readings in the module docstring."""
    return dict(eps=(46.0 * KB, 98.0 * KB), sigma=(0.3624, 0.3699), mass=(14.027, 15.035),
                kb=292880.0, b0=0.153, ka=418.4, theta0=math.radians(109.471),
                kphi=4.184, phis=0.0, n_mult=3, rc=1.0)


def make_ff(p: dict) -> FF:
    ff = FF()
    ff.eps[:] = p["eps"]; ff.sigma[:] = p["sigma"]; ff.mass[:] = p["mass"]
    ff.kb, ff.b0, ff.ka, ff.theta0 = p["kb"], p["b0"], p["ka"], p["theta0"]
    ff.kphi, ff.phis, ff.n_mult, ff.rc = p["kphi"], p["phis"], int(p["n_mult"]), p["rc"]
    ff.lj_form = int(p.get("lj_form", 0))   # 1: force-shifted variant (gradient checks only)
    return ff


def build(force: bool = False) -> str:
    """Compile the oracle (gcc, FP64, no FMA contraction, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        P, i32, i64, d = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        L.orc_topo_bonds.argtypes = [ctypes.c_int, ctypes.c_int, P, P, P]
        L.orc_topo_exclusions.argtypes = [ctypes.c_int, ctypes.c_int, P, P, P, ctypes.c_int]
        L.orc_topo_angles.argtypes = [ctypes.c_int, ctypes.c_int, P, P, ctypes.c_int]
        L.orc_topo_dihedrals.argtypes = [ctypes.c_int, ctypes.c_int, P, P, ctypes.c_int]
        L.orc_topo_home_view.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, P, P, P]
        sysargs = [i64, P, d, i32, P, P, P, P]
        L.orc_lj_brute.argtypes = sysargs + [P, P, P]
        L.orc_lj_cells.argtypes = sysargs + [P, P, P, i32]
        L.orc_lj_atoms.argtypes = sysargs + [i64, P, P, i32]
        L.orc_bin.argtypes = [i64, P, d, i32, P, P, P]
        L.orc_bonded.argtypes = [i64, i32, P, d, i32, P, i32, P, i32, P, P, P, P, P]
        L.orc_forces.argtypes = [P, P, P, P, P, P]
        L.orc_run.argtypes = [P, P, P, P, P, P, d, i64, i32, d, d, d, P, i64, P]
        L.orc_run.restype = ctypes.c_int
        L.orc_run_nh.argtypes = [P, P, P, P, P, P, d, i64, d, d, d, P, i64, P]
        L.orc_run_nh.restype = ctypes.c_int
        L.orc_traj_means.argtypes = [P, P, P, P, P, d, i64, P]
        L.orc_traj_means.restype = ctypes.c_int
        L.orc_kinetic.argtypes = [i64, i32, P, P]
        L.orc_kinetic.restype = d
        _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


# --------------------------------------------------------------------------
# topology (Sec. 3.3)

def chain_bonds(naom: int) -> np.ndarray:
    return np.array([(k, k + 1) for k in range(naom - 1)], dtype=np.int32).reshape(-1, 2)


class Topology:
    """Per-molecule-type lists built from a bond graph (Sec. 3.3)."""

    def __init__(self, naom: int, bonds: np.ndarray, types_m: np.ndarray):
        self.naom = naom
        self.bonds = _c(bonds, np.int32).reshape(-1, 2)
        self.types_m = _c(types_m, np.int32)
        nb = len(self.bonds)
        cap = 64 * naom + 64
        ei = np.zeros(naom + 1, np.int32); ex = np.zeros(cap, np.int32)
        ne = lib().orc_topo_exclusions(naom, nb, _p(self.bonds), _p(ei), _p(ex), cap)
        self.excl_index, self.excl = ei, ex[:ne].copy()
        ang = np.zeros(3 * cap, np.int32)
        na = lib().orc_topo_angles(naom, nb, _p(self.bonds), _p(ang), cap)
        self.angles = ang[:3 * na].reshape(-1, 3).copy()
        dh = np.zeros(4 * cap, np.int32)
        nd = lib().orc_topo_dihedrals(naom, nb, _p(self.bonds), _p(dh), cap)
        self.dihedrals = dh[:4 * nd].reshape(-1, 4).copy()

    def t_bonds(self):
        idx = np.zeros(self.naom + 1, np.int32); b = np.zeros(2 * len(self.bonds), np.int32)
        lib().orc_topo_bonds(self.naom, len(self.bonds), _p(self.bonds), _p(idx), _p(b))
        return idx, b

    def home_view(self, terms: np.ndarray):
        terms = _c(terms, np.int32)
        w = terms.shape[1]
        idx = np.zeros(self.naom + 1, np.int32)
        rows = np.zeros((w * len(terms), w + 1), np.int32)
        n = lib().orc_topo_home_view(self.naom, len(terms), w, _p(terms), _p(idx), _p(rows))
        return idx, rows[:n]


def chain_topology(naom: int = 150) -> Topology:
    t = np.zeros(naom, np.int32)
    t[0] = t[-1] = 1
    return Topology(naom, chain_bonds(naom), t)


# --------------------------------------------------------------------------
# forces, energies, binning, integration

class System:
    """n_mol identical molecules (atom = molecule * naom + MAIDX) in a cube L."""

    def __init__(self, topo: Topology, n_mol: int, L: float, params: dict | None = None,
                 use_cells: bool | None = None, nthreads: int = 0):
        self.topo, self.n_mol, self.L = topo, n_mol, float(L)
        self.n = n_mol * topo.naom
        self.params = dict(default_params() if params is None else params)
        self.ff = make_ff(self.params)
        if use_cells is None:
            use_cells = self.n > 3000
        self.s = Sys(n_mol, topo.naom, len(topo.bonds), len(topo.angles), len(topo.dihedrals), 0,
                     _p(topo.types_m), _p(topo.excl_index), _p(topo.excl), _p(topo.bonds),
                     _p(topo.angles), _p(topo.dihedrals), self.L, int(use_cells), nthreads)
        self.masses_m = np.array([self.params["mass"][t] for t in topo.types_m])

    def set_params(self, p: dict):
        self.params = dict(p)
        self.ff = make_ff(self.params)
        self.masses_m = np.array([self.params["mass"][t] for t in self.topo.types_m])

    def _sysargs(self, x):
        t = self.topo
        return [self.n, _p(x), self.L, t.naom, _p(t.types_m), _p(t.excl_index), _p(t.excl),
                ctypes.byref(self.ff)]

    def lj(self, x, method: str = "brute", nthreads: int = 0):
        x = _c(x, np.float64).reshape(-1, 3)
        f = np.zeros_like(x); en = np.zeros(2); vir = np.zeros(6)
        if method == "brute":
            lib().orc_lj_brute(*self._sysargs(x), _p(f), _p(en), _p(vir))
        else:
            lib().orc_lj_cells(*self._sysargs(x), _p(f), _p(en), _p(vir), nthreads)
        return f, en, vir

    def lj_atoms(self, x, atoms, nthreads: int = 0):
        x = _c(x, np.float64).reshape(-1, 3)
        sel = _c(atoms, np.int64)
        f = np.zeros((len(sel), 3))
        lib().orc_lj_atoms(*self._sysargs(x), len(sel), _p(sel), _p(f), nthreads)
        return f

    def bonded(self, x):
        x = _c(x, np.float64).reshape(-1, 3)
        t = self.topo
        f = np.zeros_like(x); en = np.zeros(3); vir = np.zeros(6)
        lib().orc_bonded(self.n_mol, t.naom, _p(x), self.L, len(t.bonds), _p(t.bonds),
                         len(t.angles), _p(t.angles), len(t.dihedrals), _p(t.dihedrals),
                         ctypes.byref(self.ff), _p(f), _p(en), _p(vir))
        return f, en, vir

    def forces(self, x):
        """total force, energies (lj, lj_shifted, bond, angle, dihedral), virial"""
        x = _c(x, np.float64).reshape(-1, 3)
        f = np.zeros_like(x); en = np.zeros(7); vir = np.zeros(6)
        lib().orc_forces(ctypes.byref(self.s), ctypes.byref(self.ff), _p(x), _p(f), _p(en), _p(vir))
        return f, en[:5], vir

    def run(self, x, v, dt: float, n_steps: int, thermostat: bool = False, T0: float = 300.0,
            tau: float = 0.1, lam: float = 1.0, sample_every: int = 1):
        """velocity Verlet; returns x, v, f, samples[(step, lj, lj_s, bond, angle, dih, ke, T)], lam"""
        x = _c(x, np.float64).reshape(-1, 3).copy()
        v = _c(v, np.float64).reshape(-1, 3).copy()
        f = np.zeros_like(x)
        rows = n_steps // max(sample_every, 1) + 2
        samples = np.zeros((rows, 8))
        lam_c = ctypes.c_double(lam)
        nr = lib().orc_run(ctypes.byref(self.s), ctypes.byref(self.ff), _p(self.masses_m), _p(x), _p(v),
                           _p(f), dt, n_steps, int(thermostat), T0, tau, KB, ctypes.byref(lam_c),
                           sample_every, _p(samples))
        return x, v, f, samples[:nr], lam_c.value

    def run_nh(self, x, v, dt: float, n_steps: int, T0: float, tau: float, xi: float = 0.0, sample_every: int = 1):
        """Leap-Frog with Nose-Hoover coupling and centre-of-mass translation
        removal (Sec. 2, Sec. 3.4), Q = tau^2 T0 / (4 pi^2); v is the on-step
        velocity.  Returns x, v, f, samples[(step, lj, lj_s, bond, angle, dih,
        ke, T, xi, eta)], xi."""
        x = _c(x, np.float64).reshape(-1, 3).copy()
        v = _c(v, np.float64).reshape(-1, 3).copy()
        f = np.zeros_like(x)
        rows = n_steps // max(sample_every, 1) + 2
        samples = np.zeros((rows, 10))
        xi_c = ctypes.c_double(xi)
        nr = lib().orc_run_nh(ctypes.byref(self.s), ctypes.byref(self.ff), _p(self.masses_m), _p(x), _p(v),
                              _p(f), dt, n_steps, T0, tau, KB, ctypes.byref(xi_c), sample_every, _p(samples))
        return x, v, f, samples[:nr], xi_c.value

    def nh_extended_energy(self, samples, T0: float, tau: float):
        """H = K + U + g kB Q xi^2 / 2 + g kB T0 eta per sample row of run_nh
        (U with the shifted LJ energy; g = 3N - 3)."""
        g = 3.0 * self.n - 3.0
        Q = tau * tau * T0 / (4.0 * np.pi ** 2)
        U = samples[:, 2] + samples[:, 3] + samples[:, 4] + samples[:, 5]
        return samples[:, 6] + U + 0.5 * g * KB * Q * samples[:, 8] ** 2 + g * KB * T0 * samples[:, 9]

    def traj_means(self, x, v, dt: float, n_steps: int):
        """(mean U, mean R_ee^2) over steps 0..n_steps of an NVE velocity-Verlet
        run; U = shifted LJ + bond + angle + dihedral, R_ee from unwrapped x."""
        x = _c(x, np.float64).reshape(-1, 3)
        v = _c(v, np.float64).reshape(-1, 3)
        out = np.zeros(2)
        lib().orc_traj_means(ctypes.byref(self.s), ctypes.byref(self.ff), _p(self.masses_m), _p(x), _p(v),
                             dt, n_steps, _p(out))
        return out

    def theta(self):
        """The differentiated parameters (eps_C32, eps_C33, sigma_C32, sigma_C33, k_phi)."""
        p = self.params
        return np.array([p["eps"][0], p["eps"][1], p["sigma"][0], p["sigma"][1], p["kphi"]])

    def with_theta(self, th):
        p = dict(self.params)
        p["eps"] = (float(th[0]), float(th[1]))
        p["sigma"] = (float(th[2]), float(th[3]))
        p["kphi"] = float(th[4])
        return p

    def fd_gradient(self, x, v, dt: float, n_steps: int, rel_h: float = 1e-4):
        """Central finite differences of traj_means in each of the five
        parameters, step rel_h * |theta_i|: array (2, 5), row 0 d<U>, row 1
        d<R_ee^2>.  The parameters are restored afterwards."""
        th0 = self.theta()
        p0 = dict(self.params)
        g = np.zeros((2, 5))
        try:
            for i in range(5):
                h = rel_h * abs(th0[i])
                tp, tm = th0.copy(), th0.copy()
                tp[i] += h; tm[i] -= h
                self.set_params(self.with_theta(tp)); jp = self.traj_means(x, v, dt, n_steps)
                self.set_params(self.with_theta(tm)); jm = self.traj_means(x, v, dt, n_steps)
                g[:, i] = (jp - jm) / (tp[i] - tm[i])
        finally:
            self.set_params(p0)
        return g

    def kinetic(self, v):
        v = _c(v, np.float64).reshape(-1, 3)
        return lib().orc_kinetic(self.n, self.topo.naom, _p(self.masses_m), _p(v))


def bin_atoms(x, L: float, M: int):
    """Stable counting sort of atoms into M^3 cells (Sec. 3.1)."""
    x = _c(x, np.float64).reshape(-1, 3)
    n = len(x)
    cell_of = np.zeros(n, np.int32); start = np.zeros(M ** 3 + 1, np.int32); perm = np.zeros(n, np.int32)
    lib().orc_bin(n, _p(x), float(L), M, _p(cell_of), _p(start), _p(perm))
    return cell_of, start, perm
