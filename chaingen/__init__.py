"""Seeded synthetic polyethylene melts (inputs only).

The generator grows united-atom chains (Sec. 2 of the paper: 150-site chains,
CH3 ends and CH2 interior, bond 0.153 nm, tetrahedral angle, trans/gauche
dihedrals) in a periodic cube at a chosen mass density, and draws Maxwell
velocities.  It holds none of the force-field or integrator arithmetic, so the
CUDA path and the FP64 oracle can both consume its output without sharing the
method's code.  All randomness is SplitMix64 keyed by the seed; the C source is
built with -ffp-contract=off so x86-64 and aarch64 produce identical bits.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "chaingen.c")
_LIB = os.path.join(_HERE, "libchaingen.so")

KB = 0.0083144626          # kJ/mol/K (CODATA 2018 R / 1000)
AMU_G = 1.66053906660e-24  # g per amu
MASS_CH2 = 14.027          # amu, Table I
MASS_CH3 = 15.035          # amu, Table I
BOND = 0.153               # nm, Table I

_lib = None


def build(force: bool = False) -> str:
    """Compile libchaingen.so next to the source (gcc, portable flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        d, i32, i64, u64 = ctypes.c_double, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
        P = ctypes.c_void_p
        lib.cg_grow_chains.argtypes = [i32, i32, d, d, d, d, u64, P]
        lib.cg_grow_chains.restype = ctypes.c_int
        lib.cg_maxwell.argtypes = [i64, P, d, d, u64, P]
        lib.cg_maxwell.restype = None
        lib.cg_uniforms.argtypes = [u64, i64, P]
        lib.cg_uniforms.restype = None
        lib.cg_splitmix64.argtypes = [u64]
        lib.cg_splitmix64.restype = u64
        lib.cg_ln_export.argtypes = [d]
        lib.cg_ln_export.restype = d
        lib.cg_exp_export.argtypes = [d]
        lib.cg_exp_export.restype = d
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def sub_seed(seed: int, k: int) -> int:
    """Independent stream k of a seed (one SplitMix64 output)."""
    return int(_load().cg_splitmix64(ctypes.c_uint64((seed * 0x100000001B3 + k) & (2**64 - 1))))


def site_masses(sites: int) -> np.ndarray:
    m = np.full(sites, MASS_CH2)
    m[0] = m[-1] = MASS_CH3
    return m


def site_types(sites: int) -> np.ndarray:
    """0 = C_32 (CH2, interior), 1 = C_33 (CH3, chain ends)."""
    t = np.zeros(sites, dtype=np.int32)
    t[0] = t[-1] = 1
    return t


def box_length(n_chains: int, sites: int = 150, density_g_cm3: float = 0.77) -> float:
    """Cube side (nm) holding n_chains chains at the mass density, rounded to a
    multiple of 2^-20 nm so that it is exactly representable in FP32."""
    mass_amu = n_chains * float(site_masses(sites).sum())
    vol_nm3 = mass_amu * AMU_G / density_g_cm3 * 1e21
    L = vol_nm3 ** (1.0 / 3.0)
    return round(L * 2**20) / 2**20


def melt(n_chains: int, sites: int = 150, seed: int = 1, T: float = 500.0,
         density_g_cm3: float = 0.77, L: float | None = None, r_min: float = 0.27,
         p_trans: float = 0.6) -> dict:
    """One periodic melt: pos (N,3) wrapped in [0,L), vel (N,3), types (N,),
    masses (N,), chain-major atom order (atom = chain*sites + index).  L is
    rounded to a multiple of 2^-20 nm so that it is exact in FP32."""
    lib = _load()
    if L is None:
        L = box_length(n_chains, sites, density_g_cm3)
    L = round(float(L) * 2**20) / 2**20     # every box side is exactly representable in FP32
    N = n_chains * sites
    pos = np.empty((N, 3), dtype=np.float64)
    relaxed = lib.cg_grow_chains(n_chains, sites, L, BOND, r_min, p_trans,
                                 ctypes.c_uint64(sub_seed(seed, 0)), _ptr(pos))
    masses = np.tile(site_masses(sites), n_chains)
    vel = np.empty((N, 3), dtype=np.float64)
    lib.cg_maxwell(N, _ptr(masses), T, KB, ctypes.c_uint64(sub_seed(seed, 1)), _ptr(vel))
    return dict(pos=pos, vel=vel, L=float(L), n_chains=n_chains, sites=sites,
                types=np.tile(site_types(sites), n_chains), masses=masses,
                T=T, seed=seed, relaxed=int(relaxed))


def maxwell(masses: np.ndarray, T: float, seed: int, stream: int = 1) -> np.ndarray:
    """Fresh Maxwell-Boltzmann velocities (N,3) in nm/ps at T kelvin for the
    given masses (amu), zero total momentum; stream 1 is the one melt() uses."""
    masses = np.ascontiguousarray(masses, dtype=np.float64)
    vel = np.empty((len(masses), 3), dtype=np.float64)
    _load().cg_maxwell(len(masses), _ptr(masses), float(T), KB, ctypes.c_uint64(sub_seed(seed, stream)), _ptr(vel))
    return vel


def unwrapped(m: dict) -> np.ndarray:
    """Positions (N,3) with every chain made continuous: site 0 as stored,
    each later site one minimum-image bond vector on from the previous."""
    p = m["pos"].reshape(m["n_chains"], m["sites"], 3)
    d = np.diff(p, axis=1)
    d -= m["L"] * np.round(d / m["L"])
    out = np.concatenate([p[:, :1], p[:, :1] + np.cumsum(d, axis=1)], axis=1)
    return out.reshape(-1, 3)


def uniforms(seed: int, n: int) -> np.ndarray:
    out = np.empty(n, dtype=np.float64)
    _load().cg_uniforms(ctypes.c_uint64(sub_seed(seed, 7)), n, _ptr(out))
    return out


def replica_recipe(n_replicas: int = 64, seed: int = 4, lo: int = 20, hi: int = 400,
                   t_lo: float = 250.0, t_hi: float = 500.0):
    """Chain counts log-uniform in [lo, hi] and temperatures uniform in
    [t_lo, t_hi], one pair per replica, from the seed."""
    lib = _load()
    u = uniforms(seed, 2 * n_replicas)
    a, b = lib.cg_ln_export(float(lo)), lib.cg_ln_export(float(hi))
    counts = [int(lib.cg_exp_export(a + (b - a) * u[2 * r]) + 0.5) for r in range(n_replicas)]
    counts = [min(max(c, lo), hi) for c in counts]
    temps = [t_lo + (t_hi - t_lo) * u[2 * r + 1] for r in range(n_replicas)]
    return counts, temps


def replicas(n_replicas: int = 64, seed: int = 4, sites: int = 150, **kw) -> list[dict]:
    counts, temps = replica_recipe(n_replicas, seed)
    out = []
    for r, (c, T) in enumerate(zip(counts, temps)):
        out.append(melt(c, sites, seed=sub_seed(seed, 100 + r), T=T, **kw))
    return out
