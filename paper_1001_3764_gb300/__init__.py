"""Python binding of the GB300 united-atom polyethylene MD engine.

Argument marshalling only: every step of the method runs in the CUDA library
libmdgb300.so behind the C ABI of include/md.h (same function names).  PyTorch
supplies device memory (the workspace) and the CUDA stream.  There is no CPU
fallback: if the library is missing this module raises.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

from . import build as _build

LIB_PATH = _build.LIB

MD_OK, MD_EINVAL, MD_ENOMEM, MD_ECUDA, MD_EOVERFLOW, MD_EUNSTABLE, MD_ETIMEOUT = 0, -1, -2, -3, -4, -5, -6
MD_PLAIN_FP32, MD_MIXED = 0, 1
MD_NVE, MD_VRESCALE, MD_NOSE_HOOVER = 0, 1, 2
MD_SCHED_GRID, MD_SCHED_PERSISTENT = 0, 1
MD_DISP_REBUILD, MD_DISP_ERROR = 0, 1
KB = 0.0083144626  # kJ/mol/K

_ERRNAMES = {MD_EINVAL: "MD_EINVAL", MD_ENOMEM: "MD_ENOMEM", MD_ECUDA: "MD_ECUDA",
             MD_EOVERFLOW: "MD_EOVERFLOW", MD_EUNSTABLE: "MD_EUNSTABLE", MD_ETIMEOUT: "MD_ETIMEOUT"}


class MDError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_ERRNAMES.get(code, code)}: {msg}")
        self.code = code


class md_params(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_double * 2), ("sigma", ctypes.c_double * 2), ("mass", ctypes.c_double * 2),
                ("kb", ctypes.c_double), ("b0", ctypes.c_double), ("ka", ctypes.c_double),
                ("theta0", ctypes.c_double), ("kphi", ctypes.c_double), ("phis", ctypes.c_double),
                ("n_mult", ctypes.c_int32), ("pad", ctypes.c_int32)]


class md_topology(ctypes.Structure):
    _fields_ = [("naom", ctypes.c_int32), ("n_bonds", ctypes.c_int32), ("bonds", ctypes.c_void_p),
                ("types", ctypes.c_void_p)]


class md_desc(ctypes.Structure):
    _fields_ = [("n_replicas", ctypes.c_int32), ("sites_per_chain", ctypes.c_int32),
                ("n_chains", ctypes.c_void_p), ("box", ctypes.c_void_p), ("pos", ctypes.c_void_p),
                ("vel", ctypes.c_void_p), ("T_target", ctypes.c_void_p), ("params", md_params),
                ("dt", ctypes.c_double), ("rc", ctypes.c_double), ("skin", ctypes.c_double),
                ("tau_t", ctypes.c_double), ("rebin_every", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("thermostat", ctypes.c_int32), ("nbr_capacity", ctypes.c_int32),
                ("lj_block", ctypes.c_int32), ("schedule", ctypes.c_int32), ("lj_lanes", ctypes.c_int32),
                ("lj_region", ctypes.c_int32), ("lj_pair_exact", ctypes.c_int32), ("topology", ctypes.c_void_p), ("displacement", ctypes.c_int32),
                ("cuda_stream", ctypes.c_void_p), ("workspace", ctypes.c_void_p),
                ("workspace_bytes", ctypes.c_size_t)]


class md_tuning(ctypes.Structure):
    _fields_ = [("skin", ctypes.c_double), ("rebin_every", ctypes.c_int32), ("lj_block", ctypes.c_int32),
                ("schedule", ctypes.c_int32), ("lj_lanes", ctypes.c_int32), ("lj_region", ctypes.c_int32),
                ("from_cache", ctypes.c_int32),
                ("us_per_step", ctypes.c_double)]


class md_adj_desc(ctypes.Structure):
    _fields_ = [("n_chains", ctypes.c_int32), ("sites_per_chain", ctypes.c_int32), ("box", ctypes.c_double),
                ("params", md_params), ("rc", ctypes.c_double), ("dt", ctypes.c_double),
                ("n_steps", ctypes.c_int32), ("checkpoint_every", ctypes.c_int32),
                ("lj_form", ctypes.c_int32), ("hvp_precision", ctypes.c_int32), ("cuda_stream", ctypes.c_void_p)]


class md_energy_t(ctypes.Structure):
    _fields_ = [("lj", ctypes.c_double), ("lj_shifted", ctypes.c_double), ("bond", ctypes.c_double),
                ("angle", ctypes.c_double), ("dihedral", ctypes.c_double), ("kinetic", ctypes.c_double),
                ("temperature", ctypes.c_double), ("total", ctypes.c_double),
                ("virial", ctypes.c_double * 6), ("pressure", ctypes.c_double)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "virial"}
        d["virial"] = list(self.virial)
        return d


EXPORTS = ["md_autotune", "md_workspace_size", "md_create", "md_step", "md_step_async", "md_sync", "md_forces", "md_energy",
           "md_rebin", "md_get_state", "md_set_state", "md_set_params", "md_set_temperature", "md_get_thermostat", "md_observables", "md_rdf",
           "md_acf_reset", "md_acf_sample", "md_acf_push", "md_acf_read", "md_early_rebins", "md_bin_study",
           "md_stream",
           "md_info", "md_get_bins", "md_get_neighbors", "md_get_cell_units", "md_profile_enable", "md_profile_read",
           "md_profile_reset", "md_launches_per_call", "md_bin_static", "md_destroy", "md_last_error",
           "md_adj_create", "md_adj_set_theta", "md_adj_forward", "md_adj_backward", "md_adj_tangent",
           "md_adj_energy", "md_adj_destroy", "md_wait_selftest"]

_lib = None


def load(path: str = LIB_PATH):
    """Load libmdgb300.so (built by build.build()); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"CUDA library {path} is missing: run paper_1001_3764_gb300.build.build() "
                          "(or __graft_entry__.build()) on a machine with nvcc")
    L = ctypes.CDLL(path)
    P, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    sig = {
        "md_autotune": ([P, i32, ctypes.c_char_p, P], ctypes.c_int),
        "md_workspace_size": ([P, P], ctypes.c_int),
        "md_create": ([P, P], ctypes.c_int),
        "md_step": ([P, i64], ctypes.c_int),
        "md_step_async": ([P, i64], ctypes.c_int),
        "md_sync": ([P], ctypes.c_int),
        "md_forces": ([P, P], ctypes.c_int),
        "md_energy": ([P, P], ctypes.c_int),
        "md_rebin": ([P], ctypes.c_int),
        "md_get_state": ([P, P, P, P], ctypes.c_int),
        "md_set_state": ([P, P, P], ctypes.c_int),
        "md_set_params": ([P, P], ctypes.c_int),
        "md_set_temperature": ([P, P], ctypes.c_int),
        "md_get_thermostat": ([P, P], ctypes.c_int),
        "md_observables": ([P, P, P, P], ctypes.c_int),
        "md_rdf": ([P, i32, P, P], ctypes.c_int),
        "md_acf_reset": ([P, i32], ctypes.c_int),
        "md_acf_sample": ([P], ctypes.c_int),
        "md_acf_push": ([P, P], ctypes.c_int),
        "md_acf_read": ([P, P, P], ctypes.c_int),
        "md_early_rebins": ([P, P], ctypes.c_int),
        "md_bin_study": ([P, i32, P], ctypes.c_int),
        "md_stream": ([P], P),
        "md_info": ([P, P, P, P, P], ctypes.c_int),
        "md_get_bins": ([P, P, P, P], ctypes.c_int),
        "md_get_neighbors": ([P, P, P], ctypes.c_int),
        "md_get_cell_units": ([P, P], ctypes.c_int),
        "md_profile_enable": ([P, i32], ctypes.c_int),
        "md_profile_read": ([P, P, P], ctypes.c_int),
        "md_profile_reset": ([P], ctypes.c_int),
        "md_launches_per_call": ([P, i64], i64),
        "md_bin_static": ([P, i32, ctypes.c_double, i32, P, P, P, P], ctypes.c_int),
        "md_destroy": ([P], None),
        "md_last_error": ([P], ctypes.c_char_p),
        "md_adj_create": ([P, P], ctypes.c_int),
        "md_adj_set_theta": ([P, P], ctypes.c_int),
        "md_adj_forward": ([P, P, P, P], ctypes.c_int),
        "md_adj_backward": ([P, P, P], ctypes.c_int),
        "md_adj_tangent": ([P, P, P, P, P, P], ctypes.c_int),
        "md_adj_energy": ([P, P], ctypes.c_int),
        "md_adj_destroy": ([P], None),
        "md_wait_selftest": ([i32], ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    _lib = L
    return L


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _check(rc, handle=None):
    if rc != MD_OK:
        raise MDError(rc, load().md_last_error(handle).decode())


def default_params() -> dict:
    """Table I of the paper with these readings: 14.027/15.035 amu masses and
    0.3624/0.3699 nm sigmas for C_32/C_33; epsilon (not printed) 46 K and 98 K
    times k_B; k_b = 292880 kJ/mol/nm^2, b0 = 0.153 nm; k_a = 418.4
    kJ/mol/rad^2, theta0 = 109.471 deg; k_phi = 4.184 kJ/mol, n = 3, phi_s = 0."""
    return dict(eps=(46.0 * KB, 98.0 * KB), sigma=(0.3624, 0.3699), mass=(14.027, 15.035),
                kb=292880.0, b0=0.153, ka=418.4, theta0=math.radians(109.471),
                kphi=4.184, phis=0.0, n_mult=3)


def make_params(p: dict) -> md_params:
    q = md_params()
    q.eps[:] = p["eps"]; q.sigma[:] = p["sigma"]; q.mass[:] = p["mass"]
    q.kb, q.b0, q.ka, q.theta0 = p["kb"], p["b0"], p["ka"], p["theta0"]
    q.kphi, q.phis, q.n_mult = p["kphi"], p["phis"], int(p["n_mult"])
    return q


# ---------------------------------------------------------------- thin wrappers (C ABI names)

def md_autotune(desc: md_desc, trial_cycles: int = 2, cache_path: str | None = None) -> dict:
    t = md_tuning()
    _check(load().md_autotune(ctypes.byref(desc), trial_cycles,
                              None if cache_path is None else cache_path.encode(), ctypes.byref(t)))
    return {k: getattr(t, k) for k, _ in t._fields_}


def md_workspace_size(desc: md_desc) -> int:
    b = ctypes.c_size_t()
    _check(load().md_workspace_size(ctypes.byref(desc), ctypes.byref(b)))
    return b.value


def md_create(desc: md_desc):
    h = ctypes.c_void_p()
    _check(load().md_create(ctypes.byref(desc), ctypes.byref(h)))
    return h


def md_step(h, n: int):
    _check(load().md_step(h, n), h)


def md_step_async(h, n: int):
    _check(load().md_step_async(h, n), h)


def md_sync(h):
    _check(load().md_sync(h), h)


def md_forces(h, n_atoms: int) -> np.ndarray:
    f = np.empty((n_atoms, 3))
    _check(load().md_forces(h, _p(f)), h)
    return f


def md_energy(h, n_replicas: int) -> list:
    out = (md_energy_t * n_replicas)()
    _check(load().md_energy(h, out), h)
    return [out[r].as_dict() for r in range(n_replicas)]


def md_rebin(h):
    _check(load().md_rebin(h), h)


def md_get_state(h, n_atoms: int):
    x = np.empty((n_atoms, 3)); v = np.empty((n_atoms, 3)); img = np.empty((n_atoms, 3), np.int32)
    _check(load().md_get_state(h, _p(x), _p(v), _p(img)), h)
    return x, v, img


def md_set_state(h, pos, vel):
    pos = np.ascontiguousarray(pos, np.float64); vel = np.ascontiguousarray(vel, np.float64)
    _check(load().md_set_state(h, _p(pos), _p(vel)), h)


def md_set_params(h, p: dict):
    q = make_params(p)
    _check(load().md_set_params(h, ctypes.byref(q)), h)


def md_set_temperature(h, T):
    T = np.ascontiguousarray(T, np.float64)
    _check(load().md_set_temperature(h, _p(T)), h)


def md_get_thermostat(h, n_replicas: int) -> np.ndarray:
    xi = np.zeros(n_replicas, np.float64)
    _check(load().md_get_thermostat(h, xi.ctypes.data), h)
    return xi


def md_stream(h) -> int:
    return load().md_stream(h) or 0


def md_info(h):
    n, c = ctypes.c_int64(), ctypes.c_int64()
    cap, M = ctypes.c_int32(), ctypes.c_int32()
    _check(load().md_info(h, ctypes.byref(n), ctypes.byref(c), ctypes.byref(cap), ctypes.byref(M)), h)
    return dict(n_atoms=n.value, n_cells=c.value, nbr_capacity=cap.value, cells_per_side=M.value)


def md_get_bins(h, n_atoms: int, n_cells: int):
    co = np.empty(n_atoms, np.int32); cs = np.empty(n_cells + 1, np.int32); pm = np.empty(n_atoms, np.int32)
    _check(load().md_get_bins(h, _p(co), _p(cs), _p(pm)), h)
    return co, cs, pm


def md_get_neighbors(h, n_atoms: int, cap: int):
    cnt = np.empty(n_atoms, np.int32); ent = np.zeros((n_atoms, cap), np.int32)
    _check(load().md_get_neighbors(h, _p(cnt), _p(ent)), h)
    return cnt, ent


def md_get_cell_units(h, n_atoms: int):
    u = np.empty((n_atoms, 3), np.float32)
    _check(load().md_get_cell_units(h, _p(u)), h)
    return u


def md_profile_enable(h, on: bool):
    _check(load().md_profile_enable(h, int(on)), h)


def md_profile_read(h):
    ms = np.zeros(5); n = np.zeros(5, np.int64)
    _check(load().md_profile_read(h, _p(ms), _p(n)), h)
    return ms, n


def md_profile_reset(h):
    _check(load().md_profile_reset(h), h)


def md_launches_per_call(h, n: int) -> int:
    return int(load().md_launches_per_call(h, n))


def md_bin_static(pos_dev: int, n_atoms: int, box: float, cells_per_side: int, cell_of_dev: int,
                  cell_start_dev: int, perm_dev: int, stream: int = 0):
    """Binning into caller DEVICE arrays (pointers as ints) with no device
    allocation; see include/md.h for limits and the shared-scratch rules."""
    _check(load().md_bin_static(ctypes.c_void_p(pos_dev), n_atoms, box, cells_per_side,
                                ctypes.c_void_p(cell_of_dev), ctypes.c_void_p(cell_start_dev),
                                ctypes.c_void_p(perm_dev), ctypes.c_void_p(stream)))


def md_destroy(h):
    if h:
        load().md_destroy(h)


def md_last_error(h=None) -> str:
    return load().md_last_error(h).decode()


def md_wait_selftest(spins: int = 1000) -> int:
    """Return code of the bounded-wait self-test (MD_ETIMEOUT when it works)."""
    return int(load().md_wait_selftest(int(spins)))


def md_adj_create(desc: md_adj_desc):
    h = ctypes.c_void_p()
    _check(load().md_adj_create(ctypes.byref(desc), ctypes.byref(h)))
    return h


def md_adj_set_theta(h, theta):
    th = np.ascontiguousarray(theta, np.float64).reshape(5)
    _check(load().md_adj_set_theta(h, _p(th)))


def md_adj_forward(h, pos, vel) -> np.ndarray:
    pos = np.ascontiguousarray(pos, np.float64); vel = np.ascontiguousarray(vel, np.float64)
    obs = np.zeros(2)
    _check(load().md_adj_forward(h, _p(pos), _p(vel), _p(obs)))
    return obs


def md_adj_backward(h, weight) -> np.ndarray:
    w = np.ascontiguousarray(weight, np.float64).reshape(2)
    g = np.zeros(5)
    _check(load().md_adj_backward(h, _p(w), _p(g)))
    return g


def md_adj_tangent(h, pos, direction):
    pos = np.ascontiguousarray(pos, np.float64); d = np.ascontiguousarray(direction, np.float64)
    gu = np.zeros_like(pos); hv = np.zeros_like(pos); dth = np.zeros(10)
    _check(load().md_adj_tangent(h, _p(pos), _p(d), _p(gu), _p(hv), _p(dth)))
    return gu, hv, dth[:5], dth[5:]


def md_adj_energy(h) -> dict:
    out = np.zeros(6)
    _check(load().md_adj_energy(h, _p(out)))
    return dict(lj_shifted=out[0], bond=out[1], angle=out[2], dihedral=out[3], r2_sum=out[4], U=out[5])


def md_adj_destroy(h):
    if h:
        load().md_adj_destroy(h)


# ---------------------------------------------------------------- convenience object

PROFILE_GROUPS = ("rebin", "nbr_build", "integrate", "lj", "bonded")


class System:
    """One or more periodic melts (replicas) stepped together on the GPU.

    `melts` is a dict or a list of dicts with keys pos (N,3), vel (N,3), L,
    n_chains, sites (the chaingen format).  Device memory is a torch uint8
    tensor handed to the library as its workspace; the library runs on a
    torch stream (`self.stream`).  The keyword arguments are the md_desc
    fields of include/md.h (lj_region, lj_block, lj_lanes and schedule shape
    the LJ kernel; lj_pair_exact=True rounds every LJ pair force once so that
    the LJ forces sum to exactly zero; displacement picks the policy for an
    atom that moved more than skin/2 between list builds).
    """

    def __init__(self, melts, precision: int = MD_MIXED, dt: float = 0.001, rc: float = 1.0,
                 skin: float = 0.1, rebin_every: int = 10, thermostat: int = MD_NVE, T_target=None,
                 tau_t: float = 0.1, params: dict | None = None, nbr_capacity: int = 0, device: int = 0,
                 use_torch_memory: bool = True, lj_block: int = 0, schedule: int = MD_SCHED_GRID,
                 lj_lanes: int = 0, autotune: bool = False, tune_cycles: int = 2, tune_cache: str | None = None,
                 topology=None, displacement: int = 0, lj_region: int = 0, lj_pair_exact: bool = False):
        import torch
        load()
        if isinstance(melts, dict):
            melts = [melts]
        self.melts = melts
        self.n_replicas = len(melts)
        self.sites = int(melts[0]["sites"])
        self.params = dict(default_params() if params is None else params)
        self._n_chains = np.array([m["n_chains"] for m in melts], np.int32)
        self._box = np.array([m["L"] for m in melts], np.float64)
        self._pos = np.ascontiguousarray(np.concatenate([m["pos"] for m in melts]), np.float64)
        self._vel = np.ascontiguousarray(np.concatenate([m["vel"] for m in melts]), np.float64)
        self.n_atoms = len(self._pos)
        self._T = None if T_target is None else np.ascontiguousarray(np.broadcast_to(
            np.asarray(T_target, np.float64), (self.n_replicas,)))
        self.device = torch.device("cuda", device)
        self.stream = torch.cuda.Stream(device=self.device)
        d = md_desc()
        d.n_replicas = self.n_replicas
        d.sites_per_chain = self.sites
        d.n_chains = _p(self._n_chains); d.box = _p(self._box)
        d.pos = _p(self._pos); d.vel = _p(self._vel)
        d.T_target = _p(self._T)
        d.params = make_params(self.params)
        d.dt, d.rc, d.skin, d.tau_t = dt, rc, skin, tau_t
        d.rebin_every, d.precision, d.thermostat = rebin_every, precision, thermostat
        d.nbr_capacity = nbr_capacity
        d.lj_block, d.schedule, d.lj_lanes = lj_block, schedule, lj_lanes
        d.lj_region = lj_region
        d.lj_pair_exact = 1 if lj_pair_exact else 0
        d.displacement = displacement
        if topology is not None:
            # (bonds [n_bonds, 2], types [naom]) of the molecule type (Sec. 3.3)
            self._tb = np.ascontiguousarray(np.asarray(topology[0], np.int32).reshape(-1, 2))
            self._tt = np.ascontiguousarray(np.asarray(topology[1], np.int32))
            self._topo = md_topology(len(self._tt), len(self._tb), _p(self._tb), _p(self._tt))
            d.topology = ctypes.cast(ctypes.pointer(self._topo), ctypes.c_void_p)
        self.tuning = md_autotune(d, tune_cycles, tune_cache) if autotune else None
        d.cuda_stream = self.stream.cuda_stream
        self.workspace = None
        if use_torch_memory:
            nbytes = md_workspace_size(d)
            self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
            addr = self.workspace.data_ptr()
            d.workspace = (addr + 255) // 256 * 256
            d.workspace_bytes = nbytes
        self.desc = d
        torch.cuda.synchronize(self.device)
        self.h = md_create(d)
        self.info = md_info(self.h)
        self.dt, self.rebin_every = dt, d.rebin_every

    def step(self, n: int, sync: bool = True):
        (md_step if sync else md_step_async)(self.h, n)

    def sync(self):
        md_sync(self.h)

    def forces(self):
        return md_forces(self.h, self.n_atoms)

    def energy(self):
        return md_energy(self.h, self.n_replicas)

    def rebin(self):
        md_rebin(self.h)

    def state(self):
        return md_get_state(self.h, self.n_atoms)

    def set_state(self, pos, vel):
        md_set_state(self.h, pos, vel)

    def set_params(self, p: dict):
        self.params = dict(p)
        md_set_params(self.h, p)

    def set_temperature(self, T):
        md_set_temperature(self.h, np.broadcast_to(np.asarray(T, np.float64), (self.n_replicas,)))

    def observables(self) -> dict:
        """Per chain: end-to-end vectors r_ee [n_chains, 3] and squared radii
        of gyration rg2 [n_chains]; per replica: trans_fraction, computed on
        the GPU from the current state."""
        n_ch = int(self._n_chains.sum())
        ree = np.zeros((n_ch, 3), np.float64)
        rg2 = np.zeros(n_ch, np.float64)
        tf = np.zeros(self.n_replicas, np.float64)
        _check(load().md_observables(self.h, ree.ctypes.data, rg2.ctypes.data, tf.ctypes.data), self.h)
        return {"r_ee": ree, "rg2": rg2, "trans_fraction": tf}

    def rdf(self, r_max: float, n_bins: int):
        """Radial distribution function of non-bonded site pairs, computed on
        the GPU (md_rdf): bin centres [n_bins], g(r) [n_replicas, n_bins] and
        the integer pair counts [n_replicas, n_bins].  Bins are
        numpy.linspace(0, r_max, n_bins + 1); g = counts / (n_pairs * shell /
        L^3) with n_pairs = N (N - 1) / 2 - n_chains (2 S - 3) per replica."""
        edges = np.linspace(0.0, float(r_max), int(n_bins) + 1)
        counts = np.zeros((self.n_replicas, int(n_bins)), np.int64)
        _check(load().md_rdf(self.h, int(n_bins), edges.ctypes.data, counts.ctypes.data), self.h)
        shell = 4.0 / 3.0 * np.pi * (edges[1:] ** 3 - edges[:-1] ** 3)
        g = np.zeros(counts.shape)
        S = self.sites
        for r in range(self.n_replicas):
            n = int(self._n_chains[r]) * S
            n_pairs = n * (n - 1) // 2 - int(self._n_chains[r]) * (2 * S - 3)
            L = float(self._box[r])
            g[r] = counts[r] / (n_pairs * shell / L ** 3)
        return 0.5 * (edges[1:] + edges[:-1]), g, counts

    def acf_reset(self, max_lag: int):
        _check(load().md_acf_reset(self.h, int(max_lag)), self.h)
        self._acf_lag = int(max_lag)

    def acf_sample(self):
        """Add the current end-to-end vectors as the next ACF sample (GPU)."""
        _check(load().md_acf_sample(self.h), self.h)

    def acf_push(self, r_ee):
        """Add a given sample of end-to-end vectors [n_chains, 3]."""
        r = np.ascontiguousarray(r_ee, np.float64).reshape(-1, 3)
        _check(load().md_acf_push(self.h, r.ctypes.data), self.h)

    def acf(self):
        """(C [n_replicas, max_lag + 1], number of samples)."""
        C = np.zeros((self.n_replicas, self._acf_lag + 1), np.float64)
        n = ctypes.c_int64(0)
        _check(load().md_acf_read(self.h, C.ctypes.data, ctypes.byref(n)), self.h)
        return C, int(n.value)

    def bin_study(self, reps: int = 5) -> dict:
        """CBIN-style host binning against the on-GPU counting sort
        (md_bin_study): mean ms per round of each part."""
        ms = np.zeros(6, np.float64)
        _check(load().md_bin_study(self.h, int(reps), ms.ctypes.data), self.h)
        keys = ("gpu_binning", "gpu_list_build", "host_position_copy", "host_binning", "host_binned_data_copy",
                "host_total")
        return dict(zip(keys, (float(v) for v in ms)))

    def early_rebins(self) -> int:
        """Rebuilds added by the displacement check so far."""
        n = ctypes.c_int64(0)
        _check(load().md_early_rebins(self.h, ctypes.byref(n)), self.h)
        return int(n.value)

    def thermostat_xi(self) -> np.ndarray:
        """Nose-Hoover friction xi (1/ps) of each replica (zeros for the
        other thermostats)."""
        return md_get_thermostat(self.h, self.n_replicas)

    def bins(self):
        return md_get_bins(self.h, self.n_atoms, self.info["n_cells"])

    def neighbors(self):
        return md_get_neighbors(self.h, self.n_atoms, self.info["nbr_capacity"])

    def close(self):
        if getattr(self, "h", None):
            md_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- adjoint

THETA_NAMES = ("eps_C32", "eps_C33", "sigma_C32", "sigma_C33", "k_phi")


class Adjoint:
    """FP64 NVE run of one melt on the GPU and the gradient of its trajectory
    means (<U>, <R_ee^2>) with respect to theta = (eps_C32, eps_C33,
    sigma_C32, sigma_C33, k_phi) by the library's adjoint kernels.

    `melt` is a chaingen-format dict; its positions may be wrapped into the
    box: md_adj_forward makes each chain continuous on the GPU (the
    end-to-end distance needs continuous chains)."""

    def __init__(self, melt: dict, n_steps: int = 500, checkpoint_every: int = 50, dt: float = 0.001,
                 rc: float = 1.0, params: dict | None = None, device: int | None = None, lj_form: int = 0,
                 hvp_fp32: bool = False):
        import torch
        if device is not None:
            torch.cuda.set_device(device)
        self.params = dict(default_params() if params is None else params)
        n_chains, sites, L = int(melt["n_chains"]), int(melt["sites"]), float(melt["L"])
        self.x0 = np.ascontiguousarray(melt["pos"], np.float64).reshape(-1, 3)
        self.v0 = np.ascontiguousarray(melt["vel"], np.float64).reshape(-1, 3)
        self.n_atoms = n_chains * sites
        desc = md_adj_desc()
        desc.n_chains, desc.sites_per_chain, desc.box = n_chains, sites, L
        desc.params = make_params(self.params)
        desc.rc, desc.dt, desc.n_steps, desc.checkpoint_every = rc, dt, n_steps, checkpoint_every
        desc.lj_form = int(lj_form)     # 1: force-shifted LJ, a variant outside the paper (gradient checks)
        desc.hvp_precision = 1 if hvp_fp32 else 0   # FP32 Hessian-vector products in the reverse pass
        self.stream = torch.cuda.Stream()
        desc.cuda_stream = self.stream.cuda_stream
        self.h = md_adj_create(desc)
        self.theta = np.array([*self.params["eps"], *self.params["sigma"], self.params["kphi"]], np.float64)
        self._forward_theta = None

    def forward(self, theta=None) -> np.ndarray:
        """(<U>, <R_ee^2>) at theta (default: the current one)."""
        if theta is not None:
            self.theta = np.array(theta, np.float64).reshape(5)
            md_adj_set_theta(self.h, self.theta)
        obs = md_adj_forward(self.h, self.x0, self.v0)
        self._forward_theta = self.theta.copy()
        return obs

    def backward(self, weight=(1.0, 0.0), theta=None) -> np.ndarray:
        """d(w0 <U> + w1 <R_ee^2>)/dtheta; reruns the forward pass first if
        the checkpoints are not those of theta."""
        if theta is not None and not np.array_equal(np.asarray(theta, np.float64), self.theta):
            self.forward(theta)
        if self._forward_theta is None or not np.array_equal(self._forward_theta, self.theta):
            self.forward()
        return md_adj_backward(self.h, weight)

    def tangent(self, pos, direction):
        """(dU/dx, H dir, dU/dtheta, d(dU/dx . dir)/dtheta) at pos."""
        return md_adj_tangent(self.h, pos, direction)

    def energy(self) -> dict:
        return md_adj_energy(self.h)

    def close(self):
        if getattr(self, "h", None):
            md_adj_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _md_adjoint_function():
    import torch

    class MDAdjoint(torch.autograd.Function):
        """theta (5,) float64 -> (<U>, <R_ee^2>) of an Adjoint's trajectory;
        backward runs the reverse pass for the incoming weights."""

        @staticmethod
        def forward(ctx, theta, adj):
            th = theta.detach().cpu().numpy().astype(np.float64)
            obs = adj.forward(th)
            ctx.adj, ctx.theta = adj, th
            return torch.tensor(obs, dtype=torch.float64)

        @staticmethod
        def backward(ctx, grad_out):
            w = grad_out.detach().cpu().numpy().astype(np.float64)
            g = ctx.adj.backward(w, theta=ctx.theta)
            return torch.tensor(g, dtype=torch.float64), None

    return MDAdjoint


def __getattr__(name):
    if name == "MDAdjoint":
        fn = _md_adjoint_function()
        globals()["MDAdjoint"] = fn
        return fn
    raise AttributeError(name)
