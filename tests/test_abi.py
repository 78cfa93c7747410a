"""C ABI: the library builds, loads and exports every entry point that
include/md.h declares; descriptor validation needs no GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

import chaingen
import paper_1001_3764_gb300 as md
from paper_1001_3764_gb300 import build as cuda_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "md.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(md_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    cuda_build.build()
    return md.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(md.EXPORTS)


def _desc(melt, **kw):
    d = md.md_desc()
    keep = []
    nc = np.array([melt["n_chains"]], np.int32); box = np.array([melt["L"]])
    pos = np.ascontiguousarray(melt["pos"]); vel = np.ascontiguousarray(melt["vel"])
    keep += [nc, box, pos, vel]
    d.n_replicas = 1; d.sites_per_chain = melt["sites"]
    d.n_chains = nc.ctypes.data; d.box = box.ctypes.data; d.pos = pos.ctypes.data; d.vel = vel.ctypes.data
    d.params = md.make_params(md.default_params())
    d.dt, d.rc, d.skin, d.tau_t, d.rebin_every = 0.001, 1.0, 0.1, 0.1, 10
    d.precision, d.thermostat = md.MD_MIXED, md.MD_NVE
    for k, v in kw.items():
        setattr(d, k, v)
    return d, keep


def test_workspace_size_without_gpu(lib):
    m = chaingen.melt(10, seed=1)
    d, keep = _desc(m)
    b = md.md_workspace_size(d)
    N = 1500
    assert b > N * (48 + 48 + 32 + 32)     # state + forces at least
    d2, keep2 = _desc(m, precision=md.MD_PLAIN_FP32)
    assert md.md_workspace_size(d2) < b


@pytest.mark.parametrize("field,value", [("dt", 0.0), ("rc", -1.0), ("rebin_every", 0), ("precision", 7),
                                         ("thermostat", 3), ("sites_per_chain", 2), ("n_replicas", 0),
                                         ("lj_block", 192), ("lj_lanes", 4), ("lj_region", 4), ("lj_pair_exact", 2),
                                         ("displacement", 5)])
def test_bad_descriptors_are_rejected(lib, field, value):
    m = chaingen.melt(10, seed=1)
    d, keep = _desc(m, **{field: value})
    with pytest.raises(md.MDError) as e:
        md.md_workspace_size(d)
    assert e.value.code == md.MD_EINVAL


def test_box_smaller_than_three_cells_is_rejected(lib):
    m = chaingen.melt(10, seed=1)
    d, keep = _desc(m)
    box = np.array([3.2]); keep.append(box); d.box = box.ctypes.data     # 3.2 < 3 * 1.1
    with pytest.raises(md.MDError) as e:
        md.md_create(d)
    assert e.value.code == md.MD_EINVAL
    assert "box" in md.md_last_error(None)


def test_thermostat_needs_targets(lib):
    m = chaingen.melt(10, seed=1)
    d, keep = _desc(m, thermostat=md.MD_VRESCALE)
    with pytest.raises(md.MDError):
        md.md_workspace_size(d)


def _adj_desc(**kw):
    d = md.md_adj_desc()
    d.n_chains, d.sites_per_chain, d.box = 4, 150, 3.4
    d.params = md.make_params(md.default_params())
    d.rc, d.dt, d.n_steps, d.checkpoint_every = 1.0, 0.001, 10, 5
    d.lj_form, d.hvp_precision = 0, 0
    for k, v in kw.items():
        setattr(d, k, v)
    return d


@pytest.mark.parametrize("field,value", [("hvp_precision", 2), ("hvp_precision", -1), ("lj_form", 3),
                                         ("n_chains", 0), ("n_steps", -1), ("checkpoint_every", 0),
                                         ("box", 0.0)])
def test_bad_adjoint_descriptors_are_rejected(lib, field, value):
    # validated before any CUDA call
    with pytest.raises(md.MDError) as e:
        md.md_adj_create(_adj_desc(**{field: value}))
    assert e.value.code == md.MD_EINVAL


def test_topology_descriptor_validation(lib):
    """md_desc.topology is checked before any GPU work: atom indices in
    range, no self or repeated bonds, types 0/1, naom equal to
    sites_per_chain, and the mixed precision form."""
    m = chaingen.melt(2, sites=6, seed=1, L=3.4)

    def size_with(bonds, types, naom=6, precision=md.MD_MIXED):
        b = np.ascontiguousarray(np.asarray(bonds, np.int32))
        t = np.ascontiguousarray(np.asarray(types, np.int32))
        topo = md.md_topology(naom, len(b) // 2, b.ctypes.data, t.ctypes.data)
        d, keep = _desc(m, precision=precision)
        d.topology = ctypes.cast(ctypes.pointer(topo), ctypes.c_void_p)
        sz = ctypes.c_size_t()
        return lib.md_workspace_size(ctypes.byref(d), ctypes.byref(sz)), keep, b, t, topo

    chain = [0, 1, 1, 2, 2, 3, 3, 4, 4, 5]
    ends = [1, 0, 0, 0, 0, 1]
    assert size_with(chain, ends)[0] == md.MD_OK
    assert size_with([0, 1, 1, 6], ends)[0] == md.MD_EINVAL          # atom out of range
    assert size_with([0, 0, 1, 2], ends)[0] == md.MD_EINVAL          # self bond
    assert size_with([0, 1, 1, 0], ends)[0] == md.MD_EINVAL          # repeated bond
    assert size_with(chain, [2, 0, 0, 0, 0, 1])[0] == md.MD_EINVAL   # unknown type
    assert size_with(chain, ends, naom=7)[0] == md.MD_EINVAL         # naom != sites_per_chain
    assert size_with(chain, ends, precision=md.MD_PLAIN_FP32)[0] == md.MD_EINVAL
