"""Host-side arithmetic of bench.py (CPU): the drift slope's units and the
DRAM-traffic lookup that the roofline object reports."""
import hashlib
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

KB = 0.0083144626   # kJ/mol/K


def test_drift_slope_is_in_kT_per_atom_per_ns():
    # a total energy rising by exactly 1e-4 kT per atom per ns at T = 500 K,
    # sampled every 1 ps over 200 ps (the units the drift measurement uses)
    n_atoms, T = 150000, 500.0
    per_ps = 1e-4 * KB * T * n_atoms / 1000.0          # kJ/mol per ps
    t = np.arange(201, dtype=float)
    e = -2.5e6 + per_ps * t
    d, se = bench._slope(t, e, np.full_like(t, T), n_atoms)
    assert d == pytest.approx(1e-4, rel=1e-9)
    assert se < 1e-12
    # the temperature that sets kT is the mean of the samples
    d2, _ = bench._slope(t, e, np.linspace(400.0, 600.0, t.size), n_atoms)
    assert d2 == pytest.approx(1e-4, rel=1e-9)
    # and the sign follows the energy
    d3, _ = bench._slope(t, e[::-1], np.full_like(t, T), n_atoms)
    assert d3 == pytest.approx(-1e-4, rel=1e-9)


def test_traffic_is_reported_only_for_the_captured_source(tmp_path, monkeypatch):
    src = tmp_path / "k_lj.cu"
    src.write_text("// kernel source\n")
    h = hashlib.sha256(src.read_bytes()).hexdigest()[:16]
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "lj_dram_traffic.txt").write_text(f"# note\nbytes_per_launch = 123456\nsource_sha256_16 = {h}\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench._traffic(str(src)) == 123456.0
    src.write_text("// changed kernel\n")
    assert bench._traffic(str(src)) is None
