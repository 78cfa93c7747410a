"""Throughput of the united-atom polyethylene MD hot path on one GB300.

Workload (N = 1): a 0.77 g/cm^3 polyethylene melt of 10,000 chains x 150
united atoms (1.5M sites, L = 35.68 nm), r_c = 1.0 nm, skin 0.1 nm, neighbour
list rebuilt every 10 steps, dt = 1 fs, NVE velocity Verlet, mixed precision
(FP32 pair and bonded math, int64 fixed-point force sums, FP64 state).
One benchmark "step" is one pass of the whole hot path: rebin + neighbour list
+ 10 MD steps (one CUDA-graph launch).  Metric: atom-steps/s of MD steps.

Under torchrun (--gpus N > 1) every rank runs its own independent replica melt
(replicas only: the method has no exchange between independent systems), and
the value is the sum over ranks ("scaling": "weak").

--impl reference times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload (the slow reference arm of this build).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

MD_STEPS_PER_BENCH_STEP = 10
N_CHAINS = 10000
SITES = 150
DT_PS = 0.001
FLOP_PER_ATOM_LJ = 69.2 * 20.0       # unique pairs within r_c per atom x flops per pair (Newton-3 count)
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12   # SMs x FP32 lanes x 2 x max SM clock
WORKLOAD = ("PE melt 10,000 chains x 150 united atoms (1.5M sites), 0.77 g/cm3, L=35.68 nm, "
            "rc=1.0 nm, skin=0.1 nm, rebin every 10 steps, dt=1 fs, NVE velocity Verlet")


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    def __init__(self, index: int):
        self.index, self.proc, self.path = index, None, None

    def start(self):
        self.path = os.path.join("/tmp", f"bench_clocks_{os.getpid()}.csv")
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [c.strip() for c in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1])); mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _traffic(kernel_src: str):
    """DRAM bytes per LJ launch from the committed ncu summary, if the kernel
    source is unchanged since the capture (else None)."""
    path = os.path.join(ROOT, "profiles", "lj_dram_traffic.txt")
    if not os.path.exists(path):
        return None
    kv = {}
    for line in open(path):
        if "=" in line and not line.startswith("#"):
            k, v = line.split("=", 1)
            kv[k.strip()] = v.strip()
    h = hashlib.sha256(open(kernel_src, "rb").read()).hexdigest()[:16]
    if kv.get("source_sha256_16") != h:
        return None
    try:
        return float(kv["bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def replica_seed(rank: int) -> int:
    """Seed of rank r's replica melt: every rank steps an independent system."""
    return 3 + 1000 * rank


def make_workload(rank: int, chains: int = N_CHAINS):
    import chaingen
    return chaingen.melt(chains, SITES, seed=replica_seed(rank), T=500.0)


def max_over_ranks(x: float, ws: int) -> float:
    """The largest of x over all ranks (the slowest rank sets the time)."""
    if ws <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(ws: int, n_atoms_per_rank: int, md_steps: int, seconds: float) -> float:
    """Whole-job atom-steps/s: the units all ranks processed over the slowest rank's time."""
    return ws * n_atoms_per_rank * md_steps / seconds


def equilibrate(md, melts, rounds=6, steps=250, seed=11):
    """Untimed set-up.  The grown chains start with hard contacts (down to
    0.22 nm); the energy they release lands in the bond and angle vibrations
    of the last-grown chains, which a global thermostat drains only slowly.
    So: `rounds` x (`steps` steps of the weak-coupling thermostat at each
    melt's T, neighbour list every 2 steps, then fresh Maxwell velocities),
    which removes the kinetic half of any hot mode's excess per round."""
    import chaingen
    single = isinstance(melts, dict)
    melts = [melts] if single else list(melts)
    T0 = [m["T"] for m in melts]
    eq = md.System(melts, precision=md.MD_MIXED, thermostat=md.MD_VRESCALE, T_target=T0, tau_t=0.05,
                   rebin_every=2)
    for r in range(rounds):
        eq.step(steps)
        x, _, _ = eq.state()
        v = np.concatenate([chaingen.maxwell(m["masses"], m["T"], seed + 7919 * k, stream=100 + r)
                            for k, m in enumerate(melts)])
        eq.set_state(x, v)
    eq.step(steps)
    x, v, _ = eq.state()
    eq.close()
    off, out = 0, []
    for m in melts:
        n = len(m["pos"])
        out.append(dict(m, pos=x[off:off + n], vel=v[off:off + n]))
        off += n
    return out[0] if single else out


def _slope(t_ps, e, T, n_atoms):
    tn = np.asarray(t_ps) * 1e-3                                   # ns
    e = np.asarray(e)
    coef, cov = np.polyfit(tn, e, 1, cov=True)                     # kJ/mol per ns
    norm = 0.0083144626 * float(np.mean(T)) * n_atoms
    return float(coef[0] / norm), float(np.sqrt(cov[0, 0]) / norm)


def drift(md, n_chains=1000, relax_ps=150, mixed_ps=200, plain_ps=50, window_ps=50, every_ps=1.0):
    """NVE energy drift (least-squares slope of the total energy with shifted
    LJ) in kT per atom per ns, on the 150k-site melt (1,000 chains, seed 2).
    After the thermostat set-up the melt warms by ~25 K over its first ~150 ps
    of NVE (most of it in the first 50 ps), and while it warms the total
    energy moves with the velocity-Verlet shadow-energy offset (it scales as
    dt^2); so NVE runs relax_ps first, then both forms start from the same
    relaxed state."""
    import chaingen
    m = equilibrate(md, chaingen.melt(n_chains, SITES, seed=2, T=500.0))
    n = len(m["pos"])
    per = int(round(every_ps / DT_PS))
    s = md.System(m, precision=md.MD_MIXED)
    try:
        s.step(int(round(relax_ps / DT_PS)))
        x, v, img = s.state()
        relaxed = dict(m, pos=x + img * m["L"], vel=v)
        out = {"sites": n, "relax_ps": relax_ps, "every_ps": every_ps}
        for name, prec, total_ps in (("mixed", md.MD_MIXED, mixed_ps), ("plain", md.MD_PLAIN_FP32, plain_ps)):
            q = s if name == "mixed" else md.System(relaxed, precision=prec)
            t, e, T = [], [], []
            nsamp = int(round(total_ps / every_ps))
            for k in range(nsamp + 1):
                en = q.energy()[0]
                t.append(k * every_ps); e.append(en["total"]); T.append(en["temperature"])
                if k < nsamp:
                    q.step(per)
            d, se = _slope(t, e, T, n)
            w = int(round(window_ps / every_ps))
            wins = [_slope(t[i:i + w + 1], e[i:i + w + 1], T[i:i + w + 1], n)[0] for i in range(0, nsamp, w)]
            wT = [float(np.mean(T[i:i + w + 1])) for i in range(0, nsamp, w)]
            out[name] = {"kT_per_atom_per_ns": d, "stderr": se, "window_ps": total_ps, "T_mean": float(np.mean(T)),
                         "per_50ps_window": wins, "per_50ps_window_T": wT}
            if q is not s:
                q.close()
        out["note"] = ("stderr assumes independent samples (an underestimate for correlated energy "
                       "fluctuations); the mixed and plain runs start from the same relaxed state")
        return out
    except md.MDError as err:
        return {"error": str(err)}
    finally:
        s.close()


def batched(md, cycles=5):
    """Config 4: 64 independent melts of 20..400 chains (log-uniform, seed 4)
    quenched at T0 ~ U(250, 500) K, mixed form, all replicas in the same
    graph-captured launches, LJ block shape / schedule / cell size chosen by
    md_autotune.  Compared with the same replicas stepped one system at a time."""
    import torch
    import chaingen
    melts = chaingen.replicas(64, seed=4)
    T0 = [m["T"] for m in melts]
    ms = equilibrate(md, melts, rounds=4)
    n_atoms = sum(len(m["pos"]) for m in ms)
    cache = os.path.join("/tmp", "md_autotune_cache.txt")
    s = md.System(ms, precision=md.MD_MIXED, thermostat=md.MD_VRESCALE, T_target=T0, tau_t=0.1,
                  autotune=True, tune_cycles=2, tune_cache=cache)
    R = s.rebin_every
    st = torch.cuda.ExternalStream(md.md_stream(s.h))
    s.step(2 * R)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(st)
    s.step(cycles * R, sync=False)
    b.record(st)
    s.sync()
    torch.cuda.synchronize()
    t_batched = a.elapsed_time(b) * 1e-3
    temps = [e["temperature"] for e in s.energy()]
    tuning = dict(s.tuning)
    s.close()
    def timed(system):
        system.step(R)
        qs = torch.cuda.ExternalStream(md.md_stream(system.h))
        torch.cuda.synchronize()
        a.record(qs)
        system.step(cycles * R, sync=False)
        b.record(qs)
        system.sync()
        torch.cuda.synchronize()
        return a.elapsed_time(b) * 1e-3

    # the same replicas one system at a time (mixed, same settings; and plain FP32)
    t_seq = {md.MD_MIXED: 0.0, md.MD_PLAIN_FP32: 0.0}
    for prec in t_seq:
        for m, T in zip(ms, T0):
            q = md.System(m, precision=prec, thermostat=md.MD_VRESCALE, T_target=T, tau_t=0.1,
                          skin=tuning["skin"], rebin_every=R, lj_block=tuning["lj_block"],
                          schedule=tuning["schedule"], lj_lanes=tuning["lj_lanes"], lj_region=tuning["lj_region"])
            t_seq[prec] += timed(q)
            q.close()
    # one plain FP32 melt with the same total number of chains
    big = equilibrate(md, chaingen.melt(sum(m["n_chains"] for m in ms), SITES, seed=4, T=400.0), rounds=2)
    q = md.System(big, precision=md.MD_PLAIN_FP32, skin=tuning["skin"], rebin_every=R,
                  lj_block=tuning["lj_block"], schedule=tuning["schedule"], lj_lanes=tuning["lj_lanes"],
                  lj_region=tuning["lj_region"])
    t_big = timed(q)
    n_big = len(big["pos"])
    q.close()
    steps = cycles * R
    return {"value": n_atoms * steps / t_batched, "unit": "atom-steps/s", "replicas": len(ms), "sites": n_atoms,
            "md_steps": steps, "sequential_value": n_atoms * steps / t_seq[md.MD_MIXED],
            "speedup_vs_sequential": t_seq[md.MD_MIXED] / t_batched,
            "sequential_plain_fp32_value": n_atoms * steps / t_seq[md.MD_PLAIN_FP32],
            "one_plain_fp32_melt_value": n_big * steps / t_big, "one_plain_fp32_melt_sites": n_big,
            "tuning": tuning, "T_final_range": [float(min(temps)), float(max(temps))]}


def adjoint(md, n_chains=50, K=500, C=50, reps=3):
    """Adjoint configuration: 50 chains x 150 sites (7,500 sites, L = 6.10
    nm), 500 NVE steps in FP64, checkpoints every 50 steps; gradient of
    (<U>, <R_ee^2>) with respect to (eps, sigma, k_phi).  Wall time of the
    synchronous forward and reverse calls (median of `reps`)."""
    import chaingen
    melt = equilibrate(md, chaingen.melt(n_chains, SITES, seed=5, T=500.0))
    adj = md.Adjoint(melt, n_steps=K, checkpoint_every=C)
    adj.forward(); adj.backward((1.0, 0.0))          # warm-up
    tf, tb = [], []
    for _ in range(reps):
        t0 = time.perf_counter(); obs = adj.forward(); t1 = time.perf_counter()
        g = adj.backward((1.0, 0.0)); t2 = time.perf_counter()
        tf.append(t1 - t0); tb.append(t2 - t1)
    adj.close()
    # the same with FP32 Hessian-vector products in the reverse pass
    adj32 = md.Adjoint(melt, n_steps=K, checkpoint_every=C, hvp_fp32=True)
    adj32.forward(); adj32.backward((1.0, 0.0))
    tb32 = []
    for _ in range(reps):
        t1 = time.perf_counter(); g32 = adj32.backward((1.0, 0.0)); tb32.append(time.perf_counter() - t1)
    adj32.close()
    n = n_chains * SITES
    f, b, b32 = float(np.median(tf)), float(np.median(tb)), float(np.median(tb32))
    return {"sites": n, "steps": K, "checkpoint_every": C, "forward_ms": f * 1e3, "backward_ms": b * 1e3,
            "gradient_atom_steps_per_s": n * K / (f + b), "obs": [float(o) for o in obs],
            "grad_U": dict(zip(md.THETA_NAMES, [float(x) for x in g])),
            "backward_ms_fp32_hvp": b32 * 1e3,
            "fp32_hvp_max_rel_diff": float(np.max(np.abs(g32 - g)) / np.max(np.abs(g))),
            "note": "FP64 state and adjoint; backward recomputes each 50-step segment from its checkpoint; "
                    "the fp32_hvp figures run the reverse pass's Hessian-vector products in FP32"}


def nvt_nose_hoover(md, melt, bench_steps=20):
    """The paper's NVT ensemble on the benchmark melt: Leap-Frog with
    Nose-Hoover coupling at 500 K (tau 0.1 ps) and centre-of-mass removal,
    mixed form, timed like the NVE loop (graph launches of one rebin cycle,
    CUDA events on the library's stream).  Outside the headline numbers; an
    error is reported instead of raised."""
    import torch
    try:
        s = md.System(melt, precision=md.MD_MIXED, thermostat=md.MD_NOSE_HOOVER, T_target=500.0, tau_t=0.1)
        try:
            st = torch.cuda.ExternalStream(md.md_stream(s.h))
            for _ in range(3):
                s.step(MD_STEPS_PER_BENCH_STEP)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record(st)
            for _ in range(bench_steps):
                s.step(MD_STEPS_PER_BENCH_STEP, sync=False)
            b.record(st)
            s.sync()
            torch.cuda.synchronize()
            ms = a.elapsed_time(b)
            n, steps = len(melt["pos"]), bench_steps * MD_STEPS_PER_BENCH_STEP
            return {"value": n * steps / (ms * 1e-3), "unit": "atom-steps/s", "ms_per_bench_step": ms / bench_steps,
                    "md_steps": steps, "T_end": float(s.energy()[0]["temperature"]),
                    "xi_end": float(s.thermostat_xi()[0])}
        finally:
            s.close()
    except Exception as err:   # noqa: BLE001 -- a side measurement must not lose the headline line
        return {"error": f"{type(err).__name__}: {err}"}


# Table III of the paper: box volumes (nm^3) and site counts of its seven
# test systems.  The engine's boxes are cubes, so each is run in the cube of
# the same volume and the same number of 150-site chains (~0.25 g/cm^3).
TABLE3 = (("I", 10 * 10 * 16, 19200), ("II", 16 * 16 * 24, 64800), ("III", 20 * 20 * 32, 117600),
          ("IV", 24 * 24 * 40, 243000), ("V", 30 * 30 * 40, 363000), ("VI", 34 * 34 * 40, 507000),
          ("VII", 40 * 40 * 40, 675000))


def binning_study(md, reps=5):
    """The paper's binning and neighbour-list study (Sec. 4.1, Tables IV and
    V) on GB300: for each Table III system, the CBIN arm (positions copied to
    the host, binned there on one thread, binned data copied back) against
    the on-GPU counting sort, and the list build (md_bin_study, mean of
    `reps` rounds, ms).  Mixed form, generated melts (no equilibration)."""
    import chaingen
    out = []
    for name, vol, n in TABLE3:
        chains = n // SITES
        L = vol ** (1.0 / 3.0)
        m = chaingen.melt(chains, SITES, seed=100 + chains, T=500.0, L=L)
        s = md.System(m, precision=md.MD_MIXED)
        t = s.bin_study(reps)
        s.close()
        out.append(dict(system=name, sites=chains * SITES, L_nm=round(m["L"], 4), **{k: round(v, 4) for k, v in t.items()},
                        host_over_gpu=t["host_total"] / t["gpu_binning"]))
    return {"unit": "ms", "reps": reps, "systems": out,
            "note": "cubes of the Table III volumes; host binning on one thread of the GPU box's host"}


def cpu_baseline(melt, steps=4, steps_1t=1):
    """The CPU-baseline leg: the FP64 oracle (cell list) on the host cores,
    `steps` velocity-Verlet steps of the benchmark melt's generated state with
    OpenMP on every core, and `steps_1t` step on one thread (steps + 1 force
    evaluations each)."""
    import oracle
    cores = os.cpu_count() or 1
    n = len(melt["pos"])
    out = {}
    for nt, k in ((cores, steps), (1, steps_1t)):
        ref = oracle.System(oracle.chain_topology(SITES), melt["n_chains"], melt["L"], use_cells=True, nthreads=nt)
        t0 = time.perf_counter()
        ref.run(melt["pos"], melt["vel"], DT_PS, k, sample_every=0)
        el = time.perf_counter() - t0
        out[nt] = (n * k / el, k, el)
    v, k, el = out[cores]
    v1, k1, el1 = out[1]
    return {"value": v, "unit": "atom-steps/s", "cores": cores, "kind": "oracle",
            "sample": f"{k} velocity-Verlet steps ({k + 1} force evaluations) of the {n}-site melt, "
                      f"FP64 cell-list oracle, OpenMP {cores} threads, {el:.1f} s",
            "one_thread": {"value": v1, "unit": "atom-steps/s", "cores": 1,
                           "sample": f"{k1} velocity-Verlet step ({k1 + 1} force evaluations) of the same melt, "
                                     f"1 thread, {el1:.1f} s"}}


def oracle_sampled_forces(melt, precision_fp32: bool, n_sample=48, seed=0):
    """Part of the CPU-baseline leg: the FP64 oracle's total force (LJ summed
    over all atoms, orc_lj_atoms, plus the bonded terms) on `n_sample` atoms
    of the generated melt, as the GPU holds it after upload (FP64, or rounded
    to FP32 for the plain form)."""
    import oracle
    x = np.array(melt["pos"], np.float64)
    if precision_fp32:
        x = x.astype(np.float32).astype(np.float64)
    rng = np.random.default_rng(seed)
    sel = np.sort(rng.choice(len(x), n_sample, replace=False))
    ref = oracle.System(oracle.chain_topology(SITES), melt["n_chains"], melt["L"], use_cells=True,
                        nthreads=os.cpu_count() or 1)
    return sel, ref.lj_atoms(x, sel) + ref.bonded(x)[0][sel]


def force_error(md, melt, sampled):
    """Per-result error of the GPU forces at 1.5M sites against the FP64
    oracle, both forms: sampled atoms of the generated state (no GPU-produced
    input reaches the oracle).  rel_rms = ||F - F_orc||_2 / ||F_orc||_2 over
    the sample; max_rel = max over atoms of max|F - F_orc| / RMS|F_orc|."""
    out = {}
    for name, prec in (("mixed", md.MD_MIXED), ("plain", md.MD_PLAIN_FP32)):
        sel, f_orc = sampled[name]
        s = md.System(melt, precision=prec)
        f = s.forces()[sel]
        s.close()
        scale = float(np.sqrt(np.mean(np.sum(f_orc ** 2, axis=1))))
        out[name] = {"rel_rms": float(np.sqrt(np.sum((f - f_orc) ** 2) / np.sum(f_orc ** 2))),
                     "max_rel": float(np.abs(f - f_orc).max() / scale), "atoms": int(len(sel))}
    out["note"] = ("generated (unrelaxed) 1.5M-site melt, seed 3; LJ over all atoms within r_c plus bonded "
                   "terms, FP64 oracle; sample drawn with numpy default_rng(0)")
    return out


def drift_headline(md, melt, steps=2000, every=20):
    """NVE energy drift at the headline configuration (1.5M sites, 2,000
    steps of 1 fs after the set-up), both forms from the same state: slope of
    the total energy (shifted LJ) sampled every `every` steps, in kT per atom
    per ns.  A 2 ps window resolves drifts far above the 1e-4 target only;
    the 150k-site 200 ps protocol (drift_kT_per_atom_per_ns) resolves it."""
    out = {"steps": steps, "every": every}
    for name, prec in (("mixed", md.MD_MIXED), ("plain", md.MD_PLAIN_FP32)):
        try:
            s = md.System(melt, precision=prec)
            t, e, T = [], [], []
            for k in range(steps // every + 1):
                en = s.energy()[0]
                t.append(k * every * DT_PS); e.append(en["total"]); T.append(en["temperature"])
                if k < steps // every:
                    s.step(every)
            s.close()
            d, se = _slope(t, e, T, len(melt["pos"]))
            out[name] = {"kT_per_atom_per_ns": d, "stderr": se, "T_mean": float(np.mean(T))}
        except md.MDError as err:
            out[name] = {"error": str(err)}
    return out


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    melt = make_workload(0)
    import oracle
    cores = os.cpu_count() or 1
    ref = oracle.System(oracle.chain_topology(SITES), melt["n_chains"], melt["L"], use_cells=True, nthreads=cores)
    x, v = melt["pos"], melt["vel"]
    ref.run(x, v, DT_PS, 0, sample_every=0)            # warm-up: one force evaluation
    t0 = time.perf_counter()
    ref.run(x, v, DT_PS, args.steps, sample_every=0)   # one MD step per bench step
    el = time.perf_counter() - t0
    n = len(x)
    value = n * args.steps / el
    cb = {"value": value, "unit": "atom-steps/s", "cores": cores, "kind": "oracle",
          "sample": f"{args.steps} velocity-Verlet steps ({args.steps + 1} force evaluations) of the "
                    f"{n}-site melt, FP64 cell-list oracle, OpenMP {cores} threads"}
    print(json.dumps({"impl": "reference", "metric": "atom-steps/s", "value": value, "unit": "atom-steps/s",
                      "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                      "ms_per_step": el / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
                      "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                      "config": {"workload": WORKLOAD, "sites": n, "md_steps_per_bench_step": 1},
                      "cpu_baseline": cb,
                      "e2e": {"value": value, "unit": "atom-steps/s", "h2d_bytes_per_step": 0,
                              "d2h_bytes_per_step": 0}}), flush=True)


def run_gpu(args):
    import torch
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    import paper_1001_3764_gb300 as md

    melt = equilibrate(md, make_workload(rank, args.chains))
    n_atoms = len(melt["pos"])

    if args.ncu_energy:
        # the kernels of md_energy (energy-form forces, reductions, kinetic
        # energy) inside cudaProfilerStart/Stop, for a launch list
        s = md.System(melt, precision=md.MD_MIXED)
        s.step(MD_STEPS_PER_BENCH_STEP)
        s.energy()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        torch.cuda.profiler.start()
        for _ in range(args.steps):
            s.energy()
        torch.cuda.profiler.stop()
        el = time.perf_counter() - t0
        s.close()
        if rank == 0:
            print(json.dumps({"ncu_energy": True, "calls": args.steps, "ms_per_call": el / args.steps * 1e3,
                              "sites": n_atoms}), flush=True)
        return

    results = {}
    forms = (("mixed", md.MD_MIXED),) if args.ncu_region else (("mixed", md.MD_MIXED), ("plain", md.MD_PLAIN_FP32))
    for name, prec in forms:
        # MD_DISP_ERROR: step graphs without conditional nodes (a profiler can
        # take them apart); the equilibrated melt never moves an atom more
        # than skin/2 between list builds, so the work is the same as with the
        # default early-rebuild policy, whose throughput is reported beside
        s = md.System(melt, precision=prec, displacement=md.MD_DISP_ERROR)
        st = torch.cuda.ExternalStream(md.md_stream(s.h))
        for _ in range(args.warmup):
            s.step(MD_STEPS_PER_BENCH_STEP)
        md.md_profile_enable(s.h, True)
        md.md_profile_reset(s.h)
        clocks = ClockSampler(local)
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        clocks.start()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if args.ncu_region:
            torch.cuda.profiler.start()
        a.record(st)
        for _ in range(args.steps):
            s.step(MD_STEPS_PER_BENCH_STEP, sync=False)
        b.record(st)
        s.sync()
        if args.ncu_region:
            torch.cuda.profiler.stop()
        torch.cuda.synchronize()
        ck = clocks.stop()
        ms = max_over_ranks(a.elapsed_time(b), ws)
        prof_ms, prof_n = md.md_profile_read(s.h)
        md.md_profile_enable(s.h, False)
        launches = md.md_launches_per_call(s.h, MD_STEPS_PER_BENCH_STEP) * args.steps
        results[name] = dict(ms=ms, clocks=ck, prof_ms=prof_ms, prof_n=prof_n, launches=launches)
        if name == "mixed" and not args.ncu_region:
            # end to end through the public API with host buffers: upload the
            # state from pinned host memory, run one cycle, read the energies
            pos_h = torch.from_numpy(np.ascontiguousarray(melt["pos"])).pin_memory().numpy()
            vel_h = torch.from_numpy(np.ascontiguousarray(melt["vel"])).pin_memory().numpy()
            s.set_state(pos_h, vel_h)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(args.steps):
                s.set_state(pos_h, vel_h)
                s.step(MD_STEPS_PER_BENCH_STEP)
                s.energy()
            e2e_s = max_over_ranks(time.perf_counter() - t0, ws)
            results[name]["e2e_s"] = e2e_s
            results[name]["e2e_h2d"] = pos_h.nbytes + vel_h.nbytes
            results[name]["e2e_d2h"] = ctypes_size_energy(md)
        s.close()

    if args.ncu_region:
        if rank == 0:
            m = results["mixed"]
            print(json.dumps({"ncu_region": True, "ms_per_step": m["ms"] / args.steps, "sites": n_atoms,
                              "launches": int(m["launches"])}), flush=True)
        return
    # the same loop with the default policy (a conditional early rebuild per step)
    if not args.ncu_region:
        s = md.System(melt, precision=md.MD_MIXED)
        st = torch.cuda.ExternalStream(md.md_stream(s.h))
        for _ in range(args.warmup):
            s.step(MD_STEPS_PER_BENCH_STEP)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(st)
        for _ in range(args.steps):
            s.step(MD_STEPS_PER_BENCH_STEP, sync=False)
        b.record(st)
        s.sync()
        torch.cuda.synchronize()
        ms_reb = max_over_ranks(a.elapsed_time(b), ws)
        results["rebuild_policy"] = dict(ms=ms_reb, early=s.early_rebins())
        s.close()
    # everything below runs outside the timed region, on rank 0
    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return
    # energy drift of both forms on the 150k-site melt, and over 2,000 steps at 1.5M
    dr = drift(md)
    dr_1p5 = drift_headline(md, melt)
    m = results["mixed"]
    md_steps = MD_STEPS_PER_BENCH_STEP * args.steps
    value = aggregate_rate(ws, n_atoms, md_steps, m["ms"] * 1e-3)
    plain_value = aggregate_rate(ws, n_atoms, md_steps, results["plain"]["ms"] * 1e-3)
    ns_day = md_steps / (m["ms"] * 1e-3) * DT_PS * 1e-3 * 86400
    lj_ms = m["prof_ms"][3] / max(m["prof_n"][3], 1)
    achieved = FLOP_PER_ATOM_LJ * n_atoms / (lj_ms * 1e-3) / 1e12
    src = os.path.join(ROOT, "paper_1001_3764_gb300", "csrc", "k_lj.cu")
    traffic = _traffic(src)
    e2e_val = aggregate_rate(ws, n_atoms, md_steps, m["e2e_s"])
    out = {
        "metric": "atom-steps/s", "value": value, "unit": "atom-steps/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": m["ms"] / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+i64+f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sites": n_atoms, "md_steps_per_bench_step": MD_STEPS_PER_BENCH_STEP,
                   "precision": "mixed (FP32 pair/bonded math, int64 fixed-point forces, FP64 state)",
                   "l2": "inputs larger than L2 (cluster lists ~0.8 GB allocated, ~50 MB read per step; state and "
                         "forces ~150 MB)",
                   "displacement_policy": "MD_DISP_ERROR (no early rebuild needed on the equilibrated melt)",
                   "parallelism": f"replicas x{ws}" if ws > 1 else "1 GPU"},
        "ns_per_day": ns_day,
        "plain_fp32": {"value": plain_value,
                       "ns_per_day": md_steps / (results["plain"]["ms"] * 1e-3) * DT_PS * 1e-3 * 86400,
                       "ms_per_step": results["plain"]["ms"] / args.steps},
        "drift_kT_per_atom_per_ns": ({k: dr[k]["kT_per_atom_per_ns"] for k in ("mixed", "plain")}
                                     if "mixed" in dr else None),
        "drift_1p5M_2000_steps": dr_1p5,
        "displacement_rebuild_policy": {
            "value": aggregate_rate(ws, n_atoms, md_steps, results["rebuild_policy"]["ms"] * 1e-3),
            "ms_per_step": results["rebuild_policy"]["ms"] / args.steps,
            "early_rebuilds": results["rebuild_policy"]["early"],
            "note": "same loop with the default MD_DISP_REBUILD policy (a displacement check and a conditional "
                    "list rebuild in every step graph); the headline uses MD_DISP_ERROR, whose graphs ncu can "
                    "profile, with the same work on this melt"},
        "roofline": {"kernel": "k_cl_force (LJ force, Eq. 2)", "bound": "alu", "achieved": achieved,
                     "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP32_PEAK_TFLOPS,
                     "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz",
                     "flop_per_atom": FLOP_PER_ATOM_LJ, "traffic": traffic},
        "e2e": {"value": e2e_val, "unit": "atom-steps/s", "h2d_bytes_per_step": m["e2e_h2d"],
                "d2h_bytes_per_step": m["e2e_d2h"]},
        "gpu_launches": int(m["launches"]),
        "clocks": m["clocks"],
    }
    if ws == 1 and not args.no_cpu_baseline:
        # the CPU-baseline leg: the oracle timed on the host cores, and its
        # sampled forces for the per-result error of both GPU forms
        gen = make_workload(rank, args.chains)
        out["cpu_baseline"] = cpu_baseline(gen)
        sampled = {"mixed": oracle_sampled_forces(gen, False), "plain": oracle_sampled_forces(gen, True)}
        out["force_err"] = force_error(md, gen, sampled)
    out["kernel_ms_per_launch"] = {g: float(t / max(n, 1)) for g, t, n in
                                   zip(md.PROFILE_GROUPS, m["prof_ms"], m["prof_n"])}
    if not args.no_binning_study:
        out["binning_study"] = binning_study(md)
    if not args.no_batched:
        out["batched"] = batched(md)
    if not args.no_adjoint:
        out["adjoint"] = adjoint(md)
    out["nvt_nose_hoover"] = nvt_nose_hoover(md, melt)
    out["drift_detail"] = dr
    print(json.dumps(out), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def ctypes_size_energy(md):
    import ctypes
    return ctypes.sizeof(md.md_energy_t)


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=50)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-batched", action="store_true", help="skip the 64-replica measurement")
    p.add_argument("--no-adjoint", action="store_true", help="skip the adjoint-gradient measurement")
    p.add_argument("--no-binning-study", action="store_true", help="skip the Table III binning study")
    p.add_argument("--chains", type=int, default=N_CHAINS, help="chains of 150 sites (default 10,000 = 1.5M sites)")
    p.add_argument("--ncu-region", action="store_true",
                   help="profile only the timed loop of the mixed form (cudaProfilerStart/Stop); "
                        "skips the plain form, e2e, drift and CPU baseline")
    p.add_argument("--ncu-energy", action="store_true",
                   help="profile only `steps` md_energy calls on the mixed form (cudaProfilerStart/Stop), "
                        "then exit")
    args = p.parse_args()
    if args.warmup < 3:
        p.error("--warmup must be at least 3 (untimed warm-up steps before the timed region)")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
