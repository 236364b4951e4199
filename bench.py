#!/usr/bin/env python3
"""Benchmark of the SU(2) heat-bath Monte Carlo on GB300.

Workload (one "step"): the 64^4 FP32 configuration -- hot start, 100
checkerboard heat-bath sweeps each followed by the plaquette and Polyakov
loop, then 25 APE smearing steps (alpha = 0.7) and Wilson loops W(R,T) for
R, T = 1..16 on the smeared spatial links.  Every step of it runs in libsu2's
kernels.  Metric: heat-bath link updates per second (100 x 4V per step).
The links (1.07 GB) are larger than L2 (129 MB), so no L2 flush is needed
between steps.

Printed as one JSON line (rank 0), with:
  roofline      the heat-bath substep kernel (the dominant one): algorithmic
                bytes per launch over its CUDA-event launch time, against the
                measured HBM copy bandwidth of MEASURED_PEAKS.json;
  cpu_baseline  the plain FP64 CPU oracle on this host, one substep of the
                same 64^4 lattice (rank 0 at N = 1 only);
  e2e           the same metric through the public API starting from a host
                configuration in pinned memory (H2D and results D2H inside the
                timed region);
  fp64 / f16q / batched / sweep_only   sub-measurements beside the FP32 path.

`--impl reference` times the CPU oracle as it stands (each step one
heat-bath substep of the same 64^4 lattice) and prints the same line shape.
Multi-GPU (torchrun): independent replicas, one lattice per rank (the
method's lattices do not shard here), weak scaling, max time over ranks.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "heat-bath link updates/s"
UNIT = "link updates/s"
DIMS = (64, 64, 64, 64)
BETA = 2.6
SWEEPS = 100
APE_STEPS, APE_ALPHA = 25, 0.7
RMAX = TMAX = 16
WORKLOAD = "su2_64^4_f32_beta2.6_hot_100sweeps_plaq_poly_ape25_W16x16"
PREC = "f32"
BATCH_SHAPES = [(8, 8, 8, 8)] * 16 + [(12, 12, 12, 12)] * 16 + [(16, 16, 16, 16)] * 16 + [(24, 24, 24, 6)] * 16


def volume(d):
    v = 1
    for x in d:
        v *= x
    return v


def config(n):
    return {"workload": WORKLOAD, "lattice": "x".join(map(str, DIMS)), "beta": BETA, "start": "hot",
            "links": "f32", "reductions": "f64", "sweeps_per_step": SWEEPS, "ape": [APE_STEPS, APE_ALPHA],
            "wilson": [RMAX, TMAX], "sampler": "kennedy-pendleton, max_tries 64",
            "l2": "inputs larger than L2 (1.07 GB links vs 129 MB L2), no flush",
            "parallelism": "replicas%d" % n if n > 1 else "single"}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    return ws, int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0"))


# ---------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_id):
        self.proc = None
        self.dev = device_id

    def start(self):
        try:
            cmd = ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits", "-lms", "200"]
            if self.dev is not None:
                cmd += ["-i", str(self.dev)]
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                smax.append(float(f[1]))
                power.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_max": max(power) if power else None}


def nvsmi_id(torch, dev):
    try:
        return "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        return None


# ---------------------------------------------------------------------------
# the GPU arm
# ---------------------------------------------------------------------------
def step(lat, hist):
    """One pass of the whole hot path on the resident lattice."""
    lat.restart("hot")
    lat.sweep_measure(SWEEPS, hist)
    lat.ape_smear(APE_ALPHA, APE_STEPS)
    return lat.wilson_loops(RMAX, TMAX, smeared=True)


def small_configs(torch):
    """The other configurations the benchmark's lattice is quoted beside, each
    run once as specified (their own sweep counts and measurements) and
    reported as link updates/s over the device time of the whole run."""
    import numpy as np
    from paper_1010_4834_gb300 import Batch, Lattice

    def timed(fn):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / 1e3

    out = {}
    # each run is preceded by a short untimed one on the same lattice (which
    # builds its sweep graphs), then the lattice restarts from its seed
    # 8^4, beta 2.4, cold, FP64: 100 sweeps, plaquette and Polyakov after each
    lat = Lattice((8, 8, 8, 8), 2.4, seed=1, start="cold", prec="f64")
    lat.sweep_measure(16)
    lat.restart("cold")
    t = timed(lambda: lat.sweep_measure(100))
    out["8^4_f64_cold_100sweeps_measured"] = 100 * 4 * 8 ** 4 / t
    lat.close()
    # 16^4, beta 2.5, hot, FP32: 500 sweeps, then 25 APE steps and W(R,T <= 8)
    lat = Lattice((16, 16, 16, 16), 2.5, seed=1, start="hot", prec="f32")

    def c2(n=500):
        lat.sweep(n)
        lat.ape_smear(0.7, 25)
        lat.wilson_loops(8, 8, smeared=True)
    c2(16)
    lat.restart("hot")
    t = timed(c2)
    out["16^4_f32_hot_500sweeps_ape25_W8x8"] = 500 * 4 * 16 ** 4 / t
    lat.close()
    # 32^3 x 4 at 16 betas in [2.2, 2.6]: 1000 measured sweeps each, FP32 and
    # F16Q; one lattice is too small to fill the GPU, so the 16 chains run
    # concurrently, each on its own stream driven by its own host thread
    from concurrent.futures import ThreadPoolExecutor
    for prec in ("f32", "f16q"):
        lats = [Lattice((32, 32, 32, 4), float(b), seed=1 + i, start="hot", prec=prec, stream=torch.cuda.Stream())
                for i, b in enumerate(np.linspace(2.2, 2.6, 16))]
        with ThreadPoolExecutor(len(lats)) as ex:
            list(ex.map(lambda x: x.sweep_measure(16), lats))
        for x in lats:
            x.restart("hot")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with ThreadPoolExecutor(len(lats)) as ex:
            list(ex.map(lambda x: x.sweep_measure(1000), lats))
        torch.cuda.synchronize()
        t = time.perf_counter() - t0
        out["32^3x4_%s_16betas_1000sweeps_measured" % prec] = 16 * 1000 * 4 * 32 ** 3 * 4 / t
        for x in lats:
            x.close()
        # the same scan as one batch: one persistent launch sweeps and
        # measures all 16 chains (su2_batch_sweep_measure); a first batch
        # picks the schedule, a fresh one from the hot start is timed
        betas = [float(b) for b in np.linspace(2.2, 2.6, 16)]
        warm = Batch([(32, 32, 32, 4)] * 16, betas, seed=1, start="hot", prec=prec)
        warm.tune(4)
        bs, G = warm.block_size, warm.groups
        warm.sweep_measure(16)
        warm.close()
        bat = Batch([(32, 32, 32, 4)] * 16, betas, seed=1, start="hot", prec=prec)
        bat.block_size, bat.groups = bs, G
        t = timed(lambda: bat.sweep_measure(1000))
        out["32^3x4_%s_16betas_1000sweeps_measured_batched" % prec] = 16 * 1000 * 4 * 32 ** 3 * 4 / t
        bat.close()
    return {"unit": UNIT, "values": out,
            "what": "each configuration's whole run (sweeps and its measurements): device time, and for the "
                    "32^3x4 scan the wall time of its 16 chains run concurrently on 16 streams, or (_batched) the "
                    "device time of one batch of the 16 chains measured in one persistent launch"}


def oracle_per_config():
    """The oracle as it stands on each configuration's lattice: two heat-bath
    sweeps from its start, serial build on one core and OpenMP build on
    every core; link updates/s (a bounded sample: the configurations' own
    sweep counts would take minutes to hours on the CPU)."""
    import oracle
    from oracle import build as oracle_build
    oracle_build.build_all()
    cases = {"C1 8^4 beta 2.4 cold": ((8, 8, 8, 8), 2.4, "cold"), "C2 16^4 beta 2.5 hot": ((16, 16, 16, 16), 2.5, "hot"),
             "C3 32^3x4 beta 2.4 cold": ((32, 32, 32, 4), 2.4, "cold"),
             "C4 24^3x6 beta 2.4 hot (largest batch member)": ((24, 24, 24, 6), 2.4, "hot"),
             "C5 64^4 beta 2.6 hot": (DIMS, BETA, "hot")}
    out = {}
    for name, (dims, beta, start) in cases.items():
        row = {}
        for label, ctx in (("1_core", None), ("all_cores", oracle.parallel)):
            ch = oracle.chain(beta, seed=1)
            nsw = 2 if volume(dims) <= 1 << 20 else 1
            with (ctx() if ctx else _null()):
                U = oracle.init_hot(list(dims), ch) if start == "hot" else oracle.init_cold(list(dims))
                t0 = time.perf_counter()
                if volume(dims) > 1 << 20 and label == "1_core":
                    upd = sum(oracle.substep(list(dims), U, ch, 0, k // 2, k % 2).updates for k in range(2))
                else:
                    upd = sum(oracle.sweep(list(dims), U, ch, sw).updates for sw in range(nsw))
                row[label] = upd / (time.perf_counter() - t0)
                if label == "all_cores":
                    row["cores"] = oracle.threads()
        out[name] = row
    return {"unit": UNIT, "values": out,
            "what": "the plain FP64 C oracle, two sweeps (64^4: one sweep on all cores, two substeps on one "
                    "core) of each configuration's lattice from its start"}


class _null:
    def __enter__(self):
        return self

    def __exit__(self, *a):
        return False


def batched_run(torch, peaks):
    """The 64-lattice batch: tuned schedule, then 200 sweeps in one persistent
    launch; link updates/s and the algorithmic GB/s at the substep's 128 B
    per update against the measured copy peak, with the ncu traffic of one
    batched launch (profiles/batched_f32.md) when it matches the source."""
    from paper_1010_4834_gb300 import Batch, inputs
    betas = inputs.batch_betas(len(BATCH_SHAPES), seed=1)
    b = Batch(BATCH_SHAPES, betas, seed=1, start="hot", prec="f32")
    groups = b.tune(4)
    b.sweep(20)
    torch.cuda.synchronize()
    a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    b.sweep(200)
    e.record()
    torch.cuda.synchronize()
    tb = a.elapsed_time(e) / 1e3
    vb = sum(volume(d) for d in BATCH_SHAPES)
    gb = 200 * 4 * vb * 128 / tb / 1e9
    out = {"value": 200 * 4 * vb / tb, "unit": UNIT,
           "achieved_gbs": round(gb, 1), "frac": round(gb / peaks["hbm_gbs"], 4), "bytes_per_update": 128,
           "what": "64 lattices (16 each of 8^4, 12^4, 16^4, 24^3x6), beta ~ U[2.0, 2.8], "
                   "FP32, 200 sweeps in one persistent cooperative launch (CUDA graph)",
           "ms_per_sweep": tb / 200 * 1e3, "groups": groups, "block_size": b.block_size,
           "schedule": "lattices dealt largest-first to G groups with CTAs in proportion to their work; "
                       "(block size, G) picked by su2_batch_tune"}
    vals = _profile_values("batched_f32.md")
    if vals.get("batch_sha") == batch_source_sha():
        try:
            out["traffic_dram_bytes_per_update"] = float(vals["dram_bytes_per_update"])
            out["traffic_l2_bytes_per_update"] = float(vals["l2_bytes_per_update"])
        except (KeyError, ValueError):
            pass
    b.close()
    return out


def batch_source_sha():
    """Hash of the batched kernel's sources (code only) and build flags."""
    h = hashlib.sha256()
    pkg = os.path.join(ROOT, "paper_1010_4834_gb300")
    for f in ("su2_batch.cu", "su2_device.cuh", "su2_hb_link.cuh", "su2_kernel_util.cuh", "su2_internal.h"):
        with open(os.path.join(pkg, "csrc", f), encoding="utf-8") as fh:
            h.update(_code_only(fh.read()).encode())
    with open(os.path.join(pkg, "build.py"), encoding="utf-8") as fh:
        h.update(_code_only(fh.read(), python=True).encode())
    return h.hexdigest()[:16]


def static_potential_run():
    """Section 5.4 on the 16^4 beta = 2.5 configuration: 200 configurations
    ten sweeps apart after 300 thermalisation sweeps, each smeared by 25 APE
    steps (alpha = 0.7) before W(R, T <= 8); V(R) at its plateau in T and the
    fitted string tension with jackknife errors, beside the paper's table."""
    from paper_1010_4834_gb300 import Lattice, potential
    lat = Lattice((16, 16, 16, 16), 2.5, seed=1, start="hot", prec="f32")
    lat.sweep(300)
    W = potential.wilson_ensemble(lat, 200, 10, alpha=0.7, n_ape=25, rmax=8, tmax=8)
    lat.close()
    res = potential.static_potential(W, rfit=6)
    return {"lattice": "16^4", "beta": 2.5, "configurations": 200, "sweeps_apart": 10,
            "ape": [25, 0.7], "V": [round(float(v), 5) for v in res["V"]],
            "dV": [round(float(v), 5) for v in res["dV"]], "T_plateau": [int(t) for t in res["T_plateau"]],
            "fit_R": [1, int(res["rfit"])], "sigma_a2": res["sigma_a2"], "sigma_a2_err": res["sigma_a2_err"],
            "a_fm": res["a_fm"], "a_fm_err": res["a_fm_err"],
            "paper_beta2.5": {"sigma_a2": 0.036623, "a_fm": 0.085682, "lattice": "24^3x32", "configurations": 1981}}


def timed_sweeps(torch, lat, n, reps=3):
    """Device time of n heat-bath sweeps (graph path), best of reps."""
    best = None
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record()
        lat.sweep(n)
        b.record()
        torch.cuda.synchronize()
        t = a.elapsed_time(b) / 1e3
        best = t if best is None else min(best, t)
    return best


def launch_seconds(torch, lat, kind, sweeps=4):
    """Average duration of one heat-bath launch of `kind` ("substep" or
    "pair"): one CUDA-event pair around the launches of `sweeps` sweeps
    issued back to back on the lattice's stream, and, for comparison, the
    mean of the same launches each bracketed by its own events with the
    stream idle between them (which adds the launch latency to every launch).
    For the substep a third figure: one event pair around 32 plain sweeps
    replayed as the library's sweep graph (8 substep launches a sweep, plus
    one sweep-counter bump every 8 sweeps), the way the benchmark's sweeps
    run the kernel; that one is returned first."""
    def one(mu, p, sw):
        if kind == "pair":
            lat.pair(mu, sw)
        else:
            lat.substep(mu, p, sw)
    parities = (0,) if kind == "pair" else (0, 1)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for sw in range(sweeps):
        for mu in range(4):
            for p in parities:
                one(mu, p, 1000 + sw)
    b.record()
    torch.cuda.synchronize()
    n = 4 * len(parities) * sweeps
    back_to_back = a.elapsed_time(b) / 1e3 / n
    in_graph = None
    if kind != "pair":
        lat.sweep(8)                      # the sweep graph exists
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        lat.sweep(32)
        b.record()
        torch.cuda.synchronize()
        in_graph = a.elapsed_time(b) / 1e3 / (8 * 32)
    times = []
    for sw in range(sweeps):
        for mu in range(4):
            for p in parities:
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                one(mu, p, 2000 + sw)
                b.record()
                torch.cuda.synchronize()
                times.append(a.elapsed_time(b) / 1e3)
    return back_to_back, n, statistics.mean(times), in_graph


def heatbath_roofline(torch, lat, kind, peaks, peak_kind):
    """The heat-bath kernel the sweeps run, against the measured copy peak.
    Algorithmic bytes per update: a substep reads the 3.5 V distinct links its
    V/2 staples need and writes V/2 (8 link transfers per update); a fused
    parity pair reads 3.5 V and writes V for V updates (4.5 transfers)."""
    V = volume(DIMS)
    lb = {"f32": 16, "f64": 32, "f16q": 8}[PREC]
    t_direct, n_launch, t_isolated, t_graph = launch_seconds(torch, lat, kind)
    t_launch = t_graph if t_graph is not None else t_direct
    timing = ("one event pair around 32 sweeps replayed as the sweep graph (256 launches)" if t_graph is not None
              else "one event pair around %d back-to-back launches" % n_launch)
    if kind == "pair":
        upd_launch, per_update, name = V, 4.5 * lb, "k_heatbath_pair<F32>"
    else:
        upd_launch, per_update, name = V // 2, 8 * lb, "k_heatbath<F32>"
    alg_bytes = int(per_update * upd_launch)
    achieved = alg_bytes / t_launch / 1e9
    return {"bound": "hbm", "kernel": name, "achieved": round(achieved, 1),
            "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": round(achieved / peaks["hbm_gbs"], 4),
            "peak_kind": peak_kind, "traffic": profiled_traffic(kind, upd_launch),
            "algorithmic_bytes_per_update": per_update,
            "algorithmic_bytes_per_launch": alg_bytes, "launch_us": round(t_launch * 1e6, 2),
            "launches_timed": 256 if t_graph is not None else n_launch, "timing": timing,
            "launch_us_direct": round(t_direct * 1e6, 2),
            "launch_us_direct_note": "one event pair around %d back-to-back direct launches" % n_launch,
            "launch_us_isolated": round(t_isolated * 1e6, 2),
            "updates_per_s_in_kernel": upd_launch / t_launch}


def reduce_over_ranks(dist, elapsed, launches, device):
    """Whole-job timing: the slowest rank's time and every rank's launches."""
    import torch
    t = torch.tensor([elapsed], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    c = torch.tensor([float(launches)], device=device, dtype=torch.float64)
    dist.all_reduce(c)
    return float(t.item()), int(c.item())


def _code_only(text, python=False):
    """Source text without comments and with whitespace runs collapsed, so
    that editing a comment does not count as changing the kernel."""
    import re
    if python:
        text = re.sub(r"#[^\n]*", " ", text)
    else:
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def source_sha():
    """Hash of the heat-bath kernels' sources (code only) and build flags."""
    h = hashlib.sha256()
    pkg = os.path.join(ROOT, "paper_1010_4834_gb300")
    for f in (os.path.join(pkg, "csrc", "su2_device.cuh"), os.path.join(pkg, "csrc", "su2_heatbath.cu"),
              os.path.join(pkg, "csrc", "su2_hb_link.cuh"), os.path.join(pkg, "csrc", "su2_pair.cu"),
              os.path.join(pkg, "csrc", "su2_kernel_util.cuh"), os.path.join(pkg, "csrc", "su2_internal.h"),
              os.path.join(pkg, "build.py")):
        with open(f, encoding="utf-8") as fh:
            h.update(_code_only(fh.read(), python=f.endswith(".py")).encode())
    return h.hexdigest()[:16]


def _profile_values(name):
    path = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(path):
        return {}
    vals = {}
    for line in open(path):
        if ":" in line and line.startswith("- "):
            k, v = line[2:].split(":", 1)
            vals[k.strip()] = v.strip().strip("`")
    return vals


def profiled_traffic(kind, updates_per_launch):
    """DRAM bytes per heat-bath launch ("substep" or "pair") from the
    committed ncu summary, scaled by updates; None if the kernel source
    changed since the capture."""
    vals = _profile_values("hb_pair_f32.md" if kind == "pair" else "hb_substep_f32.md")
    if vals.get("source_sha") != source_sha():
        return None
    try:
        return float(vals["dram_bytes_per_update"]) * updates_per_launch
    except (KeyError, ValueError):
        return None


def profiled_f64_flops():
    """FP64 flops per heat-bath link update (2 DFMA + DMUL + DADD thread
    instructions, from the committed ncu summary of an FP64 substep), or None
    if the kernel source changed since the capture."""
    vals = _profile_values("hb_substep_f64.md")
    if vals.get("source_sha") != source_sha():
        return None
    try:
        return float(vals["fp64_flops_per_update"])
    except (KeyError, ValueError):
        return None


def f64_roofline(updates_per_s, fp64_peak):
    """The FP64 heat bath against the probe-measured FP64 FMA rate (its bound:
    GB300 issues FP64 at 1/64 of the FP32 rate)."""
    fl = profiled_f64_flops()
    if fl is None or not fp64_peak:
        return {"bound": "alu", "achieved": None, "peak": fp64_peak, "unit": "FLOP/s", "frac": None,
                "note": "FP64 flops per update not profiled for this source"}
    ach = fl * updates_per_s
    return {"bound": "alu", "achieved": ach, "peak": fp64_peak, "unit": "FLOP/s", "frac": round(ach / fp64_peak, 4),
            "flops_per_update": fl, "peak_kind": "measured (su2_probe_fma, FP64)"}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def _oracle_substeps(nsub):
    """Time `nsub` heat-bath substeps of the oracle (in sweep order) on the
    benchmark's hot-start lattice with the oracle build currently bound;
    returns (link updates, seconds)."""
    import oracle
    ch = oracle.chain(BETA, seed=1)
    U = oracle.init_hot(list(DIMS), ch)
    updates = 0
    t0 = time.perf_counter()
    for k in range(nsub):
        updates += oracle.substep(list(DIMS), U, ch, k // 8, (k // 2) % 4, k % 2).updates
    return updates, time.perf_counter() - t0


def cpu_baseline():
    """The oracle as it stands (plain FP64 C) on the same 64^4 lattice: its
    OpenMP build over every host core on two sweeps (sixteen substeps), and
    the serial build on one core on the first four substeps (half a sweep)."""
    import oracle
    from oracle import build as oracle_build
    oracle_build.build_all()
    with oracle.parallel():
        cores = oracle.threads()
        upd_all, t_all = _oracle_substeps(16)
    upd_one, t_one = _oracle_substeps(4)
    lat = "x".join(map(str, DIMS))
    return {"value": upd_all / t_all, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "two heat-bath sweeps (sixteen substeps, %d link updates) of the %s beta=2.6 hot-start "
                      "lattice, the plain FP64 C oracle built with OpenMP (the sites of each substep shared "
                      "among %d threads, one per host core); %.1f s" % (upd_all, lat, cores, t_all),
            "single_core": {"value": upd_one / t_one, "unit": UNIT, "cores": 1,
                            "sample": "the first four substeps (%d link updates), serial build; %.1f s"
                                      % (upd_one, t_one)}}


def run_gpu(args):
    import torch
    ws, rank, lrank = dist_env()
    torch.cuda.set_device(lrank)
    # one dedicated stream: the library's launches and the timing events share it
    with torch.cuda.stream(torch.cuda.Stream()):
        run_gpu_on_stream(args)


def run_gpu_on_stream(args):
    import numpy as np
    import torch
    ws, rank, lrank = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(lrank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", lrank))
    else:
        dist = None
        torch.cuda.set_device(lrank)

    def barrier():
        if dist is not None:
            dist.barrier()

    from paper_1010_4834_gb300 import build as su2_build
    if rank == 0 or ws == 1:
        su2_build.build()
    barrier()
    from paper_1010_4834_gb300 import Lattice, kernel_launches, probe_fma

    V = volume(DIMS)
    lat = Lattice(DIMS, BETA, seed=1 + rank, start="hot", prec=PREC)
    hist = np.empty((SWEEPS, 4))
    for _ in range(args.warmup):
        step(lat, hist)
    torch.cuda.synchronize()
    barrier()
    clocks = ClockSampler(nvsmi_id(torch, lrank))
    clocks.start()
    n0 = kernel_launches()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record()
    for _ in range(args.steps):
        W = step(lat, hist)
    ev1.record()
    torch.cuda.synchronize()
    elapsed = ev0.elapsed_time(ev1) / 1e3
    launches = kernel_launches() - n0
    clk = clocks.stop()
    barrier()
    if dist is not None:
        elapsed, launches = reduce_over_ranks(dist, elapsed, launches, "cuda")
    updates_per_step = SWEEPS * 4 * V
    value = ws * updates_per_step * args.steps / elapsed
    plaq_last = float(hist[-1, 0])

    # roofline of the heat-bath kernel the sweeps run (the substep kernel),
    # with the fused parity pair's beside it
    peaks, peak_kind = measured_peaks()
    roofline = heatbath_roofline(torch, lat, "substep", peaks, peak_kind)
    if PREC != "f64":
        roofline["pair_kernel"] = heatbath_roofline(torch, lat, "pair", peaks, peak_kind)

    # end to end through the public API: every step starts from the
    # configuration in pinned host memory (2.15 GB canonical FP64), which the
    # copy engine brings into one of two device buffers while the previous
    # step computes (the first step's copy is not hidden); results to host
    host_cfg = torch.empty((V, 4, 4), dtype=torch.float64, pin_memory=True)
    lat.get_links(host_cfg.numpy())
    dev_cfg = [torch.empty((V, 4, 4), dtype=torch.float64, device="cuda") for _ in range(2)]
    copy_stream = torch.cuda.Stream()
    lat_stream = torch.cuda.current_stream()   # the lattice's stream
    ready = [torch.cuda.Event() for _ in range(2)]
    e2e_steps = max(1, args.steps)
    torch.cuda.synchronize()
    t0 = time.perf_counter()

    def fetch(k):
        with torch.cuda.stream(copy_stream):
            dev_cfg[k % 2].copy_(host_cfg, non_blocking=True)
            ready[k % 2].record(copy_stream)

    fetch(0)
    for i in range(e2e_steps):
        if i + 1 < e2e_steps:
            fetch(i + 1)   # buffer (i+1) % 2 was last read by step i - 1's set_links, which synchronised
        lat_stream.wait_event(ready[i % 2])
        lat.set_links(dev_cfg[i % 2])
        lat.sweep_measure(SWEEPS, hist)
        lat.ape_smear(APE_ALPHA, APE_STEPS)
        W = lat.wilson_loops(RMAX, TMAX, smeared=True)
    torch.cuda.synchronize()
    t_e2e = time.perf_counter() - t0
    e2e = {"value": ws * updates_per_step * e2e_steps / t_e2e, "unit": UNIT,
           "h2d_bytes_per_step": V * 16 * 8, "d2h_bytes_per_step": hist.nbytes + W.nbytes,
           "path": "pinned host links -> copy engine (next step's, overlapped) -> Lattice.set_links(device copy) "
                   "-> sweep_measure(100) -> ape_smear(0.7, 25) -> wilson_loops(16, 16)", "steps": e2e_steps}
    # the same through the C ABI's own host-input path: su2_set_links reads
    # the pinned host buffer itself (its conversion kernel reads host memory
    # directly), so each step's copy is not overlapped with the previous step
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        lat.set_links(host_cfg.numpy())
        lat.sweep_measure(SWEEPS, hist)
        lat.ape_smear(APE_ALPHA, APE_STEPS)
        W = lat.wilson_loops(RMAX, TMAX, smeared=True)
    torch.cuda.synchronize()
    t_dir = time.perf_counter() - t0
    e2e["host_path"] = {"value": ws * updates_per_step * e2e_steps / t_dir, "unit": UNIT,
                        "path": "pinned host links -> Lattice.set_links(host pointer: su2_set_links reads it "
                                "directly) -> sweep_measure(100) -> ape_smear(0.7, 25) -> wilson_loops(16, 16)"}
    del host_cfg, dev_cfg

    extra = {}
    if rank == 0 and not args.no_extra:
        extra["sweep_only"] = {"value": 20 * 4 * V / timed_sweeps(torch, lat, 20), "unit": UNIT,
                               "what": "FP32 64^4 heat-bath sweeps alone (graph replay), 20 sweeps"}
        # over-relaxation sweeps (Eq. 10): the same staple gather plus the old
        # link, no random numbers; 144 B per update (7 classes read for the
        # staple, the link itself read and written)
        lat.overrelax(2)
        best = None
        for _ in range(3):
            a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record()
            lat.overrelax(8)
            e.record()
            torch.cuda.synchronize()
            t = a.elapsed_time(e) / 1e3
            best = t if best is None else min(best, t)
        or_gbs = 8 * 4 * V * 144 / best / 1e9
        extra["overrelax"] = {"value": 8 * 4 * V / best, "unit": UNIT, "achieved_gbs": round(or_gbs, 1),
                              "frac": round(or_gbs / peaks["hbm_gbs"], 4),
                              "what": "FP32 64^4 over-relaxation sweeps, 8 sweeps of 8 launches; 144 B per "
                                      "update of algorithmic traffic against the measured copy peak"}
        # the paper's benchmark mode (Section 5.1): beta 6.0, hot start, one
        # heat-bath try (Creutz), the plaquette measured every sweep
        lat.set_options(1, "creutz")
        lat.set_beta(6.0)
        lat.restart("hot")
        lat.sweep_measure(5)
        a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        lat.sweep_measure(20)
        e.record()
        torch.cuda.synchronize()
        extra["paper_mode"] = {"value": 20 * 4 * V / (a.elapsed_time(e) / 1e3), "unit": UNIT,
                               "what": "64^4 FP32, beta 6.0, hot start, Creutz sampler with one try, "
                                       "plaquette and Polyakov every sweep, 20 sweeps"}
        # the layout comparison of Section 5.1 (same settings): one array of
        # all links against one array per direction, one plain kernel on both
        lat.layout_compare(1)
        ms, mismatch = lat.layout_compare(8)
        ups = [8 * 4 * V / (t / 1e3) for t in ms]
        extra["layout"] = {"library": ups[0], "plain_by_direction": ups[1], "plain_one_array": ups[2],
                           "unit": UNIT, "by_direction_over_one_array": ups[1] / ups[2],
                           "mismatched_links": mismatch,
                           "what": "8 sweeps in paper mode: the library's kernels; a plain one-thread-per-link "
                                   "kernel on the library's layout (one array per direction and parity); the same "
                                   "kernel on one site-major array (element 4 s + mu), the paper's layout"}
        lat.close()
        del lat
        fp64_peak = probe_fma("f64")
        extra["fma_peaks"] = {"f64": fp64_peak, "f32": probe_fma("f32"), "unit": "FLOP/s",
                              "what": "su2_probe_fma: eight independent FMA chains per thread over a full grid"}
        for prec, n in (("f64", 4), ("f16q", 20)):
            l2 = Lattice(DIMS, BETA, seed=1, start="hot", prec=prec)
            l2.sweep(2)
            extra[prec] = {"value": n * 4 * V / timed_sweeps(torch, l2, n, reps=2), "unit": UNIT,
                           "what": "%s 64^4 heat-bath sweeps alone, %d sweeps" % (prec, n)}
            if prec == "f64":
                extra[prec]["roofline"] = f64_roofline(extra[prec]["value"], fp64_peak)
            else:
                g = extra[prec]["value"] * 64 / 1e9          # 8 links of 8 B per update
                extra[prec]["achieved_gbs"] = round(g, 1)
                extra[prec]["frac"] = round(g / peaks["hbm_gbs"], 4)
            l2.close()
        extra["configs"] = small_configs(torch)
        c1 = extra["configs"]["values"]["8^4_f64_cold_100sweeps_measured"]
        extra["configs"]["8^4_f64_roofline"] = f64_roofline(c1, fp64_peak)
        extra["static_potential"] = static_potential_run()
        if not args.no_cpu:
            extra["oracle_configs"] = oracle_per_config()
        extra["batched"] = batched_run(torch, peaks)
    else:
        lat.close()

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        cpu = cpu_baseline()

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": elapsed / args.steps * 1e3, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic (hot start from seed)",
                "config": config(ws), "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": launches, "clocks": clk, "plaquette_last": plaq_last}
        line.update(extra)
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# the reference arm: the CPU oracle as it stands
# ---------------------------------------------------------------------------
def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    from oracle import build as oracle_build
    oracle_build.build_all()
    with oracle.parallel():
        cores = oracle.threads()
        ch = oracle.chain(BETA, seed=1)
        U = oracle.init_hot(list(DIMS), ch)
        k = 0
        for _ in range(args.warmup):
            oracle.substep(list(DIMS), U, ch, k // 8, (k // 2) % 4, k % 2)
            k += 1
        t0 = time.perf_counter()
        updates = 0
        for _ in range(args.steps):
            st = oracle.substep(list(DIMS), U, ch, k // 8, (k // 2) % 4, k % 2)
            updates += st.updates
            k += 1
        t = time.perf_counter() - t0
    value = updates / t
    sample = ("each step one heat-bath substep (%d link updates) of the %s beta=2.6 hot-start lattice, "
              "plain FP64 C oracle built with OpenMP over %d host cores"
              % (volume(DIMS) // 2, "x".join(map(str, DIMS)), cores))
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (hot start from seed)",
            "config": config(ws), "impl": "reference",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline")
    ap.add_argument("--no-extra", action="store_true", help="skip the FP64/F16Q/batched sub-measurements")
    ap.add_argument("--extent", type=int, default=None,
                    help="hypercubic extent override (small profiling cases only; not a bench line)")
    ap.add_argument("--sweeps", type=int, default=None, help="sweeps per step override (profiling only)")
    ap.add_argument("--prec", choices=["f32", "f64", "f16q"], default="f32",
                    help="link precision override (profiling only; not a bench line)")
    ap.add_argument("--batched-only", action="store_true",
                    help="run only the 64-lattice batched measurement and print it (profiling; not a bench line)")
    args = ap.parse_args()
    global DIMS, SWEEPS, WORKLOAD
    if args.extent:
        DIMS = (args.extent,) * 4
    if args.sweeps:
        SWEEPS = args.sweeps
    global PREC
    PREC = args.prec
    if args.extent or args.sweeps or PREC != "f32":
        WORKLOAD = "profiling case %s %s, %d sweeps per step" % ("x".join(map(str, DIMS)), PREC, SWEEPS)
    if args.warmup < 3 and args.impl == "ours":
        print("note: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        run_reference(args)
    elif args.batched_only:
        import torch
        torch.cuda.set_device(0)
        print(json.dumps({"batched": batched_run(torch, measured_peaks()[0])}), flush=True)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
