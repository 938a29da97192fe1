"""Benchmark: two-site gate applies/s at chi = 4096, mixed-precision vs FP64 path.

Workload (steady state of a saturated bond, the chi = 4096 configuration):
an n = 26 chain whose bonds saturate at chi = 4096 (bonds 12, 13, 14 are 4096),
initialised as a random mixed-canonical MPS (sites left of 12 left-isometries,
right of 12 right-isometries, site 12 i.i.d. complex Gaussian of unit norm;
workloads/states.py).  One step = one pass of the whole hot path on bond
(12, 13) under the canonical policy:
  * one-qubit Haar gates on sites 12 and 13,
  * the centre move back to site 12 (LQ of site 13, absorbed into site 12),
  * the theta contraction with the gate epilogue, the truncated pivoted QR
    (k = chi), Q formation and the split,
with the two-qubit gate alternating between a seeded Haar SU(4) gate
(mps_apply_2q) and a SWAP (mps_swap).  Bond dims are invariant (k = chi), so
every step is the same amount of work.  Inputs (theta is 512 MiB in c64) are
larger than L2, so no flush is needed between steps.

`value` is the mixed path's applies/s over all ranks (replicas: one independent
state per GPU, no collectives on the data path).  The FP64 path runs the same
steps for a shorter count; the fidelity deviation compares a mixed and an FP64
state after the same steps.

--impl reference times the CPU oracle (oracle/) on the host cores instead.
"""

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

CHI = 4096
N_SITES = 26
BOND_SITE = 12
METRIC = "two-site gate applies/s at chi=4096; mixed vs FP64 path at fidelity dev <=1e-6"


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def init_dist(backend):
    """Process group of the replica run, with a bounded collective timeout
    (MPS_BENCH_PG_TIMEOUT_S, default 600 s): a replica that dies or stalls before the
    timing all-reduce makes the other ranks fail with an error instead of waiting."""
    import datetime

    import torch.distributed as dist

    secs = float(os.environ.get("MPS_BENCH_PG_TIMEOUT_S", "600"))
    dist.init_process_group(backend, timeout=datetime.timedelta(seconds=secs))


def make_state(chi, n, centre, seed):
    import numpy as np

    from workloads import states

    bonds = states.max_bond_dims(n, chi)
    sites = states.random_canonical_mps(n, bonds, centre, seed=seed)
    return [np.ascontiguousarray(s) for s in sites]


def step_gates(steps, seed):
    import numpy as np

    from workloads import gates

    rng = np.random.default_rng(seed)
    seq = []
    for s in range(steps):
        u1 = gates.haar_unitary(rng, 2)
        u2 = gates.haar_unitary(rng, 2)
        g = gates.haar_unitary(rng, 4) if s % 2 == 0 else None  # None = SWAP
        seq.append((u1, u2, g))
    return seq


def do_step(m, st, i=BOND_SITE):
    u1, u2, g = st
    m.apply_1q(i, u1)
    m.apply_1q(i + 1, u2)
    if g is None:
        m.swap(i)
    else:
        m.apply_2q(i, g)


class ClockSampler:
    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) >= 9:
                    rows.append(f)
        except Exception:
            pass
        finally:
            try:
                os.unlink(self.path)
            except Exception:
                pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["clock sampling unavailable"]}
        mhz = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[j] for r in rows for j in range(4) if r[5 + j].lower() == "active"})
        return {"sm_mhz": statistics.median(mhz) if mhz else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# DRAM traffic of the panel kernel from one ncu capture (profiles/qr_panel_kernel_chi4096.md):
# the dram bytes of all 128 panel launches of one chi = 4096 gate over their algorithmic
# bytes.  The sweep's L2 reuse makes the ratio depend on the bond dimension (the share
# of the trailing matrix that stays in L2), so it is used only at the chi it was
# measured at, and only for the kernel source it was measured on (sha256 of the
# qr_panel_kernel definition in csrc/qr.cu); otherwise the traffic is null.
PANEL_NCU = {"kernel_sha256": "58a896d19a977c4b4e7f1e58bd8887db2b260c2601fc785c0f81cf7d276730c7", "chi": 4096,
             "dram_over_algorithmic": 0.7408}


def panel_kernel_source():
    """The text of qr_panel_kernel's definition in csrc/qr.cu (up to the section on the
    unpivoted cluster panel that follows it)."""
    with open(os.path.join(ROOT, "paper_2505_06119_gb300", "csrc", "qr.cu")) as f:
        src = f.read()
    start = src.index("__global__ void __launch_bounds__(PNT, 1) qr_panel_kernel")
    end = src.index("// Unpivoted panel on one thread-block cluster", start)
    return src[start:end]


def panel_traffic(alg_bytes_per_launch, chi):
    import hashlib

    if chi != PANEL_NCU["chi"]:
        return None

    try:
        sha = hashlib.sha256(panel_kernel_source().encode()).hexdigest()
    except Exception:
        return None
    if PANEL_NCU["kernel_sha256"] is None or sha != PANEL_NCU["kernel_sha256"]:
        return None
    return PANEL_NCU["dram_over_algorithmic"] * alg_bytes_per_launch


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return p, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def ours(args):
    import numpy as np
    import torch

    import __graft_entry__

    ws, rank, local = dist_env()
    if ws > 1:
        init_dist("nccl")
    torch.cuda.set_device(local)
    __graft_entry__.build()
    from paper_2505_06119_gb300 import MPS

    chi = args.chi
    n = N_SITES if chi == CHI else 2 * int(math.log2(chi)) + 2
    i = n // 2 - 1  # bonds i, i+1, i+2 all equal chi
    sites = make_state(chi, n, i, seed=1234 + rank)
    seq = step_gates(max(args.warmup + args.steps, args.fp64_warmup + args.fp64_steps), seed=99 + rank)
    stream = torch.cuda.Stream()
    sptr = stream.cuda_stream

    # --- mixed path, timed with per-kernel-class CUDA events
    tr = {"truncation": args.truncation}
    tc = {"tensor_cores": True} if args.tensor_cores else {}
    m = MPS(n, chi, precision="mixed", policy="canon", stream=sptr, profile=True, device=local, **tr, **tc)
    m.set_sites([s.astype(np.complex64) for s in sites], centre=i)
    with ClockSampler(local) as clk:
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        ms, st = time_steps_at(m, seq, args.warmup, args.steps, torch, stream, i)
    clocks = clk.summary()
    ms_step = ms / args.steps
    launches = int(sum(v["launches"] for v in st.values()))
    panel = st["panel"]
    peaks, peak_src = load_peaks()
    achieved = panel["alg_bytes"] / (panel["ms"] * 1e-3) / 1e9 if panel["ms"] > 0 else 0.0
    m.close()

    ms_step64 = None
    fid = {}
    if args.fp64_steps > 0:
        # --- FP64 path on the same steps
        m64 = MPS(n, chi, precision="fp64", policy="canon", stream=sptr, device=local, **tr)
        m64.set_sites(sites, centre=i)
        ms64, st64 = time_steps_at(m64, seq, args.fp64_warmup, args.fp64_steps, torch, stream, i)
        ms_step64 = ms64 / args.fp64_steps

        # --- deviation of the mixed path from the FP64 path: a mixed state run through
        # exactly the FP64 steps, compared result by result
        mm = MPS(n, chi, precision="mixed", policy="canon", stream=sptr, device=local, **tr, **tc)
        mm.set_sites([s.astype(np.complex64) for s in sites], centre=i)
        for stp in seq[:args.fp64_warmup + args.fp64_steps]:
            do_step_at(mm, stp, i)
        fid = fidelity_deviation(mm, m64, n, i, args, np)
        mm.close()
        m64.close()

    # --- end to end through the C ABI with host buffers (pinned), copies timed
    e2e = {"value": None, "seconds": 1.0, "steps": 0, "h2d": 0, "d2h": 0}
    if args.e2e_steps > 0:
        e2e = e2e_run(args, sites, seq, n, chi, i, sptr, local, torch, np)

    agg = replica_throughput(ms, e2e["seconds"], args.steps, e2e["steps"], ws, device="cuda")
    t_max, value = agg["t_max_ms"], agg["value"]
    e2e_v = agg["e2e_value"] if ws > 1 else e2e["value"]
    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return
    cpu = None if args.no_cpu_baseline else cpu_baseline(args)
    line = {
        "metric": METRIC,
        "value": value,
        "unit": "applies/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": t_max / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "c64",
        "data": "synthetic",
        "config": bench_config(chi, n, i, ws, args.truncation),
        "fp64_path": {"value": ws * 1e3 / ms_step64 if ms_step64 else None, "unit": "applies/s",
                      "ms_per_step": ms_step64, "steps": args.fp64_steps, "warmup": args.fp64_warmup,
                      "dtype": "c128"},
        "speedup_vs_fp64": ms_step64 / ms_step if ms_step64 else None,
        "tflops": FLOP_PER_APPLY * chi ** 3 * value / 1e12,
        "tensor_roofline": tensor_roofline(FLOP_PER_APPLY * chi ** 3 * value / 1e12, peaks, peak_src,
                                           FLOP_PER_APPLY * chi ** 3 * ws * 1e3 / ms_step64 / 1e12
                                           if ms_step64 else None),
        "fidelity_dev": fid,
        "roofline": {"bound": "hbm",
                     "kernel": ("qr_panel_kernel (pivoted-QR panel: per-step trailing GEMV)" if args.truncation == "qrcp"
                                else "panel class of the randomized split (sketch pivots and unpivoted panels: "
                                     "latency-bound; algorithmic bytes are the sketch's)"),
                     "achieved": achieved, "peak": peaks.get("hbm_gbs"), "unit": "GB/s",
                     "frac": achieved / peaks.get("hbm_gbs", 1.0),
                     "traffic": (panel_traffic(panel["alg_bytes"] / max(1, panel["launches"]), chi)
                                 if args.truncation == "qrcp" else None),
                     "traffic_unit": "bytes per launch",
                     "peak_source": peak_src,
                     "launches_timed": panel["launches"], "kernel_ms_per_step": panel["ms"] / args.steps},
        "stage_ms_per_step": {k: v["ms"] / args.steps for k, v in st.items()},
        "gpu_launches": launches,
        "clocks": clocks,
        "e2e": {"value": e2e_v, "unit": "applies/s", "h2d_bytes_per_step": e2e["h2d"],
                "d2h_bytes_per_step": e2e["d2h"], "steps": e2e["steps"]},
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


# algorithmic real flops of one full-bond two-site apply per chi^3: theta contraction
# 32, truncated pivoted QR 37.3, Q formation 13.3
FLOP_PER_APPLY = 82.7
FP64_NOMINAL_TFLOPS = 1.25  # GB300 FP64 rate (nominal; no FP64 peak is measured on this machine)
TF32_PER_BF16 = 0.5         # dense TF32 tensor rate relative to BF16 (nominal ratio 1.1 / 2.25 PF)


def tensor_roofline(tflops_mixed, peaks, peak_src, tflops_fp64):
    """Algorithmic TFLOP/s of the whole step as a fraction of the dense tensor rates:
    BF16 (the measured sustained cuBLAS rate, the step being seconds long), TF32 (that
    rate times the nominal TF32/BF16 ratio), and for the FP64 path the nominal FP64 rate."""
    bf16 = peaks.get("bf16_tflops_sustained") or peaks.get("bf16_tflops") or 1700.0
    out = {"tflops_mixed": tflops_mixed, "peak_bf16_tflops": bf16, "frac_bf16": tflops_mixed / bf16,
           "peak_tf32_tflops": bf16 * TF32_PER_BF16, "frac_tf32": tflops_mixed / (bf16 * TF32_PER_BF16),
           "peak_source": peak_src + " (bf16 sustained; tf32 = bf16 x 0.5 nominal ratio)"}
    if tflops_fp64:
        out.update({"tflops_fp64": tflops_fp64, "peak_fp64_tflops": FP64_NOMINAL_TFLOPS,
                    "frac_fp64": tflops_fp64 / FP64_NOMINAL_TFLOPS, "fp64_peak_source": "nominal"})
    return out


def fidelity_deviation(mm, m64, n, i, args, np):
    """Error of the mixed path against the FP64 path (which matches the FP64 oracle to
    1e-10) after the same steps, per result: the norm fidelity (relative), the state
    fidelity 1 - |<mix|64>|^2 / (<mix|mix><64|64>) (FP64 transfer matrices), sampled
    amplitudes (absolute and relative to the largest sampled FP64 amplitude) and the
    diagonal of R of the last split, |R_tt| for the kept pivots t < k (relative)."""
    f64 = m64.fidelity()
    fmx = mm.fidelity()
    out = {"steps": args.fp64_warmup + args.fp64_steps, "f_fp64": f64, "f_mixed": fmx,
           "norm_fidelity_rel": abs(fmx - f64) / f64,
           "scope": "after the listed steps of this workload (a per-step bar); over the 390 truncating gates "
                    "of the 40-qubit depth-20 brick-wall at chi 1024 the deviation is larger (about 4e-5 in the norm fidelity), "
                    "set by pivot decisions between residual norms closer than FP32 rounding"}
    if not args.skip_overlap:
        o = mm.overlap(m64)
        nmx = mm.overlap(mm).real
        n64 = m64.overlap(m64).real
        out["overlap"] = 1.0 - abs(o) ** 2 / (nmx * n64)
    rng = np.random.default_rng(2024)
    amax = dmax = 0.0
    for _ in range(args.amp_samples):
        bits = rng.integers(0, 2, n)
        a64 = m64.amplitude(bits)
        dmax = max(dmax, abs(mm.amplitude(bits) - a64))
        amax = max(amax, abs(a64))
    out["amplitude_max_abs"] = dmax
    out["amplitude_max_rel"] = dmax / amax if amax > 0 else None
    out["amplitude_samples"] = args.amp_samples
    # R diagonal of the last split: row t of the right site R P^T at column jpvt[t]
    p64, k64 = m64.last_pivots()
    pmx, kmx = mm.last_pivots()
    r64 = m64.get_site(i + 1).reshape(k64, -1)
    rmx = mm.get_site(i + 1).reshape(kmx, -1)
    d64 = np.abs(r64[np.arange(k64), p64[:k64]])
    dmx = np.abs(rmx[np.arange(kmx), pmx[:kmx]])
    out["r_diag_rel_max"] = float(np.max(np.abs(dmx - d64) / np.maximum(d64, 1e-300)))
    out["r_diag_rel_max_first_half"] = float(np.max(np.abs(dmx - d64)[:k64 // 2] / d64[:k64 // 2]))
    out["pivots_equal"] = bool(np.array_equal(p64[:k64], pmx[:kmx]))
    out["pivot_positions_differing"] = int(np.sum(p64[:k64] != pmx[:kmx]))
    return out


def replica_throughput(ms, e2e_seconds, steps, e2e_steps, ws, device="cuda"):
    """Whole-job throughput of ws independent replicas (no data-path collective):
    every rank timed `steps` steps in `ms` milliseconds; the job takes the slowest
    rank's time, so value = steps * ws / max_rank(ms).  Same for the end-to-end loop.
    One all-reduce (MAX) of the two times when ws > 1 (NCCL on "cuda", gloo on "cpu")."""
    import torch

    t_max, e2e_s = float(ms), float(e2e_seconds)
    if ws > 1:
        import torch.distributed as dist

        t = torch.tensor([t_max, e2e_s], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_max, e2e_s = float(t[0]), float(t[1])
    return {"t_max_ms": t_max, "value": steps * ws / (t_max * 1e-3),
            "e2e_value": (e2e_steps * ws / e2e_s) if e2e_steps else None}


def do_step_at(m, st, i):
    do_step(m, st, i)


def time_steps_at(m, seq, warmup, steps, torch, stream, i):
    for st in seq[:warmup]:
        do_step(m, st, i)
    m.sync()
    m.kernel_stats_reset()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for st in seq[warmup:warmup + steps]:
        do_step(m, st, i)
    e1.record(stream)
    m.sync()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1), m.kernel_stats()


def e2e_run(args, sites, seq, n, chi, i, sptr, local, torch, np):
    """End to end through the C ABI with the two working sites held in pinned host
    memory: every step uploads them (the state left by the previous step, centre
    on site i+1), runs the same step as the device-timed loop (1q gates, centre
    move, gate or SWAP, split) and reads the two new sites back."""
    from paper_2505_06119_gb300 import MPS

    m = MPS(n, chi, precision="mixed", policy="canon", stream=sptr, device=local, truncation=args.truncation,
            tensor_cores=args.tensor_cores)
    m.set_sites([s.astype(np.complex64) for s in sites], centre=i)
    do_step(m, seq[0], i)
    shape_a = (chi, 2, chi)
    a_h = torch.empty(shape_a, dtype=torch.complex64).pin_memory()
    b_h = torch.empty(shape_a, dtype=torch.complex64).pin_memory()
    an, bn = a_h.numpy(), b_h.numpy()
    m.get_site(i, fmt="c64", out=an)
    m.get_site(i + 1, fmt="c64", out=bn)
    steps = max(1, args.e2e_steps)
    m.sync()
    t0 = time.perf_counter()
    for st in seq[1:1 + steps]:
        m.set_site(i, an)
        m.set_site(i + 1, bn)
        m.set_centre(i + 1)
        do_step(m, st, i)
        m.get_site(i, fmt="c64", out=an)
        m.get_site(i + 1, fmt="c64", out=bn)
    m.sync()
    dt = time.perf_counter() - t0
    m.close()
    nbytes = an.nbytes + bn.nbytes
    return {"value": steps / dt, "seconds": dt, "steps": steps, "h2d": nbytes, "d2h": nbytes}


# ---------------------------------------------------------------------------
def oracle_apply_sample(chi_s, seed, nsteps=2):
    """nsteps oracle steps of the same recipe at bond chi_s (chi_s = 4096 is the
    benchmark's own workload, n = 26): returns seconds per step."""
    from oracle import mps as omps

    n = N_SITES if chi_s == CHI else 2 * int(math.log2(chi_s)) + 2
    i = n // 2 - 1
    sites = make_state(chi_s, n, i, seed)
    seq = step_gates(nsteps, seed + 1)
    o = omps.OracleMPS(n, chi_s, "canon")
    o.set_sites(sites, centre=i)
    del sites
    t0 = time.perf_counter()
    for st in seq:
        u1, u2, g = st
        o.apply_1q(i, u1)
        o.apply_1q(i + 1, u2)
        if g is None:
            o.swap(i)
        else:
            o.apply_2q(i, g)
    return (time.perf_counter() - t0) / len(seq)


def cpu_baseline(args, budget_s=None):
    """The oracle as it stands on this host's cores: a bounded sample of the same
    step recipe at chi = 1024 (an apply at chi = 4096 takes about a minute), scaled to
    the chi = 4096 unit by the cubic work ratio (1024/4096)^3."""
    from oracle import build as obuild
    from oracle import qr as oqr

    obuild.build()
    chi_s = args.cpu_chi
    secs = oracle_apply_sample(chi_s, seed=7, nsteps=args.cpu_steps)
    scale = (chi_s / args.chi) ** 3
    return {"value": scale / secs, "unit": "applies/s", "cores": oqr.num_threads(), "kind": "oracle",
            "sample": "%d oracle steps (same recipe: 1q gates, centre move, gate/SWAP, pivoted-QR split) at "
                      "chi=%d, %.2f s per step; applies/s scaled to chi=%d by (%d/%d)^3" % (
                          args.cpu_steps, chi_s, secs, args.chi, chi_s, args.chi),
            "seconds_per_sample_step": secs}


TRUNCATION_NAMES = {"qrcp": "truncated column-pivoted QR (QP3)",
                    "rqrcp": "truncated QR with randomized column pivoting (RQRCP, sketch of 40 rows)"}


def bench_config(chi, n, i, ws, truncation="qrcp"):
    return {
        "workload": "steady-state two-site apply on a saturated bond, chi_l=chi_m=chi_r=%d, n=%d, "
                    "canonical policy (centre move + 1q gates + gate/SWAP alternating per step)" % (chi, n),
        "chi": chi, "n_sites": n, "bond_site": i, "policy": "canon",
        "precision": "complex64 bulk, FP64 column norms / reflector norms / pivots",
        "truncation": TRUNCATION_NAMES[truncation],
        "l2": "inputs larger than L2 (theta %d MiB)" % (((2 * chi) ** 2 * 8) >> 20),
        "parallelism": "replicas" if ws > 1 else "single GPU",
    }


def reference(args):
    """The CPU oracle on this host's cores (the reference arm): W + K timed steps, each a
    bounded sample of the workload (one oracle step of the same recipe at chi =
    --cpu-chi; value = applies/s scaled to chi by the cubic work ratio), then, unless
    --no-ref-full, one real oracle step at chi itself, reported beside it so that the
    scaled value can be checked against a measured one."""
    ws, rank, local = dist_env()
    if rank != 0:
        return
    from oracle import build as obuild
    from oracle import qr as oqr

    obuild.build()
    chi_s = args.cpu_chi
    for w in range(args.warmup):
        oracle_apply_sample(chi_s, seed=3 + w, nsteps=1)
    times = [oracle_apply_sample(chi_s, seed=11 + s, nsteps=1) for s in range(max(1, args.steps))]
    secs = statistics.mean(times)
    scale = (chi_s / args.chi) ** 3
    value = scale / secs
    full = None
    if not args.no_ref_full:
        fs = oracle_apply_sample(args.chi, seed=1234, nsteps=1)
        full = {"chi": args.chi, "seconds": fs, "applies_per_s": 1.0 / fs,
                "scaled_over_measured": value * fs}
    scaled = value
    if full:
        value = full["applies_per_s"]  # the measured step at the line's own bond dimension
    n = N_SITES if args.chi == CHI else 2 * int(math.log2(args.chi)) + 2
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "applies/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
        "data": "synthetic",
        "config": bench_config(args.chi, n, n // 2 - 1, ws),
        "value_basis": ("value = one measured oracle step at chi=%d (full_step_measured); " % args.chi
                        if full else "value = the samples scaled to chi=%d by (%d/%d)^3; " % (
                            args.chi, chi_s, args.chi)) +
                       "each timed step is one oracle step of the same recipe at chi=%d (ms_per_step is its "
                       "wall time), scaled_value = their applies/s at chi=%d by the cubic work ratio" % (
                           chi_s, args.chi),
        "scaled_value": scaled,
        "full_step_measured": full,
        "cpu_baseline": {"value": value, "unit": "applies/s", "cores": oqr.num_threads(), "kind": "oracle",
                         "sample": "each step: 1 oracle step of the same recipe at chi=%d, scaled to chi=%d "
                                   "by (%d/%d)^3; plus one measured step at chi=%d" % (
                                       chi_s, args.chi, chi_s, args.chi, args.chi)},
        "e2e": {"value": value, "unit": "applies/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def lapack_workload(args):
    """The library CPU line: the same split through SciPy/LAPACK on this host's cores.
    For each chi: theta = gate . (A B) (zgemm), then zgeqp3 (LAPACK's pivoted QR, which
    has no truncation, so it factors the whole 2chi x 2chi theta) and zungqr for the kept
    chi columns; seconds per apply, median of --lapack-reps."""
    import numpy as np
    import scipy.linalg.lapack as la

    from workloads import gates, states

    try:
        blas = np.show_config(mode="dicts")["Build Dependencies"]["blas"]
        blas = "%s %s" % (blas.get("name"), blas.get("version"))
    except Exception:
        blas = "unknown"
    rows = []
    for chi in [int(c) for c in args.lapack_chi.split(",")]:
        rng = np.random.default_rng(chi)
        a = states.complex_gaussian(rng, (chi, 2, chi))
        b = states.complex_gaussian(rng, (chi, 2, chi))
        g = gates.haar_unitary(rng, 4).reshape(2, 2, 2, 2)
        ts = []
        for _ in range(args.lapack_reps):
            t0 = time.perf_counter()
            x = (a.reshape(2 * chi, chi) @ b.reshape(chi, 2 * chi)).reshape(chi, 2, 2, chi)
            theta = np.asfortranarray(np.einsum("abcd,lcdr->labr", g, x).reshape(2 * chi, 2 * chi))
            lw = int(la.zgeqp3(theta, lwork=-1)[3][0].real)  # workspace query: the blocked QP3
            qr_, jpvt, tau, work, info = la.zgeqp3(theta, lwork=max(lw, 1), overwrite_a=1)
            lw2 = int(la.zungqr(qr_[:, :chi], tau[:chi], lwork=-1)[1][0].real)
            q, work, info2 = la.zungqr(qr_[:, :chi], tau[:chi], lwork=max(lw2, 1))
            ts.append(time.perf_counter() - t0)
            assert info == 0 and info2 == 0
        sec = statistics.median(ts)
        rows.append({"chi": chi, "seconds_per_apply": sec, "applies_per_s": 1.0 / sec,
                     "scaled_to_chi_%d" % CHI: (chi / CHI) ** 3 / sec})
    print(json.dumps({"workload": "cpu-lapack", "blas": blas, "cores": os.cpu_count(),
                      "steps": "zgemm + gate + zgeqp3 (full) + zungqr (k = chi)", "rows": rows}), flush=True)


def layer_workload(args):
    """Layer batching (a 64-qubit chain, bonds 2..chi, random canonical state, mixed
    precision, LOCAL policy): one brick-wall layer of Haar SU(4) gates on the even and
    on the odd bonds, applied by mps_apply_layer (replayed as a CUDA graph, and with
    direct launches) and one gate at a time; per-layer milliseconds of each
    (CUDA-synchronised wall clock, after two warm-up layers)."""
    import numpy as np
    import torch

    import __graft_entry__
    from workloads import gates, states

    __graft_entry__.build()
    from paper_2505_06119_gb300 import MPS

    n = 64
    modes = args.layer_modes.split(",")
    out = {"workload": "layer", "n_sites": n, "precision": "mixed", "policy": "local", "rows": []}
    for chi in [int(c) for c in args.layer_chi.split(",")]:
        bonds_ = states.max_bond_dims(n, chi)
        if chi >= 4096:
            # saturated i.i.d. Gaussian sites (the local policy needs no canonical form, and
            # a layer's work depends only on the bond dims); generated in complex64
            rng0 = np.random.default_rng(5)
            sites = []
            for i in range(n):
                shp = (bonds_[i], 2, bonds_[i + 1])
                x = rng0.standard_normal(shp, dtype=np.float32) + 1j * rng0.standard_normal(shp, dtype=np.float32)
                sites.append((x / np.float32(np.sqrt(2.0 * bonds_[i]))).astype(np.complex64))
        else:
            sites = [s.astype(np.complex64) for s in states.random_canonical_mps(n, bonds_, n // 2, seed=5)]
        rng = np.random.default_rng(3)
        row = {"chi": chi}
        for par in (0, 1):
            bonds = list(range(par, n - 1, 2))
            gs = [gates.haar_unitary(rng, 4) for _ in bonds]
            res = {"layer_direct": None, "one_by_one": None, "graph_launches": None}
            for mode in [x for x in ("layer", "layer_direct", "one_by_one") if x in modes]:
                with MPS(n, chi, precision="mixed", policy="local", graphs=(mode == "layer")) as m:
                    for rep in range(3 if chi < 4096 else 2):  # warm-up layers (the second captures the graph)
                        m.set_sites(sites, centre=n // 2)
                        m.sync()
                        torch.cuda.synchronize()
                        t = time.perf_counter()
                        if mode != "one_by_one":
                            m.apply_layer(bonds, gs)
                        else:
                            for q, g in zip(bonds, gs):
                                m.apply_2q(q, g)
                        m.sync()
                        res[mode] = (time.perf_counter() - t) * 1e3
                    if mode == "layer":
                        res["graph_launches"] = m.layer_stats()[1]
            row["even" if par == 0 else "odd"] = {
                "gates": len(bonds), "ms_layer": res.get("layer"), "ms_layer_direct": res["layer_direct"],
                "ms_one_by_one": res["one_by_one"], "graph_launches": res["graph_launches"],
                "speedup": res["one_by_one"] / res["layer"] if res["one_by_one"] and res.get("layer") else None}
            if args.layer_even_only:
                break
        out["rows"].append(row)
    print(json.dumps(out), flush=True)


def circuit_workload(args):
    """Whole circuits (the 40-qubit depth-20 brick-wall at chi 1024 and, reduced, the 7x7
    grid random circuit), mixed and FP64
    paths under the canonical policy: two-qubit gate applies per second of each path
    (CUDA-synchronised wall clock over the whole circuit, routed gates counted once) and
    the mixed-vs-FP64 fidelity deviation at the end (both readings of the deviation:
    relative norm-fidelity difference and 1 - |<mix|64>|^2 / (<mix|mix><64|64>),
    contractions in FP64).  Grid circuits also report the SWAP count, and with the
    permutation approach (--circuit grid-perm) the norm fidelity before and after every
    permutation layer and the average norm fidelity per swap
    f_swap = (F_after / F_before)^(1 / swaps) of Sec. III-E (probe time excluded)."""
    import numpy as np
    import torch

    import __graft_entry__
    from workloads import circuits

    __graft_entry__.build()
    from paper_2505_06119_gb300 import MPS

    if args.circuit == "config2":
        n, chi = 40, 1024
        ops = circuits.brickwall(n, 20, seed=7)
        name = "40-qubit chain, depth-20 brick-wall of Haar SU(4) + SU(2), chi_max=1024, seed 7"
    else:
        rows, cols, cyc = (int(x) for x in args.grid.split("x"))
        n, chi = rows * cols, args.grid_chi
        if args.circuit == "grid":
            ops = circuits.grid_rcs(rows, cols, cyc, seed=11, singles=args.singles)
            how = "SWAP-routed vertical couplers (chains there and back)"
        else:
            ops = circuits.grid_rcs_permuted(rows, cols, cyc, seed=11, singles=args.singles)
            how = ("vertical couplers in a column-snake embedding reached by bubble-sort site "
                   "permutations between the A/B and C/D layers")
        ones = "paper 1q gate set" if args.singles == "paper" else "Haar 1q gates"
        name = ("%dx%d grid random circuit, %d cycles ABCDCDAB, %s and fSim, %s, chi_max=%d, "
                "seed 11" % (rows, cols, cyc, ones, how, chi))
    n2q = circuits.count_two_qubit(ops)
    swaps = sum(2 * (abs(op[2] - op[1]) - 1) for op in ops if op[0] == "2q") + \
        sum(circuits.inversions(op[1]) for op in ops if op[0] == "perm")
    res = {}
    states_ = {}
    for prec in ("mixed", "fp64"):
        m = MPS(n, chi, precision=prec, policy="canon")
        m.sync()
        torch.cuda.synchronize()
        layers = []
        probe_s = 0.0
        t = time.perf_counter()
        for op in ops:
            if op[0] != "perm":
                m.run([op])
                continue
            # norm fidelity before and after the permutation layer (Sec. III-E: f_swap)
            t0 = time.perf_counter()
            f0 = m.fidelity()
            probe_s += time.perf_counter() - t0
            nsw = m.permute(op[1])
            t0 = time.perf_counter()
            f1 = m.fidelity()
            probe_s += time.perf_counter() - t0
            layers.append({"swaps": nsw, "f_before": f0, "f_after": f1,
                           "f_swap": (f1 / f0) ** (1.0 / nsw) if nsw else 1.0})
        m.sync()
        dt = time.perf_counter() - t - probe_s
        res[prec] = {"seconds": dt, "two_qubit_gates_per_s": n2q / dt, "fidelity": m.fidelity(),
                     "max_bond": max(m.bond_dims())}
        if layers:
            tot_sw = sum(x["swaps"] for x in layers)
            ratio = float(np.prod([x["f_after"] / x["f_before"] for x in layers]))
            res[prec]["permutation_layers"] = layers
            res[prec]["f_swap_average"] = ratio ** (1.0 / tot_sw)
        states_[prec] = m
    mm, m64 = states_["mixed"], states_["fp64"]
    o = mm.overlap(m64)
    dev_o = 1.0 - abs(o) ** 2 / (mm.overlap(mm).real * m64.overlap(m64).real)
    dev_f = abs(res["mixed"]["fidelity"] - res["fp64"]["fidelity"]) / res["fp64"]["fidelity"]
    rng = np.random.default_rng(2024)
    amax = dmax = 0.0
    for _ in range(64):  # sampled amplitudes, mixed against FP64
        bits = rng.integers(0, 2, n)
        a64 = m64.amplitude(bits)
        dmax = max(dmax, abs(mm.amplitude(bits) - a64))
        amax = max(amax, abs(a64))
    dsc_mx, dsc_64 = mm.discarded()[0], m64.discarded()[0]
    for m in states_.values():
        m.close()
    print(json.dumps({"workload": "circuit", "circuit": name, "two_qubit_gates": n2q, "swaps": swaps, "paths": res,
                      "speedup_mixed_vs_fp64": res["fp64"]["seconds"] / res["mixed"]["seconds"],
                      "fidelity_dev": {"norm_fidelity_rel": dev_f, "overlap": dev_o, "amplitude_max_abs": dmax,
                                       "amplitude_max_rel": dmax / amax if amax else None,
                                       "discarded_total_rel": abs(dsc_mx - dsc_64) / max(dsc_64, 1e-300)}}),
          flush=True)


FP32_ALU_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12  # CUDA-core FFMA peak at the 2070 MHz maximum clock
FP64_TFLOPS = 1.25  # nominal GB300 FP64 rate


def svd_roofline(m, rows, cols, prec, seconds):
    """Algorithmic work of the Jacobi iteration of the last SVD split: every sweep forms
    the pair sums of all rows*(rows-1)/2 column pairs of theta^H (16 flop per element of
    a column of length cols), and each applied rotation updates two columns of theta^H
    and two of V (20 flop per element pair, lengths cols and rows).  The rate is taken
    over the whole apply (theta and the split included), so it is a lower bound for the
    Jacobi kernel, against the CUDA-core FP32 (mixed) or FP64 peak: the iteration runs on
    the CUDA cores, not the tensor cores."""
    sweeps, rots = m.svd_stats()
    pairs = rows * (rows - 1) // 2
    flops = min(sweeps, 40) * pairs * 16.0 * cols + rots * 20.0 * (cols + rows)
    peak = FP32_ALU_TFLOPS if prec == "mixed" else FP64_TFLOPS
    tf = flops / seconds / 1e12
    return {"jacobi_sweeps": sweeps, "jacobi_rotations": rots, "jacobi_gflop": flops / 1e9,
            "achieved_tflops": tf, "alu_peak_tflops": peak, "frac": tf / peak}


def truncation_workload(args):
    """Pivoted QR versus SVD bond truncation (Sec. IV-A.1) and norm versus overlap
    fidelity (Sec. III-E), FP64, canonical policy.  (1) An n-qubit brick-wall circuit
    run exactly (chi_max = 2^(n/2)) and truncated at several chi_max with each split:
    CUDA-synchronised wall time, norm fidelity F_bar, overlap fidelity
    F = |<exact|trunc>|^2 / (<exact|exact> <trunc|trunc>) from the GPU transfer-matrix
    overlap, and r = F_bar - F.  (2) One apply on a saturated bond (chi_l = chi_m =
    chi_r) with each split, mixed and FP64: seconds per apply and discarded weight."""
    import numpy as np
    import torch

    import __graft_entry__
    from workloads import circuits, gates, states

    __graft_entry__.build()
    from paper_2505_06119_gb300 import MPS

    n, depth = args.trunc_n, args.trunc_depth
    ops = circuits.brickwall(n, depth, seed=7)
    n2q = circuits.count_two_qubit(ops)
    chis = [int(x) for x in args.trunc_chi.split(",") if x]
    exact = MPS(n, 2 ** (n // 2), precision="fp64", policy="canon")
    if chis:
        exact.run(ops)
    fe = exact.fidelity()
    rows = []
    for chi in chis:
        for tr in ("qrcp", "svd"):
            with MPS(n, chi, precision="fp64", policy="canon", truncation=tr) as m:
                m.sync()
                torch.cuda.synchronize()
                t = time.perf_counter()
                m.run(ops)
                m.sync()
                dt = time.perf_counter() - t
                fbar = m.fidelity()
                f = abs(exact.overlap(m)) ** 2 / (fe * fbar)
                rows.append({"chi_max": chi, "split": tr, "seconds": dt, "two_qubit_gates_per_s": n2q / dt,
                             "norm_fidelity": fbar, "overlap_fidelity": f, "r": fbar - f})
    exact.close()
    gate_rows = []
    for chi in (int(x) for x in args.svd_gate_chi.split(",") if x):
        e = int(np.ceil(np.log2(chi))) + 1
        nn, i = 2 * e + 2, e
        g = gates.haar_unitary(np.random.default_rng(1234), 4)
        for prec in ("mixed", "fp64"):
            a, b = states.saturated_two_site(chi, chi, chi, seed=1234)
            for tr in ("qrcp", "svd"):
                with MPS(nn, chi, precision=prec, policy="local", truncation=tr) as m:
                    m.set_site(i, a)
                    m.set_site(i + 1, b)
                    m.apply_2q(i, g)  # warm-up (and the first kernel loads)
                    m.set_site(i, a)
                    m.set_site(i + 1, b)
                    d0 = m.discarded()[0]
                    m.sync()
                    torch.cuda.synchronize()
                    t = time.perf_counter()
                    m.apply_2q(i, g)
                    m.sync()
                    dt = time.perf_counter() - t
                    row = {"chi": chi, "precision": prec, "split": tr, "seconds": dt,
                           "discarded": m.discarded()[0] - d0}
                    if tr == "svd":
                        row.update(svd_roofline(m, 2 * chi, 2 * chi, prec, dt))
                    gate_rows.append(row)
    print(json.dumps({"workload": "truncation",
                      "circuit": "%d-qubit chain, depth-%d brick-wall of Haar SU(4) + SU(2), seed 7" % (n, depth),
                      "two_qubit_gates": n2q, "exact_norm": fe, "circuit_rows": rows,
                      "gate": "one apply on a saturated bond chi_l = chi_m = chi_r, seed 1234, LOCAL policy",
                      "gate_rows": gate_rows}), flush=True)


def iqft_workload(args):
    """Random-saturation IQFT (Sec. IV-D.1, the IQFT output-fidelity study; Sec. III-D.1): an
    n-qubit random mixed-canonical state whose bonds are filled to a fraction sigma of
    chi_max (bond min(chain bound, sigma chi)), then the IQFT on all qubits as one
    controlled-phase MPO of bond 2 per qubit, applied by zip-up, CANON policy.  Per
    sigma and precision: CUDA-synchronised seconds, the norm fidelity after the IQFT,
    and the splits (zip-up + recompression).  For the smallest sigma the gate-by-gate
    IQFT (controlled phases routed by SWAP chains) is timed too."""
    import numpy as np
    import torch

    import __graft_entry__
    from workloads import circuits, states

    __graft_entry__.build()
    from paper_2505_06119_gb300 import MPS

    n, chi = args.iqft_n, args.iqft_chi
    sigmas = [float(x) for x in args.iqft_sigma.split(",") if x]
    mpo_ops = circuits.iqft_mpo(list(range(n)))
    gate_ops = circuits.iqft_noswap(list(range(n)))
    rows = []
    for sg in sigmas:
        fill = max(1, int(round(sg * chi)))
        bonds = [min(b, fill) for b in states.max_bond_dims(n, chi)]
        sites = states.random_canonical_mps(n, bonds, 0, seed=5)
        runs = [("mpo", mpo_ops, p) for p in ("mixed", "fp64")]
        if sg == min(sigmas):
            runs.append(("gates", gate_ops, "mixed"))
        for how, ops, prec in runs:
            with MPS(n, chi, precision=prec, policy="canon") as m:
                m.set_sites(sites, centre=0)
                d0, c0 = m.discarded()
                m.sync()
                torch.cuda.synchronize()
                t = time.perf_counter()
                m.run(ops)
                m.sync()
                dt = time.perf_counter() - t
                d1, c1 = m.discarded()
                rows.append({"sigma": sg, "input_bond": max(bonds), "iqft": how, "precision": prec, "seconds": dt,
                             "norm_fidelity": m.fidelity(), "splits": c1 - c0, "discarded_sum": d1 - d0,
                             "max_bond": max(m.bond_dims())})
    print(json.dumps({"workload": "iqft", "n": n, "chi_max": chi,
                      "input": "random mixed-canonical MPS, bonds min(chain bound, sigma chi_max), seed 5",
                      "rows": rows}), flush=True)


def big_gate_workload(args):
    """One two-site apply at the paper's largest bond dimension (chi_l = chi_m = chi_r =
    args.big_chi, theta (2 chi)^2; the size of the quantum phase estimation circuit's central
    gate), mixed path, through the
    raw-pointer C call on device buffers: Gaussian sites made on the GPU, seeded.  Checks
    the norm identity ||R P^T||^2 + discarded = ||theta||^2 with ||theta||^2 =
    sum (A^H A) .* conj(B B^H) (the gate is unitary on the physical indices)."""
    import ctypes

    import numpy as np
    import torch

    import __graft_entry__
    from workloads import gates

    __graft_entry__.build()
    from paper_2505_06119_gb300 import _lib as L
    from paper_2505_06119_gb300.mps import _gate

    lib = L.load()
    chi = args.big_chi
    dev = torch.device("cuda:0")
    gen = torch.Generator(device=dev)
    gen.manual_seed(5)

    def site():
        x = torch.randn((chi, 2, chi), dtype=torch.complex64, device=dev, generator=gen)
        return x / torch.linalg.vector_norm(x)

    a, b = site(), site()
    g = gates.haar_unitary(np.random.default_rng(5), 4)
    torch.backends.cuda.matmul.allow_tf32 = False
    A2 = a.reshape(2 * chi, chi)
    B2 = b.reshape(chi, 2 * chi)
    theta2 = float(((A2.conj().T @ A2) * (B2 @ B2.conj().T).conj()).sum().real)
    sz = ctypes.c_size_t()
    code = L.MPS_PREC_MIXED
    assert lib.mps_two_site_workspace(code, chi, chi, chi, chi, ctypes.byref(sz)) == 0
    ws = torch.empty(sz.value + 256, dtype=torch.uint8, device=dev)
    base = (ws.data_ptr() + 255) // 256 * 256
    disc = torch.zeros(1, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream().cuda_stream
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    rc = lib.mps_two_site_apply(code, chi, chi, chi, chi, a.data_ptr(), b.data_ptr(), _gate(g, 16), a.data_ptr(),
                                b.data_ptr(), disc.data_ptr(), base, sz.value, stream)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    kept = float((b.abs() ** 2).sum())
    flops = 82.7 * chi ** 3
    print(json.dumps({"workload": "big_gate", "chi": chi, "theta": "%d x %d complex64" % (2 * chi, 2 * chi),
                      "rc": rc, "seconds": ms / 1e3, "applies_per_s": 1e3 / ms,
                      "tflops_algorithmic": flops / (ms * 1e-3) / 1e12,
                      "workspace_gib": sz.value / 2 ** 30,
                      "norm_identity_rel": abs(kept + disc.item() - theta2) / theta2}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--chi", type=int, default=CHI)
    ap.add_argument("--fp64-steps", type=int, default=19)
    ap.add_argument("--amp-samples", type=int, default=64)
    ap.add_argument("--tensor-cores", action="store_true",
                    help="mixed path: long complex products on the tcgen05 tensor cores (3xTF32)")
    ap.add_argument("--truncation", default="qrcp", choices=["qrcp", "rqrcp"],
                    help="split of the gate workload: the deterministic pivoted QR (the metric's) or "
                         "randomized pivoting")
    ap.add_argument("--fp64-warmup", type=int, default=1)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--cpu-chi", type=int, default=1024)
    ap.add_argument("--cpu-steps", type=int, default=6)
    ap.add_argument("--no-ref-full", action="store_true", help="reference arm: skip the real chi-sized step")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--skip-overlap", action="store_true")
    ap.add_argument("--workload", default="gate",
                    choices=["gate", "layer", "circuit", "big", "truncation", "iqft", "cpu-lapack"],
                    help="gate: the headline metric; layer: batched vs one-by-one layer times; "
                         "circuit: whole-circuit throughput and fidelity deviation; "
                         "big: one apply at a large bond dimension; "
                         "truncation: pivoted QR vs SVD splits (fidelity, runtime); "
                         "iqft: random-saturation IQFT by controlled-phase MPOs; "
                         "cpu-lapack: the split through SciPy/LAPACK on the host cores")
    ap.add_argument("--lapack-chi", default="512,1024,2048")
    ap.add_argument("--lapack-reps", type=int, default=2)
    ap.add_argument("--iqft-n", type=int, default=20)
    ap.add_argument("--iqft-chi", type=int, default=128)
    ap.add_argument("--iqft-sigma", default="0.125,0.25,0.5,1.0")
    ap.add_argument("--trunc-n", type=int, default=16)
    ap.add_argument("--trunc-depth", type=int, default=16)
    ap.add_argument("--trunc-chi", default="8,16,32")
    ap.add_argument("--svd-gate-chi", default="64,256,512")
    ap.add_argument("--big-chi", type=int, default=16384)
    ap.add_argument("--layer-chi", default="256,1024,2048")
    ap.add_argument("--layer-modes", default="layer,layer_direct,one_by_one")
    ap.add_argument("--layer-even-only", action="store_true")
    ap.add_argument("--circuit", default="config2", choices=["config2", "grid", "grid-perm"])
    ap.add_argument("--grid-chi", type=int, default=256)
    ap.add_argument("--grid", default="7x7x12", help="rows x cols x cycles of the grid circuit")
    ap.add_argument("--singles", default="paper", choices=["paper", "haar"],
                    help="one-qubit gates of the grid circuit: the paper's sqrt X/Y/W set or Haar SU(2)")
    args = ap.parse_args()
    if args.workload == "layer":
        layer_workload(args)
    elif args.workload == "circuit":
        circuit_workload(args)
    elif args.workload == "big":
        big_gate_workload(args)
    elif args.workload == "truncation":
        truncation_workload(args)
    elif args.workload == "iqft":
        iqft_workload(args)
    elif args.workload == "cpu-lapack":
        lapack_workload(args)
    elif args.impl == "reference":
        reference(args)
    else:
        ours(args)


if __name__ == "__main__":
    main()
