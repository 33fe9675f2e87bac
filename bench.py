"""Benchmark of the L-ACE exchange hot path on one GB300 (or N independent replicas).

Workload: the water-like localized-exchange system -- cubic L = 23.5 bohr,
72^3 grid, 256 occupied orbitals (Gaussian sums around 192 centres,
band-limited to 40 Ha), SCDM on the 1/8 grid subsample, overlap-of-moduli
screening at S_thr = 1e-3.  One step is the whole hot path on inputs already
in HBM: Loewdin orthonormalisation, SCDM localisation, screening, the
screened pair convolutions with E_x, the ACE build (M, Cholesky, xi) and one
ACE application to the N_P orbitals.  The metric counts the real pair
convolutions (Poisson solves) of the step.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl lace|reference]
Under torchrun each rank runs its own replica of the workload (weak scaling,
no collective on the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
from concurrent.futures import ThreadPoolExecutor
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "Fock pair-convolutions/s & ACE build ms vs plain FP64 at stated dE_x; p99 latency"
UNIT = "pair-convolutions/s"
S_THR = 1e-3
STRIDE = 2
B_ALG_PER_PAIR_FP32 = 16  # bytes per grid point per real pair (3-pass FFT model)
# sources of the pair-convolution kernels: the committed DRAM-traffic capture
# (profiles/pairconv_traffic.json) holds their hash and counts only while they match
PAIRCONV_SOURCES = ("common.cuh", "dft_packed.cuh", "f32x2.cuh", "lace_internal.cuh", "pairconv.cu", "pairconv_spec.cuh",
                    "pairconv_spec2.cuh", "pairconv_spec_s.cu", "pairconv_spec_m.cu",
                    "pairconv_spec_l.cu")


def pairconv_sources_sha256() -> str:
    import hashlib

    h = hashlib.sha256()
    for f in PAIRCONV_SOURCES:
        with open(os.path.join(ROOT, "paper_1801_09263_gb300", "csrc", f), "rb") as fh:
            h.update(f.encode() + b"\0" + fh.read())
    return h.hexdigest()


def committed_traffic():
    """(bytes per step, note) of the committed DRAM-traffic capture; bytes is
    None when the kernels changed since the capture."""
    tr = os.path.join(ROOT, "profiles", "pairconv_traffic.json")
    try:
        d = json.load(open(tr))
    except Exception:
        return None, "no committed capture"
    when = d.get("captured", "?")
    if d.get("kernel_sources_sha256") != pairconv_sources_sha256():
        return None, f"stale: the pair-convolution sources changed since the capture of {when}"
    return d["traffic_bytes_per_step"], f"ncu capture of {when} ({d.get('workload', '')})"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="lace", choices=["lace", "reference"])
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-fp64", action="store_true")
    p.add_argument("--profile-pairconv", action="store_true",
                   help="only the pair convolutions of a 64-orbital 72^3 set (for ncu captures)")
    p.add_argument("--fp64", action="store_true", help="with --profile-pairconv: FP64 path")
    p.add_argument("--profile-n", type=int, default=72, help="with --profile-pairconv: cubic grid size")
    p.add_argument("--serving", action="store_true",
                   help="only the serving stream (32 resident systems, Poisson arrivals, p50/p99 latency)")
    p.add_argument("--serve-iters", type=int, default=10, help="SCF-like iterations per system (--serving)")
    p.add_argument("--serve-systems", type=int, default=32)
    p.add_argument("--serve-slots", type=int, default=8)
    p.add_argument("--serve-rebuild-slots", type=int, default=4)
    p.add_argument("--serve-fp64", action="store_true", help="serve in the plain FP64 form (for comparison)")
    p.add_argument("--serve-no-merge", action="store_true",
                   help="serve without merged pair convolutions and REBUILD groups (for comparison)")
    p.add_argument("--no-serving", action="store_true", help="skip the serving sample of the default run")
    p.add_argument("--batched", action="store_true",
                   help="only the batched uneven instances (48 systems, persistent launch in a CUDA graph)")
    p.add_argument("--no-batched", action="store_true", help="skip the batched sample of the default run")
    p.add_argument("--batch-instances", type=int, default=48, help="instances of --batched (fewer for ncu captures)")
    p.add_argument("--no-ace96", action="store_true", help="skip the 96^3 ACE build comparison of the default run")
    p.add_argument("--ace96", action="store_true", help="only the 96^3 ACE build comparison")
    return p.parse_args()


def max_over_ranks(ms: float, world: int, device=None) -> float:
    """The slowest rank's time: every rank runs its own replica (weak scaling),
    so the job is done when the last one is."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist

    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(units: float, world: int, device=None) -> float:
    """Units processed by all ranks together."""
    if world <= 1:
        return units
    import torch
    import torch.distributed as dist

    t = torch.tensor([units], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload(seed):
    import synth

    return synth.config2_water_like(seed=seed)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for k, name in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(name)
        busy = [x for x in sm if smax and x > 0.5 * smax] or sm
        return {"sm_mhz": statistics.median(busy) if busy else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def run_lace(args, rank, world, local):
    import torch

    import paper_1801_09263_gb300 as lace
    from paper_1801_09263_gb300.build import build

    build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    sysm = workload(1801 + 1 + rank)
    n, ng = sysm.n_occ, int(np.prod(sysm.shape))
    phi_dev = torch.from_numpy(sysm.phi).to(dev)
    stream = torch.cuda.current_stream(dev)

    def barrier():
        if world > 1:
            import torch.distributed as dist

            dist.barrier()
        torch.cuda.synchronize(dev)

    def make_ctx(prec):
        ctx = lace.Lace(local, prec)
        ctx.set_stream(stream.cuda_stream)
        ctx.set_cell(sysm.cell, sysm.shape, sysm.ecut)
        return ctx

    out_dev = torch.empty_like(phi_dev)

    def step(ctx):
        ctx.load_orbitals_dev(phi_dev, n, 0, True)
        ctx.localize(STRIDE)
        npairs = ctx.screen(S_THR)
        ctx.apply_exchange(want_W=False)
        ctx.build_ace(lace.LACE_SYM_AVG)
        ctx.apply_ace_dev(phi_dev, out_dev)
        return npairs

    # ---------------- mixed precision (headline)
    ctx = make_ctx(lace.LACE_MIXED)
    for _ in range(args.warmup):
        npairs = step(ctx)
    launches0 = ctx.launch_count()
    pc_ms, ace_ms, step_ms = [], [], []
    sampler = ClockSampler(local)
    barrier()
    sampler.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        e_a = torch.cuda.Event(enable_timing=True)
        e_b = torch.cuda.Event(enable_timing=True)
        e_a.record(stream)
        npairs = step(ctx)
        e_b.record(stream)
        t = ctx.get_timings()
        pc_ms.append(t["pairconv_kernels"])
        ace_ms.append(t["ace_build"])
        e_b.synchronize()
        step_ms.append(e_a.elapsed_time(e_b))
    ev1.record(stream)
    barrier()
    clocks = sampler.stop()
    total_ms = ev0.elapsed_time(ev1)
    launches = ctx.launch_count() - launches0
    stages = ctx.get_timings()
    ex_mixed = ctx.exchange_energy(1.0)
    total_ms = max_over_ranks(total_ms, world, dev)
    value = sum_over_ranks(npairs * args.steps, world, dev) / (total_ms / 1e3)

    # ---------------- plain FP64 GPU form (same step)
    fp64 = None
    if not args.no_fp64:
        c64 = make_ctx(lace.LACE_FP64)
        step(c64)
        barrier()
        e_a = torch.cuda.Event(enable_timing=True)
        e_b = torch.cuda.Event(enable_timing=True)
        e_a.record(stream)
        np64 = step(c64)
        e_b.record(stream)
        e_b.synchronize()
        t64 = e_a.elapsed_time(e_b)
        st64 = c64.get_timings()
        ex64 = c64.exchange_energy(1.0)
        fp64 = {"pair_convolutions_per_s": np64 / (t64 / 1e3), "step_ms": t64, "n_pairs": np64,
                "pairconv_kernels_ms": st64["pairconv_kernels"], "ace_build_ms": st64["ace_build"],
                "E_x_Ha": ex64, "dE_x_mixed_vs_fp64_Ha": ex_mixed - ex64}
        c64.close()

    # ---------------- end to end through the host API (pinned host buffers)
    e2e = None
    if not args.no_e2e:
        phi_pin = torch.from_numpy(sysm.phi).pin_memory()
        w_pin = torch.empty_like(phi_pin).pin_memory()
        k_pin = torch.empty_like(phi_pin).pin_memory()
        phi_np, w_np, k_np = phi_pin.numpy(), w_pin.numpy(), k_pin.numpy()
        import ctypes as C

        def e2e_step():
            ctx._check(ctx.lib.lace_load_orbitals(ctx.h, phi_np.ctypes.data_as(C.c_void_p), n, 0, 1), "load")
            ctx.localize(STRIDE)
            ctx.screen(S_THR)
            ex = C.c_double()
            ctx._check(ctx.lib.lace_apply_exchange(ctx.h, w_np.ctypes.data_as(C.c_void_p), C.byref(ex)), "apply")
            ctx.build_ace(lace.LACE_SYM_AVG)
            ctx._check(ctx.lib.lace_apply_ace(ctx.h, phi_np.ctypes.data_as(C.c_void_p), n,
                                              k_np.ctypes.data_as(C.c_void_p)), "apply ace")
            return ex.value

        e2e_step()
        barrier()
        t0 = time.perf_counter()
        ksteps = max(1, min(args.steps, 3))
        for _ in range(ksteps):
            e2e_step()
        barrier()
        dt = max_over_ranks(time.perf_counter() - t0, world, dev)
        e2e = {"value": sum_over_ranks(npairs * ksteps, world, dev) / dt, "unit": UNIT,
               "h2d_bytes_per_step": 2 * phi_np.nbytes, "d2h_bytes_per_step": w_np.nbytes + k_np.nbytes + 8,
               "steps": ksteps}
    ctx.close()

    # ---------------- roofline of the pair-convolution kernels
    peak, peak_kind = peaks()
    pc_avg = statistics.mean(pc_ms)
    # 16 Ng bytes per real pair, plus once per application: read the occupied and
    # target orbitals ((N_occ + N_P) Ng 4 bytes) and write W (N_P Ng 4 bytes)
    alg_bytes = B_ALG_PER_PAIR_FP32 * ng * npairs + (n + n) * ng * 4 + n * ng * 4
    achieved = alg_bytes / (pc_avg / 1e3) / 1e9
    roof = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "traffic": None, "peak_kind": peak_kind,
            "kernel": "pairconv passes A+B+C (per step)", "alg_bytes_per_step": alg_bytes}
    roof["traffic"], roof["traffic_source"] = committed_traffic()
    result = {
        "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(total_ms / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "water-like localized exchange: L=23.5 bohr, 72^3, 256 occupied orbitals, "
                               "SCDM stride 2, S_thr=1e-3, step = Loewdin+SCDM+screen+pair-conv+ACE build+ACE apply",
                   "n_pairs": npairs, "kept_fraction": npairs / (n * (n + 1) / 2), "grid": list(sysm.shape),
                   "n_occ": n, "precision": "mixed (FP32 FFT, FP64 energies and N x N factorisations)",
                   "l2": "inputs (764 MB FP64 orbitals) larger than L2", "parallelism": f"replicas x{world}"},
        "stages_ms": {k: round(v, 3) for k, v in stages.items()},
        "ace_build_ms": round(statistics.mean(ace_ms), 3),
        "latency_ms": {"p50": round(statistics.median(step_ms), 3),
                       "p99": round(float(np.percentile(step_ms, 99)), 3)},
        "roofline": roof, "clocks": clocks, "gpu_launches": launches, "e2e": e2e,
        "fp64_gpu": fp64, "E_x_Ha": ex_mixed,
    }
    try:
        result["alu_peaks_measured"] = {k: round(v, 2) for k, v in lace.probe_peak_rates(local).items()}
    except Exception as exc:  # reported, not fatal
        result["alu_peaks_measured"] = {"error": str(exc)}
    if not args.no_serving:
        # the serving stream (each rank serves its own replica of it)
        del phi_dev, out_dev
        torch.cuda.empty_cache()
        result["serving"] = run_serving(local, args.serve_systems, args.serve_iters, args.serve_slots,
                                        args.serve_rebuild_slots)
        result["latency_ms"] = {"p50": result["serving"]["latency_ms"]["p50"],
                                "p99": result["serving"]["latency_ms"]["p99"],
                                "of": "serving-stream requests (submission to completion)"}
        result["step_latency_ms"] = {"p50": round(statistics.median(step_ms), 3),
                                     "p99": round(float(np.percentile(step_ms, 99)), 3)}
    if not args.no_batched:
        result["batched"] = run_batched(local)
    if not args.no_ace96:
        result["ace_96"] = run_ace96(local)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline(sysm, budget_s=15.0)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(result), flush=True)


def oracle_sample(sysm, n_targets):
    """Localised orbitals and kept pairs from the oracle, plus a target sample."""
    import oracle as O

    g = O.Grid(sysm.cell, sysm.shape)
    occ = O.lowdin(g, sysm.phi[: sysm.n_occ])
    piv, _, w = O.scdm(g, occ, STRIDE)
    s = O.overlap_moduli(g, w)
    keep = O.kept_pairs(s, S_THR, sysm.n_occ, 0)
    rng = np.random.default_rng(0)
    targets = rng.choice(sysm.n_occ, size=n_targets, replace=False)
    return g, w, keep, targets


def cpu_baseline(sysm, budget_s=15.0, prepared=None):
    """Oracle pair convolutions on the host cores, on a bounded sample of targets."""
    import oracle as O

    g, w, keep, targets = prepared or oracle_sample(sysm, 64)
    done, t0 = 0, time.perf_counter()
    used = []
    for j in targets:
        cols = keep[:, j:j + 1]
        O.apply_exchange_columns(g, w, w[j:j + 1], cols)
        done += int(cols.sum())
        used.append(int(j))
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return {"value": round(done / dt, 2), "unit": UNIT, "cores": len(os.sched_getaffinity(0)), "kind": "oracle",
            "sample": f"oracle K psi_j for {len(used)} localized targets ({done} pair convolutions, scipy.fft "
                      f"workers={len(os.sched_getaffinity(0))}) of the same 72^3 workload"}


def run_reference(args, rank, world):
    if rank != 0:
        return
    sysm = workload(1801 + 1)
    prepared = oracle_sample(sysm, 64)
    for _ in range(args.warmup):
        cpu_baseline(sysm, budget_s=2.0, prepared=prepared)
    vals, t0 = [], time.perf_counter()
    for _ in range(args.steps):
        vals.append(cpu_baseline(sysm, budget_s=8.0, prepared=prepared))
    total = time.perf_counter() - t0
    v = statistics.mean(x["value"] for x in vals)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(1e3 * total / args.steps, 1), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "water-like localized exchange: L=23.5 bohr, 72^3, 256 occupied orbitals, "
                               "SCDM stride 2, S_thr=1e-3 (oracle pair convolutions on a target sample)"},
        "cpu_baseline": {"value": v, "unit": UNIT, "kind": "oracle", "cores": vals[0]["cores"],
                         "sample": vals[0]["sample"]},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


SERVE_RATE = 200.0        # offered requests per second over all systems
SERVE_MAX_INNER = 8       # inner-loop K_ACE applications per ACE rebuild at most
SERVE_BLOCK = 32          # functions per application (a block of trial vectors)
SERVE_EPS = 1e-3          # SCF-like drift of the orbitals between rebuilds
SERVE_INNER_EPS = 1e-2    # the inner loop's block moves by SERVE_INNER_EPS x decay^k at its k-th step
SERVE_INNER_DECAY = 0.5
SERVE_CADENCE_TOL = 1e-5  # rebuild once the block's ACE energy moves by less than this (relative)


def run_serving(local, n_systems, iters, slots, rebuild_slots, fp64_sample=4, fp64=False, merging=True):
    """The serving stream: resident systems (N log-uniform in [32, 512],
    2/3/5-smooth cubic grids in [48, 128]), each an SCF-like client running
    the double loop of the paper (Sec. 2): an outer iteration is a REBUILD
    (orthonormalise, SCDM, screen, pair convolutions, ACE build); its inner
    loop applies that ACE projector (APPLY: K_ACE on a block of SERVE_BLOCK
    functions) to a block that moves by SERVE_INNER_EPS x SERVE_INNER_DECAY^k
    at step k, until the server reports the block's ACE energy converged
    (relative change below SERVE_CADENCE_TOL; at most SERVE_MAX_INNER
    applies); then the orbitals drift by SERVE_EPS and the next REBUILD
    follows, for `iters` outer iterations.  Request k of a system arrives at
    its Poisson time (rate SERVE_RATE / n_systems per system, seeded) and is
    submitted at max(arrival, completion of request k-1, the client's own
    host work for it): a client sends its next request only after the
    previous result, and prepares it (drift, next block) on a host thread.  Latency = submission to
    completion (the server's), response = arrival to completion.  Mixed
    precision (or plain FP64 with fp64=True); memory admission with the
    default budget (90% of free device memory); queued REBUILDs on one grid
    size are admitted in groups and share pass launches (merged pair
    convolutions)."""
    import synth
    import torch

    import paper_1801_09263_gb300 as lace

    torch.cuda.set_device(local)
    systems = synth.serving_systems(n_systems=n_systems)
    t0 = time.perf_counter()
    # the client's orbitals, inner-loop blocks and results live in pinned host memory
    phis, blocks, outs = [], [], []
    for s in systems:
        nb = min(SERVE_BLOCK, s.n_occ)
        phis.append(synth.serving_orbitals(
            s, torch.empty((s.n_occ,) + s.shape, dtype=torch.float64, pin_memory=True).numpy()))
        blocks.append(torch.empty((nb,) + s.shape, dtype=torch.float64, pin_memory=True).numpy())
        outs.append(torch.empty((nb,) + s.shape, dtype=torch.float64, pin_memory=True).numpy())
    gen_s = time.perf_counter() - t0
    rng = np.random.default_rng(1801 + 4 + 1000)
    nreq_max = iters * (SERVE_MAX_INNER + 1)
    gaps = rng.exponential(n_systems / SERVE_RATE, size=(n_systems, nreq_max))
    arrivals = np.cumsum(gaps, axis=1)
    srv = lace.Server(local, lace.LACE_FP64 if fp64 else lace.LACE_MIXED, slots=slots, rebuild_slots=rebuild_slots)
    if not merging:
        srv.set_pair_merging(False, 0.0)
    sids = [srv.add_system(s.cell, s.shape, s.ecut, s.n_occ, 0, S_THR) for s in systems]
    for sid in sids:
        srv.set_rebuild_tolerance(sid, SERVE_CADENCE_TOL)
    step = [0] * n_systems        # requests sent
    outer = [0] * n_systems       # REBUILDs sent
    inner = [0] * n_systems       # APPLYs sent since the last REBUILD
    next_kind = ["rebuild"] * n_systems
    outstanding = [None] * n_systems
    lat = {"rebuild": [], "apply": []}
    resp = []
    pairs = 0
    ex_last = [None] * n_systems
    inner_counts, due_count = [], 0
    peak_running, peak_bytes = 0, 0
    fails = []

    def prep_rebuild(k, drift):
        # SCF-like drift of the orbitals; the inner loop's block starts from them
        t = time.perf_counter()
        if drift:
            synth.perturb_in_place(phis[k], SERVE_EPS)
        blocks[k][...] = phis[k][: len(blocks[k])]
        return time.perf_counter() - t

    def prep_apply(k, i):
        # the inner loop's block moves less at every step
        t = time.perf_counter()
        if i > 0:
            synth.perturb_in_place(blocks[k], SERVE_INNER_EPS * SERVE_INNER_DECAY ** i)
        return time.perf_counter() - t

    # the clients' host work (drift of up to 4 GB of orbitals a system) runs
    # on a thread pool so that one client's preparation does not hold up the
    # others' submissions
    pool = ThreadPoolExecutor(max_workers=max(1, min(16, os.cpu_count() or 1)))
    prep = [None] * n_systems
    prep_s = 0.0
    t_start = time.perf_counter()
    done_all = 0
    finished = [False] * n_systems
    while done_all < n_systems:
        now = time.perf_counter() - t_start
        for k in range(n_systems):
            if finished[k]:
                continue
            cur = outstanding[k]
            if cur is not None:
                rid, kind = cur
                r = srv.poll(rid, wait=False)
                if r is None:
                    continue
                outstanding[k] = None
                if r["status"] != 0:
                    fails.append({"system": k, "kind": kind, "status": r["status"], "error": r["error"]})
                lat[kind].append(r["latency_ms"])
                resp.append(1e3 * (time.perf_counter() - t_start - arrivals[k][step[k] - 1]))
                if kind == "rebuild":
                    pairs += r["n_pairs"]
                    ex_last[k] = r["ex"] if r["status"] == 0 else None
                    next_kind[k] = "apply"
                else:
                    due = r["rebuild_due"]
                    due_count += int(due)
                    if due or inner[k] >= SERVE_MAX_INNER:
                        inner_counts.append(inner[k])
                        next_kind[k] = "rebuild" if outer[k] < iters else "done"
                    else:
                        next_kind[k] = "apply"
                if next_kind[k] == "done":
                    finished[k] = True
                    done_all += 1
                    continue
            if outstanding[k] is None and prep[k] is None:
                # the client's own work before its next request, on a host thread
                if next_kind[k] == "rebuild":
                    prep[k] = pool.submit(prep_rebuild, k, outer[k] > 0)
                else:
                    prep[k] = pool.submit(prep_apply, k, inner[k])
            if outstanding[k] is None and prep[k].done() and now >= arrivals[k][step[k]]:
                prep_s += prep[k].result()
                prep[k] = None
                if next_kind[k] == "rebuild":
                    outstanding[k] = (srv.submit_rebuild(sids[k], phis[k]), "rebuild")
                    outer[k] += 1
                    inner[k] = 0
                else:
                    outstanding[k] = (srv.submit_apply(sids[k], blocks[k], outs[k]), "apply")
                    inner[k] += 1
                step[k] += 1
        st = srv.stats()
        peak_running = max(peak_running, st["running"])
        peak_bytes = max(peak_bytes, st["bytes_resident"])
        time.sleep(0.0005)
    makespan = time.perf_counter() - t_start
    pool.shutdown()
    merge = srv.merge_stats()
    srv.close()
    # accuracy: the last rebuild of the smallest systems against the plain FP64 GPU form
    order = sorted((k for k in range(n_systems) if ex_last[k] is not None),
                   key=lambda k: systems[k].n_occ * int(np.prod(systems[k].shape)))
    dex = []
    for k in order[:fp64_sample]:
        s = systems[k]
        with lace.Lace(local, lace.LACE_FP64) as c64:
            c64.set_cell(s.cell, s.shape, s.ecut)
            c64.load_orbitals(phis[k], s.n_occ, 0, True)
            c64.localize(STRIDE)
            c64.screen(S_THR)
            _, ex64 = c64.apply_exchange(want_W=False)
        dex.append(abs(ex_last[k] - ex64))
    all_lat = lat["rebuild"] + lat["apply"]

    def pct(v, q):
        return round(float(np.percentile(v, q)), 3) if v else None

    return {
        "workload": f"{n_systems} resident systems, N log-uniform [32,512], cubic 2/3/5-smooth grids [48,128], "
                    f"{iters} SCF-like outer iterations x (1 rebuild + applies of {SERVE_BLOCK} orbitals until the "
                    f"block's ACE energy moves by < {SERVE_CADENCE_TOL:g} relative, at most {SERVE_MAX_INNER}), "
                    f"Poisson arrivals {SERVE_RATE:g} req/s offered, closed loop per system, {slots} slots "
                    f"({rebuild_slots} for rebuilds), "
                    f"S_thr={S_THR:g}, {'plain FP64' if fp64 else 'mixed precision'}, "
                    f"{'merged pair convolutions of same-grid REBUILD groups' if merging else 'no merging'}",
        "requests": len(all_lat), "failed": fails[:8], "n_failed": len(fails),
        "latency_ms": {"p50": pct(all_lat, 50), "p99": pct(all_lat, 99),
                       "rebuild_p50": pct(lat["rebuild"], 50), "rebuild_p99": pct(lat["rebuild"], 99),
                       "apply_p50": pct(lat["apply"], 50), "apply_p99": pct(lat["apply"], 99)},
        "response_ms": {"p50": pct(resp, 50), "p99": pct(resp, 99), "of": "arrival to completion"},
        "latency_from": "submission to completion (each system submits its next request once the previous completed)",
        "served_req_per_s": round(len(all_lat) / makespan, 1), "offered_req_per_s": SERVE_RATE,
        "merged_pair_convolutions": merge,
        "inner_applies_per_rebuild": {"mean": round(float(np.mean(inner_counts)), 2) if inner_counts else None,
                                      "max": int(max(inner_counts)) if inner_counts else None,
                                      "ended_by_convergence": due_count, "outer_iterations": len(inner_counts)},
        "pair_convolutions_per_s": round(pairs / makespan, 1), "pair_convolutions": int(pairs),
        "makespan_s": round(makespan, 3), "peak_running": peak_running,
        "peak_resident_GB": round(peak_bytes / 1e9, 2),
        "dE_x_vs_fp64_gpu_Ha": {"max": max(dex) if dex else None, "systems": len(dex)},
        "orbital_generation_s": round(gen_s, 1),
        "client_host_prep_s": round(prep_s, 1),
    }


ACE96_ORACLE = os.path.join(ROOT, "tests", "golden", "ace96_oracle_sample.json")


def run_ace96(local, reps=3):
    """ACE build and apply on the 96^3 workload: 256 water-like occupied + 128
    extra orbitals (N_P = 384), S_thr = 1e-3.  Mixed precision (tcgen05 3xBF16
    M' and xi, FP64 Cholesky) and the plain FP64 GPU form, both on the FP64
    oracle's SCDM points: ACE build ms (CUDA events), E_x, and K_ACE on 8
    random probes, each against the oracle's values stored in
    tests/golden/ace96_oracle_sample.json (written by the committed script
    beside it from oracle/ alone: E_x and K_ACE psi on 512 seeded points per
    probe, scaled by the probe's largest |K_ACE psi|) and against each other."""
    import synth
    import torch

    import paper_1801_09263_gb300 as lace

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if not os.path.exists(ACE96_ORACLE):
        return {"error": "tests/golden/ace96_oracle_sample.json missing (run tests/golden/make_ace96_oracle.py)"}
    with open(ACE96_ORACLE) as f:
        gold = json.load(f)
    sysm = synth.config3_water_like_with_extras()
    phi = torch.from_numpy(sysm.phi).to(dev)
    probe = torch.from_numpy(np.random.default_rng(gold["probe"]["seed"]).standard_normal(
        (gold["probe"]["count"],) + sysm.shape)).to(dev)
    pts = torch.tensor(gold["sample_points"], dtype=torch.long, device=dev)
    k_ref = np.array(gold["k_ace_sample"])
    k_scale = np.array(gold["k_ace_max_abs"])
    out = {}
    for name, prec in (("mixed", lace.LACE_MIXED), ("fp64", lace.LACE_FP64)):
        with lace.Lace(local, prec) as c:
            c.set_stream(torch.cuda.current_stream(dev).cuda_stream)
            c.set_cell(sysm.cell, sysm.shape, sysm.ecut)
            c.load_orbitals_dev(phi, 256, 128, True)
            c.set_pivots(np.array(gold["pivots"], dtype=np.int64))
            npairs = c.screen(S_THR)
            c.apply_exchange(want_W=False)
            builds = []
            for _ in range(reps):
                c.build_ace(lace.LACE_SYM_AVG)
                builds.append(c.get_timings()["ace_build"])
            kp = torch.empty_like(probe)
            c.apply_ace_dev(probe, kp)
            torch.cuda.synchronize(dev)
            t = c.get_timings()
            ex = c.exchange_energy(1.0)
            ks = kp.reshape(kp.shape[0], -1)[:, pts].cpu().numpy()
            out[name] = {"ace_build_ms": round(statistics.median(builds), 3), "ace_apply_ms_8": round(t["ace_apply"], 3),
                         "pairconv_ms": round(t["pairconv_kernels"], 3), "n_pairs": npairs, "E_x_Ha": ex,
                         "dE_x_vs_oracle_Ha": ex - gold["E_x_Ha"],
                         "max_rel_dK_psi_vs_oracle": float(np.max(np.abs(ks - k_ref) / k_scale[:, None])),
                         "kprobe": kp}
    dk = (out["mixed"]["kprobe"] - out["fp64"]["kprobe"]).abs().max() / out["fp64"]["kprobe"].abs().max()
    for v in out.values():
        del v["kprobe"]
    return {"workload": "water-like L=23.5 bohr, 96^3, 256 occupied + 128 extra orbitals (N_P=384), SCDM stride 2, "
                        "S_thr=1e-3; both forms on the FP64 oracle's SCDM points",
            "oracle": {"E_x_Ha": gold["E_x_Ha"], "n_pairs": gold["n_pairs"],
                       "sample": f"K_ACE psi of {gold['probe']['count']} probes on {len(gold['sample_points'])} "
                                 "seeded grid points each (tests/golden/ace96_oracle_sample.json)"},
            "mixed": out["mixed"], "fp64_gpu": out["fp64"],
            "ace_build_speedup_vs_fp64": round(out["fp64"]["ace_build_ms"] / out["mixed"]["ace_build_ms"], 1),
            "dE_x_mixed_vs_fp64_Ha": out["mixed"]["E_x_Ha"] - out["fp64"]["E_x_Ha"],
            "max_rel_dK_psi_mixed_vs_fp64": float(dk)}


def run_batched(local, steps=5, n_instances=48):
    """Batched uneven instances: 48 cubic cells (L ~ U[10, 20] bohr, 2/3/5-smooth
    grids in [32, 64], N log-uniform in [16, 128], S_thr = 1e-3), localised
    exchange + ACE build for all of them per step through one lace_batch:
    run 1 eager (with the launch-shape autotuning), run 2 captures the CUDA
    graph, then `steps` timed runs replay it (host wall clock per run; the
    device time of the pair convolutions and of the whole graph from the
    library's events)."""
    import synth
    import torch

    import paper_1801_09263_gb300 as lace

    torch.cuda.set_device(local)
    inst = synth.batch_instances(n_instances=n_instances)
    phis = [synth.serving_orbitals(s) for s in inst]
    with lace.Batch([(s.cell, s.shape, s.ecut, s.n_occ, S_THR) for s in inst], device=local) as b:
        for q, p in enumerate(phis):
            b.set_orbitals(q, p)
        t0 = time.perf_counter()
        ex, st = b.run()
        first_s = time.perf_counter() - t0
        b.run()
        walls, pcs, hots, setups = [], [], [], []
        for _ in range(steps):
            t0 = time.perf_counter()
            ex, st = b.run()
            walls.append(1e3 * (time.perf_counter() - t0))
            inf = b.info()
            pcs.append(inf["pairconv_ms"])
            hots.append(inf["hot_ms"])
            setups.append(inf["setup_ms"])
        npairs = sum(len(b.context(q).get_pairs()) for q in range(len(inst)))
        inf = b.info()
    wall = statistics.median(walls)
    return {
        "workload": f"{n_instances} cubic cells, L~U[10,20] bohr, 2/3/5-smooth grids [32,64], N log-uniform [16,128], "
                    f"S_thr={S_THR:g}, localised exchange + ACE build per instance, mixed precision",
        "instances": n_instances, "failed": int((st != 0).sum()), "pair_convolutions": int(npairs),
        "step_ms": round(wall, 3), "instances_per_s": round(n_instances / (wall / 1e3), 1),
        "pair_convolutions_per_s": round(npairs / (wall / 1e3), 1),
        "setup_ms": round(statistics.median(setups), 3),
        "pairconv_device_ms": round(statistics.median(pcs), 3),
        "graph_device_ms": round(statistics.median(hots), 3),
        "pair_convolutions_per_s_device": round(npairs / (statistics.median(pcs) / 1e3), 1),
        "launch_shape": {"threads": inf["threads"], "ctas_per_sm": inf["ctas_per_sm"], "chunks": inf["chunks"],
                         "tuned_ms": inf["tune_ms"]},
        "graph_replays": inf["graph_replays"], "first_run_s": round(first_s, 3),
        "E_x_Ha_sum": float(np.sum(ex)),
    }


def run_profile(args, local):
    """Pair convolutions only: 64 orbitals on the 72^3 grid (--profile-n), every pair (2080)."""
    import synth
    import torch

    import paper_1801_09263_gb300 as lace
    from paper_1801_09263_gb300.build import build

    build()
    torch.cuda.set_device(local)
    n = args.profile_n
    L = 23.5 * n / 72.0
    sysm = synth.small_localized_system(7, (L, L, L), (n, n, n), 40.0 * min(1.0, (n / 72.0) ** 2), 48, 64)
    ctx = lace.Lace(local, lace.LACE_FP64 if args.fp64 else lace.LACE_MIXED)
    ctx.set_cell(sysm.cell, sysm.shape, sysm.ecut)
    ctx.load_orbitals(sysm.phi, sysm.n_occ, 0, False)
    for _ in range(max(1, args.steps)):
        ctx.apply_exchange(want_W=False)
    t = ctx.get_timings()
    npairs = sysm.n_occ * (sysm.n_occ + 1) // 2
    print(json.dumps({"profile": "pairconv", "grid": n, "n_pairs": npairs, "pairconv_ms": t["pairconv_kernels"],
                      "us_per_pair": 1e3 * t["pairconv_kernels"] / npairs}), flush=True)
    ctx.close()


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.profile_pairconv:
        run_profile(args, local)
    elif args.ace96:
        from paper_1801_09263_gb300.build import build

        build()
        print(json.dumps({"ace_96": run_ace96(local)}), flush=True)
    elif args.batched:
        from paper_1801_09263_gb300.build import build

        build()
        print(json.dumps({"batched": run_batched(local, steps=max(1, args.steps), n_instances=args.batch_instances)}),
              flush=True)
    elif args.serving:
        from paper_1801_09263_gb300.build import build

        build()
        print(json.dumps({"serving": run_serving(local, args.serve_systems, args.serve_iters, args.serve_slots,
                                                 args.serve_rebuild_slots, fp64=args.serve_fp64,
                                                 merging=not args.serve_no_merge)}), flush=True)
    elif args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_lace(args, rank, world, local)


if __name__ == "__main__":
    main()
