#!/usr/bin/env python
"""Throughput of the fused effective-field + stochastic LLG hot path.

Workload: 128^3 simple-cubic lattice (2,097,152 spins), periodic; exchange
shells J1=1.0, J2=-0.2, J3=0.05 meV, bulk DMI D=0.2 meV (first shell),
K=0.05 meV along z, mu_s=2; random initial spins (seed 1); stochastic Heun at
T=10 K with the Philox thermal field (seed 1), alpha=0.1, dt=1e-3 ps; FP32.
One benchmark step = one run of the workload's 10,000 LLG time steps (each
time step = predictor + corrector kernel).  The spin state (32 MB) is smaller
than L2, so L2 is flushed (256 MB write) before every timed step, outside the
step's CUDA-event bracket.

Multi-GPU: replicas only (independent replicas, one per rank, different noise
streams); the value is the spin-updates of all ranks over the slowest rank.

`--impl reference` times the FP64 CPU oracle on the host cores instead (one
LLG time step of the same lattice per benchmark step).
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "LLG spin-updates/s (% of HBM roofline); time to max-torque<1e-6 vs plain"
UNIT = "spin-updates/s"
LLG_STEPS = 10000
# algorithmic bytes per spin and launch (FP32 records of 16 B):
#   predictor: read n, write predictor state and folded corrector term (3 x 16)
#   corrector: read predictor state and folded term, write n          (3 x 16)
# algorithmic bytes per spin and launch of the two LLG kernel classes (FP32
# records): Heun reads n, writes np and q; reads np and q, writes n.  Depondt
# and SIB correctors also read n.  RK4: stage 0 (counted as the predictor)
# reads n, writes acc and the stage state; stages 1-2 read the stage state,
# n and acc and write acc and the next state; stage 3 reads the stage state,
# n and acc and writes n (the three counted as the corrector).
SOLVER_BYTES = {"heun": {"llg_predictor": 48, "llg_corrector": 48},
                "depondt": {"llg_predictor": 48, "llg_corrector": 64},
                "sib": {"llg_predictor": 48, "llg_corrector": 64},
                "rk4": {"llg_predictor": 48, "llg_corrector": (80 + 80 + 64) / 3}}
# the method's own algorithmic bytes per spin and time step (FP32 records),
# which the roofline fraction is charged with: a two-stage step reads n and
# writes the predictor n^p (32 B), then reads n and n^p and writes n' (48 B);
# the field and the thermal noise are recomputed, not stored.  (The kernels
# above move 96 B for Heun because they store the folded corrector term q in
# place of recomputing the stencil on n and the noise.)  RK4 has no two-stage
# figure and is charged with the design's bytes.
METHOD_STEP_BYTES = {"heun": 80, "depondt": 80, "sib": 80}
# the lean FP32 Heun passes (whole 32 x 8 tiles) pack q into the predicted
# record's pad word plus 8 bytes: read n, write n^p|q_x and q_yz (40 B); read
# those, write n (40 B)
LEAN_HEUN_BYTES = {"llg_predictor": 40, "llg_corrector": 40}
CORRECTOR_LAUNCHES = {"heun": 1, "depondt": 1, "sib": 1, "rk4": 3}
KERNEL_SOURCES = ["paper_1901_11350_gb300/csrc/field_llg.cu", "paper_1901_11350_gb300/csrc/cubic.cu",
                  "paper_1901_11350_gb300/csrc/cubic_lean.cu",
                  "paper_1901_11350_gb300/csrc/common.cuh"]
# GNEB: bytes per spin and iteration of the method's three passes with FP32
# records (read n, write g 32; read the three images and g 64; read n, g, v
# and write n, v 80, plus the per-image reductions' re-reads, about 190) and
# of this design's four passes (move 80, field 48, tangent 80, force 96)
GNEB_METHOD_BYTES = 190
GNEB_DESIGN_BYTES = 304


def rank_info():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")),
            int(os.environ.get("WORLD_SIZE", "1")))


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def source_hash():
    h = hashlib.sha256()
    for p in KERNEL_SOURCES:
        fp = os.path.join(ROOT, p)
        if os.path.exists(fp):
            h.update(open(fp, "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel sources."""
    fp = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        d = json.load(open(fp))
    except (OSError, ValueError):
        return None
    e = d.get(kernel)
    if not e or e.get("source_sha") != source_hash():
        return None
    return e.get("dram_bytes_per_launch")


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.out = tempfile.NamedTemporaryFile(mode="w+", suffix=".csv", delete=False)

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.out, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        self.out.flush()
        rows = []
        try:
            with open(self.out.name) as f:
                for line in f:
                    p = [x.strip() for x in line.split(",")]
                    if len(p) >= 9:
                        rows.append(p)
        finally:
            os.unlink(self.out.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no nvidia-smi samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


def max_over_ranks(value, device="cpu"):
    """Largest `value` over all ranks of the default process group (the
    value itself without one)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.item()


def whole_job_rate(world, units_per_rank, slowest_ms):
    """Units of all replicas over the slowest rank's time (weak scaling)."""
    return world * units_per_rank / (slowest_ms / 1e3)


def cpu_baseline(cfg, seconds=12.0, max_steps=64):
    """The FP64 oracle, as it stands, on the host cores: full lattice, a
    bounded number of LLG time steps."""
    import oracle
    from paper_1901_11350_gb300 import inputs as I
    g, h, r = cfg["geometry"], cfg["hamiltonian"], cfg["run"]
    o = oracle.System(g, h)
    n = I.random_spins(o.N, cfg["spin_seed"])
    kw = dict(solver=r["solver"], dt=r["dt"], alpha=r["alpha"], T=r["T"], seed=r["seed"])
    t0 = time.perf_counter()
    n = o.llg(n, 1, **kw)
    t1 = time.perf_counter() - t0
    steps = max(1, min(max_steps, int(seconds / max(t1, 1e-6))))
    t0 = time.perf_counter()
    n = o.llg(n, steps, step0=1, **kw)
    el = time.perf_counter() - t0
    return {"value": o.N * steps / el, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
            "sample": "%d FP64 %s steps (T = %g K) of the full %s lattice (%d spins), %.1f s" % (
                steps, r["solver"], r["T"], "x".join(str(x) for x in g["n_cells"]), o.N, el)}


def oracle_rate(step, units_per_call, seconds=10.0, max_calls=1000):
    """Units per second of `step()` (one oracle call doing units_per_call
    units of work), timed for about `seconds` on the host cores."""
    t0 = time.perf_counter()
    step()
    t1 = time.perf_counter() - t0
    calls = max(1, min(max_calls, int(seconds / max(t1, 1e-6))))
    t0 = time.perf_counter()
    for _ in range(calls):
        step()
    el = time.perf_counter() - t0
    return units_per_call * calls / el, calls, el


def run_reference(args):
    rank, _, world = rank_info()
    if rank != 0:
        return 0
    import oracle
    from paper_1901_11350_gb300 import inputs as I
    cfg = I.cfg_sc_128()
    g, h, r = cfg["geometry"], cfg["hamiltonian"], cfg["run"]
    o = oracle.System(g, h)
    n = I.random_spins(o.N, cfg["spin_seed"])
    kw = dict(solver=r["solver"], dt=r["dt"], alpha=r["alpha"], T=r["T"], seed=r["seed"])
    for k in range(args.warmup):
        n = o.llg(n, 1, step0=k, **kw)
    times = []
    for k in range(args.steps):
        t0 = time.perf_counter()
        n = o.llg(n, 1, step0=args.warmup + k, **kw)
        times.append(time.perf_counter() - t0)
    el = sum(times)
    value = o.N * args.steps / el
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": cfg["name"], "spins": o.N, "llg_steps_per_bench_step": 1,
                      "solver": "heun", "T_K": r["T"], "l2": "n/a (host)"},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
                            "sample": "1 FP64 stochastic-Heun step of the full 128x128x128 lattice per step"},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))
    return 0


def run_gpu(args):
    import torch
    import torch.distributed as dist
    from paper_1901_11350_gb300 import binding as Bd
    from paper_1901_11350_gb300 import build
    from paper_1901_11350_gb300 import inputs as I

    rank, local, world = rank_info()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    build.build()
    cfg = I.cfg_sc_128(args.side)
    g, h, r = cfg["geometry"], cfg["hamiltonian"], cfg["run"]
    S = args.llg_steps
    ctx = Bd.Context(g, h, "f32")
    if args.generic:
        ctx.set_option("generic_stencil", 1)
    ctx.set_option("cubic_lean", args.cubic_lean)
    if args.cubic_rows:
        rw = [int(x) for x in args.cubic_rows.split(",")]
        ctx.set_option("cubic_rows", rw[0])
        if len(rw) > 1:
            ctx.set_option("cubic_rows_corr", rw[1])
    if args.zc:
        zc = [int(x) for x in args.zc.split(",")]
        ctx.set_option("planes_per_cta", zc[0])
        if len(zc) > 1:
            ctx.set_option("planes_per_cta_corr", zc[1])
    N = ctx.N
    host0 = torch.zeros((N, 4), dtype=torch.float32)
    host0[:, :3] = torch.from_numpy(I.random_spins(N, cfg["spin_seed"])).float()
    host0 = host0.pin_memory()
    n = host0.to("cuda")
    kw = dict(solver=args.solver, dt=r["dt"], alpha=r["alpha"],
              T=r["T"] if args.temperature is None else args.temperature, seed=r["seed"], replica=rank)
    lean = args.solver == "heun" and bool(ctx.get_option("cubic_lean"))
    bps = LEAN_HEUN_BYTES if lean else SOLVER_BYTES[args.solver]
    bytes_per_step = bps["llg_predictor"] + CORRECTOR_LAUNCHES[args.solver] * bps["llg_corrector"]
    if not args.zc and not args.generic and not args.cubic_rows:
        ctx.autotune(n)  # tile height and planes per CTA, chosen by timing before the timed region
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    st = torch.cuda.current_stream()
    step = 0
    for k in range(args.warmup):
        flush.fill_(k & 0xFF)
        ctx.llg_step(n, S, step0=step, **kw)
        step += S
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        for k in range(args.steps):
            flush.fill_((k + 1) & 0xFF)
            ev[k][0].record(st)
            ctx.llg_step(n, S, step0=step, **kw)
            ev[k][1].record(st)
            step += S
        torch.cuda.synchronize()
    el_ms = sum(a.elapsed_time(b) for a, b in ev)
    el_ms = max_over_ranks(el_ms, "cuda")
    # per-kernel durations: a separate pass with CUDA events around every
    # launch (the events keep consecutive launches from overlapping, so they
    # stay out of the timed region above)
    prof_steps = min(args.steps, 2)
    ctx.profile(True)
    for k in range(prof_steps):
        flush.fill_((k + 7) & 0xFF)
        ctx.llg_step(n, S, step0=step, **kw)
        step += S
    torch.cuda.synchronize()
    ctx.profile(False)
    kern = {}
    for name in ("llg_predictor", "llg_corrector"):
        ms, cnt = ctx.profile_read(name)
        kern[name] = (ms, cnt)
    if world > 1:
        dist.barrier()
    value = whole_job_rate(world, N * S * args.steps, el_ms)
    finite = bool(torch.isfinite(n).all().item())

    # end to end through the public API: pinned host state in, state out
    host_out = torch.empty_like(host0).pin_memory()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    e0.record(st)
    for k in range(args.steps):
        nd = host0.to("cuda", non_blocking=True)
        ctx.llg_step(nd, S, step0=step, **kw)
        host_out.copy_(nd, non_blocking=True)
        step += S
    e1.record(st)
    torch.cuda.synchronize()
    e2e_value = whole_job_rate(world, N * S * args.steps, max_over_ranks(e0.elapsed_time(e1), "cuda"))

    peaks, peak_kind = measured_peaks()
    # the roofline unit is one LLG time step (its predictor and corrector
    # launches together), timed by the CUDA events around the timed region:
    # per-launch events would serialise the two passes' overlap
    step_s = el_ms / 1e3 / (S * args.steps) * world
    method_bytes = METHOD_STEP_BYTES.get(args.solver, bytes_per_step)
    achieved = method_bytes * N / step_s / 1e9
    tr = [ncu_traffic(k) for k in ("llg_predictor", "llg_corrector")] if args.solver == "heun" and not args.generic \
        else [None]
    tot_ms = sum(v[0] for v in kern.values())
    roof = {"bound": "hbm", "kernel": "llg_step (predictor + corrector launch of one time step)",
            "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"],
            "traffic": None if None in tr else sum(tr), "peak_source": peak_kind,
            "algorithmic_bytes_per_spin_step": method_bytes,
            "algorithmic_bytes_per_step": method_bytes * N, "us_per_step": step_s * 1e6,
            "timing": "CUDA events around the timed region, %d LLG steps" % (S * args.steps),
            "design_bytes_per_spin_step": bytes_per_step,
            "design_frac": bytes_per_step * N / step_s / 1e9 / peaks["hbm_gbs"],
            "kernel_share": {k: {"share": v[0] / tot_ms if tot_ms else None, "launches": v[1],
                                 "avg_launch_us": 1e3 * v[0] / max(v[1], 1)} for k, v in kern.items()},
            "kernel_share_timing": "serialised: CUDA events around every launch, %d profiled bench steps after "
                                   "the timed region (shares, not the kernels' speed inside the step)" % prof_steps}
    clocks = clk.summary()
    if world > 1:
        dist.destroy_process_group()
    if rank != 0:
        return 0
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": el_ms / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": cfg["name"], "spins": N, "llg_steps_per_bench_step": S, "solver": args.solver,
                      "kernel_path": "generic" if args.generic else (
                          "cubic27" if ctx.get_option("has_cubic_path") else "generic"),
                      "planes_per_cta": ctx.get_option("planes_per_cta"),
                      "planes_per_cta_corr": ctx.get_option("planes_per_cta_corr"),
                      "columns_per_thread": [ctx.get_option("cubic_rows"), ctx.get_option("cubic_rows_corr")],
                      "lean_heun_passes": lean,
                      "T_K": r["T"], "thermal_rng": "philox4x32-10", "l2": "flushed (256 MB write) before each step",
                      "parallelism": "replicas" if world > 1 else "single"},
           "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": N * 16, "d2h_bytes_per_step": N * 16},
           "gpu_launches": ((1 + CORRECTOR_LAUNCHES[args.solver]) * S + 1) * args.steps, "roofline": roof, "clocks": clocks,
           "finite": finite}
    if not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(dict(cfg, run=dict(r, solver=args.solver)))
    if world == 1 and not args.no_relax:
        # the metric's second half: time to converge relaxations, against the
        # plain FP64 method on the same GPU
        out["relaxation"] = {"gneb": gneb_result(args, compact=True),
                             "warm_start": warmstart_result(args, args.relax_systems, compact=True)}
    print(json.dumps(out))
    return 0


def run_gneb(args):
    print(json.dumps(gneb_result(args)))
    return 0


def gneb_result(args, compact=False):
    """Batched GNEB workload (48 skyrmion-collapse chains): device seconds to
    max force < 1e-5 meV/rad, batched FP32 against the plain FP64 loop over
    chains through the single-chain entry point, on the same GPU."""
    import numpy as np
    import torch
    from paper_1901_11350_gb300 import build
    from paper_1901_11350_gb300 import gneb_batch as G

    torch.cuda.set_device(torch.cuda.current_device())
    build.build()
    t0 = time.perf_counter()
    chains = G.prepare(n_chains=args.chains, seed=4, precision="f32")
    prep_s = time.perf_counter() - t0
    kw = dict(dt=0.2, k_spring=1.0, tol=1e-5, chunk=args.gneb_chunk)
    tune = None
    if args.gneb_persistent < 0:
        # launch mode of the batched iterations chosen by the autotuner on
        # the full batch (one launch per pass, or the persistent kernel)
        from paper_1901_11350_gb300 import binding as Bd
        offs, Ms, off = [], [], 0
        for ch in chains:
            offs.append(off)
            Ms.append(ch.M)
            off += ch.M * ch.N
        x = torch.cat([ch.ctx.spins(ch.chain0).reshape(-1, 4) for ch in chains])
        choice, t0_ms, t1_ms = Bd.gneb_batch_autotune([ch.ctx for ch in chains], x, torch.zeros_like(x), offs, Ms,
                                                      n_trial=16, k_spring=kw["k_spring"], dt=kw["dt"])
        tune = {"per_pass_ms": t0_ms, "persistent_ms": t1_ms, "trial_iterations": 16}
        del x
        pk = dict(persistent=bool(choice))
    else:
        pk = dict(persistent=bool(args.gneb_persistent))
    G.run_batched(chains[:2], **dict(kw, chunk=10, tol=0.0, max_iter=10), **pk)  # warm-up (graph, tables)
    state, batch_s = G.run_batched(chains, **kw, **pk)
    if args.gneb_no_reference:  # profiling aid: the batched run alone
        return {"metric": "GNEB device seconds to max force < 1e-5 meV/rad, all chains", "value": batch_s,
                "unit": "s", "higher_is_better": False, "reference": None, "persistent": pk["persistent"],
                "iterations": {"max": max(state[k]["iters"] for k in state)}}
    ref, ref_s = G.run_per_chain(chains, precision="f64", **kw)
    from paper_1901_11350_gb300 import binding as Bd
    # barrier heights in FP64: image energies of the converged FP32 chains
    # re-evaluated by an FP64 context, against the FP64 loop's own chains
    bar32, bar64 = [], []
    for k, ch in enumerate(chains):
        c64 = Bd.Context(ch.draw["geometry"], ch.draw["hamiltonian"], "f64")
        x = state[k]["x"].reshape(ch.M, ch.N, 4).double()
        E = np.array([c64.energy(x[m].contiguous())[0].item() for m in range(ch.M)])
        bar32.append(E.max() - E[0])
        bar64.append(ref[k]["E"].max() - ref[k]["E"][0])
        c64.close()
    bar32, bar64 = np.array(bar32), np.array(bar64)
    spins = sum(c.M * c.N for c in chains)
    out = {"metric": "GNEB device seconds to max force < 1e-5 meV/rad, all chains", "value": batch_s, "unit": "s",
           "higher_is_better": False, "dtype": "f32 forces, f64 energies", "data": "synthetic",
           "config": {"workload": "gneb%d_skyrmion_collapse" % len(chains), "chains": len(chains),
                      "launch": "persistent" if pk["persistent"] else "per pass (CUDA graph)",
                      "launch_autotune": tune,
                      "spins_all_images": spins, "images": [c.M for c in chains],
                      "sides": [c.draw["L"] for c in chains], "redraws": sum(c.draw["attempt"] for c in chains),
                      "dt": kw["dt"], "k_spring": kw["k_spring"], "check_every": kw["chunk"]},
           "iterations": {"max": max(state[k]["iters"] for k in state), "min": min(state[k]["iters"] for k in state)},
           "all_converged": bool(all(state[k]["fmax"] < kw["tol"] for k in state)),
           "reference": {"kind": "plain FP64 loop over chains (sp_gneb_step), same GPU", "value": ref_s, "unit": "s",
                         "all_converged": bool(all(ref[k]["fmax"] < kw["tol"] for k in ref))},
           "speedup_vs_reference": ref_s / batch_s,
           "barrier_meV": {"min": float(bar64.min()), "max": float(bar64.max())},
           "barrier_rel_diff_f32_batch_vs_f64": {"max": float(np.max(np.abs(bar32 - bar64) / np.abs(bar64))),
                                                 "median": float(np.median(np.abs(bar32 - bar64) / np.abs(bar64)))},
           "setup_s": prep_s}
    # per-iteration roofline over the full batch (GNEB_METHOD_BYTES; the
    # design's passes move GNEB_DESIGN_BYTES: move 80 (read F, v, x; write v,
    # x), field 48 (x, next image; write Pg), tangent 80 (three images, Pg;
    # write tau), force 96 (tau, Pg, F, v; write v, F))
    import torch
    offs, Ms, ctxs, off = [], [], [], 0
    for ch in chains:
        offs.append(off)
        Ms.append(ch.M)
        ctxs.append(ch.ctx)
        off += ch.M * ch.N
    x = torch.cat([ch.ctx.spins(ch.chain0).reshape(-1, 4) for ch in chains])
    v = torch.zeros_like(x)
    Bd.gneb_batch_step(ctxs, x, v, offs, Ms, n_iter=16, k_spring=1.0, climbing=True, dt=kw["dt"])
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(st)
    Bd.gneb_batch_step(ctxs, x, v, offs, Ms, n_iter=64, k_spring=1.0, climbing=True, dt=kw["dt"])
    e1.record(st)
    torch.cuda.synchronize()
    it_s = e0.elapsed_time(e1) / 64 / 1e3
    peaks, pk = measured_peaks()
    gbs = GNEB_METHOD_BYTES * off / it_s / 1e9
    out["roofline"] = {"bound": "hbm", "kernel": "one GNEB iteration of all chains (move, field, tangent, force)",
                       "achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": gbs / peaks["hbm_gbs"],
                       "traffic": None, "peak_source": pk, "algorithmic_bytes_per_spin_iteration": GNEB_METHOD_BYTES,
                       "design_bytes_per_spin_iteration": GNEB_DESIGN_BYTES,
                       "design_frac": GNEB_DESIGN_BYTES * off / it_s / 1e9 / peaks["hbm_gbs"],
                       "ms_per_iteration": it_s * 1e3}
    # the oracle on the largest chain, scaled to the spin-iterations this run needed
    import oracle
    big = max(range(len(chains)), key=lambda k: chains[k].M * chains[k].N)
    ch = chains[big]
    o = oracle.System(ch.draw["geometry"], ch.draw["hamiltonian"])
    ost = {"x": ch.chain0, "v": None}

    def oiter():
        ost["x"], ost["v"], _, _, _ = o.gneb(ost["x"], ost["v"], n_iter=1, k_spring=1.0, climbing=True, dt=kw["dt"])

    rate, calls, el = oracle_rate(oiter, ch.M * ch.N, seconds=6.0 if compact else 10.0)
    work = sum(state[k]["iters"] * chains[k].M * chains[k].N for k in state)
    out["cpu_baseline"] = {"value": work / rate, "unit": "s", "cores": oracle.threads(), "kind": "oracle",
                           "sample": "%d FP64 GNEB iterations of the largest chain (%d images x %d spins) in %.1f s; "
                                     "%.3g spin-iterations/s, scaled to the %.3g spin-iterations of the batched run"
                                     % (calls, ch.M, ch.N, el, rate, work)}
    if compact:
        for k in ("images", "sides"):
            out["config"].pop(k)
    return out


def run_hex_dipole(args):
    """512x512 hexagonal monolayer with the FFT dipole term, FP32 Depondt
    (alpha=0.5, dt=1e-3 ps), 2000 steps: spin-updates/s and the split
    between the dipole pipeline and the LLG kernels."""
    import torch
    from paper_1901_11350_gb300 import binding as Bd
    from paper_1901_11350_gb300 import build
    from paper_1901_11350_gb300 import inputs as I

    torch.cuda.set_device(0)
    build.build()
    cfg = I.cfg_hex_dipole()
    g, h, r = cfg["geometry"], cfg["hamiltonian"], cfg["run"]
    ctx = Bd.Context(g, h, "f32")
    N = ctx.N
    n = ctx.spins(I.random_spins(N, cfg["spin_seed"]))
    kw = dict(solver=r["solver"], dt=r["dt"], alpha=r["alpha"])
    S = args.llg_steps if args.llg_steps != LLG_STEPS else r["n_steps"]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    for k in range(args.warmup):
        flush.fill_(k)
        ctx.llg_step(n, 50, **kw)
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    tot = 0.0
    for k in range(args.steps):
        flush.fill_(k + 1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        ctx.llg_step(n, S, **kw)
        e1.record(st)
        torch.cuda.synchronize()
        tot += e0.elapsed_time(e1)
    # per-kernel split from a separate profiled pass (events around launches)
    ctx.profile(True)
    ctx.llg_step(n, S, **kw)
    torch.cuda.synchronize()
    ctx.profile(False)
    kern = {k: ctx.profile_read(k) for k in ("llg_predictor", "llg_corrector", "dipole")}
    dip_ms, dip_n = kern["dipole"]
    # algorithmic bytes of one dipole evaluation (FP32): row spectra written
    # (3 x n1 x (P0/2+1) complex), read+written by the column pass, kernel
    # tensor read (6 x P1 x (P0/2+1) real), read by the inverse rows, moments
    # read and field written (16 B per spin each)
    n0, n1 = g["n_cells"][0], g["n_cells"][1]
    P0, P1 = 2 * n0, 2 * n1
    half = P0 // 2 + 1
    spec = 3 * n1 * half * 8
    dip_bytes = spec + 2 * spec + 6 * P1 * half * 4 + spec + 2 * 16 * N
    peaks, _ = measured_peaks()
    out = {"metric": "LLG spin-updates/s, dipolar monolayer", "value": N * S * args.steps / (tot / 1e3),
           "unit": UNIT, "higher_is_better": True, "dtype": "f32", "data": "synthetic", "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": tot / args.steps,
           "config": {"workload": cfg["name"], "spins": N, "llg_steps_per_bench_step": S, "solver": r["solver"],
                      "fft_grid": [P0, P1]},
           "kernels": {k: {"total_ms": v[0], "launches": v[1]} for k, v in kern.items()},
           "dipole": {"us_per_evaluation": 1e3 * dip_ms / max(dip_n, 1), "algorithmic_bytes": dip_bytes,
                      "achieved_GBs": dip_bytes / (dip_ms / max(dip_n, 1) / 1e3) / 1e9, "peak_GBs": peaks["hbm_gbs"]},
           "finite": bool(torch.isfinite(n).all().item())}
    dip_gbs = dip_bytes / (dip_ms / max(dip_n, 1) / 1e3) / 1e9
    out["roofline"] = {"bound": "hbm", "kernel": "dipole_field (row, column x kernel, inverse-row FFT passes)",
                       "achieved": dip_gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                       "frac": dip_gbs / peaks["hbm_gbs"], "traffic": None,
                       "algorithmic_bytes_per_launch": dip_bytes,
                       "note": "per dipole evaluation (the largest share of a step); its 46 MB working set stays "
                               "in L2, so the passes are latency-bound rather than DRAM-bound"}
    if not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(cfg, seconds=10.0, max_steps=50)
    print(json.dumps(out))
    return 0


def run_mc(args):
    """Metropolis Monte Carlo of the simple-cubic ferromagnet (J = 1 meV,
    periodic, B = 0): all temperatures of a grid as replicas of one launch;
    per temperature args.mc_thermal sweeps with the adaptive cone (target
    acceptance 0.5) and args.mc_samples sampled sweeps with the cone fixed.
    Reports spin-updates/s and the critical temperature from the Binder
    cumulant crossings of the sizes and the susceptibility peak."""
    import numpy as np
    import torch
    from paper_1901_11350_gb300 import binding as Bd
    from paper_1901_11350_gb300 import build
    from paper_1901_11350_gb300 import inputs as I

    torch.cuda.set_device(0)
    build.build()
    sizes = [int(v) for v in args.mc_sizes.split(",")]
    T = np.round(np.arange(args.mc_tmin, args.mc_tmax + 1e-9, args.mc_dt), 6)
    R = len(T)
    kB = 0.08617333262
    res, tot_updates, tot_s = {}, 0.0, 0.0
    st_cuda = torch.cuda.current_stream()
    for L in sizes:
        ctx = Bd.Context(I.simple_cubic(L, L, L, periodic=(True, True, True), mu_s=2.0), dict(J=[1.0]), "f32")
        ctx.set_option("mc_resident", args.mc_resident)
        N = ctx.N
        x = ctx.spins(I.ferromagnet(N))[None].repeat(R, 1, 1).contiguous()
        cone = torch.full((R,), 0.5, dtype=torch.float64, device="cuda")
        stats = torch.zeros((R, 8), dtype=torch.float64, device="cuda")
        ctx.mc_sweeps(x, T, args.warmup, seed=L, target_accept=0.5, sample=False, cone=cone, stats=stats)
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        torch.cuda.synchronize()
        e0.record(st_cuda)
        ctx.mc_sweeps(x, T, args.mc_thermal, seed=L, sweep0=args.warmup, target_accept=0.5, sample=False, cone=cone,
                      stats=stats)
        e1.record(st_cuda)
        stats.zero_()
        ctx.mc_sweeps(x, T, args.mc_samples, seed=L, sweep0=args.warmup + args.mc_thermal, target_accept=0.0,
                      sample=True, cone=cone, stats=stats)
        e2.record(st_cuda)
        torch.cuda.synchronize()
        secs = e0.elapsed_time(e2) / 1e3
        sweeps = args.mc_thermal + args.mc_samples
        tot_updates += float(sweeps) * N * R
        tot_s += secs
        s = stats.cpu().numpy()
        n = s[:, 5]
        m, m2, m4, E, E2 = (s[:, k] / n for k in range(5))
        res[L] = dict(N=N, colours=ctx.mc_colours(), resident=ctx.get_option("mc_resident") == 1 and N <= 2048,
                      seconds=secs, thermal_s=e0.elapsed_time(e1) / 1e3, m=m, m2=m2, m4=m4,
                      U4=1 - m4 / (3 * m2 ** 2), chi=N * (m2 - m ** 2) / (kB * T), cv=(E2 - E ** 2) / (kB * T ** 2) / N,
                      accept=s[:, 6] / s[:, 7], cone=cone.cpu().numpy())
    # Binder-cumulant crossings of consecutive sizes (linear interpolation)
    cross = []
    for a, b in zip(sizes[:-1], sizes[1:]):
        d = res[a]["U4"] - res[b]["U4"]
        for k in range(R - 1):
            if d[k] < 0 <= d[k + 1] or d[k] > 0 >= d[k + 1]:
                cross.append(float(T[k] + (T[k + 1] - T[k]) * d[k] / (d[k] - d[k + 1])))
                break
    Lmax = max(sizes)
    chi = res[Lmax]["chi"]
    k = int(np.argmax(chi))
    tpk = float(T[k])
    if 0 < k < R - 1:  # parabola through the peak and its neighbours
        y0, y1, y2 = chi[k - 1], chi[k], chi[k + 1]
        den = y0 - 2 * y1 + y2
        if den != 0:
            tpk = float(T[k] + 0.5 * (T[1] - T[0]) * (y0 - y2) / den)
    out = {"metric": "Metropolis spin-updates/s, simple-cubic ferromagnet (Tc validation)",
           "value": tot_updates / tot_s, "unit": "spin-updates/s", "n_gpus": 1, "higher_is_better": True,
           "dtype": "f32 field and trials, f64 observables", "data": "synthetic",
           "config": {"workload": "mc_sc_ferromagnet_tc", "sizes": sizes, "temperatures_K": [float(t) for t in T],
                      "thermal_sweeps": args.mc_thermal, "sample_sweeps": args.mc_samples, "J_meV": 1.0,
                      "target_accept": 0.5, "colours": {str(L): r["colours"] for L, r in res.items()},
                      "l2": "inputs resident in L2 (at most 29 x 30^3 x 16 B = 12.5 MB): a sweep's cost is "
                            "instruction issue, not DRAM"},
           "tc_K": {"binder_crossings": cross, "binder_mean": float(np.mean(cross)) if cross else None,
                    "chi_peak_L%d" % Lmax: tpk, "expected_high_T_series": 16.71, "paper_mc": 16.60},
           "per_size": {str(L): {"seconds": r["seconds"], "spins": r["N"],
                                 "kernel": "k_mc_resident" if r["resident"] else "k_mc_colour",
                                 "us_per_sweep_adaptive": 1e6 * r["thermal_s"] / max(args.mc_thermal, 1),
                                 "us_per_sweep_sampled": 1e6 * (r["seconds"] - r["thermal_s"]) / max(args.mc_samples, 1),
                                 "m": [round(float(v), 5) for v in r["m"]], "U4": [round(float(v), 5) for v in r["U4"]],
                                 "chi": [round(float(v), 3) for v in r["chi"]], "cv": [round(float(v), 5) for v in r["cv"]],
                                 "accept": [round(float(v), 3) for v in r["accept"]]}
                        for L, r in res.items()}}
    peaks, kind = measured_peaks()
    # algorithmic bytes of a trial: the spin's record read and written (the
    # neighbours' records come from L2 within a colour sweep)
    gbs = 32 * out["value"] / 1e9
    out["roofline"] = {"bound": "hbm", "kernel": "k_mc_colour", "achieved": gbs, "peak": peaks["hbm_gbs"],
                       "unit": "GB/s", "frac": gbs / peaks["hbm_gbs"], "traffic": None, "peak_source": kind,
                       "algorithmic_bytes_per_trial": 32,
                       "note": "bound by instruction issue, not DRAM: the neighbour records come from L2 or "
                               "shared memory; ncu of the resident kernel shows the issue slots of its SMs 80% busy"}
    if not args.no_cpu_baseline:
        import oracle
        Lm = max(sizes)
        o = oracle.System(I.simple_cubic(Lm, Lm, Lm, periodic=(True, True, True), mu_s=2.0), dict(J=[1.0]))
        x0 = I.ferromagnet(o.N)[None]
        state = {"x": x0}

        def sweep():
            state["x"], _, _ = o.mc(state["x"], [16.5], 1, seed=1, target_accept=0.5, sample=True)

        v, calls, el = oracle_rate(sweep, o.N)
        out["cpu_baseline"] = {"value": v, "unit": "spin-updates/s", "cores": oracle.threads(), "kind": "oracle",
                               "sample": "%d Metropolis sweeps of one %d^3 replica at 16.5 K, %.1f s" % (calls, Lm, el)}
    print(json.dumps(out))
    return 0


def run_sllg(args):
    """Stochastic LLG sampling of the simple-cubic ferromagnet (J = 1 meV,
    periodic, B = 0; Appendix "Stochastic LLG"): every temperature of the grid
    is a replica of one batch (sp_llg_step_replicas), stochastic Heun with
    alpha = args.sllg_alpha and dt = args.sllg_dt; args.sllg_thermal steps,
    then args.sllg_samples steps with the observables accumulated after
    every args.sllg_every steps (sp_sample).  Reports spin-updates/s and the
    critical temperature from the Binder-cumulant crossings of the sizes and
    the susceptibility peak of the largest."""
    import numpy as np
    import torch
    from paper_1901_11350_gb300 import binding as Bd
    from paper_1901_11350_gb300 import build
    from paper_1901_11350_gb300 import inputs as I

    torch.cuda.set_device(0)
    build.build()
    sizes = [int(v) for v in args.mc_sizes.split(",")]
    T = np.round(np.arange(args.mc_tmin, args.mc_tmax + 1e-9, args.mc_dt), 6)
    R = len(T)
    kB = 0.08617333262
    every = args.sllg_every
    n_samp = args.sllg_samples // every
    kw = dict(solver="heun", dt=args.sllg_dt, alpha=args.sllg_alpha)
    res, tot_updates, tot_s = {}, 0.0, 0.0
    st_cuda = torch.cuda.current_stream()
    for L in sizes:
        ctx = Bd.Context(I.simple_cubic(L, L, L, periodic=(True, True, True), mu_s=2.0), dict(J=[1.0]), "f32")
        if args.generic:
            ctx.set_option("generic_stencil", 1)
        if args.zc:
            zc = [int(v) for v in args.zc.split(",")]
            ctx.set_option("planes_per_cta", zc[0])
            if len(zc) > 1:
                ctx.set_option("planes_per_cta_corr", zc[1])
        N = ctx.N
        x = ctx.spins(I.ferromagnet(N))[None].repeat(R, 1, 1).contiguous()
        stats = torch.zeros((R, 8), dtype=torch.float64, device="cuda")
        step = 0
        ctx.llg_step_replicas(x, T, max(args.warmup, 1), seed=L, step0=step, **kw)
        step += max(args.warmup, 1)
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        torch.cuda.synchronize()
        e0.record(st_cuda)
        ctx.llg_step_replicas(x, T, args.sllg_thermal, seed=L, step0=step, **kw)
        step += args.sllg_thermal
        e1.record(st_cuda)
        for k in range(n_samp):
            ctx.llg_step_replicas(x, T, every, seed=L, step0=step, **kw)
            step += every
            ctx.sample(x, stats)
        e2.record(st_cuda)
        torch.cuda.synchronize()
        secs = e0.elapsed_time(e2) / 1e3
        steps = args.sllg_thermal + n_samp * every
        tot_updates += float(steps) * N * R
        tot_s += secs
        s = stats.cpu().numpy()
        n = s[:, 5]
        m, m2, m4, E, E2 = (s[:, k] / n for k in range(5))
        res[L] = dict(N=N, seconds=secs, thermal_s=e0.elapsed_time(e1) / 1e3, m=m, m2=m2, m4=m4,
                      U4=1 - m4 / (3 * m2 ** 2), chi=N * (m2 - m ** 2) / (kB * T), cv=(E2 - E ** 2) / (kB * T ** 2) / N,
                      finite=bool(torch.isfinite(x).all().item()))
    cross = []
    for a, b in zip(sizes[:-1], sizes[1:]):
        d = res[a]["U4"] - res[b]["U4"]
        for k in range(R - 1):
            if d[k] < 0 <= d[k + 1] or d[k] > 0 >= d[k + 1]:
                cross.append(float(T[k] + (T[k + 1] - T[k]) * d[k] / (d[k] - d[k + 1])))
                break
    Lmax = max(sizes)
    chi = res[Lmax]["chi"]
    k = int(np.argmax(chi))
    tpk = float(T[k])
    if 0 < k < R - 1:
        y0, y1, y2 = chi[k - 1], chi[k], chi[k + 1]
        den = y0 - 2 * y1 + y2
        if den != 0:
            tpk = float(T[k] + 0.5 * (T[1] - T[0]) * (y0 - y2) / den)
    out = {"metric": "stochastic-LLG spin-updates/s, simple-cubic ferromagnet (Tc validation)",
           "value": tot_updates / tot_s, "unit": "spin-updates/s", "n_gpus": 1, "higher_is_better": True,
           "dtype": "f32 field and steps, f64 observables", "data": "synthetic",
           "config": {"workload": "sllg_sc_ferromagnet_tc", "sizes": sizes, "temperatures_K": [float(t) for t in T],
                      "thermal_steps": args.sllg_thermal, "sample_steps": n_samp * every, "sample_every": every,
                      "solver": "heun", "dt_ps": args.sllg_dt, "alpha": args.sllg_alpha, "J_meV": 1.0,
                      "start": "ferromagnet along z", "thermal_rng": "philox4x32-10, one stream per replica"},
           "tc_K": {"binder_crossings": cross, "binder_mean": float(np.mean(cross)) if cross else None,
                    "chi_peak_L%d" % Lmax: tpk, "expected_high_T_series": 16.71, "paper_sllg": 16.92},
           # method kernels: predictor + corrector per step of each size's batch, one observable pass per
           # sample (the graph replays add one step-counter kernel per 32 steps, not counted)
           "gpu_launches": sum(2 * (args.sllg_thermal + n_samp * every) + n_samp for _ in sizes),
           # algorithmic bytes of a spin update: the two LLG passes, 48 B each
           "roofline": {"bound": "hbm", "kernel": "LLG predictor + corrector, all replica batches",
                        "achieved": 96 * tot_updates / tot_s / 1e9, "peak": measured_peaks()[0]["hbm_gbs"],
                        "unit": "GB/s", "frac": 96 * tot_updates / tot_s / 1e9 / measured_peaks()[0]["hbm_gbs"],
                        "traffic": None, "algorithmic_bytes_per_update": 96,
                        "note": "includes the observable passes and the small lattices' launch latency"},
           "per_size": {str(L): {"seconds": r["seconds"], "spins": r["N"], "finite": r["finite"],
                                 "m": [round(float(v), 5) for v in r["m"]], "U4": [round(float(v), 5) for v in r["U4"]],
                                 "chi": [round(float(v), 3) for v in r["chi"]], "cv": [round(float(v), 5) for v in r["cv"]]}
                        for L, r in res.items()}}
    if not args.no_cpu_baseline:
        # one replica of the largest lattice near Tc, stepped by the oracle
        out["cpu_baseline"] = cpu_baseline(dict(
            geometry=I.simple_cubic(Lmax, Lmax, Lmax, periodic=(True, True, True), mu_s=2.0),
            hamiltonian=dict(J=[1.0]), spin_seed=1,
            run=dict(solver="heun", dt=args.sllg_dt, alpha=args.sllg_alpha, T=16.5, seed=Lmax)), seconds=10.0,
            max_steps=200)
    print(json.dumps(out))
    return 0


def run_square32(args):
    """32x32 square lattice, open, J=1, interfacial D=0.3, K=0.1 z, B=1 T z,
    mu_s=2: 1000 deterministic Depondt steps in FP64 (dt=1e-3 ps,
    alpha=0.3) on the default path, with the other paths timed beside it
    (single CTA, 27-point, generic; and FP32); the oracle on the host cores."""
    import numpy as np
    import torch
    from paper_1901_11350_gb300 import binding as Bd
    from paper_1901_11350_gb300 import build
    from paper_1901_11350_gb300 import inputs as I

    torch.cuda.set_device(0)
    build.build()
    cfg = I.cfg_square_32()
    g, h, r = cfg["geometry"], cfg["hamiltonian"], cfg["run"]
    kw = dict(solver=r["solver"], dt=r["dt"], alpha=r["alpha"])
    S = r["n_steps"]
    res = {}
    st = torch.cuda.current_stream()
    # default: FP64 per-spin kernels in small blocks over many SMs; cubic: the
    # 27-point path; f32_*: the FP32 single-CTA path and the FP32 per-spin
    # kernels with one launch per pass
    for path in ("default", "cubic", "f32_single_cta", "f32_generic"):
        c = Bd.Context(g, h, "f32" if path.startswith("f32") else "f64")
        c.set_option("small_path", 1 if path in ("default", "f32_single_cta") else 0)
        if path == "f32_generic":
            c.set_option("generic_stencil", 1)
        n = c.spins(I.random_spins(c.N, cfg["spin_seed"]))
        for _ in range(args.warmup):
            c.llg_step(n, S, **kw)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        torch.cuda.synchronize()
        for k in range(args.steps):
            ev[k][0].record(st)
            c.llg_step(n, S, **kw)
            ev[k][1].record(st)
        torch.cuda.synchronize()
        ms = sum(a.elapsed_time(b) for a, b in ev) / args.steps
        res[path] = ms
    N = 1024
    out = {"metric": "LLG steps/s, 32x32 square lattice, FP64 Depondt (1000 steps per run)",
           "value": S / (res["default"] / 1e3), "unit": "steps/s", "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": res["default"], "higher_is_better": True, "dtype": "f64",
           "data": "synthetic", "config": {"workload": cfg["name"], "spins": N, "llg_steps_per_bench_step": S},
           "paths_ms_per_run": res, "spin_updates_per_s": N * S / (res["default"] / 1e3)}
    if not args.no_cpu_baseline:
        import oracle
        o = oracle.System(g, h)
        x = I.random_spins(N, cfg["spin_seed"])
        t0 = time.perf_counter()
        k = 0
        while time.perf_counter() - t0 < 5.0:
            x = o.llg(x, 50, **kw)
            k += 50
        sec = time.perf_counter() - t0
        out["cpu_baseline"] = {"value": k / sec, "unit": "steps/s", "cores": oracle.threads(), "kind": "oracle",
                               "sample": "%d FP64 Depondt steps of the same lattice, %.1f s" % (k, sec)}
    print(json.dumps(out))
    return 0


def run_hessian(args):
    """Covariant Hessian-vector products on a 2048x2048 hexagonal monolayer
    (FP32, interfacial DMI, anisotropy, field): product rate and HBM
    roofline (algorithmic bytes: read n and v, write H v, 3 x 16 B per
    spin); and the lowest mode of a 128x128 skyrmion state by 64 Lanczos
    steps (FP64)."""
    import numpy as np
    import torch
    from paper_1901_11350_gb300 import binding as Bd
    from paper_1901_11350_gb300 import build
    from paper_1901_11350_gb300 import inputs as I

    torch.cuda.set_device(0)
    build.build()
    h = dict(J=[1.0], dmi_kind="interfacial", D=[0.3], K=[0.05], Khat=[[0, 0, 1]], B=[0, 0, 1.5])
    g = I.hexagonal(2048, 2048, periodic=(True, True), mu_s=2.0)
    c = Bd.Context(g, h, "f32")
    N = c.N
    n = c.spins(I.random_spins(N, 1))
    v = c.spins(I.random_spins(N, 2))
    out = torch.empty_like(n)
    for _ in range(args.warmup):
        c.hessian_apply(n, v, out)
    K = 200
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(st)
    for _ in range(K):
        c.hessian_apply(n, v, out)
    e1.record(st)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / K
    peaks, kind = measured_peaks()
    gbs = 48.0 * N / (ms / 1e3) / 1e9
    # lowest mode of a relaxed skyrmion (Lanczos, FP64)
    g2 = I.hexagonal(128, 128, periodic=(True, True), mu_s=2.0)
    c2 = Bd.Context(g2, h, "f64")
    r = I.site_positions(g2)
    x = c2.spins(I.neel_skyrmion(r, r.mean(axis=0), 6.0, I.SKYRMION_HELICITY))
    c2.minimise(x, c2.spins(np.zeros((c2.N, 3))), dt=0.2, tol=1e-8, max_iter=20000)
    c2.lowest_mode(x, krylov=8)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lam, _ = c2.lowest_mode(x, krylov=64)
    lanczos_s = time.perf_counter() - t0
    out_j = {"metric": "covariant Hessian-vector products/s, 2048x2048 hexagonal monolayer (FP32)",
             "value": 1e3 / ms, "unit": "products/s", "n_gpus": 1, "higher_is_better": True, "dtype": "f32",
             "data": "synthetic", "ms_per_step": ms,
             "config": {"workload": "hessian_hex2048", "spins": N, "products_timed": K,
                        "l2": "working set (201 MB) larger than L2"},
             "roofline": {"bound": "hbm", "achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                          "frac": gbs / peaks["hbm_gbs"], "traffic": None, "peak_source": kind,
                          "algorithmic_bytes_per_launch": 48 * N},
             "lanczos": {"lattice": [128, 128], "state": "relaxed Neel skyrmion", "krylov": 64,
                         "seconds": lanczos_s, "lowest_eigenvalue_meV": lam}}
    if not args.no_cpu_baseline:
        # the oracle's product on a 512x512 crop of the workload (the full
        # lattice's products are independent per spin: the rate carries over)
        import oracle
        gs = I.hexagonal(512, 512, periodic=(True, True), mu_s=2.0)
        o = oracle.System(gs, h)
        ns, vs = I.random_spins(o.N, 1), I.random_spins(o.N, 2)
        rate, calls, el = oracle_rate(lambda: o.hessian_apply(ns, vs), o.N)
        out_j["cpu_baseline"] = {"value": rate / N, "unit": "products/s", "cores": oracle.threads(), "kind": "oracle",
                                 "sample": "%d FP64 products on a 512x512 lattice in %.1f s (%.3g spins/s), "
                                           "scaled to the 2048x2048 lattice" % (calls, el, rate)}
    print(json.dumps(out_j))
    return 0


# (lattice side, channels from the level below or the previous layer,
# upsampled, skip channels, output channels): the distinct convolution shapes
# of the network at 128 x 128
UNET_SHAPES = [(128, 32, 0, 0, 32), (128, 64, 1, 32, 32), (64, 64, 0, 0, 64), (32, 128, 0, 0, 128),
               (32, 256, 1, 128, 128), (16, 256, 0, 0, 256)]


def unet_layer_times(batch, reps=20):
    """Per-shape device times of the 3x3 convolution (forward) and its
    weight gradient for each convolution kernel, batch `batch` (CUDA events
    around `reps` launches after three warm-up launches)."""
    import torch
    from paper_1901_11350_gb300 import unet as UN

    old = UN.conv_kernel()
    g = torch.Generator(device="cuda").manual_seed(0)

    def rnd(*shape):
        return (torch.randn(*shape, device="cuda", generator=g) * 0.5).to(torch.bfloat16)

    def timed(fn):
        for _ in range(3):
            fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    out = []
    for L, c0, up, c1, co in UNET_SHAPES:
        h = L // 2 if up else L
        s0, s1 = rnd(batch, h, h, c0), (rnd(batch, L, L, c1) if c1 else None)
        dz, w = rnd(batch, L, L, co), rnd(co, 9, c0 + c1) * 0.05
        flops = 2.0 * batch * L * L * co * 9 * (c0 + c1)
        row = {"L": L, "cin": c0 + c1, "cout": co, "upsampled": bool(up)}
        for k in ("mma", "tcgen05", "tcgen05_ws", "tcgen05_halo"):
            UN.set_conv_kernel(k)
            ms = timed(lambda: UN.conv3x3_forward(s0, w, None, src1=s1, up0=bool(up)))
            row["forward_" + k] = {"ms": ms, "tflops": flops / ms / 1e9}
            if k in ("mma", "tcgen05"):  # kernels 2 and 3 share the weight gradient of kernel 1
                ms = timed(lambda: UN.conv3x3_wgrad(s0, dz, src1=s1, up0=bool(up)))
                row["wgrad_" + k] = {"ms": ms, "tflops": flops / ms / 1e9}
            UN.check_device_error()
        out.append(row)
    UN.set_conv_kernel(old)
    return out


def run_unet(args):
    """The warm-start network alone (BF16 U-Net, 128x128 inputs, batch 64):
    training samples/s of a full step (forward, backward, Adam) and
    prediction samples/s, on held-out draws; tensor-core roofline."""
    import numpy as np
    import torch
    from paper_1901_11350_gb300 import build
    from paper_1901_11350_gb300 import inputs as I
    from paper_1901_11350_gb300 import unet as UN
    from paper_1901_11350_gb300 import warmstart as W

    torch.cuda.set_device(0)
    build.build()
    if args.conv_kernel:
        UN.set_conv_kernel(args.conv_kernel)
    L, bm = 128, 64
    net = UN.UNet(L, bm, I.unet_init(0))
    draws = [I.warmstart_draw(I.WARMSTART_SEEDS["heldout"], 100000 + i, L) for i in range(bm)]
    s = W._records(np.stack([d["spins"] for d in draws]))
    f = W._features(draws)
    t = torch.zeros_like(s)
    t[..., 2] = 1.0
    flops = W.unet_flops(L)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    st = torch.cuda.current_stream()
    res = {}
    for name, fn, mult in (("train_step", lambda: net.train_step(s, f, t, 1e-4), 3), ("predict", lambda: net.predict(s, f), 1)):
        for _ in range(args.warmup):
            fn()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        torch.cuda.synchronize()
        for k in range(args.steps):
            flush.fill_(k & 0xFF)
            ev[k][0].record(st)
            fn()
            ev[k][1].record(st)
        torch.cuda.synchronize()
        ms = sum(a.elapsed_time(b) for a, b in ev) / args.steps
        res[name] = (ms, mult * bm * flops / (ms / 1e3) / 1e12)
    UN.check_device_error()
    # end to end: pinned host batch in, loss out, every step
    hs, hf, ht = s.cpu().pin_memory(), f.cpu().pin_memory(), t.cpu().pin_memory()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(st)
    for k in range(args.steps):
        loss = net.train_step(hs.to("cuda", non_blocking=True), hf.to("cuda", non_blocking=True),
                              ht.to("cuda", non_blocking=True), 1e-4)
        loss.item()
    e1.record(st)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / args.steps
    peaks, kind = measured_peaks()
    ms, tf = res["train_step"]
    out = {"metric": "U-Net training samples/s (BF16, 128x128, forward + backward + Adam)", "value": bm / (ms / 1e3),
           "unit": "samples/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
           "config": {"workload": "unet_hex128_b64", "batch": bm, "lattice": [L, L],
                      "widths": [32, 64, 128, 256], "conv_kernel": UN.conv_kernel(),
                      "l2": "flushed (256 MB write) before each step"},
           "e2e": {"value": bm / (e2e_ms / 1e3), "unit": "samples/s", "h2d_bytes_per_step": 2 * bm * L * L * 16 + bm * 16,
                   "d2h_bytes_per_step": 8},
           "roofline": {"bound": "tensor", "achieved": tf, "peak": peaks["bf16_tflops"], "unit": "TFLOP/s",
                        "frac": tf / peaks["bf16_tflops"], "traffic": None,
                        "peak_source": kind + " bf16 burst", "flop_per_sample_forward": flops,
                        "note": "whole training step (all kernels) against the convolution FLOPs x 3"},
           "predict": {"ms": res["predict"][0], "tflops": res["predict"][1],
                       "frac": res["predict"][1] / peaks["bf16_tflops"], "samples_per_s": bm / (res["predict"][0] / 1e3)}}
    if args.unet_layers:
        del net
        out["layers"] = unet_layer_times(bm)
    print(json.dumps(out))
    return 0


def run_warmstart(args):
    print(json.dumps(warmstart_result(args, args.systems)))
    return 0


def warmstart_result(args, systems, compact=False):
    """Learned warm start (BF16 U-Net, 128x128 periodic hexagonal lattices):
    device seconds until every held-out system has FP64 max torque < 1e-6 meV,
    for the unaided FP64 minimiser and for network prediction + FP32 + FP64,
    plus the network's own tensor-core throughput.  Needs trained parameters
    (``python -m paper_1901_11350_gb300.warmstart --out <prefix>``)."""
    import numpy as np
    import torch
    from paper_1901_11350_gb300 import build
    from paper_1901_11350_gb300 import inputs as I
    from paper_1901_11350_gb300 import unet as UN
    from paper_1901_11350_gb300 import warmstart as W

    torch.cuda.set_device(torch.cuda.current_device())
    build.build()
    params = W.load_params(args.weights)
    L, bm = 128, 64
    net = UN.UNet(L, bm, params)
    # network throughput: forward (predict) and training step on one batch
    draws = [I.warmstart_draw(I.WARMSTART_SEEDS["heldout"], 100000 + i, L) for i in range(bm)]
    s = W._records(np.stack([d["spins"] for d in draws]))
    f = W._features(draws)
    flops = W.unet_flops(L)
    times = {}
    for name, fn in (("predict", lambda: net.predict(s, f)), ("train_step", lambda: net.loss_grad(s, f, s))):
        for _ in range(args.warmup):
            fn()
        with W._Timer() as t:
            for _ in range(10):
                fn()
        times[name] = t.seconds / 10
    net.set_params(params)  # loss_grad above changed no parameter, but keep the state clean
    peaks, kind = measured_peaks()
    tf_pred = bm * flops / times["predict"] / 1e12
    tf_train = 3 * bm * flops / times["train_step"] / 1e12
    rep = W.evaluate(net, I.WARMSTART_SEEDS["heldout"], systems, L, max_iter=args.eval_max_iter,
                     polish_max_iter=5000, chunk=systems, per_system=args.per_system, log=lambda m: None)
    warm, una = rep["warm"], rep["unaided"]
    loop = rep["unaided_per_system_loop"]
    out = {"metric": "device seconds to FP64 max torque < 1e-6 meV for all systems, warm start vs unaided FP64",
           "value": warm["batched_seconds"], "unit": "s", "higher_is_better": False,
           "dtype": "bf16 network, f32 then f64 minimiser", "data": "synthetic", "n_gpus": 1,
           "config": {"workload": "warmstart_hex128", "systems": systems, "lattice": [L, L],
                      "max_iter": args.eval_max_iter, "params": os.path.basename(args.weights)},
           "unaided_fp64": {"batched_seconds": una["batched_seconds"], "per_system_loop_seconds_est":
                            loop["est_seconds_all"], "per_system_loop_sample": loop},
           "arms": {k: rep[k] for k in ("unaided", "batched", "warm", "uniform")},
           "speedup_vs_unaided_per_system_loop": loop["est_seconds_all"] / warm["batched_seconds"],
           "network": {"flop_per_sample_forward": flops, "batch": bm,
                       "predict_ms": 1e3 * times["predict"], "train_step_ms": 1e3 * times["train_step"],
                       "roofline": {"bound": "tensor", "achieved": tf_pred, "peak": peaks["bf16_tflops"],
                                    "unit": "TFLOP/s", "frac": tf_pred / peaks["bf16_tflops"], "traffic": None,
                                    "peak_kind": kind + " bf16 burst"},
                       "train_tflops": tf_train}}
    if compact:
        out["arms"] = {k: {kk: rep[k][kk] for kk in ("converged", "matched", "mean_iterations", "batched_seconds")
                           if kk in rep[k]} for k in ("unaided", "batched", "warm", "uniform")}
        out["unaided_fp64"].pop("per_system_loop_sample")
    return out


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--llg-steps", type=int, default=LLG_STEPS)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--temperature", type=float, default=None, help="override T (profiling aid)")
    ap.add_argument("--zc", default="", help="units per CTA of the 27-point path, P or P,C for predictor and "
                    "corrector (profiling aid; default: chosen by sp_autotune)")
    ap.add_argument("--generic", action="store_true", help="force the generic neighbour-list kernels")
    ap.add_argument("--cubic-lean", type=int, default=1, choices=[0, 1],
                    help="0: the general 27-point Heun passes even where the lean ones fit")
    ap.add_argument("--cubic-rows", default="", help="columns per thread of the 27-point kernels, R or R,C for "
                                                     "predictor and corrector (default: chosen by sp_autotune)")
    ap.add_argument("--solver", default="heun", choices=["heun", "depondt", "sib", "rk4"],
                    help="sc128: LLG solver (the workload is stochastic Heun; the others for comparison)")
    ap.add_argument("--workload", default="sc128", choices=["sc128", "gneb48", "hex512", "warmstart", "unet", "mc30", "hessian",
                                                        "square32", "sllg30"])
    ap.add_argument("--mc-sizes", default="10,15,20,30", help="mc30: lattice sides")
    ap.add_argument("--mc-thermal", type=int, default=10000, help="mc30: thermalisation sweeps")
    ap.add_argument("--mc-samples", type=int, default=100000, help="mc30: sampled sweeps")
    ap.add_argument("--mc-tmin", type=float, default=10.0)
    ap.add_argument("--mc-tmax", type=float, default=24.0)
    ap.add_argument("--mc-dt", type=float, default=0.5, help="mc30, sllg30: temperature step (K)")
    ap.add_argument("--mc-resident", type=int, default=1, choices=[0, 1],
                    help="mc30: 0 forces one launch per colour on every size")
    ap.add_argument("--sllg-thermal", type=int, default=20000, help="sllg30: thermalisation steps")
    ap.add_argument("--sllg-samples", type=int, default=100000, help="sllg30: sampled steps")
    ap.add_argument("--sllg-every", type=int, default=10, help="sllg30: steps between samples")
    ap.add_argument("--sllg-dt", type=float, default=1e-3, help="sllg30: time step (ps)")
    ap.add_argument("--sllg-alpha", type=float, default=1.0, help="sllg30: damping")
    ap.add_argument("--systems", type=int, default=200, help="warmstart: held-out systems")
    ap.add_argument("--eval-max-iter", type=int, default=30000, help="warmstart: iteration cap per relaxation")
    ap.add_argument("--per-system", type=int, default=4, help="warmstart: systems timed in the one-system loop")
    ap.add_argument("--weights", default=os.path.join(ROOT, "paper_1901_11350_gb300", "weights",
                                                      "warmstart_hex128.npz"))
    ap.add_argument("--chains", type=int, default=48)
    ap.add_argument("--gneb-chunk", type=int, default=50)
    ap.add_argument("--gneb-no-reference", action="store_true", help="gneb48: skip the FP64 per-chain loop (profiling aid)")
    ap.add_argument("--gneb-persistent", type=int, default=-1, choices=[-1, 0, 1],
                    help="gneb48: 1 = one persistent cooperative launch per call, 0 = one launch per pass, "
                         "-1 (default) = chosen by the autotuner")
    ap.add_argument("--conv-kernel", default="", choices=["", "mma", "tcgen05", "tcgen05_ws", "tcgen05_halo"],
                    help="unet: convolution kernel of the timed steps (default: the library's)")
    ap.add_argument("--unet-layers", action="store_true",
                    help="unet: add per-shape forward and weight-gradient times of every convolution kernel")
    ap.add_argument("--side", type=int, default=128, help="lattice side (profiling aid; the workload is 128)")
    ap.add_argument("--no-relax", action="store_true",
                    help="sc128: skip the relaxation half of the metric (GNEB batch, warm start)")
    ap.add_argument("--relax-systems", type=int, default=64,
                    help="sc128: held-out systems of the warm-start part of the relaxation half")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "gneb48":
        return run_gneb(args)
    if args.workload == "hex512":
        return run_hex_dipole(args)
    if args.workload == "warmstart":
        return run_warmstart(args)
    if args.workload == "unet":
        return run_unet(args)
    if args.workload == "mc30":
        return run_mc(args)
    if args.workload == "hessian":
        return run_hessian(args)
    if args.workload == "sllg30":
        return run_sllg(args)
    if args.workload == "square32":
        return run_square32(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
