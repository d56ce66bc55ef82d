#!/usr/bin/env python
"""Benchmark of the RTT Monte Carlo hot path on GB300.

One *step* is one Monte Carlo iteration of every chain of the workload: the
local energy of the configuration the iteration starts from and one
systematic single-spin Metropolis sweep (Sec. 3.3; TFIM of Sec. 4), i.e. one
local-energy sample per chain.  The library runs the energy on a second
stream beside the sweep (the sweep of a 4096-chain batch fills 32 of the 152
SMs).  Default workload: 6x6 open TFIM (N = 36, h = 3.0), R = 2 (L = 72),
chi = 64, 4096 chains; synthetic seeded tensors.

value        local-energy samples/s = chains x steps / summed device step time
e2e          the same through host buffers: every step copies the chains'
             spins and amplitudes from pinned host memory, runs the step and
             copies E_loc, spins and amplitudes back (all inside the timing)
roofline     dominant kernel: algorithmic flops per launch / its mean launch
             time (library event profiler on the launching stream) against
             the FP32 (or FP64) CUDA-core peak, or the measured bf16 tensor peak;
             step_* : the flops of every kernel of a step / the step time
             (kernels of one step overlap, so per-kernel times add up to more
             than the step)
cpu_baseline the FP64 oracle on this host's cores, bounded sample

--impl reference runs the FP64 CPU oracle as the reference arm.
Multi-GPU (torchrun): independent chain shards per rank (chain0 = rank * B),
weak scaling, no data-path collective.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("local-energy samples/s & effective samples/s at ≤1e-4 rel. energy error, 1 GB300")
SM_COUNT = 152
FP32_LANES_PER_SM = 128
FP64_LANES_PER_SM = 2


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default: a per-workload count that runs for seconds)")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="learned_16x16")
    ap.add_argument("--precision", default="fp16x3", choices=["fp32", "fp64", "bf16x3", "fp16x3"])
    ap.add_argument("--chains", type=int, default=0, help="override the workload's chain count")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--sweeps", type=int, default=0,
                    help="physical-space workloads: dual Monte Carlo sweeps per state (default 100)")
    ap.add_argument("--gram-schmidt", default="first", choices=["none", "first", "all"],
                    help="physical-space workloads: the basis of the dual Monte Carlo")
    args = ap.parse_args()
    if args.steps is None:
        args.steps = DEFAULT_STEPS.get(args.workload, 20)
    return args


# timed steps when --steps is not given: each runs for seconds
DEFAULT_STEPS = {"learned_16x16": 20, "plain_16x16": 20, "plain_6x6": 1000, "vhdd_6x6": 500, "prec_10x10": 50,
                 "tiny_fp64": 1000, "batched64": 3, "dual_6x6": 500, "physical_6x6": 3,
                 "physical_10x10": 2}

# executed tensor flops (dense-equivalent) per algorithmic flop of the
# split-precision site products: three hi/lo products (x3); the chi = 64
# split-row sweep also contracts both spin slices (x2), the other tensor-core
# kernels take the row's slice through a 2:4-sparse operand
def executed_per_alg(kernel: str, chi: int) -> float:
    return 6.0 if (kernel == "tc_sweep" and chi == 64) else 3.0


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0}, "fallback"


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-i", str(self.index), "-lms", "200"], stdout=subprocess.PIPE,
                stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (FileNotFoundError, OSError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- L2 flush
class L2Flush:
    """Evicts the 129 MB L2 between timed steps, outside the timed events:
    writes a 256 MiB buffer, then reads another 256 MiB buffer so that the
    written lines are written back before the next step, which starts with a
    cold, clean L2."""

    def __init__(self):
        import torch
        self.torch = torch
        n = 256 * 2**20 // 4
        self.w = torch.empty(n, dtype=torch.float32, device="cuda")
        self.r = torch.ones(n, dtype=torch.float32, device="cuda")
        self.sink = torch.empty((), dtype=torch.float32, device="cuda")

    def __call__(self):
        self.w.zero_()
        self.torch.sum(self.r, dim=0, out=self.sink)


# ---------------------------------------------------------------- DRAM traffic
# dram__bytes_read.sum + dram__bytes_write.sum of one launch of a kernel, from
# an ncu capture of that kernel as it is built now, keyed by (workload,
# precision, kernel, chains); a kernel with no current capture reports None.
# The 16x16 rows kernel was captured at 1024 chains (397.6 MB read + 9.7 MB
# written): the environment rows and spins every (tile, row) CTA reads, 337 MB,
# grow with the chains and the site tensors' 67 MB do not, so 8192 chains
# move 8 x 340.7 MB + 67 MB.
_ROWS16_TRAFFIC_8192 = 8 * (397.6e6 + 9.7e6 - 67.1e6) + 67.1e6
MEASURED_TRAFFIC = {
    ("learned_16x16", "fp16x3", "tc_rows", 8192): _ROWS16_TRAFFIC_8192,
    ("plain_16x16", "fp16x3", "tc_rows", 8192): _ROWS16_TRAFFIC_8192,
    ("plain_16x16", "fp16x3", "tc_rows", 1024): 397.6e6 + 9.7e6,
}


def measured_traffic(args, kernel, B):
    return MEASURED_TRAFFIC.get((args.workload, args.precision, kernel, B))


# ---------------------------------------------------------------- algorithmic work
def site_steps(N: int, R: int, kernel: str, path=None) -> int:
    """Row-site vector-matrix products one chain needs in one launch (periodic
    path; pass the path for a general one)."""
    if path is not None and not np.array_equal(path, np.tile(path[:N], len(path) // N)):
        L = len(path)
        first = {int(i): k for k, i in reversed(list(enumerate(path)))}
        last = {int(i): k for k, i in enumerate(path)}
        kmin = min(last.values()) + 1
        kind = kernel.split("_", 1)[1] if kernel.startswith(("simt_", "tc_")) else kernel
        if kind == "sweep":             # per proposal j: sites j..L-1 (the part after the
            return sum(L - j for j in range(N))   # spin's last site rebuilt from b_R)
        if kind == "rows":
            return sum(last[i] - first[i] + 1 for i in range(N)) + (L - N)
        if kind == "right_env":
            return L - kmin
        if kind == "left_env":
            return N
        if kind == "chain_init":
            return L
        return 0
    span = (R - 1) * N + 1
    if kernel in ("simt_sweep", "tc_sweep"):
        return (N - 1) + N * span + N            # right env + flip rows + l_j update
    if kernel in ("simt_rows", "tc_rows"):
        return N * span + (R - 1) * N            # N flip rows + the unflipped row
    if kernel in ("simt_right_env", "tc_right_env"):
        return N - 1
    if kernel in ("simt_left_env", "tc_left_env"):
        return N
    if kernel in ("simt_chain_init", "tc_chain_init"):
        return R * N
    return 0


# ---------------------------------------------------------------- reference arm (oracle)
def run_reference(args):
    """The reference arm: the FP64 oracle, as it stands, on this host's cores,
    each step a bounded sample of the workload's step (one chain per core for
    the learned-proposal workload, two per core otherwise)."""
    from concurrent.futures import ThreadPoolExecutor
    from oracle import oracle as orc
    from paper_2604_22718_gb300 import inputs
    w = inputs.WORKLOADS[args.workload]
    inst = inputs.workload(args.workload)
    o = orc.Oracle(inst)
    cores = os.cpu_count() or 1
    N = inst.n_spins
    learned = args.workload == "learned_16x16"
    # the binding splits a batch across threads only when it holds at least two
    # chains per thread; the learned workload's chains run one per thread here
    per_step = cores if learned else 2 * cores
    spins = inputs.initial_spins(w["seed"], per_step, N)
    mant, ex = o.init_chains(spins)
    if learned:
        from oracle import made as omade
        H = 512
        p = omade.masked_params(inputs.made_init_weights(w["seed"], N, H), N, H)
        order = inst.path[:N].astype(np.int64)
        exe = ThreadPoolExecutor(cores)

        def step(t):
            # the learned proposal, then the local sweep with its energy
            prop, lq_new = omade.sample(p, order, per_step, w["seed"], 0, t, N)
            lq_cur = omade.log_prob(p, spins, order)
            la_cur = o.log_amplitudes(spins)[0]
            la_new, _, m_new, e_new = o.log_amplitudes(prop)
            for c in range(per_step):
                if omade.indep_mh_decide(la_cur[c], lq_cur[c], la_new[c], lq_new[c],
                                         omade.accept_uniform(w["seed"], c, t, N)):
                    spins[c], mant[c], ex[c] = prop[c], m_new[c], e_new[c]

            def one(c):
                o.mcmc(w["seed"], spins[c:c + 1], mant[c:c + 1], ex[c:c + 1], t, 1,
                       measure_every=1, chain0=c)
            list(exe.map(one, range(per_step)))
    else:
        def step(t):
            o.mcmc(w["seed"], spins, mant, ex, t, 1, measure_every=1, threads=cores)
    t_total = 0.0
    for t in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        step(t)
        dt = time.perf_counter() - t0
        if t >= args.warmup:
            t_total += dt
    value = per_step * args.steps / t_total
    what = ("1 local sweep + E_loc (C oracle, one chain per thread) and 1 learned independence "
            "proposal (numpy FP64)" if learned else "1 sweep + E_loc")
    line = {
        "metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "impl": "reference",
        "config": {"workload": _workload_desc(args.workload, inst, per_step), "chains": per_step,
                   "sample": f"{per_step} chains per step (bounded sample of the "
                             f"{w['chains']}-chain workload), {what} each"},
        "cpu_baseline": {"value": value, "unit": "samples/s", "cores": cores, "kind": "oracle",
                         "sample": f"{per_step} chains x {args.steps} steps, {cores} threads"},
        "e2e": {"value": value, "unit": "samples/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def _workload_desc(name, inst, chains):
    R = inst.path.shape[0] // inst.n_spins
    return (f"{name}: {inst.lx}x{inst.ly} open TFIM N={inst.n_spins} J={inst.J} h={inst.h}, "
            f"R={R} L={inst.path.shape[0]} chi={inst.chi}, {chains} chains, "
            f"1 sweep + E_loc per step")


def cpu_baseline(inst, w, seed):
    """The FP64 oracle on this host's cores: ~20 core-seconds of CPU work."""
    from oracle import oracle as orc
    from paper_2604_22718_gb300 import inputs
    o = orc.Oracle(inst)
    cores = os.cpu_count() or 1
    # warm call (library load, first-touch), then a timed calibration
    warm = inputs.initial_spins(seed + 3, 2, inst.n_spins)
    wm, we = o.init_chains(warm)
    o.mcmc(seed, warm, wm, we, 0, 1, measure_every=1, threads=1)
    cal = 2 * cores
    spins = inputs.initial_spins(seed + 1, cal, inst.n_spins)
    mant, ex = o.init_chains(spins)
    t0 = time.perf_counter()
    o.mcmc(seed, spins, mant, ex, 0, 1, measure_every=1, threads=cores)
    dt = time.perf_counter() - t0
    cpu_per_chain = dt * cores / cal
    n = int(min(20000, max(cal, 20.0 / max(cpu_per_chain, 1e-6))))
    n = max(cores, (n // cores) * cores)
    spins = inputs.initial_spins(seed + 2, n, inst.n_spins)
    mant, ex = o.init_chains(spins)
    t0 = time.perf_counter()
    o.mcmc(seed, spins, mant, ex, 0, 1, measure_every=1, threads=cores)
    dt = time.perf_counter() - t0
    return {"value": n / dt, "unit": "samples/s", "cores": cores, "kind": "oracle",
            "sample": f"{n} chains x 1 sweep + E_loc (FP64 oracle, {cores} threads, "
                      f"{dt:.1f} s wall)"}


def batched_sample_flops(inst) -> float:
    """Algorithmic flops of one sample (sweep + right environment + rows) of an instance."""
    N, R, chi = inst.n_spins, inst.path.shape[0] // inst.n_spins, inst.chi
    steps = site_steps(N, R, "simt_sweep") + site_steps(N, R, "simt_right_env") + \
        site_steps(N, R, "simt_rows")
    return steps * 2.0 * chi * chi


def cpu_baseline_batched(insts, per, seed):
    """The FP64 oracle on this host's cores for the batched workload, bounded:
    for each chi of the workload its instance with the fewest site steps runs
    one sweep + E_loc on one chain per host thread; the flop rate of those runs,
    divided by the workload's mean algorithmic flops per sample, is the oracle's
    samples/s on the whole workload."""
    from oracle import oracle as orc
    from paper_2604_22718_gb300 import inputs
    cores = os.cpu_count() or 1
    picks = {}
    for inst in insts:
        if inst.chi not in picks or batched_sample_flops(inst) < batched_sample_flops(picks[inst.chi]):
            picks[inst.chi] = inst
    done_flops, wall = 0.0, 0.0
    for chi, inst in sorted(picks.items()):
        o = orc.Oracle(inst)
        warm = inputs.initial_spins(seed + 3, 1, inst.n_spins)
        wm, we = o.init_chains(warm)
        o.mcmc(seed, warm, wm, we, 0, 1, measure_every=1, threads=1)
        spins = inputs.initial_spins(seed + chi, cores, inst.n_spins)
        mant, ex = o.init_chains(spins)
        t0 = time.perf_counter()
        o.mcmc(seed, spins, mant, ex, 0, 1, measure_every=1, threads=cores)
        wall += time.perf_counter() - t0
        done_flops += cores * batched_sample_flops(inst)
    mean_flops = sum(batched_sample_flops(i) for i in insts) / len(insts)
    return {"value": done_flops / wall / mean_flops, "unit": "samples/s", "cores": cores,
            "kind": "oracle",
            "sample": f"one chain per thread x 1 sweep + E_loc of the smallest instance of each chi "
                      f"({sorted(picks)}), {wall:.1f} s wall; its flop rate over the workload's mean "
                      f"{mean_flops:.3g} algorithmic flops per sample"}


# ---------------------------------------------------------------- our arm
def run_ours(args):
    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    from paper_2604_22718_gb300 import inputs, rtt

    from paper_2604_22718_gb300 import dist as rdist
    w = inputs.WORKLOADS[args.workload]
    inst = inputs.workload(args.workload)
    B_total = (args.chains or w["chains"]) * world
    chain0, B = rdist.shard(B_total, rank, world)
    N = inst.n_spins
    R = inst.path.shape[0] // N
    m = rtt.RTT(inst, args.precision, seed=w["seed"])
    m.reserve(B)
    # every rank's chains are its block of one seeded start: N ranks run the
    # chains of one GPU, chain by chain
    spins = torch.from_numpy(inputs.initial_spins(w["seed"], B_total, N)[chain0:chain0 + B].copy()).cuda()
    _, _, state = m.log_amplitudes(spins)
    K, W = args.steps, args.warmup
    trace = torch.empty((K, B), dtype=torch.float64, device="cuda")
    scratch_row = torch.empty((1, B), dtype=torch.float64, device="cuda")
    acc = torch.zeros(B, dtype=torch.int64, device="cuda")
    flush = L2Flush()
    stream = torch.cuda.current_stream()
    sweep = 0
    for _ in range(W):
        m.mcmc_sweep(spins, state, sweep, 1, 1, scratch_row, None, chain0=chain0)
        sweep += 1
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    clocks = ClockSampler(dev)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    t_wall0 = time.perf_counter()
    for t in range(K):
        flush()                             # L2 flush outside the timed events
        starts[t].record(stream)
        m.mcmc_sweep(spins, state, sweep, 1, 1, trace[t:t + 1], acc, chain0=chain0)
        ends[t].record(stream)
        sweep += 1
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall0
    clk = clocks.stop()
    # per-kernel times from a separate profiled pass (the event profiler stays
    # off inside the timed region)
    n_prof = min(K, 20)
    sp_p, st_p = spins.clone(), state.clone()
    torch.cuda.synchronize()
    m.profile(True)
    for t in range(n_prof):
        flush()
        m.mcmc_sweep(sp_p, st_p, 900000 + t, 1, 1, scratch_row, None, chain0=chain0)
    torch.cuda.synchronize()
    prof = {k: (v[0] * K / n_prof, v[1] * K / n_prof) for k, v in m.profile_read().items()}
    m.profile(False)
    del sp_p, st_p
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    total_ms = sum(step_ms)
    if dist:
        tt = torch.tensor([total_ms], dtype=torch.float64, device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        total_ms = float(tt.item())
        dist.barrier()
    value = B_total * K / (total_ms / 1e3)
    stats = m.observables(trace, acc, K * N)
    ess_per_s = value / (2.0 * stats["tau_int"])

    # dominant kernel roofline
    peaks, peak_kind = measured_peaks()
    dom = max((k for k in prof if k != "eloc_reduce"), key=lambda k: prof[k][1]) if prof else None
    roof = None
    if dom:
        launches, ms = prof[dom]
        flops = 2.0 * inst.chi * inst.chi * site_steps(N, R, dom, inst.path) * B
        achieved = flops / (ms / launches / 1e3) / 1e12
        if args.precision in ("bf16x3", "fp16x3"):
            # fp16 and bf16 dense tensor rates are equal on this part; the
            # burst peak for a timed region under a second, else the sustained
            long_region = total_ms / 1e3 > 1.0
            peak = peaks["bf16_tflops_sustained" if long_region else "bf16_tflops"]
            bound, pk = "tensor", (f"bf16 dense {'sustained' if long_region else 'burst'} "
                                   f"({peak_kind}); fp16 = bf16 rate; executed = "
                                   f"{executed_per_alg(dom, inst.chi):g}x algorithmic")
        else:
            lanes = FP32_LANES_PER_SM if args.precision == "fp32" else FP64_LANES_PER_SM
            peak = SM_COUNT * lanes * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
            bound, pk = "alu", (f"{args.precision} CUDA-core fma peak: {SM_COUNT} SMs x {lanes} "
                                f"lanes x 2 flop x {peaks.get('sm_max_mhz', 2070.0):.0f} MHz")
        mult = executed_per_alg(dom, inst.chi) if bound == "tensor" else 1.0
        executed = achieved * mult
        step_flops = sum(2.0 * inst.chi * inst.chi * site_steps(N, R, k, inst.path) * B * v[0]
                         for k, v in prof.items()) / K
        step_tf = step_flops / (total_ms / K / 1e3) / 1e12
        roof = {"bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": measured_traffic(args, dom, B), "kernel": dom,
                "executed_tflops": executed, "executed_frac": executed / peak,
                "peak_source": pk, "flops_per_launch": flops,
                "launch_ms": ms / launches,
                "kernel_share": ms / sum(v[1] for v in prof.values()),
                "step_tflops": step_tf, "step_frac": step_tf / peak,
                "step_executed_frac": step_tf * mult / peak}
    launches_total = int(round(sum(v[0] for v in prof.values())))

    # end to end through host buffers
    e2e = None
    if not args.no_e2e:
        spins_h = spins.cpu().pin_memory()
        state_h = state.cpu().pin_memory()
        eloc_h = torch.empty((1, B), dtype=torch.float64).pin_memory()
        spins_d = torch.empty_like(spins)
        state_d = torch.empty_like(state)
        row_d = torch.empty((1, B), dtype=torch.float64, device="cuda")
        e_st = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
        e_en = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
        torch.cuda.synchronize()
        for t in range(K):
            flush()
            e_st[t].record(stream)
            spins_d.copy_(spins_h, non_blocking=True)
            state_d.copy_(state_h, non_blocking=True)
            m.mcmc_sweep(spins_d, state_d, sweep, 1, 1, row_d, None, chain0=chain0)
            eloc_h.copy_(row_d, non_blocking=True)
            spins_h.copy_(spins_d, non_blocking=True)
            state_h.copy_(state_d, non_blocking=True)
            e_en[t].record(stream)
            sweep += 1
        torch.cuda.synchronize()
        e2e_ms = sum(s.elapsed_time(e) for s, e in zip(e_st, e_en))
        if dist:
            tt = torch.tensor([e2e_ms], dtype=torch.float64, device="cuda")
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            e2e_ms = float(tt.item())
        e2e = {"value": B_total * K / (e2e_ms / 1e3), "unit": "samples/s",
               "h2d_bytes_per_step": B * N + 16 * B,
               "d2h_bytes_per_step": 8 * B + B * N + 16 * B}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": world, "steps": K,
            "warmup": W, "ms_per_step": total_ms / K, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp32": "f32", "fp64": "f64", "bf16x3": "bf16x3",
                      "fp16x3": "fp16x3"}[args.precision],
            "data": "synthetic",
            "config": {"workload": _workload_desc(args.workload, inst, B), "chains_per_gpu": B,
                       "precision": args.precision, "parallelism": f"replicas over chains x{world}",
                       "l2": "flushed (256 MiB write + 256 MiB read) between timed steps, outside the events"},
            "ess_per_s": ess_per_s, "tau_int": stats["tau_int"], "accept_rate": stats["accept_rate"],
            "e_mean": stats["mean"], "e_se": stats["se"], "v_score": stats["v_score"],
            "roofline": roof, "gpu_launches": launches_total,
            "kernels": {k: {"launches": v[0], "ms": v[1]} for k, v in prof.items()},
            "clocks": clk, "e2e": e2e, "wall_s_timed_region": t_wall,
        }
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(inst, w, w["seed"])
        print(json.dumps(line), flush=True)
    m.close()
    if dist:
        dist.destroy_process_group()


def run_batched(args):
    """Batched form: the 64-instance workload (lattices {4,6,8,12}^2, R {2,3,4},
    chi {32,64,128,256}, h ~ U[2.5,3.5]): the FP32 instances in one persistent
    launch per step and, unless --precision fp32, the chi 64 / 128 instances in
    the split precision on the tensor cores; against the same instances run as
    separate per-instance launches."""
    import torch
    from paper_2604_22718_gb300 import inputs, rtt
    torch.cuda.set_device(0)
    insts = inputs.batched_instances()
    per = args.chains or 1024
    chains = [per] * len(insts)
    K, W = args.steps, args.warmup
    tc_prec = args.precision if args.precision in ("fp16x3", "bf16x3") else None
    precs = [tc_prec if (tc_prec and inst.chi in (64, 128)) else "fp32" for inst in insts]
    n_tc = sum(p != "fp32" for p in precs)
    b = rtt.RTTBatch(insts, chains, precisions=precs)
    cache = os.path.join(ROOT, "paper_2604_22718_gb300", "_build", "batch_tiles.json")
    os.makedirs(os.path.dirname(cache), exist_ok=True)
    t0 = time.perf_counter()
    b.tune(cache, probe_chains=min(per, 64))
    tune_s = time.perf_counter() - t0
    spins = torch.cat([torch.from_numpy(inputs.initial_spins(3000 + i, c, inst.n_spins).ravel())
                       for i, (inst, c) in enumerate(zip(insts, chains))]).cuda()
    st = b.init(spins)
    e = torch.empty(b.total_chains, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    for t in range(W):
        b.step(spins, st, t, e)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    clocks = ClockSampler(torch.cuda.current_device())
    torch.cuda.synchronize()
    clocks.start()
    for t in range(K):
        ev[t][0].record(stream)
        b.step(spins, st, W + t, e)
        ev[t][1].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = sum(a.elapsed_time(z) for a, z in ev)
    value = b.total_chains * K / (ms / 1e3)
    # the same instances as separate launches (one rtt handle each, one sweep + E_loc)
    handles = [rtt.RTT(inst, precs[i], seed=22722 + i) for i, inst in enumerate(insts)]
    sps, sts, trs = [], [], []
    for i, (m, inst) in enumerate(zip(handles, insts)):
        sp = torch.from_numpy(inputs.initial_spins(3000 + i, per, inst.n_spins)).cuda()
        _, _, s_ = m.log_amplitudes(sp)
        sps.append(sp)
        sts.append(s_)
        trs.append(torch.empty((1, per), dtype=torch.float64, device="cuda"))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for m, sp, s_, tr in zip(handles, sps, sts, trs):
        m.mcmc_sweep(sp, s_, 0, 1, 1, tr)
    e1.record(stream)
    torch.cuda.synchronize()
    sep_ms = e0.elapsed_time(e1)
    flops = sum(per * batched_sample_flops(inst) for inst in insts)
    # end to end: each step's spins and chain states from pinned host buffers,
    # its energies, spins and states back to them
    e2e = None
    if not args.no_e2e:
        sp_h = spins.cpu().pin_memory()
        st_h = st.cpu().pin_memory()
        e_h = torch.empty(b.total_chains, dtype=torch.float64).pin_memory()
        sp_d, st_d = torch.empty_like(spins), torch.empty_like(st)
        ee = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        torch.cuda.synchronize()
        for t in range(K):
            ee[t][0].record(stream)
            sp_d.copy_(sp_h, non_blocking=True)
            st_d.copy_(st_h, non_blocking=True)
            b.step(sp_d, st_d, W + K + t, e)
            e_h.copy_(e, non_blocking=True)
            sp_h.copy_(sp_d, non_blocking=True)
            st_h.copy_(st_d, non_blocking=True)
            ee[t][1].record(stream)
        torch.cuda.synchronize()
        e2e_ms = sum(a.elapsed_time(z) for a, z in ee)
        nbytes = spins.numel() + st.numel() * st.element_size()
        e2e = {"value": b.total_chains * K / (e2e_ms / 1e3), "unit": "samples/s",
               "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes + 8 * b.total_chains}
    achieved = flops / (ms / K / 1e3) / 1e12
    peaks, kind = measured_peaks()
    peak = SM_COUNT * FP32_LANES_PER_SM * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    line = {
        "metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": 1, "steps": K,
        "warmup": W, "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if not tc_prec else f"f32+{tc_prec}", "data": "synthetic",
        "config": {"workload": f"batched64: {len(insts)} instances x {per} chains, lattices "
                               "{4,6,8,12}^2, R {2,3,4}, chi {32,64,128,256}; FP32 instances in one "
                               "persistent launch per step through a CUDA graph"
                               + (f", chi 64 and 128 instances ({n_tc}) in {tc_prec} on the tensor cores"
                                  if tc_prec else ""), "chains": b.total_chains},
        "separate_launches_ms_per_step": sep_ms, "speedup_vs_separate": sep_ms / (ms / K),
        "tune_s": tune_s,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": None, "kernel": "k_batch",
                     "peak_source": "fp32 CUDA-core fma peak; achieved counts the whole step's "
                                    "algorithmic flops, tensor-core instances included"},
        # per tensor-core instance and step: sweep, left and right environments, rows, reduction
        "gpu_launches": K * (1 + 5 * n_tc), "clocks": clk, "e2e": e2e,
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_batched(insts, per, 22722)
    print(json.dumps(line), flush=True)
    for m in handles:
        m.close()
    b.close()


# launches of one rtt_indep_mh call with tensor-core (BF16) inference that the
# RTT handle's profiler does not see, from its host code: log q(s): W2 to BF16,
# inputs, layer 1, ReLU to BF16, layer 2, output layer, loss (7); sampling:
# init, ReLU to BF16, per position the tensor-core layer and the draw, and
# between positions the first-layer update (3N - 1 + 2); the decision (1).
# (psi of the proposals is the handle's amplitude kernel, profiled with it.)
def indep_mh_launches(N: int) -> int:
    return 7 + (3 * N + 1) + 1


def run_learned(args):
    """Learned-proposal form, the metric's configuration: 16x16 open TFIM
    (N = 256, h = 3.044), R = 2 (L = 512), chi = 128, 8192 chains, FP16X3
    site products.  A MADE 256 -> 512 -> 512 -> 256 is trained (library
    call) on 2^20 configurations of the plain local sampler (8192 chains x 128
    thinned sweeps); then each step is one mixed iteration of every chain: one
    learned independence proposal (BF16 tensor-core inference) and one local
    sweep with the local energy of the configuration entering it.

    value     mixed samples/s over exactly K timed steps (CUDA events on the
              launching stream, L2 flushed between steps outside the events,
              no profiler)
    ess_per_s value / (2 tau_int), tau_int (Sokal window) from a trace of
              max(K, 128) iterations whose first K are the timed steps
    plain     local flips only, FP16X3, same start, same protocol
    plain_fp32 the plain FP32 sampler on the CUDA cores (2 timed steps; tau_int
              of the FP16X3 local-flip trace, the same Markov kernel)
    gate      FP16X3 against the FP64 oracle on 48 sampled configurations:
              mean local energy within 1e-4 relative
    roofline  dominant kernel from a separate profiled pass"""
    import torch
    from paper_2604_22718_gb300 import inputs, rtt, dist as rdist
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    tdist = None
    if world > 1:
        import torch.distributed as tdist
        torch.cuda.set_device(local)
        tdist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    name = "learned_16x16"
    w = inputs.WORKLOADS[name]
    inst = inputs.workload(name)
    N = inst.n_spins
    R = inst.path.shape[0] // N
    B_total = (args.chains or w["chains"]) * world
    chain0, B = rdist.shard(B_total, rank, world)
    prec = args.precision
    K, W = args.steps, args.warmup
    T_tau = max(K, 128)
    n_data_sweeps = 128
    epochs = 20
    stream = torch.cuda.current_stream()
    m = rtt.RTT(inst, prec, seed=w["seed"])
    m.reserve(B)
    # every rank's chains are its block of one seeded start
    sp = torch.from_numpy(inputs.initial_spins(w["seed"], B_total, N)[chain0:chain0 + B].copy()).cuda()
    _, _, st = m.log_amplitudes(sp)
    t0 = time.perf_counter()
    m.mcmc_sweep(sp, st, 0, 16, chain0=chain0)                       # burn-in
    data = torch.empty((n_data_sweeps * B, N), dtype=torch.uint8, device="cuda")
    for r in range(n_data_sweeps):
        m.mcmc_sweep(sp, st, 16 + r, 1, chain0=chain0)
        data[r * B:(r + 1) * B].copy_(sp)
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    order = inst.path[:N].astype(np.int32)
    made = rtt.MADE(N, 512, order, inputs.made_init_weights(w["seed"], N, 512), seed=w["seed"])
    t0 = time.perf_counter()
    hist = made.fit(data, epochs=epochs, batch=1024, lr=1e-3, seed=w["seed"])
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    del data
    sp0, st0 = sp.clone(), st.clone()
    flush = L2Flush()
    sweep_base = 16 + n_data_sweeps

    def iterate(spins, state, t, mixed, row=None, acc=None):
        if mixed:
            rtt.indep_mh(m, made, spins, state, t, acc, chain0=chain0)
        m.mcmc_sweep(spins, state, t, 1, 1, row, chain0=chain0)

    def run(mixed):
        """W warm-up iterations, K timed ones (events), then untimed ones up to
        T_tau; returns (timed ms, trace [T_tau][B], acceptances, clocks)."""
        s2, st2 = sp0.clone(), st0.clone()
        tr = torch.empty((T_tau, B), dtype=torch.float64, device="cuda")
        junk = torch.empty((1, B), dtype=torch.float64, device="cuda")
        acc = torch.zeros(B, dtype=torch.int64, device="cuda")
        base = sweep_base + (100000 if mixed else 0)
        for t in range(W):
            iterate(s2, st2, base + t, mixed, junk)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(K)]
        clocks = ClockSampler(dev)
        torch.cuda.synchronize()
        if tdist:
            tdist.barrier()
        torch.cuda.synchronize()
        clocks.start()
        # an NVTX range marks the timed steps (profilers can filter on it)
        torch.cuda.nvtx.range_push("rtt_timed_mixed" if mixed else "rtt_timed_plain")
        for t in range(K):
            flush()
            ev[t][0].record(stream)
            iterate(s2, st2, base + W + t, mixed, tr[t:t + 1], acc)
            ev[t][1].record(stream)
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        clk = clocks.stop()
        if tdist:
            tdist.barrier()
        ms = sum(a.elapsed_time(z) for a, z in ev)
        for t in range(K, T_tau):
            iterate(s2, st2, base + W + t, mixed, tr[t:t + 1], acc)
        torch.cuda.synchronize()
        return ms, tr, acc, clk, (s2, st2)

    ms_m, tr_m, acc_m, clk, (sp_m, st_m) = run(True)
    ms_p, tr_p, _, clk_p, _ = run(False)
    ms_m, ms_p = _max_over_ranks(tdist, ms_m), _max_over_ranks(tdist, ms_p)
    obs_m = m.observables(tr_m)
    obs_p = m.observables(tr_p)
    value = B_total * K / (ms_m / 1e3)
    value_p = B_total * K / (ms_p / 1e3)
    ess_m = value / (2.0 * obs_m["tau_int"])
    ess_p = value_p / (2.0 * obs_p["tau_int"])

    # profiled pass (not timed): per-kernel CUDA-event times of the handle's
    # kernels over two mixed iterations
    s3, st3 = sp_m.clone(), st_m.clone()
    junk = torch.empty((1, B), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    m.profile(True)
    n_prof = 2
    t0 = time.perf_counter()
    for t in range(n_prof):
        iterate(s3, st3, 500000 + t, True, junk)
    torch.cuda.synchronize()
    prof = m.profile_read()
    m.profile(False)
    del s3, st3
    launches_per_step = sum(v[0] for v in prof.values()) / n_prof + indep_mh_launches(N)
    peaks, peak_kind = measured_peaks()
    dom = max((k for k in prof if k != "eloc_reduce"), key=lambda k: prof[k][1])
    launches, kms = prof[dom]
    flops = 2.0 * inst.chi * inst.chi * site_steps(N, R, dom, inst.path) * B
    achieved = flops / (kms / launches / 1e3) / 1e12
    long_region = ms_m / 1e3 > 1.0
    peak = peaks["bf16_tflops_sustained"] if long_region else peaks["bf16_tflops"]
    kind_txt = "sustained" if long_region else "burst"
    step_flops = sum(2.0 * inst.chi * inst.chi * site_steps(N, R, k, inst.path) * B * v[0]
                     for k, v in prof.items()) / n_prof
    step_tf = step_flops / (ms_m / K / 1e3) / 1e12
    roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": measured_traffic(args, dom, B), "kernel": dom,
            "flops_per_launch": flops, "launch_ms": kms / launches,
            "peak_source": f"bf16 dense {kind_txt} ({peak_kind}; timed region "
                           f"{ms_m / 1e3:.1f} s); fp16 = bf16 rate",
            "frac_of_burst": achieved / peaks["bf16_tflops"],
            "executed_per_algorithmic": executed_per_alg(dom, inst.chi),
            "kernel_share": kms / sum(v[1] for v in prof.values()),
            "step_tflops": step_tf, "step_frac": step_tf / peak}

    # end to end through host buffers: spins and amplitudes from pinned host
    # memory, one mixed iteration, E_loc, spins and amplitudes back, every step
    e2e = None
    if not args.no_e2e:
        sp_h = sp_m.cpu().pin_memory()
        st_h = st_m.cpu().pin_memory()
        el_h = torch.empty((1, B), dtype=torch.float64).pin_memory()
        sp_d, st_d = torch.empty_like(sp_m), torch.empty_like(st_m)
        row_d = torch.empty((1, B), dtype=torch.float64, device="cuda")
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(K)]
        torch.cuda.synchronize()
        for t in range(K):
            flush()
            ev[t][0].record(stream)
            sp_d.copy_(sp_h, non_blocking=True)
            st_d.copy_(st_h, non_blocking=True)
            iterate(sp_d, st_d, 600000 + t, True, row_d)
            el_h.copy_(row_d, non_blocking=True)
            sp_h.copy_(sp_d, non_blocking=True)
            st_h.copy_(st_d, non_blocking=True)
            ev[t][1].record(stream)
        torch.cuda.synchronize()
        e2e_ms = _max_over_ranks(tdist, sum(a.elapsed_time(z) for a, z in ev))
        e2e = {"value": B_total * K / (e2e_ms / 1e3), "unit": "samples/s",
               "h2d_bytes_per_step": B * N + 16 * B,
               "d2h_bytes_per_step": 8 * B + B * N + 16 * B}

    # the plain FP32 sampler (CUDA cores) on the same chains: 1 warm-up, 2 timed
    m32 = rtt.RTT(inst, "fp32", seed=w["seed"])
    m32.reserve(B)
    s32 = sp0.clone()
    _, _, st32 = m32.log_amplitudes(s32)
    junk = torch.empty((1, B), dtype=torch.float64, device="cuda")
    m32.mcmc_sweep(s32, st32, sweep_base, 1, 1, junk, chain0=chain0)
    ev32 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
            for _ in range(2)]
    torch.cuda.synchronize()
    for t in range(2):
        flush()
        ev32[t][0].record(stream)
        m32.mcmc_sweep(s32, st32, sweep_base + 1 + t, 1, 1, junk, chain0=chain0)
        ev32[t][1].record(stream)
    torch.cuda.synchronize()
    ms32 = _max_over_ranks(tdist, sum(a.elapsed_time(z) for a, z in ev32))
    m32.close()
    del s32, st32
    value32 = B_total * 2 / (ms32 / 1e3)
    ess32 = value32 / (2.0 * obs_p["tau_int"])

    line = None
    if rank == 0:
        gate = precision_gate(m, inst, sp_m[:48].clone())
        line = {
            "metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": world, "steps": K,
            "warmup": W, "ms_per_step": ms_m / K, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": prec, "data": "synthetic",
            "config": {"workload": _workload_desc(name, inst, B_total) +
                       "; each step also makes one learned independence proposal per chain "
                       "(MADE 256-512-512-256 trained on the plain sampler's configurations, "
                       "BF16 tensor-core inference)",
                       "chains_per_gpu": B, "precision": prec,
                       "parallelism": f"replicas over chains x{world} (each rank trains its own "
                                      "proposal on its own chains)",
                       "training_configs": n_data_sweeps * B, "epochs": epochs,
                       "l2": "flushed (256 MiB write + 256 MiB read) between timed steps, "
                             "outside the events"},
            "ess_per_s": ess_m, "tau_int": obs_m["tau_int"], "tau_trace_iterations": T_tau,
            "indep_acceptance": float(acc_m.sum()) / (B * T_tau),
            "e_mean": obs_m["mean"], "e_se": obs_m["se"], "v_score": obs_m["v_score"],
            "plain": {"samples_per_s": value_p, "ess_per_s": ess_p, "tau_int": obs_p["tau_int"],
                      "e_mean": obs_p["mean"], "e_se": obs_p["se"],
                      "what": "local flips only, same precision and start"},
            "plain_fp32": {"samples_per_s": value32, "ess_per_s": ess32, "steps": 2,
                           "what": "the plain sampler on the FP32 CUDA cores; tau_int of the "
                                   "local-flip trace above (same Markov kernel)"},
            "ess_speedup_vs_plain_fp32": ess_m / ess32,
            "ess_speedup_vs_plain_same_precision": ess_m / ess_p,
            "gate_rel_err": gate["rel_err"], "gate_ok": gate["rel_err"] <= 1e-4,
            "gate": gate,
            "roofline": roof, "gpu_launches": int(round(launches_per_step * K)),
            "kernels_per_step": {k: {"launches": v[0] / n_prof, "ms": v[1] / n_prof}
                                 for k, v in prof.items()},
            "made_nll_first_last_epoch": [hist[0], hist[-1]] if hist else None,
            "data_s": t_data, "train_s": t_train, "clocks": clk, "clocks_plain": clk_p,
            "e2e": e2e,
        }
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline_learned(inst, w["seed"], made)
        print(json.dumps(line), flush=True)
    made.close()
    m.close()
    if tdist:
        tdist.destroy_process_group()


def _max_over_ranks(tdist, ms):
    if not tdist:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device="cuda")
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return float(t.item())


def precision_gate(m, inst, spins):
    """Metric gate (R12): the local energies of the same configurations from
    the split-precision handle and the FP64 oracle; relative error of the mean
    (relative to the mean, or to the mean |E_loc| when the mean is near zero)."""
    from oracle import oracle as orc
    e = m.local_energy(spins).cpu().numpy()
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    e_o = orc.Oracle(inst).local_energies(spins.cpu().numpy(), threads=cores)
    dt = time.perf_counter() - t0
    scale = max(abs(float(e_o.mean())), float(np.mean(np.abs(e_o))))
    return {"rel_err": abs(float(e.mean()) - float(e_o.mean())) / scale,
            "configs": int(spins.shape[0]), "max_abs_err": float(np.max(np.abs(e - e_o))),
            "e_mean": float(e.mean()), "e_mean_fp64": float(e_o.mean()), "oracle_s": dt}


def cpu_baseline_learned(inst, seed, made_gpu):
    """The FP64 oracle on this host's cores, one mixed iteration (one local
    sweep with its local energy, and one learned independence proposal with the
    trained weights) for one chain per core."""
    from oracle import oracle as orc
    from oracle import made as omade
    from paper_2604_22718_gb300 import inputs
    cores = os.cpu_count() or 1
    o = orc.Oracle(inst)
    N = inst.n_spins
    n = cores
    spins = inputs.initial_spins(seed + 5, n, N)
    p = omade.unpack(made_gpu.params().astype(np.float64), N, made_gpu.hidden)
    order = inst.path[:N].astype(np.int64)
    from concurrent.futures import ThreadPoolExecutor

    def one(c):
        s = spins[c:c + 1].copy()
        mant, ex = o.init_chains(s)
        o.mcmc(seed, s, mant, ex, 0, 1, measure_every=1, chain0=c)
        return s

    t0 = time.perf_counter()
    with ThreadPoolExecutor(cores) as exe:
        out = list(exe.map(one, range(n)))
    # the learned proposal: ancestral sampling, log q of both states, psi(s'),
    # the decision
    cur = np.concatenate(out)
    prop, lq_new = omade.sample(p, order, n, seed, 0, 0, N)
    lq_cur = omade.log_prob(p, cur, order)
    la_new = o.log_amplitudes(prop)[0]
    la_cur = o.log_amplitudes(cur)[0]
    for c in range(n):
        omade.indep_mh_decide(la_cur[c], lq_cur[c], la_new[c], lq_new[c],
                              omade.accept_uniform(seed, c, 0, N))
    dt = time.perf_counter() - t0
    return {"value": n / dt, "unit": "samples/s", "cores": cores, "kind": "oracle",
            "sample": f"{n} chains x 1 mixed iteration (local sweep + E_loc in the C oracle, "
                      f"one chain per thread; learned proposal in numpy FP64), {dt:.1f} s wall"}


def run_dual(args):
    """Dual Monte Carlo (Sec. 3.3): M = 3 states of the plain_6x6 kind, 4096
    chains each; one step = rtt_dual_step: for every state a the mixed local
    energies and overlap ratios against all b of the configurations a's chains
    start from (second stream), beside one sweep of a's chains."""
    import torch
    from paper_2604_22718_gb300 import inputs, rtt
    name = "dual_6x6"
    w = inputs.WORKLOADS[name]
    states = inputs.workload_states(name)
    M, N = len(states), states[0].n_spins
    B = args.chains or w["chains"]
    hs = [rtt.RTT(s, args.precision, seed=w["seed"] + 100 * m) for m, s in enumerate(states)]
    spins = [torch.from_numpy(inputs.initial_spins(w["seed"] + m, B, N)).cuda() for m in range(M)]
    sts = [h.log_amplitudes(x)[2] for h, x in zip(hs, spins)]
    K, W = args.steps, args.warmup
    e = torch.empty((K, M, M, B), dtype=torch.float64, device="cuda")
    r = torch.empty((K, M, M, B), dtype=torch.float64, device="cuda")
    flush = L2Flush()
    stream = torch.cuda.current_stream()
    for t in range(W):
        rtt.dual_step(hs, spins, sts, t, e[0], r[0])
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    clocks = ClockSampler(torch.cuda.current_device())
    torch.cuda.synchronize()
    for h in hs:
        h.profile(True)
    clocks.start()
    for t in range(K):
        flush()
        ev[t][0].record(stream)
        rtt.dual_step(hs, spins, sts, W + t, e[t], r[t])
        ev[t][1].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    prof = {}
    for h in hs:
        for k, (n, ms) in h.profile_read().items():
            a = prof.setdefault(k, [0, 0.0])
            a[0] += n
            a[1] += ms
        h.profile(False)
    total_ms = sum(a.elapsed_time(z) for a, z in ev)
    value = M * B * K / (total_ms / 1e3)
    Ht, St, Hse, Sse = (np.zeros((M, M)) for _ in range(4))
    for a in range(M):
        for b in range(M):
            so = hs[a].observables(e[:, a, b, :].contiguous())
            sr = hs[a].observables(r[:, a, b, :].contiguous())
            Ht[a, b], Hse[a, b], St[a, b], Sse[a, b] = so["mean"], so["se"], sr["mean"], sr["se"]
    eig, c0 = rtt.dual_solve(Ht, St)
    dom = max(prof, key=lambda k: prof[k][1])
    launches, ms = prof[dom]
    R = states[0].path.shape[0] // N
    chi = states[0].chi
    flops = 2.0 * chi * chi * site_steps(N, R, dom) * B
    achieved = flops / (ms / launches / 1e3) / 1e12
    peaks, kind = measured_peaks()
    peak = peaks["bf16_tflops_sustained"]
    step_flops = sum(2.0 * chi * chi * site_steps(N, R, k) * B * v[0] for k, v in prof.items()) / K
    step_tf = step_flops / (total_ms / K / 1e3) / 1e12
    # oracle baseline on a bounded sample: mixed energies against all states and one sweep
    from oracle import oracle as orc
    from oracle import dual as odual
    cores = os.cpu_count() or 1
    nb = 48
    orcs = [orc.Oracle(s) for s in states]
    t0 = time.perf_counter()
    for a in range(M):
        sp = inputs.initial_spins(w["seed"] + a, nb, N)
        for b in range(M):
            odual.mixed_local_energies(orcs[a], orcs[b], sp, threads=cores)
        mant, ex = orcs[a].init_chains(sp)
        orcs[a].mcmc(w["seed"], sp, mant, ex, 0, 1, record=False, threads=cores)
    cpu_s = time.perf_counter() - t0
    line = {
        "metric": "dual Monte Carlo samples/s (chains x states per step; each sample carries "
                  "M mixed local energies and M overlap ratios)",
        "value": value, "unit": "samples/s", "n_gpus": 1, "steps": K, "warmup": W,
        "ms_per_step": total_ms / K, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"fp32": "f32", "fp64": "f64", "bf16x3": "bf16x3",
                                       "fp16x3": "fp16x3"}[args.precision],
        "data": "synthetic",
        "config": {"workload": f"{name}: {M} states of 6x6 open TFIM N=36 h=3.0, R=2 L=72 chi=64, "
                               f"{B} chains per state, rtt_dual_step per step",
                   "l2": "flushed (256 MiB write + 256 MiB read) between timed steps"},
        "mixed_local_energies_per_s": M * M * B * K / (total_ms / 1e3),
        "H_tilde": Ht.tolist(), "S_tilde": St.tolist(), "H_tilde_se": Hse.tolist(),
        "S_tilde_se": Sse.tolist(), "eigenvalues": [[float(z.real), float(z.imag)] for z in eig],
        "lowest_combination": c0.tolist(),
        "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": None, "kernel": dom,
                     "executed_frac": executed_per_alg(dom, chi) * achieved / peak, "step_tflops": step_tf,
                     "step_executed_frac": executed_per_alg(dom, chi) * step_tf / peak,
                     "peak_source": f"bf16 dense sustained ({kind}); fp16 = bf16 rate"},
        "kernels": {k: {"launches": v[0], "ms": v[1]} for k, v in prof.items()},
        "gpu_launches": sum(v[0] for v in prof.values()), "clocks": clk,
        "cpu_baseline": {"value": M * nb / cpu_s, "unit": "samples/s", "cores": cores,
                         "kind": "oracle",
                         "sample": f"{nb} chains per state: {M * M} mixed-energy sets + {M} sweeps "
                                   f"(FP64 oracle, {cores} threads, {cpu_s:.1f} s)"},
    }
    print(json.dumps(line), flush=True)
    for h in hs:
        h.close()


def rounding_flops(L: int, D2: int, chi: int) -> float:
    """Dense operation counts of one TT rounding of a two-term sum (bond D2
    rounded to chi): per site the product with the carried factor, a
    Householder QR with explicit Q (4 m n^2 - 4 n^3 / 3, m >= n), and a thin SVD
    with both factors (6 m n^2 + 20 n^3, m >= n) plus the product with U S."""

    def qr(m, n):
        m, n = max(m, n), min(m, n)
        return 4.0 * m * n * n - 4.0 * n ** 3 / 3.0

    def svd(m, n):
        m, n = max(m, n), min(m, n)
        return 6.0 * m * n * n + 20.0 * n ** 3

    f = 0.0
    for k in range(L):
        rl = min(2 ** min(k, 30), D2)
        dl = 1 if k == 0 else D2
        dr = 1 if k == L - 1 else D2
        f += 2.0 * (2 * rl) * dl * dr
        if k < L - 1:
            f += qr(2 * rl, dr)
        if k >= 1:
            r1 = min(chi, 2 ** min(L - 1 - k, 30))
            f += svd(rl, 2 * r1)
            t = min(chi, rl, 2 * r1)
            f += 2.0 * (2 * min(2 ** min(k - 1, 30), D2)) * rl * t
    return f


def run_replica(args):
    """Replica-space optimization (Sec. 3.1, Sec. 4): one step = one application
    of 1 - tau H-bar to the TT phi -- every term's rank-1 MPO, the tree of
    two-term sums each rounded to rank chi, phi - tau S rounded and scaled --
    from phi^(0) = 1.  After the timed steps the RTT psi = C phi is sampled
    with the library's FP64 sampler for its energy (not timed)."""
    import torch
    from paper_2604_22718_gb300 import inputs, rtt
    name = args.workload
    w = inputs.REPLICA_WORKLOADS[name]
    lx, ly, order, chi, tau, h = w["lx"], w["ly"], w["orderings"], w["chi"], w["tau"], w["h"]
    N = lx * ly
    path = inputs.path_sum([inputs.ordering(o, lx, ly) for o in order])
    L = path.shape[0]
    terms = inputs.hbar_terms(w["kind"], lx, ly, h, orderings=order)
    eta, ops = rtt.replica_lift(N, path, terms)
    K_terms = len(eta)
    levels, n = 0, K_terms
    while n > 1:
        n = n // 2 + n % 2
        levels += 1
    tt_prec = "fp64" if args.precision == "fp64" else "fp32"
    plan = rtt.TTPlan(L, chi, eta, ops, precision=tt_prec)
    phi0 = inputs.replica_ones(L, chi)
    phi = torch.from_numpy(phi0).cuda()
    K, W = args.steps, args.warmup
    ln = torch.empty(W + K, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    for t in range(W):
        plan.power(phi, tau, 1, ln[t:t + 1])
    flush = L2Flush()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    clocks = ClockSampler(torch.cuda.current_device())
    torch.cuda.synchronize()
    clocks.start()
    for t in range(K):
        flush()
        ev[t][0].record(stream)
        plan.power(phi, tau, 1, ln[W + t:W + t + 1])
        ev[t][1].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    total_ms = sum(a.elapsed_time(z) for a, z in ev)
    step_ms = total_ms / K
    value = K / (total_ms / 1e3)
    ct = min(2 * chi, 16)
    n1 = K_terms // 2                       # first level: sums of two rank-chi terms
    flops_step = (n1 * rounding_flops(L, 2 * chi, ct) + (K_terms - 1 - n1) * rounding_flops(L, 2 * ct, ct)
                  + rounding_flops(L, chi + ct, chi))
    achieved = flops_step / (step_ms / 1e3) / 1e12
    peaks, _ = measured_peaks()
    lanes = FP64_LANES_PER_SM if tt_prec == "fp64" else FP32_LANES_PER_SM
    peak = SM_COUNT * lanes * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    lognorm = ln.cpu().numpy()
    # end to end: phi from pinned host memory, one step, phi and its log-norm back
    e2e = None
    if not args.no_e2e:
        host_phi = torch.from_numpy(phi.cpu().numpy()).pin_memory()
        host_ln = torch.empty(1, dtype=torch.float64).pin_memory()
        dphi = torch.empty_like(phi)
        dln = torch.empty(1, dtype=torch.float64, device="cuda")
        ke = min(K, 200)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for t in range(ke):
            dphi.copy_(host_phi, non_blocking=True)
            plan.power(dphi, tau, 1, dln)
            host_phi.copy_(dphi, non_blocking=True)
            host_ln.copy_(dln, non_blocking=True)
        torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t0
        nb = phi.numel() * 8
        e2e = {"value": ke / e2e_s, "unit": "steps/s", "h2d_bytes_per_step": nb,
               "d2h_bytes_per_step": nb + 8}
    # the energy of psi = C phi, sampled (FP64, the TT's cores with b_L = b_R = e_0)
    e0v = np.zeros(chi)
    e0v[0] = 1.0
    inst = inputs.RTTInstance(n_spins=N, path=path.astype(np.int32), tensors=phi.cpu().numpy(),
                              b_left=e0v, b_right=e0v.copy(), bonds=inputs.open_bonds(lx, ly),
                              J=1.0, h=h, name=name, lx=lx, ly=ly, R=len(order))
    hh = rtt.RTT(inst, "fp64", seed=22730)
    B, burn, meas = 4096, 50, 200
    sp = torch.from_numpy(inputs.initial_spins(22731, B, N)).cuda()
    st = hh.log_amplitudes(sp)[2]
    hh.mcmc_sweep(sp, st, 0, burn)
    tr = torch.empty((meas, B), dtype=torch.float64, device="cuda")
    hh.mcmc_sweep(sp, st, burn, meas, measure_every=1, trace=tr)
    obs = hh.observables(tr)
    hh.close()
    cpu = None
    if not args.no_cpu_baseline:
        from oracle import replica as orp
        tt = orp.tt_ones(L)
        t0 = time.perf_counter()
        nsteps = 0
        while time.perf_counter() - t0 < 15.0 and nsteps < 1000:
            tt, _ = orp.power_step(tt, eta, ops, tau, chi)
            nsteps += 1
        cpu_s = time.perf_counter() - t0
        cpu = {"value": nsteps / cpu_s, "unit": "steps/s", "cores": 1, "kind": "oracle",
               "sample": f"{nsteps} steps of the same workload from phi^(0) = 1 (numpy FP64 "
                         f"oracle, one thread, {cpu_s:.1f} s)"}
    launches = K * (levels + 1)
    line = {
        "metric": "replica-space optimization steps/s (1 - tau H-bar on the TT, rounded to chi)",
        "value": value, "unit": "steps/s", "n_gpus": 1, "steps": K, "warmup": W,
        "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp64": "f64", "fp32": "f32"}[tt_prec], "data": "synthetic",
        "config": {"workload": f"{name}: {lx}x{ly} open TFIM h={h}, path "
                               f"{'+'.join(order)} (L={L}), H-bar_{w['kind']} ({K_terms} terms, "
                               f"{levels} tree levels, pairwise sums rounded to rank {min(2 * chi, 16)}), "
                               f"chi={chi}, tau={tau}, phi0 = 1",
                   "l2": "flushed (256 MiB write + 256 MiB read) between timed steps"},
        "roundings_per_s": K_terms * value,
        "launch_ms": step_ms / (levels + 1),
        "site_step_us": 1e3 * step_ms / (levels + 1) / (2 * L),
        "log_norm_last": float(lognorm[-1]),
        "energy": {"E_per_site": obs["mean"] / N, "se_per_site": obs["se"] / N,
                   "v_score": obs["v_score"], "tau_int": obs["tau_int"], "chains": B,
                   "sweeps": meas, "sampler": "FP64 SIMT, general path"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": None, "kernel": "k_tt_round",
                     "flops_per_step": flops_step,
                     "peak_source": ("FP64 CUDA-core peak, 152 SMs x 2 FP64 FMA lanes x 2070 MHz"
                                     if tt_prec == "fp64" else
                                     "FP32 CUDA-core peak, 152 SMs x 128 FP32 FMA lanes x 2070 MHz"),
                     "note": "latency-bound: each rounding is a chain of 2 L dependent small "
                             "factorizations on one warp"},
        "gpu_launches": launches, "clocks": clk, "e2e": e2e, "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)
    plan.close()


def run_physical(args):
    """Physical-space optimization (Sec. 3.2; Sec. 4, Table 1) on 6x6 or 10x10:
    from the replica-space result (H-bar_HV, 30 or 60 steps from phi^(0) = 1),
    iterations with the operators {1, O_X, O_ZZ,HV, O_ZZ,DD'}: operator states,
    dual Monte Carlo (4096 chains x 100 sweeps per state unless --chains /
    --sweeps say otherwise), the generalized eigenproblem and the combined TT.
    One step = one iteration; the sampled energy of each result (not timed) is
    reported beside lambda_0."""
    import torch
    from paper_2604_22718_gb300 import inputs, rtt
    from paper_2604_22718_gb300.physical import PhysicalOptimizer
    lx = ly = int(args.workload.split("_")[1].split("x")[0])
    start_steps = 30 if lx <= 6 else 60
    order = ("V", "H", "D", "Dp")
    chi, tau, h = 2, 0.1, 3.0
    N = lx * ly
    path = inputs.path_sum([inputs.ordering(o, lx, ly) for o in order])
    L = path.shape[0]
    ops = [("1", []),
           ("X", inputs.replica_terms(lx, ly, order, [], 1.0)),
           ("ZZ_HV", inputs.replica_terms(lx, ly, order, [("H", 1.0, "H"), ("V", 1.0, "V")], 0.0)),
           ("ZZ_DDp", inputs.replica_terms(lx, ly, order, [("D", 1.0, "D"), ("Dp", 1.0, "Dp")], 0.0))]
    eta, hops = rtt.replica_lift(N, path, inputs.hbar_terms("HV", lx, ly, h, orderings=order))
    prec = "fp64" if args.precision == "fp64" else "fp32"
    plan = rtt.TTPlan(L, chi, eta, hops, precision=prec)
    phi = torch.from_numpy(inputs.replica_ones(L, chi)).cuda()
    plan.power(phi, tau, start_steps)
    opt = PhysicalOptimizer(N, path, inputs.open_bonds(lx, ly), 1.0, h, chi, ops, precision=prec,
                            tt_precision=prec)
    B, S, burn = args.chains or 4096, args.sweeps or 100, 20
    BE = 4096           # chains of the (untimed) energy of each result
    gs = "" if args.gram_schmidt == "none" else args.gram_schmidt
    pilot = max(S // 5, 10) if gs else 0
    spins0 = inputs.initial_spins(22741, B, N)
    e_start = opt.energy(phi, BE, 200, 50, 22742)
    K, W = args.steps, args.warmup
    for t in range(W):
        opt.step(phi.clone(), spins0, B, S, burn, 22750 + t, gram_schmidt=gs)
    clocks = ClockSampler(torch.cuda.current_device())
    torch.cuda.synchronize()
    clocks.start()
    rows, total = [], 0.0
    for t in range(K):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = opt.step(phi, spins0, B, S, burn, 22760 + t, gram_schmidt=gs)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        total += dt
        phi = res["phi"]
        obs = opt.energy(phi, BE, 200, 50, 22770 + t)
        rows.append({"lambda0_per_site": float(res["lambda"][0].real) / N,
                     "E_per_site": obs["mean"] / N, "se_per_site": obs["se"] / N,
                     "v_score": obs["v_score"], "c": [float(x) for x in res["c"]], "s": dt,
                     "phases_s": {k: round(v, 4) for k, v in res["timing"].items()}})
    clk = clocks.stop()
    value = K / total
    M = len(ops)
    dual_samples = M * B * (S + pilot)
    cpu = None
    if not args.no_cpu_baseline:
        from oracle import replica as orp
        from oracle import oracle as orc
        from oracle import dual as odual
        # the oracle's own inputs of the same shapes: a seeded rank-chi TT, its
        # own lifting, a Gram-Schmidt basis of the same pattern (the cost does
        # not depend on the values)
        tt = orp.unpadded(inputs.replica_start(22744, L, chi))
        lifted = [orp.lift(terms, path, N) if terms
                  else (np.ones(1), np.zeros((1, L), dtype=np.uint8)) for _, terms in ops]
        t0 = time.perf_counter()
        phis = [orp.apply_operator(tt, e, o, opt.chi_s, chi_tree=min(2 * opt.chi_s, 16))[0]
                for e, o in lifted]
        t_tt = time.perf_counter() - t0
        e0v = np.zeros(opt.chi_s)
        e0v[0] = 1.0
        insts = [inputs.RTTInstance(n_spins=N, path=path.astype(np.int32),
                                    tensors=orp.padded(p, opt.chi_s),
                                    b_left=e0v, b_right=e0v.copy(), bonds=inputs.open_bonds(lx, ly),
                                    J=1.0, h=h) for p in phis]
        T = np.eye(M)
        if gs:
            for m in range(1, M):
                T[m, :1 if gs == "first" else m] = -0.5
        main = [insts[0]] + [odual.direct_sum([insts[a] for a in range(M) if T[m, a] != 0.0],
                                              T[m][T[m] != 0.0]) for m in range(1, M)]
        nb = 64
        cores = os.cpu_count() or 1
        sp = inputs.initial_spins(22743, nb, N)

        def unit(states, pairs, swept):
            """Oracle seconds for one sweep of each state in swept and the mixed
            energies of the (a, b) pairs, on nb chains."""
            oc = [orc.Oracle(i) for i in states]
            xs = [sp.copy() for _ in oc]
            t_sw = t_mx = 0.0
            for a in swept:
                mant, ex = oc[a].init_chains(xs[a])
                t = time.perf_counter()
                oc[a].mcmc(22744, xs[a], mant, ex, 0, 1, record=False, threads=cores)
                t_sw += time.perf_counter() - t
            for a, b in pairs:
                t = time.perf_counter()
                odual.mixed_local_energies(oc[a], oc[b], xs[a], threads=cores)
                t_mx += time.perf_counter() - t
            return t_sw, t_mx

        all_pairs = [(a, b) for a in range(M) for b in range(M)]
        t_sw, t_mx = unit(main, all_pairs, range(M))
        t_mc = ((S + burn) * t_sw + S * t_mx) * B / nb
        if gs:              # the pilot on the raw states: psi^1 alone for "first"
            p_sw, p_mx = (unit(insts, [(0, b) for b in range(1, M)], [0]) if gs == "first"
                          else unit(insts, all_pairs, range(M)))
            t_mc += ((pilot + burn) * p_sw + pilot * p_mx) * B / nb
        cpu_it = t_tt * 2 + t_mc
        cpu = {"value": 1.0 / cpu_it, "unit": "iterations/s", "cores": cores, "kind": "oracle",
               "sample": f"on a seeded rank-{chi} TT of the same shape: "
                         f"operator TTs timed in full ({t_tt:.1f} s, counted twice for the "
                         f"combination), dual Monte Carlo timed on {nb} chains x 1 sweep and "
                         f"{M}x{M} mixed energies of the states it runs on, scaled to {B} chains x "
                         f"{S + burn} sweeps with {S} measured"
                         + (f", plus the pilot ({pilot + burn} sweeps, {pilot} measured)" if pilot
                            else "")
                         + f" (FP64 oracle, {cores} threads)"}
    line = {
        "metric": "physical-space optimization iterations/s (operator TTs, dual Monte Carlo, "
                  "eigenproblem, combined TT)",
        "value": value, "unit": "iterations/s", "n_gpus": 1, "steps": K, "warmup": W,
        "ms_per_step": 1e3 * total / K, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"fp64": "f64", "fp32": "f32"}[prec], "data": "synthetic",
        "config": {"workload": f"{args.workload}: {lx}x{ly} open TFIM h={h}, path V+H+D+Dp (L={L}), "
                               f"chi={chi}, operators 1, O_X, O_ZZ,HV, O_ZZ,DD' ({M} states of rank "
                               f"{opt.chi_s}), start = "
                               f"{start_steps} steps of "
                               f"H-bar_HV from phi0 = 1; dual Monte Carlo {B} chains x {S} sweeps "
                               f"(+{burn} burn-in) per state"
                               + (f" on the Gram-Schmidt states (against psi^1 only)" if gs == "first"
                                  else " on the Gram-Schmidt states" if gs else "")
                               + (f" after a {pilot}-sweep pilot" if gs else "")
                               + f", {prec.upper()} sampler and TT arithmetic",
                   "timing": "host wall clock around each iteration (synchronized), includes "
                             "handle creation and the host eigen-solver"},
        "dual_samples_per_s": dual_samples * value,
        "start": {"E_per_site": e_start["mean"] / N, "se_per_site": e_start["se"] / N,
                  "v_score": e_start["v_score"]},
        "iterations": rows,
        "roofline": None,
        "roofline_note": "composite of kernels measured in the dual_6x6 and replica_* lines",
        "clocks": clk, "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)
    opt.close()
    plan.close()


def main():
    args = parse()
    if args.impl == "reference":
        if int(os.environ.get("RANK", "0")) != 0:
            return
        run_reference(args)
        return
    if args.workload == "batched64":
        if int(os.environ.get("RANK", "0")) == 0:
            run_batched(args)
        return
    if args.workload == "learned_16x16":
        if int(os.environ.get("RANK", "0")) == 0:
            run_learned(args)
        return
    if args.workload in ("physical_6x6", "physical_10x10"):
        if int(os.environ.get("RANK", "0")) == 0:
            run_physical(args)
        return
    if args.workload.startswith("replica_"):
        if int(os.environ.get("RANK", "0")) == 0:
            run_replica(args)
        return
    if args.workload == "dual_6x6":
        if int(os.environ.get("RANK", "0")) == 0:
            run_dual(args)
        return
    run_ours(args)


if __name__ == "__main__":
    main()
