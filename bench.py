"""Walker-step throughput of the GB300 ph-AFQMC library.

One bench step is one measurement block of the hot path: 20 imaginary-time
steps of every walker (force bias, field draw, one-body operator, Taylor
propagation, overlaps, weights), with orthonormalisation every 2 steps and
the local energy plus comb population control at the end of the block. The
metric is walker-steps per second over the whole job.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload c2|c1|c3] [--precision fp64|fp32|tf32|tf32x3]

Under torchrun (N > 1) every rank runs an independent replica (its own Philox
stream tag); there is no data-path collective. The reference arm times the
FP64 CPU oracle on the host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "walker-steps/s"
BLOCK = 20  # imaginary-time steps per bench step (one measurement/comb block)
PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}
# FP64 and FP32 SIMT peaks from unit counts: 152 SMs at the 2070 MHz maximum
# clock; FP32 128 FMA lanes per SM, FP64 from the nominal 1.25 TFLOP/s.
SM_COUNT, SM_MAX_MHZ = 152, 2070.0
FP32_SIMT_TFLOPS = SM_COUNT * 128 * 2 * SM_MAX_MHZ * 1e6 / 1e12
FP64_TFLOPS = 1.25
TF32_OVER_BF16 = 0.5   # nominal dense TF32 : BF16 tensor throughput


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c2")
    ap.add_argument("--precision", default="tf32x3")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64-compare", action="store_true",
                    help="skip the FP64 GPU comparison run (speed and energy)")
    ap.add_argument("--no-serving", action="store_true",
                    help="skip the serving-loop measurement (p50/p99 per block)")
    ap.add_argument("--no-shapes", action="store_true",
                    help="skip the other workload shapes (TM-atom, multi-determinant)")
    return ap.parse_args()


def workload(name, rank=0):
    from synth import CONFIGS
    s = CONFIGS[name]()
    return s.replace(run_id=rank)


def describe(s):
    return (f"{s.name}: M={s.M} N={s.n_up}+{s.n_dn} n_chol={s.n_chol} "
            f"W={s.n_walkers} dtau={s.dtau} det={s.n_det}")


# ------------------------------------------------------------------ peaks

def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return dict(PEAKS_FALLBACK), "fallback"


def roofline_for(kernel_stats, precision, peaks, src, s, workload_name, taylor_fused=None):
    """Dominant kernel of the timed region against its bound. The propagate
    group runs on the tensor cores unless the propagation path is the
    CUDA-core series (taylor_fused = 0, or 4 for block-diagonal Cholesky
    vectors; when the path is not given, the CUDA-core series is assumed
    above M = 64), where it is rated against the FP32 CUDA-core peak. BF16X3 propagates with BF16 products (BF16 peak);
    its other contractions are TF32X3 (TF32 peak)."""
    best = max(kernel_stats.items(), key=lambda kv: kv[1]["total_ms"])
    name, st = best
    avg_s = st["total_ms"] / max(1, st["launches"]) / 1e3
    # 0: the CUDA-core series; 4: the block-diagonal series on the CUDA cores
    prop_tc = (taylor_fused not in (0, 4)) if taylor_fused is not None else s.M <= 64
    tensor_groups = ("force_bias", "one_body", "energy") + (("propagate",) if prop_tc else ())
    if st["is_bytes"]:
        bound, unit = "hbm", "GB/s"
        achieved = st["work"] / avg_s / 1e9
        peak = peaks["hbm_gbs"]
        peak_src = f"hbm_gbs ({src})"
    elif precision in ("tf32", "tf32x3", "bf16x3") and name not in tensor_groups:
        # the small inverses, QR and field draws run on the CUDA cores in FP32
        bound, unit = "alu", "TFLOP/s"
        achieved = st["work"] / avg_s / 1e12
        peak = FP32_SIMT_TFLOPS
        peak_src = "FP32 CUDA cores: 152 SM x 128 lanes x 2 x 2070 MHz"
    elif precision == "fp64":
        bound, unit = "alu", "TFLOP/s"
        achieved = st["work"] / avg_s / 1e12
        peak = FP64_TFLOPS
        peak_src = "FP64 nominal 1.25 TFLOP/s"
    elif precision == "fp32":
        bound, unit = "alu", "TFLOP/s"
        achieved = st["work"] / avg_s / 1e12
        peak = FP32_SIMT_TFLOPS
        peak_src = "FP32 SIMT: 152 SM x 128 lanes x 2 x 2070 MHz"
    elif precision == "bf16x3" and name == "propagate":
        bound, unit = "tensor", "TFLOP/s"
        achieved = st["work"] / avg_s / 1e12
        peak = peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"])
        peak_src = f"bf16 sustained ({src})"
    else:
        bound, unit = "tensor", "TFLOP/s"
        achieved = st["work"] / avg_s / 1e12
        peak = peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"]) * TF32_OVER_BF16
        peak_src = f"bf16 sustained ({src}) x 0.5 nominal TF32 ratio"
    traffic = lookup_traffic(name, precision, workload_name)
    return {"kernel": name, "bound": bound, "achieved": round(achieved, 3),
            "peak": round(peak, 3), "unit": unit, "frac": round(achieved / peak, 4),
            "peak_source": peak_src,
            "traffic": traffic,
            "launches": st["launches"], "avg_launch_us": round(avg_s * 1e6, 2),
            "work_per_launch": st["work"]}


def lookup_traffic(kernel, precision, workload_name):
    """DRAM bytes per launch from the committed ncu summary, if one matches
    the kernel group, precision and workload."""
    p = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(p):
        return None
    for line in open(p):
        t = line.split()
        if (len(t) >= 5 and not line.startswith("#") and t[0] == kernel and t[1] == precision
                and t[2] == workload_name):
            return float(t[3])
    return None


# ------------------------------------------------------------------ clocks

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.rows = []
        self.proc = None
        self.index = index

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = sorted(float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit())
        mx = max((float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()), default=None)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            for i, n in enumerate(names):
                if len(r) > 4 + i and r[4 + i].lower() == "active":
                    reasons.add(n)
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(self.rows)}


# ------------------------------------------------------------------ CPU oracle

_WORKER_SYSTEM = {}


def _oracle_init(name):
    # never raise here: a failing pool initializer respawns workers forever
    try:
        from synth import CONFIGS
        import oracle.afqmc  # noqa: F401
        _WORKER_SYSTEM[name] = CONFIGS[name]().replace(measure_every=0, pc_every=0)
    except Exception as e:  # reported by the first task
        _WORKER_SYSTEM["error"] = repr(e)


def _oracle_worker(args):
    name, walker_ids, n_steps = args
    if "error" in _WORKER_SYSTEM:
        raise RuntimeError(_WORKER_SYSTEM["error"])
    from oracle import afqmc as O
    s = _WORKER_SYSTEM[name]
    run = O.OracleRun(s, walker_ids=walker_ids)
    t0 = time.perf_counter()
    run.run(n_steps)
    if n_steps >= BLOCK:
        run.local_energies()      # the block's one energy measurement
    return time.perf_counter() - t0


def cpu_oracle(name, budget_s=20.0):
    """The FP64 oracle as it stands, one process per host core (spawned, one
    BLAS thread each), each following its own walkers for a few steps plus
    one energy measurement. Returns (walker-steps/s, cores, sample text)."""
    import multiprocessing as mp
    from synth import CONFIGS
    s = CONFIGS[name]()
    cores = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    # probe: one walker, one step, to size the sample to the budget
    env = dict(os.environ, OPENBLAS_NUM_THREADS="1", OMP_NUM_THREADS="1")
    old = {k: os.environ.get(k) for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS")}
    os.environ.update({"OPENBLAS_NUM_THREADS": "1", "OMP_NUM_THREADS": "1"})
    try:
        with ctx.Pool(cores, initializer=_oracle_init, initargs=(name,)) as pool:
            t1 = pool.map(_oracle_worker, [(name, [0], 2)])[0]
            per_ws = max(t1 / 2.0, 1e-5)
            steps = BLOCK        # one block: ortho every 2, energy at the end
            per_core = max(1, int(budget_s / (per_ws * steps)))
            per_core = min(per_core, max(1, s.n_walkers // cores))
            jobs = [(name, list(range(c * per_core, (c + 1) * per_core)), steps)
                    for c in range(cores)]
            t0 = time.perf_counter()
            pool.map(_oracle_worker, jobs)
            wall = time.perf_counter() - t0
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    ws = cores * per_core * steps
    sample = (f"{describe(s)}; {cores} processes x {per_core} walkers x {steps} steps "
              f"(orthonormalisation every 2, one local-energy evaluation at the end, "
              f"no comb); full M, N, n_chol")
    return ws / wall, cores, sample


# ------------------------------------------------------------------ GPU arm

def max_over_ranks(x, device):
    """The slowest rank's value (every rank gets it): the job's time is the
    time of its slowest replica."""
    import torch
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(units_per_rank, world, max_ms):
    """Units all ranks processed per second of the slowest rank's time."""
    return units_per_rank * world / (max_ms / 1e3)


def flush_l2(buf):
    buf.add_(1.0)


def run_ours(args, rank, world):
    import numpy as np
    import torch
    from paper_1804_03310_gb300 import Afqmc

    s = workload(args.workload, rank)
    s = s.replace(measure_every=BLOCK, pc_every=BLOCK, ortho_every=2)
    torch.cuda.set_device(rank % max(1, torch.cuda.device_count()))
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        return _timed(args, s, stream, rank, world)


def _timed(args, s, stream, rank, world):
    import torch
    from paper_1804_03310_gb300 import Afqmc
    ctx = Afqmc.from_system(s, precision=args.precision, stream=stream.cuda_stream)
    flush = torch.zeros(256 * 1024 * 1024 // 4, device="cuda", dtype=torch.float32)
    for _ in range(args.warmup):
        ctx.afqmc_propagate(BLOCK)
    torch.cuda.synchronize()
    ctx.afqmc_set_kernel_timing(True)
    n0 = ctx.afqmc_launch_count()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    total_ms = 0.0
    with ClockSampler(rank % max(1, torch.cuda.device_count())) as clk:
        for _ in range(args.steps):
            flush_l2(flush)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            ctx.afqmc_propagate(BLOCK)
            b.record(stream)
            b.synchronize()
            total_ms += a.elapsed_time(b)
    torch.cuda.synchronize()
    launches = ctx.afqmc_launch_count() - n0
    from paper_1804_03310_gb300 import KERNEL_IDS
    kstats = {k: ctx.afqmc_kernel_stats(k) for k in KERNEL_IDS}
    kstats = {k: v for k, v in kstats.items() if v["launches"] > 0}
    kstats["_taylor_fused"] = ctx.afqmc_get_tuning().get("taylor_fused") if args.precision in (
        "tf32", "tf32x3", "bf16x3") else 0
    ctx.afqmc_synchronize()
    hist = ctx.afqmc_energy_history()
    ctx.close()
    if world > 1:
        total_ms = max_over_ranks(total_ms, "cuda")
    e2e = None if args.no_e2e else run_e2e(args, s)
    return s, total_ms, launches, kstats, clk.summary(), hist, e2e


def run_e2e(args, s):
    """Same metric through the public API with host buffers: create (host
    inputs copied to the device), K blocks each ending with the weights and
    local energies read back to the host, destroy."""
    import numpy as np
    import torch
    from paper_1804_03310_gb300 import Afqmc
    h2d = (s.h1.nbytes + s.L.nbytes + s.C_up.nbytes + s.C_dn.nbytes + s.occ_up.nbytes
           + s.occ_dn.nbytes + s.ci.nbytes)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ctx = Afqmc.from_system(s, precision=args.precision)
    d2h = 0
    for _ in range(args.steps):
        ctx.afqmc_propagate(BLOCK)
        w, lo = ctx.afqmc_weights()
        e, em = ctx.afqmc_local_energy()
        d2h += w.nbytes + lo.nbytes + e.nbytes + 8
    ctx.close()
    wall = time.perf_counter() - t0
    return {"value": round(s.n_walkers * BLOCK * args.steps / wall, 1), "unit": METRIC,
            "h2d_bytes_per_step": int(h2d / args.steps),
            "d2h_bytes_per_step": int(d2h / args.steps),
            "includes": "context creation with setup precompute, host read-back every block"}


def fp64_compare(args, s, hist):
    """The plain FP64 GPU path on the same workload and seed: its
    walker-steps/s over two timed blocks, the cuBLAS DGEMM rate of this GPU
    (the FP64 roofline), and the paired difference of the mixed energies
    recorded at the same steps (both runs draw the same fields)."""
    import numpy as np
    import torch
    from paper_1804_03310_gb300 import Afqmc
    n_blocks = min(3, args.warmup + args.steps)
    stream = torch.cuda.Stream()
    ctx = Afqmc.from_system(s, precision="fp64", stream=stream.cuda_stream)
    times = []
    for b in range(n_blocks):
        a = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ctx.afqmc_propagate(BLOCK)
        e.record(stream)
        e.synchronize()
        times.append(a.elapsed_time(e))
    ctx.close()
    timed = times[1:] if len(times) > 1 else times
    v64 = s.n_walkers * BLOCK * len(timed) / (sum(timed) / 1e3)
    # cuBLAS DGEMM on this GPU, the measured FP64 denominator
    n = 4096
    x = torch.randn(n, n, dtype=torch.float64, device="cuda")
    y = torch.randn(n, n, dtype=torch.float64, device="cuda")
    for _ in range(2):
        torch.matmul(x, y)
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    e = torch.cuda.Event(enable_timing=True)
    a.record()
    reps = 5
    for _ in range(reps):
        torch.matmul(x, y)
    e.record()
    e.synchronize()
    dgemm = 2.0 * n ** 3 * reps / (a.elapsed_time(e) / 1e3) / 1e12
    return {"value": round(v64, 1), "unit": METRIC, "blocks_timed": len(timed),
            "dgemm_tflops": round(dgemm, 3),
            "energy_check": energy_check(args.precision),
            "energy_check_shapes": energy_check_shapes(args.precision)}


def energy_check_shapes(precision):
    """Paired energy deviation at the full-size shapes: the H-chain shape
    (200 steps), the TM-atom shape (100 steps) and the multi-determinant
    shape (60 steps: without the comb its walkers die off from about step
    50), each in `precision` and in FP64 on the GPU with the
    same seed, comb off, one measurement every 20 steps. Walker i of one run
    is walker i of the other, so the difference of the mixed estimates is
    the precision error alone, whether or not the energy still drifts."""
    import numpy as np
    from synth import CONFIGS
    from paper_1804_03310_gb300 import Afqmc
    out = {}
    precs = [precision] + [p for p in ("tf32x3", "bf16x3") if p != precision]
    for name, n_steps in (("c2", 200), ("c3", 100), ("c4", 60)):
        s = CONFIGS[name]().replace(pc_every=0, measure_every=20)
        e = {}
        for p in ["fp64"] + precs:
            with Afqmc.from_system(s, precision=p) as ctx:
                ctx.afqmc_propagate(n_steps)
                e[p] = ctx.afqmc_energy_history()[:, 1]
        out[name] = {"steps": n_steps, "measurements": int(len(e["fp64"])),
                     "e_fp64_last": round(float(e["fp64"][-1]), 6)}
        for p in precs:
            d = (e[p] - e["fp64"]) * 1e3
            out[name][p] = {"max_abs_mHa": round(float(np.max(np.abs(d))), 6),
                            "mean_mHa": round(float(np.mean(d)), 6)}
    return out


def energy_check(precision, n_steps=600):
    """Mixed energies of the plain 10-orbital system (5+5 electrons, 40 dense
    fields, 512 walkers, dt = 0.01, comb off) in `precision` and on the FP64
    GPU path with the same seed: walker i of one run is walker i of the
    other, so the difference, measurement by measurement, is the precision
    error alone."""
    import numpy as np
    from synth import config_c1
    from paper_1804_03310_gb300 import Afqmc
    s = config_c1().replace(n_walkers=512, pc_every=0)
    out = {}
    for p in ("fp64", precision):
        with Afqmc.from_system(s, precision=p) as ctx:
            ctx.afqmc_propagate(n_steps)
            out[p] = ctx.afqmc_energy_history()[:, 1]
    d = (out[precision] - out["fp64"]) * 1e3
    return {"workload": f"{s.name}: M={s.M} N={s.n_up}+{s.n_dn} n_chol={s.n_chol} "
                        f"W={s.n_walkers} dtau={s.dtau}, {n_steps} steps, shared draws, comb off",
            "measurements": int(len(d)),
            "max_abs_mHa": round(float(np.max(np.abs(d))), 6),
            "mean_mHa": round(float(np.mean(d)), 6)}


def serving_leg(precision, n_runs=20, rate=20.0, seed=5, blocks=10, steps=50, mf_subtract=1):
    """The serving loop under a Poisson stream of independent runs drawn from
    the serving mix at its stated ranges: M in 20..200, N per spin M/5..M/3,
    n_chol 4M..6M, 128..2048 walkers, dt = 0.005, `blocks` blocks of `steps`
    steps each (energy once per block, comb every 10 steps), with the
    reference determinant's mean field subtracted (without it the phaseless
    cut empties a third of these random-trial populations). Inputs are
    drawn before the clock starts; submissions follow the arrival times;
    runs use the fixed launch heuristics (no per-request tuning); p50/p99 are
    the server's own per-block latencies. Offered load = the submitted runs'
    walker-steps over the arrival window; served = completed walker-steps
    over the elapsed time."""
    import numpy as np
    from synth.systems import serving_run
    from paper_1804_03310_gb300 import Inputs, Server
    rng = np.random.default_rng(seed)
    systems = [serving_run(rng, k) for k in range(n_runs)]
    runs = [Inputs.from_system(sy, precision=precision, autotune=False,
                               mf_subtract=mf_subtract) for sy in systems]
    gaps = rng.exponential(1.0 / rate, size=n_runs)
    srv = Server()
    t0 = time.perf_counter()
    t_arrive = 0.0
    ids = []
    for inp, gap in zip(runs, gaps):
        now = time.perf_counter() - t0
        if now < t_arrive:
            time.sleep(t_arrive - now)
        ids.append(srv.afqmc_server_submit(inp, blocks, steps))
        t_arrive += gap
    window = time.perf_counter() - t0
    srv.afqmc_server_wait(-1, 900)
    st = srv.afqmc_server_stats()
    failures = []
    for i in ids:
        info = srv.afqmc_server_poll(i)
        if info["state"] != "done":
            failures.append(f"run {i}: {info['state']} {info['message']}")
    srv.close()
    offered = sum(sy.n_walkers for sy in systems) * blocks * steps
    return {"workload": (f"{n_runs} runs, Poisson arrivals {rate}/s, M 20..200, N/spin M/5..M/3, "
                         f"n_chol 4M..6M, W 128..2048, {blocks} blocks of {steps} steps "
                         f"(comb every 10), {precision}, mean field "
                         f"{'subtracted' if mf_subtract else 'kept'}"),
            "m_drawn": [int(sy.M) for sy in systems],
            "completed": int(st["completed"]), "failed": int(st["failed"]),
            "p50_block_ms": round(st["p50_ms"], 3), "p99_block_ms": round(st["p99_ms"], 3),
            "walker_steps_per_s": round(st["walker_steps"] / st["elapsed_s"], 1),
            "offered_walker_steps_per_s": round(offered / max(window, 1e-9), 1),
            "elapsed_s": round(st["elapsed_s"], 3), "max_active_seen": int(st["max_active_seen"]),
            "failures": failures[:4]}


def _blocks(s, precision, n_blocks, **kw):
    """Mean device ms per 20-step block after one warm-up block, and the
    per-kernel-group totals over the timed blocks."""
    import torch
    from paper_1804_03310_gb300 import Afqmc, KERNEL_IDS
    stream = torch.cuda.Stream()
    ctx = Afqmc.from_system(s, precision=precision, stream=stream.cuda_stream, **kw)
    ctx.afqmc_propagate(BLOCK)
    stream.synchronize()
    ctx.afqmc_set_kernel_timing(True)
    total = 0.0
    for _ in range(n_blocks):
        a = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ctx.afqmc_propagate(BLOCK)
        e.record(stream)
        e.synchronize()
        total += a.elapsed_time(e)
    ks = {k: ctx.afqmc_kernel_stats(k) for k in KERNEL_IDS}
    ctx.close()
    return total / n_blocks, {k: round(v["total_ms"], 3) for k, v in ks.items() if v["launches"]}


def islands_leg(s, precision, value):
    """The bench workload with FP64 arithmetic islands beside the default
    FP32 arithmetic there: fp64_islands = 2, the QR alone in FP64 (the form
    the TM-atom configuration states: FP64 only for the orthonormalisation,
    the log-determinants and the weights), and fp64_islands = 1, the small
    inverse as well."""
    import torch
    from paper_1804_03310_gb300 import Afqmc
    out = {}
    for mode, key in ((2, "qr"), (1, "qr_and_inverse")):
        stream = torch.cuda.Stream()
        ctx = Afqmc.from_system(s, precision=precision, fp64_islands=mode,
                                stream=stream.cuda_stream)
        ctx.afqmc_propagate(BLOCK)
        stream.synchronize()
        total = 0.0
        n = 3
        for _ in range(n):
            a = torch.cuda.Event(enable_timing=True)
            e = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            ctx.afqmc_propagate(BLOCK)
            e.record(stream)
            e.synchronize()
            total += a.elapsed_time(e)
        ctx.close()
        v = s.n_walkers * BLOCK * n / (total / 1e3)
        out[key] = {"fp64_islands": mode, "value": round(v, 1), "unit": METRIC,
                    "ms_per_block": round(total / n, 3),
                    "ratio_to_default": round(v / value, 3)}
    return out


def batch_leg(precision, n_blocks=4):
    """Multi-system batching: four systems of uneven M, N, n_chol and walker
    counts advanced by afqmc_batch_propagate (one graph launch per 20-step
    block, every member a branch of it) against the same systems advanced
    one after another on one stream."""
    import torch
    from synth import make_system
    from paper_1804_03310_gb300 import Afqmc, Batch
    shapes = [(24, 8, 8, 100, 512), (40, 10, 9, 180, 384), (60, 20, 20, 260, 256),
              (90, 15, 15, 400, 256)]
    systems = [make_system(f"batch_{k}", M=M, n_up=nu, n_dn=nd, n_chol=G, ham_seed=10 + k,
                           l_kind="dense", l_sigma=0.05 * math.sqrt(10.0 / M), trial="eig",
                           dtau=0.005, n_walkers=W, seed=10 + k, ortho_every=2,
                           measure_every=BLOCK, pc_every=BLOCK, run_id=k)
               for k, (M, nu, nd, G, W) in enumerate(shapes)]
    ws = sum(s.n_walkers for s in systems) * BLOCK * n_blocks

    def make():
        return [Afqmc.from_system(s, precision=precision) for s in systems]

    # one after another
    ctxs = make()
    for c in ctxs:
        c.afqmc_propagate(BLOCK)
        c.afqmc_synchronize()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(n_blocks):
        for c in ctxs:
            c.afqmc_propagate(BLOCK)
    for c in ctxs:
        c.afqmc_synchronize()
    seq = time.perf_counter() - t0
    for c in ctxs:
        c.close()
    # batched
    ctxs = make()
    b = Batch(ctxs, BLOCK)
    b.afqmc_batch_propagate(1)
    b.afqmc_batch_synchronize()
    t0 = time.perf_counter()
    b.afqmc_batch_propagate(n_blocks)
    b.afqmc_batch_synchronize()
    bat = time.perf_counter() - t0
    launches = b.afqmc_batch_launches()
    b.close()
    for c in ctxs:
        c.close()
    return {"workload": "; ".join(f"M={M} N={nu}+{nd} n_chol={G} W={W}"
                                  for (M, nu, nd, G, W) in shapes) + f", {precision}",
            "blocks": n_blocks, "batched_value": round(ws / bat, 1),
            "sequential_value": round(ws / seq, 1), "unit": METRIC,
            "speedup": round(seq / bat, 3), "graph_launches": int(launches)}


def ndet_leg(precision, ndets=(1, 10, 50, 200, 500)):
    """Cost of the multi-determinant step against the number of
    determinants (the shape of the paper's N_det study, Sec. III): the
    multi-determinant workload's system with the trial truncated or extended
    to N_det determinants, one 20-step block timed after a warm-up block."""
    from synth import config_c4
    out = []
    for nd in ndets:
        s = config_c4(n_det=nd).replace(measure_every=BLOCK, pc_every=BLOCK, ortho_every=2)
        try:
            ms, _ = _blocks(s, precision, 1)
        except Exception as e:   # e.g. a trial too large for the on-chip energy kernel
            out.append({"n_det": nd, "error": str(e)[:160]})
            continue
        out.append({"n_det": nd, "ms_per_block": round(ms, 3),
                    "value": round(s.n_walkers * BLOCK / (ms / 1e3), 1)})
    base = out[0].get("ms_per_block")
    for r in out:
        if base and "ms_per_block" in r:
            r["cost_vs_1_det"] = round(r["ms_per_block"] / base, 3)
    return {"workload": "M=80 N=10+10 n_chol=400 W=1024, " + precision, "unit": METRIC,
            "points": out}


def cs_leg(precision, W=2048, n_steps=800):
    """Correlated sampling (Sec. V): the ionisation energy E(cation) -
    E(neutral) of the 10-orbital system (5+5 and 5+4 electrons, same
    Hamiltonian and orbitals, comb off, energy every 10 steps) with shared
    field paths (equal seed and Philox tag) against independent paths. The
    reblocked standard error of the difference series is the figure of
    merit: the variance ratio is the factor of sampling time correlated
    sampling saves at equal error bar."""
    import numpy as np
    from synth import make_system
    from paper_1804_03310_gb300 import Afqmc
    kw = dict(M=10, n_chol=40, ham_seed=0, l_kind="dense", l_sigma=0.05, trial="eig",
              dtau=0.01, n_walkers=W, seed=17, ortho_every=5, measure_every=10, pc_every=0)
    out = {}
    t0 = time.perf_counter()
    for label, ids in (("correlated", (3, 3)), ("independent", (3, 4))):
        e = []
        for nd, rid in ((5, ids[0]), (4, ids[1])):
            sy = make_system("cs", n_up=5, n_dn=nd, run_id=rid, **kw)
            with Afqmc.from_system(sy, precision=precision) as ctx:
                ctx.afqmc_propagate(n_steps)
                e.append(ctx.afqmc_energy_history()[:, 1])
        d = (e[1] - e[0])[10:]
        out[label] = {"ip_ha": round(float(np.mean(d)), 6),
                      "stderr_ha": round(reblocked_error(d), 7)}
    r = (out["independent"]["stderr_ha"] / max(out["correlated"]["stderr_ha"], 1e-300)) ** 2
    return {"workload": (f"M=10 N=5+5 / 5+4 n_chol=40 W={W} dtau=0.01, {n_steps} steps, "
                         f"comb off, {precision}"),
            **out, "variance_ratio": round(r, 2),
            "seconds": round(time.perf_counter() - t0, 2)}


def reblocked_error(x):
    """Standard error of a serially correlated series (blocking analysis)."""
    import numpy as np
    x = np.asarray(x, dtype=np.float64)
    best = 0.0
    while len(x) >= 4:
        best = max(best, float(np.std(x, ddof=1) / np.sqrt(len(x))))
        n = len(x) // 2 * 2
        x = 0.5 * (x[0:n:2] + x[1:n:2])
    return best


def precisions_leg(s, n_blocks=3):
    """The bench workload in each reduced precision (same seed): walker-steps/s
    per mode; the energy deviation of each mode is in fp64_gpu."""
    out = {}
    for prec in ("fp32", "tf32x3", "bf16x3"):
        ms, _ = _blocks(s, prec, n_blocks)
        out[prec] = {"value": round(s.n_walkers * BLOCK / (ms / 1e3), 1),
                     "ms_per_block": round(ms, 3)}
    return out


def shapes_leg(precision):
    """The other workload shapes of the scope, each in its stated arithmetic
    and in FP64 on the GPU (same walkers and seed): the TM-atom shape
    (M = 150, BF16 hi + lo arithmetic; its shell-structured Cholesky vectors
    take the block-diagonal path, timed beside the dense path with the
    operator streamed by TMA) and the multi-determinant shape (200
    determinants, batched SMW ratios) in the bench's precision."""
    from synth import CONFIGS
    out = {}
    for name, prec in (("c3", "bf16x3"), ("c4", precision)):
        s = CONFIGS[name]().replace(measure_every=BLOCK, pc_every=BLOCK, ortho_every=2)
        ms, kms = _blocks(s, prec, 2)
        ms64, _ = _blocks(s, "fp64", 1)
        v = s.n_walkers * BLOCK / (ms / 1e3)
        v64 = s.n_walkers * BLOCK / (ms64 / 1e3)
        out[name] = {"workload": describe(s), "precision": prec,
                     "value": round(v, 1), "unit": METRIC, "ms_per_block": round(ms, 3),
                     "fp64_value": round(v64, 1), "speedup": round(v / v64, 2),
                     "kernels_ms_2_blocks": kms}
        if name == "c3":   # the dense path on the same inputs
            msd, kmsd = _blocks(s, prec, 2, block_sparse=2)
            out[name]["dense"] = {"value": round(s.n_walkers * BLOCK / (msd / 1e3), 1),
                                  "ms_per_block": round(msd, 3), "kernels_ms_2_blocks": kmsd,
                                  "block_sparse_speedup": round(msd / ms, 2)}
    return out


def weight_forms_leg(s, precision, n_steps=200):
    """The weight forms and the mean-field subtraction (Sec. II) on the bench
    workload: walker-steps/s of each (two timed blocks; the local-energy form
    evaluates the energy every step), the paired energy deviation of each
    against the FP64 GPU path with the same draws (comb off, n_steps steps,
    one measurement every 20), and the walkers the phaseless cut leaves
    alive after 60 steps at dt = 0.02 (comb off) with and without the
    subtraction."""
    import numpy as np
    from paper_1804_03310_gb300 import Afqmc
    out = {}
    for mode, mf in ((0, 0), (0, 1), (1, 0), (1, 1)):
        key = f"{'local_energy' if mode else 'hybrid'}{'_mf' if mf else ''}"
        v = s.replace(weight_mode=mode, mf_subtract=mf)
        ms, _ = _blocks(v, precision, 2)
        r = {"value": round(s.n_walkers * BLOCK / (ms / 1e3), 1), "ms_per_block": round(ms, 3)}
        if mode or mf:
            p = v.replace(pc_every=0, measure_every=20)
            e = {}
            for prec in ("fp64", precision):
                with Afqmc.from_system(p, precision=prec) as ctx:
                    ctx.afqmc_propagate(n_steps)
                    e[prec] = ctx.afqmc_energy_history()[:, 1]
                    w, _ = ctx.afqmc_weights()
                    if prec == "fp64":   # how far the comb-off population has degenerated
                        r["end_killed"] = int(np.count_nonzero(w <= 0))
                        r["end_top_weight_share"] = round(float(w.max() / w.sum()), 4)
            d = (e[precision] - e["fp64"]) * 1e3
            r["paired_max_abs_mHa"] = round(float(np.max(np.abs(d))), 6)
            r["paired_median_abs_mHa"] = round(float(np.median(np.abs(d))), 6)
            r["e_fp64_last"] = round(float(e["fp64"][-1]), 6)
        out[key] = r
    alive = {}
    for mf in (0, 1):
        p = s.replace(pc_every=0, measure_every=0, dtau=0.02, mf_subtract=mf)
        with Afqmc.from_system(p, precision=precision) as ctx:
            ctx.afqmc_propagate(60)
            w, _ = ctx.afqmc_weights()
        alive["mean_field_subtracted" if mf else "plain"] = int(np.count_nonzero(w > 0))
    out["alive_after_60_steps_dt0.02"] = alive
    out["paired_steps"] = n_steps
    return out


def dtype_of(precision):
    return {"fp64": "f64", "fp32": "f32", "tf32": "tf32", "tf32x3": "tf32x3",
            "bf16x3": "bf16x3"}[precision]


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        if rank != 0:
            return 0
        return reference_arm(args)
    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    s, total_ms, launches, kstats, clocks, hist, e2e = run_ours(args, rank, world)
    if rank != 0:
        return 0
    peaks, src = load_peaks()
    fused = kstats.pop("_taylor_fused", None)
    value = whole_job_value(s.n_walkers * BLOCK * args.steps, world, total_ms)
    line = {
        "metric": METRIC, "value": round(value, 1), "unit": METRIC, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(total_ms / args.steps, 4),
        "ms_per_imaginary_step": round(total_ms / args.steps / BLOCK, 5),
        "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": dtype_of(args.precision),
        "data": "synthetic (seeded Hamiltonian and trial of the workload's shape)",
        "config": {"workload": describe(s), "precision": args.precision,
                   "step": (f"one bench step = one block of {BLOCK} imaginary-time steps "
                            "(ortho every 2, energy + comb at the end); ms_per_step is per "
                            "block, ms_per_imaginary_step per imaginary-time step"),
                   "l2": "flushed (256 MB write) between timed iterations",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "gpu_launches": int(launches),
        "roofline": roofline_for(kstats, args.precision, peaks, src, s, args.workload, fused),
        "kernels_ms": {k: round(v["total_ms"], 3) for k, v in kstats.items()},
        "clocks": clocks,
        "energy_last": float(hist[-1][1]) if len(hist) else None,
    }
    if e2e:
        line["e2e"] = e2e

    def leg(key, fn):
        # an optional leg that fails reports its error instead of ending the run
        try:
            line[key] = fn()
        except Exception as e:  # noqa: BLE001
            line[key] = {"error": f"{type(e).__name__}: {str(e)[:200]}"}

    if not args.no_fp64_compare and world == 1 and args.precision != "fp64":
        def f64_leg():
            f64 = fp64_compare(args, s, hist)
            f64["speedup"] = round(value / f64["value"], 2)
            return f64
        leg("fp64_gpu", f64_leg)
    if not args.no_serving and world == 1:
        leg("serving", lambda: serving_leg(args.precision))
    if not args.no_shapes and world == 1 and args.precision != "fp64":
        leg("shapes", lambda: shapes_leg(args.precision))
        leg("precisions", lambda: precisions_leg(s))
        leg("fp64_islands", lambda: islands_leg(s, args.precision, value))
        leg("batch", lambda: batch_leg(args.precision))
        leg("ndet_sweep", lambda: ndet_leg(args.precision))
        leg("correlated_sampling", lambda: cs_leg(args.precision))
        leg("weight_forms", lambda: weight_forms_leg(s, args.precision))
    if not args.no_cpu_baseline and world == 1:
        v, cores, sample = cpu_oracle(args.workload)
        line["cpu_baseline"] = {"value": round(v, 2), "unit": METRIC, "cores": cores,
                                "kind": "oracle", "sample": sample}
    print(json.dumps(line))
    return 0


def reference_arm(args):
    from synth import CONFIGS
    s = CONFIGS[args.workload]()
    vals = []
    t0 = time.perf_counter()
    for _ in range(args.warmup + args.steps):
        v, cores, sample = cpu_oracle(args.workload, budget_s=8.0)
        vals.append(v)
    wall = time.perf_counter() - t0
    timed = vals[args.warmup:]
    value = sum(timed) / len(timed)
    line = {"metric": METRIC, "value": round(value, 2), "unit": METRIC, "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(wall / max(1, len(vals)) * 1e3, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": describe(s), "precision": "fp64 (CPU oracle)"},
            "cpu_baseline": {"value": round(value, 2), "unit": METRIC, "cores": cores,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": round(value, 2), "unit": METRIC, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


if __name__ == "__main__":
    sys.exit(main())
