"""Benchmark of the spectral point-mass filter hot path on GB300.

Workload (default, --workload c4): 4096 independent 2-D filters, each with its
own seeded stable A and diagonal Q, axis sizes drawn from {32, 48, 64, 96,
128}, linear measurement z = x + v (R = 0.1^2 I), dt = 0.05.  One step = one
epoch of every filter (Bayes measurement update + spectral time update), one
graph-replayed launch of the batched fused kernel.  --workload c2 | c3 | c5 |
c6 select the 128 x 128 oscillator, the 96^3 bearing filter, the serving
population and the 4-D coordinated turn.

metric : grid-point updates per second (points x epochs / device time)
value  : the tensor-core path at the chosen precision (default BF16X6, the
         split-BF16 format within 1e-5, for the 2-D workloads c2 / c4 / c5;
         FP16X3 for the 3-D and 4-D ones), inputs resident in HBM, L2 flushed
         between timed steps
e2e    : the same through the public C-ABI call with the measurements taken
         from host memory and the moments read back every step
fp64_gpu : the plain float64 GPU path on the same workload (comparator)
cpu_baseline : the float64 oracle on a bounded sample, on the host cores,
         with the parity of the same sample on the GPU

Multi-GPU: filters are independent, so N ranks run N replicas ("replicas
only"), barriers and a max-over-ranks timing, no data-path collective.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "grid-pt updates/s vs plain FP64 GPU at ≤1e-5 L1 err; p50/p99 filter latency"
UNIT = "grid-pt updates/s"


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if ws > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("gloo", rank=rank, world_size=ws)
        pg = dist
    return ws, rank, local, pg


def _barrier(pg):
    if pg is not None:
        pg.barrier()


def _max_over_ranks(pg, x):
    if pg is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


_SCENARIOS = {
    "c2": "w.c2_scenario(epochs={e})",
    "c2small": "w.c2_scenario(N=(64, 64), epochs={e})",
    "c3": "w.c3_scenario(epochs={e})",
    "c6": "w.c6_scenario(epochs={e})",
}


def _scenario_expr(name, epochs):
    """Python expression (over `import workloads as w`) that builds the workload
    with at least `epochs` seeded epochs (the trajectory continues past the
    configured count when a run needs more steps)."""
    if name not in _SCENARIOS:
        raise SystemExit(f"unknown workload {name}")
    floor = 20 if name == "c6" else 50
    return _SCENARIOS[name].format(e=max(floor, epochs))


def _scenario(name, epochs=50):
    import workloads as w   # noqa: F401  (used by the expression)
    return eval(_scenario_expr(name, epochs))


def leg_epochs(workload, steps, warmup):
    """Epochs of the seeded scenario that each leg of a single-filter bench
    run consumes (timed steps after the warm-up, the end-to-end loop, the
    float64 comparator, the oracle parity sample); the scenario is built with
    the largest of them, so every leg indexes inside it."""
    nx = {"c2": 2, "c2small": 2, "c3": 3, "c6": 4}[workload]
    f64 = max(3, min(steps // 4, {2: 40, 3: 5, 4: 10}[nx]))
    return {"timed": warmup + steps, "e2e": 3 + steps, "fp64": warmup + f64,
            "parity": {2: 60, 3: 10, 4: 2}[nx]}


def _launch_names(sc):
    return "k_fused2d" if sc.cfg.nx == 2 else "k_slices_fwd+k_lines_axis0+k_slices_inv"


# DRAM bytes (read + write) per launch of the timed kernel, from one ncu capture
# of the current kernel (profiles/): the 128 x 128 fused kernel, and the batch
# kernel per grid point (captured on 2048 filters, scaled by the points).
# Bytes a served request uploads: its StepItem (slot, flags, z[3]) and the
# TimeConsts of its time update (32 + 5 x 16 x 8 + 64 x 10 x 8 + 5 x 8 bytes).
STEP_ITEM_BYTES = 32
TIME_CONSTS_BYTES = 5832
TRAFFIC_C2 = 345344.0
# DRAM bytes per grid point of one C4 epoch (the four kernels' dram__bytes_read
# + dram__bytes_write, one ncu capture of the full batch), per format; absent
# where not captured for the current kernels
TRAFFIC_C4_PER_POINT = {"bf16x6": 13.373, "fp16x3": 13.434}
BATCH_KERNEL = "k_front2d + k_fused2d_planned<128|96|64> (one graph per epoch)"


def _flops_per_step(N):
    """Algorithmic transform flops of one epoch: forward + inverse per axis, 2 N_m flops per point each."""
    P = 1
    for n in N:
        P *= n
    return 4.0 * P * sum(N)


# Method variants of the single-filter workloads (--psi, --realign): the
# diffusion multiplier (Euler product or exact-in-time) and the fill of a
# re-aligned frame (multilinear or band-limited shear passes, n_x = 2).
MODES = {"psi": "euler", "realign": "multilinear"}


def _apply_modes(sc):
    sc.cfg.realign_mode = MODES["realign"]
    return sc


def time_gpu(sc, precision, steps, warmup, flush_mb=512):
    """Device time of `steps` epochs (CUDA events around each pmf_step, L2 flushed between)."""
    import torch
    from paper_2412_07240_gb300 import Filter
    f = Filter(sc.cfg, precision=precision, psi_mode=MODES["psi"])
    assert len(sc.z) >= warmup + steps
    flush = torch.empty(flush_mb * (1 << 20) // 4, dtype=torch.float32, device="cuda")
    K = len(sc.z)
    for k in range(warmup):
        f.step(sc.meas, sc.z[k], sc.dt)
    f.sync()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    l0 = f.launches
    for k in range(steps):
        flush.fill_(float(k))
        ev[k][0].record()
        f.step(sc.meas, sc.z[warmup + k], sc.dt)
        ev[k][1].record()
    torch.cuda.synchronize()
    f.sync()
    launches = f.launches - l0
    ms = [a.elapsed_time(b) for a, b in ev]
    return f, ms, launches


def time_e2e(sc, precision, steps):
    """Wall time of steps through the public API: measurement from host, moments read back."""
    import torch
    from paper_2412_07240_gb300 import Filter
    f = Filter(sc.cfg, precision=precision, psi_mode=MODES["psi"])
    for k in range(3):
        f.step(sc.meas, sc.z[k], sc.dt)
        f.moments()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(3, 3 + steps):
        f.step(sc.meas, sc.z[k], sc.dt)
        f.moments()
    t1 = time.perf_counter()
    return (t1 - t0) * 1e3 / steps


def oracle_sample(name, epochs, threads=1, total=None):
    """Run the float64 oracle on the first `epochs` epochs of workload `name`
    (a scenario of `total` epochs, default `epochs`) in a single-threaded
    subprocess."""
    env = dict(os.environ)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[v] = str(threads)
    code = f"""
import json, sys, time
sys.path.insert(0, {ROOT!r})
import numpy as np
import workloads as w
from oracle.filter import OracleFilter
sc = {_scenario_expr(name, max(epochs, total or 0))}
sc.cfg.realign_mode = {MODES["realign"]!r}
f = OracleFilter(sc.cfg, psi_mode={MODES["psi"]!r})
t = time.perf_counter()
for k in range({epochs}):
    f.meas_update(sc.meas, sc.z[k])
    f.time_update(sc.dt)
dt = time.perf_counter() - t
np.save(sys.argv[1], f.P)
print(json.dumps({{"seconds": dt, "epochs": {epochs}}}))
"""
    import tempfile
    with tempfile.TemporaryDirectory() as td:
        out = os.path.join(td, "p.npy")
        r = subprocess.run([sys.executable, "-c", code, out], env=env, capture_output=True, text=True,
                           timeout=600)
        if r.returncode != 0:
            raise RuntimeError(r.stderr)
        res = json.loads(r.stdout.strip().splitlines()[-1])
        import numpy as np
        res["P"] = np.load(out)
    return res


def _oracle_env():
    env = dict(os.environ)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[v] = "1"
    return env


def _oracle_proc(code, timeout=900):
    """Run oracle code in a single-threaded subprocess; its last stdout line is JSON."""
    r = subprocess.run([sys.executable, "-c", code], env=_oracle_env(), capture_output=True, text=True,
                       timeout=timeout)
    if r.returncode != 0:
        raise RuntimeError(r.stderr)
    return json.loads(r.stdout.strip().splitlines()[-1])


def _oracle_par(code, nproc, timeout=900):
    """Run `code` as `nproc` concurrent single-threaded processes, one per host
    core, on disjoint shares of a sample of independent filters.  Child r gets
    "r nproc" as argv, sets its share up, prints "ready", waits for one line on
    stdin, runs and prints a JSON line with "points", "t0" and "t1" (wall
    clock around its compute).  Returns the summed points, the span from the
    first start to the last end, and the per-child results."""
    procs = [subprocess.Popen([sys.executable, "-c", code, str(r), str(nproc)], env=_oracle_env(),
                              stdin=subprocess.PIPE, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True)
             for r in range(nproc)]
    try:
        for p in procs:
            if p.stdout.readline().strip() != "ready":
                raise RuntimeError(p.communicate(timeout=timeout)[1])
        for p in procs:
            p.stdin.write("go\n")
            p.stdin.flush()
        res = []
        for p in procs:
            out, err = p.communicate(timeout=timeout)
            if p.returncode != 0:
                raise RuntimeError(err)
            res.append(json.loads(out.strip().splitlines()[-1]))
    finally:
        for p in procs:
            if p.poll() is None:
                p.kill()
    span = max(r["t1"] for r in res) - min(r["t0"] for r in res)
    return {"points": sum(r["points"] for r in res), "seconds": span, "children": res}


_SHARE_SRC = """
def _share(work, nproc):
    # work of a filter ~ P * sum(N) (one dense transform per axis); largest
    # first, each unit to the least loaded process (ties: lowest rank)
    load, owner = [0] * nproc, [0] * len(work)
    for u in sorted(range(len(work)), key=lambda u: (-work[u], u)):
        r = min(range(nproc), key=lambda q: (load[q], q))
        owner[u] = r
        load[r] += work[u]
    return owner
"""


def _oracle_cores(n_units):
    return max(1, min(os.cpu_count() or 1, n_units))


def c4_sample_ids(count, nsample=256):
    """Indices of the filters the oracle samples from the batch (all sizes)."""
    import numpy as np
    return np.linspace(0, count - 1, min(nsample, count)).astype(int)


C4_CHECKPOINTS = (8, 25, 50, 100)


def oracle_c4_sample(count, checkpoints=C4_CHECKPOINTS, nsample=256, outdir=None):
    """The float64 oracle on `nsample` filters spread over the batch (all sizes),
    max(checkpoints) epochs each (the workload's whole horizon), the filters
    dealt to one single-threaded process per host core: grid-point updates and
    the wall span.  With `outdir`, each child also saves the weights and frame
    of its filters after each checkpoint epoch there (outside the timed span)
    for the parity comparison."""
    epochs = max(checkpoints)
    code = f"""
import json, sys, time
sys.path.insert(0, {ROOT!r})
import numpy as np
import workloads as w
from oracle.filter import OracleFilter
rank, nproc = int(sys.argv[1]), int(sys.argv[2])
{_SHARE_SRC}cfgs, meas, dt, truth, z = w.c4_batch(count={count}, epochs={epochs})
idx = np.linspace(0, len(cfgs) - 1, min({nsample}, len(cfgs))).astype(int)
owner = _share([int(np.prod(cfgs[i].N)) * sum(cfgs[i].N) for i in idx], nproc)
idx = [i for i, o in zip(idx, owner) if o == rank]
print("ready", flush=True)
sys.stdin.readline()
pts, t0, done, failed = 0, time.time(), [], []
for i in idx:
    f = OracleFilter(cfgs[i])
    k = 0
    try:
        for k in range({epochs}):
            f.meas_update(meas, z[i, k])
            f.time_update(dt)
            if k + 1 in {tuple(checkpoints)!r}:
                done.append((i, k + 1, f.P.copy(), f.c.copy(), f.M.copy()))
        k = {epochs}
    except Exception:     # the oracle cannot carry this filter on (degenerate normaliser or frame)
        failed.append(int(i))
    pts += int(np.prod(cfgs[i].N)) * k
t1 = time.time()
if {outdir!r} is not None:
    for i, k, P, c, M in done:
        np.savez(f"{outdir}/{{i}}_{{k}}.npz", P=P, c=c, M=M)
print(json.dumps({{"points": pts, "t0": t0, "t1": t1, "filters": len(idx), "failed": failed}}))
"""
    cores = _oracle_cores(nsample)
    t = _oracle_par(code, cores)
    t.update(filters=min(nsample, count), epochs=epochs, cores=cores,
             failed=sorted(i for r in t["children"] for i in r.get("failed", [])))
    return t


def oracle_c5_sample(n_filters, per_dim=(30, 20, 5), reqs=5):
    """The float64 oracle on the first requests of a few serving filters of each
    dimension (same filter population as the served one), the filters dealt
    round-robin to one single-threaded process per host core."""
    code = f"""
import json, sys, time
sys.path.insert(0, {ROOT!r})
import numpy as np
import workloads as w
from oracle.filter import OracleFilter
rank, nproc = int(sys.argv[1]), int(sys.argv[2])
{_SHARE_SRC}wl = w.c5_serving(n_filters={n_filters}, duration=0.3, seed=5)
picks = []
for d, want in zip((1, 2, 3), {per_dim!r}):
    got = 0
    for i, c in enumerate(wl.cfgs):
        if c.nx != d or got == want:
            continue
        r = np.nonzero(wl.ids == i)[0][:{reqs}]
        if len(r) < {reqs}:
            continue
        picks.append((i, r))
        got += 1
owner = _share([int(np.prod(wl.cfgs[i].N)) * sum(wl.cfgs[i].N) * len(r) for i, r in picks], nproc)
print("ready", flush=True)
sys.stdin.readline()
pts, t0 = 0, time.time()
for (i, r), o in zip(picks, owner):
    if o != rank:
        continue
    c = wl.cfgs[i]
    f = OracleFilter(c)
    for q in r:
        f.meas_update(wl.meas[i], wl.z[q, :c.nx])
        f.time_update(min(float(wl.taus[q]), 0.6))
    pts += int(np.prod(c.N)) * len(r)
print(json.dumps({{"points": pts, "t0": t0, "t1": time.time(), "filters": len(picks)}}))
"""
    cores = _oracle_cores(sum(per_dim))
    t = _oracle_par(code, cores)
    t.update(filters=list(per_dim), requests_each=reqs, cores=cores)
    return t


def run_reference(args, ws, rank, pg):
    """The oracle arm: float64 oracle on the host cores, bounded sample per step."""
    if rank != 0:
        return
    if args.workload in ("c4", "c5"):
        if args.workload == "c4":
            t = oracle_c4_sample(args.count)
            name, sample = f"c4_batch_{args.count}x2d_mixed", (f"{t['filters']} filters spread over the batch, "
                                                                f"{t['epochs']} epochs each, one single-threaded "
                                                                f"process per core")
        else:
            n = args.count if args.count != 4096 else 10000
            t = oracle_c5_sample(n)
            name, sample = f"c5_serving_{n}_mixed", (f"first {t['requests_each']} requests of "
                                                     f"{t['filters']} 1-D/2-D/3-D filters, one single-threaded "
                                                     f"process per core")
        value = t["points"] / t["seconds"]
        ms = None
        if args.workload == "c4":
            # one epoch of the whole workload at the sampled rate
            import workloads as w
            cfgs = w.c4_batch(count=args.count, epochs=1)[0]
            ms = sum(c.N[0] * c.N[1] for c in cfgs) / value * 1e3
        line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic (seeded filters and measurements)",
                "config": {"workload": name, "parallelism": "replicas",
                           "ms_per_step": "one epoch of the whole workload at the sampled rate"
                           if ms is not None else "no per-step figure (request replay)"},
                "cpu_baseline": {"value": value, "unit": UNIT, "cores": t["cores"], "kind": "oracle",
                                 "sample": sample},
                "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return
    sc = _apply_modes(_scenario(args.workload, args.warmup + args.steps))
    P = 1
    for n in sc.cfg.N:
        P *= n
    t = oracle_sample(args.workload, args.warmup + args.steps)
    per = t["seconds"] / t["epochs"]
    value = P / per
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded truth and measurements)",
            "config": {"workload": sc.name, "grid": list(sc.cfg.N), "epochs_timed": t["epochs"],
                       "parallelism": "replicas"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{t['epochs']} epochs of the {sc.name} filter, single thread"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# tensor-core products per K step of each format (split planes)
MMA_PRODUCTS = {"bf16x6": 6, "fp16x3": 3, "bf16x3": 3, "tf32": 1}
# dense tensor rate of each format relative to bf16 (nominal figures)
MMA_RATE = {"bf16x6": 1.0, "fp16x3": 1.0, "bf16x3": 1.0, "tf32": 1.1 / 2.25}


def executed_mma_flops(cfgs, precision):
    """Tensor-core flops one epoch of the batch issues.  Every GEMM stage is a
    128 (lines, unused ones included) x N x K product per split-format
    product, N = K = the axis size; the GEMM form runs six stages per filter
    (regrid, Hartley transform and inverse along each axis), the FFT form the
    two regrid stages only.  The regrid GEMMs are counted for every filter."""
    from paper_2412_07240_gb300 import _binding, lib_path
    path = os.path.join(os.path.dirname(lib_path()), "autotune_2d.json")
    rec = json.load(open(path)) if os.path.exists(path) else {}
    code = _binding.PREC[precision]
    env = os.environ.get("PMF_2D_FORM")
    total = 0.0
    for c in cfgs:
        e = rec.get(f"2d:{c.N[0]}x{c.N[1]}:{code}")
        fft = env == "fft" if env in ("gemm", "fft") else bool(e is not None and e["form"])
        stages_per_axis = 1 if fft else 3
        total += MMA_PRODUCTS[precision] * 2.0 * 128 * stages_per_axis * (c.N[0] ** 2 + c.N[1] ** 2)
    return total


def transform_forms(cfgs, precision):
    """Filters per Hartley form (tensor-core GEMM or shared-memory FFT), from the
    2-D autotuner's record beside the library, and the record's entries."""
    from paper_2412_07240_gb300 import _binding, lib_path
    path = os.path.join(os.path.dirname(lib_path()), "autotune_2d.json")
    rec = json.load(open(path)) if os.path.exists(path) else {}
    code = _binding.PREC[precision]
    counts, used = {"gemm": 0, "fft": 0}, {}
    for c in cfgs:
        key = f"2d:{c.N[0]}x{c.N[1]}:{code}"
        e = rec.get(key)
        if os.environ.get("PMF_2D_FORM") in ("gemm", "fft"):
            counts[os.environ["PMF_2D_FORM"]] += 1
        elif e is None:
            counts["gemm"] += 1           # sizes without an FFT form
        else:
            counts["fft" if e["form"] else "gemm"] += 1
            used[key] = e
    return {"filters": counts, "autotune": used}


def bench_batch(args, ws, rank, pg):
    """The 4096-filter batch: one fused launch per epoch over all filters."""
    import numpy as np
    import torch
    import workloads as w
    from paper_2412_07240_gb300 import Batch, Filter
    epochs = args.warmup + args.steps + 1
    cfgs, meas, dt, truth, z = w.c4_batch(count=args.count, epochs=epochs)
    P = np.array([c.N[0] * c.N[1] for c in cfgs], dtype=np.int64)
    ids = np.arange(len(cfgs))
    b = Batch(cfgs, [meas] * len(cfgs), precision=args.precision)
    flush = torch.empty(512 * (1 << 20) // 4, dtype=torch.float32, device="cuda")
    for k in range(args.warmup):
        b.step(ids, z[:, k], dt)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    l0 = b.launches
    _barrier(pg)
    with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        for k in range(args.steps):
            flush.fill_(float(k))
            ev[k][0].record()
            b.step(ids, z[:, args.warmup + k], dt)
            ev[k][1].record()
        torch.cuda.synchronize()
    launches = b.launches - l0
    ms = [a.elapsed_time(c) for a, c in ev]
    t_ms = _max_over_ranks(pg, sum(ms))
    value = ws * P.sum() * args.steps / (t_ms * 1e-3)
    bad = int((b.status() != 0).sum())
    # end to end: measurements from host, moments back, every epoch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ne = min(20, args.steps)
    for k in range(ne):
        b.step(ids, z[:, args.warmup + k], dt)
        b.moments(strict=False)
    e2e_ms = (time.perf_counter() - t0) * 1e3 / ne
    # plain float64 per-filter path on a subset, scaled by points
    sub = ids[:: max(1, len(ids) // 64)]
    fs = [Filter(cfgs[i], precision="fp64") for i in sub]
    for f, i in zip(fs, sub):
        f.step(meas, z[i, 0], dt)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for f, i in zip(fs, sub):
        f.step(meas, z[i, 1], dt)
    e1.record()
    torch.cuda.synchronize()
    fp64_rate = P[sub].sum() / (e0.elapsed_time(e1) * 1e-3)
    flops = float(sum(4.0 * c.N[0] * c.N[1] * (c.N[0] + c.N[1]) for c in cfgs))
    kernel_ms = float(np.mean(ms))
    peaks, src = _peaks()
    ach = flops / (kernel_ms * 1e-3) / 1e12
    ex_flops = executed_mma_flops(cfgs, args.precision)
    ex_ach = ex_flops / (kernel_ms * 1e-3) / 1e12
    ex_peak = peaks.get("bf16_tflops") * MMA_RATE[args.precision]
    # the epoch's algorithmic intensity (flops / 8 B per point) is below the
    # bf16 ridge, so the HBM roofline binds: float32 weights in and out
    alg_bytes = 8.0 * float(P.sum())
    gbs = alg_bytes / (kernel_ms * 1e-3) / 1e9
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": f"f32 ({args.precision} split GEMMs)",
            "data": "synthetic (seeded truth and measurements)",
            "config": {"workload": f"c4_batch_{len(cfgs)}x2d_mixed", "points": int(P.sum()),
                       "precision": args.precision, "l2": "flushed between timed steps",
                       "parallelism": f"replicas x{ws}"},
            "e2e": {"value": ws * P.sum() / (e2e_ms * 1e-3), "unit": UNIT,
                    # copied per filter: a 32-byte step item (slot, flags, z[3]) and a
                    # 4-byte id in, a 64-byte gather record (mean, cov, status, pad) out
                    "h2d_bytes_per_step": int(len(cfgs) * 36), "d2h_bytes_per_step": int(len(cfgs) * 64),
                    "ms_per_step": e2e_ms},
            "gpu_launches": int(launches),
            "fp64_gpu": {"value": fp64_rate, "unit": UNIT, "filters_timed": int(len(sub))},
            "latency_ms": {"p50": float(np.percentile(ms, 50)), "p99": float(np.percentile(ms, 99))},
            "degenerate_filters": bad,
            "transform_forms": transform_forms(cfgs, args.precision),
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": peaks.get("hbm_gbs"), "unit": "GB/s",
                         "frac": gbs / peaks.get("hbm_gbs"),
                         "traffic": (TRAFFIC_C4_PER_POINT[args.precision] * float(P.sum())
                                     if args.precision in TRAFFIC_C4_PER_POINT else None),
                         "kernel": BATCH_KERNEL, "bytes_per_launch": alg_bytes,
                         "peak_source": f"hbm_gbs ({src})",
                         "tensor": {"achieved": ach, "peak": peaks.get("bf16_tflops"), "unit": "TFLOP/s",
                                    "frac": ach / peaks.get("bf16_tflops"), "flops_per_launch": flops,
                                    "note": "algorithmic transform flops (forward + inverse per axis)",
                                    "executed": {"achieved": ex_ach, "peak": ex_peak, "unit": "TFLOP/s",
                                                 "frac": ex_ach / ex_peak, "flops_per_launch": ex_flops,
                                                 "note": "tensor-core flops issued (M = 128 lanes, every "
                                                         "split product, regrid GEMMs included)"}}},
            "clocks": clk.summary()}
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        import tempfile
        with tempfile.TemporaryDirectory() as td:
            t = oracle_c4_sample(len(cfgs), outdir=td)
            # parity of the sample: the same filters in a batch of their own,
            # the workload's whole horizon from their priors, weights against
            # the oracle's at the checkpoint epochs
            sid = c4_sample_ids(len(cfgs))
            pc, pm, pdt, _, pz = w.c4_batch(count=len(cfgs), epochs=t["epochs"])
            g = Batch([pc[i] for i in sid], [pm] * len(sid), precision=args.precision)
            errs, flipped, gbad = [], [], set()
            for k in range(t["epochs"]):
                g.step(np.arange(len(sid)), pz[sid, k], pdt)
                if k + 1 not in C4_CHECKPOINTS:
                    continue
                gst = g.status()
                for j, i in enumerate(sid):
                    if gst[j] != 0:
                        gbad.add(j)
                    fn = os.path.join(td, f"{i}_{k + 1}.npz")
                    if j in gbad or not os.path.exists(fn):
                        continue
                    ref = np.load(fn)
                    Pg, cg, Mg = g.pdf(j)
                    e = float(np.abs(Pg - ref["P"]).sum() / np.abs(ref["P"]).sum())
                    scale = np.abs(ref["M"]).max()
                    same = (np.abs(cg - ref["c"]).max() <= 1e-9 * scale and
                            np.abs(Mg - ref["M"]).max() <= 1e-9 * scale)
                    (errs if same else flipped).append(e)
            g.close()
        line["cpu_baseline"] = {"value": t["points"] / t["seconds"], "unit": UNIT, "cores": t["cores"],
                                "kind": "oracle",
                                "sample": f"{t['filters']} filters spread over the batch, {t['epochs']} epochs "
                                          "each, one single-threaded process per core"}
        line["rel_l1_vs_oracle"] = max(errs) if errs else None
        if errs:
            q = np.quantile(errs, [0.5, 0.99])
            line["rel_l1_quantiles"] = {"p50": float(q[0]), "p99": float(q[1]), "max": max(errs),
                                        "over_1e-5": int(sum(e > 1e-5 for e in errs))}
        line["rel_l1_sample"] = (f"max over {len(errs)} (filter, epoch) pairs of the {t['filters']} sampled "
                                 f"filters at epochs {list(C4_CHECKPOINTS)} whose frame equals the oracle's, "
                                 "same filters in a batch of their own, both on their own regrid decisions; "
                                 f"{len(flipped)} pairs on a neighbouring regrid lattice point (rel L1 up to "
                                 f"{max(flipped) if flipped else 0.0:.1e}); {len(gbad)} filters degenerate on "
                                 f"the GPU, {len(t['failed'])} stopped in the oracle")
    if rank == 0:
        print(json.dumps(line))


def bench_serve(args, ws, rank, pg):
    """The serving workload: 10k resident filters of mixed dimension, a Poisson
    request log replayed in real time through the request server."""
    import numpy as np
    import torch
    import workloads as w
    from paper_2412_07240_gb300 import Filter, Server
    n = args.count if args.count != 4096 else 10000
    warm = 0.5
    cap_s = args.capacity_log      # log seconds after the timed window, replayed all at once
    wl = w.c5_serving(n_filters=n, rate=args.rate, duration=args.duration + warm + cap_s, seed=5 + rank)
    P = np.array([int(np.prod(c.N)) for c in wl.cfgs], dtype=np.int64)
    srv = Server(max_filters=n, precision=args.precision, hbm_budget=int(120e9))
    t0 = time.perf_counter()
    fid = np.array([srv.admit(c, m) for c, m in zip(wl.cfgs, wl.meas)], dtype=np.int32)
    admit_s = time.perf_counter() - t0
    ids = fid[wl.ids]
    k = int(np.searchsorted(wl.t_arrival, warm))
    kend = int(np.searchsorted(wl.t_arrival, warm + args.duration))
    srv.replay(wl.t_arrival[:k], ids[:k], wl.z[:k], wl.taus[:k])          # warm-up requests
    sel = slice(k, kend)
    _barrier(pg)
    with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        lat, st = srv.replay(wl.t_arrival[sel] - warm, ids[sel], wl.z[sel], wl.taus[sel])
    wall = _max_over_ranks(pg, st["wall_s"] * 1e3) * 1e-3
    pts = float(P[wl.ids[sel]].sum())
    value = ws * pts / wall
    # capacity: the continuation of the log (each filter's next requests, so
    # the measurements stay consistent with its state), every request queued
    # at once: the rate the server sustains when it never waits for arrivals
    capacity = None
    if kend < len(wl.t_arrival):
        csel = slice(kend, None)
        clat, cst = srv.replay(np.zeros(len(wl.t_arrival) - kend), ids[csel], wl.z[csel], wl.taus[csel])
        cwall = _max_over_ranks(pg, cst["wall_s"] * 1e3) * 1e-3
        capacity = {"requests_per_s": ws * float(cst["requests"]) / cwall,
                    "grid_pt_updates_per_s": ws * float(P[wl.ids[csel]].sum()) / cwall,
                    "requests": int(cst["requests"]), "wall_s": cwall,
                    "mean_batch": cst["mean_batch"], "max_batch": int(cst["max_batch"]),
                    "note": "next requests of every filter, all queued at t = 0 (no arrival waits)"}
    # plain float64 per-filter path on a sample of each dimension
    rng = np.random.default_rng(0)
    f64_pts, f64_s = 0.0, 0.0
    for d in (1, 2, 3):
        cand = [i for i, c in enumerate(wl.cfgs) if c.nx == d]
        for i in rng.choice(cand, size=min(len(cand), 8 if d < 3 else 3), replace=False):
            f = Filter(wl.cfgs[i], precision="fp64")
            r = np.nonzero(wl.ids == i)[0][:3]
            for q in r[:1]:
                f.step(wl.meas[i], wl.z[q, :d], min(wl.taus[q], 0.6))
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for q in r[1:]:
                f.step(wl.meas[i], wl.z[q, :d], min(wl.taus[q], 0.6))
            e1.record()
            torch.cuda.synchronize()
            f64_pts += P[i] * len(r[1:])
            f64_s += e0.elapsed_time(e1) * 1e-3
            f.close()
    nreq = int(st["requests"])
    # algorithmic transform flops of the served requests: forward + inverse per axis
    served = wl.ids[sel]
    per_filter = np.array([4.0 * np.prod(c.N) * sum(c.N) for c in wl.cfgs])
    flops = float(per_filter[served].sum())
    peaks, peak_src = _peaks()
    peak = peaks.get("bf16_tflops", 1900.0)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": int(st["batches"]),
            "warmup": k, "ms_per_step": wall * 1e3 / max(1.0, st["batches"]), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": f"f32 ({args.precision} split GEMMs, 1-D float32)",
            "data": "synthetic (seeded filters, Poisson arrivals, exact-discretisation truth)",
            "config": {"workload": f"c5_serving_{n}_mixed", "rate_per_s": args.rate, "duration_s": args.duration,
                       "filters": n, "resident_points": int(P.sum()), "resident_bytes": srv.bytes,
                       "hbm_budget": int(120e9), "admission_s": admit_s, "precision": args.precision,
                       "parallelism": f"replicas x{ws}"},
            "requests_per_s": ws * nreq / wall,
            "latency_ms": {"p50": float(np.percentile(lat, 50) * 1e3), "p99": float(np.percentile(lat, 99) * 1e3),
                           "max": float(lat.max() * 1e3)},
            "batches": {"count": int(st["batches"]), "mean": st["mean_batch"], "max": int(st["max_batch"])},
            "capacity": capacity,
            "e2e": {"value": value, "unit": UNIT,
                    "h2d_bytes_per_step": int(st["mean_batch"] * (STEP_ITEM_BYTES + TIME_CONSTS_BYTES)),
                    "d2h_bytes_per_step": 0, "note": "the replay is end to end: requests from host arrays; the results stay resident "
                            "(read on demand), so nothing is copied back per batch"},
            "gpu_launches": int(st["launches"]),
            "fp64_gpu": {"value": f64_pts / f64_s if f64_s > 0 else None, "unit": UNIT,
                         "sample": "8 1-D, 8 2-D, 3 3-D filters, plain float64 path, one update each"},
            "roofline": {"bound": "tensor", "achieved": flops / wall / 1e12, "peak": peak, "unit": "TFLOP/s",
                         "frac": flops / wall / 1e12 / peak, "traffic": None,
                         "kernel": "all serving launches (1-D CUDA-core, 2-D fused, 3-D pipelines)",
                         "peak_source": f"bf16_tflops ({peak_src})",
                         "flops": flops, "note": "algorithmic transform flops of the served requests / wall"},
            "clocks": clk.summary()}
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        t = oracle_c5_sample(n)
        line["cpu_baseline"] = {"value": t["points"] / t["seconds"], "unit": UNIT, "cores": t["cores"],
                                "kind": "oracle",
                                "sample": f"first {t['requests_each']} requests of {t['filters']} 1-D/2-D/3-D "
                                          "filters, one single-threaded process per core"}
    if rank == 0:
        print(json.dumps(line))
    srv.close()


def bench_4d(args, ws, rank, pg, local):
    """The 4-D coordinated-turn terrain filter of Sec. VI (34^4 grid): the
    float32 4-D kernels (any precision but fp64), the float64 path beside
    them, and the RMSE/ASTD of Sec. VI over seeded Monte Carlo runs."""
    import numpy as np
    import torch
    import workloads as w
    from paper_2412_07240_gb300 import Degenerate, Filter
    legs = leg_epochs("c6", args.steps, args.warmup)
    sc = _apply_modes(_scenario("c6", max(legs.values()) + 1))
    P = 1
    for n in sc.cfg.N:
        P *= n
    prec = args.precision
    _barrier(pg)
    with ClockSampler(local) as clk:
        f, ms, launches = time_gpu(sc, prec, args.steps, args.warmup)
    t_ms = _max_over_ranks(pg, sum(ms))
    value = ws * P * args.steps / (t_ms * 1e-3)
    e2e_ms = _max_over_ranks(pg, time_e2e(sc, prec, min(args.steps, len(sc.z) - 3)))
    f.close()
    f64, ms64, l64 = time_gpu(sc, "fp64", legs["fp64"] - args.warmup, args.warmup)
    ms64_step = _max_over_ranks(pg, sum(ms64) / len(ms64))
    f64.close()

    # RMSE / ASTD over M runs of T + 1 filtering estimates (Sec. VI): one
    # terrain, a fresh seeded trajectory per run; runs are split over ranks
    T, M = 20, args.mc
    se, var, used, lost = np.zeros(4), np.zeros(4), 0, 0
    for m in range(rank, M, ws):
        run = _apply_modes(w.c6_scenario(seed=100 + m, epochs=T + 1))
        g = Filter(run.cfg, precision=prec, psi_mode=MODES["psi"])
        try:
            for k in range(T + 1):
                g.meas_update(run.meas, run.z[k])
                mean, cov = g.moments()
                se += (run.truth[k] - mean) ** 2
                var += np.diag(cov)
                if k < T:
                    g.time_update(run.dt)
            used += 1
        except Degenerate:
            lost += 1
        finally:
            g.close()
    if pg is not None:
        t = torch.tensor(np.concatenate([se, var, [used, lost]]), dtype=torch.float64)
        pg.all_reduce(t)
        se, var, used, lost = t[:4].numpy(), t[4:8].numpy(), int(t[8]), int(t[9])
    cnt = max(1, used) * (T + 1)
    # algorithmic transform flops of one epoch: regrid + forward (one fused
    # matrix) and inverse, 4 axes, 2 N_m flops per point each
    flops = 2 * 2.0 * P * sum(sc.cfg.N)
    kernel_ms = float(np.mean(ms))
    achieved = flops / (kernel_ms * 1e-3) / 1e12
    f32_peak = 152 * 128 * 2 * 2.07e9 / 1e12
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 (float32 grid and contractions; float64 exponents, frame and moment totals)",
        "data": "synthetic (seeded truth, synthetic terrain, Gaussian-mixture noise)",
        "config": {"workload": sc.name, "grid": list(sc.cfg.N), "precision": "float32 4-D kernels",
                   "dt": sc.dt, "dt_sub": sc.cfg.dt_sub,
                   "step": "one epoch: Bayes measurement update + spectral time update",
                   "l2": "flushed between timed steps (512 MB write)", "parallelism": f"replicas x{ws}"},
        "e2e": {"value": ws * P / (e2e_ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": 392,
                "d2h_bytes_per_step": 8 * (4 + 16), "ms_per_step": e2e_ms},
        "gpu_launches": int(launches),
        "fp64_gpu": {"value": ws * P / (ms64_step * 1e-3), "unit": UNIT, "ms_per_step": ms64_step,
                     "launches_per_step": l64 / max(1, len(ms64))},
        "latency_ms": {"p50": float(np.percentile(ms, 50)), "p99": float(np.percentile(ms, 99))},
        "accuracy": {"runs": used, "degenerate_runs": lost, "estimates_per_run": T + 1,
                     "rmse": np.sqrt(se / cnt).tolist(), "astd": np.sqrt(var / cnt).tolist(),
                     "state": ["p_x", "v_x", "p_y", "v_y"],
                     "paper_table_I_spectral": {"rmse": [14.4769, 13.0677, 9.8878, 6.8588],
                                                "astd": [18.8222, 15.0611, 13.1594, 8.807],
                                                "time_s": 0.41649,
                                                "note": "SRTM terrain and the paper's CPU; context only"}},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": f32_peak, "unit": "TFLOP/s",
                     "frac": achieved / f32_peak, "traffic": None,
                     "kernel": "whole epoch (8 float32 axis contractions + exponents + multiplier)",
                     "peak_source": "float32 FMA: 152 SMs x 128 lanes x 2 x 2.07 GHz",
                     "flops_per_launch": flops},
        "clocks": clk.summary(),
    }
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        epochs = legs["parity"]
        t = oracle_sample("c6", epochs, total=len(sc.z))
        per = t["seconds"] / t["epochs"]
        line["cpu_baseline"] = {"value": P / per, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"{epochs} epochs of the {sc.name} filter, single thread"}
        # parity of a sample: both filters on their own regrid decisions; an
        # update whose frames differ (a float32 decision on a neighbouring
        # lattice point) is counted, the weights of the others compared
        from oracle.filter import OracleFilter
        g = Filter(sc.cfg, precision=prec, psi_mode=MODES["psi"])
        o = OracleFilter(sc.cfg, psi_mode=MODES["psi"])
        worst, differ = 0.0, 0

        def _upd():
            nonlocal worst, differ
            Pg, cg, Mg = g.pdf()
            scale = np.abs(o.M).max()
            if np.abs(cg - o.c).max() > 1e-9 * scale or np.abs(Mg - o.M).max() > 1e-9 * scale:
                differ += 1
            else:
                worst = max(worst, float(np.abs(Pg - o.P).sum() / np.abs(o.P).sum()))
        for k in range(epochs):
            g.meas_update(sc.meas, sc.z[k])
            o.meas_update(sc.meas, sc.z[k])
            _upd()
            g.time_update(sc.dt)
            o.time_update(sc.dt)
            _upd()
        g.close()
        line["rel_l1_vs_oracle"] = worst
        line["rel_l1_sample"] = (f"{epochs} epochs, every update, both on their own regrid decisions; "
                                 f"{differ} updates with differing frames not compared")
    if rank == 0:
        print(json.dumps(line))


def default_precision(workload):
    """The split format of a workload: BF16X6 (the split-BF16 format within
    1e-5) where the tensor-core kernels have it (2-D: c2, c4, c5, whose 3-D
    filters the server runs in FP16X3), FP16X3 for the 3-D and 4-D paths."""
    return "fp16x3" if workload in ("c3", "c6") else "bf16x6"


def make_parser():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default="c4")
    ap.add_argument("--precision", default=None,
                    help="tensor-core format (default bf16x6 for c2/c4/c5, fp16x3 for c3/c6)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--count", type=int, default=4096, help="filters of the c4 batch workload (c5: 10000)")
    ap.add_argument("--rate", type=float, default=200e3, help="c5: aggregate request rate per second")
    ap.add_argument("--duration", type=float, default=60.0, help="c5: seconds of requests replayed")
    ap.add_argument("--capacity-log", type=float, default=2.0,
                    help="c5: seconds of further log replayed all at once for the capacity figure")
    ap.add_argument("--mc", type=int, default=50, help="c6: Monte Carlo runs for RMSE/ASTD")
    ap.add_argument("--psi", default="euler", choices=["euler", "exact"],
                    help="c2/c3/c6: diffusion multiplier (Euler product or exact in time)")
    ap.add_argument("--realign", default="multilinear", choices=["multilinear", "shear"],
                    help="c2: fill of a re-aligned frame (shear: band-limited, n_x = 2)")
    return ap


def main(argv=None):
    args = make_parser().parse_args(argv)
    args.warmup = max(3, args.warmup)
    args.precision = args.precision or default_precision(args.workload)
    MODES["psi"], MODES["realign"] = args.psi, args.realign
    ws, rank, local, pg = _dist()
    if args.impl == "reference":
        run_reference(args, ws, rank, pg)
        return

    import numpy as np
    import torch
    torch.cuda.set_device(local)
    if args.workload in ("c4", "c5", "c6"):
        if args.workload == "c6":
            bench_4d(args, ws, rank, pg, local)
        else:
            (bench_batch if args.workload == "c4" else bench_serve)(args, ws, rank, pg)
        if pg is not None:
            pg.destroy_process_group()
        return
    legs = leg_epochs(args.workload, args.steps, args.warmup)
    sc = _apply_modes(_scenario(args.workload, max(legs.values()) + 1))
    P = 1
    for n in sc.cfg.N:
        P *= n
    peaks, peak_src = _peaks()

    # fused tensor-core path
    _barrier(pg)
    with ClockSampler(local) as clk:
        f, ms, launches = time_gpu(sc, args.precision, args.steps, args.warmup)
    t_ms = _max_over_ranks(pg, sum(ms))
    ms_per_step = t_ms / args.steps
    value = ws * P * args.steps / (t_ms * 1e-3)

    # end to end through the public API
    e2e_ms = _max_over_ranks(pg, time_e2e(sc, args.precision, min(args.steps, len(sc.z) - 3)))
    meas_bytes = 176      # pmf_meas struct (host) per step
    mom_bytes = 8 * (len(sc.cfg.N) + len(sc.cfg.N) ** 2)

    # plain float64 GPU path on the same workload
    f64, ms64, l64 = time_gpu(sc, "fp64", legs["fp64"] - args.warmup, args.warmup)
    ms64_step = _max_over_ranks(pg, sum(ms64) / len(ms64))

    kernel_ms = float(np.mean(ms))
    flops = _flops_per_step(sc.cfg.N)
    achieved_tflops = flops / (kernel_ms * 1e-3) / 1e12
    peak = peaks.get("bf16_tflops", 1900.0)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": f"f32 ({args.precision} split GEMMs, fp64 frame/moments)" if args.precision != "fp64" else "f64",
        "data": "synthetic (seeded truth and measurements)",
        "config": {"workload": sc.name, "grid": list(sc.cfg.N), "precision": args.precision,
                   "psi": MODES["psi"], "realign": MODES["realign"],
                   "step": "one epoch: Bayes measurement update + spectral time update",
                   "l2": "flushed between timed steps (512 MB write)", "parallelism": f"replicas x{ws}"},
        "e2e": {"value": ws * P / (e2e_ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": meas_bytes,
                "d2h_bytes_per_step": mom_bytes, "ms_per_step": e2e_ms},
        "gpu_launches": int(launches),
        "fp64_gpu": {"value": ws * P / (ms64_step * 1e-3), "unit": UNIT, "ms_per_step": ms64_step,
                     "launches_per_step": l64 / max(1, len(ms64))},
        "latency_ms": {"p50": float(np.percentile(ms, 50)), "p99": float(np.percentile(ms, 99))},
        "roofline": {"bound": "tensor", "achieved": achieved_tflops, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved_tflops / peak,
                     "traffic": TRAFFIC_C2 if sc.name.startswith("c2") and tuple(sc.cfg.N) == (128, 128) else None,
                     "kernel": _launch_names(sc), "peak_source": f"bf16_tflops ({peak_src})",
                     "flops_per_launch": flops},
        "clocks": clk.summary(),
    }
    if rank == 0 and ws == 1 and not args.no_cpu_baseline and sc.cfg.nx in (2, 3):
        epochs = legs["parity"]
        t = oracle_sample(args.workload, epochs, total=len(sc.z))
        per = t["seconds"] / t["epochs"]
        # parity of the sample: same epochs on the GPU path from the prior
        g = type(f)(sc.cfg, precision=args.precision, psi_mode=MODES["psi"])
        for k in range(epochs):
            g.step(sc.meas, sc.z[k], sc.dt)
        Pg = g.pdf()[0]
        err = float(np.abs(Pg - t["P"]).sum() / np.abs(t["P"]).sum())
        line["cpu_baseline"] = {"value": P / per, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"{epochs} epochs of the {sc.name} filter, single thread"}
        line["rel_l1_vs_oracle"] = err
    if rank == 0:
        print(json.dumps(line))
    if pg is not None:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
