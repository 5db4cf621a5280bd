#!/usr/bin/env python3
"""Throughput benchmark of the COLA hot path on GB300 (one JSON line on stdout).

A "step" here is one pass of the whole hot path over one batch: Philox white noise -> 2LPT
initial conditions -> the nsteps+1 force evaluations of eq. ALCtimestep (deposit, 3-D FFT,
k-space Green's function, inverse FFTs, gather + COLA kick/drift) -> CIC density -> P(k).
The metric is particle-updates per second: np^3 * nsteps / (wall time of one step).

The headline workload is the largest single-GPU configuration, 1024^3 particles on a 2048^3
mesh in a 1000 Mpc/h box; the paper's own Sec. 2 run (256^3 particles, 768^3 mesh, 100 Mpc/h)
is measured the same way and reported as `paper_scale`.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

Multi-GPU (torchrun): every rank runs an independent realisation (different seed); there is no
collective on the data path ("replicas only", weak scaling); value = sum over ranks / max time.
--impl reference times the float64 CPU oracle on the host cores instead (rank 0 only).
"""
import argparse
import concurrent.futures
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "cola_1024p_2048g_L1000"  # the largest single-GPU configuration (headline)
PAPER_WORKLOAD = "cola_256p_768g_L100"  # the paper's Sec. 2 run (second line)
METRIC = "COLA particle-updates/s (N_p x steps / s), fwd and fwd+adjoint, on 1 GB300 vs plain GPU"
UNIT = "particle-updates/s"
NSTEPS = 10


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-ensemble", action="store_true")
    ap.add_argument("--no-fof", action="store_true")
    ap.add_argument("--no-paper-scale", action="store_true")
    return ap.parse_args()


# ---- distributed plumbing ----------------------------------------------------------------
def dist_setup(backend):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group(backend=backend)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world, device=None):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---- clocks during the timed region ------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.samples = []
        self.window = None
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(gpu_id), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True, bufsize=1)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 7:
                self.samples.append((time.time(), parts))

    def mark(self, t0, t1):
        self.window = (t0, t1)

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        t0, t1 = self.window
        sel = [p for (t, p) in self.samples if t0 - 0.15 <= t <= t1 + 0.15] or [p for _, p in self.samples[-3:]]
        if not sel:
            return None
        def num(x):
            try:
                return float(x)
            except ValueError:
                return None

        sm = [num(p[0]) for p in sel if num(p[0]) is not None]
        mx = [num(p[1]) for p in sel if num(p[1]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for p in sel for i in range(4) if p[3 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(sel)}


# ---- roofline bookkeeping ------------------------------------------------------------------------
def algorithmic_bytes(name, n_p, ng):
    """Minimum bytes a launch of kernel `name` must move (float32 / complex64 / int32 data).
    H = n^2 (n/2 + 1) complex modes of a half spectrum, 8 bytes each."""
    np3, ng3 = n_p**3, ng**3
    n = int(name.rsplit("_", 1)[1]) if name.rsplit("_", 1)[-1].isdigit() else ng
    H = n * n * (n // 2 + 1) * 8
    if name.startswith("fft_cols"):
        return 2 * H                       # in-place complex column pass: read + write
    if name.startswith("fft_x_r2c") or name.startswith("fft_x_c2r_"):
        return H + n**3 * 4                # real rows <-> half-spectrum rows
    if name.startswith("deposit_fftx"):
        return 12 * np3 + H                # fixed-point coordinates per particle, half spectrum out
    if name.startswith("fft_z_green"):
        return H + 2 * H                   # delta_k in; B and Gz out
    if name.startswith("fft_y_inv3"):
        return 2 * H + 3 * H               # B, Gz in; C, Gy, Gz out
    if name.startswith("fft_x_c2r3"):
        return 3 * (H + n**3 * 4)          # three half spectra in, three real meshes out
    table = {
        "deposit_4x4": 12 * np3 + 4 * ng3,   # fixed-point coordinates per particle, delta rows written once
        "deposit_4x2": 12 * np3 + 4 * ng3,
        "deposit_2x2": 12 * np3 + 4 * ng3,
        "kspace_force": 4 * 8 * ng * ng * (ng // 2 + 1),
        "gather_kick_drift": 72 * np3 + 12 * ng3,  # s, v, s1, s2 in, s, v out; 3 force meshes once
        "gather_binned": 28 * np3 + 12 * ng3,  # index + coordinates in, force out; 3 force meshes once
        "gather_binned4": 32 * np3 + 12 * ng3,  # the same with the force as one float4 per particle
        "kick_drift": 84 * np3,            # force, s, v, s1, s2 in; s, v out
        "kick_drift4": 88 * np3,           # the same with the force read as one float4
        "keys": 16 * np3,
        "scatter": 32 * np3,               # key + displacement in; index + fixed-point coordinates out
        "power_bin": 8 * ng * ng * (ng // 2 + 1),
    }
    return table.get(name)


# the sources the force-evaluation kernels are compiled from (their measured DRAM traffic stays
# valid while these are unchanged)
FORCE_SOURCES = ("cola_internal.cuh", "fft.cuh", "particle_bodies.cuh", "pm_bodies.cuh", "pm_common.cuh",
                 "pm_fft_kernels.cu", "pm_kernels.cu", "tma.cuh")


def kernel_source_digest():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1301_0322_gb300", "csrc")
    for f in FORCE_SOURCES:
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(f.encode() + fh.read())
    return h.hexdigest()[:16]


def measured_traffic(name, workload):
    """dram read+write bytes per launch from a committed ncu summary, if taken on this source."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        data = json.load(open(path))
    except Exception:
        return None
    rec = data.get(workload, {}).get(name)
    if not rec or rec.get("source_digest") != kernel_source_digest():
        return None
    return rec.get("dram_bytes_per_launch")


def hbm_peak():
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ---- the float64 oracle as a CPU baseline ------------------------------------------------------
_ORACLE_STATE = {}


def oracle_sample(workload):
    """One COLA step (PM force at a_0, kick to a_1/2, drift to a_1) of the float64 oracle on a
    periodic sub-volume of the workload at the same resolution: the box side, the particles and
    the mesh cells per side divided by d = max(2, np / 128) (1/8 of the 256^3/768^3 workload,
    1/512 of the 1024^3/2048^3 one).  The 2LPT initial conditions are set up once, untimed.
    Returns (particle-updates/s, seconds, description, particles in the sample)."""
    import numpy as np

    from oracle import cola as oc
    from oracle import lpt
    from oracle.cosmology import Cosmology, time_grid
    from paper_1301_0322_gb300 import inputs

    n_p, ng, box, seed = inputs.WORKLOADS[workload]
    d = max(2, n_p // 128)
    n_p, ng, box = n_p // d, ng // d, box / d
    if workload not in _ORACLE_STATE:
        cosmo = Cosmology(**inputs.COSMOLOGY)
        cfg = oc.ColaConfig(n_p=n_p, n_g=ng, box=box, cosmo=cosmo, nsteps=NSTEPS)
        w = inputs.gaussian_noise(n_p, seed).reshape(n_p, n_p, n_p).astype(np.float64)
        s1, s2 = lpt.ic_2lpt(w, box, cosmo)
        a, mid = time_grid(cfg.a_init, cfg.a_final, NSTEPS)
        g = cosmo.growth(a)
        coef = (cosmo.kick_cola(a[0], mid[0], a[0], cfg.n_lpt), cosmo.drift_cola(a[0], a[1], mid[0], cfg.n_lpt))
        _ORACLE_STATE[workload] = (cfg, s1, s2, a, g, coef)
    cfg, s1, s2, a, g, (ck, cd) = _ORACLE_STATE[workload]
    s = g["D1"][0] * s1 + g["D2"][0] * s2
    v = np.zeros_like(s)
    t0 = time.perf_counter()
    acc = oc.acceleration(s, cfg, a[0])
    v = v + ck * (acc - g["T2D1"][0] * s1 - g["T2D2"][0] * s2)
    s = s + cd * v + (g["D1"][1] - g["D1"][0]) * s1 + (g["D2"][1] - g["D2"][0]) * s2
    dt = time.perf_counter() - t0
    desc = (f"one float64 oracle COLA step (PM force, kick, drift) on a {box:g} Mpc/h sub-volume at the "
            f"workload's resolution ({n_p}^3 particles, {ng}^3 mesh, 1/{d**3} of the workload; the FFT's "
            f"N log N share is that of the smaller mesh)")
    return n_p**3 / dt, dt, desc, n_p**3


def reference_arm(args):
    rank, world, _ = dist_setup("gloo")
    if rank != 0:
        barrier(world)
        return
    cores = os.cpu_count()
    times = []
    for i in range(args.warmup + args.steps):
        _, dt, desc, n_sub = oracle_sample(args.workload)
        if i >= args.warmup:
            times.append(dt)
    per_step = statistics.mean(times)
    value = n_sub / per_step
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_step * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args.workload, world),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    barrier(world)


# ---- the GB300 arm ------------------------------------------------------------------------------------
# kernels of one force evaluation (binning, mesh passes, gather, kick/drift) by profiler label
EVAL_KERNELS = ("keys", "scan_reduce", "scan_blocks", "scan_apply", "scatter", "deposit_fftx_", "fft_cols_fwd_",
                "fft_z_green_", "fft_y_inv3_", "fft_x_c2r3_", "gather_binned", "kick_drift", "gather_kick_drift",
                "gather_binned4", "kick_drift4")


def eval_floor_bytes(n_p, ng):
    """Algorithmic floor of one force evaluation: 56 bytes per mesh cell (deposit write 8, r2c read 8
    + write 4, three c2r read 4 + write 4, gather read 12) plus 84 bytes per particle (deposit read
    12, kick/drift read 48 and write 24)."""
    return 56 * ng**3 + 84 * n_p**3


def workload_config(workload, world):
    from paper_1301_0322_gb300 import inputs
    n_p, ng, box, _ = inputs.WORKLOADS[workload]
    return {"workload": workload, "particles": f"{n_p}^3", "mesh": f"{ng}^3", "box_mpc_h": box,
            "nsteps": NSTEPS, "step": "noise + 2LPT IC + 11 force evaluations + density + P(k)",
            "mode": "forward", "parallelism": "replicas" if world > 1 else "single",
            "l2": "inputs larger than L2 (meshes of several GB)"}


class HostSink:
    """Device -> host copy of a float32 device array into a pageable host array through a ring of
    pinned staging chunks: a helper thread issues one cudaMemcpyAsync per chunk on a copy stream
    (after `ready` has been recorded) and copies each landed chunk into the destination while the
    next one is in flight, split over `workers` (a thread pool shared by the sinks: one thread
    copies about 13 GB/s of host memory, the device sends about 190).  `enqueued()` returns the
    event after the last chunk's copy once the thread has issued it (the caller's stream waits on
    it before reusing the source)."""

    def __init__(self, torch, chunk_elems, nslots, copy_stream, workers):
        self.torch = torch
        self.slots = [torch.empty(chunk_elems, dtype=torch.float32, pin_memory=True) for _ in range(nslots)]
        self.done = [torch.cuda.Event() for _ in range(nslots)]
        self.cs = copy_stream
        self.chunk = chunk_elems
        self.workers = workers
        self.nparts = max(1, workers._max_workers)
        self.thread = None
        self.last = None
        self.issued = threading.Event()

    def start(self, src, dst, ready):
        self.issued.clear()
        self.thread = threading.Thread(target=self._run, args=(src.reshape(-1), dst.reshape(-1), ready))
        self.thread.start()

    def _run(self, src, dst, ready):
        torch = self.torch
        n, c, ns = src.numel(), self.chunk, len(self.slots)
        ranges = [(a, min(n, a + c)) for a in range(0, n, c)]
        pending = [None] * ns
        with torch.cuda.device(src.device), torch.cuda.stream(self.cs):
            self.cs.wait_event(ready)
            for i, (a, b) in enumerate(ranges):
                k = i % ns
                if pending[k] is not None:
                    self._land(k, pending[k], dst)
                self.slots[k][:b - a].copy_(src[a:b], non_blocking=True)
                self.done[k].record(self.cs)
                pending[k] = (a, b)
            self.last = self.done[(len(ranges) - 1) % ns]
            self.issued.set()
            for j in range(len(ranges), len(ranges) + ns):
                k = j % ns
                if pending[k] is not None:
                    self._land(k, pending[k], dst)
                    pending[k] = None

    def _land(self, k, ab, dst):
        import numpy as np
        a, b = ab
        self.done[k].synchronize()
        src, out = self.slots[k].numpy(), dst.numpy()
        step = -(-(b - a) // self.nparts)
        parts = [(lo, min(b - a, lo + step)) for lo in range(0, b - a, step)]
        for f in [self.workers.submit(np.copyto, out[a + lo:a + hi], src[lo:hi]) for lo, hi in parts]:
            f.result()

    def enqueued(self):
        self.issued.wait()
        return self.last

    def join(self):
        self.thread.join()


def measure_workload(args, workload, dev, rank, world, with_fof):
    """Time `args.steps` whole runs of `workload` (after `args.warmup` untimed ones) on the device,
    the per-kernel split, the roofline of the dominant kernel and of a whole force evaluation, and
    the same runs end to end with host buffers."""
    import ctypes

    import torch

    import paper_1301_0322_gb300 as cola
    from paper_1301_0322_gb300 import inputs

    n_p, ng, box, seed = inputs.WORKLOADS[workload]
    plan = cola.Plan(np_side=n_p, ng=ng, box=box, nsteps=NSTEPS, device=dev, **inputs.COSMOLOGY)
    h = plan.handle
    lib = cola.load_library()
    n3 = n_p**3
    nbins = ng // 2
    s = plan._empty((3, n3))
    # v, s1 and s2 share one allocation, and the noise sits in the v slot (the initial conditions
    # transform it before they write v); the final density and its transform go to the plan's
    # own force meshes (cola_density_power), free after the last step
    pool = plan._empty(9 * n3)
    v, s1, s2 = (pool[i * 3 * n3:(i + 1) * 3 * n3].view(3, n3) for i in range(3))
    noise = pool[:n3]
    k, pk = plan._empty(nbins, torch.float64), plan._empty(nbins, torch.float64)
    nm = plan._empty(nbins, torch.int64)

    def one_step(sd):
        cola.cola_noise(h, sd, noise)
        cola.cola_ic_2lpt(h, noise, s, v, s1, s2)
        for i in range(NSTEPS + 1):
            cola.cola_step(h, i, s, v, s1, s2)
        cola.cola_density_power(h, s, nbins, k, pk, nm)

    base_seed = seed + 1000 * rank
    gpu_id = str(torch.cuda.get_device_properties(dev).uuid)
    gpu_id = gpu_id if gpu_id.startswith("GPU-") else "GPU-" + gpu_id
    sampler = ClockSampler(gpu_id) if rank == 0 else None
    for i in range(args.warmup):
        one_step(base_seed + i)
    plan.status()
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    cnt0 = ctypes.c_uint64()
    lib.cola_launch_count(ctypes.byref(cnt0))
    lib.cola_profile(h, 1)
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t_wall0 = time.time()
    ev0.record(stream)
    for i in range(args.steps):
        one_step(base_seed + 100 + i)
    ev1.record(stream)
    ev1.synchronize()
    t_wall1 = time.time()
    torch.cuda.synchronize()
    lib.cola_profile(h, 0)
    cnt1 = ctypes.c_uint64()
    lib.cola_launch_count(ctypes.byref(cnt1))
    barrier(world)
    plan.status()
    ms_step = max_over_ranks(ev0.elapsed_time(ev1) / args.steps, world, dev)
    clocks = None
    if sampler:
        sampler.mark(t_wall0, t_wall1)
        clocks = sampler.stop()
    # per-kernel device time from the events recorded around every launch (on the launch stream)
    nmax = 256
    names = ctypes.create_string_buffer(64 * nmax)
    launches = (ctypes.c_int64 * nmax)()
    msk = (ctypes.c_double * nmax)()
    count = ctypes.c_int32()
    lib.cola_profile_read(h, nmax, names, launches, msk, ctypes.byref(count))
    kernels = {}
    for i in range(count.value):
        nm_ = names.raw[64 * i:64 * (i + 1)].split(b"\0", 1)[0].decode()
        kernels[nm_] = {"launches": int(launches[i]), "ms": float(msk[i])}
    total_ms = ms_step * args.steps
    peak, peak_kind = hbm_peak()
    for name, kv in kernels.items():
        kv["share"] = kv["ms"] / total_ms
        alg = algorithmic_bytes(name, n_p, ng)
        kv["avg_launch_ms"] = kv["ms"] / kv["launches"]
        if alg and name in ("power_bin", "cross_bin"):
            alg /= kv["launches"] / args.steps  # one spectrum read, over the shell-range launches of a P(k)
        if alg:
            kv["bytes_per_launch"] = alg
            kv["achieved_gbs"] = alg / (kv["avg_launch_ms"] * 1e-3) / 1e9
            kv["frac"] = kv["achieved_gbs"] / peak
    dom = max(kernels, key=lambda x: kernels[x]["ms"])
    alg = algorithmic_bytes(dom, n_p, ng)
    avg_ms = kernels[dom]["avg_launch_ms"]
    achieved = alg / (avg_ms * 1e-3) / 1e9 if alg else None
    # one force evaluation against the algorithmic floor of the scope table: one launch of each of
    # its kernels, at the mean duration of that kernel's launches (the density and P(k) at the end
    # of a run launch the binning, the fused deposit and the forward passes once more)
    ev_ms = sum(kv["ms"] / kv["launches"] for nm_, kv in kernels.items()
                if any(nm_ == e or (e.endswith("_") and nm_ == e + str(ng)) for e in EVAL_KERNELS))
    floor = eval_floor_bytes(n_p, ng)
    roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "peak_source": peak_kind,
                "unit": "GB/s", "frac": (achieved / peak) if achieved else None,
                "traffic": measured_traffic(dom, workload), "bytes_per_launch": alg, "avg_launch_ms": avg_ms,
                "force_evaluation": {"floor_bytes": floor, "ms": ev_ms,
                                     "achieved_gbs": floor / (ev_ms * 1e-3) / 1e9,
                                     "frac": floor / (ev_ms * 1e-3) / 1e9 / peak,
                                     "floor": "56 B per mesh cell + 84 B per particle"}}
    value = world * n3 * NSTEPS / (ms_step * 1e-3)

    # end to end through the public API with host buffers: the noise arrives from pinned host
    # memory, s, v and P(k) go back to pageable host arrays through pinned staging chunks
    e2e = None
    if not args.no_e2e:
        copy_stream = torch.cuda.Stream(device=dev)
        chunk = min(3 * n3, 64 << 20)  # 256 MB chunks
        pool = concurrent.futures.ThreadPoolExecutor(max_workers=os.cpu_count() or 8)
        # one copy stream per sink: in a shared stream, chunks of s issued after v's first ones
        # would queue behind v's wait for the end of the steps
        sink_s, sink_v = (HostSink(torch, chunk, 3, torch.cuda.Stream(device=dev), pool) for _ in range(2))
        h_noise = torch.empty(n3, dtype=torch.float32, pin_memory=True)
        h_s = torch.zeros((3, n3), dtype=torch.float32)  # pageable (zeros: pages touched once here)
        h_v = torch.zeros((3, n3), dtype=torch.float32)
        h_pk = torch.empty(nbins, dtype=torch.float64, pin_memory=True)
        cola.cola_noise(h, base_seed, noise)
        h_noise.copy_(noise)
        e_noise = plan._empty(n3)  # its own slot, so that the next run's noise arrives during this run
        ev_ic, ev_s, ev_steps, ev_noise = (torch.cuda.Event() for _ in range(4))
        e_noise.copy_(h_noise)
        ev_noise.record(stream)
        torch.cuda.synchronize()
        ke = max(1, min(args.steps, 3 if ng >= 1536 else 5))

        def e2e_step():
            stream.wait_event(ev_noise)  # this run's noise has arrived
            cola.cola_ic_2lpt(h, e_noise, s, v, s1, s2)
            ev_ic.record(stream)
            with torch.cuda.stream(copy_stream):  # the next run's noise, host -> device
                copy_stream.wait_event(ev_ic)
                e_noise.copy_(h_noise, non_blocking=True)
                ev_noise.record(copy_stream)
            for i in range(NSTEPS + 1):
                cola.cola_step(h, i, s, v, s1, s2)
                if i == NSTEPS - 1:  # s is final here (the last evaluation kicks v only)
                    ev_s.record(stream)
                    sink_s.start(s, h_s, ev_s)
            ev_steps.record(stream)
            sink_v.start(v, h_v, ev_steps)  # v leaves during the density and P(k)
            cola.cola_density_power(h, s, nbins, k, pk, nm)
            h_pk.copy_(pk, non_blocking=True)
            stream.wait_event(sink_s.enqueued())
            stream.wait_event(sink_v.enqueued())  # the next run's initial conditions write v

        def e2e_join():
            sink_s.join()
            sink_v.join()
            stream.wait_event(ev_noise)

        e2e_step()
        e2e_join()
        torch.cuda.synchronize()
        barrier(world)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        t0 = time.perf_counter()
        for _ in range(ke):
            e2e_step()
            e2e_join()  # the host arrays hold this run's s and v before the next run starts
        e1.record(stream)
        e1.synchronize()
        wall = (time.perf_counter() - t0) * 1e3 / ke
        ms_e2e = max_over_ranks(max(e0.elapsed_time(e1) / ke, wall), world, dev)
        # the host arrays hold the last run's results
        assert torch.equal(h_pk, pk.cpu()), "host copy of P(k) differs from the device result"
        assert torch.equal(h_s[:, -4096:], s[:, -4096:].cpu()), "host copy of s differs from the device result"
        assert torch.equal(h_v[:, -4096:], v[:, -4096:].cpu()), "host copy of v differs from the device result"
        e2e = {"value": world * n3 * NSTEPS / (ms_e2e * 1e-3), "unit": UNIT, "ms_per_step": ms_e2e,
               "h2d_bytes_per_step": 4 * n3, "d2h_bytes_per_step": 2 * 12 * n3 + 8 * nbins,
               "steps": ke, "host_arrays": "s, v pageable (through 256 MB pinned staging chunks); noise, P(k) pinned"}
        pool.shutdown()
        del sink_s, sink_v, h_s, h_v, h_noise, e_noise

    # halo finding on the final state of the last run (Sec. 3.2: b = 0.2, >= 25 particles)
    fof = None
    if with_fof and not args.no_fof and rank == 0:
        thresholds = [25, 50, 100, 200, 400, 800, 1600, 3200]
        group = plan._empty(n3, torch.int32)
        size = plan._empty(n3, torch.int32)
        n_ge = plan._empty(len(thresholds), torch.int64)
        for _ in range(2):
            cola.cola_fof(h, s, 1, 5, 25, group, size, thresholds, n_ge)
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        cola.cola_fof(h, s, 1, 5, 25, group, size, thresholds, n_ge)
        f1.record(stream)
        f1.synchronize()
        plan.status()
        rho_crit = 2.775e11  # h^2 M_sun / Mpc^3
        m_p = rho_crit * inputs.COSMOLOGY["omega_m"] * box**3 / n3
        fof = {"ms": f0.elapsed_time(f1), "linking_length": 0.2, "nmin": 25, "particle_mass_msun_h": m_p,
               "halos": int(n_ge[0]),
               "n_ge": {f"{t * m_p:.3g}": int(c) for t, c in zip(thresholds, n_ge.tolist())},
               "state": f"final state of the last timed {workload} run"}
    del plan, pool, s
    torch.cuda.empty_cache()
    return {
        "workload": workload, "value": value, "ms_per_step": ms_step, "roofline": roofline, "e2e": e2e,
        "clocks": clocks, "fof": fof, "gpu_launches": int(cnt1.value - cnt0.value),
        "config": workload_config(workload, world),
        "kernels": {kk: {"launches": kv["launches"], "ms_per_step": round(kv["ms"] / args.steps, 4),
                         "share": round(kv["share"], 4),
                         **({"frac": round(kv["frac"], 4), "achieved_gbs": round(kv["achieved_gbs"], 1)}
                            if "frac" in kv else {})}
                    for kk, kv in sorted(kernels.items(), key=lambda x: -x[1]["ms"])},
    }


def cpu_baseline(workload):
    reps, vals, desc, spent = 0, [], "", 0.0
    while spent < 10.0 and reps < 4:
        val, dt, desc, _ = oracle_sample(workload)
        vals.append(val)
        spent += dt
        reps += 1
    return {"value": statistics.median(vals), "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{desc}; median of {reps} repetitions"}


def gb300_arm(args):
    import torch

    rank, world, local = dist_setup("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    head = measure_workload(args, args.workload, dev, rank, world, with_fof=args.workload == PAPER_WORKLOAD)
    paper = None
    if args.workload != PAPER_WORKLOAD and not args.no_paper_scale:
        paper = measure_workload(args, PAPER_WORKLOAD, dev, rank, world, with_fof=True)

    # forward + adjoint on the differentiable workload, through the autograd wrapper
    fwd_adj = None
    if not args.no_adjoint:
        fwd_adj = adjoint_timing(args, dev, rank, world)
        torch.cuda.empty_cache()

    # the 48-box mock ensemble: batched persistent kernels + graphs against sequential single boxes
    ens = None
    if not args.no_ensemble:
        ens = ensemble_timing(args, dev, rank, world)
        torch.cuda.empty_cache()

    cpu = cpu_paper = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.workload)
        if paper is not None:
            cpu_paper = cpu_baseline(PAPER_WORKLOAD)

    if rank == 0:
        line = {
            "metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": head["config"], "roofline": head["roofline"], "cpu_baseline": cpu, "e2e": head["e2e"],
            "clocks": head["clocks"], "gpu_launches": head["gpu_launches"],
            "paper_scale": None if paper is None else {
                k_: paper[k_] for k_ in ("workload", "value", "ms_per_step", "roofline", "e2e", "clocks",
                                         "gpu_launches", "kernels")},
            "fwd_adjoint": fwd_adj, "ensemble": ens, "fof": head["fof"] or (paper or {}).get("fof"),
            "kernels": head["kernels"],
        }
        if paper is not None:
            line["paper_scale"]["unit"] = UNIT
            line["paper_scale"]["cpu_baseline"] = cpu_paper
        print(json.dumps(line), flush=True)
    barrier(world)


def adjoint_timing(args, dev, rank, world):
    """Particle-updates/s of forward + gradient (loss = sum (delta - delta_target)^2, gradient
    with respect to the white noise) on the 128^3 / 256^3, L = 200 Mpc/h workload, and the cost
    of the backward pass relative to the forward pass."""
    import torch

    import paper_1301_0322_gb300 as cola
    from paper_1301_0322_gb300 import inputs

    name = "cola_128p_256g_L200"
    n_p, ng, box, seed = inputs.WORKLOADS[name]
    plan = cola.Plan(np_side=n_p, ng=ng, box=box, nsteps=NSTEPS, adjoint=True, device=dev, **inputs.COSMOLOGY)
    with torch.no_grad():
        target = cola.cola_density_from_noise(plan.noise(seed), plan).double()
    noise = plan.noise(seed + 1000 + rank)
    stream = torch.cuda.current_stream()

    def fwd_bwd():
        x = noise.clone().requires_grad_(True)
        loss = ((cola.cola_density_from_noise(x, plan).double() - target) ** 2).sum()
        loss.backward()
        return x.grad

    def fwd_only():
        with torch.no_grad():
            return ((cola.cola_density_from_noise(noise, plan).double() - target) ** 2).sum()

    for _ in range(max(3, args.warmup)):
        fwd_bwd()
        fwd_only()
    torch.cuda.synchronize()
    barrier(world)
    k = max(3, min(args.steps, 20))
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    e0.record(stream)
    for _ in range(k):
        fwd_bwd()
    e1.record(stream)
    for _ in range(k):
        fwd_only()
    e2.record(stream)
    e2.synchronize()
    ms_fb = max_over_ranks(e0.elapsed_time(e1) / k, world, dev)
    ms_f = max_over_ranks(e1.elapsed_time(e2) / k, world, dev)
    return {"value": world * n_p**3 * NSTEPS / (ms_fb * 1e-3), "unit": UNIT, "workload": name,
            "ms_per_step": ms_fb, "forward_ms": ms_f, "backward_over_forward": (ms_fb - ms_f) / ms_f,
            "step": "forward with per-evaluation checkpoints + density + loss + adjoint to the noise"}


def ensemble_timing(args, dev, rank, world):
    """Particle-updates/s of the 48-box mock ensemble (16 x 64^3/128^3 L=100, 16 x 96^3/192^3
    L=150, 16 x 128^3/256^3 L=200 Mpc/h, seeds 100..147): noise + 2LPT IC + 11 force
    evaluations + density + P(k) for all boxes, the steps replayed from CUDA graphs with the
    launch shape the autotuner picked; against the same work done box after box with
    single-box plans (one plan per box size)."""
    import ctypes

    import torch

    import paper_1301_0322_gb300 as cola
    from paper_1301_0322_gb300 import inputs

    boxes = inputs.ENSEMBLE_48
    seeds = [sd + 1000 * rank for sd in inputs.ENSEMBLE_48_SEEDS]
    e = cola.Ensemble(boxes, device=dev, nsteps=NSTEPS, **inputs.COSMOLOGY)
    nbins = 32
    noise = e.noise(seeds)
    s, v, s1, s2 = e.ic_2lpt(noise)
    best, tune_ms = e.tune(s, reps=3)
    delta = e._empty(e.cells_total)
    kk, pk = e._empty((e.nbox, nbins), torch.float64), e._empty((e.nbox, nbins), torch.float64)
    nm = e._empty((e.nbox, nbins), torch.int64)
    h = e.handle
    sd_arr = seeds

    def ens_step():
        cola.cola_ensemble_noise(h, sd_arr, noise)
        cola.cola_ensemble_ic_2lpt(h, noise, s, v, s1, s2)
        for i in range(NSTEPS + 1):
            cola.cola_ensemble_step(h, i, s, v, s1, s2)
        cola.cola_ensemble_density(h, s, delta)
        cola.cola_ensemble_power(h, delta, nbins, kk, pk, nm)

    stream = torch.cuda.current_stream()
    reps = max(2, min(args.steps, 5))

    def timed(fn):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        barrier(world)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        e1.synchronize()
        return max_over_ranks(e0.elapsed_time(e1) / reps, world, dev)

    ms_ens = timed(ens_step)
    e.status()
    # per-kernel split of one ensemble run (direct launches with events)
    lib = cola.load_library()
    lib.cola_ensemble_profile(h, 1)
    ens_step()
    lib.cola_ensemble_profile(h, 0)
    nmax = 64
    names = ctypes.create_string_buffer(64 * nmax)
    launches = (ctypes.c_int64 * nmax)()
    msk = (ctypes.c_double * nmax)()
    count = ctypes.c_int32()
    lib.cola_ensemble_profile_read(h, nmax, names, launches, msk, ctypes.byref(count))
    kernels = {}
    for i in range(count.value):
        nm_ = names.raw[64 * i:64 * (i + 1)].split(b"\0", 1)[0].decode()
        kernels[nm_] = {"launches": int(launches[i]), "ms": float(msk[i])}
    peak, peak_kind = hbm_peak()
    sized = ("keys", "scatter", "gather_kick_drift", "gather_binned", "kick_drift")
    for name, kv in kernels.items():
        alg = 0
        if name.startswith("ens_"):  # multi-box kernels: one launch covers every box
            base = name[len("ens_"):]
            for n_p, ng, _ in boxes:
                if base in sized:
                    a = algorithmic_bytes(base, n_p, ng)
                elif base == "fft_y":
                    a = algorithmic_bytes(f"fft_cols_{ng}", n_p, ng)
                else:
                    a = algorithmic_bytes(f"{base}_{ng}", n_p, ng)
                alg = alg + a if a is not None and alg is not None else None
        else:  # per-box launches: bytes of one box of the launch's size (mean over the boxes)
            suffix = name.rsplit("_", 1)[-1]
            of_size = [b for b in boxes if not suffix.isdigit() or b[1] == int(suffix)]
            parts = [algorithmic_bytes(name, n_p, ng) for n_p, ng, _ in of_size]
            alg = sum(parts) / len(parts) if parts and None not in parts else None
        avg = kv["ms"] / kv["launches"]
        kv["avg_launch_ms"] = avg
        if alg:
            kv["bytes_per_launch"] = alg
            kv["achieved_gbs"] = alg / (avg * 1e-3) / 1e9
            kv["frac"] = kv["achieved_gbs"] / peak
    del e
    torch.cuda.empty_cache()

    # sequential single-box runs of the same 48 boxes
    plans = {}
    for n_p, ng, box in boxes:
        if (n_p, ng, box) not in plans:
            p = cola.Plan(np_side=n_p, ng=ng, box=box, nsteps=NSTEPS, device=dev, **inputs.COSMOLOGY)
            n3 = n_p**3
            bufs = [p._empty(n3)] + [p._empty((3, n3)) for _ in range(4)] + [p._empty(ng**3)]
            bufs += [p._empty(nbins, torch.float64), p._empty(nbins, torch.float64), p._empty(nbins, torch.int64)]
            plans[(n_p, ng, box)] = (p, bufs)

    def seq_step():
        for (n_p, ng, box), sd in zip(boxes, seeds):
            p, (nz, ss, vv, a1, a2, dd, k_, p_, m_) = plans[(n_p, ng, box)]
            hh = p.handle
            cola.cola_noise(hh, sd, nz)
            cola.cola_ic_2lpt(hh, nz, ss, vv, a1, a2)
            for i in range(NSTEPS + 1):
                cola.cola_step(hh, i, ss, vv, a1, a2)
            cola.cola_density(hh, ss, None, dd)
            cola.cola_power(hh, dd, nbins, k_, p_, m_)

    ms_seq = timed(seq_step)
    for p, _ in plans.values():
        p.status()
    updates = world * sum(b[0] ** 3 for b in boxes) * NSTEPS
    return {"workload": "ensemble_48: 16x 64^3/128^3 L100 + 16x 96^3/192^3 L150 + 16x 128^3/256^3 L200, seeds 100..147",
            "value": updates / (ms_ens * 1e-3), "unit": UNIT, "ms_per_step": ms_ens,
            "sequential_single_box": {"value": updates / (ms_seq * 1e-3), "ms_per_step": ms_seq},
            "speedup_vs_sequential": ms_seq / ms_ens,
            "tuning": {"threads": best.threads, "tile_shape": best.tile_shape, "blocks_per_sm": best.blocks_per_sm,
                       "radix": best.radix, "launch": best.launch, "mesh_streams": best.mesh_streams},
            "tune_candidates_ms": [round(float(x), 4) for x in tune_ms],
            "step": "noise + 2LPT IC + 11 force evaluations (CUDA graph per step) + density + P(k), all boxes",
            "kernels": {k_: {kk_: (round(vv_, 5) if isinstance(vv_, float) else vv_) for kk_, vv_ in kv.items()}
                        for k_, kv in sorted(kernels.items(), key=lambda x: -x[1]["ms"])},
            "peak_gbs": peak, "peak_source": peak_kind}


if __name__ == "__main__":
    a = parse_args()
    if a.impl == "reference":
        reference_arm(a)
    else:
        gb300_arm(a)
