"""Throughput of the two-component pseudopotential D3Q19 step on one GB300.

Workload (default): primary drainage in a synthetic sphere pack, 128^3 voxels,
spheres of radius 8 by seeded relaxed random sequential addition to porosity
0.38, 8 reservoir slices per end, non-wetting component injected at z = 0
under a fixed capillary pressure, NEEM inlet/outlet, contact angle 45 deg,
viscosity ratio 10, FP32.  A step is one full time step over every fluid
voxel (density, wall density, force, collision, streaming, bounce-back, open
planes).  Throughput counts fluid-node updates per second (MLUPS over fluid
nodes; the all-voxel rate is in ``config``).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
For N > 1 run under torchrun: every rank runs an independent replica.

``--workload adjoint_pack_96`` times the reverse pass: a 96^3 sphere pack
(radius 6, porosity 0.40), 500 steps of imbibition in FP32, loss = smooth
non-wetting saturation, gradients with respect to the per-voxel wettability
and the inlet density, checkpoints every 50 steps; adjoint steps per second
next to forward steps per second on the same lattice.

``--workload batched_sweep_64`` instead times the batched sweep: 64
independent sphere packs (edges 48..112, radius 4..8, porosity 0.35..0.45,
viscosity ratio in {1, 5, 10, 50}, contact angle in {30, 60, 90, 120} deg)
stepped together as one batch (three launches per step for all samples, CUDA
graph replay, autotuned block size), next to the same samples stepped one
after another as solo lattices; aggregate MLUPS over all fluid nodes.
"""
import argparse
import hashlib
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

METRIC = "MLUPS (2-component D3Q19)"
UNIT = "MLUPS"
# algorithmic bytes per fluid-node update: the 18 moving population pairs and
# the rest pair, read once and written once, plus the node's voxel index
ALGO_BYTES = {"fp32": 2 * (18 * 8 + 8) + 4, "fp64": 2 * (18 * 16 + 16) + 4,
              "fp16dev": 2 * (18 * 4 + 8) + 4, "bf16dev": 2 * (18 * 4 + 8) + 4}
DTYPE = {"fp32": "f32", "fp64": "f64", "fp16dev": "f32 (f16 storage)", "bf16dev": "f32 (bf16 storage)"}
WORKLOAD = "drainage_pack_128"
# algorithmic bytes per fluid node and time step of the reverse-mode job
# (record + reverse): the recorded forward step, then in the reverse sweep
# the recomputed step, the recomputed state stored and read back, and the
# adjoint population pairs read and written, plus the node's voxel index
ADJ_BYTES = 308 + 304 + 304 + 304 + 4
NOMINAL_HBM_GBS = 7900.0  # GB300 HBM3e, nominal


def workload_setup():
    from paper_2207_01534_gb300 import inputs

    solid, r1, r2 = inputs.drainage_pack_128()
    tau = inputs.tau_for_viscosity_ratio(10.0)
    xi = inputs.xi_of_theta(45.0)
    # inlet density of component 1 for a capillary pressure Pc = P_in - P_out of
    # 0.02 with the Eq. 12 pressure (inlet: rho2 ~ 0.03; outlet: rho2 = 1, rho1 ~ 0.03)
    G, minor, pc = 3.5, 0.03, 0.02
    rho_in1 = _pc_inlet(G, minor, pc)
    kw = dict(tau=tau, G=G, xi=xi, periodic=(1, 1, 0), open_axis=2, rho_in1=rho_in1, rho_out2=1.0)
    cfg = {"workload": WORKLOAD, "grid": [128, 128, 128], "sphere_radius": 8, "porosity": 0.38, "reservoir": 8,
           "M": 10, "theta_deg": 45, "G": G, "Pc": pc, "n_fluid": int((solid == 0).sum()),
           "lups_basis": "fluid nodes", "l2": "inputs larger than L2 (populations alone 146 MB)"}
    return solid, r1, r2, kw, cfg


BATCH_WORKLOAD = "batched_sweep_64"
ADJOINT_WORKLOAD = "adjoint_pack_96"


def _pc_inlet(G=3.5, minor=0.03, pc=0.02):
    from paper_2207_01534_gb300 import drivers

    return drivers.inlet_density(pc, G, minor, 1.0)


def batch_setup(count=64, edges=(48, 112)):
    """Geometries of the batched sweep, built in a spawn pool of host processes."""
    import concurrent.futures as cf
    import multiprocessing as mp

    from paper_2207_01534_gb300 import inputs

    specs = inputs.batched_sweep(count, edge_lo=edges[0], edge_hi=edges[1])
    workers = min(len(specs), os.cpu_count() or 1)
    with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        geo = list(ex.map(inputs.batched_sample, specs))
    samples, states = [], []
    for spec, (solid, r1, r2) in zip(specs, geo):
        samples.append(dict(solid=solid, tau=inputs.tau_for_viscosity_ratio(spec["M"]), G=3.5,
                            xi=inputs.xi_of_theta(spec["theta_deg"]), periodic=(1, 1, 0), open_axis=2,
                            rho_in1=_pc_inlet(), rho_out2=1.0))
        states.append((r1, r2))
    nf = [int((kw["solid"] == 0).sum()) for kw in samples]
    name = BATCH_WORKLOAD if (count, tuple(edges)) == (64, (48, 112)) else "batched_sweep_%d_edges_%d_%d" % (
        count, edges[0], edges[1])
    cfg = {"workload": name, "samples": len(specs), "edges": [sp["n"] for sp in specs],
           "n_fluid_total": int(sum(nf)), "n_voxels_total": int(sum(kw["solid"].size for kw in samples)),
           "M": sorted({sp["M"] for sp in specs}), "theta_deg": sorted({sp["theta_deg"] for sp in specs}),
           "Pc": 0.02, "reservoir": 6, "lups_basis": "fluid nodes",
           "l2": "inputs larger than L2 (populations of all samples exceed 1 GB)"}
    return samples, states, cfg


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def snapshot(self):
        """One reading now (besides the periodic ones): taken right after the
        timed steps are enqueued it sees the GPU under load even when the
        timed region is shorter than the sampling period."""
        try:
            r = subprocess.run(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=10)
            for line in r.stdout.splitlines():
                if line.strip():
                    self.rows.append([c.strip() for c in line.split(",")])
        except (OSError, subprocess.SubprocessError):
            pass

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.th.join(timeout=2)
        sm = [float(r[1]) for r in self.rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({names[k] for r in self.rows if len(r) >= 9 for k in range(4) if r[5 + k] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(sm)}


# the files that define and instantiate the split passes (k_dens, k_wall,
# k_fused) whose DRAM traffic profiles/traffic.json records
TRAFFIC_SOURCES = ("lbm_internal.h", "lbm_kernels.cuh", "lbm_ops.inl", "lbm_fp32.cu", "lbm_fp64.cu", "lbm_fp16.cu",
                   "lbm_bf16.cu", "lbm_fixed.cuh", "lbm_push.cuh", "lbm_push.cu")


def kernel_source_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2207_01534_gb300", "csrc")
    for f in TRAFFIC_SOURCES:
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic(kernel, storage):
    """DRAM bytes per launch of `kernel` with `storage` from the committed ncu
    summary, or None when there is none for the current kernel sources."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
    except (OSError, ValueError):
        return None
    e = d.get(WORKLOAD, {}).get(storage, {}).get(kernel)
    if not e or e.get("source_hash") != kernel_source_hash():
        return None
    return e.get("dram_bytes_per_launch")


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback"


def oracle_rate(solid, r1, r2, kw, steps, budget_s=30.0):
    """The FP64 oracle on the host cores: MLUPS over fluid nodes."""
    import oracle

    o = oracle.Oracle(solid, **kw)
    o.init_densities(r1, r2)
    o.step(1)  # first touch
    t0 = time.perf_counter()
    done = 0
    while done < steps and (time.perf_counter() - t0) < budget_s:
        o.step(1)
        done += 1
    dt = time.perf_counter() - t0
    nf = int((solid == 0).sum())
    return nf * done / dt / 1e6, done, dt


def reference_sample(solid, r1, r2, kw, total_steps, budget_updates=6e8):
    """The workload itself when total_steps full oracle steps stay within the
    budget of node updates (about two minutes of the oracle on 16 cores), else
    the largest centred cubic crop of it (8-slice reservoirs, drainage start)
    that does."""
    from paper_2207_01534_gb300 import inputs

    nf = int((solid == 0).sum())
    if nf * total_steps <= budget_updates:
        return solid, r1, r2, "the whole %s lattice" % WORKLOAD
    for n in range(min(solid.shape) - 16, 15, -16):
        c = inputs.crop(solid, n, reservoir=8)
        if int((c == 0).sum()) * total_steps <= budget_updates:
            c1, c2 = inputs.drainage_init(c, 8)
            return c, c1, c2, "a centred %d^3 crop of the %s lattice (8-slice reservoirs)" % (n, WORKLOAD)
    c = inputs.crop(solid, 16, reservoir=4)
    c1, c2 = inputs.drainage_init(c, 4)
    return c, c1, c2, "a centred 16^3 crop of the %s lattice" % WORKLOAD


# ---- ranks: one process per GPU, each stepping its own replica of the
# workload (no data exchange); the job's time is the slowest rank's and its
# value counts the units of every rank

def dist_init(world, backend="nccl"):
    """The process group for world > 1 ranks (MASTER_ADDR / MASTER_PORT / RANK /
    WORLD_SIZE from the environment); None for one rank."""
    if world <= 1:
        return None
    import torch.distributed as dist

    dist.init_process_group(backend)
    return dist


def barrier(dist):
    if dist is not None:
        dist.barrier()


def max_over_ranks(dist, ms, device):
    """The slowest rank's value of ms (every rank receives it)."""
    if dist is None:
        return ms
    import torch

    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, world, ms):
    """Millions of units per second over all ranks: every rank processed
    units_per_rank within the job time ms (milliseconds)."""
    return units_per_rank * world / (ms / 1e3) / 1e6


def dist_finish(dist):
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


def run_reference(args, rank, world):
    if rank != 0:  # the oracle runs once, on rank 0's host cores
        return
    solid, r1, r2, kw, cfg = workload_setup()
    cores = os.cpu_count() or 1
    solid, r1, r2, what = reference_sample(solid, r1, r2, kw, args.steps + max(args.warmup, 0))
    nf = int((solid == 0).sum())
    import oracle

    o = oracle.Oracle(solid, **kw)
    o.init_densities(r1, r2)
    o.step(max(args.warmup, 0))
    t0 = time.perf_counter()
    o.step(args.steps)
    dt = time.perf_counter() - t0
    v = nf * args.steps / dt / 1e6
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": cfg, "impl": "reference",
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "each step: one FP64 oracle step of %s (%d fluid nodes)" % (what, nf)},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def form_rate(lbm, solid, r1, r2, kw, nf, storage, kernel, steps, warmup=50):
    """One storage form or schedule on the headline workload: MLUPS over
    `steps` graph-replayed steps (CUDA events on the lattice's stream) and
    the collide-stream pass's device time from event-timed steps."""
    import torch

    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        lat = lbm.Lattice(solid, kernel=kernel, storage=storage, stream=stream.cuda_stream, **kw)
        lat.init_densities(r1, r2)
        lat.step(warmup)
        lat.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        lat.step(steps)
        ev1.record(stream)
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1)
        kms = lat.step_timed(200) / 200
        lat.synchronize()
        lat.close()
    peak, _ = peaks()
    algo = ALGO_BYTES[storage]
    out = {"value": nf * steps / (ms / 1e3) / 1e6, "unit": UNIT, "ms_per_step": ms / steps, "steps": steps,
           "storage": storage, "kernel_schedule": kernel,
           "step_frac": algo * nf / (ms / steps / 1e3) / 1e9 / peak}
    if kms[2] > 0:
        out["collide_stream_ms"] = float(kms[2])
        out["collide_stream_frac"] = algo * nf / (float(kms[2]) / 1e3) / 1e9 / peak
    return out


def other_forms(args, lbm, solid, r1, r2, kw, nf, value, dist, local):
    """The 16-bit storage forms, the push schedule, the batched sweep and the
    adjoint, each measured after the headline FP32 number in the same run on
    the same GPU and reported against it."""
    forms = {"basis": "measured after the headline number, same run and GPU; each form on its own stream with "
                      "inputs resident; ratios against the headline FP32 split-schedule value"}
    for st in ("fp16dev", "bf16dev"):
        f = form_rate(lbm, solid, r1, r2, kw, nf, st, "auto", 2000)
        f["over_fp32"] = f["value"] / value
        forms[st] = f
    f = form_rate(lbm, solid, r1, r2, kw, nf, "fp32", "push", 2000)
    f["over_split"] = f["value"] / value
    forms["push"] = f
    sub = argparse.Namespace(**vars(args))
    sub.steps, sub.warmup, sub.storage = 100, 10, "fp32"
    b = batch_line(sub, 1, dist, local)
    forms["batch"] = {"workload": BATCH_WORKLOAD, "value": b["value"], "unit": UNIT, "steps": sub.steps,
                      "samples": b["config"].get("samples", args.batch_count),
                      "batch_over_solo": b["config"]["batch_over_solo"],
                      "solo_sequential_mlups": b["config"]["solo_sequential_mlups"],
                      "step_frac": b["roofline"]["frac"]}
    # the same batch stepped by one persistent cooperative launch per 256 steps
    sub.kernel = "persistent"
    bp = batch_line(sub, 1, dist, local, solo=False)
    forms["batch_persistent"] = {"workload": BATCH_WORKLOAD, "value": bp["value"], "unit": UNIT, "steps": sub.steps,
                                 "gpu_launches": bp["gpu_launches"], "over_batch": bp["value"] / b["value"],
                                 "over_solo": bp["value"] / b["config"]["solo_sequential_mlups"]}
    a = adjoint_line(args, 1, dist, local)
    forms["adjoint"] = {"workload": ADJOINT_WORKLOAD, "value": a["value"], "unit": UNIT, "steps": a["steps"],
                        "adjoint_over_forward_time": a["config"]["adjoint_over_forward_time"],
                        "forward_steps_per_s": a["config"]["forward_steps_per_s"],
                        "roofline_frac": a["roofline"]["frac"],
                        "algorithmic_bytes_per_node_step": ADJ_BYTES}
    return forms


def run_ours(args, rank, world):
    import torch

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = dist_init(world)
    from paper_2207_01534_gb300 import lbm

    lbm.load()
    solid, r1, r2, kw, cfg = workload_setup()
    nf = cfg["n_fluid"]
    nvox = solid.size
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        lat = lbm.Lattice(solid, kernel=args.kernel, storage=args.storage, stream=stream.cuda_stream, **kw)
        lat.init_densities(r1, r2)
        lat.step(args.warmup)
        lat.synchronize()

        # device-timed region: K steps on the context stream, inputs resident
        clocks = ClockSampler(local)
        l0 = lat.info()["launches"]
        barrier(dist)
        torch.cuda.synchronize()
        clocks.start()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        lat.step(args.steps)
        ev1.record(stream)
        clocks.snapshot()  # the steps are enqueued: the GPU is running them
        torch.cuda.synchronize()
        clocks.snapshot()
        clk = clocks.stop()
        launches = lat.info()["launches"] - l0
        ms = max_over_ranks(dist, ev0.elapsed_time(ev1), "cuda")
        sat = lat.saturation()
        assert np.isfinite(sat).all(), sat

        # per-kernel device time (events around each launch) over up to 1000 steps
        nt = min(args.steps, 1000)
        kms = lat.step_timed(nt) / nt
        lat.synchronize()
    names = ("dens", "wall", "fused", "plane", "pipeline")
    dominant = names[int(np.argmax(kms))]
    value = whole_job_rate(nf * args.steps, world, ms)
    peak, peak_kind = peaks()
    fused_ms = float(kms[2]) if kms[2] > 0 else float(kms.max())
    algo = ALGO_BYTES[args.storage]
    achieved = algo * nf / (fused_ms / 1e3) / 1e9
    step_bytes_rate = algo * nf / (ms / args.steps / 1e3) / 1e9
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": measured_traffic({"auto": "k_fused", "split": "k_fused", "push": "k_fused_push"}.get(args.kernel),
                                        args.storage),
            "kernel": {"brick": "k_brick", "push": "k_fused_push", "fused": "k_pipe", "flow": "k_flow"}.get(args.kernel,
                                                                                                         "k_fused"),
            "peak_kind": peak_kind,
            "peak_nominal": NOMINAL_HBM_GBS, "frac_nominal": achieved / NOMINAL_HBM_GBS,
            "algorithmic_bytes_per_node": algo, "kernel_ms": {names[k]: float(kms[k]) for k in range(5)},
            "step_frac": step_bytes_rate / peak}
    del lat
    torch.cuda.synchronize()

    # end to end through the public API with host buffers: create (geometry
    # upload), initial densities upload, K steps, fields and saturation read
    # back.  The inputs sit in pinned host memory (the binding passes
    # contiguous arrays through, so the library copies from these buffers).
    solid_h = torch.from_numpy(np.ascontiguousarray(solid, dtype=np.uint8)).pin_memory().numpy()
    r1_h = torch.from_numpy(np.ascontiguousarray(r1, dtype=np.float64)).pin_memory().numpy()
    r2_h = torch.from_numpy(np.ascontiguousarray(r2, dtype=np.float64)).pin_memory().numpy()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lat2 = lbm.Lattice(solid_h, kernel=args.kernel, storage=args.storage, **kw)
    lat2.init_densities(r1_h, r2_h)
    lat2.step(args.steps)
    fields = lat2.fields(("rho1", "rho2"))
    s2 = lat2.saturation()
    dt = time.perf_counter() - t0
    del lat2, fields
    h2d = solid.nbytes + r1.nbytes + r2.nbytes
    d2h = 2 * nvox * 8 + 4 * 8
    e2e = {"value": nf * args.steps / dt / 1e6, "unit": UNIT, "h2d_bytes_per_step": h2d / args.steps,
           "d2h_bytes_per_step": d2h / args.steps}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle

        v, done, cdt = oracle_rate(solid, r1, r2, kw, steps=args.cpu_steps)
        oracle.set_threads(1)
        v1, done1, cdt1 = oracle_rate(solid, r1, r2, kw, steps=3, budget_s=15.0)
        oracle.set_threads(os.cpu_count() or 1)
        cpu = {"value": v, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
               "sample": "%d full steps of the %s workload (%.1f s); one core: %d steps (%.1f s)" % (
                   done, WORKLOAD, cdt, done1, cdt1),
               "value_one_core": v1}
    cfg = dict(cfg)
    cfg.update({"parallelism": "replicas" if world > 1 else "single", "kernel_schedule": args.kernel,
                "storage": args.storage,
                "voxel_mlups": nvox * args.steps * world / (ms / 1e3) / 1e6})
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": DTYPE[args.storage], "data": "synthetic", "config": cfg, "roofline": roof,
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches), "clocks": clk,
            "saturation": {"S_w": sat[0], "S_nw_smooth": sat[1]}}
    if world == 1 and not args.no_forms and args.kernel == "auto" and args.storage == "fp32":
        line["forms"] = other_forms(args, lbm, solid, r1, r2, kw, nf, value, dist, local)
    if rank == 0:
        print(json.dumps(line), flush=True)
    dist_finish(dist)


def run_batch(args, rank, world):
    import torch

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = dist_init(world)
    line = batch_line(args, world, dist, local)
    if rank == 0:
        print(json.dumps(line), flush=True)
    dist_finish(dist)


def batch_line(args, world, dist, local, solo=True):
    import tempfile

    samples, states, cfg = batch_setup(args.batch_count, tuple(args.batch_edges))
    import torch

    from paper_2207_01534_gb300 import lbm

    lbm.load()
    nf = cfg["n_fluid_total"]
    stream = torch.cuda.Stream()
    cache = args.tune_cache or os.path.join(tempfile.gettempdir(), "lbm_autotune.json")
    with torch.cuda.stream(stream):
        bkern = "persistent" if args.kernel == "persistent" else "split"
        b = lbm.Batch([dict(kw, storage=args.storage, kernel=bkern) for kw in samples], stream=stream.cuda_stream)
        for smp, (r1, r2) in zip(b.samples, states):
            smp.init_densities(r1, r2)
        b.step(args.warmup)
        block = b.autotune(cache)
        b.step(2)
        b.synchronize()
        clocks = ClockSampler(local)
        l0 = b.info()["launches"]
        barrier(dist)
        torch.cuda.synchronize()
        clocks.start()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        b.step(args.steps)
        ev1.record(stream)
        clocks.snapshot()
        torch.cuda.synchronize()
        clocks.snapshot()
        clk = clocks.stop()
        launches = b.info()["launches"] - l0
        ms = max_over_ranks(dist, ev0.elapsed_time(ev1), "cuda")
        sats = [smp.saturation() for smp in b.samples]
        assert np.isfinite(np.array(sats)).all()
        b.close()
        del b
        torch.cuda.synchronize()

        # the same samples as solo lattices stepped one after another
    # end to end through the public API with host buffers: create (geometry
    # upload), initial densities upload, K steps, fields and saturation read
    # back.  The inputs sit in pinned host memory (the binding passes
    # contiguous arrays through, so the library copies from these buffers).
    solid_h = torch.from_numpy(np.ascontiguousarray(solid, dtype=np.uint8)).pin_memory().numpy()
    r1_h = torch.from_numpy(np.ascontiguousarray(r1, dtype=np.float64)).pin_memory().numpy()
    r2_h = torch.from_numpy(np.ascontiguousarray(r2, dtype=np.float64)).pin_memory().numpy()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lat2 = lbm.Lattice(solid_h, kernel=args.kernel, storage=args.storage, **kw)
    lat2.init_densities(r1_h, r2_h)
    lat2.step(args.steps)
    fields = lat2.fields(("rho1", "rho2"))
    s2 = lat2.saturation()
    dt = time.perf_counter() - t0
    del lat2, fields
    h2d = solid.nbytes + r1.nbytes + r2.nbytes
    d2h = 2 * nvox * 8 + 4 * 8
    e2e = {"value": nf * args.steps / dt / 1e6, "unit": UNIT, "h2d_bytes_per_step": h2d / args.steps,
           "d2h_bytes_per_step": d2h / args.steps}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle

        v, done, cdt = oracle_rate(solid, r1, r2, kw, steps=args.cpu_steps)
        oracle.set_threads(1)
        v1, done1, cdt1 = oracle_rate(solid, r1, r2, kw, steps=3, budget_s=15.0)
        oracle.set_threads(os.cpu_count() or 1)
        cpu = {"value": v, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
               "sample": "%d full steps of the %s workload (%.1f s); one core: %d steps (%.1f s)" % (
                   done, WORKLOAD, cdt, done1, cdt1),
               "value_one_core": v1}
    cfg = dict(cfg)
    cfg.update({"parallelism": "replicas" if world > 1 else "single", "kernel_schedule": args.kernel,
                "storage": args.storage,
                "voxel_mlups": nvox * args.steps * world / (ms / 1e3) / 1e6})
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": DTYPE[args.storage], "data": "synthetic", "config": cfg, "roofline": roof,
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches), "clocks": clk,
            "saturation": {"S_w": sat[0], "S_nw_smooth": sat[1]}}
    if world == 1 and not args.no_forms and args.kernel == "auto" and args.storage == "fp32":
        line["forms"] = other_forms(args, lbm, solid, r1, r2, kw, nf, value, dist, local)
    if rank == 0:
        print(json.dumps(line), flush=True)
    dist_finish(dist)


def run_batch(args, rank, world):
    import torch

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = dist_init(world)
    line = batch_line(args, world, dist, local)
    if rank == 0:
        print(json.dumps(line), flush=True)
    dist_finish(dist)


def batch_line(args, world, dist, local, solo=True):
    import tempfile

    samples, states, cfg = batch_setup(args.batch_count, tuple(args.batch_edges))
    import torch

    from paper_2207_01534_gb300 import lbm

    lbm.load()
    nf = cfg["n_fluid_total"]
    stream = torch.cuda.Stream()
    cache = args.tune_cache or os.path.join(tempfile.gettempdir(), "lbm_autotune.json")
    with torch.cuda.stream(stream):
        bkern = "persistent" if args.kernel == "persistent" else "split"
        b = lbm.Batch([dict(kw, storage=args.storage, kernel=bkern) for kw in samples], stream=stream.cuda_stream)
        for smp, (r1, r2) in zip(b.samples, states):
            smp.init_densities(r1, r2)
        b.step(args.warmup)
        block = b.autotune(cache)
        b.step(2)
        b.synchronize()
        clocks = ClockSampler(local)
        l0 = b.info()["launches"]
        barrier(dist)
        torch.cuda.synchronize()
        clocks.start()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        b.step(args.steps)
        ev1.record(stream)
        clocks.snapshot()
        torch.cuda.synchronize()
        clocks.snapshot()
        clk = clocks.stop()
        launches = b.info()["launches"] - l0
        ms = max_over_ranks(dist, ev0.elapsed_time(ev1), "cuda")
        sats = [smp.saturation() for smp in b.samples]
        assert np.isfinite(np.array(sats)).all()
        b.close()
        del b
        torch.cuda.synchronize()

        # the same samples as solo lattices stepped one after another
        solo_runs = []
        for kw, (r1, r2) in zip(samples, states) if solo else []:
            g = lbm.Lattice(kernel="split", storage=args.storage, stream=stream.cuda_stream, **kw)
            g.init_densities(r1, r2)
            g.step(args.warmup + 2)
            solo_runs.append(g)
        torch.cuda.synchronize()
        ev0.record(stream)
        for g in solo_runs:
            g.step(args.steps)
        ev1.record(stream)
        torch.cuda.synchronize()
        ms_solo = ev0.elapsed_time(ev1) if solo else float("nan")
        for g in solo_runs:
            g.close()
        del solo_runs
        torch.cuda.synchronize()

    # end to end through the public API with host buffers
    t0 = time.perf_counter()
    b2 = lbm.Batch([dict(kw, storage=args.storage) for kw in samples])
    for smp, (r1, r2) in zip(b2.samples, states):
        smp.init_densities(r1, r2)
    b2.step(args.steps)
    s2 = [smp.saturation() for smp in b2.samples]
    dt = time.perf_counter() - t0
    b2.close()
    h2d = sum(kw["solid"].nbytes + r1.nbytes + r2.nbytes for kw, (r1, r2) in zip(samples, states))
    d2h = 32 * len(samples)
    value = whole_job_rate(nf * args.steps, world, ms)
    peak, peak_kind = peaks()
    algo = ALGO_BYTES[args.storage]
    achieved = algo * nf / (ms / args.steps / 1e3) / 1e9
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": None,
            "kernel": ("whole batched step (k_persist: all steps of a launch, grid barriers between the passes)"
                       if bkern == "persistent" else "whole batched step (k_dens_table + k_wall_table + k_fused_table)"),
            "peak_kind": peak_kind, "algorithmic_bytes_per_node": algo}
    cfg = dict(cfg)
    cfg.update({"parallelism": "replicas" if world > 1 else "single", "storage": args.storage, "block": block,
                "batch_schedule": bkern, "solo_sequential_mlups": nf * args.steps / (ms_solo / 1e3) / 1e6,
                "batch_over_solo": ms_solo / ms})
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": DTYPE[args.storage], "data": "synthetic", "config": cfg, "roofline": roof,
            "cpu_baseline": None, "gpu_launches": int(launches), "clocks": clk,
            "e2e": {"value": nf * args.steps / dt / 1e6, "unit": UNIT, "h2d_bytes_per_step": h2d / args.steps,
                    "d2h_bytes_per_step": d2h / args.steps}}
    return line


def run_adjoint(args, rank, world):
    import torch

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = dist_init(world)
    line = adjoint_line(args, world, dist, local)
    if rank == 0:
        print(json.dumps(line), flush=True)
    dist_finish(dist)


def adjoint_line(args, world, dist, local):
    import torch

    from paper_2207_01534_gb300 import inputs

    solid, r1, r2 = inputs.adjoint_pack_96()
    from paper_2207_01534_gb300 import lbm

    lbm.load()
    nsteps, every = args.adjoint_steps, min(args.checkpoint_every, args.adjoint_steps)
    nf = int((solid == 0).sum())
    kw = dict(tau=inputs.tau_for_viscosity_ratio(10.0), G=3.5, xi=inputs.xi_of_theta(45.0), periodic=(1, 1, 0),
              open_axis=2, rho_in1=_pc_inlet(pc=0.0), rho_out2=1.0, sample=(8, 88))
    stream = torch.cuda.Stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
    with torch.cuda.stream(stream):
        lat = lbm.Lattice(solid, storage="fp32", kernel="split", stream=stream.cuda_stream, **kw)
        gx = torch.zeros(solid.shape, dtype=torch.float32, device="cuda")
        # warm-up: one record + reverse pass of the timed length, so the
        # checkpoint, segment and density buffers are allocated before timing
        lat.init_densities(r1, r2)
        lat.record(nsteps, every)
        lat.adjoint(1.0, gx)
        barrier(dist)
        torch.cuda.synchronize()
        clocks = ClockSampler(local)
        clocks.start()
        lat.init_densities(r1, r2)
        l0 = lat.info()["launches"]
        ev[0].record(stream)
        lat.step(nsteps)
        ev[1].record(stream)
        clocks.snapshot()
        lat.init_densities(r1, r2)
        ev[2].record(stream)
        lat.record(nsteps, every)
        ev[3].record(stream)
        J, grin = lat.adjoint(1.0, gx)
        ev[4].record(stream)
        torch.cuda.synchronize()
        clocks.snapshot()
        clk = clocks.stop()
        launches = lat.info()["launches"] - l0
        t_fwd = ev[0].elapsed_time(ev[1]) / 1e3
        t_rec = ev[2].elapsed_time(ev[3]) / 1e3
        t_adj = ev[3].elapsed_time(ev[4]) / 1e3
        gmax = float(gx.abs().max())
        mem = lat.info()["device_bytes"]
    t_job = max_over_ranks(dist, (t_rec + t_adj) * 1e3, "cuda") / 1e3
    fwd_rate = nsteps / t_fwd
    adj_rate = nsteps / (t_rec + t_adj)
    value = whole_job_rate(nf * nsteps, world, t_job * 1e3)
    peak, peak_kind = peaks()
    achieved = ADJ_BYTES * nf * nsteps / (t_rec + t_adj) / 1e9
    cfg = {"workload": ADJOINT_WORKLOAD, "grid": [96, 96, 96], "sphere_radius": 6, "porosity": 0.40, "reservoir": 8,
           "steps": nsteps, "checkpoint_every": every, "n_fluid": nf, "M": 10, "theta_deg": 45, "Pc": 0.0,
           "loss": "smooth S_nw of the sample slab", "storage": "fp32", "parallelism": "replicas" if world > 1 else "single",
           "forward_steps_per_s": fwd_rate, "adjoint_steps_per_s": adj_rate,
           "adjoint_over_forward_time": (t_rec + t_adj) / t_fwd, "record_s": t_rec, "reverse_s": t_adj,
           "device_bytes": mem, "J": J, "dJ_drho_in1": grin, "max_abs_dJ_dxi": gmax,
           "l2": "inputs larger than L2 (checkpoints and segment states exceed 1 GB)"}
    line = {"metric": "adjoint MLUPS (forward record + reverse, 2-component D3Q19)", "value": value, "unit": UNIT,
            "n_gpus": world, "steps": nsteps, "warmup": 1, "ms_per_step": t_job * 1e3 / nsteps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": cfg, "gpu_launches": int(launches), "clocks": clk,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": None, "peak_kind": peak_kind,
                         "kernel": "record + reverse passes (forward, recompute, adjoint kernels)",
                         "algorithmic_bytes_per_node_step": ADJ_BYTES,
                         "bytes_basis": "record 308 (a forward step) + recompute 304 + segment state stored and "
                                        "read 304 + adjoint populations read and written 304 + voxel index 4"}}
    return line


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    # 6000 steps of the 128^3 workload take about 0.55 s: long enough for several
    # clock samples (every 200 ms) under load
    ap.add_argument("--steps", type=int, default=6000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", default="ours", choices=("ours", "reference"))
    ap.add_argument("--kernel", default="auto",
                    choices=("auto", "split", "flow", "fused", "wave", "push", "brick", "persistent"))
    ap.add_argument("--storage", default="fp32", choices=("fp32", "fp64", "fp16dev", "bf16dev"))
    ap.add_argument("--cpu-steps", type=int, default=60)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="skip the 16-bit, push, batch and adjoint forms")
    ap.add_argument("--workload", default=WORKLOAD, choices=(WORKLOAD, BATCH_WORKLOAD, ADJOINT_WORKLOAD))
    ap.add_argument("--tune-cache", default=None, help="autotuner JSON cache (batched workload)")
    ap.add_argument("--batch-count", type=int, default=64, help="samples (batched workload)")
    ap.add_argument("--batch-edges", type=int, nargs=2, default=(48, 112), help="edge range (batched workload)")
    ap.add_argument("--adjoint-steps", type=int, default=500, help="recorded steps (adjoint workload)")
    ap.add_argument("--checkpoint-every", type=int, default=50, help="checkpoint interval (adjoint workload)")
    args = ap.parse_args()
    assert args.warmup >= 0 and args.steps > 0
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.workload == BATCH_WORKLOAD:
        run_batch(args, rank, world)
    elif args.workload == ADJOINT_WORKLOAD:
        run_adjoint(args, rank, world)
    else:
        run_ours(args, rank, world)


if __name__ == "__main__":
    main()
