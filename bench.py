"""Benchmark of the IMPM elastomer substep on GB300.

Workload: the 4,194,304-particle sensor pad (128x128x32 cells at dx =
0.3125 mm, sphere indenter, press 1 mm / slip 3 mm / rotate 30 deg over
20,000 substeps, 128x128 surface readout every 100 substeps).  One bench
step = 100 IMPM substeps (every relative-rest pass of Algorithm 1 included)
plus the surface readout of that frame.  Metric: particle-updates/s, one
update = one particle through one P2G -> grid -> G2P pass.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun every rank runs its own replica of the pad (independent
instances shard with no data-path collective); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
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

METRIC = "MPM particle-updates/s (4.2M pts, FP32) & surrogate vs MPM frames/s at ≤2% err"
UNIT = "particle-updates/s"
SUBSTEPS_PER_STEP = 100
BYTES_PER_UPDATE = 96          # x (12 B) + F (36 B), read once and written once per committed update


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([a.strip() for a in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                for nm, val in zip(names, r[5:9]):
                    if val.lower().startswith("active"):
                        reasons.add(nm)
            except Exception:
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _kernel_hash():
    """Hash of the fused transfer kernel's source (its section of
    tsim_kernels.cu plus the device header it includes)."""
    csrc = os.path.join(ROOT, "paper_2405_02914_gb300", "csrc")
    k = open(os.path.join(csrc, "tsim_kernels.cu")).read()
    a, b = k.index("// ---------------------------------------------------------------- fused transfer"), \
        k.index("size_t transfer_smem_bytes()")
    h = hashlib.sha256(k[a:b].encode())
    h.update(open(os.path.join(csrc, "tsim_device.cuh"), "rb").read())
    return h.hexdigest()[:16]


def _traffic(n_particles):
    """DRAM bytes per commit launch from the committed ncu summary, if it was
    taken on the current kernel source (else None)."""
    try:
        with open(os.path.join(ROOT, "profiles", "transfer_commit_traffic.json")) as f:
            t = json.load(f)
        if t.get("kernel_hash") != _kernel_hash():
            return None
        return float(t["dram_bytes_per_particle"]) * n_particles
    except Exception:
        return None


def cpu_baseline(scene, max_seconds=15.0):
    """The FP64 oracle as it stands, single-threaded, on the first substeps."""
    import oracle as O
    from paper_2405_02914_gb300 import inputs as I
    x, tag = I.gel_particles(scene.gel)
    v, C, F = I.rest_state(x.shape[0])
    st = O.State(x, v, C, F, tag)
    s, ind = O.make_scene(scene), O.make_indenter(scene.ind)
    done, passes, t0 = 0, 0, time.perf_counter()
    while True:
        pl, _ = O.run(s, ind, scene.keyframes, done, 1, st)
        done += 1
        passes += int(pl.sum())
        el = time.perf_counter() - t0
        if el > max_seconds or done >= 50:
            break
    return {"value": x.shape[0] * passes / el, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "first %d substeps (%d passes) of a %d-particle scene of this workload, FP64 oracle, "
                      "serial, %.1f s" % (done, passes, x.shape[0], el)}


def aggregate_ranks(ms, e2e_s, updates, e2e_updates, world, device):
    """Whole-job figures of the replicas: the slowest rank's times (max) and
    the work of all ranks (sum); world = 1 returns the inputs."""
    if world <= 1:
        return ms, e2e_s, updates, e2e_updates
    import torch
    import torch.distributed as dist
    tt = torch.tensor([ms, e2e_s], device=device, dtype=torch.float64)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    uu = torch.tensor([updates, e2e_updates], device=device, dtype=torch.float64)
    dist.all_reduce(uu, op=dist.ReduceOp.SUM)
    return float(tt[0]), float(tt[1]), float(uu[0]), float(uu[1])


def run_reference(args, scene):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle as O
    from paper_2405_02914_gb300 import inputs as I
    x, tag = I.gel_particles(scene.gel)
    v, C, F = I.rest_state(x.shape[0])
    st = O.State(x, v, C, F, tag)
    s, ind = O.make_scene(scene), O.make_indenter(scene.ind)
    k = 0
    for _ in range(args.warmup):
        O.run(s, ind, scene.keyframes, k, 1, st)
        k += 1
    passes, t0 = 0, time.perf_counter()
    for _ in range(args.steps):
        pl, _ = O.run(s, ind, scene.keyframes, k, 1, st)
        passes += int(pl.sum())
        k += 1
    el = time.perf_counter() - t0
    val = x.shape[0] * passes / el
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / max(args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "pad4m: 4,194,304-particle press-slip-rotate sensor pad",
                       "step": "1 IMPM substep (bounded sample of the 100-substep GPU step)"},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": "%d substeps after %d warm-up substeps, FP64 oracle, serial"
                                       % (args.steps, args.warmup)},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


SURROGATE_WEIGHTS = os.path.join(ROOT, "paper_2405_02914_gb300", "weights", "surrogate_pad64.npz")


def surrogate_leg(n_traj=8, threshold=0.02):
    """Surrogate vs IMPM surface frames/s on held-out trajectories of the
    surrogate's pad (64x64x16 cells, 128x128 frames at dx/2 pitch every 100
    substeps): IMPM frames/s measured on the frames it makes here, network
    frames/s at inference batch 256 on device-resident inputs, per-frame error
    against those IMPM frames, and the frames/s served when frames whose
    predicted error exceeds ``threshold`` x press depth fall back to IMPM."""
    if not os.path.exists(SURROGATE_WEIGHTS):
        return {"unavailable": "no trained parameters at %s" % os.path.relpath(SURROGATE_WEIGHTS, ROOT)}
    import numpy as np
    from paper_2405_02914_gb300 import inputs as I
    from paper_2405_02914_gb300 import surrogate as G
    params, meta = G.load_params(SURROGATE_WEIGHTS)
    fr = G.generate(I.surrogate_scenes(n_traj, seed=1))
    mpm_fps = fr.mpm_frames / fr.mpm_seconds
    pred = G.predict(params, fr)
    err = G.frame_errors(pred, fr)
    ind = G.indicator(pred, fr)
    del pred
    summ = G.serve_summary(err, ind, threshold)
    t_batch = G.time_inference(params, batch=256)
    surr_fps = 256 / t_batch
    n_fb = summ["fallback_frac"] * len(fr)
    served = len(fr) / (len(fr) / surr_fps + n_fb / mpm_fps)
    tflops = G.forward_flops() * 256 / t_batch / 1e12
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peak, src = float(json.load(f)["bf16_tflops"]), "measured"
    except Exception:
        peak, src = 1900.0, "fallback"
    return {"frames_per_s": surr_fps, "mpm_frames_per_s": mpm_fps, "served_frames_per_s": served,
            "speedup_served": served / mpm_fps, "speedup_network": surr_fps / mpm_fps,
            "threshold": threshold, "frames": len(fr), "trajectories": n_traj, **summ,
            "inference_batch": 256, "frame": "128x128x3 displacement + indicator",
            "roofline": {"bound": "tensor", "achieved": tflops, "peak": peak, "unit": "TFLOP/s",
                         "frac": tflops / peak, "peak_source": src,
                         "kernel": "k_conv_fwd_tc (tcgen05.mma kind::f16, BF16 in, FP32 accumulate in TMEM), whole forward"},
            "weights": os.path.relpath(SURROGATE_WEIGHTS, ROOT), "trained": meta}


def workload(name, seed):
    """Scenes of a named workload and its description."""
    from paper_2405_02914_gb300 import inputs as I
    if name == "pad4m":
        return [I.scene_pad4m(seed=seed)], ("pad4m: 128x128x32 cells, dx=0.3125 mm, 4,194,304 particles, "
                                            "press-slip-rotate")
    if name == "press65k":
        return [I.scene_press65k()], "press65k: 32x32x8 cells, dx=0.625 mm, 65,536 particles, sphere press"
    if name == "large33m":
        return [I.scene_large33m()], ("large33m: 256x256x64 cells, dx=0.234375 mm, 33,554,432 particles, "
                                      "Perlin plate press-slip-rotate")
    sc = I.batch_scenes(n=64, seed=seed)
    n = sum(s.gel.n_particles for s in sc)
    return sc, "batch64: 64 instances, grids 48x48x12..128x128x32, %d particles, lockstep" % n


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="tsim", choices=["tsim", "reference"])
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="pad4m", choices=["pad4m", "press65k", "batch64", "large33m"])
    ap.add_argument("--no-surrogate", action="store_true", help="skip the surrogate vs IMPM frames/s leg")
    ap.add_argument("--autotune", type=int, default=600,
                    help="substeps of online launch-configuration tuning before the timed region (0: off)")
    ap.add_argument("--no-graph", action="store_true",
                    help="launch kernels one by one (profilers cannot see inside graphs with loops)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    from paper_2405_02914_gb300 import inputs as I
    scenes, wl_desc = workload(args.workload, args.seed)
    scene = scenes[0]
    if args.impl == "reference":
        return run_reference(args, scene)

    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_2405_02914_gb300 import tsim as T

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()

    # inputs resident in HBM before the timed region
    d_in = []
    for sc in scenes:
        x, tag = I.gel_particles(sc.gel)
        v, C, F = I.rest_state(x.shape[0])
        d_in.append([torch.from_numpy(a).to(dev) for a in (x, v, C, F)] +
                    [torch.from_numpy(tag.view(np.int32)).to(dev)])
        del x, tag, v, C, F
    n = sum(sc.gel.n_particles for sc in scenes)
    ctx = T.tsim_create([T.gel_desc(sc.gel) for sc in scenes], [T.material_desc(sc.mat) for sc in scenes],
                        stream)
    T.tsim_set_solver(ctx, T.solver_desc(scene.solver))
    for i, sc in enumerate(scenes):
        T.tsim_set_indenter(ctx, i, T.indenter_desc(sc.ind))
        T.tsim_set_trajectory(ctx, i, sc.keyframes)
    T.tsim_use_graph(ctx, not args.no_graph)
    T.tsim_profile(ctx, True)
    outs = [(torch.empty((sc.readout_px, sc.readout_px), device=dev),
             torch.empty((sc.readout_px, sc.readout_px, 3), device=dev)) for sc in scenes]

    def reset():
        T.tsim_set_substep(ctx, 0)
        for i in range(len(scenes)):
            T.tsim_write_particles(ctx, i, *d_in[i])

    def read_all(host=False):
        for i, sc in enumerate(scenes):
            h, nrm = (h_hosts[i], n_hosts[i]) if host else outs[i]
            T.tsim_read_surface(ctx, i, sc.readout_px, sc.readout_px, sc.readout_pitch, h, nrm)

    def one_step():
        T.tsim_step(ctx, SUBSTEPS_PER_STEP)
        read_all()

    reset()
    for _ in range(args.warmup):
        one_step()
    tuning = T.tsim_get_tuning(ctx)
    if args.autotune > 0:
        tuning = T.tsim_autotune(ctx, args.autotune)
    reset()
    T.tsim_kernel_time(ctx)                    # drop warm-up timings
    s0 = T.tsim_stats(ctx)

    clocks = ClockSampler(local)
    clocks.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        one_step()
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    s1 = T.tsim_stats(ctx)
    launches, k_ms = T.tsim_kernel_time(ctx)
    updates = s1.particle_updates - s0.particle_updates
    passes = s1.passes - s0.passes
    substeps = s1.substeps - s0.substeps

    # end to end through the public API with host buffers (pinned)
    kf_hosts = [T.keyframes(sc.keyframes) for sc in scenes]
    h_hosts = [torch.empty((sc.readout_px, sc.readout_px), pin_memory=True) for sc in scenes]
    n_hosts = [torch.empty((sc.readout_px, sc.readout_px, 3), pin_memory=True) for sc in scenes]

    def e2e_step():
        for i in range(len(scenes)):
            T.tsim_set_trajectory(ctx, i, kf_hosts[i])
        T.tsim_step(ctx, SUBSTEPS_PER_STEP)
        read_all(host=True)

    reset()
    T.tsim_profile(ctx, False)
    e2e_step()
    reset()
    s2 = T.tsim_stats(ctx)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        e2e_step()
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    s3 = T.tsim_stats(ctx)
    e2e_updates = s3.particle_updates - s2.particle_updates
    T.tsim_destroy(ctx)

    t_max, e2e_max, tot_updates, e2e_tot = aggregate_ranks(ms, e2e_s, updates, e2e_updates, world, dev)
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    value = tot_updates / (t_max * 1e-3)
    peak, peak_kind = _peaks()
    avg_commit_ms = k_ms / max(launches, 1)
    achieved = n * BYTES_PER_UPDATE / (avg_commit_ms * 1e-3) / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "%s, %d substeps + surface readout per step" % (wl_desc, SUBSTEPS_PER_STEP),
                   "instances": len(scenes),
                   "particles": n, "substeps_timed": int(substeps), "passes_timed": int(passes),
                   "mean_passes_per_substep": passes / max(substeps * len(scenes), 1),
                   "particle_substeps_per_s": n * substeps * world / (t_max * 1e-3),
                   "substep_ms": t_max / max(substeps, 1),
                   "parallelism": "replicas" if world > 1 else "single",
                   "l2": "inputs larger than L2 (particle state %d MB per parity)" % (n * 52 // 2 ** 20),
                   "tuning": tuning},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": _traffic(n),
                     "kernel": "k_transfer<COMMIT> (fused G2P -> F,x move -> re-bin -> P2G)",
                     "launches_timed": launches, "avg_launch_ms": avg_commit_ms,
                     "bytes_per_launch": n * BYTES_PER_UPDATE, "peak_source": peak_kind},
        "e2e": {"value": e2e_tot / e2e_max, "unit": UNIT,
                "h2d_bytes_per_step": sum(20 * len(k) for k in kf_hosts),
                "d2h_bytes_per_step": sum(16 * sc.readout_px ** 2 for sc in scenes)},
        "gpu_launches": None,
        "clocks": clk,
    }
    # own kernels launched in the timed region: per substep round_begin, grid, check,
    # commit transfer; per extra pass transfer, grid, check; per step 3 readout kernels
    extra = passes - substeps
    line["gpu_launches"] = int(4 * substeps + 3 * extra + 3 * args.steps * len(scenes)) * world
    if args.workload != "pad4m":
        line["metric"] = UNIT + " (%s)" % args.workload
    if not args.no_surrogate and world == 1:
        try:
            line["surrogate"] = surrogate_leg()
        except Exception as e:          # reported, never silently replaced by another path
            line["surrogate"] = {"error": "%s: %s" % (type(e).__name__, e)}
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(scene)
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
