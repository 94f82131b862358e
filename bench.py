"""Benchmark of the IMPM elastomer substep on GB300.

Workload: the 4,194,304-particle sensor pad (128x128x32 cells at dx =
0.3125 mm, sphere indenter, press 1 mm / slip 3 mm / rotate 30 deg over
20,000 substeps, 128x128 surface readout every 100 substeps).  One bench
step = 1000 IMPM substeps (every relative-rest pass of Algorithm 1
included) as ten frames of 100 substeps, each followed by its surface
readout; the default 20 steps time the whole trajectory from rest.  Metric:
particle-updates/s, one update = one particle through one P2G -> grid -> G2P
pass; the line also gives the rate per phase of the trajectory.

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
FRAMES_PER_STEP = 10           # one bench step: ten readout frames (1000 substeps of pad4m)
# algorithmic bytes of one particle-update (one particle through one P2G -> grid
# -> G2P pass): x, v, C, F (96 B) read and written
BYTES_PER_UPDATE = 192
# what the fused G2P2G layout must move at least: a commit pass reads and
# writes x and F (96 B); a repeat pass only reads them (48 B)
G2P2G_COMMIT = 96
G2P2G_REPEAT = 48


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


def _traffic(n_particles, kind):
    """DRAM bytes per launch of the commit or repeat transfer from the
    committed ncu summary, if it was taken on the current kernel source (else
    None)."""
    try:
        with open(os.path.join(ROOT, "profiles", "transfer_traffic.json")) as f:
            t = json.load(f)
        if t.get("kernel_hash") != _kernel_hash() or kind not in t:
            return None
        return float(t[kind]["dram_bytes_per_particle"]) * n_particles
    except Exception:
        return None


def _oracle_sample(scene, threads, max_seconds):
    """Substeps of the workload's scene from rest on the FP64 oracle until
    max_seconds have passed (at most 50 substeps); threads = 1 is the serial
    oracle, otherwise its all-cores variant with that many threads."""
    import oracle as O
    from paper_2405_02914_gb300 import inputs as I
    x, tag = I.gel_particles(scene.gel)
    v, C, F = I.rest_state(x.shape[0])
    st = O.State(x, v, C, F, tag)
    s, ind = O.make_scene(scene), O.make_indenter(scene.ind)
    done, passes, t0 = 0, 0, time.perf_counter()
    while True:
        if threads == 1:
            pl, _ = O.run(s, ind, scene.keyframes, done, 1, st)
        else:
            pl, _ = O.run_par(s, ind, scene.keyframes, done, 1, st, threads)
        done += 1
        passes += int(pl.sum())
        el = time.perf_counter() - t0
        if el > max_seconds or done >= 50:
            break
    return x.shape[0] * passes / el, done, passes, el, x.shape[0]


RENDER_SPP, RENDER_BOUNCES = 128, 4


def render_setup(height, scene):
    """LEDs, albedo and description of the sensor image of a readout."""
    from paper_2405_02914_gb300 import inputs as I
    H, W = height.shape
    pitch = scene.readout_pitch
    leds = I.sensor_leds(W, H, pitch, scene.gel.height, "gelsight")
    return leds, I.base_texture(W, H, seed=1), pitch


def render_leg(height, scene, stream, reps=5):
    """The sensor image (path tracing, 128 samples per pixel, 4 reflections)
    of the last frame's surface, CUDA events around each render."""
    import torch
    from paper_2405_02914_gb300 import tsim as T
    leds, alb, pitch = render_setup(height, scene)
    H, W = height.shape
    d = T.render_desc(leds, RENDER_SPP, RENDER_BOUNCES, 0.0, 1)
    ta = torch.from_numpy(alb).to(height.device)
    out = torch.empty((H, W, 3), device=height.device)
    T.tsim_render(height, ta, pitch, d, out, stream)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(reps + 1)]
    ev[0].record(stream)
    for r in range(reps):
        T.tsim_render(height, ta, pitch, d, out, stream)
        ev[r + 1].record(stream)
    torch.cuda.synchronize()
    ms = ev[0].elapsed_time(ev[-1]) / reps
    paths = W * H * RENDER_SPP
    return {"ms_per_frame": ms, "paths_per_s": paths / (ms * 1e-3), "frames_per_s": 1e3 / ms,
            "pixels": [W, H], "spp": RENDER_SPP, "max_bounces": RENDER_BOUNCES, "leds": "4 (red, green, blue, white)",
            "bound": "alu", "mean_rgb": [float(v) for v in out.mean(dim=(0, 1)).cpu()]}


def cpu_baseline(scene, max_seconds=12.0, height=None):
    """The FP64 oracle as it stands on the host cores: all cores (the record)
    and one core (nested), each on the first substeps of the same scene; with
    a height field also the oracle's sensor image of it (one core)."""
    import oracle as O
    render = None
    if height is not None:
        import numpy as np
        from oracle import render_oracle as RO
        leds, alb, pitch = render_setup(height, scene)
        spp = 8
        t0 = time.perf_counter()
        RO.render(np.asarray(height, dtype=np.float64), alb.astype(np.float64), pitch,
                  RO.make_desc(leds, spp, RENDER_BOUNCES, 0.0, 1))
        el = time.perf_counter() - t0
        paths = height.shape[0] * height.shape[1] * spp
        render = {"paths_per_s": paths / el, "cores": 1, "kind": "oracle",
                  "sample": "the same frame at %d samples per pixel (%d paths), FP64, %.2f s" % (spp, paths, el)}
    cores = O.threads()
    v1, d1, p1, e1, n = _oracle_sample(scene, 1, max_seconds)
    out1 = {"value": v1, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "first %d substeps (%d passes) of the %d-particle scene from rest, FP64 oracle, serial, "
                      "%.1f s" % (d1, p1, n, e1)}
    if cores <= 1:
        out1["nproc"] = os.cpu_count()
        if render:
            out1["render"] = render
        return out1
    va, da, pa, ea, _ = _oracle_sample(scene, cores, max_seconds)
    out = {"value": va, "unit": UNIT, "cores": cores, "kind": "oracle", "nproc": os.cpu_count(),
           "sample": "first %d substeps (%d passes) of the %d-particle scene from rest, FP64 oracle, all-cores "
                     "variant (%d threads, private grids summed in thread order), %.1f s" % (da, pa, n, cores, ea),
           "single_thread": out1}
    if render:
        out["render"] = render
    return out


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
    """The FP64 oracle as it stands on all host cores (rank 0 only): W warm-up
    substeps, then K timed substeps of the workload's scene from rest, one
    substep per step (a bounded sample of the GPU step)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle as O
    from paper_2405_02914_gb300 import inputs as I
    cores = O.threads()
    x, tag = I.gel_particles(scene.gel)
    v, C, F = I.rest_state(x.shape[0])
    st = O.State(x, v, C, F, tag)
    s, ind = O.make_scene(scene), O.make_indenter(scene.ind)
    k = 0
    for _ in range(args.warmup):
        O.run_par(s, ind, scene.keyframes, k, 1, st, cores)
        k += 1
    passes, t0 = 0, time.perf_counter()
    for _ in range(args.steps):
        pl, _ = O.run_par(s, ind, scene.keyframes, k, 1, st, cores)
        passes += int(pl.sum())
        k += 1
    el = time.perf_counter() - t0
    val = x.shape[0] * passes / el
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / max(args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "pad4m: 4,194,304-particle press-slip-rotate sensor pad",
                       "step": "1 IMPM substep (bounded sample of the GPU step of %d substeps)"
                               % (FRAMES_PER_STEP * scene.readout_every)},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle", "nproc": os.cpu_count(),
                             "sample": "%d substeps after %d warm-up substeps from rest, FP64 oracle, all-cores "
                                       "variant (%d threads)" % (args.steps, args.warmup, cores)},
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
    # a fallback frame pays IMPM for its trajectory's prefix up to that frame
    served = len(fr) / G.served_seconds(ind > threshold, fr.traj, fr.substep, 100, surr_fps, mpm_fps)
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


def batch_leg(n_sub=300, warm=60, tune=600):
    """The batched workload as an extra record: 64 uneven instances (grids
    48x48x12 .. 128x128x32, about 105M particles) in one context, CUDA-graph
    stepping with the autotuned launch configuration; particle-updates/s over
    n_sub substeps after warm-up (CUDA events on the stream)."""
    import torch
    from paper_2405_02914_gb300 import inputs as I
    from paper_2405_02914_gb300 import tsim as T
    scenes = I.batch_scenes(n=64, seed=0)
    stream = torch.cuda.current_stream()
    t0 = time.perf_counter()
    sim = T.Sim(scenes, stream=stream, use_graph=True)
    setup_s = time.perf_counter() - t0
    try:
        tuning = T.tsim_autotune(sim.ctx, tune)
        sim.step(warm)
        s0 = sim.stats()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.step(n_sub)
        e1.record(stream)
        torch.cuda.synchronize()
        T.tsim_sync(sim.ctx)
        s1 = sim.stats()
        ms = e0.elapsed_time(e1)
    finally:
        sim.close()
    n = sum(sc.gel.n_particles for sc in scenes)
    upd = s1.particle_updates - s0.particle_updates
    return {"value": upd / (ms * 1e-3), "unit": UNIT, "instances": len(scenes), "particles": n,
            "substeps_timed": n_sub, "after_substeps": tune + warm,
            "mean_passes_per_instance_substep": (s1.passes - s0.passes) / (n_sub * len(scenes)),
            "ms": ms, "setup_s": setup_s, "tuning": tuning, "spill_max": int(s1.spill_max)}


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


def profile_state(args, scene):
    """Profiling aid for a phase of the trajectory: --save-state advances the
    scene --at substeps (CUDA graph) and writes x, v, C, F to PATH (.npz);
    --load-state writes that state back, sets the substep counter to --at
    and runs --substeps substeps with kernels launched one by one (what a
    profiler can see), then prints the passes they took."""
    import numpy as np
    import torch
    from paper_2405_02914_gb300 import inputs as I
    from paper_2405_02914_gb300 import tsim as T
    torch.cuda.set_device(0)
    if args.save_state:
        sim = T.Sim(scene, use_graph=True)
        sim.step(args.at)
        T.tsim_sync(sim.ctx)
        x, v, C, F = sim.particles()
        sim.close()
        np.savez(args.save_state, x=x, v=v, C=C, F=F, at=args.at)
        print("saved the state at substep %d to %s" % (args.at, args.save_state))
        return
    z = np.load(args.load_state)
    if int(z["at"]) != args.at:
        raise SystemExit("the state was saved at substep %d, not %d" % (int(z["at"]), args.at))
    tag = I.gel_particles(scene.gel)[1]
    sim = T.Sim(scene, use_graph=False, states=[(z["x"], z["v"], z["C"], z["F"], tag)])
    T.tsim_set_substep(sim.ctx, args.at)
    sim.step(args.substeps)
    T.tsim_sync(sim.ctx)
    print("substeps %d..%d, passes %s" % (args.at, args.at + args.substeps - 1, sim.log(args.substeps)[0].tolist()))
    sim.close()


def _phases(kf):
    """Substep ranges of the trajectory's phases from its keyframes: the
    press, slip and rotation segments of press_slip_rotate, then the hold."""
    names = ["press", "slip", "rotate"]
    rows = [int(r[0]) for r in kf]
    out = []
    for i in range(len(rows) - 1):
        a, b = rows[i], rows[i + 1]
        d = kf[i + 1, 1:] - kf[i, 1:]
        if abs(d[3]) > 0:
            nm = "rotate"
        elif abs(d[0]) > 0 or abs(d[1]) > 0:
            nm = "slip"
        else:
            nm = "press" if i == 0 else names[min(i, 2)]
        out.append((nm, a, b))
    out.append(("hold", rows[-1], 1 << 40))
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="tsim", choices=["tsim", "reference"])
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="pad4m", choices=["pad4m", "press65k", "batch64", "large33m"])
    ap.add_argument("--no-surrogate", action="store_true", help="skip the surrogate vs IMPM frames/s leg")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end pass (profiling runs)")
    ap.add_argument("--no-batch", action="store_true", help="skip the 64-instance batched record")
    ap.add_argument("--no-render", action="store_true", help="skip the sensor-image (path tracing) leg")
    ap.add_argument("--render-only", action="store_true",
                    help="profiling aid: only the sensor image of a synthetic 128 x 128 pressed membrane")
    ap.add_argument("--autotune", type=int, default=600,
                    help="substeps of online launch-configuration tuning before the timed region (0: off)")
    ap.add_argument("--no-graph", action="store_true",
                    help="launch kernels one by one (profilers cannot see inside graphs with loops)")
    ap.add_argument("--save-state", metavar="PATH",
                    help="profiling aid: advance the workload's first scene --at substeps and save its state")
    ap.add_argument("--load-state", metavar="PATH",
                    help="profiling aid: load a saved state and run --substeps substeps from --at, kernel by kernel")
    ap.add_argument("--at", type=int, default=0)
    ap.add_argument("--substeps", type=int, default=3)
    ap.add_argument("--object-particles", action="store_true",
                    help="represent the indenter by particles (8 per cell) instead of its SDF contact")
    ap.add_argument("--mu-kinetic", type=float, default=0.0,
                    help="kinetic friction coefficient of the slip (0: the static one, the default workload)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    from paper_2405_02914_gb300 import inputs as I
    scenes, wl_desc = workload(args.workload, args.seed)
    if args.object_particles:
        from paper_2405_02914_gb300 import inputs as I
        scenes = [I.with_object_particles(sc) for sc in scenes]
        wl_desc += ", indenter as %d particles" % len(scenes[0].ind.obj)
    if args.mu_kinetic > 0:
        for sc in scenes:
            sc.ind.mu_k = min(args.mu_kinetic, sc.ind.mu)
        wl_desc += ", kinetic friction %g" % args.mu_kinetic
    scene = scenes[0]
    if args.impl == "reference":
        return run_reference(args, scene)
    if args.save_state or args.load_state:
        return profile_state(args, scene)
    if args.render_only:
        import numpy as np
        import torch
        n, p = scene.readout_px, scene.readout_pitch
        y, x = np.mgrid[0:n, 0:n]
        r2 = (((x + 0.5) - n / 2) ** 2 + ((y + 0.5) - n / 2) ** 2) * p ** 2
        h = scene.gel.height - 1e-3 * np.exp(-r2 / (2 * 3e-3 ** 2))         # a 1 mm press of a 3 mm radius
        frame = torch.from_numpy(np.ascontiguousarray(h, dtype=np.float32)).to("cuda:0")
        print(json.dumps({"render": render_leg(frame, scene, torch.cuda.current_stream())}), flush=True)
        return

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
    every = scene.readout_every
    sub_per_step = FRAMES_PER_STEP * every

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
        if sc.ind.obj is not None:
            T.tsim_set_object_particles(ctx, i, sc.ind.obj, sc.ind.obj_m)
        T.tsim_set_trajectory(ctx, i, sc.keyframes)
    T.tsim_use_graph(ctx, not args.no_graph)
    T.tsim_profile(ctx, True)
    outs = [(torch.empty((sc.readout_px, sc.readout_px), device=dev),
             torch.empty((sc.readout_px, sc.readout_px, 3), device=dev)) for sc in scenes]
    h_hosts = [torch.empty((sc.readout_px, sc.readout_px), pin_memory=True) for sc in scenes]
    n_hosts = [torch.empty((sc.readout_px, sc.readout_px, 3), pin_memory=True) for sc in scenes]

    def reset():
        T.tsim_set_substep(ctx, 0)
        for i in range(len(scenes)):
            T.tsim_write_particles(ctx, i, *d_in[i])

    def read_all(host=False):
        for i, sc in enumerate(scenes):
            h, nrm = (h_hosts[i], n_hosts[i]) if host else outs[i]
            T.tsim_read_surface(ctx, i, sc.readout_px, sc.readout_px, sc.readout_pitch, h, nrm)

    def one_step(events=None):
        # ten frames: `every` substeps, then the surface readout of the frame
        for _ in range(FRAMES_PER_STEP):
            T.tsim_step(ctx, every)
            read_all()
            if events is not None:
                e = torch.cuda.Event(enable_timing=True)
                e.record(stream)
                events.append(e)

    reset()
    for _ in range(args.warmup):
        one_step()
    tuning = T.tsim_get_tuning(ctx)
    if args.autotune > 0:
        tuning = T.tsim_autotune(ctx, args.autotune)
    reset()
    T.tsim_pass_time(ctx)                      # drop warm-up timings
    s0 = T.tsim_stats(ctx)

    clocks = ClockSampler(local)
    clocks.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    frame_ev = [e0]
    for _ in range(args.steps):
        one_step(frame_ev)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(frame_ev[-1])
    s1 = T.tsim_stats(ctx)
    commits, commit_ms, loop_ms = T.tsim_pass_time(ctx)
    T.tsim_sync(ctx)
    updates = s1.particle_updates - s0.particle_updates
    passes = s1.passes - s0.passes
    substeps = s1.substeps - s0.substeps
    per_sub = T.tsim_read_log(ctx, 0, int(substeps))[0].astype(np.int64) if substeps <= 32768 else None
    frame_ms = np.array([frame_ev[i].elapsed_time(frame_ev[i + 1]) for i in range(len(frame_ev) - 1)])
    n0 = scene.gel.n_particles
    phases = {}
    if per_sub is not None and len(scenes) == 1:
        for nm, a, b in _phases(scene.keyframes):
            f0, f1 = a // every, min(b, int(substeps)) // every
            if f1 <= f0:
                continue
            p = int(per_sub[f0 * every:f1 * every].sum())
            t = float(frame_ms[f0:f1].sum())
            ph = phases.setdefault(nm, {"substeps": 0, "passes": 0, "ms": 0.0})
            ph["substeps"] += (f1 - f0) * every
            ph["passes"] += p
            ph["ms"] += t
        for ph in phases.values():
            ph["mean_passes_per_substep"] = ph["passes"] / ph["substeps"]
            ph["particle_updates_per_s"] = n0 * ph["passes"] / (ph["ms"] * 1e-3)
            ph["particle_substeps_per_s"] = n0 * ph["substeps"] / (ph["ms"] * 1e-3)

    # end to end through the public API with host buffers (pinned): the
    # trajectory goes up and every frame's surface comes back each step
    e2e_s, e2e_updates, kf_hosts = 0.0, 0.0, [T.keyframes(sc.keyframes) for sc in scenes]
    if not args.no_e2e:
        def e2e_step():
            for i in range(len(scenes)):
                T.tsim_set_trajectory(ctx, i, kf_hosts[i])
            for _ in range(FRAMES_PER_STEP):
                T.tsim_step(ctx, every)
                read_all(host=True)

        T.tsim_profile(ctx, False)
        reset()
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
    repeat = passes - substeps * len(scenes)
    avg_commit_ms = commit_ms / max(commits, 1)
    avg_repeat_ms = loop_ms / max(repeat, 1) if repeat > 0 else None
    bytes_launch = n * BYTES_PER_UPDATE

    def roof(kernel, avg_ms, launches, total_ms, g2p2g_bytes, traffic):
        ach = bytes_launch / (avg_ms * 1e-3) / 1e9
        return {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                "traffic": traffic, "kernel": kernel, "launches_timed": int(launches), "avg_launch_ms": avg_ms,
                "total_ms": total_ms, "bytes_per_launch": bytes_launch,
                "bytes_per_particle_update": BYTES_PER_UPDATE,
                "g2p2g_bytes_per_particle": g2p2g_bytes,
                "frac_g2p2g_bytes": n * g2p2g_bytes / (avg_ms * 1e-3) / 1e9 / peak,
                "peak_source": peak_kind}

    r_commit = roof("k_transfer<COMMIT> (accepted pass: fused G2P -> F, x move -> re-bin -> P2G)", avg_commit_ms,
                    commits, commit_ms, G2P2G_COMMIT, _traffic(n, "commit"))
    rooflines = {"commit": r_commit}
    if avg_repeat_ms is not None:
        r_rep = roof("k_transfer<ITER> (repeat pass: fused G2P -> P2G; each timed pass includes its grid update "
                     "and check, CUDA events around the loop node)", avg_repeat_ms, repeat, loop_ms,
                     G2P2G_REPEAT, _traffic(n, "repeat"))
        rooflines["repeat"] = r_rep
    dom = max(rooflines.values(), key=lambda r: r["total_ms"])
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "%s, %d substeps per step (%d frames of %d substeps, each with its surface readout)"
                               % (wl_desc, sub_per_step, FRAMES_PER_STEP, every),
                   "instances": len(scenes),
                   "particles": n, "substeps_timed": int(substeps), "passes_timed": int(passes),
                   "mean_passes_per_substep": passes / max(substeps * len(scenes), 1),
                   "particle_substeps_per_s": n * substeps * world / (t_max * 1e-3),
                   "substep_ms": t_max / max(substeps, 1),
                   "phases": phases,
                   "parallelism": "replicas" if world > 1 else "single",
                   "l2": "inputs larger than L2 (particle state %d MB per parity)" % (n * 52 // 2 ** 20),
                   "tuning": tuning},
        "roofline": dict(dom),
        "rooflines": rooflines,
        "e2e": {"value": e2e_tot / e2e_max if e2e_max > 0 else None, "unit": UNIT,
                "h2d_bytes_per_step": sum(20 * len(k) for k in kf_hosts),
                "d2h_bytes_per_step": FRAMES_PER_STEP * sum(16 * sc.readout_px ** 2 for sc in scenes)},
        "gpu_launches": None,
        "clocks": clk,
    }
    # own kernels launched in the timed region: per substep round_begin, grid update
    # (with the check), commit transfer and its spill branch; per repeat pass transfer,
    # spill branch, grid update; per frame the step's end marker and 3 readout kernels
    # (and the object particles' P2G with each transfer when the indenter is particles)
    obj = 1 if any(sc.ind.obj is not None for sc in scenes) else 0
    line["gpu_launches"] = int((4 + obj) * substeps + (3 + obj) * max(repeat, 0) +
                               (1 + 3 * len(scenes)) * args.steps * FRAMES_PER_STEP) * world
    if args.workload != "pad4m":
        line["metric"] = UNIT + " (%s)" % args.workload
    if not args.no_batch and world == 1 and args.workload == "pad4m":
        try:
            line["batch64"] = batch_leg()
        except Exception as e:          # reported, never silently replaced by another path
            line["batch64"] = {"error": "%s: %s" % (type(e).__name__, e)}
    if not args.no_surrogate and world == 1:
        try:
            line["surrogate"] = surrogate_leg()
        except Exception as e:          # reported, never silently replaced by another path
            line["surrogate"] = {"error": "%s: %s" % (type(e).__name__, e)}
    frame = outs[0][0]
    if not args.no_render and world == 1:
        try:
            line["render"] = render_leg(frame, scene, stream)
        except Exception as e:          # reported, never silently replaced by another path
            line["render"] = {"error": "%s: %s" % (type(e).__name__, e)}
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(scene, height=None if args.no_render else frame.cpu().numpy())
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
