"""Learned surface surrogate around the IMPM simulator.

* ``generate``: runs seeded trajectories through the batched IMPM (one
  context, many instances, CUDA-graph stepping) and records, every
  ``every`` substeps, the indenter heightmap (tsim_read_indenter_height) and
  the surface displacement field (tsim_read_displacement) on a 128 x 128
  pixel window at dx/2 pitch, plus the pose and material scalars of the
  frame.  The frames stay on the device.  ``generate_chunks`` writes them
  to disk one batch of trajectories per file and resumes an interrupted
  run at the first missing chunk; ``load_chunks`` reads them back.
* ``features``: the network input of a set of frames, x[B,H,W,12] =
  [heightmap, pixel x, pixel y, press depth, slip x, slip y, rotation,
  E, nu, mu, press rate, tangential rate] (lengths in mm, scalars
  broadcast; the rates carry the loading speed, on which the dynamic part of
  the simulated response depends).
* ``train``: Adam on the masked displacement loss with the residual
  indicator channel (include/tsurr.h), all in the library's kernels.
* ``evaluate`` / ``serve``: per-frame error against the IMPM frames,
  the predicted error from the indicator channel, and the fallback rule:
  a frame whose predicted RMS error exceeds ``threshold`` x press depth is
  served by the simulator instead.
* ``foil``: a no-learning predictor (the penetration of the indenter into
  the undeformed surface, Gaussian-smoothed, as a vertical displacement)
  that the trained network is compared against.

The paper has no learned component; this is a project addition.  PyTorch
only holds device memory and assembles batches.
"""
from __future__ import annotations

import dataclasses
import json
import math
import os
import re
import time

import numpy as np

from . import inputs as I
from . import tsim as T
from . import tsurr as S

MM = 1e-3
CLIP = 2e-3            # heightmap clip (m): columns that miss the indenter read +2 mm
N_SCALARS = 9          # per-frame scalars broadcast as channels 3..11


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("the surrogate pipeline needs a CUDA device")
    return torch


def trajectory_state(kf: np.ndarray, k: float):
    """Tip (3) and yaw of the piecewise-linear keyframe trajectory at substep k."""
    kf = np.asarray(kf, np.float64)
    s = kf[:, 0]
    if k <= s[0]:
        row = kf[0, 1:]
    elif k >= s[-1]:
        row = kf[-1, 1:]
    else:
        j = int(np.searchsorted(s, k, side="right")) - 1
        a = (k - s[j]) / (s[j + 1] - s[j])
        row = (1 - a) * kf[j, 1:] + a * kf[j + 1, 1:]
    return row[:3], row[3]


RATE_LEVER = 3e-3      # rotation rate enters the tangential rate as the speed at 3 mm from the axis


def frame_scalars(scene: I.Scene, k: int) -> np.ndarray:
    """[press depth, slip x, slip y, rotation, E, nu, mu, press rate, tangential
    rate] at substep k, normalised: lengths in mm, material constants centred
    on their ranges, rates in mm per 1000 substeps over the substep ending at k
    (the tangential rate adds the slip speed and the rotation speed at
    RATE_LEVER from the axis)."""
    tip, yaw = trajectory_state(scene.keyframes, k)
    tip0, yaw0 = trajectory_state(scene.keyframes, 0)
    tipp, yawp = trajectory_state(scene.keyframes, k - 1)
    press = max(0.0, scene.gel.height - tip[2])
    m = scene.mat
    press_rate = (tipp[2] - tip[2]) / MM * 1e3
    tang_rate = (float(np.hypot(tip[0] - tipp[0], tip[1] - tipp[1])) + abs(yaw - yawp) * RATE_LEVER) / MM * 1e3
    return np.array([press / MM, (tip[0] - tip0[0]) / MM, (tip[1] - tip0[1]) / MM, yaw - yaw0,
                     (m.E - 1.9e5) / 1e5, (m.nu - 0.44) / 0.04, (scene.ind.mu - 0.6) / 0.4,
                     press_rate, tang_rate], np.float32)


@dataclasses.dataclass
class Frames:
    """A frame dataset on the device."""
    height: "object"          # [N, P, P] float32, indenter heightmap (mm)
    scalars: "object"         # [N, 9] float32
    disp: "object"            # [N, P, P, 3] float32, surface displacement (mm)
    press: np.ndarray         # [N] trajectory press depth (mm)
    traj: np.ndarray          # [N] trajectory index
    substep: np.ndarray       # [N]
    mpm_seconds: float = 0.0  # device time of the IMPM stepping that made them
    mpm_frames: int = 0

    def __len__(self):
        return int(self.press.shape[0])

    def subset(self, idx):
        idx = np.asarray(idx)
        torch = _torch()
        ti = torch.as_tensor(idx, device=self.height.device)
        return Frames(self.height[ti], self.scalars[ti], self.disp[ti], self.press[idx], self.traj[idx],
                      self.substep[idx], self.mpm_seconds, self.mpm_frames)


def _run_chunk(chunk, every, px, pitch, x_ref):
    """IMPM of one batch of trajectories; returns (H, U, seconds, passes per instance-substep)."""
    torch = _torch()
    nf = chunk[0].n_substeps // every
    H = torch.empty((len(chunk), nf, px, px), dtype=torch.float32, device="cuda")
    U = torch.empty((len(chunk), nf, px, px, 3), dtype=torch.float32, device="cuda")
    sim = T.Sim(chunk, use_graph=True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    secs = 0.0
    try:
        for f in range(nf):
            ev0.record()
            sim.step(every)
            ev1.record()
            ev1.synchronize()
            secs += ev0.elapsed_time(ev1) / 1e3
            for i in range(len(chunk)):
                T.tsim_read_indenter_height(sim.ctx, i, px, px, pitch, CLIP, out=H[i, f])
                T.tsim_read_displacement(sim.ctx, i, x_ref, px, px, pitch, out=U[i, f])
        st = T.tsim_stats(sim.ctx)
    finally:
        sim.close()
    return H, U, secs, st.passes / max(1, st.substeps) / len(chunk)


def generate(scenes, every: int = 100, batch: int = 64, log=None, retries: int = 3, traj0: int = 0,
             device: str = "cuda") -> Frames:
    """IMPM frames of ``scenes`` (all on the same pad), ``batch`` trajectories
    per context.  A trajectory whose simulation latches an error (the message
    names its instance) is left out and the rest of its batch is run again.
    Trajectory indices start at traj0."""
    torch = _torch()
    px = scenes[0].readout_px
    pitch = scenes[0].readout_pitch
    gel = scenes[0].gel
    x_ref = torch.from_numpy(np.ascontiguousarray(I.gel_particles(gel)[0])).to(device)
    hs, ss, us, pr, tr, sk = [], [], [], [], [], []
    mpm_s, mpm_frames, dropped = 0.0, 0, []
    for c0 in range(0, len(scenes), batch):
        ids = list(range(c0, min(len(scenes), c0 + batch)))
        nsub = scenes[ids[0]].n_substeps
        assert all(scenes[j].n_substeps == nsub and scenes[j].gel == gel for j in ids)
        nf = nsub // every
        for attempt in range(retries + 1):
            try:
                H, U, secs, passes = _run_chunk([scenes[j] for j in ids], every, px, pitch, x_ref)
                break
            except T.TsimError as e:
                m = re.search(r"instance (\d+)", str(e))
                if m is None or attempt == retries:
                    raise
                bad = ids.pop(int(m.group(1)))
                dropped.append(bad)
                if log:
                    log("trajectory %d left out: %s" % (bad, e))
        mpm_s += secs
        mpm_frames += nf * len(ids)
        for i, j in enumerate(ids):
            for f in range(nf):
                k = (f + 1) * every
                ss.append(frame_scalars(scenes[j], k))
                pr.append(scenes[j].meta.get("press", 0.0) / MM)
                tr.append(traj0 + j)
                sk.append(k)
        hs.append((H / MM).reshape(-1, px, px))
        us.append((U / MM).reshape(-1, px, px, 3))
        if log:
            log("generated %d/%d trajectories, %.1f s of IMPM, %.2f passes per instance-substep"
                % (ids[-1] + 1, len(scenes), mpm_s, passes))
    out = Frames(torch.cat(hs), torch.from_numpy(np.stack(ss)).to(device), torch.cat(us), np.array(pr, np.float64),
                 np.array(tr), np.array(sk), mpm_s, mpm_frames)
    out.dropped = [traj0 + j for j in dropped]
    return out


def generate_chunks(scenes, out_dir: str, every: int = 100, batch: int = 64, log=None, retries: int = 3,
                    device: str = "cuda"):
    """The frames of ``scenes`` written to out_dir as one file per batch of
    trajectories (chunk_00000.npz, ...; written to a temporary name, then
    renamed).  A chunk already on disk is kept, so an interrupted run resumes
    at the first missing chunk.  Returns the chunk paths."""
    os.makedirs(out_dir, exist_ok=True)
    paths = []
    for ci, c0 in enumerate(range(0, len(scenes), batch)):
        path = os.path.join(out_dir, "chunk_%05d.npz" % ci)
        paths.append(path)
        if os.path.exists(path):
            if log:
                log("chunk %d on disk, kept" % ci)
            continue
        fr = generate(scenes[c0:c0 + batch], every, batch, log, retries, traj0=c0, device=device)
        tmp = path + ".part.npz"
        np.savez(tmp, height=fr.height.cpu().numpy(), scalars=fr.scalars.cpu().numpy(), disp=fr.disp.cpu().numpy(),
                 press=fr.press, traj=fr.traj, substep=fr.substep, mpm_seconds=fr.mpm_seconds,
                 mpm_frames=fr.mpm_frames, dropped=np.array(fr.dropped, dtype=np.int64))
        os.replace(tmp, path)
    return paths


def load_chunks(out_dir: str, device: str = "cuda") -> Frames:
    """The frames of every chunk file in out_dir, in chunk order, on the device."""
    torch = _torch()
    files = sorted(f for f in os.listdir(out_dir) if f.startswith("chunk_") and f.endswith(".npz")
                   and not f.endswith(".part.npz"))
    zs = [np.load(os.path.join(out_dir, f)) for f in files]
    out = Frames(torch.from_numpy(np.concatenate([z["height"] for z in zs])).to(device),
                 torch.from_numpy(np.concatenate([z["scalars"] for z in zs])).to(device),
                 torch.from_numpy(np.concatenate([z["disp"] for z in zs])).to(device),
                 np.concatenate([z["press"] for z in zs]), np.concatenate([z["traj"] for z in zs]),
                 np.concatenate([z["substep"] for z in zs]), float(sum(float(z["mpm_seconds"]) for z in zs)),
                 int(sum(int(z["mpm_frames"]) for z in zs)))
    out.dropped = [int(j) for z in zs for j in z["dropped"]]
    return out


def features(fr: Frames, idx=None):
    """Network input x[B, P, P, 12] for frames ``idx`` (all when None),
    assembled by the library's kernel (tsurr_features)."""
    h = fr.height if idx is None else fr.height[idx]
    sc = fr.scalars if idx is None else fr.scalars[idx]
    return S.tsurr_features(h.contiguous(), sc.contiguous())


def train(fr: Frames, steps: int, batch: int = 32, lr: float = 1e-3, seed: int = 0, params=None, log=None,
          log_every: int = 1000, weight: str = "press", warmup: int = 200):
    """Train from ``params`` (seeded init when None); returns (params, losses).

    ``weight="press"`` weights each frame by 1/press_depth^2 (through the
    loss mask, normalised to mean 1 over the dataset) so that the loss
    follows the error measure, which is relative to the press depth."""
    torch = _torch()
    P = fr.height.shape[1]
    net = S.tsurr_create(batch, P, P)
    try:
        S.tsurr_set_params(net, S.init_params(seed) if params is None else params)
        if weight == "press":
            w = 1.0 / np.maximum(fr.press, 0.05) ** 2
            w = torch.as_tensor(w / w.mean(), dtype=torch.float32, device="cuda")
        else:
            w = torch.ones(len(fr), dtype=torch.float32, device="cuda")
        rng = np.random.default_rng(seed)
        losses = []
        t0 = time.time()
        for step in range(1, steps + 1):
            idx = torch.as_tensor(rng.integers(0, len(fr), batch), device="cuda")
            x = features(fr, idx)
            t = fr.disp[idx].contiguous()
            m = w[idx].view(batch, 1, 1).expand(batch, P, P).contiguous()
            losses.append(S.tsurr_backward(net, x, t, m))
            # linear warm-up, then cosine decay to 2 % of the peak rate
            c = 0.02 + 0.98 * 0.5 * (1 + math.cos(math.pi * (step - 1) / steps))
            lr_t = lr * min(1.0, step / max(1, warmup)) * c
            S.tsurr_adam(net, lr_t, 0.9, 0.999, 1e-8, step)
            if log and (step % log_every == 0 or step == steps):
                log("step %d loss %.5f (%.1f s)" % (step, float(np.mean(losses[-log_every:])), time.time() - t0))
        return S.tsurr_get_params(net), np.array(losses)
    finally:
        S.tsurr_destroy(net)


def predict(params, fr: Frames, batch: int = 256):
    """Network output y[N, P, P, 4] (mm) for all frames."""
    torch = _torch()
    P = fr.height.shape[1]
    net = S.tsurr_create(batch, P, P)
    try:
        S.tsurr_set_params(net, params)
        y = torch.empty((len(fr), P, P, 4), dtype=torch.float32, device="cuda")
        for a in range(0, len(fr), batch):
            idx = torch.arange(a, min(len(fr), a + batch), device="cuda")
            S.tsurr_forward(net, features(fr, idx), out=y[a:a + idx.numel()])
        torch.cuda.synchronize()
        return y
    finally:
        S.tsurr_destroy(net)


def frame_errors(pred, fr: Frames):
    """Per-frame RMS over the pixels of |u_pred - u_IMPM|, divided by the
    trajectory's press depth."""
    torch = _torch()
    d = pred[..., :3] - fr.disp
    rms = torch.sqrt((d * d).sum(-1).mean(dim=(1, 2))).cpu().numpy()
    return rms / fr.press


def indicator(pred, fr: Frames):
    """Predicted per-frame RMS error (indicator channel), divided by press
    depth, reduced by the library's kernel (tsurr_indicator)."""
    torch = _torch()
    press = torch.as_tensor(np.asarray(fr.press, np.float32), device=pred.device)
    return S.tsurr_indicator(pred.contiguous(), press).cpu().numpy().astype(np.float64)


def foil(fr: Frames, sigma_px: float):
    """No-learning prediction: u_z = -(Gaussian-smoothed indenter penetration)."""
    torch = _torch()
    pen = torch.clamp(-fr.height, min=0.0).unsqueeze(1)
    r = max(1, int(math.ceil(3 * sigma_px)))
    g = torch.exp(-0.5 * (torch.arange(-r, r + 1, device="cuda", dtype=torch.float32) / sigma_px) ** 2)
    g = g / g.sum()
    import torch.nn.functional as F
    sm = F.conv2d(F.pad(pen, (r, r, 0, 0), mode="replicate"), g.view(1, 1, 1, -1))
    sm = F.conv2d(F.pad(sm, (0, 0, r, r), mode="replicate"), g.view(1, 1, -1, 1))
    out = torch.zeros((len(fr),) + tuple(fr.height.shape[1:]) + (4,), device="cuda")
    out[..., 2] = -sm[:, 0]
    return out


def fit_foil(fr: Frames, sigmas=(0.5, 1, 2, 3, 4, 6, 8, 12)):
    """The foil's one parameter, chosen by its error on ``fr``."""
    best = None
    for s in sigmas:
        e = float(np.median(frame_errors(foil(fr, s), fr)))
        if best is None or e < best[1]:
            best = (s, e)
    return best[0]


def serve_summary(err, ind, threshold: float = 0.02):
    """Fallback rule and the error of what is served: frames whose indicator
    exceeds ``threshold`` go to the simulator (served error 0)."""
    fb = ind > threshold
    served = np.where(fb, 0.0, err)
    return dict(n=int(err.size), fallback_frac=float(fb.mean()), served_within=float((served <= threshold).mean()),
                surrogate_within=float((err <= threshold).mean()), median_err=float(np.median(err)),
                p90_err=float(np.percentile(err, 90)), max_served_err=float(served.max()))


def served_seconds(fallback, traj, substep, every: int, surr_fps: float, mpm_fps: float) -> float:
    """Time to serve all frames when the flagged ones fall back to IMPM: every
    frame pays its network inference (1/surr_fps), and a trajectory with a
    fallback frame pays IMPM for its whole prefix up to its last flagged
    frame ((substep / every) frames at 1/mpm_fps each; earlier flagged frames
    of the same trajectory come out of that run)."""
    fallback = np.asarray(fallback, bool)
    traj = np.asarray(traj)
    frames = np.asarray(substep) // every
    t = fallback.size / surr_fps
    for j in np.unique(traj[fallback]):
        t += frames[fallback & (traj == j)].max() / mpm_fps
    return float(t)


def time_inference(params, P: int = 128, batch: int = 256, reps: int = 20, warmup: int = 3, seed: int = 0):
    """Seconds per batch of the network forward on device-resident inputs
    (CUDA events on the launching stream)."""
    torch = _torch()
    net = S.tsurr_create(batch, P, P)
    try:
        S.tsurr_set_params(net, params)
        x = torch.from_numpy(I.surrogate_batch(seed, batch, P, P)[0]).cuda()
        y = torch.empty((batch, P, P, 4), dtype=torch.float32, device="cuda")
        for _ in range(warmup):
            S.tsurr_forward(net, x, out=y)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            S.tsurr_forward(net, x, out=y)
        e1.record()
        e1.synchronize()
        return e0.elapsed_time(e1) / 1e3 / reps
    finally:
        S.tsurr_destroy(net)


def forward_flops(P: int = 128, stored: bool = False) -> float:
    """Multiply-add FLOPs of one P x P frame through the nine convolutions (2
    per multiply-add) on the real channels (12 inputs of the first layer, 4
    outputs of the last); stored=True counts the 16-wide padded input and
    output that the kernels compute."""
    tot, hw = 0.0, P * P
    sizes = [hw, hw / 4, hw / 16, hw / 64, hw / 64, hw / 16, hw / 4, hw, hw]
    last = len(I.SURR_CONVS) - 1
    for li, ((cin, cout), npix) in enumerate(zip(I.SURR_CONVS, sizes)):
        if not stored:
            cin = I.SURR_CIN if li == 0 else cin
            cout = I.SURR_COUT if li == last else cout
        tot += 2.0 * npix * cout * 9 * cin
    return tot


def save(path, params, meta: dict):
    np.savez_compressed(path, params=np.asarray(params, np.float32), meta=json.dumps(meta))


def load_params(path):
    z = np.load(path, allow_pickle=False)
    return z["params"], json.loads(str(z["meta"]))
