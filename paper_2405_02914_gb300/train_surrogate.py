"""Generate IMPM frames, train the surface surrogate, evaluate it on held-out
trajectories and write the parameters plus a JSON report.

    python -m paper_2405_02914_gb300.train_surrogate --train 320 --test 64 \
        --variants 20000:1e-3:press --out weights.npz --report report.json

Training trajectories use dataset seed 0, held-out ones seed 1, so the two
sets never share a trajectory.  Each variant ``steps:lr:weighting`` trains
from the same seeded initialisation on the same frames; the one with the
lowest median held-out error is written to ``--out``.  ``--diag`` saves the
per-frame errors and trajectory parameters of the held-out set.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

from . import inputs as I
from . import surrogate as G


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=320, help="training trajectories")
    ap.add_argument("--test", type=int, default=64, help="held-out trajectories")
    ap.add_argument("--variants", default="20000:1e-3:press")
    ap.add_argument("--batch", type=int, default=32)
    ap.add_argument("--every", type=int, default=100, help="substeps between frames")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--init", default=None, help="start from these parameters (.npz)")
    ap.add_argument("--out", required=True)
    ap.add_argument("--report", required=True)
    ap.add_argument("--diag", default=None)
    ap.add_argument("--cache", default=None,
                    help="write the frames to this directory, one file per batch of trajectories, and resume "
                         "from the chunks already there")
    a = ap.parse_args(argv)

    def log(msg):
        print("[%7.1f s] %s" % (time.time() - t0, msg), flush=True)

    t0 = time.time()
    train_sc = I.surrogate_scenes(a.train, seed=0)
    test_sc = I.surrogate_scenes(a.test, seed=1)
    if a.cache:
        for name, sc in (("train", train_sc), ("test", test_sc)):
            G.generate_chunks(sc, os.path.join(a.cache, name), every=a.every, log=log)
        train_fr = G.load_chunks(os.path.join(a.cache, "train"))
        test_fr = G.load_chunks(os.path.join(a.cache, "test"))
    else:
        train_fr = G.generate(train_sc, every=a.every, log=log)
        test_fr = G.generate(test_sc, every=a.every, log=log)
    log("frames: %d training, %d held-out" % (len(train_fr), len(test_fr)))
    sigma = G.fit_foil(train_fr.subset(np.arange(0, len(train_fr), 7)))
    foil_err = G.frame_errors(G.foil(test_fr, sigma), test_fr)
    mpm_fps = test_fr.mpm_frames / test_fr.mpm_seconds
    init = G.load_params(a.init)[0] if a.init else None
    results, best = [], None
    for v in a.variants.split(","):
        steps, lr, weight = v.split(":")
        steps, lr = int(steps), float(lr)
        params, losses = G.train(train_fr, steps, batch=a.batch, lr=lr, seed=a.seed, params=init, log=log,
                                 weight=weight)
        pred = G.predict(params, test_fr)
        err = G.frame_errors(pred, test_fr)
        ind = G.indicator(pred, test_fr)
        del pred
        summ = G.serve_summary(err, ind)
        r = dict(variant=v, final_loss=float(np.mean(losses[-200:])), surrogate=summ,
                 gain_median=float(np.median(foil_err) / max(np.median(err), 1e-12)))
        log(json.dumps(r))
        results.append(r)
        if best is None or summ["median_err"] < best[0]:
            best = (summ["median_err"], params, err, ind, v, steps, lr, weight)
    _, params, err, ind, v, steps, lr, weight = best
    G.save(a.out, params, dict(variant=v, steps=steps, lr=lr, weight=weight, train=a.train, every=a.every,
                               batch=a.batch))
    t_batch = G.time_inference(params)
    surr_fps = 256 / t_batch
    summ = G.serve_summary(err, ind)
    n_fb = summ["fallback_frac"] * len(test_fr)
    eff_fps = len(test_fr) / (len(test_fr) / surr_fps + n_fb / mpm_fps)
    report = dict(train_trajectories=a.train, test_trajectories=a.test, train_frames=len(train_fr),
                  test_frames=len(test_fr), dropped=dict(train=train_fr.dropped, test=test_fr.dropped),
                  batch=a.batch, every=a.every, variants=results, chosen=v, surrogate=summ,
                  foil=dict(sigma_px=sigma, median_err=float(np.median(foil_err)),
                            within=float((foil_err <= 0.02).mean())),
                  gain_median=float(np.median(foil_err) / max(np.median(err), 1e-12)),
                  surrogate_frames_per_s=surr_fps, mpm_frames_per_s=mpm_fps, served_frames_per_s=eff_fps,
                  forward_tflops=G.forward_flops() * 256 / t_batch / 1e12,
                  mpm_seconds=dict(train=train_fr.mpm_seconds, test=test_fr.mpm_seconds),
                  wall_seconds=time.time() - t0)
    with open(a.report, "w") as f:
        json.dump(report, f, indent=1)
    if a.diag:
        meta = [test_sc[j].meta for j in test_fr.traj]
        np.savez_compressed(a.diag, err=err, ind=ind, foil=foil_err, substep=test_fr.substep, traj=test_fr.traj,
                            press=test_fr.press, kind=np.array([m["kind"] for m in meta]),
                            slip=np.array([m["slip"] for m in meta]), rot=np.array([m["rotate"] for m in meta]),
                            mu=np.array([m["mu"] for m in meta]), E=np.array([m["E"] for m in meta]),
                            nu=np.array([m["nu"] for m in meta]))
    log(json.dumps(report))
    return 0


if __name__ == "__main__":
    sys.exit(main())
