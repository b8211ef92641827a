"""Clustered visibility cache (Section 3.6) on the 16-room scene.

Clusters the lights with k-means, trains the clustered cache online for a
few frames, then runs inference and the two-step sampler with its shadow ray
on a top-down heightfield view and prints the time of each stage (CUDA
events) and the accumulated estimate's error against the exact DI.

    python -m paper_2506_05930_gb300.examples.clustered_frame --width 480 --height 270
"""
import argparse

import numpy as np
import torch

import nvc_synth as S
from paper_2506_05930_gb300 import nvc


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--width", type=int, default=1920)
    ap.add_argument("--height", type=int, default=1080)
    ap.add_argument("--lights", type=int, default=1024)
    ap.add_argument("--train-frames", type=int, default=20)
    ap.add_argument("--frames", type=int, default=4)
    ap.add_argument("--weights", default="sum", choices=["sum", "visibility"],
                    help="first-step cluster weights (NVC_CLUSTER_WEIGHT_*)")
    args = ap.parse_args()

    cfg = S.config_by_name("clustered_1080p")
    k = cfg.n_outputs
    sc = S.scene_rooms(seed=1, n_lights=args.lights)
    gb = S.gbuffer_heightfield(seed=1, width=args.width, height=args.height)
    assign, _ = nvc.nvc_kmeans_lights(sc.lights, S.kmeans_init(args.lights, k, seed=0), 10)
    clusters = nvc.Clusters(assign, k, weights=args.weights)
    scene = nvc.Scene.from_synth(sc)
    pos = torch.from_numpy(gb.pos).cuda()
    nrm = torch.from_numpy(gb.nrm).cuda()
    cache = nvc.VisibilityCache(cfg)
    cache.set_params(S.init_params(cfg, seed=0))
    loss = torch.empty(1, dtype=torch.float64, device="cuda")
    vis = torch.empty((gb.n, k), device="cuda")
    light = torch.empty(gb.n, dtype=torch.int32, device="cuda")
    W = torch.empty(gb.n, device="cuda")
    est = torch.empty(gb.n, device="cuda")
    acc = torch.zeros(gb.n, dtype=torch.float64, device="cuda")
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    times = np.zeros(3)
    for f in range(args.train_frames + args.frames):
        ev[0].record()
        nvc.nvc_train_step_clustered(cache.handle, scene, clusters, pos, 5, f, loss)
        ev[1].record()
        nvc.nvc_infer(cache.handle, pos, vis)
        ev[2].record()
        nvc.nvc_sample_clustered(scene, clusters, vis, pos, nrm, 7, f, light=light, weight=W,
                                 estimate=est)
        ev[3].record()
        if f >= args.train_frames:
            acc += est.double()
            torch.cuda.synchronize()
            times += [ev[i].elapsed_time(ev[i + 1]) for i in range(3)]
    exact = torch.empty(gb.n, device="cuda")
    nvc.nvc_exact_di(scene, pos, nrm, exact)
    torch.cuda.synchronize()
    mean = acc.cpu().numpy() / args.frames
    ex = exact.cpu().numpy().astype(np.float64)
    times /= max(args.frames, 1)
    print(f"{gb.width}x{gb.height}, {args.lights} lights, k = {k}, {args.weights} weights: "
          f"train {times[0]:.3f} ms, "
          f"infer {times[1]:.3f} ms, sample + shadow ray {times[2]:.3f} ms; "
          f"loss {loss.item():.4f}; relative RMS error of the {args.frames}-frame mean "
          f"{np.sqrt(np.mean((mean - ex) ** 2)) / max(np.sqrt(np.mean(ex ** 2)), 1e-30):.3f}")
    cache.close()


if __name__ == "__main__":
    main()
