"""The 1080p frame workload (Sections 3.1-3.4): the heightfield + boxes view
with 32 point lights (or --lights), trained online for a few frames and then rendered as
whole frames (training step, fused inference + WRS + Neural DI), with the
time of each stage printed (CUDA events).

The shading variant is set directly (no autotuning), so that a profiler
sees a fixed sequence of launches: `--pretrain` training steps, then
`--frames` frames, each one training-data launch, one training launch, the
Adam, the shading launch and the frame counter.

    python -m paper_2506_05930_gb300.examples.frame_1080p --variant 7 --frames 3
"""
import argparse

import torch

import nvc_synth as S
from paper_2506_05930_gb300 import nvc


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--width", type=int, default=1920)
    ap.add_argument("--height", type=int, default=1080)
    ap.add_argument("--variant", type=int, default=7, help="fused shading variant (0-7)")
    ap.add_argument("--lights", type=int, default=32,
                    help="point lights = network outputs (above 32: variant 0 or 5)")
    ap.add_argument("--pretrain", type=int, default=5)
    ap.add_argument("--frames", type=int, default=3)
    ap.add_argument("--warm", type=int, default=0,
                    help="untimed frames before the timed ones (the first one loads the kernels)")
    ap.add_argument("--table-precision", default=None, choices=["fp16", "fp32"],
                    help="table features of the fused inference (default: the workload's)")
    args = ap.parse_args()

    cfg = S.config_by_name("frame_1080p").with_(n_outputs=args.lights)
    sc = S.scene_heightfield(seed=1, n_lights=args.lights, n_spheres=32, n_boxes=32)
    gb = S.gbuffer_heightfield(seed=1, width=args.width, height=args.height)
    scene = nvc.Scene.from_synth(sc)
    n = gb.n
    view = nvc.View(torch.from_numpy(gb.pos).cuda(), torch.from_numpy(gb.nrm).cuda(), 0,
                    torch.empty(n, dtype=torch.int32, device="cuda"), torch.empty(n, device="cuda"),
                    torch.empty(n, device="cuda"), torch.empty(n, device="cuda"))
    cache = nvc.VisibilityCache(cfg)
    cache.set_params(S.init_params(cfg, seed=0))
    if args.table_precision:
        nvc.nvc_set_table_precision(cache.handle, args.table_precision)
    nvc.nvc_set_shade_variant(cache.handle, args.variant)
    loss = torch.empty(1, dtype=torch.float64, device="cuda")
    for f in range(args.pretrain):
        nvc.nvc_train_step(cache.handle, scene, view.pos, 1, f, loss)
    # untimed frames: the first launch of each kernel also loads it
    for f in range(args.warm):
        nvc.nvc_frame(cache.handle, scene, [view], 0, 1, args.pretrain + f, loss, use_graph=False)
    args.pretrain += args.warm
    nvc.nvc_set_profiling(cache.handle, True)
    nvc.nvc_stage_times(cache.handle)
    for f in range(args.frames):
        nvc.nvc_frame(cache.handle, scene, [view], 0, 1, args.pretrain + f, loss, use_graph=False)
    ms, launches = nvc.nvc_stage_times(cache.handle)
    torch.cuda.synchronize()
    names = ("training data", "training fwd+bwd", "Adam", "shade")
    print("per frame (ms):", ", ".join(f"{a} {m / args.frames:.4f}" for a, m in zip(names, ms)),
          f"| launches {launches}, loss {loss.item():.5f}, picked",
          int((view.idx >= 0).sum().item()), "of", n)
    cache.close()


if __name__ == "__main__":
    main()
