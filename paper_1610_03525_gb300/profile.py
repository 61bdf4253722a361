"""Run one generator configuration a few times on cuda:0 (a target for ncu).

    python -m paper_1610_03525_gb300.profile --kind c1 --size 8192 8192 --spc 1024 --octaves 12 --reps 3

Kinds: c1, c2, perlin_s5, perlin_s3, opensimplex; three sizes make a 3D
volume.  No timing is done here; numbers come from the profiler.
"""
from __future__ import annotations

import argparse


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--kind", default="c1", choices=["c1", "c2", "perlin_s5", "perlin_s3", "opensimplex"])
    ap.add_argument("--size", type=int, nargs="+", default=[8192, 8192])
    ap.add_argument("--spc", type=int, default=1024)
    ap.add_argument("--octaves", type=int, default=12)
    ap.add_argument("--origin", type=int, nargs="+", default=[0, 0, 0])
    ap.add_argument("--dtype", default="f32", choices=["f32", "f16"])
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--shape", default="auto", choices=["auto", "8x4", "16x2"], help="2D thread shape")
    ap.add_argument("--coarse", default="auto", choices=["auto", "runs", "tile"], help="2D coarse-octave mode")
    ap.add_argument("--tune-cache", default=None, help="launch-config table to load (as bench.py --tune-cache)")
    args = ap.parse_args()

    import torch

    import paper_1610_03525_gb300 as P

    dims = len(args.size)
    dtype = P.PTG_F16 if args.dtype == "f16" else P.PTG_F32
    d = P.make_desc(dims=dims, size=tuple(args.size), spc=args.spc, origin=tuple(args.origin) + (0,) * 3,
                    octaves=args.octaves, smoothness=P.PTG_C2 if args.kind == "c2" else P.PTG_C1,
                    variant=(P.PTG_PERLIN_S3 if args.kind == "perlin_s3" else P.PTG_PERLIN_S5) |
                    {"auto": P.PTG_SHAPE_AUTO, "8x4": P.PTG_SHAPE_8X4, "16x2": P.PTG_SHAPE_16X2}[args.shape] |
                    {"auto": P.PTG_COARSE_AUTO, "runs": P.PTG_COARSE_RUNS, "tile": P.PTG_COARSE_TILE}[args.coarse],
                    dtype=dtype)
    out = torch.empty(tuple(reversed(args.size)), dtype=torch.float16 if dtype == P.PTG_F16 else torch.float32,
                      device="cuda")
    ctx = P.ptg_create(0)
    if args.tune_cache:
        P.ptg_autotune(ctx, 0, args.tune_cache)
    fn = {"c1": P.ptg_field, "c2": P.ptg_field, "perlin_s5": P.ptg_perlin, "perlin_s3": P.ptg_perlin,
          "opensimplex": P.ptg_opensimplex}[args.kind]
    shape = ""
    if dims == 2 and args.kind != "opensimplex":
        rw, nt = P.ptg_launch_config(ctx, d, P.METHOD_PERLIN if args.kind.startswith("perlin") else P.METHOD_FIELD)
        shape = " (thread shape %dx%d, %d octaves at the tile nodes)" % (rw, 32 // rw, nt)
    for _ in range(args.reps):
        fn(ctx, d, out)
    torch.cuda.synchronize()
    ctx.close()
    print("ran %d x %s %s%s" % (args.reps, args.kind, "x".join(map(str, args.size)), shape))


if __name__ == "__main__":
    main()
