"""Run one compress + decompress of a synthetic field on cuda:0 (a small,
self-contained case for profilers such as ncu).

    python -m paper_1706_03791_gb300.run_case --kind blobs3d --shape 100 500 500 --reps 2 --chunk 256
"""
from __future__ import annotations

import argparse
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--kind", default="blobs3d", choices=["blobs3d", "grf2d"])
    ap.add_argument("--shape", type=int, nargs="+", default=[100, 500, 500])
    ap.add_argument("--ebrel", type=float, default=1e-4)
    ap.add_argument("--layers", type=int, default=1)
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--chunk", type=int, default=0, help="Huffman chunk length (0: the context's autotuned length, else whole rows)")
    args = ap.parse_args()
    import torch
    from paper_1706_03791_gb300 import build, szgb
    from synthetic import fields
    build.build()
    if args.kind == "blobs3d":
        x = fields.blobs3d(*args.shape, seed=2) if args.shape != [100, 500, 500] else fields.workload_3d()
    else:
        x = fields.grf2d(*args.shape, seed=1)
    xd = torch.from_numpy(x).cuda()
    ctx = szgb.Context(0)
    for _ in range(args.reps):
        s, st = ctx.compress(xd, eb_rel=args.ebrel, layers=args.layers, m=0, chunk_points=args.chunk)
        y = ctx.decompress(s)
    torch.cuda.synchronize()
    err = float((y.double() - xd.double()).abs().max())
    print("ok points=%d bytes=%d m=%d maxerr/eb=%.6f" % (x.size, s.numel(), st.m, err / st.eb_f))


if __name__ == "__main__":
    main()
