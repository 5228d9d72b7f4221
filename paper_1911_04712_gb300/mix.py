"""Run the standard mix of uneven boxes as one batch.

The mix (``workloads.box_mix``): boxes with integer edges U{6..24}, density
3, 4 or 5, a, gamma and kT drawn from their ranges, seeds 0..nbox-1.  The
whole mix is packed into one ``Batch`` and stepped; the throughput is timed
with CUDA events (states resident on the device).

    python -m paper_1911_04712_gb300.mix --nbox 512 --steps 100 --stencil half
"""

from __future__ import annotations

import argparse
import json


def main() -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--nbox", type=int, default=512)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--stencil", choices=("full", "half"), default="half")
    args = ap.parse_args()

    import torch

    from . import batch as B
    from .workloads import box_mix, uniform_box_state

    specs = box_mix(args.nbox, master_seed=args.seed)
    states = [uniform_box_state(s.L, rho=s.rho, kT=s.kT, seed=s.seed) for s in specs]
    descs = [B.make_desc(s.L, len(st[0]), a=s.a, gamma=s.gamma, kT=s.kT, dt=s.dt, seed=s.seed)
             for s, st in zip(specs, states)]
    stream = torch.cuda.current_stream()
    bt = B.Batch(descs, stream=stream.cuda_stream, stencil=1 if args.stencil == "half" else 0)
    for k, (x, v) in enumerate(states):
        bt.set_state(k, x, v)
    bt.step(args.warmup)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    bt.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    n = sum(len(x) for x, _ in states)
    ms = e0.elapsed_time(e1)
    print(json.dumps({"boxes": args.nbox, "particles": n, "steps": args.steps,
                      "stencil": args.stencil, "ms_per_step": ms / max(args.steps, 1),
                      "particle_steps_per_s": n * args.steps / (ms / 1000.0) if ms > 0 else None}))
    bt.close()
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
