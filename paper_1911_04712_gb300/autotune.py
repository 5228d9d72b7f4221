"""Autotuner of the direct force kernel, per density band.

For each stencil and each density band it times the force stage of every
kernel variant (threads per block x pair-list capacity x drain) with the
library's per-stage CUDA events and keeps the fastest, twice: on one
periodic box of the band's density (the single-box table) and on a packed
batch of small boxes of that density with edges U{6..24} (the packed
table).  The result is a JSON table {"full": [{"rho_upper", "rho",
"variant", "ms": [...]}, ...], "half": [...], "full_packed": [...],
"half_packed": [...]} that ``batch.py`` installs into the library
(dpd_tuning_set) when it loads.

    python -m paper_1911_04712_gb300.autotune --out tuning_gb300.json
"""

from __future__ import annotations

import argparse
import json
import sys

# (upper bound of the band, density the band is measured at)
BANDS = [(3.5, 3.0), (4.5, 4.0), (5.5, 5.0), (7.5, 6.5), (1e9, 10.0)]


def _time_packed(B, stencil, rho, var, nbox, steps, warmup, seed, stream):
    from .workloads import box_mix, uniform_box_state
    specs = box_mix(nbox, master_seed=seed, rhos=(rho,))
    states = [uniform_box_state(s.L, rho=s.rho, kT=s.kT, seed=s.seed) for s in specs]
    descs = [B.make_desc(s.L, len(st[0]), a=s.a, gamma=s.gamma, kT=s.kT, dt=s.dt, seed=s.seed)
             for s, st in zip(specs, states)]
    bt = B.Batch(descs, stream=stream, stencil=stencil, variant=var)
    for k, (x, v) in enumerate(states):
        bt.set_state(k, x, v)
    bt.step(warmup)
    ms = bt.profile(steps)[4]
    bt.close()
    return ms


def tune(L: float = 80.0, steps: int = 10, warmup: int = 3, seed: int = 0, nbox: int = 96,
         verbose=True) -> dict:
    import torch

    from . import batch as B
    from . import dpd as D
    from .workloads import uniform_box_state

    D.lib()
    stream = torch.cuda.current_stream()
    table = {}
    for name, stencil in (("full", 0), ("half", 1)):
        rows = []
        for upper, rho in BANDS:
            x, v = uniform_box_state(L, rho=rho, seed=seed)
            times = []
            for var in range(B.NUM_FORCE_VARIANTS):
                box = D.Box(L, seed=seed, stencil=stencil, stream=stream)
                box.set_param(D.PARAM_FORCE_VARIANT, var)
                box.set_state(x, v)
                box.step(warmup)
                times.append(box.profile(steps)[4])
                box.close()
            best = min(range(len(times)), key=times.__getitem__)
            rows.append({"rho_upper": upper, "rho": rho, "variant": best,
                         "threads_listcap": list(B.variant_info(best)),
                         "ms": [round(t, 5) for t in times]})
            if verbose:
                print(f"{name} rho={rho}: best variant {best} {B.variant_info(best)} "
                      f"{times[best]:.4f} ms (variant 0: {times[0]:.4f})", file=sys.stderr)
        table[name] = rows
        rows = []
        for upper, rho in BANDS:
            times = [_time_packed(B, stencil, rho, var, nbox, steps, warmup, seed,
                                  stream.cuda_stream)
                     for var in range(B.NUM_FORCE_VARIANTS)]
            best = min(range(len(times)), key=times.__getitem__)
            rows.append({"rho_upper": upper, "rho": rho, "variant": best,
                         "threads_listcap": list(B.variant_info(best)),
                         "ms": [round(t, 5) for t in times]})
            if verbose:
                print(f"{name} packed rho={rho}: best variant {best} {B.variant_info(best)} "
                      f"{times[best]:.4f} ms (variant 0: {times[0]:.4f})", file=sys.stderr)
        table[name + "_packed"] = rows
    table["box"] = {"L": L, "steps": steps,
                    "what": "force-stage ms per step: one box per band (full, half), or a "
                            f"batch of {nbox} boxes with edges U{{6..24}} at the band's "
                            "density (full_packed, half_packed)"}
    return table


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=None)
    ap.add_argument("--L", type=float, default=80.0)
    ap.add_argument("--steps", type=int, default=10)
    args = ap.parse_args()
    table = tune(args.L, args.steps)
    text = json.dumps(table, indent=1)
    if args.out:
        with open(args.out, "w") as f:
            f.write(text + "\n")
    print(text)


if __name__ == "__main__":
    main()
