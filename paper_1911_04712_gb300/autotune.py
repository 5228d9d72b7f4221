"""Autotuner of the direct force kernel, per density band.

For each stencil and each density band it fills a periodic box of the
band's representative density, times the force stage of every kernel
variant (threads per block x pair-list capacity) with the library's
per-stage CUDA events, and keeps the fastest.  The result is a JSON table
{"full": [{"rho_upper", "rho", "variant", "ms": [...]}, ...], "half": [...]}
that ``batch.py`` installs into the library (dpd_tuning_set) when it loads.

    python -m paper_1911_04712_gb300.autotune --out tuning_gb300.json
"""

from __future__ import annotations

import argparse
import json
import sys

# (upper bound of the band, density the band is measured at)
BANDS = [(3.5, 3.0), (4.5, 4.0), (5.5, 5.0), (7.5, 6.5), (1e9, 10.0)]


def tune(L: float = 48.0, steps: int = 10, warmup: int = 3, seed: int = 0, verbose=True) -> dict:
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
    table["box"] = {"L": L, "steps": steps, "what": "force-stage ms per step, one box per band"}
    return table


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=None)
    ap.add_argument("--L", type=float, default=48.0)
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
