"""Flow SU(N) configurations on the twisted l x l x Nl x Nl box and report E, Q, P and the rate.

    python -m paper_2107_03747_gb300.sun_flow --N 4 --l 8 --configs 16 --steps 10

Seeded configurations exp(i amp omega_a lambda_a / 2) (generalised Gell-Mann lambda_a), twist
n_01 = k, RK3 steps of eps in FP64 through tgf_sun_stage, E/Q/P/S through tgf_sun_measure at the
end.  Prints one JSON line: the observables of the first configuration and the measured
site-RK3-steps/s (CUDA events around the steps after two warm-up steps).
"""
from __future__ import annotations

import argparse
import json

from . import binding as tgf
from . import inputs as I


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--N", type=int, default=2)
    ap.add_argument("--l", type=int, default=8)
    ap.add_argument("--k", type=int, default=1)
    ap.add_argument("--configs", type=int, default=16)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--eps", type=float, default=0.01)
    ap.add_argument("--amp", type=float, default=0.3)
    a = ap.parse_args()
    import torch

    N, l = a.N, a.l
    L = (l, l, N * l, N * l)
    V = l * l * N * l * N * l
    b = tgf.SunBatch(N, [L] * a.configs, [(a.k, 0, 0, 0, 0, 0)] * a.configs)
    b.set_links([I.random_links(L, s, a.amp, N=N) for s in range(a.configs)])
    for _ in range(2):
        b.step(a.eps)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(a.steps):
        b.step(a.eps)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / max(1, a.steps)
    m = b.measure((a.steps + 2) * a.eps)
    print(json.dumps({"N": N, "extent": L, "configs": a.configs, "ms_per_step": ms,
                      "site_steps_per_s": V * a.configs / ms * 1e3,
                      "t": m[0][0], "E": m[0][1], "Q": m[0][2], "P": m[0][3], "S": m[0][4]}))


if __name__ == "__main__":
    main()
