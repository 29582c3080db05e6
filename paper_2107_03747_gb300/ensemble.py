"""Twisted ensembles and lambda_TGF, the way the paper measures it (Sec. 3.1).

Chains of the twisted Wilson action are generated on the GPU with the paper's hybrid algorithm
(tgf_mc_sweeps: one heat-bath sweep and L~ over-relaxation sweeps per hybrid sweep, L~ hybrid
sweeps between measurements).  Every measurement flows a copy of each chain's field to
sqrt(8t) = c L~ in FP32 and reads the clover E and Q there; lambda_TGF = N(c, L~) t^2 <E d_Q> /
(3 <d_Q>) (eq. lambdat_latt) with N(c, L~) of eq. (latt_norm), d_Q = [|Q| < 1/2].  Errors are a
jackknife over chains (the chains are independent).

    python -m paper_2107_03747_gb300.ensemble --l 4 --beta 20 --chains 256 --therm 50 --rounds 16
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import binding as tgf
from . import inputs as I


def generate_and_measure(beta, l=4, chains=256, therm=50, rounds=16, c=0.3, seed=2107, n_or=None, eps=0.01):
    """E and Q at sqrt(8t) = c L~ for `rounds` measurements of `chains` chains started at the
    twist-eater.  Returns (L~, t, E[rounds, chains], Q[rounds, chains])."""
    import torch

    L = I.tgf_extent(l)
    Lt = 3 * l
    n_or = Lt if n_or is None else n_or
    t = (c * Lt) ** 2 / 8.0
    mc = tgf.FlowBatch([L] * chains, "fp64")
    mc.set_links([I.twist_eater(L, 1)] * chains)
    fl = tgf.FlowBatch([L] * chains, "fp32")
    canon = torch.empty(mc.canonical_numel(), dtype=torch.float64, device=mc.device)
    tgf.tgf_mc_sweeps(mc.prec, mc.lat, mc.links, beta, therm, n_or, seed, 0)
    sweep = therm
    E = np.zeros((rounds, chains))
    Q = np.zeros((rounds, chains))
    rows = np.arange(chains)
    for r in range(rounds):
        tgf.tgf_mc_sweeps(mc.prec, mc.lat, mc.links, beta, Lt, n_or, seed, sweep)
        sweep += Lt
        tgf.tgf_unpack(mc.prec, mc.lat, mc.links, canon)
        tgf.tgf_pack(fl.prec, fl.lat, canon, fl.links)
        obs, nrec = fl.flow(eps, t, measure_every=1 << 20)
        o = obs.cpu().numpy()
        last = np.asarray(nrec) - 1
        if not np.allclose(o[rows, last, 0], t):
            raise RuntimeError("flow did not reach t")
        E[r] = o[rows, last, 1]
        Q[r] = o[rows, last, 2]
    torch.cuda.synchronize()
    return Lt, t, E, Q


def jackknife_lambda(c, Lt, t, E, Q):
    """lambda_TGF over all measurements and its jackknife error over chains (columns)."""
    lam = tgf.tgf_lambda(c, Lt, t, E.ravel(), Q.ravel())[0]
    n = E.shape[1]
    jk = np.array([tgf.tgf_lambda(c, Lt, t, np.delete(E, j, axis=1).ravel(), np.delete(Q, j, axis=1).ravel())[0]
                   for j in range(n)])
    return lam, math.sqrt((n - 1) / n * np.sum((jk - jk.mean()) ** 2))


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--l", type=int, default=4, help="short extent l of the l x l x 3l x 3l box (L~ = 3l)")
    ap.add_argument("--beta", type=float, default=20.0, help="18 b = 6/g0^2")
    ap.add_argument("--chains", type=int, default=256)
    ap.add_argument("--therm", type=int, default=50, help="hybrid sweeps before the first measurement")
    ap.add_argument("--rounds", type=int, default=16, help="measurements per chain, L~ hybrid sweeps apart")
    ap.add_argument("--n-or", type=int, default=None, help="over-relaxation sweeps per hybrid sweep (default L~)")
    ap.add_argument("--c", type=float, default=0.3)
    ap.add_argument("--seed", type=int, default=2107)
    a = ap.parse_args()
    t0 = time.time()
    Lt, t, E, Q = generate_and_measure(a.beta, a.l, a.chains, a.therm, a.rounds, a.c, a.seed, a.n_or)
    out = {"l": a.l, "Ltilde": Lt, "beta": a.beta, "c": a.c, "t": t, "chains": a.chains, "rounds": a.rounds,
           "seconds": time.time() - t0}
    if a.rounds:
        lam, err = jackknife_lambda(a.c, Lt, t, E, Q)
        out.update(lambda_tgf=lam, error=err, kept=int(np.sum(np.abs(Q) < 0.5)), measurements=int(Q.size))
    print(json.dumps(out))


if __name__ == "__main__":
    main()
