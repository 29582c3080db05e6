"""Writes the stored oracle trajectories under tests/golden/ (calls only oracle/ and the input generators).

Run from the repository root:  python tests/golden/make_golden.py
"""
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import tgf_oracle as O  # noqa: E402
from paper_2107_03747_gb300 import inputs as I  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def write_flow(name, L, seed, amp, eps, t_end, note):
    U = I.random_links(L, seed, amp)
    t0 = time.time()
    _, rec = O.flow(U, eps, t_end, I.default_twist(1))
    with open(os.path.join(HERE, name), "w") as f:
        f.write(f"# {note}\n")
        f.write(f"# written by tests/golden/make_golden.py with oracle/tgf_oracle.py (FP64 CPU), {time.time() - t0:.1f} s\n")
        f.write(f"# L = {L}, seed = {seed}, amp = {amp}, twist n_01 = 1, eps = {eps}, t_end = {t_end}\n")
        f.write("# t E Q P S\n")
        for r in rec:
            f.write(" ".join(repr(float(x)) for x in r) + "\n")


if __name__ == "__main__":
    write_flow("flow_l4_seed0.txt", (4, 4, 12, 12), 0, 0.3, 0.01, 0.18,
               "4x4x12x12 twisted SU(3), links exp(i 0.3 omega T) from seed 0, RK3 eps=0.01 to t=c^2 l^2/8 (c=0.3)")
    write_flow("flow_l2_seed3.txt", (2, 2, 6, 6), 3, 0.5, 0.02, 0.1,
               "2x2x6x6 twisted SU(3), links exp(i 0.5 omega T) from seed 3, RK3 eps=0.02 to t=0.1")
