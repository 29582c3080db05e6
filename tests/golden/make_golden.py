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


def write_flow(name, L, seed, amp, eps, t_end, note, batched=False):
    """Oracle flow of one configuration, every record; `batched` draws the field as a member of
    the mixed-size ensemble (amplitude from the seed's stream) instead of with amplitude `amp`."""
    if batched:
        amp, U = I.batched_member(seed, L)
    else:
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


FILES = {
    "flow_l4_seed0.txt": lambda n: write_flow(
        n, (4, 4, 12, 12), 0, 0.3, 0.01, 0.18,
        "4x4x12x12 twisted SU(3), links exp(i 0.3 omega T) from seed 0, RK3 eps=0.01 to t=c^2 l^2/8 (c=0.3)"),
    "flow_l2_seed3.txt": lambda n: write_flow(
        n, (2, 2, 6, 6), 3, 0.5, 0.02, 0.1,
        "2x2x6x6 twisted SU(3), links exp(i 0.5 omega T) from seed 3, RK3 eps=0.02 to t=0.1"),
    # the coupling's own flow time on the L~ = 12 box: sqrt(8t) = c L~ with c = 0.3 (Sec. 3.1), 162 steps
    "flow_l4_seed0_paper_scale.txt": lambda n: write_flow(
        n, (4, 4, 12, 12), 0, 0.3, 0.01, 1.62,
        "4x4x12x12 twisted SU(3), links exp(i 0.3 omega T) from seed 0, RK3 eps=0.01 to sqrt(8t)=0.3*12, t=1.62"),
    # member 1 (l = 6) of the 256-configuration mixed ensemble, to t = c^2 l^2/8 = 0.405: 40 steps + one of 0.005
    "flow_l6_batched1.txt": lambda n: write_flow(
        n, (6, 6, 18, 18), 1, None, 0.01, 0.405,
        "6x6x18x18 twisted SU(3), mixed-ensemble member seed 1 (amplitude from its stream), RK3 eps=0.01 to "
        "t=c^2 l^2/8=0.405 (c=0.3)", batched=True),
}


if __name__ == "__main__":
    names = sys.argv[1:] or sorted(FILES)
    for name in names:
        FILES[name](name)
