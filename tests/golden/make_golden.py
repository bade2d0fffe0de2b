"""Write the closed-form lattice fixture (lattice_w1.txt) from oracle.closed_form only.

Run from the repository root: python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
from oracle import closed_form  # noqa: E402


def main():
    a = 10.0 ** (1.0 / 3.0)
    s = closed_form.lattice_sums(np.eye(3) * a, 12.0, 100 ** 3, nbins=200)
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "lattice_w1.txt")
    with open(out, "w") as f:
        f.write("# Perfect simple cubic lattice, 100^3 sites, spacing (1/0.1)^(1/3), rc = 12 (the 1M workload\n")
        f.write("# without jitter). Written by tests/golden/make_golden.py from oracle.closed_form.\n")
        f.write("neighbours_per_site %d\n" % s["nvec"])
        f.write("count %d\n" % s["count"])
        f.write("suminvr %.17g\n" % s["suminvr"])
        f.write("energy %.17g\n" % s["energy"])
        f.write("virial_diag %.17g\n" % s["virial"][0, 0])
        f.write("hist200 %s\n" % " ".join(str(int(v)) for v in s["hist"]))
    print(out)


if __name__ == "__main__":
    main()
