"""Writes the stored exact values under tests/golden/ from oracle/ only.

kaufman_lnZ.txt: ln Z of the L x L periodic Ising ferromagnet (Kaufman 1949,
evaluated with mpmath at 50 digits by oracle.exact.kaufman_lnZ) at
beta = i/200, i = 0..200, for L in {4, 8, 16, 32, 64}.  The GPU host has no
mpmath, so the GPU free-energy checks read these values.

Run from the repository root:  python tests/golden/make_golden.py
"""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import exact  # noqa: E402


def main():
    out = os.path.join(ROOT, "tests", "golden", "kaufman_lnZ.txt")
    with open(out, "w") as fh:
        fh.write("# L beta lnZ   (Kaufman 1949 closed form, mpmath 50 digits; "
                 "written by tests/golden/make_golden.py)\n")
        for L in (4, 8, 16, 32, 64):
            for i in range(201):
                b = i / 200
                fh.write(f"{L} {b!r} {exact.kaufman_lnZ(L, b)!r}\n")


if __name__ == "__main__":
    main()
