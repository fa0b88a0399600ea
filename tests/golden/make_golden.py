"""Write the exact-DOS fixtures in this folder.  Calls only ``oracle/``.

    python tests/golden/make_golden.py            # L = 8, 16, 32
    python tests/golden/make_golden.py 64 128     # larger lattices

Each file lists, per realisable energy E of the L x L periodic 2D Ising model
(J = 1), the exact ln g(E) from Kaufman's closed form (Beale's method); the
L = 8 file also carries the integer g(E).  Source: oracle/exact_dos.py
(multiprecision DFT up to L = 32, prime-field evaluation + CRT above; the two
agree exactly where both run).
"""
import math
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import exact_dos  # noqa: E402


def write_ising(L):
    g = exact_dos.ising_kaufman(L) if L <= 32 else exact_dos.ising_kaufman_modular(L)
    path = os.path.join(HERE, f"ising_L{L}_exact_lng.txt")
    with open(path, "w") as f:
        f.write(f"# 2D Ising L={L} periodic, J=1: exact ln g(E) (Kaufman closed form, Beale's method)\n")
        f.write("# written by tests/golden/make_golden.py from oracle/exact_dos.py\n")
        f.write("# E ln_g" + (" g" if L <= 8 else "") + "\n")
        for E in sorted(g):
            line = f"{E} {math.log(g[E]):.17g}" if L <= 32 else f"{E} {math.log(g[E]):.13g}"
            if L <= 8:
                line += f" {g[E]}"
            f.write(line + "\n")
    return path


if __name__ == "__main__":
    sizes = [int(a) for a in sys.argv[1:]] or [8, 16, 32]
    for L in sizes:
        print(write_ising(L))
