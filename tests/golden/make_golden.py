"""Write the oracle's golden fixtures (calls only ``oracle/`` and the input synthesiser).

The paper prints no worked numeric example (its figures carry no values), so
these fixtures freeze the oracle's own answer on small cases.  They guard the
oracle across hosts (x86-64 here, AArch64 next to the GPU) and across edits:
a change to the oracle's arithmetic that moves them must say, in its commit
message, which passage of the paper justifies it.

    python -m tests.golden.make_golden      # rewrites the .txt files
"""
import os

import numpy as np

import oracle
from paper_1812_06007_gb300 import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))

CASES = {
    # Section 3 PowerURV on a Section 5-style matrix Haar diag(sigma) Haar
    "urv_64x48_q2_plain": dict(m=64, n=48, decades=8.0, q=2, reorth=False),
    "urv_64x48_q2_reorth": dict(m=64, n=48, decades=8.0, q=2, reorth=True),
    "urv_40x40_q0": dict(m=40, n=40, decades=4.0, q=0, reorth=True),
}


def compute_case(name):
    c = CASES[name]
    A = W.test_matrix_np(c["m"], c["n"], W.sigma_profile("exponential", c["n"], decades=c["decades"]))
    U, R, V = oracle.urv(A, c["q"], c["reorth"], W.SEED_G)
    G = oracle.gaussian(W.SEED_G, c["n"], c["n"])
    return {
        "G_head": G[:4, :4],
        "R_diag": np.diag(R)[None, :12],
        "R_row0": R[:1, :12],
        "V_head": V[:6, :4],
        "U_head": U[:6, :4],
    }


def save_fixture(path, arrays, header):
    with open(path, "w") as f:
        f.write(f"# {header}\n")
        for key, a in arrays.items():
            a = np.atleast_2d(a)
            f.write(f"{key} {a.shape[0]} {a.shape[1]}\n")
            for row in a:
                f.write(" ".join(repr(float(x)) for x in row) + "\n")


def load_fixture(path):
    out = {}
    with open(path) as f:
        lines = [ln for ln in f.read().splitlines() if ln and not ln.startswith("#")]
    i = 0
    while i < len(lines):
        key, r, c = lines[i].split()
        r, c = int(r), int(c)
        out[key] = np.array([[float(x) for x in lines[i + 1 + k].split()] for k in range(r)])
        i += 1 + r
    return out


def main():
    for name in CASES:
        c = CASES[name]
        hdr = (f"oracle PowerURV (Section 3): m={c['m']} n={c['n']} q={c['q']} reorth={c['reorth']}, "
               f"A = Haar diag(10^(-{c['decades']}(j-1)/(n-1))) Haar (Section 5 recipe), seed_G={W.SEED_G}")
        save_fixture(os.path.join(HERE, name + ".txt"), compute_case(name), hdr)


if __name__ == "__main__":
    main()
