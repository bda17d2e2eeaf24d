"""Write table2_synthetic_ours.txt: the synthetic rows of Table 2 (Sec. 5)
reproduced with the oracle (rates of Table 1 from the spectra of A^T A and X,
M-ADMM from its error map).  Calls only the oracle and the input generators.

The paper does not state m, p, the seed or the mean of the "Nonzero-Mean"
row; the choices here: m = 10 contiguous blocks (p = 50 for 500 x 500,
p = 100 for 1000 x 500), seed 0, mean 1.

Run from the repository root:  python tests/golden/make_table2_synthetic.py
"""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import apc_oracle as O  # noqa: E402
from paper_1708_01413_gb300 import inputs  # noqa: E402

ROWS = (
    ("Standard_Gaussian", dict(n=500, N=500, mean=0.0), 10),
    ("Nonzero_Mean_Gauss", dict(n=500, N=500, mean=1.0), 10),
    ("Standard_Tall_Gaus", dict(n=500, N=1000, mean=0.0), 10),
)
METHODS = ("DGD", "D-NAG", "D-HBM", "M-ADMM", "B-Cimmino", "APC")


def main():
    lines = ["# Synthetic rows of Table 2 (Sec. 5) reproduced with the oracle: convergence times",
             "# T = 1/(-log rho) from the rates of Table 1 (spectra of A^T A and X) and the modified",
             "# ADMM's error map.  Inputs: inputs.gaussian_system(n, seed=0, N, mean); m = 10",
             "# contiguous blocks.  Written by tests/golden/make_table2_synthetic.py.",
             "# columns: problem, " + ", ".join(METHODS) + ", kappa(A^T A), kappa(X)"]
    for name, kw, m in ROWS:
        A, _, b = inputs.gaussian_system(kw["n"], 0, N=kw["N"], mean=kw["mean"])
        row = O.table2_row(A, b, inputs.even_offsets(kw["N"], m))
        vals = " ".join(f"{row[k]:.3g}" for k in METHODS)
        lines.append(f"{name:<19}{vals} {row['kappa_AtA']:.3g} {row['kappa_X']:.3g}")
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "table2_synthetic_ours.txt")
    with open(out, "w") as fh:
        fh.write("\n".join(lines) + "\n")
    print("\n".join(lines))


if __name__ == "__main__":
    main()
