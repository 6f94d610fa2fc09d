"""Writes the stored expected values under tests/golden/ by calling only the oracle.

Run from the repository root:  python tests/golden/make_golden.py
Each value is the oracle's own exact diagonalisation of the Heisenberg model on the
small geometries of the Numerical Experiments section of arXiv:2011.12453 (Kagome
2x2x3 and triangular 3x4 tori), in the S_z = 0 sector.
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import heisenberg as hz  # noqa: E402
from paper_2011_12453_gb300 import workloads as W  # noqa: E402


def main():
    out = {"_source": "tests/golden/make_golden.py (oracle.heisenberg.ground_state, S_z = 0 sector, J = 1)"}
    for name, g, k in [("kagome_2x2x3", W.kagome(2), 2), ("triangular_3x4", W.triangular(3, 4), 2)]:
        w, _, codes = hz.ground_state(g.n_sites, g.edges, g.J, k=k)
        out[name] = {"n_sites": g.n_sites, "n_edges": g.n_edges, "sector_size": int(len(codes)),
                     "E": [float(x) for x in w]}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "ed_energies.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=2)
        f.write("\n")
    print(json.dumps(out, indent=2))


if __name__ == "__main__":
    main()
