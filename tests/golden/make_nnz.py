"""Writes nnz.json: the number of non-zero sample-voxel weights of P (Eq. 1,
discretised) per workload and multigrid level, counted by the FP64 oracle.
The benchmark uses these counts as the algorithmic work of one projector or
transpose call (one multiply-add per weight). Calls only oracle/."""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import oracle as orc  # noqa: E402
from paper_1001_0599_gb300 import synthetic  # noqa: E402


def main():
    out = {"_doc": "non-zero weights of P per workload and multigrid level (0 = finest), from orc_count_terms"}
    for name, levels in (("small", 1), ("paper", 3), ("lowdose", 3), ("cube40", 3)):
        wl = synthetic.workload(name)
        g = orc.Geometry.from_workload(wl)
        out[name] = {str(l): orc.count_terms(g.coarse(2 ** l) if l else g) for l in range(levels)}
        print(name, out[name], flush=True)
    with open(os.path.join(HERE, "nnz.json"), "w") as fh:
        json.dump(out, fh, indent=1)


if __name__ == "__main__":
    main()
