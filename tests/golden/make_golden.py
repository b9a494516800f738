"""Writes the stored expected values under tests/golden/.

Inputs come from the seeded generator (graphgen); expected values come only
from the CPU oracle (oracle/). Run from the repository root:

    python tests/golden/make_golden.py
"""
import hashlib
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import graphgen as gg  # noqa: E402
import oracle  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def main():
    r, c = gg.rmat(14, 16, seed=1)
    h = hashlib.sha256(r.tobytes() + c.tobytes()).hexdigest()
    src = gg.max_degree_vertex(r)
    depth, _ = oracle.bfs(r, c, src)
    hist = np.bincount(depth[depth >= 0])
    with open(os.path.join(HERE, "rmat_s14_seed1.txt"), "w") as f:
        f.write("# R-MAT scale 14, edge factor 16, (a,b,c)=(0.57,0.19,0.19), seed 1,\n"
                "# symmetrised, self-loops and duplicates removed (graphgen).\n"
                "# bfs_levels = oracle queue-BFS vertex count per depth from the\n"
                "# max-degree source (paper Sec. 5.1 semantics).\n")
        f.write(f"n={r.size - 1}\nm={c.size}\nsha256={h}\nsrc={src}\n")
        f.write("bfs_levels=" + ",".join(str(int(x)) for x in hist) + "\n")
        f.write(f"unreached={int((depth < 0).sum())}\n")


if __name__ == "__main__":
    main()
