"""Writes tests/golden/two_view_matches.txt: the oracle's match list for the seeded single-pair scene
(1500 points in a 10 m cube, 2000 keypoints per image, band 4 px, ratio 4/5).  Calls only oracle/ and scenes/.

    python tests/golden/make_golden.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import scenes  # noqa: E402


def main():
    sc = scenes.two_view()
    A, B = sc.images
    pr = sc.pairs[0]
    mj, nc = oracle.match_pair(A.xy, A.desc, B.xy, B.desc, pr.F, pr.d, pr.p, pr.q)
    m = oracle.matches_from_match_j(mj)
    with open(os.path.join(HERE, "two_view_matches.txt"), "w") as fh:
        fh.write("# oracle match list, scenes.two_view() (seed 1512_06235 + 1), d = 4 px, ratio 4/5\n")
        fh.write(f"# n_cand {nc}\n")
        for i, j in m:
            fh.write(f"{i} {j}\n")


if __name__ == "__main__":
    main()
