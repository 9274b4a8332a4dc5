"""Writes oracle_sphere_scene.txt: the FP64 oracle's output on the seeded
64x48 sphere scene (radius 0.10 m at 0.80 m, plane at 1.5 m, 1 mm noise;
window radius 3, 3 iterations) at a fixed set of pixels.  It calls only the
oracle and the input generator; the test compares the oracle with this file
to catch unintended changes of its arithmetic."""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import synth   # noqa: E402

PIXELS = [(32, 24), (30, 22), (35, 26), (38, 24), (26, 24), (10, 10), (5, 40), (60, 3), (0, 0), (63, 47)]


def compute():
    s = synth.sphere_scene(0)
    p = oracle.params(*s.intrinsics, r=3, T=3)
    f = oracle.curvature_pixels(s.depth, p, np.array(PIXELS), nthreads=1)
    return f


def main():
    f = compute()
    with open(os.path.join(HERE, "oracle_sphere_scene.txt"), "w") as fh:
        fh.write("# u v status k1 k2 n_x n_y n_z  (oracle, sphere scene seed 0, r=3, T=3, k=1e-4)\n")
        for (u, v), st, a, b, n in zip(PIXELS, f.status, f.k1, f.k2, f.normal):
            fh.write(f"{u} {v} {st} {a:.12e} {b:.12e} {n[0]:.12e} {n[1]:.12e} {n[2]:.12e}\n")


if __name__ == "__main__":
    main()
