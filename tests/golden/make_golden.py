"""Write tests/golden/oracle_sphere_f6.txt: FP64 oracle sums on a small sphere.

Regression fixture for the oracle (run from the repository root):
    python tests/golden/make_golden.py
It calls only ``oracle/`` (and ``synth/`` for the mesh and the seeded density); the
stored values are the direct single-, double- and adjoint-double-layer sums (Sec. II.A,
Eqs. kernel and kernel_pol) at every 9th of the 720 centroids of a frequency-6
geodesic unit sphere, density uniform in [-1, 1] (seed 6), weights folded in.
"""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import synth  # noqa: E402
from oracle.quadrature import quadrature_points  # noqa: E402

PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_sphere_f6.txt")


def compute():
    m = synth.geodesic_sphere(6)
    xyz, w, nrm = quadrature_points(m.tri, m.sph)
    sig = synth.uniform_density(m.n, 6)
    idx = np.arange(0, m.n, 9)
    q = sig * w
    out = {"idx": idx}
    out["sl"] = oracle.direct("sl", xyz, xyz, q, idx=idx, nthreads=1)
    out["dl"] = oracle.direct("dl", xyz, xyz, q, src_nrm=nrm, idx=idx, nthreads=1)
    out["adl"] = oracle.direct("adl", xyz, xyz, q, trg_nrm=nrm, idx=idx, nthreads=1)
    return out


def main():
    r = compute()
    with open(PATH, "w") as f:
        f.write("# target_index sl dl adl  (oracle FP64; geodesic sphere f=6, 720 points, seed 6)\n")
        for i, t in enumerate(r["idx"]):
            f.write("%d %.17e %.17e %.17e\n" % (t, r["sl"][i], r["dl"][i], r["adl"][i]))


if __name__ == "__main__":
    main()
