"""Write the stored expected values under tests/golden/ from the oracle only.

cfg1_fom.json: receiver pressures of the config-1 model (1x1x2 m cavity,
8x8x16 nodes, shell ring, one unit shell load) at all 181 frequencies
20..200 Hz, by the oracle's dense GEPP of the scaled system (paper Sec. 2,
Eq. 1; Eq. 8), and LAPACK's 1-norm condition estimate (zgecon) of that scaled
matrix at each frequency, which bounds how far two correct FP64 solutions of
slightly differently rounded matrices can differ.
Run:  python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np
import scipy.linalg.lapack as lapack
import scipy.sparse as sp

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import workloads as W  # noqa: E402
from oracle import fem, fom  # noqa: E402


def main():
    w = W.config1()
    asm = fem.assemble(w.model)
    F = fem.load_matrix(w.model, w.loads, w.n_rhs)
    rc = fem.receiver_dofs(w.model, w.receivers)
    p, _ = fom.sweep(asm, w.freqs_hz, F, rc, method="dense")
    kappa = []
    for f in w.freqs_hz:
        om = 2 * np.pi * f
        r, c = fom.equilibrate(asm, om)
        As = (sp.diags(r) @ asm.A(om) @ sp.diags(c)).toarray()
        anorm = np.abs(As).sum(axis=0).max()
        lu, piv, info = lapack.zgetrf(As)
        rcond, info2 = lapack.zgecon(lu, anorm, norm="1")
        kappa.append(float(1.0 / rcond))
    out = {"workload": w.name, "source": "oracle.fom.sweep(method='dense')",
           "freqs_hz": w.freqs_hz.tolist(), "receivers": [list(r) for r in w.receivers],
           "p_re": p.real.tolist(), "p_im": p.imag.tolist(), "kappa1_scaled": kappa}
    with open(os.path.join(HERE, "cfg1_fom.json"), "w") as fh:
        json.dump(out, fh)
    print("wrote cfg1_fom.json", p.shape)


if __name__ == "__main__":
    main()
