"""Tune the bare mass m0 of each synthetic configuration and write synth/m0_table.json.

Test infrastructure only (see ``oracle/__init__.py``): this script uses the
oracle's operator to place the spectrum; the table it writes is an input of
both the oracle and the CUDA path.

The paper measures at a "mass gap" near critical mass (Section 3, Figs. 1-5)
without defining it.  Reading: the spectrum of D(m0) is the spectrum of D(0)
shifted by m0, and m0 is chosen per configuration so that the smallest real
part of the spectrum is 1e-3.  When the leftmost eigenvalue is real (the
common case) this makes min |lambda(D)| = 1e-3.  The leftmost eigenvalues of
D(0) come from shift-invert Arnoldi (scipy eigs, sparse LU) around the shift 0 (left of
the spectrum of D(0) for beta = 6.0), refined once around the first estimate.

Usage:  python -m oracle.tune_m0 64:0-9 256:0-9
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np
import scipy.sparse.linalg as spla

import synth
from . import dirac

TARGET = 1e-3


def _near(A, sigma, k, tol):
    """k eigenvalues of A nearest sigma: Arnoldi on (A - sigma)^{-1} with a sparse LU."""
    import scipy.sparse as sp
    lu = spla.splu((A - sigma * sp.identity(A.shape[0], dtype=A.dtype, format="csc")).tocsc())
    op = spla.LinearOperator(A.shape, matvec=lu.solve, dtype=np.complex128)
    mu = spla.eigs(op, k=k, which="LM", return_eigenvectors=False, tol=tol, ncv=max(40, 3 * k))
    return sigma + 1.0 / mu


def leftmost_eigs(U, k=12):
    A = dirac.stencil_sparse(dirac.wilson_stencil(U, 0.0)).tocsc()
    # rough pass around 0, then an accurate pass just left of the smallest real part found
    vals = _near(A, 0.0, 6, 1e-6)
    sigma = float(np.min(vals.real)) - 0.005
    return _near(A, sigma, k, 1e-12)


def tune(L, config):
    U = synth.gauge_field(L, config)
    vals = leftmost_eigs(U)
    i = int(np.argmin(vals.real))
    m0 = TARGET - float(vals[i].real)
    shifted = vals + m0
    return {
        "m0": m0,
        "lambda_min_re": float(vals[i].real),
        "lambda_min_im": float(vals[i].imag),
        "min_abs_eig": float(np.min(np.abs(shifted))),
        "fingerprint": synth.fingerprint(U),
        "sweeps": synth.default_sweeps(L),
        "beta": synth.BETA,
    }


def main(argv):
    path = os.path.join(os.path.dirname(synth.__file__), "m0_table.json")
    table = {"what": "bare mass m0 per synthetic configuration; written by oracle/tune_m0.py",
             "reading": "m0 = 1e-3 - min Re lambda(D(0)); leftmost eigenvalues by shift-invert Arnoldi",
             "entries": {}}
    if os.path.exists(path):
        with open(path) as f:
            table = json.load(f)
    for spec in argv:
        L, rng = spec.split(":")
        lo, hi = (int(v) for v in rng.split("-")) if "-" in rng else (int(rng), int(rng))
        for c in range(lo, hi + 1):
            t0 = time.time()
            e = tune(int(L), c)
            table["entries"][f"{int(L)}:{c}"] = e
            print(f"L={L} c={c} m0={e['m0']:.12f} lam=({e['lambda_min_re']:.6f},{e['lambda_min_im']:.2e}) "
                  f"min|lam|={e['min_abs_eig']:.3e} ({time.time() - t0:.1f}s)", flush=True)
            tmp = path + f".{os.getpid()}.tmp"
            with open(tmp, "w") as f:
                json.dump(table, f, indent=1, sort_keys=True)
            os.replace(tmp, path)  # readers never see a half-written table


if __name__ == "__main__":
    main(sys.argv[1:])
