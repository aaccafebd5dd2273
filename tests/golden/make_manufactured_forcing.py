"""Writes manufactured_forcing.json: the external forcing of Test 1 of §6.4 as a double
Fourier series in x and t.  Calls only the oracle.

The manufactured solution (h = 2 + sin 2 pi x, eta* = 2 + sin 2 pi x sin(omega t),
u* = cos 2 pi x cos(omega t), L = 1, omega = 10) is a trigonometric polynomial of degree 1
in x and in omega t, and the right-hand side and d/dt (G u) are polynomials in those
fields and their derivatives, so the forcing is a trigonometric polynomial of low degree
in both variables.  Sampling the oracle's forcing (oracle.manufactured_forcing_1d) on
NX x-points and MT times per period, with both counts above twice the degrees, and taking
the discrete Fourier transform therefore gives its coefficients exactly up to rounding.

    S(x, t) = sum c * X_j(2 pi j x) * T_k(k omega t),  X, T in {cos, sin}

Each entry of "eta" / "U" is [j, k, X, T, c].  g = 1: the paper's non-dimensional gravity
(§2.1).

Usage: python tests/golden/make_manufactured_forcing.py
"""
import json
import math
import os
import sys

import numpy as np

sys.path.insert(0, os.path.join(os.path.dirname(__file__), "..", ".."))
from oracle import sgn_oracle as O  # noqa: E402

OMEGA, L, G = 10.0, 1.0, 1.0
NX, MT = 32, 32
KEEP = 1e-12                       # relative size below which a coefficient is rounding


def series(field_of):
    """field_of(x, t) on the NX grid -> list of [j, k, X, T, c] for the nonzero terms."""
    x = np.arange(NX) * L / NX
    ts = np.arange(MT) * (2.0 * math.pi / OMEGA) / MT
    S = np.stack([field_of(x, t) for t in ts])            # [MT, NX]
    F = np.fft.fft2(S) / (NX * MT)                         # F[k, j]
    out = []
    scale = np.abs(F).max()
    assert np.abs(F[MT // 2, :]).max() <= KEEP * scale      # degrees below the sample counts
    assert np.abs(F[:, NX // 2]).max() <= KEEP * scale
    for k in range(MT // 2):
        for j in range(NX // 2):
            # a = F[k, j], b = F[-k, j]; for real S the (+-k, +-j) terms sum to
            # 2 Re{a e^{i(kwt + 2 pi j x)}} + 2 Re{b e^{i(2 pi j x - kwt)}}
            a, b = F[k, j], F[(-k) % MT, j]
            if k == 0 and j == 0:
                terms = {("cos", "cos"): a.real}
            elif k == 0:
                terms = {("cos", "cos"): 2 * a.real, ("sin", "cos"): -2 * a.imag}
            elif j == 0:
                terms = {("cos", "cos"): 2 * a.real, ("cos", "sin"): -2 * a.imag}
            else:
                terms = {("cos", "cos"): 2 * (a.real + b.real),
                         ("sin", "sin"): 2 * (b.real - a.real),
                         ("cos", "sin"): 2 * (b.imag - a.imag),
                         ("sin", "cos"): -2 * (a.imag + b.imag)}
            for (X, T), c in terms.items():
                if abs(c) > KEEP * scale:
                    out.append([j, k, X, T, float(c)])
    return out


def evaluate(entries, x, t):
    f = {"cos": np.cos, "sin": np.sin}
    return sum(c * f[X](2 * math.pi * j * x / L) * f[T](k * OMEGA * t)
               for j, k, X, T, c in entries)


def main():
    eta = series(lambda x, t: O.manufactured_forcing_1d(x, t, L, G, OMEGA)[0])
    U = series(lambda x, t: O.manufactured_forcing_1d(x, t, L, G, OMEGA)[1])
    # the series reproduces the oracle's forcing at times off the samples: to rounding on
    # the fitting grid, and on a finer grid within the oracle's own rounding there (its
    # third derivatives amplify rounding by ~k_max^3)
    for nx, tol in ((NX, 1e-12), (256, 1e-9)):
        x = np.arange(nx) * L / nx
        for t in (0.0137, 0.41, 0.999):
            se, sU = O.manufactured_forcing_1d(x, t, L, G, OMEGA)
            assert np.abs(evaluate(eta, x, t) - se).max() <= tol * np.abs(se).max()
            assert np.abs(evaluate(U, x, t) - sU).max() <= tol * np.abs(sU).max()
    spec = {"source": "Test 1 of §6.4 (manufactured solution), forcing of Eq:DAE_DSWE",
            "L": L, "g": G, "omega": OMEGA, "eta": eta, "U": U}
    path = os.path.join(os.path.dirname(__file__), "manufactured_forcing.json")
    with open(path, "w") as fh:
        json.dump(spec, fh, indent=0)
        fh.write("\n")
    print(path, len(eta), "eta terms,", len(U), "U terms")


if __name__ == "__main__":
    main()
