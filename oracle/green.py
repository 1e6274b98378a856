"""2D free-space Green's function of the Helmholtz operator (pin only).

TEST INFRASTRUCTURE: see the package header for who may import this.

For -Lap u - k^2 u = delta in the plane, the outgoing solutions are
(i/4) H0^(1)(k r) and -(i/4) H0^(2)(k r) = conj((i/4) H0^(1)(k r)) for real k.
With the damping sign of Eq. 3.1, w^2 m (1 - i gamma), the wavenumber inside
an absorbing layer has a negative imaginary part, so the bounded solution is
the H0^(2) branch: the discrete solution u approximates
conj((i/4) H0^(1)(k r)).  The Hankel function is scipy's, called.
"""
from __future__ import annotations

import numpy as np
from scipy.special import hankel1


def green_h1(k: float, r) -> np.ndarray:
    """(i/4) H0^(1)(k r)."""
    return 0.25j * hankel1(0, k * np.asarray(r, dtype=np.float64))
