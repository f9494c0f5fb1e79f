"""Closed-form flow solutions used to pin the oracle (textbook results the paper's method
reduces to; none is printed in the paper itself)."""
import numpy as np
from scipy import special


def plane_poiseuille(y, y_lo, y_hi, g, nu):
    """Steady force-driven flow between plates: u = g/(2 nu) (y - y_lo)(y_hi - y)."""
    return g / (2.0 * nu) * (y - y_lo) * (y_hi - y)


def pipe_startup(r, t, R, g, nu, nterms=60):
    """Start-up flow in a circular pipe from rest under a constant body force g:
    u = g R^2/(4 nu) [1 - r^2/R^2 - 8 sum_n J0(l_n r/R) / (l_n^3 J1(l_n)) exp(-l_n^2 nu t/R^2)]."""
    lam = special.jn_zeros(0, nterms)
    s = np.zeros_like(np.asarray(r, dtype=np.float64))
    for ln in lam:
        s = s + special.j0(ln * r / R) / (ln ** 3 * special.j1(ln)) * np.exp(-ln ** 2 * nu * t / R ** 2)
    return g * R ** 2 / (4.0 * nu) * (1.0 - (r / R) ** 2 - 8.0 * s)


def womersley(r, t, R, A, omega, nu):
    """Periodic pipe flow under g(t) = A cos(omega t):
    u = Re{ A/(i omega) [1 - J0(i^{3/2} Wo r/R) / J0(i^{3/2} Wo)] e^{i omega t} }."""
    wo = R * np.sqrt(omega / nu)
    i32 = np.exp(1j * 3.0 * np.pi / 4.0)
    shape = 1.0 - special.jv(0, i32 * wo * r / R) / special.jv(0, i32 * wo)
    return np.real(A / (1j * omega) * shape * np.exp(1j * omega * t))
