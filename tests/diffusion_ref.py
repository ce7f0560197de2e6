"""Equilibrium-diffusion reference for the asymptotic Marshak wave.

In the asymptotic diffusion limit (Sec. 4.1, eq. diffu) radiation and gas
share one temperature and the total energy obeys
    d(C_v T + a T^4)/dt = d/dx ( 4 a c T^3 / (3 chi(T)) dT/dx ),
with chi = 300 T^-3 here.  This module integrates that equation on a fine
finite-volume grid with backward Euler and a fixed-point (lagged
conductivity) iteration per step, T = T_source at the x = 0 face and no flux
at the far wall: an independent numerical solution of the limit the paper
compares its Marshak run against (its semi-analytic solution is not given).
Test infrastructure only.
"""
import numpy as np
from scipy.linalg import solve_banded


def marshak_diffusion(t_end, a_rad, c, cv, L=0.66, n=660, nt=1000, T_source=1.0, T0=1e-3,
                      chi0=300.0):
    dx = L / n
    x = (np.arange(n) + 0.5) * dx
    T = np.full(n, T0)
    dt = t_end / nt

    def cond(T):  # 4 a c T^3 / (3 chi), chi = chi0 T^-3
        return 4.0 * a_rad * c * T ** 6 / (3.0 * chi0)

    Ks = cond(T_source)
    for _ in range(nt):
        U_old = cv * T + a_rad * T ** 4
        for _ in range(50):
            U = cv * T + a_rad * T ** 4
            dU = cv + 4.0 * a_rad * T ** 3
            K = cond(T)
            Kf = 0.5 * (K[1:] + K[:-1])          # interior faces
            K0 = 0.5 * (Ks + K[0])               # the source face, half a cell away
            g = np.empty(n + 1)
            g[0] = K0 * (T[0] - T_source) / (0.5 * dx)
            g[1:n] = Kf * (T[1:] - T[:-1]) / dx
            g[n] = 0.0
            res = (U - U_old) / dt - (g[1:] - g[:-1]) / dx
            main = dU / dt
            main[0] += K0 / (0.5 * dx * dx)
            main[:-1] += Kf / (dx * dx)
            main[1:] += Kf / (dx * dx)
            up = np.zeros(n)
            lo = np.zeros(n)
            up[1:] = -Kf / (dx * dx)
            lo[:-1] = -Kf / (dx * dx)
            dT = solve_banded((1, 1), np.vstack([up, main, lo]), -res)
            T = np.maximum(T + dT, 0.5 * T0)
            if np.max(np.abs(dT) / T) < 1e-10:
                break
    return x, T


def front(x, T, level=0.5):
    """Position where T first drops below `level` (linear interpolation)."""
    i = int(np.argmax(T < level))
    if i == 0:
        return float("nan")
    return float(x[i - 1] + (level - T[i - 1]) * (x[i] - x[i - 1]) / (T[i] - T[i - 1]))
