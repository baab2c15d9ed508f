"""Green-Kubo oracle: heat-current autocorrelation (HCACF) and the running thermal
conductivity -- TEST INFRASTRUCTURE ONLY (imported by tests/ and bench.py's CPU legs).

The paper computes the potential part of the heat current (Eq. 30) so that thermal
conductivity can be obtained from it (Sec. 2.3 and its thermal-transport references).
It does not print the Green-Kubo relation.  This module uses the textbook one:

    C_a(t_m)     = < J_a(0) J_a(t_m) >,  averaged over every time origin in the series:
                   C_a(m) = 1/(T - m) * sum_{t=0}^{T-m-1} J_a(t) J_a(t+m)
    kappa_a(t_m) = 1 / (k_B T^2 V) * integral_0^{t_m} C_a(t) dt   (trapezoid rule)

J is the total (extensive) heat current in eV A / fs, so C is in (eV A / fs)^2 and
kappa, with V in A^3 and T in K, is converted to W / (m K).  Only the diagonal
components a = x, y, z are formed.  Plain numpy, fp64, one dot product per lag.
"""
from __future__ import annotations

import numpy as np

K_B = 8.617333262e-5               # eV / K
EV_PER_FS_A_K_TO_W_PER_M_K = 1.602176634e-19 / (1e-15 * 1e-10)


def hcacf(j: np.ndarray, n_lags: int) -> np.ndarray:
    """C[m, a] for m < n_lags from the (T, 3) series j (rows = consecutive steps)."""
    j = np.asarray(j, dtype=np.float64)
    T = j.shape[0]
    if not 1 <= n_lags <= T:
        raise ValueError("need 1 <= n_lags <= number of rows")
    c = np.empty((n_lags, 3))
    for m in range(n_lags):
        for a in range(3):
            c[m, a] = np.dot(j[: T - m, a], j[m:, a]) / (T - m)
    return c


def running_kappa(c: np.ndarray, dt_fs: float, volume: float, temperature: float) -> np.ndarray:
    """kappa[m, a] in W/(m K): trapezoid integral of C from lag 0 to lag m."""
    c = np.asarray(c, dtype=np.float64)
    pref = EV_PER_FS_A_K_TO_W_PER_M_K / (K_B * temperature * temperature * volume)
    k = np.zeros_like(c)
    for m in range(1, c.shape[0]):
        k[m] = k[m - 1] + 0.5 * (c[m - 1] + c[m]) * dt_fs
    return k * pref
