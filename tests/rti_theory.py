"""Linear growth rate of the viscous single-mode Rayleigh-Taylor instability
(the relation the paper's RTI study compares against), for the tests."""
import math


def growth_rate(k: float, rho_h: float, rho_l: float, mu: float, g: float = 1.0) -> float:
    """Growth rate n > 0 for equal dynamic viscosities mu and no surface
    tension: the root of
    -{g k / n^2 (a_l - a_h) + 1}(a_h q_l + a_l q_h - k) - 4 k a_l a_h = 0,
    q_i = sqrt(k^2 + n / nu_i), a_i = rho_i / (rho_l + rho_h), nu_i = mu / rho_i
    (Eq. SinglePhaseGrowth), by bisection below the inviscid rate sqrt(At g k)."""
    ah, al = rho_h / (rho_h + rho_l), rho_l / (rho_h + rho_l)
    nuh, nul = mu / rho_h, mu / rho_l

    def f(n):
        ql, qh = math.sqrt(k * k + n / nul), math.sqrt(k * k + n / nuh)
        return -(g * k / (n * n) * (al - ah) + 1.0) * (ah * ql + al * qh - k) - 4.0 * k * al * ah
    lo, hi = 1e-12, math.sqrt((ah - al) * g * k)
    assert f(lo) > 0 > f(hi)
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if f(mid) > 0:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)
