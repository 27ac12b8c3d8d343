"""Test infrastructure: the Sedov-Taylor point-blast similarity constant xi0(gamma).

A strong spherical blast of energy E in a cold uniform gas of density rho0 has shock radius
R(t) = xi0 * (E t^2 / rho0)^(1/5).  With eta = r/R, u = R' phi(eta), rho = rho0 psi(eta),
p = rho0 R'^2 f(eta) (R' = dR/dt = 2R/(5t), so R'' = -3 R'^2 / (2R)), the Euler equations
reduce to three ODEs (continuity, momentum, entropy), linear in (phi', psi', f'):
    psi phi' + (phi - eta) psi'                       = -2 psi phi / eta
    (phi - eta) phi' + f' / psi                       = 3 phi / 2
    -gamma (phi - eta) psi' / psi + (phi - eta) f'/f  = 3
with the strong-shock jump conditions at eta = 1: phi = f = 2/(gamma+1),
psi = (gamma+1)/(gamma-1).  Energy conservation then fixes
    xi0^5 = 25 / (16 pi I),   I = int_0^1 eta^2 (psi phi^2 / 2 + f/(gamma-1)) d eta.
Derived here from the equations and integrated numerically (scipy).
"""
import math

import numpy as np
from scipy.integrate import solve_ivp


def _rhs(eta, y, g):
    phi, psi, f, _ = y
    a = phi - eta
    A = np.array([[psi, a, 0.0],
                  [a, 0.0, 1.0 / psi],
                  [0.0, -g * a / psi, a / f]])
    b = np.array([-2.0 * psi * phi / eta, 1.5 * phi, 3.0])
    dphi, dpsi, df = np.linalg.solve(A, b)
    dI = eta * eta * (0.5 * psi * phi * phi + f / (g - 1.0))
    return [dphi, dpsi, df, dI]


def xi0(gamma, eta_min=1e-6):
    g = float(gamma)
    y1 = [2.0 / (g + 1.0), (g + 1.0) / (g - 1.0), 2.0 / (g + 1.0), 0.0]
    sol = solve_ivp(_rhs, (1.0, eta_min), y1, args=(g,), rtol=1e-11, atol=1e-14, method="DOP853")
    if not sol.success:
        raise RuntimeError(sol.message)
    I = -sol.y[3, -1]  # integrated from 1 down to eta_min
    return (25.0 / (16.0 * math.pi * I)) ** 0.2


def shock_radius(t, E=1.0, rho0=1.0, gamma=5.0 / 3.0):
    return xi0(gamma) * (E * t * t / rho0) ** 0.2
