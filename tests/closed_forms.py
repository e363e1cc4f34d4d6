"""Closed-form results that pin the oracle (independent of Algorithms 1-4).

Each function states the passage or the textbook result it writes out.
"""
import math

import numpy as np


def eq21a_velocity(a, DP):
    """Model I, D_G = 0, L = 2: <v> = L J_I with J_I of Eq. 21a and alpha of Eq. 22.

    Valid for a > 1 (Sec. 3, Eqs. 21-23).
    """
    ap = math.exp(a / (DP * (a - 1.0)))
    am = math.exp(a / (DP * (a + 1.0)))
    J = (ap - am) / (4.0 * DP * (ap - 1.0) * (am - 1.0))
    return 2.0 * J


def eq21b_velocity(Fa, Fb, tau, printed_sign=False):
    """Model II, D_G = 0, L = 2: <v> = L J_II, Eq. 21b with beta of Eq. 22.

    As printed the numerator reads (beta_+ - beta_-); re-deriving the current
    from Eq. 20b, and the adiabatic limit tau -> oo (the weighted mean of the
    two constant-force sliding velocities), both give (beta_- - beta_+).  The
    corrected sign is the default.  D_D = F_a F_b tau (Eq. 17).
    """
    DD = Fa * Fb * tau
    bp = math.exp(1.0 / ((Fa + 1.0) * (Fb - 1.0) * tau))
    bm = math.exp(1.0 / ((Fa - 1.0) * (Fb + 1.0) * tau))
    num = (bp - bm) if printed_sign else (bm - bp)
    return 2.0 * num / (4.0 * DD * (bp - 1.0) * (bm - 1.0))


def pwl_sliding_velocity(F):
    """Deterministic velocity in the Eq. 2 potential under a constant force |F| > 1.

    The particle crosses the two unit ramps at speeds |F| + 1 and |F| - 1,
    so a period of length 2 takes 1/(|F|+1) + 1/(|F|-1) time units.
    """
    s = abs(F)
    return math.copysign(2.0 / (1.0 / (s + 1.0) + 1.0 / (s - 1.0)), F)


def stratonovich_velocity(V0, F, D, L=1.0, nx=512, nz=256):
    """Stationary velocity of x' = -V'(x) + F + sqrt(2D) xi, V = V0 sin(2 pi x / L).

    Stratonovich's formula (e.g. Risken, "The Fokker-Planck Equation", Sec. 11.3):
      <v> = L D (1 - exp(-F L / D)) / int_0^L dx int_0^L dz exp{[V(x+z) - V(x) - F z] / D}.
    x: trapezoid rule (periodic integrand, spectrally accurate);
    z: Gauss-Legendre on [0, L].
    """
    x = np.arange(nx) * (L / nx)
    zg, wg = np.polynomial.legendre.leggauss(nz)
    z = 0.5 * L * (zg + 1.0)
    w = 0.5 * L * wg
    V = lambda y: V0 * np.sin(2.0 * np.pi * y / L)
    expo = (V(x[:, None] + z[None, :]) - V(x[:, None]) - F * z[None, :]) / D
    inner = np.exp(expo) @ w
    integral = inner.sum() * (L / nx)
    return L * D * (1.0 - math.exp(-F * L / D)) / integral


def inertial_free_variance(gamma, Q, t):
    """x' = v, v' = -gamma v + sqrt(2 gamma Q) xi, x(0) = v(0) = 0 (Ornstein-Uhlenbeck velocity).

    Var v = Q (1 - e^{-2 g t});
    Var x = (2Q/g) [t - 2(1 - e^{-g t})/g + (1 - e^{-2 g t})/(2 g)];
    Cov(x, v) = (Q/g) (1 - e^{-g t})^2.
    """
    g = gamma
    vv = Q * (1.0 - math.exp(-2.0 * g * t))
    xx = (2.0 * Q / g) * (t - 2.0 * (1.0 - math.exp(-g * t)) / g
                          + (1.0 - math.exp(-2.0 * g * t)) / (2.0 * g))
    xv = (Q / g) * (1.0 - math.exp(-g * t)) ** 2
    return xx, xv, vv


def driven_linear_velocity(gamma, a, omega, F, v0, t):
    """Noise-free v' = -gamma v + a cos(omega t) + F, v(0) = v0: exact solution."""
    g = gamma
    vp = lambda s: F / g + a * (g * math.cos(omega * s) + omega * math.sin(omega * s)) / (g * g + omega * omega)
    return vp(t) + (v0 - vp(0.0)) * math.exp(-g * t)


def driven_linear_position(gamma, a, omega, F, v0, t):
    """x(t) - x(0) for the same noise-free linear equation (integral of the velocity)."""
    g = gamma
    den = g * g + omega * omega
    # integral of the particular solution
    ip = F * t / g + a * (g * math.sin(omega * t) / omega + (1.0 - math.cos(omega * t))) / den
    c = v0 - (F / g + a * g / den)
    return ip + c * (1.0 - math.exp(-g * t)) / g
