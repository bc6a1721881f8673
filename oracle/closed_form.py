"""Closed forms used to pin the Monte Carlo oracle (test infrastructure only).

* Black-Scholes price and Greeks for a lognormal terminal price with total
  log-variance ``w`` -- the limit the Heston scheme reduces to with one step
  (S_T exactly lognormal with variance v0*T) and with zero vol-of-vol.
* The Heston (1993) semi-closed form via the characteristic function of
  ln S_T, written in the branch-cut-safe form of Albrecher, Mayer, Schoutens
  and Tistaert (2007).  The paper quotes its values ("real price" 6.8061,
  Delta 0.6958, Rho 62.7752 for the Table "Heston model parameters", Sec. 3)
  but prints no formula; Delta = P1 and Rho = K T e^{-rT} P2 follow from the
  homogeneity of the price in (S0, K).  Vega (d/dv0) differentiates the
  integrand (the characteristic function is exp(C + D v0 + ...), so the
  derivative multiplies it by D); Gamma and Theta are Richardson-extrapolated
  central differences of the closed form.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import integrate
from scipy.special import ndtr

SQRT_2PI = math.sqrt(2.0 * math.pi)


def _npdf(x):
    return math.exp(-0.5 * x * x) / SQRT_2PI


def bs_total_variance(S0, K, T, r, w, dw_dv0=0.0, dw_dT=0.0, is_put=False):
    """Black-Scholes with total log-variance w over [0, T].

    Returns dict price, delta, gamma, vega (= dPrice/dw * dw/dv0), rho,
    theta (= -dPrice/dT with w moving by dw/dT)."""
    sw = math.sqrt(w)
    d1 = (math.log(S0 / K) + r * T + 0.5 * w) / sw
    d2 = d1 - sw
    D = math.exp(-r * T)
    call = S0 * ndtr(d1) - K * D * ndtr(d2)
    dP_dw = S0 * _npdf(d1) / (2.0 * sw)          # same for call and put
    gamma = _npdf(d1) / (S0 * sw)
    if not is_put:
        price = call
        delta = ndtr(d1)
        rho = K * T * D * ndtr(d2)
        dP_dT_w = r * K * D * ndtr(d2)           # dPrice/dT at fixed w
    else:
        price = call - S0 + K * D
        delta = ndtr(d1) - 1.0
        rho = -K * T * D * ndtr(-d2)
        dP_dT_w = -r * K * D * ndtr(-d2)
    return dict(price=price, delta=delta, gamma=gamma, vega=dP_dw * dw_dv0, rho=rho,
                theta=-(dP_dT_w + dP_dw * dw_dT))


# ---------------------------------------------------------------------------
# Heston characteristic function (little-trap form)
# ---------------------------------------------------------------------------

def heston_cf(w, S0, v0, kappa, theta, xi, rho, r, T):
    """E[exp(i w ln S_T)] and the coefficient D(w) of v0 in its exponent.

    w may be complex.  d = sqrt((rho xi i w - kappa)^2 + xi^2 (i w + w^2)),
    g = (b - d) / (b + d) with b = kappa - rho xi i w."""
    iw = 1j * w
    b = kappa - rho * xi * iw
    d = np.sqrt(b * b + xi * xi * (iw + w * w))
    g = (b - d) / (b + d)
    e = np.exp(-d * T)
    C = iw * (math.log(S0) + r * T) + (kappa * theta / (xi * xi)) * (
        (b - d) * T - 2.0 * np.log((1.0 - g * e) / (1.0 - g)))
    Dv = ((b - d) / (xi * xi)) * (1.0 - e) / (1.0 - g * e)
    return np.exp(C + Dv * v0), Dv


def _probabilities(S0, K, T, r, v0, kappa, theta, xi, rho, with_vega=False):
    """P1, P2 (and their v0-derivatives): P_j = 1/2 + (1/pi) int_0^inf Re[e^{-iu ln K} f_j(u) / (iu)] du,
    f_2(u) = phi(u), f_1(u) = phi(u - i) / phi(-i), phi(-i) = S0 e^{rT}."""
    lnK = math.log(K)
    fwd = S0 * math.exp(r * T)
    args = (S0, v0, kappa, theta, xi, rho, r, T)

    def integrand(u, j, deriv):
        if j == 1:
            phi, Dv = heston_cf(u - 1j, *args)
            phi = phi / fwd
        else:
            phi, Dv = heston_cf(u + 0j, *args)
        val = phi * Dv if deriv else phi
        return (np.exp(-1j * u * lnK) * val / (1j * u)).real

    def integral(j, deriv):
        tot = 0.0
        edges = [0.0, 5.0, 20.0, 60.0, 150.0, 400.0, 1000.0]
        for a, b in zip(edges[:-1], edges[1:]):
            val, _ = integrate.quad(integrand, a, b, args=(j, deriv), limit=400,
                                    epsabs=1e-14, epsrel=1e-13)
            tot += val
        return tot / math.pi

    P1 = 0.5 + integral(1, False)
    P2 = 0.5 + integral(2, False)
    if not with_vega:
        return P1, P2
    return P1, P2, integral(1, True), integral(2, True)


def heston_call_price(S0, K, T, r, v0, kappa, theta, xi, rho):
    P1, P2 = _probabilities(S0, K, T, r, v0, kappa, theta, xi, rho)
    return S0 * P1 - K * math.exp(-r * T) * P2


def heston_price_greeks(S0, K, T, r, v0, kappa, theta, xi, rho, is_put=False, h_rel=1e-3):
    """Heston closed-form price and Greeks: dict price, delta, gamma, vega (d/dv0), rho, theta (-d/dT)."""
    P1, P2, dP1, dP2 = _probabilities(S0, K, T, r, v0, kappa, theta, xi, rho, with_vega=True)
    D = math.exp(-r * T)
    call = S0 * P1 - K * D * P2
    vega = S0 * dP1 - K * D * dP2

    def delta_at(s):
        return _probabilities(s, K, T, r, v0, kappa, theta, xi, rho)[0]

    def price_at(t):
        return heston_call_price(S0, K, t, r, v0, kappa, theta, xi, rho)

    def richardson(f, x, h):
        c1 = (f(x + h) - f(x - h)) / (2 * h)
        c2 = (f(x + h / 2) - f(x - h / 2)) / h
        return (4 * c2 - c1) / 3

    gamma = richardson(delta_at, S0, h_rel * S0)
    theta_call = -richardson(price_at, T, h_rel * T)
    if not is_put:
        return dict(price=call, delta=P1, gamma=gamma, vega=vega, rho=K * T * D * P2,
                    theta=theta_call)
    return dict(price=call - S0 + K * D, delta=P1 - 1.0, gamma=gamma, vega=vega,
                rho=-K * T * D * (1.0 - P2), theta=theta_call + r * K * D)
