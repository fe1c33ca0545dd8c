"""Closed-form transport solutions of the paper's two validation cases.

TEST INFRASTRUCTURE ONLY (see ``oracle/vag_oracle.py``).

* Sec. 5.1 (one fracture, time dependent): matrix and fracture concentrations
  obtained by integrating along the characteristics of u = 1 - x.
* Sec. 5.2 (four intersecting fractures, stationary).  The printed c_{f,3}
  carries the factor exp(-beta_1 / (4 k_1 tan(theta_1))); integrating
  -k_2 c' + beta_2 c = beta_2 c_{m,3} with c_{m,3}(y) = c_{f,1}((y - 1/4) /
  tan(theta_1)) gives exp(+beta_1 / (4 k_1 tan(theta_1))).  The derived sign is
  used here; ``tests/test_oracle_analytic.py`` checks every closed form
  against its ordinary differential equation.
"""
from __future__ import annotations

import numpy as np


class OneFracture:
    """Sec. 5.1: fracture from (0, 1/4) to (1, 1/4 + tan(theta)),
    k = Lambda_f cos^2(theta), beta = sin(theta) / d_f (k > 1 assumed)."""

    def __init__(self, tan_theta=0.5, lam_f=20.0, d_f=0.01):
        th = np.arctan(tan_theta)
        self.tan = tan_theta
        self.k = lam_f * np.cos(th) ** 2
        self.beta = np.sin(th) / d_f
        assert self.k > 1

    def c_f(self, x, t):
        x = np.asarray(x, float)
        t = np.broadcast_to(np.asarray(t, float), x.shape)
        out = np.zeros_like(x)
        mid = (t > x / self.k) & (t < x)
        out[mid] = np.exp(-self.beta / (self.k - 1.0) * (x[mid] - t[mid]))
        out[t >= x] = 1.0
        return out

    def y_frac(self, x):
        return 0.25 + x * self.tan

    def c_m(self, x, y, t):
        x = np.asarray(x, float); y = np.asarray(y, float)
        out = np.where(t > x, 1.0, 0.0)
        # below the fracture and above y = 1/4: fed by the fracture
        below = (y < self.y_frac(x)) & (y > 0.25)
        xf = (4 * y[below] - 1) / (4 * self.tan)
        tt = t + xf - x[below]
        val = np.where(t > x[below] - xf, self.c_f(xf, tt), 0.0)
        out[below] = val
        return out


class FourFractures:
    """Sec. 5.2 stationary solution."""

    def __init__(self, tan1=5.0 / 8.0, tan2=0.25, lam_f1=200.0, lam_f3=400.0, d_f1=0.01, d_f3=0.01):
        t1 = np.arctan(tan1); t2 = np.arctan(tan2)
        self.tan1, self.tan2 = tan1, tan2
        self.b1 = np.sin(t1) / d_f1
        self.k1 = lam_f1 * np.cos(t1) ** 2
        self.b2 = np.cos(t2) / d_f3
        self.k2 = lam_f3 * np.cos(t2) * np.sin(t2)
        self.r = lam_f3 * d_f3 * np.sin(t2) / (lam_f1 * d_f1 * np.cos(t1))
        s = 1.0 / (4.0 * (1.0 + tan1 * tan2))
        self.x0 = s * (3.0 - tan2)
        self.y0 = s * (1.0 + 3.0 * tan1)
        self.r1 = self.b1 / self.k1 + self.b2 / self.k2 * tan1
        self.r2 = self.b2 / self.k2 + self.b1 / (self.k1 * tan1)
        self.c0 = (np.exp(-self.b1 / self.k1 * self.x0)
                   + self.r * np.exp(-self.b2 / self.k2 * (1 - self.y0))) / (self.r + 1)

    # fractures -------------------------------------------------------------
    def cf1(self, x):
        return np.exp(-self.b1 / self.k1 * np.asarray(x, float))

    def cf4(self, y):
        return np.exp(-self.b2 / self.k2 * (1.0 - np.asarray(y, float)))

    def cf2(self, x):
        x = np.asarray(x, float)
        e = -3.0 * self.b2 / (4.0 * self.k2)
        return np.exp(-self.b1 / self.k1 * x) * (
            self.c0 * np.exp(self.b1 / self.k1 * self.x0)
            + self.b1 / (self.k1 * self.r1) * (np.exp(self.r1 * x + e) - np.exp(self.r1 * self.x0 + e)))

    def cf3(self, y):
        y = np.asarray(y, float)
        g = self.b1 / (4.0 * self.k1 * self.tan1)        # derived sign: +
        lo = np.maximum(y, 0.25)
        return np.exp(self.b2 / self.k2 * y) * (
            self.c0 * np.exp(-self.b2 / self.k2 * self.y0)
            + self.b2 / (self.k2 * self.r2) * (np.exp(-self.r2 * lo + g) - np.exp(-self.r2 * self.y0 + g)))

    def line1_y(self, x):
        return 0.25 + self.tan1 * np.asarray(x, float)

    def line2_x(self, y):
        return 0.75 - self.tan2 * np.asarray(y, float)

    def c_m(self, x, y):
        x = np.asarray(x, float); y = np.asarray(y, float)
        above1 = y > self.line1_y(x)
        left2 = x < self.line2_x(y)
        out = np.zeros_like(x)
        # Omega_2: above line 1, right of line 2
        m2 = above1 & ~left2
        out[m2] = self.cf4(y[m2])
        # Omega_3: below line 1, left of line 2
        m3 = ~above1 & left2
        yy = y[m3]
        out[m3] = np.where(yy > 0.25, self.cf1((yy - 0.25) / self.tan1), 0.0)
        # Omega_4: below line 1, right of line 2
        m4 = ~above1 & ~left2
        yy = y[m4]
        out[m4] = np.where(yy < self.y0, self.cf3(yy), self.cf2((yy - 0.25) / self.tan1))
        return out
