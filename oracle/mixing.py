"""Oracle modified Broyden mixing (D. D. Johnson, PRB 38, 12807 (1988)), the scheme the paper uses
for the response Hxc potential (Sec. 3.2, Sec. 5.1; alpha_mix = 0.3 and nmix = 4 by default,
Appendix B).

Test infrastructure only (see the package docstring).

With input vectors x_i, residuals F_i = g(x_i) - x_i and the normalised differences
dF_i = (F_{i+1} - F_i) / |F_{i+1} - F_i|,  dx_i = (x_{i+1} - x_i) / |F_{i+1} - F_i|,
Johnson's update with weights w_i = 1 and w0 = 0.01 is

    a_ij  = w0^2 delta_ij + w_i w_j <dF_i|dF_j>,     beta = a^-1
    c_k   = w_k <dF_k|F>,   gamma_l = sum_k c_k beta_kl
    x_new = x + alpha F - sum_l w_l gamma_l (dx_l + alpha dF_l)

using the last ``nmix`` pairs.  Complex vectors are mixed as real vectors of (Re, Im) parts, so
<a|b> = Re sum conj(a) b.
"""

from __future__ import annotations

import numpy as np


class Broyden:
    def __init__(self, alpha=0.3, nmix=4, w0=0.01):
        self.alpha = float(alpha)
        self.nmix = int(nmix)
        self.w0 = float(w0)
        self.df, self.dx = [], []
        self.x_prev = None
        self.f_prev = None

    @staticmethod
    def _dot(a, b):
        return float(np.real(np.vdot(a, b)))

    def step(self, x, f):
        """x: current input vector, f: its residual g(x) - x.  Returns the next input vector."""
        if self.x_prev is not None:
            dF = f - self.f_prev
            nrm = np.sqrt(self._dot(dF, dF))
            if nrm > 0:
                self.df.append(dF / nrm)
                self.dx.append((x - self.x_prev) / nrm)
                if len(self.df) > self.nmix:
                    self.df.pop(0)
                    self.dx.pop(0)
        self.x_prev = x.copy()
        self.f_prev = f.copy()
        x_new = x + self.alpha * f
        m = len(self.df)
        if m:
            a = np.array([[self._dot(self.df[i], self.df[j]) for j in range(m)] for i in range(m)])
            a += self.w0 ** 2 * np.eye(m)
            beta = np.linalg.inv(a)
            c = np.array([self._dot(self.df[k], f) for k in range(m)])
            gamma = c @ beta
            for l in range(m):
                x_new = x_new - gamma[l] * (self.dx[l] + self.alpha * self.df[l])
        return x_new
