"""Closed-form Gaussian solutions used to pin the split-step oracle.

A 1D Gaussian psi(q) = exp(-A q^2/2 + B q + C) (A, B, C complex, Re A > 0)
stays Gaussian under every factor of a Strang step for the oscillator
V = q^2/2 and for the free particle:

* potential factor exp(-i kappa q^2/2)     : A <- A + i kappa
* free drift for time tau, exp(-i k^2 tau/2) in k-space:
      d = 1 + i A tau,  A <- A/d,  B <- B/d,  C <- C + i tau B^2/(2d) - ln(d)/2
  (Fourier-transform the Gaussian, multiply, transform back).

Applying these in the V/2-K-V/2 order gives the EXACT discrete trajectory of
the split-step method on the infinite line, global phase included, so a grid
solver that is spectrally accurate must reproduce it to round-off plus
truncation.  Imaginary time replaces tau by -i tau and kappa by -i kappa.

Also the continuum coherent state of the unit oscillator (the physics the
splitting approximates to O(dt^2)).
"""
import numpy as np


class Gauss1D:
    def __init__(self, A, B, C):
        self.A, self.B, self.C = complex(A), complex(B), complex(C)

    @classmethod
    def displaced_ground(cls, q0=0.0, p0=0.0):
        """pi^(-1/4) exp(-(q - q0)^2/2 + i p0 q)."""
        return cls(1.0, q0 + 1j * p0, -q0 * q0 / 2.0 - 0.25 * np.log(np.pi))

    @classmethod
    def packet(cls, sigma, q0=0.0, p0=0.0):
        """(2 pi sigma^2)^(-1/4) exp(-(q - q0)^2/(4 sigma^2) + i p0 q)."""
        A = 1.0 / (2.0 * sigma * sigma)
        return cls(A, A * q0 + 1j * p0,
                   -A * q0 * q0 / 2.0 - 0.25 * np.log(2 * np.pi * sigma * sigma))

    def kick(self, kappa):
        self.A += 1j * kappa

    def drift(self, tau):
        d = 1.0 + 1j * self.A * tau
        self.C += 1j * tau * self.B ** 2 / (2.0 * d) - 0.5 * np.log(d)
        self.A /= d
        self.B /= d

    def strang_ho(self, dt, nsteps, imag=False):
        """nsteps Strang steps for V = q^2/2: kick dt/2, drift dt, kick dt/2."""
        f = -1j if imag else 1.0
        for _ in range(nsteps):
            self.kick(f * dt / 2.0)
            self.drift(f * dt)
            self.kick(f * dt / 2.0)
        return self

    def strang_ho_kvk(self, dt, nsteps):
        """nsteps real-time steps of the other ordering for V = q^2/2:
        drift dt/2, kick dt, drift dt/2."""
        for _ in range(nsteps):
            self.drift(dt / 2.0)
            self.kick(dt)
            self.drift(dt / 2.0)
        return self

    def __call__(self, q):
        return np.exp(-self.A * q * q / 2.0 + self.B * q + self.C)


def product3(fx, fy, fz, x, y, z):
    return fz(z)[:, None, None] * fy(y)[None, :, None] * fx(x)[None, None, :]


def coherent_1d(q, t, q0):
    """Continuum coherent state of H = p^2/2 + q^2/2 started at
    pi^(-1/4) exp(-(q - q0)^2/2):
    pi^(-1/4) exp(-(q - q0 cos t)^2/2 - i q0 q sin t + i (q0^2/4) sin 2t - i t/2)."""
    return np.pi ** -0.25 * np.exp(-(q - q0 * np.cos(t)) ** 2 / 2.0 - 1j * q0 * q * np.sin(t)
                                   + 1j * q0 * q0 / 4.0 * np.sin(2 * t) - 0.5j * t)
