"""Analytic potentials used to pin the oracle.

* Uniform sphere: Sec. 6.1.1 (double-sphere test), potential of sphere i with
  mass M_i = 4/3 pi a_i^3 rho:  -G M (3 a^2 - d^2) / (2 a^3) inside,
  -G M / d outside.
* Smooth sphere rho = rho0 (1 - d^2/a^2)^2 for d < a: the same construction
  (enclosed mass, Gauss' law) for a density whose first derivative is also
  continuous, so the discretisation error is free of the mass-representation
  jitter the paper describes for the uniform sphere.
* Radial shell (App. A, radial problem) and the polar model problem
  u = sin 2 theta with its source (App. A, polar problem).
"""
import numpy as np


def sph_to_cart(r, th, ph):
    return r * np.sin(th) * np.cos(ph), r * np.sin(th) * np.sin(ph), r * np.cos(th)


def cyl_to_cart(R, ph, z):
    return R * np.cos(ph), R * np.sin(ph), z


def uniform_sphere_potential(d, a, rho=1.0, G=1.0):
    M = 4.0 / 3.0 * np.pi * a**3 * rho
    return np.where(d < a, -G * M * (3 * a**2 - d**2) / (2 * a**3), -G * M / np.maximum(d, 1e-300))


def smooth_sphere_density(d, a, rho0=1.0):
    return np.where(d < a, rho0 * (1.0 - (d / a) ** 2) ** 2, 0.0)


def smooth_sphere_potential(d, a, rho0=1.0, G=1.0):
    M = 32.0 * np.pi * rho0 * a**3 / 105.0
    inner = (-G * M / a
             - 4.0 * np.pi * G * rho0 * (19.0 * a**2 / 210.0
                                          - (d**2 / 6.0 - d**4 / (10 * a**2) + d**6 / (42 * a**4))))
    return np.where(d < a, inner, -G * M / np.maximum(d, 1e-300))


def radial_shell_potential(r, R1, R2):
    """App. A: solution of (1/r^2) d/dr (r^2 du/dr) = 4 pi rho, rho = 1 on [R1, R2]."""
    return np.where(r < R1, -2 * np.pi * (R2**2 - R1**2),
                    np.where(r <= R2, -2 * np.pi / (3 * r) * (3 * R2**2 * r - 2 * R1**3 - r**3),
                             -4 * np.pi / (3 * r) * (R2**3 - R1**3)))


def polar_source(th):
    """App. A: f(theta) for u = sin 2 theta."""
    return (2 * np.cos(th) * np.cos(2 * th) - 4 * np.sin(th) * np.sin(2 * th)) / np.sin(th)
