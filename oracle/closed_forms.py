"""Closed-form solutions on a dielectric sphere (test infrastructure).

Derived by separation of variables from the interface problem of the paper
(eq. poissonboltzmann): Laplace inside with point charges scaled by 1/eps_int,
screened Laplace (Yukawa) outside, continuity of phi and eps dphi/dn at r = a.
Potentials are in the paper's units (G = 1/(4 pi r)).
"""
import numpy as np


def born_energy(a: float, q: float, eps_int: float, eps_ext: float, kappa: float) -> float:
    """Delta G of one charge q at the centre of a sphere of radius a:
    q^2/(8 pi a) [1/(eps_ext (1 + kappa a)) - 1/eps_int]."""
    return q * q / (8.0 * np.pi * a) * (1.0 / (eps_ext * (1.0 + kappa * a)) - 1.0 / eps_int)


def born_surface_values(a: float, q: float, eps_int: float, eps_ext: float, kappa: float):
    """(phi on the surface, interior normal derivative) for the centred charge."""
    phi = q / (4.0 * np.pi * eps_ext * (1.0 + kappa * a) * a)
    dphi_int = -q / (4.0 * np.pi * eps_int * a * a)
    return phi, dphi_int


def _g_ratios(x: float, nmax: int):
    """g_n = x k_n'(x)/k_n(x) for the decaying modified spherical Bessel
    functions, n = 0..nmax, through the ratio rho_n = k_{n-1}/k_n:
    k_{n+1} = k_{n-1} + (2n+1)/x k_n  =>  rho_{n+1} = 1/(rho_n + (2n+1)/x),
    k_n' = -k_{n-1} - (n+1)/x k_n      =>  g_n = -x rho_n - (n+1)."""
    g = np.empty(nmax + 1)
    if x == 0.0:  # Laplace exterior r^-(n+1)
        return -(np.arange(nmax + 1) + 1.0)
    g[0] = -(1.0 + x)
    rho = x / (1.0 + x)  # k_0 / k_1
    for n in range(1, nmax + 1):
        g[n] = -x * rho - (n + 1.0)
        rho = 1.0 / (rho + (2.0 * n + 1.0) / x)
    return g


def _legendre(nmax: int, c: float):
    p = np.empty(nmax + 1)
    p[0] = 1.0
    if nmax >= 1:
        p[1] = c
    for n in range(1, nmax):
        p[n + 1] = ((2 * n + 1) * c * p[n] - n * p[n - 1]) / (n + 1)
    return p


def kirkwood_reaction_potential(a, xq, q, eps_int, eps_ext, kappa, nmax=200):
    """phi_reac at every charge position for charges inside a sphere of radius a:
    phi_reac(x_i) = sum_k q_k/(4 pi eps_int a) sum_n (r_i r_k/a^2)^n P_n(cos g_ik) C_n,
    C_n = ((n+1) eps_int + eps_ext g_n) / (n eps_int - eps_ext g_n)."""
    xq = np.asarray(xq, dtype=np.float64).reshape(-1, 3)
    q = np.asarray(q, dtype=np.float64).reshape(-1)
    g = _g_ratios(kappa * a, nmax)
    n = np.arange(nmax + 1)
    C = ((n + 1) * eps_int + eps_ext * g) / (n * eps_int - eps_ext * g)
    rr = np.linalg.norm(xq, axis=1)
    phi = np.zeros(len(q))
    for i in range(len(q)):
        for k in range(len(q)):
            if rr[i] == 0.0 or rr[k] == 0.0:
                c = 1.0
            else:
                c = float(np.dot(xq[i], xq[k]) / (rr[i] * rr[k]))
            P = _legendre(nmax, min(1.0, max(-1.0, c)))
            s = (rr[i] * rr[k] / (a * a)) ** n
            phi[i] += q[k] / (4.0 * np.pi * eps_int * a) * float(np.sum(s * P * C))
    return phi


def kirkwood_energy(a, xq, q, eps_int, eps_ext, kappa, nmax=200):
    """Delta G = 1/2 sum_i q_i phi_reac(x_i) for charges inside the sphere."""
    q = np.asarray(q, dtype=np.float64).reshape(-1)
    return 0.5 * float(np.dot(q, kirkwood_reaction_potential(a, xq, q, eps_int, eps_ext, kappa, nmax)))


def sphere_constant_eigs(a: float, kappa: float):
    """Operators applied to the constant 1 on a sphere of radius a:
    (V1, K1, D1), with T1 = K1. Integrals over the sphere in the chord length
    rho = |x - y| (dS = 2 pi rho drho / ... over rho in [0, 2a]):
      V1 = (1 - e^{-2 kappa a}) / (2 kappa)
      K1 = -(1 - e^{-2 kappa a}) / (2 kappa a) + e^{-2 kappa a} / 2
      D1 = (1/2 + K1) (1 + kappa a) / a
    and the Laplace limits a, -1/2, 0."""
    if kappa == 0.0:
        return a, -0.5, 0.0
    e = np.exp(-2.0 * kappa * a)
    V1 = (1.0 - e) / (2.0 * kappa)
    K1 = -(1.0 - e) / (2.0 * kappa * a) + 0.5 * e
    D1 = (0.5 + K1) * (1.0 + kappa * a) / a
    return V1, K1, D1


def laplace_sphere_eigs(a: float, n: int):
    """Laplace operators on spherical harmonics of degree n on a sphere of radius a:
    V = a/(2n+1), K = T = -1/(2(2n+1)), D = n(n+1)/(a(2n+1))."""
    return a / (2 * n + 1), -1.0 / (2.0 * (2 * n + 1)), n * (n + 1) / (a * (2 * n + 1))
