"""Couplings for the small-sphere tests.

The sphere form factors are the printed expression of Eq.
sphere_density_operator times kappa = 1/(2 pi sqrt(n_orb)), the torus's
normalisation.  The couplings multiply the squared form factors, so a test
that wants the strong coupling of the printed scale on a small sphere takes
u / kappa^2 = 4 pi^2 n_orb u (and the anisotropy likewise); only the fixed
U_0 = 1 term is then weaker by kappa^2.
"""
import math


def sphere_u(u, norb):
    return u * 4.0 * math.pi ** 2 * norb
