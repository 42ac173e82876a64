"""Anisotropic scattering of the family dsigma/dOmega = sigma(v) (1 + beta cos theta) / (4 pi)
(oracle, FP64; test infrastructure: only tests/ use it).

Sec. 2.4 separates the two cross sections the method uses: the Monte Carlo's scattering
probability takes the total cross section sigma (Eq. dm-update-prob), the gas's exchange rates
the momentum-transfer cross section sigma_bar = int (1 - cos theta) dsigma/dOmega dOmega
(Eqs. scrA, scrB), and the two sides stay equal and opposite in expectation only if each uses
its own.  The power-law runs are isotropic (sigma = sigma_bar); for this family, with
-1 <= beta <= 1 and theta the angle between the relative velocity before and after the
collision, <cos theta> = beta / 3 and so

    sigma_bar = sigma (1 - beta / 3).

The post-collision direction: cos theta has the density (1 + beta m) / 2 on [-1, 1], whose
cumulative distribution is F(m) = [(m + 1) + beta (m^2 - 1) / 2] / 2.  With c = 2u - 1 the
isotropic cosine the step draws anyway (the same stream word), F(m) = u has the root

    m = (2c + beta) / (1 + sqrt((1 - beta)^2 + 2 beta (1 + c)))

(the quadratic's root written without the cancellation of small beta); beta = 0 gives m = c.
The azimuth phi is the step's isotropic azimuth, measured in an orthonormal basis (e1, e2)
perpendicular to the incoming direction n, built by the branch-free construction of Duff et
al. (2017), "Building an orthonormal basis, revisited", JCGT 6(1):

    n' = m n + sqrt(1 - m^2) (cos phi e1 + sin phi e2).

With beta = 0 the step keeps its isotropic form n' = (sin theta cos phi, sin theta sin phi,
cos theta) in the fixed axes, which has the same distribution.

Parity: pinned by the closed-form F (the root inverts it), the moments of the sampled cosine,
|n'| = 1 with n.n' = m, and the statistical equivalence of the Monte Carlo's momentum and
energy changes with the sigma_bar expectations (tests/test_oracle_aniso.py).
"""
import numpy as np


def sbar_factor(beta):
    """sigma_bar / sigma = 1 - <cos theta> = 1 - beta / 3."""
    return 1.0 - float(beta) / 3.0


def check_beta(beta):
    beta = float(beta)
    if not (-1.0 <= beta <= 1.0):
        raise ValueError("beta must lie in [-1, 1] (dsigma/dOmega >= 0)")
    return beta


def cdf(m, beta):
    """F(m) of cos theta for the density (1 + beta m) / 2 on [-1, 1]."""
    m = np.asarray(m, dtype=np.float64)
    return 0.5 * ((m + 1.0) + 0.5 * beta * (m * m - 1.0))


def cos_from_isotropic(c, beta):
    """The cosine with density (1 + beta m) / 2 at the quantile u = (c + 1) / 2."""
    c = np.asarray(c, dtype=np.float64)
    if beta == 0.0:
        return c
    disc = (1.0 - beta) ** 2 + 2.0 * beta * (1.0 + c)
    return (2.0 * c + beta) / (1.0 + np.sqrt(np.maximum(disc, 0.0)))


def onb(n):
    """Two unit vectors (e1, e2) with (e1, e2, n) orthonormal (Duff et al. 2017)."""
    x, y, z = n
    s = 1.0 if z >= 0.0 else -1.0
    a = -1.0 / (s + z)
    b = x * y * a
    e1 = np.array([1.0 + s * x * x * a, s * b, -s * x])
    e2 = np.array([b, s + y * y * a, -y])
    return e1, e2


def new_direction(n_old, c, phi, beta):
    """The post-collision unit direction n' from the step's (cos theta, phi) draws c, phi."""
    if beta == 0.0:
        st = np.sqrt(max(0.0, 1.0 - c * c))
        return np.array([st * np.cos(phi), st * np.sin(phi), c])
    m = float(cos_from_isotropic(c, beta))
    st = np.sqrt(max(0.0, 1.0 - m * m))
    e1, e2 = onb(n_old)
    return m * n_old + st * (np.cos(phi) * e1 + np.sin(phi) * e2)
