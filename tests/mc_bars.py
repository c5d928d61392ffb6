"""Statistical bars of the Monte Carlo parity tests.

A Monte Carlo estimate is compared with an exact value through z = (estimate - exact) / SE.
The bar "within 3 standard errors" is read as a false-alarm probability: one comparison at
|z| <= 3 fails by chance with probability 2 (1 - Phi(3)) = 0.27 %.  A test that makes m
comparisons keeps that family-wise rate by bounding every |z| by z_bar(m), with
2 (1 - Phi(z_bar(m))) = 0.0027 / m (Bonferroni), so z_bar(1) = 3; and it also bounds the sum of
the m squared z-scores by the 0.9973 quantile of the chi-square law with m degrees of freedom,
which catches a bias spread thinly over many comparisons that no single |z| shows.
"""
from scipy import stats

FALSE_ALARM = 2.0 * stats.norm.sf(3.0)       # 0.0027: one comparison at 3 SE


def z_bar(m):
    """|z| bound of each of m comparisons (family-wise false-alarm rate 0.27 %)."""
    m = max(int(m), 1)
    return float(stats.norm.isf(FALSE_ALARM / (2.0 * m)))


def chi2_bar(m):
    """Bound of the sum of m squared z-scores (the chi-square(m) 0.9973 quantile)."""
    return float(stats.chi2.isf(FALSE_ALARM, max(int(m), 1)))


def t_bar(m, dof):
    """|t| bound of each of m comparisons whose standard error is estimated from the spread of
    dof + 1 independent batch means (Student's t with dof degrees of freedom)."""
    m = max(int(m), 1)
    return float(stats.t.isf(FALSE_ALARM / (2.0 * m), dof))
