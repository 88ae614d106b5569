"""Data preprocessing: mass-to-light ratio maps from a colour (Eq. 20, App. C).

When no stellar-population M/L map is available, log10 (M/L)_alpha = a + b (m_beta -
m_gamma) from two bands' magnitudes.  The error of log10 M/L propagates the magnitude
errors and adds the relation's scatter sigma_alpha in quadrature (App. C); the linear map
and its (first-order) error are what the likelihood's M/L term compares with.  Defaults
are the paper's choice for NGC 7683: alpha = gamma = SDSS i, beta = SDSS g, a = -0.70,
b = 0.89, sigma_alpha = 0.07 (App. C).  Host-side numpy; off the likelihood's hot path.
"""
from __future__ import annotations

import numpy as np

LN10 = float(np.log(10.0))


def ml_from_colour(m_beta, m_gamma, err_beta=0.0, err_gamma=0.0, a=-0.70, b=0.89, sigma_alpha=0.07):
    """(M/L, delta M/L, log10 M/L, delta log10 M/L) per pixel for magnitudes m_beta, m_gamma."""
    m_beta = np.asarray(m_beta, dtype=np.float64)
    m_gamma = np.asarray(m_gamma, dtype=np.float64)
    log_ml = a + b * (m_beta - m_gamma)
    err_log = np.sqrt(b * b * (np.square(err_beta) + np.square(err_gamma)) + sigma_alpha ** 2)
    ml = np.power(10.0, log_ml)
    return ml, ml * LN10 * err_log, log_ml, err_log + 0.0 * log_ml
