"""Image-morphology diagnostics oracle, Sec. 6.2-6.3, Eqs. (92)-(107).

Test infrastructure only.  Plain numpy with exactly rounded sums
(``math.fsum``); no blocking or reordering beyond the definitions.  The image
is row-major ``I[j, i]`` on the cell-centred screen X_i = x_min + (i + 1/2) dX,
Y_j = y_min + (j + 1/2) dY, and every integral is the pixel sum times dX dY.

Readings (the paper is silent): the "emitting image region" of the
peak-to-mean contrast is the set of pixels with I > 0; the left/right split
uses strict inequalities at pixel centres; the radial profile bins
rho_0 = sqrt(X^2 + Y^2) with width dX starting at 0, takes the mean intensity
per non-empty bin, breaks argmax ties toward the smallest radius and reports
the bin centre as rho_peak.
"""
from __future__ import annotations

import math

import numpy as np

NAMES = ["F", "X_c", "Y_c", "C", "rho_bar", "d_img", "w_img", "A_LR", "P", "rho_peak",
         "d_peak", "theta_peak"]


def screen_centres(nx, ny, x_min, x_max, y_min, y_max):
    dx = (x_max - x_min) / nx
    dy = (y_max - y_min) / ny
    X = x_min + (np.arange(nx) + 0.5) * dx
    Y = y_min + (np.arange(ny) + 0.5) * dy
    return X, Y, dx, dy


def _fsum(a) -> float:
    return math.fsum(np.asarray(a, dtype=np.float64).ravel().tolist())


def diagnostics(I, x_min, x_max, y_min, y_max, theta_g=1.0) -> dict:
    I = np.asarray(I, dtype=np.float64)
    ny, nx = I.shape
    X, Y, dx, dy = screen_centres(nx, ny, x_min, x_max, y_min, y_max)
    XX, YY = np.meshgrid(X, Y)                      # [ny, nx]
    dA = dx * dy
    F = _fsum(I) * dA                                                   # Eq. (92)
    Xc = _fsum(XX * I) * dA / F                                         # Eq. (93)
    Yc = _fsum(YY * I) * dA / F
    C = math.sqrt(Xc * Xc + Yc * Yc)                                    # Eq. (94)
    rho = np.sqrt((XX - Xc) ** 2 + (YY - Yc) ** 2)                      # Eq. (95)
    rho_bar = _fsum(rho * I) * dA / F                                   # Eq. (96)
    d_img = 2.0 * rho_bar                                               # Eq. (97)
    w_img = math.sqrt(_fsum((rho - rho_bar) ** 2 * I) * dA / F)         # Eq. (98)
    FR = _fsum(I[XX > Xc]) * dA                                         # Eq. (100)
    FL = _fsum(I[XX < Xc]) * dA
    # Eq. (99); undefined (nan) when all flux sits on the centroid column
    A_LR = (FR - FL) / (FR + FL) if FR + FL != 0.0 else math.nan
    pos = I[I > 0]
    P = float(I.max()) / (_fsum(pos) / pos.size)                        # Eq. (101)
    rho0 = np.sqrt(XX ** 2 + YY ** 2)                                   # Eq. (105)
    dr = dx
    b = np.floor(rho0 / dr).astype(np.int64)
    best_b, best_v = -1, -math.inf
    for k in range(int(b.max()) + 1):
        sel = I[b == k]
        if sel.size == 0:
            continue
        v = _fsum(sel) / sel.size
        if v > best_v:
            best_v, best_b = v, k
    rho_peak = (best_b + 0.5) * dr
    d_peak = 2.0 * rho_peak                                             # Eq. (106)
    theta_peak = d_peak * theta_g                                       # Eq. (107)
    return dict(F=F, X_c=Xc, Y_c=Yc, C=C, rho_bar=rho_bar, d_img=d_img, w_img=w_img,
                A_LR=A_LR, P=P, rho_peak=rho_peak, d_peak=d_peak, theta_peak=theta_peak)


def relative_change(Q, Q_kerr):
    """delta Q_i = (Q_i - Q_Kerr) / Q_Kerr, Eq. (102)."""
    return (Q - Q_kerr) / Q_kerr


def angular_scale(d, theta_g):
    """theta = d theta_g, Eq. (104)."""
    return d * theta_g


def rho_peak_smooth(I, x_min, x_max, y_min, y_max):
    """Differentiable reading of rho_peak (Eq. 105): the vertex of the parabola
    through the mean intensities of the argmax bin and its two neighbours,
    (b + 1/2 + delta) dX with delta = (m_- - m_+) / (2 (m_- - 2 m_0 + m_+));
    delta = 0 at the ends of the profile or for a flat triple."""
    I = np.asarray(I, dtype=np.float64)
    ny, nx = I.shape
    X, Y, dx, dy = screen_centres(nx, ny, x_min, x_max, y_min, y_max)
    XX, YY = np.meshgrid(X, Y)
    b = np.floor(np.sqrt(XX ** 2 + YY ** 2) / dx).astype(np.int64)
    means = {}
    for k in range(int(b.max()) + 1):
        sel = I[b == k]
        if sel.size:
            means[k] = _fsum(sel) / sel.size
    best = max(sorted(means), key=lambda k: (means[k], -k))
    delta = 0.0
    if best - 1 in means and best + 1 in means:
        mm, m0, mp = means[best - 1], means[best], means[best + 1]
        D = mm - 2.0 * m0 + mp
        if D != 0.0:
            delta = 0.5 * (mm - mp) / D
    return (best + 0.5 + delta) * dx
