"""Analysis helpers of the two-phase tests: the analytic capillary-wave
solution of Section 3.4 and interface measurements on order-parameter fields.
Plain NumPy/SciPy; nothing here runs the scheme."""
from __future__ import annotations

import numpy as np


def capillary_wave_htilde(t, re: float):
    """Scaled interface displacement h~(t) = (h_eq - h_0(t)) / A_p of a small
    capillary wave between two fluids of equal density and viscosity (the
    analytic solution quoted in Section 3.4), in the scaled units of that
    section: lengths by L, times by T_c, so sigma = nu = 1 / Re, k = 2 pi.
    omega_0 = sqrt(sigma k^3 / 2), eps = nu k^2 / omega_0, z_i the roots of
    z^4 - sqrt(eps w0) z^3 - eps w0 z^2 + (eps w0)^(3/2) z + w0^2 = 0 and
    h~ = sum_i z_i w0^2 / (Z_i (z_i^2 - eps w0)) exp((z_i^2 - eps w0) t)
         erfc(z_i sqrt(t)).
    The product exp(z^2 t) erfc(z sqrt(t)) is evaluated as the Faddeeva
    function w(i z sqrt(t)), which stays finite for every root."""
    from scipy.special import wofz

    sigma = nu = 1.0 / re
    k = 2.0 * np.pi
    w0 = np.sqrt(sigma * k ** 3 / 2.0)
    ew = nu * k * k  # eps * omega_0
    z = np.roots([1.0, -np.sqrt(ew), -ew, ew ** 1.5, w0 ** 2])
    t = np.asarray(t, dtype=np.float64)
    out = np.zeros(t.shape, dtype=complex)
    for i in range(4):
        zi = np.prod([z[j] - z[i] for j in range(4) if j != i])
        out += (z[i] * w0 ** 2 / (zi * (z[i] ** 2 - ew)) * np.exp(-ew * t)
                * wofz(1j * z[i] * np.sqrt(t)))
    return out.real


def local_extrema(t, f, kind: str = "max"):
    """Times of the interior local maxima (or minima) of a sampled signal,
    refined by a parabola through the three samples around each."""
    t = np.asarray(t, dtype=np.float64)
    f = np.asarray(f, dtype=np.float64)
    s = 1.0 if kind == "max" else -1.0
    out = []
    for i in range(1, len(f) - 1):
        a, b, c = s * f[i - 1], s * f[i], s * f[i + 1]
        if b > a and b >= c:
            den = a - 2.0 * b + c
            d = 0.5 * (a - c) / den if den != 0 else 0.0
            out.append(t[i] + d * (t[i + 1] - t[i]))
    return out


def zero_crossing(col):
    """Position of the first sign change of a 1D profile, linearly
    interpolated between the two samples around it."""
    col = np.asarray(col, dtype=np.float64)
    j = int(np.where(np.diff(np.sign(col)) != 0)[0][0])
    return j + col[j] / (col[j] - col[j + 1])


def cap_angle(phi):
    """Apparent contact angle (degrees) of a drop (phi > 0) sitting on the
    wall row 0 and centred on the middle column of the grid: height h on the
    centre line and half base b on the wall row, both at phi = 0; a circular
    cap has tan(theta / 2) = h / b."""
    ny, nx = phi.shape
    centre = 0.5 * (phi[:, (nx - 1) // 2] + phi[:, nx // 2])
    h = zero_crossing(centre)
    half = phi[0, nx // 2:]
    b = zero_crossing(half) + nx // 2 - (nx - 1) / 2.0
    return float(np.degrees(2.0 * np.arctan(h / b))), float(h), float(b)


def oscillation_period(t, h):
    """Period of a damped oscillation that starts at its maximum: the time of
    the first local maximum after the signal has first turned negative
    (small wiggles of the start-up transient are skipped).  None if that
    maximum has not been reached yet."""
    h = np.asarray(h, dtype=np.float64)
    neg = np.where(h < 0.0)[0]
    if len(neg) == 0:
        return None
    i0 = int(neg[0])
    maxima = local_extrema(t[i0:], h[i0:], "max")
    return maxima[0] if maxima else None
