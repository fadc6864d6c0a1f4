"""Table 1 quantities of the differentially heated cavity (Sec. 3.3), from fields
on an H x H grid of cell-centred nodes (helper of the validation tests)."""
import numpy as np


def _peak(profile, coord):
    """Maximum of a sampled profile refined by the parabola through the largest
    sample and its two neighbours; returns (value, location)."""
    k = int(np.argmax(profile))
    if 0 < k < len(profile) - 1:
        y0, y1, y2 = profile[k - 1], profile[k], profile[k + 1]
        den = y0 - 2 * y1 + y2
        if den != 0:
            d = 0.5 * (y0 - y2) / den
            return y1 - 0.25 * (y0 - y2) * d, coord[k] + d * (coord[1] - coord[0])
    return profile[k], coord[k]


def table1_quantities(ux, uy, H, alpha):
    """u_max on the vertical midline and its height, v_max on the horizontal
    midline and its abscissa; velocities in units of alpha/H, positions of H."""
    c = (np.arange(H) + 0.5) / H
    um = 0.5 * (ux[:, H // 2 - 1] + ux[:, H // 2]) * H / alpha
    vm = 0.5 * (uy[H // 2 - 1, :] + uy[H // 2, :]) * H / alpha
    u_max, y_max = _peak(um, c)
    v_max, x_max = _peak(vm, c)
    return u_max, y_max, v_max, x_max
