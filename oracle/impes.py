"""Two-phase flow by the improved IMPES scheme (Section 6), FP64 NumPy.

Test infrastructure only (see the package docstring).

Fluid model: S* = (S - s_wc) / (1 - s_wc - s_or) clipped to [0, 1],
k_rw = S*^2, k_ro = (1 - S*)^2, total mobility lambda = k_rw/mu_w + k_ro/mu_o,
fractional flow f_w = (k_rw/mu_w) / lambda.

Pressure step, Eq. (IMP): the pressure system with permeability lambda(S) kappa
and, at the cells a producer crosses, the well term q = W (p_BH - p),
W = WI kappa^x lambda(S): (A + W) p = q_inj + W p_BH.

Saturation sub-steps, Eq. (ES): phi (S^{m+1} - S^m) / dt = q_w - div(F),
F = f_w(S_up) v on every face (S_up: the cell the flow leaves), q_w = q_inj at
the injector and f_w(S) W (p_BH - p) at a producer; dt = DS_max / max |dS/dt|.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .tpfa import velocity


@dataclass
class Fluid:
    mu_w: float = 0.3       # cP (Section 6)
    mu_o: float = 3.0
    s_wc: float = 0.2
    s_or: float = 0.2


def mobilities(S, fl: Fluid):
    """(lambda, f_w) of the fluid model at saturation S."""
    s = np.clip((np.asarray(S, dtype=np.float64) - fl.s_wc) / (1.0 - fl.s_wc - fl.s_or), 0.0, 1.0)
    mw = s * s / fl.mu_w
    mo = (1.0 - s) ** 2 / fl.mu_o
    return mw + mo, mw / (mw + mo)


def well_index(hx: float, hy: float, rw: float) -> float:
    """The well index of Section 6: (1/hx^2 + 1/hy^2) / ((2/pi)(hy/hx log(r1/rw) +
    hx/hy log(r2/rw)) - 1), r1 = sqrt(9 hx^2 + hy^2) / 2, r2 = sqrt(hx^2 + 9 hy^2) / 2."""
    r1 = np.sqrt(9.0 * hx * hx + hy * hy) / 2.0
    r2 = np.sqrt(hx * hx + 9.0 * hy * hy) / 2.0
    return (1.0 / hx ** 2 + 1.0 / hy ** 2) / ((2.0 / np.pi) * (hy / hx * np.log(r1 / rw) + hx / hy * np.log(r2 / rw))
                                              - 1.0)


def pressure_terms(S, kappa3, wi, q_inj, p_bh: float, fl: Fluid):
    """(lambda(S) kappa, W, b) of Eq. (IMP); kappa3 (3, ...), the others like S."""
    lam, _ = mobilities(S, fl)
    ke = np.asarray(kappa3, dtype=np.float64) * lam[None]
    W = np.asarray(wi, dtype=np.float64) * np.asarray(kappa3, dtype=np.float64)[0] * lam
    return ke, W, np.asarray(q_inj, dtype=np.float64) + W * p_bh


def saturation_rate(S, v, p, W, p_bh: float, q_inj, phi, h, fl: Fluid):
    """dS/dt of every cell (Eq. (ES)): upstream face fluxes, the well sources."""
    S = np.asarray(S, dtype=np.float64)
    _, fw = mobilities(S, fl)
    div = np.zeros_like(S)
    for d, ax in ((0, 2), (1, 1), (2, 0)):
        vf = v[d]
        nxt = np.roll(fw, -1, axis=ax)                      # f_w of the +d neighbour
        F = np.where(vf >= 0.0, fw, nxt) * vf              # flux through each cell's +d face
        sl = [slice(None)] * 3
        sl[ax] = slice(-1, None)
        F[tuple(sl)] = 0.0                                  # boundary faces: no flow
        Fm = np.roll(F, 1, axis=ax)                         # flux through the -d face
        sl[ax] = slice(0, 1)
        Fm[tuple(sl)] = 0.0
        div += (F - Fm) / h[d]
    qw = np.asarray(q_inj) + fw * np.asarray(W) * (p_bh - np.asarray(p))
    return (qw - div) / np.asarray(phi)


def transport(S, v, p, W, p_bh: float, q_inj, phi, h, M: int, ds_max: float, fl: Fluid):
    """M sub-steps of Eq. (ES); returns (S, total time)."""
    S = np.array(S, dtype=np.float64)
    t = 0.0
    for _ in range(M):
        r = saturation_rate(S, v, p, W, p_bh, q_inj, phi, h, fl)
        m = float(np.abs(r).max())
        dt = ds_max / m if m > 0 else 0.0
        S = S + dt * r
        t += dt
    return S, t


def face_velocity(T, p, h):
    """The total velocity of the pressure p (Eq. (velocity) with lambda in T)."""
    return velocity(T, p, h)
