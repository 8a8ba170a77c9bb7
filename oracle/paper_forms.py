"""The paper's own closed forms, written out as printed (with the readings noted).

Test infrastructure only: used by tests/, the smoke check and bench.py's CPU
baseline; the library never imports or calls it.

Used only to pin the paper's formulas against the oracle's direct interface
solves (core.spectral_amp, background.background_coefficients).  Everything is
in the paper's absolute coordinates (waves e^{+- i k_y y}), so it is evaluated
only at moderate depths and moderate lambda in the tests.

Readings of the printed formulas:
  * exponents e^{-2 k_y (d_l - d_{l-1})} in the R~ and T~ recursions and in
    Case I are read as e^{2 i k_y (d_l - d_{l-1})} (as printed in Cases II/III);
  * the downward recursion starts from R~_{L,L+1} = 0 (the Remark of Sec. 3.1);
  * the reaction components carry i/(2 k_{l',y}) (the printed 1/(2 k_{l',y})
    lacks the factor i that the free-space Sommerfeld identity requires).

Sources: Fresnel R, T (Sec. 3.1, after eq. MutiLayerHelmEquation),
eqs. Rellrecursionup, Rellrecursiondown, generaltransmission (recursions),
eqs. densityinsourcelayer, disity1, disity2 (densities, Cases I-III),
eqs. reflections, equivalent_imag_for_source, equivalent_imag_for_target,
planewavekernel (images and the uniform plane-wave kernel), and the
background-field coefficients A_l, B_l of Sec. 2.2.
"""

from __future__ import annotations

import numpy as np


def _ky(k, lam):
    s = np.sqrt(np.asarray(k, dtype=np.complex128) ** 2 - np.asarray(lam, dtype=np.complex128) ** 2)
    return np.where(s.imag < 0, -s, s)


class PaperLayers:
    """R, T, R~ (both directions) and T~ at one lambda, as functions of layer indices."""

    def __init__(self, medium, lam):
        self.d = -np.asarray(medium.interfaces, dtype=np.float64).reshape(-1)  # d_0 < d_1 < ...
        self.k = np.asarray(medium.k, dtype=np.float64)
        self.eta = np.asarray(medium.eta, dtype=np.float64)
        self.L = self.d.size
        self.lam = complex(lam)
        self.ky = _ky(self.k, self.lam)
        L = self.L
        # Rt_up[l] = R~_{l, l-1} (looking up from layer l), Rt_dn[l] = R~_{l, l+1}
        self.Rt_up = np.zeros(L + 1, dtype=np.complex128)
        self.Rt_dn = np.zeros(L + 1, dtype=np.complex128)
        for l in range(0, L):  # R~_{l+1,l} from R~_{l,l-1}
            R = self.R(l + 1, l)
            if l == 0:
                self.Rt_up[1] = R
            else:
                e = self.e2(l)
                self.Rt_up[l + 1] = (R + self.Rt_up[l] * e) / (1.0 + R * self.Rt_up[l] * e)
        for l in range(L - 1, -1, -1):  # R~_{l,l+1} from R~_{l+1,l+2}
            R = self.R(l, l + 1)
            if l == L - 1:
                self.Rt_dn[l] = R
            else:
                e = self.e2(l + 1)
                self.Rt_dn[l] = (R + self.Rt_dn[l + 1] * e) / (1.0 + R * self.Rt_dn[l + 1] * e)

    def H(self, l):
        return self.d[l] - self.d[l - 1]

    def e2(self, l):
        """e^{2 i k_{l,y} (d_l - d_{l-1})} for an interior layer (0 for the half-spaces)."""
        if l <= 0 or l >= self.L:
            return 0.0
        return np.exp(2j * self.ky[l] * self.H(l))

    def R(self, a, b):
        """Fresnel reflection R_{ab} for adjacent layers."""
        ka, kb = self.eta[a] * self.ky[a], self.eta[b] * self.ky[b]
        return (ka - kb) / (ka + kb)

    def T(self, a, b):
        ka, kb = self.eta[a] * self.ky[a], self.eta[b] * self.ky[b]
        return 2.0 * ka / (ka + kb)

    def Tt(self, lp, l):
        """General transmission T~_{l' l} from layer l' to layer l (eq. generaltransmission)."""
        if l == lp:
            return 1.0 + 0j
        if l < lp:
            v = 1.0 + 0j
            for m in range(lp - 1, l - 1, -1):
                num = self.T(m + 1, m) * np.exp(1j * (self.ky[m] - self.ky[m + 1]) * self.d[m])
                den = 1.0 + self.R(m + 1, m) * self.Rt_up[m] * self.e2(m)
                v = num * v / den
            return v
        v = 1.0 + 0j
        for m in range(lp + 1, l + 1):
            num = self.T(m - 1, m) * np.exp(1j * (self.ky[m - 1] - self.ky[m]) * self.d[m - 1])
            den = 1.0 + self.R(m - 1, m) * self.Rt_dn[m] * self.e2(m)
            v = num * v / den
        return v

    def sigma(self, l, lp):
        """Densities sigma^{ud}, sigma^{uu}, sigma^{dd}, sigma^{du} of component (l, l')."""
        Ru, Rd = self.Rt_up[lp], self.Rt_dn[lp]
        den = 1.0 - Rd * Ru * self.e2(lp)
        s_ud = Rd / den
        s_du = Ru / den
        s_uu = Ru * s_ud
        s_dd = s_uu
        if l == lp:
            return {"ud": s_ud, "uu": s_uu, "dd": s_dd, "du": s_du}
        T = self.Tt(lp, l)
        if l < lp:
            ud = T * s_ud
            uu = T * (1.0 + s_uu * self.e2(lp))
            return {"ud": ud, "uu": uu, "dd": self.Rt_up[l] * ud, "du": self.Rt_up[l] * uu}
        du = T * s_du
        dd = T * (1.0 + s_dd * self.e2(lp))
        return {"du": du, "dd": dd, "uu": self.Rt_dn[l] * du, "ud": self.Rt_dn[l] * dd}


def tau(d, m, a):
    """Reflection of a height about the interface y = -d_m (eq. reflections)."""
    return -2.0 * d[m] - a


def source_image(d, l, lp, star, ys):
    """Equivalent polarization coordinate (eq. equivalent_imag_for_source)."""
    if star == "d":
        return tau(d, lp, ys) if l <= lp else ys
    return ys if l < lp else tau(d, lp - 1, ys)


def target_image(d, l, lp, comp, y):
    """Effective target location (eq. equivalent_imag_for_target)."""
    if comp == "uu":
        return y if l < lp else tau(d, l, y)
    if comp == "ud":
        return y if l <= lp else tau(d, l, y)
    if comp == "du":
        return tau(d, l - 1, y) if l < lp else y
    return tau(d, l - 1, y) if l <= lp else y  # "dd"


def nonzero_components(L, l, lp):
    """The components that the Remark of Sec. 3.1 does not set to zero."""
    out = []
    for comp in ("ud", "uu", "dd", "du"):
        if l == 0 and comp in ("dd", "du"):
            continue
        if l == L and comp in ("uu", "ud"):
            continue
        if lp == 0 and comp in ("uu", "du"):
            continue
        if lp == L and comp in ("ud", "dd"):
            continue
        out.append(comp)
    return out


def reaction_spectral(medium, lam, l, lp, y, ys, dx: float = 0.0):
    """Sum over components of E(lambda, tau^(r), tau^(r')) sigma i/(2 k_{l',y}) (uniform form)."""
    P = PaperLayers(medium, lam)
    d = P.d
    sig = P.sigma(l, lp)
    tot = 0.0 + 0j
    for comp in nonzero_components(P.L, l, lp):
        yh = target_image(d, l, lp, comp, y)
        yb = source_image(d, l, lp, comp[1], ys)
        sg = np.sign(yh - yb)
        E = np.exp(1j * P.lam * dx + sg * (1j * P.ky[l] * yh - 1j * P.ky[lp] * yb))
        tot += E * sig[comp] * 1j / (2.0 * P.ky[lp])
    return tot


def background_paper(medium, theta: float):
    """A_l, B_l of the background field in the paper's absolute form (Sec. 2.2)."""
    k0 = float(np.asarray(medium.k)[0])
    kx = k0 * np.cos(theta)
    P = PaperLayers(medium, kx)
    L = P.L
    A = np.zeros(L + 1, dtype=np.complex128)
    B = np.zeros(L + 1, dtype=np.complex128)
    A[0] = P.Rt_dn[0] * np.exp(2j * P.ky[0] * P.d[0])
    B[L] = P.Tt(0, L)
    for l in range(1, L):
        A[l] = P.Rt_dn[l] * P.Tt(0, l) * np.exp(2j * P.ky[l] * P.d[l])
        B[l] = P.Tt(0, l)
    return kx, P.ky, A, B
