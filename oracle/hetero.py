"""Plain CPU oracle of the heterodyned (relative-binning) log-likelihood.

TEST INFRASTRUCTURE ONLY: the test suite and ``bench.py``'s CPU legs are the only callers; the
library never imports this module.

The paper (Sec. 1, on LISA-Black-Hole and Cornish's heterodyning) describes the idea: relative to a
reference signal h0 near the truth, the likelihood splits into a constant precomputed once and
parts that vary slowly with frequency and need only a coarse frequency sampling. This module
restates it in the relative-binning form (Zackay, Dai & Venumadhav 2018; per-mode ratios as in
Leslie, Dai & Pratten 2021):

* for every mode lm and channel c, the ratio r(f) = h_lm,c(theta; f) / h0_lm,c(f) varies slowly,
  so inside coarse bin b = [f_b, f_b+1) it is taken as linear: r ~ r0 + r1 (f - f_b), from its
  values at the two edges;
* the data and reference enter through per-bin sums over the fine grid ("summary data"), computed
  once:
    A_o[b, lm, c]      = sum_k w_c conj(d_c,k) h0_lm,c,k (f_k - f_b)^o,            o = 0, 1
    B_o[b, lm, l'm', c] = sum_k w_c h0_lm,c,k conj(h0_l'm',c,k) (f_k - f_b)^o,     o = 0, 1, 2
  with w_c = 4 / (S_c T) (Eq. eq_inner_product);
* per sample, <d|h>_c = sum_b sum_lm Re[A0 r0 + A1 r1] and
  <h|h>_c = sum_b sum_lm,l'm' Re[B0 r0 r0'* + B1 (r1 r0'* + r0 r1'*) + B2 r1 r1'*], and
  log L = sum_c (<d|h> - <h|h>/2 - <d|d>/2) (Eq. eq_ll_fd).

The coarse edges are uniform in the relative-binning phase metric
  Phi(f) = sum_gamma sgn(gamma) (f / f*_gamma)^gamma,  gamma in {-5/3, -2/3, 1, 5/3, 7/3},
with f* = f_lo for negative and f_hi for positive exponents. This bounds how far the PN phase
difference between two nearby waveforms can change inside a bin. The edges are snapped to
fine-grid bins.
"""
from __future__ import annotations

import math

import numpy as np

from oracle import oracle as O

MSUN_S = 4.925490947641267e-6
GAMMAS = (-5.0 / 3.0, -2.0 / 3.0, 1.0, 5.0 / 3.0, 7.0 / 3.0)
MODES = ((2, 2), (2, 1), (3, 3), (3, 2), (4, 4))


def band_end(theta0, mode_mask: int) -> float:
    """Largest taper end m F_isco over the modes in the mask (the reference's last frequency)."""
    fisco = 6.0 ** -1.5 / (2.0 * math.pi * theta0[0] * MSUN_S)
    return max(m * fisco for bit, (_, m) in enumerate(MODES) if (mode_mask >> bit) & 1)


def phase_metric(f, flo: float, fhi: float):
    return sum(math.copysign(1.0, g) * (np.asarray(f, dtype=float) / (flo if g < 0 else fhi)) ** g for g in GAMMAS)


# Fractions of each mode's taper end m F_isco that get a forced edge: 1 - 0.1 * 0.7^j, j = 0..10. The
# Planck taper runs from 0.9 to 1 and its shape changes fastest near the end, so the marks close in
# geometrically; the last, 0.9972, is where the weight is ~1e-15, and above it the ratio is carried
# forward.
TAPER_MARKS = tuple(1.0 - 0.1 * 0.7 ** j for j in range(11))


def taper_marks(T: float, k0: int, theta0, mode_mask: int):
    """Per mode in the mask: (bit, [grid indices of the first bins at or above each TAPER_MARKS
    fraction of m F_isco], kend = the last bin below m F_isco)."""
    fisco = 6.0 ** -1.5 / (2.0 * math.pi * theta0[0] * MSUN_S)
    out = []
    for bit, (_, m) in enumerate(MODES):
        if (mode_mask >> bit) & 1:
            fe = m * fisco
            out.append((bit, [int(math.ceil(a * fe * T)) - k0 for a in TAPER_MARKS], int(math.ceil(fe * T)) - k0 - 1))
    return out


def default_edges(T: float, k0: int, nb: int, theta0, mode_mask: int, nbins: int) -> np.ndarray:
    """Fine-grid indices e_0 = 0 < ... < e_M = kmax of the coarse bins: nbins steps uniform in the
    phase metric between the first grid frequency and the reference's band end, snapped to the
    grid, plus each mode's taper marks (TAPER_MARKS); candidates strictly between a mode's last mark
    and its last in-band bin are dropped, because there the taper weight falls towards zero and the
    ratio h/h0 is not smooth (the ratio is carried forward over that stretch instead, see
    Hetero.ratios). kmax = the last grid bin below the band end (at most nb - 1)."""
    flo = k0 / T
    kmax = min(nb - 1, int(math.ceil(band_end(theta0, mode_mask) * T)) - k0 - 1)
    fhi = (k0 + kmax) / T
    p0, p1 = phase_metric(flo, flo, fhi), phase_metric(fhi, flo, fhi)
    cand = {0, kmax}
    for j in range(1, nbins):
        target = p0 + (p1 - p0) * j / nbins
        a, b = flo, fhi                      # bisection for phase_metric(f) = target
        for _ in range(200):
            mid = 0.5 * (a + b)
            if phase_metric(mid, flo, fhi) < target:
                a = mid
            else:
                b = mid
        cand.add(int(round(0.5 * (a + b) * T)) - k0)
    marks = taper_marks(T, k0, theta0, mode_mask)
    for _, ks, _ in marks:
        cand.update(ks)
    keep = [k for k in cand if 0 <= k <= kmax and
            (k == kmax or not any(ks[-1] < k <= kend for _, ks, kend in marks))]
    return np.array(sorted(keep), dtype=np.int64)


class Hetero:
    """Summary data of one detector (oracle Detector with data and PSD) for a reference theta0."""

    def __init__(self, odet, theta0, mode_mask: int, edges):
        self.odet, self.mask = odet, int(mode_mask)
        self.theta0 = np.asarray(theta0, dtype=float).copy()
        self.e = np.asarray(edges, dtype=np.int64)
        T, k0 = odet.T, odet.k0
        K = int(self.e[-1]) + 1
        f = (k0 + np.arange(K)) / T
        self.fe = (k0 + self.e) / T
        self.modes = [bit for bit in range(5) if (mode_mask >> bit) & 1]
        h0 = np.array([O.response(odet.det, self.theta0, 1 << bit, f) for bit in self.modes])   # [md][c][k]
        w = 4.0 / (odet.psd[:, :K] * T)                                                          # [c][k]
        d = odet.data[:, :K]
        M = self.e.size - 1
        nm = len(self.modes)
        self.A = np.zeros((2, M, nm, 3), complex)
        self.B = np.zeros((3, M, nm, nm, 3), complex)
        for b in range(M):
            lo, hi = int(self.e[b]), int(self.e[b + 1]) + (1 if b == M - 1 else 0)
            df = f[lo:hi] - self.fe[b]
            wd = w[:, lo:hi] * np.conj(d[:, lo:hi])
            for o in range(2):
                self.A[o, b] = np.einsum("ck,mck->mc", wd * df ** o, h0[:, :, lo:hi])
            for o in range(3):
                self.B[o, b] = np.einsum("ck,mck,nck->mnc", w[:, lo:hi] * df ** o, h0[:, :, lo:hi],
                                         np.conj(h0[:, :, lo:hi]))
        self.h0e = h0[:, :, self.e]                                                               # [md][c][edge]
        self.dd = np.sum(np.abs(odet.data) ** 2 * 4.0 / (odet.psd * T), axis=1)                 # [c], full grid

    def ratios(self, theta):
        """r = h / h0 at the edges, per mode and channel. Past a mode's last taper mark (where the
        taper weight falls towards zero, and beyond the band end where h0 vanishes) the ratio of
        the previous edge is carried forward; so is it where h0 is exactly zero."""
        h = np.array([O.response(self.odet.det, theta, 1 << bit, self.fe) for bit in self.modes])
        klast = {bit: ks[-1] for bit, ks, _ in taper_marks(self.odet.T, self.odet.k0, self.theta0, self.mask)}
        r = np.zeros_like(h)
        for i in range(self.fe.size):
            for mi, bit in enumerate(self.modes):
                for c in range(3):
                    h0 = self.h0e[mi, c, i]
                    if self.e[i] <= klast[bit] and h0 != 0.0:
                        r[mi, c, i] = h[mi, c, i] / h0
                    elif i > 0:
                        r[mi, c, i] = r[mi, c, i - 1]
        return r                                                                                  # [md][c][edge]

    def loglike(self, theta) -> dict:
        r = self.ratios(theta)
        r0 = r[:, :, :-1]
        r1 = (r[:, :, 1:] - r[:, :, :-1]) / np.diff(self.fe)
        r0, r1 = np.moveaxis(r0, 2, 0), np.moveaxis(r1, 2, 0)                                     # [b][md][c]
        dh = np.real(np.einsum("bmc,bmc->c", self.A[0], r0) + np.einsum("bmc,bmc->c", self.A[1], r1))
        hh = np.real(np.einsum("bmnc,bmc,bnc->c", self.B[0], r0, np.conj(r0))
                     + np.einsum("bmnc,bmc,bnc->c", self.B[1], r1, np.conj(r0))
                     + np.einsum("bmnc,bmc,bnc->c", self.B[1], r0, np.conj(r1))
                     + np.einsum("bmnc,bmc,bnc->c", self.B[2], r1, np.conj(r1)))
        return {"logl": float(np.sum(dh - 0.5 * hh - 0.5 * self.dd)), "dh": dh, "hh": hh, "dd": self.dd}


def loglike_network(hets, theta) -> dict:
    rs = [h.loglike(theta) for h in hets]
    return {"logl": sum(r["logl"] for r in rs), "dh": np.array([r["dh"] for r in rs]),
            "hh": np.array([r["hh"] for r in rs]), "dd": np.array([r["dd"] for r in rs])}
