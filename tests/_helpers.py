"""Shared helpers of the GPU parity tests: build both sides on the same seeded inputs."""
import json
import math
import os

import numpy as np

from paper_2602_12011_gb300 import workloads as W

AU_S = 499.00478383615643       # 1 au / c [s]

# Parity bar (Eq. eq_ll_fd, Eq. eq_inner_product), relative 1e-10 on each quantity's own scale:
#   log L          : 1/2 <d|d> + |<d|h>| + 1/2 <h|h>  (log L itself is ~0 for noise-free data at the
#                    true parameters, so a relative bar on log L alone is ill-posed)
#   <h|h>_{I,c}    : <h|h>_{I,c} itself
#   <d|h>_{I,c}    : sqrt(<d|d>_{I,c} <h|h>_{I,c}), the Cauchy-Schwarz bound of <d|h> (an error dh in
#                    the signal moves <d|h> by at most sqrt(<d|d><dh|dh>))
# plus the rounding floor of the arithmetic both sides compute in (unit roundoff U64 = 2^-53, or
# U_DW = 2^-48 for the double-word geometry of PE_PREC_MIXED), from two sources per bin:
#   - the T channel (X + Y + Z)/sqrt3 cancels to O((pi f L)^2) of X, Y, Z, whose rounding is of the
#     size of the A/E signal: an absolute error ~ u max(|A|, |E|) per bin;
#   - phases of magnitude Phi (TaylorF2 phase plus the Doppler phase, up to ~1e6 rad) are known to
#     ~u Phi rad, an error ~ u Phi |h| per bin.
# With Q_{I,c} = sum_b w_c (max(|A_b|, |E_b|)^2 + Phi_b^2 |h_c,b|^2), Cauchy-Schwarz bounds the
# effect on <h|h> by 2 kappa u sqrt(<h|h> Q) and on <d|h> by kappa u sqrt(<d|d> Q). Q is of the
# size of <h|h> for A and E, so the floor matters only for the suppressed T channel and for
# phases beyond ~1e5 rad. kappa = 8: the oracle's own rounding, measured against its long double
# twin (test_oracle_rounding_against_long_double), needs kappa < 0.1 there.
U64 = 2.0 ** -53
U_DW = 2.0 ** -48
KAPPA = 8.0
REL = 1e-10


def grid_f(T, k0, nb):
    return (k0 + np.arange(nb)) / T


def oracle_detector(O, det, T, k0, nb, inj, inj_mask, noise_seed):
    """Data = oracle injection + noise from the seeded normals; PSD = oracle model."""
    nrm = None if noise_seed is None else W.normals(nb, noise_seed)
    data = O.make_data(det, inj, inj_mask, T, k0, nb, nrm)
    psd = O.psd(det, grid_f(T, k0, nb))
    return O.Detector(det, T, k0, nb, data, psd)


def library_detector(Lb, odet):
    """Library detector fed with the oracle's data and PSD (identical inputs on both sides)."""
    d = Lb.Detector(odet.det, odet.T, odet.k0, odet.nb)
    d.set_data(odet.data, odet.psd)
    return d


def scale_of(dh, hh, dd):
    return 0.5 * np.sum(dd) + abs(np.sum(dh)) + 0.5 * np.sum(hh)


def record_margin(name, ratio):
    """Append the worst error/tolerance ratio of a check to the file named by PE_PARITY_LOG (if set):
    a ratio of 0.01 means the check passed with two orders of magnitude to spare."""
    path = os.environ.get("PE_PARITY_LOG")
    if not path:
        return
    with open(path, "a") as fh:
        fh.write(json.dumps({"check": name, "worst_err_over_tol": float(ratio)}) + "\n")


def phase_magnitude(O, theta, mask, f):
    """Per bin, the largest phase magnitude any active mode carries: |Psi_lm(f)| (the oracle's
    TaylorF2 phase, 2 pi f t_c included) plus the Doppler phase bound 2 pi f (1 au)."""
    P = np.zeros_like(f)
    for bit, (l, m) in enumerate(W.MODES):
        if (mask >> bit) & 1:
            P = np.maximum(P, np.abs(O.mode(theta, l, m, f)[2]))
    return P + 2 * math.pi * f * AU_S


def floor_terms(O, ods, theta, mask):
    """Q[s][I][c] = sum_b w_c (max(|A_b|, |E_b|)^2 + Phi_b^2 |h_c,b|^2) from the oracle's per-bin
    signal and weights w_c = 4/(S_c T) (see the rounding floor above)."""
    from concurrent.futures import ThreadPoolExecutor
    theta = np.atleast_2d(theta)

    def one(args):
        s, i = args
        od = ods[i]
        f = grid_f(od.T, od.k0, od.nb)
        h = O.response(od.det, theta[s], mask & 0x1F, f)
        w = 4.0 / (od.psd * od.T)
        ae2 = np.maximum(np.abs(h[0]), np.abs(h[1])) ** 2
        P2 = phase_magnitude(O, theta[s], mask & 0x1F, f) ** 2
        return s, i, np.sum(w * (ae2[None, :] + P2[None, :] * np.abs(h) ** 2), axis=1)

    Q = np.zeros((theta.shape[0], len(ods), 3))
    jobs = [(s, i) for s in range(theta.shape[0]) for i in range(len(ods))]
    with ThreadPoolExecutor(max_workers=min(16, len(jobs))) as ex:   # ctypes releases the GIL
        for s, i, q in ex.map(one, jobs):
            Q[s, i] = q
    return Q


def assert_loglike_parity(gpu, ref_logl, ref_dhhh, dd, Q, rel=REL, u=U64, name="loglike"):
    """gpu: dict from _lib.loglike (host arrays, with dhhh). ref_*: oracle batch outputs.
    dd: <d|d> per (detector, channel), shape [ndet][3] (or [3] for one detector). Q: floor_terms of
    the same samples, [B][ndet][3]."""
    B, ndet = ref_dhhh.shape[0], ref_dhhh.shape[1]
    dd = np.asarray(dd, dtype=np.float64).reshape(ndet, 3)
    Q = np.asarray(Q, dtype=np.float64).reshape(B, ndet, 3)
    worst = {"logl": 0.0, "hh": 0.0, "dh": 0.0}
    for s in range(B):
        dh = ref_dhhh[s, :, :, 0]
        hh = ref_dhhh[s, :, :, 1]
        sc = scale_of(dh, hh, dd)
        err = abs(gpu["logl"][s] - ref_logl[s])
        worst["logl"] = max(worst["logl"], err / (rel * sc))
        assert err <= rel * sc, "sample %d: logL gpu %.17g oracle %.17g err %.3g scale %.3g" % (
            s, gpu["logl"][s], ref_logl[s], err, sc)
        g = np.asarray(gpu["dhhh"][s])
        # <h|h> per (detector, channel) on its own magnitude (exactly 0 when no bin is active)
        e_hh = np.abs(g[:, :, 1] - hh)
        t_hh = rel * hh + 2 * KAPPA * u * np.sqrt(hh * Q[s])
        worst["hh"] = max(worst["hh"], float(np.max(np.where(t_hh > 0, e_hh / np.where(t_hh > 0, t_hh, 1), 0))))
        assert np.all((e_hh <= t_hh) | ((hh == 0) & (g[:, :, 1] == 0))), (
            "sample %d: <h|h> err/<h|h> %s, err/tol %s" % (s, e_hh / np.maximum(hh, 1e-300), e_hh / t_hh))
        # <d|h> per (detector, channel) on the Cauchy-Schwarz scale sqrt(<d|d><h|h>)
        e_dh = np.abs(g[:, :, 0] - dh)
        t_dh = rel * np.sqrt(dd * hh) + KAPPA * u * np.sqrt(dd * Q[s])
        worst["dh"] = max(worst["dh"], float(np.max(np.where(t_dh > 0, e_dh / np.where(t_dh > 0, t_dh, 1), 0))))
        assert np.all((e_dh <= t_dh) | ((hh == 0) & (g[:, :, 0] == 0))), (
            "sample %d: <d|h> err/sqrt(<d|d><h|h>) %s, err/tol %s" % (
                s, e_dh / np.maximum(np.sqrt(dd * hh), 1e-300), e_dh / t_dh))
    for k, v in worst.items():
        record_margin("%s:%s" % (name, k), v)


def assert_signal_parity(h, ref, name, phi, rel=REL, u=U64, kappa=64.0):
    """Per-bin A/E/T signal against the oracle's direct evaluation: rel |h_c| per bin, plus the
    rounding floor kappa u (Phi |h_c| + max(|A|, |E|) + max_b |h_c|):
    - Phi |h_c|: phases of magnitude Phi (phase_magnitude) carry ~u Phi rad on either side;
    - max(|A|, |E|): T = (X + Y + Z)/sqrt(3) cancels to O((pi f L)^2) of the link terms, which
      round at the size of the A/E signal;
    - max_b |h_c|: near a zero of a channel's transfer function the absolute rounding of the
      uncancelled terms remains.
    kappa = 64: the oracle alone, against its long double twin, needs up to ~16 (its TaylorF2 phase
    is a sum of rounded terms), and the library rounds independently."""
    ae = np.maximum(np.abs(ref[0]), np.abs(ref[1]))
    worst = 0.0
    for c in range(3):
        err = np.abs(h[c] - ref[c])
        tol = rel * np.abs(ref[c]) + kappa * u * (phi * np.abs(ref[c]) + ae + np.abs(ref[c]).max())
        ok = tol > 0
        worst = max(worst, float(np.max(err[ok] / tol[ok])) if ok.any() else 0.0)
        assert np.all(err <= tol), (name, c, np.max(err / (np.abs(ref[c]) + 1e-300)), np.max(err[ok] / tol[ok]))
    record_margin(name, worst)


def grad_tolerance(g_ref, hh, F_ii, rel=1e-9):
    """Bar of one gradient component against the oracle's dual-number gradient (Sec. 2.3, the
    adjoint of Eq. eq_ll_fd): rel * (|g_i| + sqrt((1 + <h|h>) F_ii)).

    g_i = <d - h | d_i h>. A relative error e of the signal's derivative moves the noise part
    <n | d_i h> by about e sqrt(F_ii) (its standard deviation is sqrt(F_ii)); an error e of the signal
    moves <h | d_i h> by at most e sqrt(<h|h> F_ii). No <d|d> enters the scale."""
    return rel * (abs(g_ref) + math.sqrt((1.0 + hh) * max(F_ii, 0.0)))


def max_active_bins(theta, T, k0, nb):
    """Upper bound of the active bins of a sample (largest mode, m = 4, ends at 4 F_isco)."""
    M = theta[0] * 4.925490947641267e-6
    fisco = 6 ** -1.5 / (2 * math.pi * M)
    return int(min(nb, max(0, math.ceil(4 * fisco * T) - k0)))
