"""Shared helpers of the GPU parity tests: build both sides on the same seeded inputs."""
import math

import numpy as np

from paper_2602_12011_gb300 import workloads as W

# Parity bar on log L (Eq. eq_ll_fd): |dlogL| <= REL * (1/2 <d|d> + |<d|h>| + 1/2 <h|h>), the
# likelihood's own scale (log L itself is ~0 for noise-free data at the true parameters).
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


def assert_loglike_parity(gpu, ref_logl, ref_dhhh, dd_per_det, rel=REL):
    """gpu: dict from _lib.loglike (host arrays, with dhhh). ref_*: oracle batch outputs."""
    B = ref_logl.shape[0]
    for s in range(B):
        dh = ref_dhhh[s, :, :, 0]
        hh = ref_dhhh[s, :, :, 1]
        sc = scale_of(dh, hh, dd_per_det)
        err = abs(gpu["logl"][s] - ref_logl[s])
        assert err <= rel * sc, "sample %d: logL gpu %.17g oracle %.17g err %.3g scale %.3g" % (
            s, gpu["logl"][s], ref_logl[s], err, sc)
        # per (detector, channel) components on the same scale
        d = np.abs(gpu["dhhh"][s] - ref_dhhh[s]).max()
        assert d <= rel * sc, "sample %d: <d|h>/<h|h> err %.3g scale %.3g" % (s, d, sc)


def max_active_bins(theta, T, k0, nb):
    """Upper bound of the active bins of a sample (largest mode, m = 4, ends at 4 F_isco)."""
    M = theta[0] * 4.925490947641267e-6
    fisco = 6 ** -1.5 / (2 * math.pi * M)
    return int(min(nb, max(0, math.ceil(4 * fisco * T) - k0)))
