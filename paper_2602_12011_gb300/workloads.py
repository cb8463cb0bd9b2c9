"""Seeded synthetic workloads: detector descriptions, frequency-grid index ranges, parameter
draws and standard-normal noise draws.

This module holds none of the method's arithmetic (no waveform, response, PSD or likelihood
formula): it only states the inputs, so that the CUDA path and the CPU oracle consume the same
numbers. Random numbers come from numpy's PCG64 with the seeds listed here.

Workloads follow the paper's performance and PE set-ups (Sec. 3.1-3.2): frequency bins
f_k = k/T from numpy.fft.rfftfreq at a 10 s cadence truncated to [1e-4, 5e-2] Hz; the injected
source of Table tab_pe_res for the sky position, inclination, phase and polarisation.
"""
from __future__ import annotations

import math

import numpy as np

# Mode-mask bits: (2,2), (2,1), (3,3), (3,2), (4,4).
MODES = ((2, 2), (2, 1), (3, 3), (3, 2), (4, 4))
MODE_22 = 0x1
MODE_ALL = 0x1F

DEG = math.pi / 180.0

# Detector descriptions (orbit 0: heliocentric Keplerian; 1: geocentric). Initial revolution
# angles -20 deg (Taiji), 0 (LISA), +20 deg (TianQin), Sec. 3.2.
LISA = dict(name="LISA", orbit=0, arm_m=2.5e9, alpha0=0.0, cartwheel0=0.0, tdi_gen=20, psd_shaping=1,
            oms_m_rtHz=15e-12, acc_ms2_rtHz=3e-15)
TAIJI = dict(name="Taiji", orbit=0, arm_m=3.0e9, alpha0=-20.0 * DEG, cartwheel0=0.0, tdi_gen=20, psd_shaping=1,
             oms_m_rtHz=8e-12, acc_ms2_rtHz=3e-15)
TIANQIN = dict(name="TianQin", orbit=1, arm_m=1.7e8, alpha0=20.0 * DEG, geo_period_s=3.65 * 86400.0,
               geo_lon=120.5 * DEG, geo_lat=-4.7 * DEG, tdi_gen=20, psd_shaping=0,
               oms_m_rtHz=1e-12, acc_ms2_rtHz=1e-15)

F_LO, F_HI = 1e-4, 5e-2


def grid(T: float, f_lo: float = F_LO, f_hi: float = F_HI):
    """Index range of the bins f_k = k/T inside [f_lo, f_hi]: returns (k0, nbins)."""
    k0 = int(math.ceil(f_lo * T - 1e-9))
    k1 = int(math.floor(f_hi * T + 1e-9))
    return k0, k1 - k0 + 1


# Parameter vector order: Mtot[Msun], q=m1/m2>=1, chi1, chi2, dL[Gpc], iota, phi_c, lambda, beta,
# psi, t_c[s].
PARAM_NAMES = ("Mtot", "q", "chi1", "chi2", "dL", "iota", "phi_c", "lambda", "beta", "psi", "t_c")


def theta_injection(T: float, tc_frac: float = 0.8) -> np.ndarray:
    """The single-source workload: Mtot 1e6 Msun, q 2, spins 0.5/0.3, dL 25.8 Gpc; inclination,
    phase, sky position and polarisation of Table tab_pe_res; t_c at tc_frac of the span."""
    return np.array([1e6, 2.0, 0.5, 0.3, 25.8, 0.4, 1.3, 1.375, -1.2108, 2.659, tc_frac * T])


def draw_prior(B: int, seed: int, T: float, tc_lo: float = 0.75, tc_hi: float = 0.85) -> np.ndarray:
    """B samples: Mtot ~ U[1e5, 1e7], q ~ U[1, 10], chi ~ U[-0.99, 0.99], isotropic sky and
    orientation, psi ~ U[0, pi), phi_c ~ U[0, 2 pi), dL ~ U[1, 50] Gpc, t_c ~ U[tc_lo, tc_hi] T."""
    rng = np.random.Generator(np.random.PCG64(seed))
    th = np.empty((B, 11))
    th[:, 0] = rng.uniform(1e5, 1e7, B)
    th[:, 1] = rng.uniform(1.0, 10.0, B)
    th[:, 2] = rng.uniform(-0.99, 0.99, B)
    th[:, 3] = rng.uniform(-0.99, 0.99, B)
    th[:, 4] = rng.uniform(1.0, 50.0, B)
    th[:, 5] = np.arccos(rng.uniform(-1.0, 1.0, B))
    th[:, 6] = rng.uniform(0.0, 2 * math.pi, B)
    th[:, 7] = rng.uniform(0.0, 2 * math.pi, B)
    th[:, 8] = np.arcsin(rng.uniform(-1.0, 1.0, B))
    th[:, 9] = rng.uniform(0.0, math.pi, B)
    th[:, 10] = rng.uniform(tc_lo, tc_hi, B) * T
    return th


def normals(nbins: int, seed: int) -> np.ndarray:
    """Standard-normal draws for the noise of three channels: array [3][nbins][2] (Re, Im)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal((3, nbins, 2))


# Named workloads (seeds fixed).
SEED_NOISE_SINGLE = 12011
SEED_BATCH_HM = 2602
SEED_BATCH_NET = 2603


def single_22():
    """Plain path: one LISA-like detector, (2,2) only, T = 2^20 s, one parameter point."""
    T = 2.0 ** 20
    k0, nb = grid(T)
    return dict(name="lisa_22_T2^20", dets=[(LISA, T, k0, nb)], theta=theta_injection(T)[None, :],
                mode_mask=MODE_22, inj=theta_injection(T), inj_mask=MODE_22, noise_seed=SEED_NOISE_SINGLE)


def batch_hm(B: int = 1024):
    """One LISA-like detector, modes 22/21/33/32/44, T = 2^22 s, B prior samples."""
    T = 2.0 ** 22
    k0, nb = grid(T)
    return dict(name="lisa_hm_T2^22_B%d" % B, dets=[(LISA, T, k0, nb)], theta=draw_prior(B, SEED_BATCH_HM, T),
                mode_mask=MODE_ALL, inj=theta_injection(T), inj_mask=MODE_ALL, noise_seed=SEED_NOISE_SINGLE)


def network_hm(B: int = 4096):
    """LISA (2^22 s) + Taiji (2^21 s) + TianQin (2^20 s), 5 modes, B samples with t_c inside
    every span (t_c ~ U[0.75, 0.85] 2^20 s)."""
    Ts = (2.0 ** 22, 2.0 ** 21, 2.0 ** 20)
    dets = []
    for det, T in zip((LISA, TAIJI, TIANQIN), Ts):
        k0, nb = grid(T)
        dets.append((det, T, k0, nb))
    inj = theta_injection(2.0 ** 20)
    return dict(name="network_hm_B%d" % B, dets=dets, theta=draw_prior(B, SEED_BATCH_NET, 2.0 ** 20),
                mode_mask=MODE_ALL, inj=inj, inj_mask=MODE_ALL, noise_seed=SEED_NOISE_SINGLE)
