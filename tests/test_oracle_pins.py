"""Pins of the FP64 CPU oracle against closed forms, limits, identities and brute force.

Each test fixes one part of the oracle to something other than the oracle itself (a textbook
closed form, a limit the paper's equations reduce to, an exact algebraic identity, or a
brute-force evaluation), so that a dropped term, a wrong sign or index or a transposed operand
in the oracle fails at least one of them. Paper references are to arXiv:2602.12011.
"""
import math

import numpy as np
import pytest

from paper_2602_12011_gb300 import workloads as W

MSUN_S = 4.925490947641267e-6
GPC_S = 1.02927125054339e17
C_SI = 299792458.0

TH = np.array([1e6, 2.0, 0.5, 0.3, 25.8, 0.4, 1.3, 1.375, -1.2108, 2.659, 0.8 * 2.0 ** 20])


def chirp_mass_s(th):
    M = th[0] * MSUN_S
    eta = th[1] / (1 + th[1]) ** 2
    return eta ** 0.6 * M


# -------------------------------------------------------------------------------------------
# Spin-weighted spherical harmonics
# -------------------------------------------------------------------------------------------
def ylm_closed(l, m, i):
    """Closed forms of -2Y_lm(iota, 0) (Ajith et al. 2007, arXiv:0709.0093, Eq. II.9 list)."""
    c2, s2 = math.cos(i / 2), math.sin(i / 2)
    pi = math.pi
    table = {
        (2, 2): math.sqrt(5 / (64 * pi)) * (1 + math.cos(i)) ** 2,
        (2, -2): math.sqrt(5 / (64 * pi)) * (1 - math.cos(i)) ** 2,
        (2, 1): math.sqrt(5 / (16 * pi)) * math.sin(i) * (1 + math.cos(i)),
        (2, -1): math.sqrt(5 / (16 * pi)) * math.sin(i) * (1 - math.cos(i)),
        (3, 3): -math.sqrt(21 / (2 * pi)) * c2 ** 5 * s2,
        (3, -3): math.sqrt(21 / (2 * pi)) * c2 * s2 ** 5,
        (3, 2): math.sqrt(7 / pi) / 2 * c2 ** 4 * (3 * math.cos(i) - 2),
        (3, -2): math.sqrt(7 / (4 * pi)) * (3 * math.cos(i) + 2) * s2 ** 4,
        (4, 4): 3 * math.sqrt(7 / pi) * c2 ** 6 * s2 ** 2,
        (4, -4): 3 * math.sqrt(7 / pi) * c2 ** 2 * s2 ** 6,
    }
    return table[(l, m)]


LMS = [(2, 2), (2, -2), (2, 1), (2, -1), (3, 3), (3, -3), (3, 2), (3, -2), (4, 4), (4, -4)]


@pytest.mark.parametrize("lm", LMS)
def test_sylm_wigner_matches_closed_forms(oracle_mod, lm):
    for i in np.linspace(0.0, math.pi, 13):
        assert oracle_mod.sylm(lm[0], lm[1], i) == pytest.approx(ylm_closed(lm[0], lm[1], i), abs=1e-14)


def test_sylm_orthonormal(oracle_mod):
    # integral over the sphere of -2Y_lm -2Y*_l'm = delta_ll' (Gauss-Legendre in cos(iota)).
    x, w = np.polynomial.legendre.leggauss(40)
    io = np.arccos(x)
    def integ(l1, l2, m):
        y1 = np.array([oracle_mod.sylm(l1, m, i) for i in io])
        y2 = np.array([oracle_mod.sylm(l2, m, i) for i in io])
        return 2 * math.pi * np.sum(w * y1 * y2)
    for l, m in [(2, 2), (2, -2), (2, 1), (3, 3), (3, 2), (3, -2), (4, 4), (4, -4), (4, 2), (4, 1)]:
        assert integ(l, l, m) == pytest.approx(1.0, abs=1e-12)
    for (l1, l2, m) in [(2, 3, 2), (2, 4, 2), (3, 4, 3), (2, 3, -2), (2, 3, 1)]:
        assert abs(integ(l1, l2, m)) < 1e-12


# -------------------------------------------------------------------------------------------
# Waveform
# -------------------------------------------------------------------------------------------
def test_face_on_22_newtonian_amplitude(oracle_mod):
    """|h+| of the face-on (2,2) SPA signal = sqrt(5/24) pi^(-2/3) Mc^(5/6) f^(-7/6) / D."""
    th = TH.copy(); th[5] = 0.0
    f = np.geomspace(1e-4, 3e-3, 9)
    hp, hc = oracle_mod.polarizations(th, W.MODE_22, f)
    Mc = chirp_mass_s(th)
    D = th[4] * GPC_S
    ref = math.sqrt(5 / 24) * math.pi ** (-2 / 3) * Mc ** (5 / 6) * f ** (-7 / 6) / D
    np.testing.assert_allclose(np.abs(hp), ref, rtol=1e-12)
    np.testing.assert_allclose(hc, -1j * hp, rtol=1e-13, atol=0)


def test_tf_newtonian_limit(oracle_mod):
    """t_c - t_f -> (5/256) Mc^(-5/3) (pi f)^(-8/3) as v -> 0 (Eq. eq_tf at Newtonian order)."""
    th = TH.copy()
    M = th[0] * MSUN_S
    Mc = chirp_mass_s(th)
    for v in (1e-3, 3e-3):
        f = v ** 3 / (math.pi * M)
        _, tf, _ = oracle_mod.mode(th, 2, 2, [f])
        newt = 5.0 / 256.0 * Mc ** (-5 / 3) * (math.pi * f) ** (-8 / 3)
        assert (th[10] - tf[0]) / newt == pytest.approx(1.0, abs=10 * v * v)


@pytest.mark.parametrize("q", [1.0, 2.0, 7.0])
def test_tf_matches_taylort2_to_2p5pn(oracle_mod, q):
    """Non-spinning t_f against the published TaylorT2 time t(v) to 2.5PN (Buonanno et al. 2009):
    t_c - t = 5M/(256 eta v^8) [1 + tau2 v^2 + tau3 v^3 + tau4 v^4 + tau5 v^5 + O(v^6)]."""
    th = TH.copy(); th[1] = q; th[2] = th[3] = 0.0
    M = th[0] * MSUN_S
    eta = q / (1 + q) ** 2
    pi = math.pi
    tau2 = 743 / 252 + 11 * eta / 3
    tau3 = -32 * pi / 5
    tau4 = 3058673 / 508032 + 5429 * eta / 504 + 617 * eta ** 2 / 72
    tau5 = -(7729 / 252 - 13 * eta / 3) * pi
    for v in (0.01, 0.02, 0.04):
        f = v ** 3 / (pi * M)
        _, tf, _ = oracle_mod.mode(th, 2, 2, [f])
        series = 1 + tau2 * v ** 2 + tau3 * v ** 3 + tau4 * v ** 4 + tau5 * v ** 5
        ratio = (th[10] - tf[0]) / (5 * M / (256 * eta * v ** 8))
        assert abs(ratio - series) < 2000 * v ** 6


def _taylorf2_from_energy_and_flux():
    """TaylorF2 coefficients alpha_k(eta) re-derived by energy balance, independently of their
    published form: dt/dv = -(dE/dv)/F with the circular-orbit binding energy E (3PN) and the
    gravitational-wave flux F (3.5PN, with its ln(16 x) tail term) of comparable-mass binaries
    (Blanchet, Living Rev. Relativ. 17, 2 (2014), the non-spinning circular-orbit energy and
    flux). Writing dt/dv = (5M/(32 eta)) v^-9 g(v), g = 1 + sum_k g_k v^k, the stationary-phase
    phase 2 pi f t(v) - 2 phi(v) with phi' = v^3 t'/M is (3/(128 eta v^5)) sum_k alpha_k v^k up
    to terms constant or linear in f, with alpha_k = 40 g_k / ((k-8)(k-5)) for k != 5, 8. The
    v^5 term integrates to a logarithm (alpha_5's ln v coefficient: -(40/3) g_5); at v^6 the
    flux's ln v term gives alpha_6 = -20 g_6c + 10 g_6l plus -20 g_6l ln v, for g_6 = g_6c +
    g_6l ln v. Returns sympy expressions in eta."""
    sp = pytest.importorskip("sympy")
    et, L = sp.symbols("eta L")
    R, pi, gE = sp.Rational, sp.pi, sp.EulerGamma
    N = 8
    # E / mu in powers of v (x = v^2) and F / ((32/5) eta^2 x^5); L stands for ln(16 x)
    Ek = {2: -R(1, 2), 4: -R(1, 2) * (-R(3, 4) - et / 12), 6: -R(1, 2) * (-R(27, 8) + R(19, 8) * et - et ** 2 / 24),
          8: -R(1, 2) * (-R(675, 64) + (R(34445, 576) - R(205, 96) * pi ** 2) * et - R(155, 96) * et ** 2
                         - R(35, 5184) * et ** 3)}
    Fk = {0: 1, 2: -R(1247, 336) - R(35, 12) * et, 3: 4 * pi,
          4: -R(44711, 9072) + R(9271, 504) * et + R(65, 18) * et ** 2,
          5: (-R(8191, 672) - R(583, 24) * et) * pi,
          6: (R(6643739519, 69854400) + R(16, 3) * pi ** 2 - R(1712, 105) * gE - R(856, 105) * L
              + (-R(134543, 7776) + R(41, 48) * pi ** 2) * et - R(94403, 3024) * et ** 2 - R(775, 324) * et ** 3),
          7: (-R(16285, 504) + R(214745, 1728) * et + R(193385, 3024) * et ** 2) * pi}
    F = [sp.sympify(Fk.get(k, 0)) for k in range(N)]
    num = [sp.sympify(0)] * N                     # -(dE/dv) / v
    for k, c in Ek.items():
        num[k - 2] += -k * c
    inv = [sp.sympify(1)] + [sp.sympify(0)] * (N - 1)   # 1/F as a series (F_0 = 1)
    for n in range(1, N):
        inv[n] = sp.expand(-sum(F[j] * inv[n - j] for j in range(1, n + 1)))
    g = [sp.expand(sum(num[j] * inv[n - j] for j in range(n + 1))) for n in range(N)]
    assert g[0] == 1 and g[1] == 0
    out = {k: 40 * g[k] / ((k - 8) * (k - 5)) for k in (2, 3, 4, 7)}
    d6 = sp.diff(g[6], L)                          # L = ln 16 + 2 ln v
    c6 = g[6].subs(L, 0) + d6 * sp.log(16)
    out["6c"] = -20 * c6 + 20 * d6
    out["6l"] = -40 * d6
    out["5l"] = -R(40, 3) * g[5]
    return et, out


@pytest.mark.parametrize("q", [1.0, 3.0, 1e9])
def test_taylorf2_coefficients_from_energy_balance(oracle_mod, q):
    """The oracle's non-spinning PN phase coefficients, alpha_2 ... alpha_7 with their eta
    dependence (3PN and 3.5PN included) and the ln v terms of alpha_5 and alpha_6, against the
    energy-balance derivation above. The oracle's coefficients are read off its Psi_PN(v) by a
    least-squares fit on the basis v^0..v^7, v^5 ln v, v^6 ln v (Psi_PN has exactly that form).
    Only alpha_5's constant, which joins phi_c, is convention and not compared."""
    et, ref = _taylorf2_from_energy_and_flux()
    eta = q / (1 + q) ** 2
    th = TH.copy()
    th[1] = q
    th[2] = th[3] = 0.0
    vs = np.linspace(0.03, 0.3, 80)
    y = np.array([oracle_mod.psi_pn(th, v) for v in vs]) * 128 * eta * vs ** 5 / 3
    B = np.column_stack([vs ** k for k in range(8)] + [vs ** 5 * np.log(vs), vs ** 6 * np.log(vs)])
    sc = np.abs(B).max(axis=0)
    c = np.linalg.lstsq(B / sc, y, rcond=None)[0] / sc
    got = {2: c[2], 3: c[3], 4: c[4], 7: c[7], "6c": c[6], "6l": c[9], "5l": c[8]}
    assert abs(c[0] - 1.0) < 1e-12 and abs(c[1]) < 1e-9
    for k, expr in ref.items():
        want = float(expr.subs(et, eta).evalf(30))
        assert got[k] == pytest.approx(want, rel=1e-7), (k, got[k], want)


def test_spin_orbit_coefficient_in_the_test_mass_limit(oracle_mod):
    """The 1.5PN spin-orbit term of alpha_3, -16 pi + 4 beta with beta -> (113/12) chi_1 as
    eta -> 0, against the same energy-balance derivation for a test mass on a prograde circular
    equatorial orbit of a Kerr black hole of spin chi_1: the exact Bardeen-Press-Teukolsky
    energy E/mu = (1 - 2 w^2 + a w^3) / sqrt(1 - 3 w^2 + 2 a w^3) - 1 (w^2 = M/r), written in
    u = (M Omega)^(1/3) through w^3 = u^3 / (1 - a u^3), and the test-mass flux to 1.5PN,
    1 - (1247/336) u^2 + (4 pi - (11/4) a) u^3 (Tagoshi, Shibata, Tanaka & Sasaki 1996)."""
    sp = pytest.importorskip("sympy")
    u, a = sp.symbols("u a")
    w = u * (1 - a * u ** 3) ** sp.Rational(-1, 3)
    E = (1 - 2 * w ** 2 + a * w ** 3) / sp.sqrt(1 - 3 * w ** 2 + 2 * a * w ** 3) - 1
    Es = sp.expand(sp.series(E, u, 0, 6).removeO())
    f = 1 - sp.Rational(1247, 336) * u ** 2 + (4 * sp.pi - sp.Rational(11, 4) * a) * u ** 3
    g = sp.expand(sp.series(-sp.diff(Es, u) / (u * f), u, 0, 4).removeO())
    alpha3 = sp.expand(40 * g.coeff(u, 3) / ((3 - 8) * (3 - 5)))
    chi1 = 0.6
    th = TH.copy()
    th[1] = 1e9
    th[2], th[3] = chi1, 0.0
    eta = th[1] / (1 + th[1]) ** 2
    vs = np.linspace(0.03, 0.3, 80)
    y = np.array([oracle_mod.psi_pn(th, v) for v in vs]) * 128 * eta * vs ** 5 / 3
    B = np.column_stack([vs ** k for k in range(8)] + [vs ** 5 * np.log(vs), vs ** 6 * np.log(vs)])
    sc = np.abs(B).max(axis=0)
    c = np.linalg.lstsq(B / sc, y, rcond=None)[0] / sc
    want = float(alpha3.subs(a, chi1))
    assert c[3] == pytest.approx(want, rel=1e-7), (c[3], want)


def _spin_energy_balance(q, chi1, chi2):
    """alpha_3 and alpha_4 of the PN phase with their aligned-spin terms, by energy balance
    through 2PN (the series algebra of _taylorf2_from_energy_and_flux, numerically). G = c = M = 1,
    m_1 = q/(1+q), S_i = m_i^2 chi_i along the orbital angular momentum, S = S_1 + S_2,
    Sigma = S_2/m_2 - S_1/m_1, delta = m_1 - m_2. Circular-orbit energy and flux with their spin
    parts (Kidder, Phys. Rev. D 52, 821 (1995); Blanchet, Living Rev. Relativ. 17, 2 (2014)):
      E / (-mu x/2) = 1 + (-3/4 - eta/12) x + (14/3 S + 2 delta Sigma) x^(3/2)
                      + (-27/8 + 19/8 eta - eta^2/24 + (S_1.S_2 - 3 S_1.L S_2.L) / eta) x^2,
      F / F_N = 1 + (-1247/336 - 35/12 eta) x + (4 pi - 4 S - 5/4 delta Sigma) x^(3/2)
                + (-44711/9072 + 9271/504 eta + 65/18 eta^2 + (-103 S_1.S_2 + 289 S_1.L S_2.L) / (48 eta)) x^2.
    For aligned spins S_1.S_2 = S_1.L S_2.L = eta^2 chi_1 chi_2."""
    m1, m2 = q / (1 + q), 1 / (1 + q)
    eta, delta = m1 * m2, m1 - m2
    S = m1 ** 2 * chi1 + m2 ** 2 * chi2
    Sig = m2 * chi2 - m1 * chi1
    ss = eta * chi1 * chi2                      # S_1 S_2 / eta for aligned spins
    E = {2: -0.5, 4: -0.5 * (-0.75 - eta / 12), 5: -0.5 * (14 / 3 * S + 2 * delta * Sig),
         6: -0.5 * (-27 / 8 + 19 / 8 * eta - eta ** 2 / 24 + (1 - 3) * ss)}
    F = {0: 1.0, 2: -1247 / 336 - 35 / 12 * eta, 3: 4 * math.pi - 4 * S - 1.25 * delta * Sig,
         4: -44711 / 9072 + 9271 / 504 * eta + 65 / 18 * eta ** 2 + (-103 + 289) / 48 * ss}
    N = 5
    num = [0.0] * N                             # -(dE/dv) / v
    for k, c in E.items():
        num[k - 2] += -k * c
    Fs = [F.get(k, 0.0) for k in range(N)]
    inv = [1.0] + [0.0] * (N - 1)               # 1/F as a series
    for n in range(1, N):
        inv[n] = -sum(Fs[j] * inv[n - j] for j in range(1, n + 1))
    g = [sum(num[j] * inv[n - j] for j in range(n + 1)) for n in range(N)]
    return 40 * g[3] / ((3 - 8) * (3 - 5)), 40 * g[4] / ((4 - 8) * (4 - 5))


@pytest.mark.parametrize("q,chi1,chi2", [(1.0, 0.5, -0.3), (3.0, 0.9, 0.2), (8.0, -0.7, 0.6), (1.5, 0.95, 0.95)])
def test_spin_terms_from_energy_balance(oracle_mod, q, chi1, chi2):
    """The oracle's alpha_3 (1.5PN spin-orbit, with its eta dependence) and alpha_4 (2PN
    spin-spin) for comparable masses and aligned spins, against energy balance with the spin parts
    of the energy and flux (_spin_energy_balance). The oracle keeps exactly these spin orders (no
    self-spin terms, no higher spin-orbit terms), so only alpha_3 and alpha_4 are compared; their
    non-spinning parts are pinned on their own above."""
    eta = q / (1 + q) ** 2
    th = TH.copy()
    th[1], th[2], th[3] = q, chi1, chi2
    vs = np.linspace(0.03, 0.3, 80)
    y = np.array([oracle_mod.psi_pn(th, v) for v in vs]) * 128 * eta * vs ** 5 / 3
    B = np.column_stack([vs ** k for k in range(8)] + [vs ** 5 * np.log(vs), vs ** 6 * np.log(vs)])
    sc = np.abs(B).max(axis=0)
    c = np.linalg.lstsq(B / sc, y, rcond=None)[0] / sc
    a3, a4 = _spin_energy_balance(q, chi1, chi2)
    assert c[3] == pytest.approx(a3, rel=1e-7, abs=1e-6), (c[3], a3)
    assert c[4] == pytest.approx(a4, rel=1e-7, abs=1e-6), (c[4], a4)


def _biww_polarizations(iota, q, psi):
    """(H+ - i Hx) of a circular binary at orders x^0, x^(1/2), x^1, from the 1PN polarisations of
    Blanchet, Iyer, Will & Wiseman, Class. Quantum Grav. 13, 575 (1996) (as restated in Blanchet,
    Living Rev. Relativ. 17, 2 (2014)); h+,x = (2 G mu x / (c^2 R)) sum_p x^(p/2) H^(p/2)+,x, psi the
    orbital phase from the ascending node, Delta = (m1 - m2)/M. The zero-frequency memory term of
    H+^(0) is left out (it belongs to the m = 0 modes)."""
    c, s = math.cos(iota), math.sin(iota)
    nu = q / (1 + q) ** 2
    D = (q - 1) / (q + 1)
    hp0 = -(1 + c * c) * np.cos(2 * psi)
    hx0 = -2 * c * np.sin(2 * psi)
    hp1 = -s * D * ((5 / 8 + c * c / 8) * np.cos(psi) - (9 / 8 + 9 * c * c / 8) * np.cos(3 * psi))
    hx1 = s * c * D * (-0.75 * np.sin(psi) + 2.25 * np.sin(3 * psi))
    hp2 = ((19 / 6 + 1.5 * c * c - c ** 4 / 3 + nu * (-19 / 6 + 11 / 6 * c * c + c ** 4)) * np.cos(2 * psi)
           - 4 / 3 * s * s * (1 + c * c) * (1 - 3 * nu) * np.cos(4 * psi))
    hx2 = (c * (17 / 3 - 4 / 3 * c * c + nu * (-13 / 3 + 4 * c * c)) * np.sin(2 * psi)
           - 8 / 3 * c * s * s * (1 - 3 * nu) * np.sin(4 * psi))
    return hp0 - 1j * hx0, hp1 - 1j * hx1, hp2 - 1j * hx2


@pytest.mark.parametrize("q", [1.5, 3.0, 8.0])
@pytest.mark.parametrize("iota", [0.3, 1.1, 2.2])
def test_higher_mode_phases_reproduce_the_1pn_polarisations(oracle_mod, q, iota):
    """The complex mode factors of the oracle (the +-i of H21 and H33, their relative sign, the
    signs of H32 and H44), summed as h+ - i hx = sum_lm h_lm -2Y_lm(iota, 0) with
    h_lm ~ sqrt(16 pi/5) H_lm x^(p/2) e^(-i m psi) and h_(l,-m) = (-1)^l conj(h_lm), against the 1PN
    polarisations of a circular binary, order by order in x^(1/2). The modes the oracle does not
    carry but the polarisations contain at these orders are added from Blanchet's review: H31 =
    i Delta/(12 sqrt(14)) at x^(1/2); H42 = sqrt(5)/63 (1 - 3 nu) and the 1PN term of H22,
    -107/42 + 55 nu/42, at x^1. The polarisations measure psi from the ascending node; the
    oracle's phase origin is 3 pi/2 behind it, a convention fixed by the x^0 order up to pi (a
    shift by pi exchanges the bodies and flips the odd orders, which must not match then)."""
    nu = q / (1 + q) ** 2
    D = (q - 1) / (q + 1)
    k = math.sqrt(16 * math.pi / 5)
    orders = {0: [(2, 2, oracle_mod.hhat(q, 2, 2, 1.0))],
              1: [(2, 1, oracle_mod.hhat(q, 2, 1, 1.0)), (3, 3, oracle_mod.hhat(q, 3, 3, 1.0)),
                  (3, 1, 1j * D / (12 * math.sqrt(14)))],
              2: [(3, 2, oracle_mod.hhat(q, 3, 2, 1.0)), (4, 4, oracle_mod.hhat(q, 4, 4, 1.0)),
                  (4, 2, math.sqrt(5) / 63 * (1 - 3 * nu)), (2, 2, -107 / 42 + 55 * nu / 42)]}

    def modes_sum(p, psi):
        h = np.zeros(psi.shape, dtype=complex)
        for l, m, H in orders[p]:
            h += k * (H * np.exp(-1j * m * psi) * oracle_mod.sylm(l, m, iota)
                      + (-1) ** l * np.conj(H) * np.exp(1j * m * psi) * oracle_mod.sylm(l, -m, iota))
        return h

    psi = np.linspace(0.0, 2 * math.pi, 64, endpoint=False)
    ref = _biww_polarizations(iota, q, psi)
    for p in range(3):
        assert np.abs(modes_sum(p, psi + 1.5 * math.pi) - ref[p]).max() < 1e-13, p
    # the other origin allowed by the x^0 order flips the x^(1/2) order (exchanged bodies)
    assert np.abs(modes_sum(1, psi + 0.5 * math.pi) - ref[1]).max() > 0.1 * np.abs(ref[1]).max()


def _newtonian_multipole_flux(m1, m2, r, n=64):
    """Energy flux of a Newtonian circular binary (masses m1, m2, separation r; G = c = M = 1),
    split by multipole and by harmonic of the orbital frequency, from the multipole expansion of
    the flux (Thorne, Rev. Mod. Phys. 52, 299 (1980)):
      F = sum_l (l+1)(l+2) / ((l-1) l l! (2l+1)!!) <(d^(l+1) I_L)^2>
          + 4 l (l+2) / ((l-1) (l+1)! (2l+1)!!) <(d^(l+1) J_L)^2>,
    with the symmetric trace-free mass moments I_L = sum_A m_A x_A^<L> and current moments
    J_L = sum_A m_A [x_A^(L-1) (x_A x v_A)]^STF. The moments are sampled over one orbit; their time
    derivatives and averages are taken harmonic by harmonic from a discrete Fourier transform
    (the moments are trigonometric polynomials). Returns {(kind, l): {harmonic k: flux}}."""
    M = m1 + m2
    w = math.sqrt(M / r ** 3)
    t = np.arange(n) * 2 * math.pi / (w * n)
    d = np.eye(3)
    bodies = []
    for mA, s in ((m1, m2 / M), (m2, -m1 / M)):
        x = np.stack([s * r * np.cos(w * t), s * r * np.sin(w * t), 0 * t], axis=1)
        v = np.stack([-s * r * w * np.sin(w * t), s * r * w * np.cos(w * t), 0 * t], axis=1)
        bodies.append((mA, x, v, (x * x).sum(1), np.cross(x, v)))
    I2 = sum(mA * (np.einsum("ti,tj->tij", x, x) - r2[:, None, None] * d / 3) for mA, x, v, r2, Lv in bodies)
    I3 = sum(mA * (np.einsum("ti,tj,tk->tijk", x, x, x) - r2[:, None, None, None] / 5 * (
        np.einsum("ti,jk->tijk", x, d) + np.einsum("tj,ik->tijk", x, d) + np.einsum("tk,ij->tijk", x, d)))
        for mA, x, v, r2, Lv in bodies)
    dd = np.einsum("ij,kl->ijkl", d, d) + np.einsum("ik,jl->ijkl", d, d) + np.einsum("il,jk->ijkl", d, d)
    I4 = sum(mA * (np.einsum("ti,tj,tk,tl->tijkl", x, x, x, x)
                   - r2[:, None, None, None, None] / 7 * sum(np.einsum(e, d, x, x) for e in (
                       "ij,tk,tl->tijkl", "ik,tj,tl->tijkl", "il,tj,tk->tijkl", "jk,ti,tl->tijkl",
                       "jl,ti,tk->tijkl", "kl,ti,tj->tijkl"))
                   + (r2 ** 2)[:, None, None, None, None] / 35 * dd) for mA, x, v, r2, Lv in bodies)
    # x . (x x v) = 0, so only the traces named here survive
    J2 = sum(mA * 0.5 * (np.einsum("ti,tj->tij", x, Lv) + np.einsum("ti,tj->tij", Lv, x)) for mA, x, v, r2, Lv in bodies)
    J3 = sum(mA * ((np.einsum("ti,tj,tk->tijk", x, x, Lv) + np.einsum("ti,tj,tk->tijk", x, Lv, x)
                    + np.einsum("ti,tj,tk->tijk", Lv, x, x)) / 3
                   - r2[:, None, None, None] / 15 * (np.einsum("ij,tk->tijk", d, Lv) + np.einsum("ik,tj->tijk", d, Lv)
                                                    + np.einsum("jk,ti->tijk", d, Lv)))
             for mA, x, v, r2, Lv in bodies)

    def split(T, l, kind):
        if kind == "I":
            coef = (l + 1) * (l + 2) / ((l - 1) * l * math.factorial(l) * _dfact(2 * l + 1))
        else:
            coef = 4 * l * (l + 2) / ((l - 1) * math.factorial(l + 1) * _dfact(2 * l + 1))
        c = np.fft.fft(T, axis=0) / n
        return {k: coef * 2 * np.sum(np.abs(c[k]) ** 2) * (k * w) ** (2 * (l + 1)) for k in range(1, n // 2)}

    return {("I", 2): split(I2, 2, "I"), ("I", 3): split(I3, 3, "I"), ("I", 4): split(I4, 4, "I"),
            ("J", 2): split(J2, 2, "J"), ("J", 3): split(J3, 3, "J")}, w


def _dfact(n):
    return math.prod(range(n, 0, -2))


@pytest.mark.parametrize("q", [1.5, 3.0, 8.0])
def test_higher_mode_amplitudes_match_multipole_flux(oracle_mod, q):
    """|H_lm| of the four higher modes (mass octupole 33, current quadrupole 21, current octupole
    32, mass hexadecapole 44) against the flux each multipole of a Newtonian binary radiates at
    harmonic m, relative to the (2,2) flux (_newtonian_multipole_flux). The flux of mode (l,m) and
    (l,-m) together is (R^2/8 pi) (m omega)^2 |h_lm|^2; the oracle's stationary-phase amplitudes
    at the same orbital frequency F give |h_lm / h_22| = |h~_lm(mF) / h~_22(2F)| sqrt(m/2). The
    (2,2) flux itself is pinned to the quadrupole formula here too."""
    m1, m2 = q / (1 + q), 1 / (1 + q)
    r = 1e4                                   # M/r = v^2 = 1e-4
    fl, w = _newtonian_multipole_flux(m1, m2, r)
    F22 = fl[("I", 2)][2]
    assert F22 == pytest.approx(32 / 5 * (m1 * m2) ** 2 * w ** (10 / 3), rel=1e-12)
    th = TH.copy()
    th[1] = q
    th[2] = th[3] = 0.0
    F = (1 / r) ** 1.5 / (2 * math.pi * th[0] * MSUN_S)   # orbital frequency: M omega = v^3
    h22 = abs(oracle_mod.mode(th, 2, 2, [2 * F])[0][0])
    for (l, m), key in (((3, 3), ("I", 3)), ((2, 1), ("J", 2)), ((4, 4), ("I", 4)), ((3, 2), ("J", 3))):
        hlm = abs(oracle_mod.mode(th, l, m, [m * F])[0][0])
        ratio_oracle = (m / 2) ** 2 * (hlm / h22 * math.sqrt(m / 2)) ** 2
        assert ratio_oracle == pytest.approx(fl[key][m] / F22, rel=1e-9), ((l, m), ratio_oracle, fl[key][m] / F22)


@pytest.mark.parametrize("lm", list(W.MODES))
def test_tf_is_phase_derivative(oracle_mod, lm):
    """t_f = (1/2 pi) dPsi/df (Eq. eq_tf with Phi = -Psi) against a central difference."""
    f = np.geomspace(2e-4, 3e-3, 7)
    _, tf, _ = oracle_mod.mode(TH, lm[0], lm[1], f)
    h = f * 1e-6
    _, _, pp = oracle_mod.mode(TH, lm[0], lm[1], f + h)
    _, _, pm = oracle_mod.mode(TH, lm[0], lm[1], f - h)
    fd = (pp - pm) / (2 * h) / (2 * math.pi)
    np.testing.assert_allclose(tf, fd, rtol=1e-7)


@pytest.mark.parametrize("lm", [(2, 1), (3, 3), (3, 2), (4, 4)])
def test_mode_phase_scaling_identity(oracle_mod, lm):
    """Psi_lm(f) = (m/2) Psi_22(2f/m) + (m-2) pi/8 and t_f^lm(f) = t_f^22(2f/m): the (l,m)
    harmonic at frequency f is the orbit at orbital frequency f/m."""
    l, m = lm
    f = np.geomspace(2e-4, 2e-3, 6)
    _, tf, ps = oracle_mod.mode(TH, l, m, f)
    _, tf22, ps22 = oracle_mod.mode(TH, 2, 2, 2 * f / m)
    np.testing.assert_allclose(ps - m / 2 * ps22, (m - 2) * math.pi / 8, atol=1e-9 * np.abs(ps).max())
    np.testing.assert_allclose(tf, tf22, rtol=1e-13)


def test_odd_m_modes_vanish_for_equal_masses(oracle_mod):
    th = TH.copy(); th[1] = 1.0
    f = np.geomspace(1e-4, 3e-3, 5)
    for l, m in ((2, 1), (3, 3)):
        h, _, _ = oracle_mod.mode(th, l, m, f)
        assert np.all(h == 0)
    h, _, _ = oracle_mod.mode(th, 2, 2, f)
    assert np.all(np.abs(h) > 0)


def test_face_on_only_m2_and_circular(oracle_mod):
    """iota = 0: only m = 2 harmonics reach the observer and h_x = -i h_+ (circular)."""
    th = TH.copy(); th[5] = 0.0
    f = np.geomspace(1e-4, 3e-3, 5)
    for bit, (l, m) in enumerate(W.MODES):
        hp, hc = oracle_mod.polarizations(th, 1 << bit, f)
        if m == 2:
            assert np.all(np.abs(hp) > 0)
            np.testing.assert_allclose(hc, -1j * hp, rtol=1e-14)
        else:
            assert np.all(hp == 0) and np.all(hc == 0)


def test_22_inclination_dependence(oracle_mod):
    """(2,2) only: h+ = sqrt(5/16pi) (1+cos^2 i)/2 H22, hx = -i sqrt(5/16pi) cos i H22."""
    f = np.geomspace(1e-4, 3e-3, 5)
    for inc in (0.3, 1.1, 2.0, 2.9):
        th = TH.copy(); th[5] = inc
        hp, hc = oracle_mod.polarizations(th, W.MODE_22, f)
        H, _, _ = oracle_mod.mode(th, 2, 2, f)
        k = math.sqrt(5 / (16 * math.pi))
        np.testing.assert_allclose(hp, k * (1 + math.cos(inc) ** 2) / 2 * H, rtol=1e-13)
        np.testing.assert_allclose(hc, -1j * k * math.cos(inc) * H, rtol=1e-13)


def test_mode_symmetry_explicit_plus_minus_m(oracle_mod):
    """h_{l,-m} = (-1)^l h*_lm: summing both signs of m explicitly,
    h+ + i hx = sum_lm H~_lm Y_lm and h+ - i hx = sum_lm (-1)^l H~_lm Y_{l,-m} for f > 0."""
    f = np.geomspace(1e-4, 3e-3, 5)
    for inc in (0.4, 1.7, 2.8):
        th = TH.copy(); th[5] = inc
        hp, hc = oracle_mod.polarizations(th, W.MODE_ALL, f)
        sp = np.zeros_like(hp); sm = np.zeros_like(hp)
        for l, m in W.MODES:
            H, _, _ = oracle_mod.mode(th, l, m, f)
            sp += H * ylm_closed(l, m, inc)
            sm += (-1) ** l * H * ylm_closed(l, -m, inc)
        np.testing.assert_allclose(hp + 1j * hc, sp, rtol=1e-12, atol=1e-12 * np.abs(sp).max())
        np.testing.assert_allclose(hp - 1j * hc, sm, rtol=1e-12, atol=1e-12 * np.abs(sp).max())


def test_planck_taper_edges(oracle_mod):
    M = TH[0] * MSUN_S
    Fisco = 6 ** -1.5 / (2 * math.pi * M)
    for m in (1, 2, 3, 4):
        assert oracle_mod.taper(TH, 0.9 * Fisco * m * (1 - 1e-12), m) == 1.0
        assert oracle_mod.taper(TH, Fisco * m, m) == 0.0
        assert oracle_mod.taper(TH, 0.95 * Fisco * m, m) == pytest.approx(0.5, abs=1e-12)
        fs = np.linspace(0.9, 1.0, 50) * Fisco * m
        w = np.array([oracle_mod.taper(TH, x, m) for x in fs])
        assert np.all(np.diff(w) <= 0)


def _taper_flatness(w, F1, F2):
    """Defining properties of the McKechan-Robinson-Sathyaprakash window as a falling edge on
    [F1, F2]; returns a list of the properties that fail (empty when all hold).
    - C-infinity flat at both ends: the finite-difference derivatives of orders 1..4, scaled by
      (F2 - F1)^k, vanish (below 1e-6) at 2 % of the width from either end, and shrink towards it;
    - faster than any power at the end: the log slope d ln w / d ln(F2 - F) exceeds 0.5 a/delta
      (> 50 at delta = a/100; a power law delta^p has slope p);
    - antisymmetric about the midpoint: w(F1 + x) + w(F2 - x) = 1."""
    a = F2 - F1
    bad = []

    def deriv(F, k, h):
        c = [1.0]
        for _ in range(k):               # binomial central-difference weights of order k
            c = [x - y for x, y in zip(c + [0.0], [0.0] + c)]
        pts = [F + (j - k / 2.0) * h for j in range(k + 1)]
        return sum(cj * w(p) for cj, p in zip(c, pts)) / h ** k

    for k in (1, 2, 3, 4):
        for end, sgn in ((F1, 1.0), (F2, -1.0)):
            vals = [abs(deriv(end + sgn * d * a, k, 0.002 * a)) * a ** k for d in (0.04, 0.02)]
            if not (vals[1] <= 1e-6 and vals[1] <= vals[0]):
                bad.append("derivative %d at %s: %s" % (k, "F1" if sgn > 0 else "F2", vals))
    for d in (1e-2, 3e-3):
        lo, hi = F2 - d * a * 1.01, F2 - d * a / 1.01
        wl, wh = w(lo), w(hi)
        slope = (math.log(wl) - math.log(wh)) / (math.log(d * 1.01) - math.log(d / 1.01)) if wl > 0 and wh > 0 else 0.0
        if not slope > 0.5 / d:
            bad.append("log slope %.3g at delta %g" % (slope, d))
    for x in np.linspace(0.05, 0.95, 19):
        if abs(w(F1 + x * a) + w(F2 - x * a) - 1.0) > 1e-14:
            bad.append("antisymmetry at %g" % x)
    return bad


def test_planck_taper_is_cinf_flat(oracle_mod):
    """The window's interior shape (Sec. 2.3 falling edge, read as the McKechan et al. 2010 Planck
    window): flat to every order at both ends, antisymmetric about the midpoint. A raised-cosine
    edge and a C^2 smoothstep edge, written here, fail the same checks."""
    for th0 in (TH, np.r_[3e5, TH[1:]]):
        M = th0[0] * MSUN_S
        Fisco = 6 ** -1.5 / (2 * math.pi * M)
        F1, F2 = 0.9 * Fisco, Fisco
        for m in (1, 2, 3, 4):
            assert _taper_flatness(lambda Fo: oracle_mod.taper(th0, Fo * m, m), F1, F2) == []

    def cosine(Fo, F1=0.9, F2=1.0):
        x = min(max((Fo - F1) / (F2 - F1), 0.0), 1.0)
        return 0.5 * (1.0 + math.cos(math.pi * x))

    def smoothstep(Fo, F1=0.9, F2=1.0):
        x = min(max((Fo - F1) / (F2 - F1), 0.0), 1.0)
        return 1.0 - x ** 3 * (10.0 - 15.0 * x + 6.0 * x * x)

    assert _taper_flatness(cosine, 0.9, 1.0) != []
    assert _taper_flatness(smoothstep, 0.9, 1.0) != []


# -------------------------------------------------------------------------------------------
# Geometry: sky basis and orbits
# -------------------------------------------------------------------------------------------
def test_sky_basis_orthonormal(oracle_mod):
    for lam, bet, psi in ((1.375, -1.2108, 2.659), (4.0, 0.3, 0.1), (0.2, 1.4, 1.9)):
        th = TH.copy(); th[7], th[8], th[9] = lam, bet, psi
        k, ep, ec = oracle_mod.sky_basis(th)
        src = np.array([math.cos(bet) * math.cos(lam), math.cos(bet) * math.sin(lam), math.sin(bet)])
        np.testing.assert_allclose(k, -src, atol=1e-15)
        for e in (ep, ec):
            np.testing.assert_allclose(e, e.T, atol=1e-15)
            assert abs(np.trace(e)) < 1e-15
            np.testing.assert_allclose(e @ k, 0, atol=1e-15)
        assert np.sum(ep * ep) == pytest.approx(2.0, abs=1e-14)
        assert np.sum(ec * ec) == pytest.approx(2.0, abs=1e-14)
        assert abs(np.sum(ep * ec)) < 1e-14


@pytest.mark.parametrize("det", [W.LISA, W.TAIJI])
def test_heliocentric_orbit_geometry(oracle_mod, det):
    AU_S = 499.00478383615643
    L = det["arm_m"] / C_SI
    for t in (0.0, 1e6, 1.3e7, -4e8):
        x = oracle_mod.orbit(det, t)
        arms = [np.linalg.norm(x[i] - x[j]) for i, j in ((0, 1), (1, 2), (2, 0))]
        np.testing.assert_allclose(arms, L, rtol=1e-2)
        alpha = det["alpha0"] + 2 * math.pi * t / 31557600.0
        c = x.mean(axis=0)
        np.testing.assert_allclose(c, AU_S * np.array([math.cos(alpha), math.sin(alpha), 0.0]), atol=0.02 * L)
        nrm = np.cross(x[1] - x[0], x[2] - x[0]); nrm /= np.linalg.norm(nrm)
        assert abs(nrm[2]) == pytest.approx(0.5, abs=2e-2)       # plane tilted 60 deg to the ecliptic
        x1 = oracle_mod.orbit(det, t + 31557600.0)
        np.testing.assert_allclose(x1, x, atol=1e-9 * AU_S)


def test_geocentric_orbit_geometry(oracle_mod):
    det = W.TIANQIN
    AU_S = 499.00478383615643
    L = det["arm_m"] / C_SI
    lon, lat = det["geo_lon"], det["geo_lat"]
    nhat = np.array([math.cos(lat) * math.cos(lon), math.cos(lat) * math.sin(lon), math.sin(lat)])
    for t in (0.0, 1e5, 3e6):
        x = oracle_mod.orbit(det, t)
        arms = [np.linalg.norm(x[i] - x[j]) for i, j in ((0, 1), (1, 2), (2, 0))]
        np.testing.assert_allclose(arms, L, rtol=1e-12)
        alpha = det["alpha0"] + 2 * math.pi * t / 31557600.0
        np.testing.assert_allclose(x.mean(axis=0), AU_S * np.array([math.cos(alpha), math.sin(alpha), 0.0]),
                                   atol=1e-11 * AU_S)
        nrm = np.cross(x[1] - x[0], x[2] - x[0]); nrm /= np.linalg.norm(nrm)
        np.testing.assert_allclose(nrm, nhat, atol=1e-12)
        x1 = oracle_mod.orbit(det, t + det["geo_period_s"])
        np.testing.assert_allclose(x1 - x1.mean(axis=0), x - x.mean(axis=0), atol=1e-9)


# -------------------------------------------------------------------------------------------
# Response
# -------------------------------------------------------------------------------------------
@pytest.mark.parametrize("lm", [(2, 2), (3, 3)])
@pytest.mark.parametrize("rs", [(1, 2), (2, 1), (1, 3), (3, 2)])
def test_link_sinc_form_equals_time_shift_form(oracle_mod, lm, rs):
    """Eq. eq_fd_resp is the Fourier transform of Eq. eq_td_resp under h(t - t0) -> e^{-2 pi i f t0}:
    y~_rs = [e^{-2 pi i f (L + k.x_s)} - e^{-2 pi i f k.x_r}] / (2 (1 - k.n_rs)) n_rs.h~.n_rs."""
    det = W.LISA
    L = det["arm_m"] / C_SI
    bit = W.MODES.index(lm)
    f = np.geomspace(1e-4, 4e-2, 7)
    th = TH.copy(); th[0] = 2e5
    y = oracle_mod.link(det, th, lm[0], lm[1], f, rs[0], rs[1])
    k, ep, ec = oracle_mod.sky_basis(th)
    hp, hc = oracle_mod.polarizations(th, 1 << bit, f)
    _, tf, _ = oracle_mod.mode(th, lm[0], lm[1], f)
    for i in range(f.size):
        x = oracle_mod.orbit(det, tf[i])
        xr, xs = x[rs[0] - 1], x[rs[1] - 1]
        n = (xr - xs) / np.linalg.norm(xr - xs)
        nhn = hp[i] * (n @ ep @ n) + hc[i] * (n @ ec @ n)
        ref = (np.exp(-2j * math.pi * f[i] * (L + k @ xs)) - np.exp(-2j * math.pi * f[i] * (k @ xr))) \
            / (2 * (1 - k @ n)) * nhn
        assert abs(y[i] - ref) <= 1e-11 * abs(ref)


def test_fd_link_response_against_time_domain_dft(oracle_mod):
    """R6, a sanity check of the SPA response, not a parity pin: the single-link response of
    Eq. eq_td_resp, evaluated sample by sample in the time domain with the moving orbit, then
    Fourier transformed, agrees with the frequency-domain form Eq. eq_fd_resp (geometry at t_f,
    Eq. eq_tf) to the accuracy of the stationary-phase treatment of the orbit.

    The time-domain (2,2) polarisations are the inverse DFT of the oracle's band-limited
    frequency-domain ones (10 s sampling, 2^16 samples, 3.5e-4 Hz to the taper end, t_c inside the
    window). Delayed samples h(t - L - k.x_s(t)) and h(t - k.x_r(t)) come from cubic splines of the
    sampled signal; the orbit comes from the oracle every 100 s, splined."""
    from scipy.interpolate import CubicSpline
    det = W.LISA
    L = det["arm_m"] / C_SI
    dt, N = 10.0, 2 ** 16
    Tw = N * dt
    th = np.array([1e6, 2.0, 0.3, 0.1, 10.0, 0.6, 0.7, 1.2, 0.4, 0.9, 6.0e5])
    fk = np.arange(N // 2 + 1) / Tw
    flo, fend = 3.5e-4, 2.0 * 6 ** -1.5 / (2 * math.pi * th[0] * MSUN_S)
    band = (fk >= flo) & (fk < fend)
    hp = np.zeros(fk.size, complex)
    hc = np.zeros(fk.size, complex)
    hp[band], hc[band] = oracle_mod.polarizations(th, W.MODE_22, fk[band])
    # smooth turn-on over [flo, 1.5 flo] so the time-domain signal starts without ringing
    ramp = np.clip((fk - flo) / (0.5 * flo), 0.0, 1.0)
    win = np.where(band, np.sin(0.5 * math.pi * ramp) ** 2, 0.0)
    hp *= win
    hc *= win
    t = np.arange(N) * dt
    sp = CubicSpline(t, np.fft.irfft(hp, n=N) / dt)
    sc = CubicSpline(t, np.fft.irfft(hc, n=N) / dt)
    tc = np.arange(-100.0, Tw + 200.0, 100.0)
    xs_all = np.array([oracle_mod.orbit(det, ti) for ti in tc])          # [time][spacecraft][xyz]
    xfun = CubicSpline(tc, xs_all, axis=0)
    x = xfun(t)
    k, ep, ec = oracle_mod.sky_basis(th)
    for (r, s_) in ((1, 2), (3, 1)):
        xr, xs = x[:, r - 1], x[:, s_ - 1]
        n = (xr - xs) / np.linalg.norm(xr - xs, axis=1)[:, None]
        fp = np.einsum("ti,ij,tj->t", n, ep, n)
        fc = np.einsum("ti,ij,tj->t", n, ec, n)
        t1 = t - L - xs @ k
        t2 = t - xr @ k
        y = (fp * (sp(t1) - sp(t2)) + fc * (sc(t1) - sc(t2))) / (2.0 * (1.0 - n @ k))
        ytd = np.fft.rfft(y) * dt
        sel = (fk > 2.0 * flo) & (fk < 0.6 * fend)
        yfd = oracle_mod.link(det, th, 2, 2, fk[sel], r, s_)
        err = np.abs(ytd[sel] - yfd)
        ref = np.abs(yfd)
        # measured: 2.7e-4 of the maximum and 2.4e-4 median; with the geometry frozen at t_c
        # instead of t_f the same comparison gives 4.4e-2 and 6.5e-3
        assert np.max(err) < 2e-3 * ref.max()
        assert np.median(err / ref) < 1e-3


def test_long_wavelength_limit(oracle_mod):
    """fL -> 0: X_1.5 -> 2 (2 pi f L)^2 [n13.h.n13 - n12.h.n12] e^{-2 pi i f k.xbar} and
    X_2.0 -> 4 i (2 pi f L) X_1.5, with relative corrections O(f L)."""
    det15 = dict(W.LISA, tdi_gen=15)
    L = det15["arm_m"] / C_SI
    th = TH.copy()
    f = np.array([1e-6, 3e-6])
    x15 = oracle_mod.response_xyz(det15, th, W.MODE_22, f)[0]
    x20 = oracle_mod.response_xyz(W.LISA, th, W.MODE_22, f)[0]
    k, ep, ec = oracle_mod.sky_basis(th)
    hp, hc = oracle_mod.polarizations(th, W.MODE_22, f)
    _, tf, _ = oracle_mod.mode(th, 2, 2, f)
    for i in range(f.size):
        x = oracle_mod.orbit(det15, tf[i])
        def nhn(a, b):
            n = (x[a] - x[b]) / np.linalg.norm(x[a] - x[b])
            return hp[i] * (n @ ep @ n) + hc[i] * (n @ ec @ n)
        xbar = x.mean(axis=0)
        ref = 2 * (2 * math.pi * f[i] * L) ** 2 * (nhn(0, 2) - nhn(0, 1)) * np.exp(-2j * math.pi * f[i] * (k @ xbar))
        eps = 2 * math.pi * f[i] * L
        assert abs(x15[i] - ref) < 5 * eps * abs(ref)
        assert abs(x20[i] - 4j * eps * x15[i]) < 5 * eps * abs(x20[i])


def test_tdi20_is_tdi15_times_one_minus_z4(oracle_mod):
    det15 = dict(W.LISA, tdi_gen=15)
    L = W.LISA["arm_m"] / C_SI
    f = np.geomspace(1e-4, 4e-2, 11)
    th = TH.copy(); th[0] = 2e5
    a = oracle_mod.response_xyz(det15, th, W.MODE_ALL, f)
    b = oracle_mod.response_xyz(W.LISA, th, W.MODE_ALL, f)
    z = np.exp(-2j * math.pi * f * L)
    np.testing.assert_allclose(b, (1 - z ** 4) * a, rtol=1e-12, atol=1e-12 * np.abs(b).max())


def test_cyclic_permutation_by_constellation_rotation(oracle_mod):
    """Rotating the heliocentric constellation by 2 pi/3 relabels spacecraft i -> i+1, so
    X(rotated) = Y and Y(rotated) = Z: the Y and Z channels are the cyclic permutations of X."""
    f = np.geomspace(1e-4, 4e-2, 9)
    th = TH.copy(); th[0] = 3e5
    rot = dict(W.LISA, cartwheel0=2 * math.pi / 3)
    a = oracle_mod.response_xyz(W.LISA, th, W.MODE_ALL, f)
    b = oracle_mod.response_xyz(rot, th, W.MODE_ALL, f)
    sc = np.abs(a).max()
    np.testing.assert_allclose(b[0], a[1], atol=1e-11 * sc)
    np.testing.assert_allclose(b[1], a[2], atol=1e-11 * sc)
    np.testing.assert_allclose(b[2], a[0], atol=1e-11 * sc)


def test_aet_from_xyz_and_t_suppression(oracle_mod):
    f = np.geomspace(1e-5, 1e-3, 12)
    th = TH.copy()
    xyz = oracle_mod.response_xyz(W.LISA, th, W.MODE_ALL, f)
    aet = oracle_mod.response(W.LISA, th, W.MODE_ALL, f)
    X, Y, Z = xyz
    np.testing.assert_allclose(aet[0], (Z - X) / math.sqrt(2), rtol=1e-13, atol=1e-13 * np.abs(X).max())
    np.testing.assert_allclose(aet[1], (X - 2 * Y + Z) / math.sqrt(6), rtol=1e-13, atol=1e-13 * np.abs(X).max())
    np.testing.assert_allclose(aet[2], (X + Y + Z) / math.sqrt(3), rtol=1e-13, atol=1e-13 * np.abs(X).max())
    ratio = np.abs(aet[2]) / np.abs(aet[0])
    slope = np.polyfit(np.log(f), np.log(ratio), 1)[0]
    assert slope >= 1.0


# -------------------------------------------------------------------------------------------
# Noise and likelihood
# -------------------------------------------------------------------------------------------
def test_psd_aet_is_rotation_of_xyz_covariance(oracle_mod):
    """S_A, S_E, S_T are the diagonal of the A/E/T rotation of the equal-arm XYZ noise covariance
    (diagonal S_X = 16 sin^2 x [S_oms + (3 + cos 2x) S_acc], off-diagonal
    -8 sin^2 x cos x [S_oms + 4 S_acc]); TDI 2.0 multiplies by |1 - z^4|^2."""
    for det in (W.LISA, W.TIANQIN, dict(W.LISA, tdi_gen=15)):
        f = np.geomspace(1e-4, 5e-2, 17)
        S = oracle_mod.psd(det, f)
        L = det["arm_m"] / C_SI
        x = 2 * math.pi * f * L
        Soms = (det["oms_m_rtHz"] * 2 * math.pi * f / C_SI) ** 2
        Sacc = (det["acc_ms2_rtHz"] / (2 * math.pi * f * C_SI)) ** 2
        if det.get("psd_shaping", 1):
            Soms = Soms * (1 + (2e-3 / f) ** 4)
            Sacc = Sacc * (1 + (0.4e-3 / f) ** 2) * (1 + (f / 8e-3) ** 4)
        SX = 16 * np.sin(x) ** 2 * (Soms + (3 + np.cos(2 * x)) * Sacc)
        CXY = -8 * np.sin(x) ** 2 * np.cos(x) * (Soms + 4 * Sacc)
        R = np.array([[-1 / math.sqrt(2), 0, 1 / math.sqrt(2)],
                      [1 / math.sqrt(6), -2 / math.sqrt(6), 1 / math.sqrt(6)],
                      [1 / math.sqrt(3), 1 / math.sqrt(3), 1 / math.sqrt(3)]])
        fac = np.abs(1 - np.exp(-2j * x) ** 2) ** 2 if det["tdi_gen"] == 20 else np.ones_like(f)
        for i in range(f.size):
            Cm = np.full((3, 3), CXY[i]) + np.eye(3) * (SX[i] - CXY[i])
            Ca = R @ Cm @ R.T * fac[i]
            # the rotation cancels to O(x^2) in T, so its rounding is relative to S_X
            np.testing.assert_allclose(np.diag(Ca), S[:, i], rtol=1e-12, atol=1e-13 * SX[i] * fac[i])
            assert np.abs(Ca - np.diag(np.diag(Ca))).max() < 1e-13 * SX[i] * fac[i]


def test_oracle_rounding_against_long_double(oracle_mod):
    """The oracle's own FP64 rounding, measured against the same template evaluated in long double
    (or_response_ld), stays inside the rounding floor the GPU parity tests allow (tests/_helpers.py):
    per bin 1e-10 |h| + 32 u (Phi |h| + max(|A|, |E|) + max |h|) (the GPU bar takes 64), and per
    channel <h|h> within 1e-10 <h|h> + 2 u sqrt(<h|h> Q) (the GPU bar takes 8x that). On this x86
    host long double has a 64-bit significand; the check is skipped where long double is double."""
    from tests import _helpers as H
    if np.finfo(np.longdouble).nmant < 60:
        pytest.skip("long double has no extra precision on this platform")
    T = 2.0 ** 16
    k0, nb = W.grid(T)
    f = H.grid_f(T, k0, nb)
    ths = [np.array([3e5, 2.0, 0.5, 0.3, 25.8, 0.4, 1.3, 1.375, -1.2108, 2.659, 0.8 * T]),
           np.array([1e5, 7.0, -0.5, 0.9, 5.0, 2.4, 0.3, 4.0, 0.9, 0.6, 0.78 * T])] + list(W.draw_prior(3, 5, T))
    for det in (W.LISA, W.TIANQIN, dict(W.LISA, tdi_gen=15), W.TAIJI):
        w = 4.0 / (oracle_mod.psd(det, f) * T)
        for th in ths:
            for mask in (0x01, 0x10, 0x1F):
                a = oracle_mod.response(det, th, mask, f)
                b = oracle_mod.response_ld(det, th, mask, f)
                phi = H.phase_magnitude(oracle_mod, th, mask, f)
                ae = np.maximum(np.abs(b[0]), np.abs(b[1]))
                for c in range(3):
                    tol = 1e-10 * np.abs(b[c]) + 32 * H.U64 * (phi * np.abs(b[c]) + ae + np.abs(b[c]).max())
                    assert np.all(np.abs(a[c] - b[c]) <= tol), (det["name"], th[0], mask, c)
                hh_a, hh_b = np.sum(w * np.abs(a) ** 2, axis=1), np.sum(w * np.abs(b) ** 2, axis=1)
                Q = np.sum(w * (ae[None, :] ** 2 + phi[None, :] ** 2 * np.abs(b) ** 2), axis=1)
                assert np.all(np.abs(hh_a - hh_b) <= 1e-10 * hh_b + 2 * H.U64 * np.sqrt(hh_b * Q)), (
                    det["name"], th[0], mask, np.abs(hh_a - hh_b) / hh_b)


def _welch_psd(x, dt, nseg):
    """One-sided PSD of a real series by Welch averaging (Hann window, no overlap):
    P_k = 2 dt |sum_n w_n x_n e^{-2 pi i k n/N}|^2 / sum_n w_n^2, averaged over segments."""
    n = x.size // nseg
    seg = x[:n * nseg].reshape(nseg, n)
    w = 0.5 - 0.5 * np.cos(2 * math.pi * np.arange(n) / n)
    X = np.fft.rfft(seg * w, axis=1)
    return np.fft.rfftfreq(n, dt), 2.0 * dt * np.mean(np.abs(X) ** 2, axis=0) / np.sum(w * w)


def _single_link_noise_from_time_series(dt=1.0, n=1 << 23, nseg=2048, seed=20611):
    """Time-domain definitions of the two noise terms in fractional frequency (Sec. 3.2: test-mass
    acceleration and optical-metrology (OMS) noise), simulated:
    - OMS: white displacement noise x(t) of one-sided PSD a_oms^2 [m^2/Hz]; y = (dx/dt)/c, the
      derivative by a central difference;
    - acceleration: white acceleration a(t) of one-sided PSD a_acc^2 [m^2 s^-4/Hz]; y = v/c with
      v(t) = integral of a dt (a running sum).
    Returns the band frequencies and the averaged periodograms per unit a_oms^2 and a_acc^2, with
    the discrete operators' transfer functions divided out of the derivative and the running sum
    (both tend to 1 as f dt -> 0; the band keeps f dt <= 0.02)."""
    g = np.random.Generator(np.random.PCG64(seed))
    sig = 1.0 / math.sqrt(2.0 * dt)                 # white noise of unit one-sided PSD
    xd = g.standard_normal(n + 2) * sig
    y_oms = (xd[2:] - xd[:-2]) / (2.0 * dt) / C_SI
    acc = g.standard_normal(n) * sig
    y_acc = np.cumsum(acc) * dt / C_SI
    f, P_oms = _welch_psd(y_oms, dt, nseg)
    _, P_acc = _welch_psd(y_acc, dt, nseg)
    u = 2 * math.pi * f * dt
    band = (f >= 2e-3) & (f <= 0.02 / dt)
    P_oms = P_oms[band] / (np.sin(u[band]) / u[band]) ** 2
    P_acc = P_acc[band] / ((u[band] / 2) / np.sin(u[band] / 2)) ** 2
    return f[band], P_oms, P_acc


def _band_ratios(f, P, S):
    edges = np.geomspace(f[0], f[-1] * (1 + 1e-9), 7)
    return np.array([np.mean(P[(f >= lo) & (f < hi)] / S[(f >= lo) & (f < hi)]) for lo, hi in zip(edges[:-1], edges[1:])])


def test_psd_unit_conversion_against_time_domain_noise(oracle_mod):
    """The oracle's single-link OMS and acceleration terms in fractional frequency against averaged
    periodograms of simulated displacement and acceleration noise converted in the time domain
    (y = x'/c and y = (1/c) int a dt). The single-link terms are read from the oracle's S_A with the
    other noise switched off (TDI 1.5, no shaping): S_A = 8 sin^2 x (2 + cos x) S_oms and
    8 sin^2 x (6 + 4 cos x + 2 cos 2x) S_acc, the A/E/T algebra pinned by the covariance test.
    The estimate has ~1-2 % statistical error per band (bar 5 %); a dropped 2 pi, a missing 1/c or a wrong
    power of f, planted in copies written here, fails."""
    f, P_oms, P_acc = _single_link_noise_from_time_series()
    base = dict(W.TIANQIN, tdi_gen=15, psd_shaping=0)
    x = 2 * math.pi * f * base["arm_m"] / C_SI
    S_oms = oracle_mod.psd(dict(base, oms_m_rtHz=1.0, acc_ms2_rtHz=0.0), f)[0] / (8 * np.sin(x) ** 2 * (2 + np.cos(x)))
    S_acc = oracle_mod.psd(dict(base, oms_m_rtHz=0.0, acc_ms2_rtHz=1.0), f)[0] / (
        8 * np.sin(x) ** 2 * (6 + 4 * np.cos(x) + 2 * np.cos(2 * x)))
    r_oms, r_acc = _band_ratios(f, P_oms, S_oms), _band_ratios(f, P_acc, S_acc)
    assert np.all(np.abs(r_oms - 1) < 0.05), r_oms
    assert np.all(np.abs(r_acc - 1) < 0.05), r_acc
    planted = {"oms without 2 pi": (f / C_SI) ** 2, "oms with f^1": 2 * math.pi * f / C_SI ** 2,
               "acc without 1/c": 1 / (2 * math.pi * f) ** 2, "acc with f^-1": 1 / (2 * math.pi * f * C_SI ** 2),
               "acc two-sided": 0.5 / (2 * math.pi * f * C_SI) ** 2}
    for name, S in planted.items():
        P = P_oms if name.startswith("oms") else P_acc
        assert np.any(np.abs(_band_ratios(f, P, S) - 1) > 0.05), name


def test_parseval_brute_force_dft(oracle_mod):
    """White noise of variance sigma^2 at cadence dt has one-sided PSD 2 sigma^2 dt; with the
    DFT d~_k = dt sum_j n_j e^{-2 pi i jk/N}, sum_j n_j^2/sigma^2 = <d|d> exactly when the series
    has no DC or Nyquist content (Eq. eq_inner_product, Eq. eq_diag_Sigma_to_Sn)."""
    N, dt, sigma = 256, 10.0, 1.7e-20
    rng = np.random.Generator(np.random.PCG64(7))
    n = rng.standard_normal(N) * sigma
    j = np.arange(N)
    n = n - n.mean() - ((-1.0) ** j) * np.mean(n * (-1.0) ** j)
    T = N * dt
    ks = np.arange(1, N // 2)
    dft = np.array([dt * np.sum(n * np.exp(-2j * math.pi * j * k / N)) for k in ks])
    data = np.stack([dft, dft, dft])
    psd = np.full((3, ks.size), 2 * sigma ** 2 * dt)
    D = oracle_mod.Detector(W.LISA, T, 1, ks.size, data, psd)
    r = oracle_mod.loglike([D], TH, 0)
    ref = np.sum(n ** 2) / sigma ** 2
    np.testing.assert_allclose(r["dd"][0], ref, rtol=1e-12)
    assert r["logl"] == pytest.approx(-1.5 * ref, rel=1e-12)


def _single(oracle_mod, normals_seed=None, T=2.0 ** 20, mask=W.MODE_22, det=W.LISA, th=None):
    k0, nb = W.grid(T)
    f = (k0 + np.arange(nb)) / T
    th = TH if th is None else th
    nrm = None if normals_seed is None else W.normals(nb, normals_seed)
    d = oracle_mod.make_data(det, th, mask, T, k0, nb, nrm)
    return oracle_mod.Detector(det, T, k0, nb, d, oracle_mod.psd(det, f))


def test_noiseless_injection(oracle_mod):
    D = _single(oracle_mod, None, mask=W.MODE_ALL)
    r = oracle_mod.loglike([D], TH, W.MODE_ALL)
    snr2 = r["hh"].sum()
    assert snr2 > 1e4
    assert abs(r["logl"]) < 1e-12 * snr2
    np.testing.assert_allclose(r["dh"], r["hh"], rtol=1e-13)
    np.testing.assert_allclose(r["dd"], r["hh"], rtol=1e-13)


def test_noise_chi2(oracle_mod):
    """-1/2 <n|n> per channel has mean -N_b and variance N_b (Re, Im ~ N(0, S T/4))."""
    T = 2.0 ** 16
    k0, nb = W.grid(T)
    th = TH.copy(); th[4] = 1e12          # signal negligible
    vals = []
    for seed in range(6):
        D = _single(oracle_mod, 100 + seed, T=T, th=th)
        r = oracle_mod.loglike([D], th, W.MODE_22)
        vals.extend(list(-0.5 * r["dd"][0]))
    vals = np.array(vals)
    assert abs(vals.mean() + nb) < 5 * math.sqrt(nb / vals.size)
    assert vals.var() == pytest.approx(nb, rel=0.8)


def test_tdi15_and_tdi20_whitened_products_agree(oracle_mod):
    """TDI 2.0 multiplies every channel's signal by (1 - z^4) and its PSD by |1 - z^4|^2 (Sec. 2.1,
    Sec. 3.2), so with noise-free data every whitened product, hence log L, <d|h>, <h|h> and the
    SNR, is the same for the two generations; only bins with 1 - z^4 = 0 would differ, and none
    lies on the grid."""
    T = 2.0 ** 14
    k0, nb = W.grid(T)
    f = (k0 + np.arange(nb)) / T
    inj = TH.copy(); inj[0] = 3e5; inj[10] = 0.8 * T
    res = []
    for det in (dict(W.LISA, tdi_gen=15), W.LISA):
        d = oracle_mod.make_data(det, inj, W.MODE_ALL, T, k0, nb, None)
        D = oracle_mod.Detector(det, T, k0, nb, d, oracle_mod.psd(det, f))
        ths = np.vstack([inj, inj + np.array([2e3, 0.05, 0.1, -0.1, 1.0, 0.05, 0.3, 0.01, 0.02, 0.1, 3.0])])
        res.append([oracle_mod.loglike([D], th, W.MODE_ALL) for th in ths])
    for a, b in zip(*res):
        scale = 0.5 * a["dd"].sum() + abs(a["dh"].sum()) + 0.5 * a["hh"].sum()
        assert scale > 1e3
        assert abs(a["logl"] - b["logl"]) < 1e-11 * scale
        np.testing.assert_allclose(b["hh"], a["hh"], rtol=1e-11)
        np.testing.assert_allclose(b["dh"], a["dh"], rtol=1e-11, atol=1e-11 * scale)


def test_residual_form_equals_component_form(oracle_mod):
    D = _single(oracle_mod, 12011, mask=W.MODE_ALL)
    for dq in (0.0, 1e-3, 0.1):
        th = TH.copy(); th[1] += dq; th[7] += dq
        r = oracle_mod.loglike([D], th, W.MODE_ALL)
        scale = 0.5 * r["dd"].sum() + abs(r["dh"].sum()) + 0.5 * r["hh"].sum()
        assert abs(r["logl"] - r["logl_resid"]) < 1e-13 * scale


# -------------------------------------------------------------------------------------------
# Gradient and Fisher (Sec. 2.2 and the AD discussion of Sec. 2.3)
# -------------------------------------------------------------------------------------------
def test_grad_dl_closed_form(oracle_mod):
    D = _single(oracle_mod, 12011, mask=W.MODE_ALL)
    th = TH.copy(); th[0] *= 1.0001; th[10] += 3.0
    r = oracle_mod.loglike([D], th, W.MODE_ALL)
    ll, g = oracle_mod.grad([D], th, W.MODE_ALL)
    assert ll == pytest.approx(r["logl"], rel=1e-14)
    ref = -(r["dh"].sum() - r["hh"].sum()) / th[4]
    assert g[4] == pytest.approx(ref, rel=1e-10)


def test_fisher_closed_forms(oracle_mod):
    D = _single(oracle_mod, None, mask=W.MODE_22)
    F = oracle_mod.fisher([D], TH, W.MODE_22)
    r = oracle_mod.loglike([D], TH, W.MODE_22)
    hh = r["hh"].sum()
    assert F[4, 4] == pytest.approx(hh / TH[4] ** 2, rel=1e-10)
    assert F[6, 6] == pytest.approx(4 * hh, rel=1e-10)
    np.testing.assert_allclose(F, F.T, rtol=1e-13, atol=1e-13 * np.abs(F).max())
    ev = np.linalg.eigvalsh(F / np.sqrt(np.outer(np.diag(F), np.diag(F))))
    assert ev.min() > -1e-9


def test_fisher_equals_jt_w_j(oracle_mod):
    T = 2.0 ** 18
    k0, nb = W.grid(T)
    th = TH.copy(); th[10] = 0.8 * T
    D = _single(oracle_mod, None, T=T, mask=W.MODE_ALL, th=th)
    F = oracle_mod.fisher([D], th, W.MODE_ALL)
    f = (k0 + np.arange(nb)) / T
    J = oracle_mod.response_jac(W.LISA, th, W.MODE_ALL, f)       # [n][3][2][11]
    w = 4.0 / (D.psd * T)                                         # [3][n]
    Fr = np.einsum("cn,ncri,ncrj->ij", w, J, J)
    np.testing.assert_allclose(F, Fr, rtol=1e-10, atol=1e-12 * np.abs(F).max())


def test_drho_diota_symbolic(oracle_mod):
    """The paper's own derivative check (Fig. fig_nerr_diota): for the (2,2) mode,
    rho^2(iota) = a ((1+c^2)/2)^2 + b c^2 + e c (1+c^2)/2 with c = cos(iota), so d rho/d iota is
    known symbolically once a, b, e are fitted from three inclinations; the dual-number gradient
    must agree to near machine precision and central differences only at a good step."""
    T = 2.0 ** 20
    k0, nb = W.grid(T)
    f = (k0 + np.arange(nb)) / T
    zero = np.zeros((3, nb), dtype=np.complex128)
    D = oracle_mod.Detector(W.LISA, T, k0, nb, zero, oracle_mod.psd(W.LISA, f))
    def rho2(inc):
        th = TH.copy(); th[5] = inc
        return -2 * oracle_mod.loglike([D], th, W.MODE_22)["logl"]
    incs = np.array([0.3, 1.2, 2.2])
    c = np.cos(incs)
    A = np.stack([((1 + c ** 2) / 2) ** 2, c ** 2, c * (1 + c ** 2) / 2], axis=1)
    a, b, e = np.linalg.solve(A, [rho2(i) for i in incs])
    inc = TH[5]
    ci, si = math.cos(inc), math.sin(inc)
    r2 = a * ((1 + ci ** 2) / 2) ** 2 + b * ci ** 2 + e * ci * (1 + ci ** 2) / 2
    assert rho2(inc) == pytest.approx(r2, rel=1e-11)
    dr2 = (a * (1 + ci ** 2) * ci + 2 * b * ci + e * ((1 + ci ** 2) / 2 + ci * ci)) * (-si)
    drho_sd = dr2 / (2 * math.sqrt(r2))
    ll, g = oracle_mod.grad([D], TH, W.MODE_22)
    rho = math.sqrt(-2 * ll)
    drho_ad = -g[5] / rho
    assert drho_ad == pytest.approx(drho_sd, rel=1e-9)
    h = 1e-5
    drho_nd = (math.sqrt(rho2(inc + h)) - math.sqrt(rho2(inc - h))) / (2 * h)
    assert drho_nd == pytest.approx(drho_sd, rel=1e-6)


def test_grad_matches_central_differences(oracle_mod):
    D = _single(oracle_mod, 12011, mask=W.MODE_ALL, T=2.0 ** 19,
                th=np.r_[TH[:10], 0.8 * 2.0 ** 19])
    th = np.r_[TH[:10], 0.8 * 2.0 ** 19]
    th = th + np.array([1e3, 0.01, 0.02, -0.02, 0.1, 0.01, 0.05, 0.002, 0.002, 0.01, 2.0])
    ll, g = oracle_mod.grad([D], th, W.MODE_ALL)
    steps = np.array([1.0, 1e-5, 1e-5, 1e-5, 1e-4, 1e-6, 1e-6, 1e-7, 1e-7, 1e-6, 1e-3])
    for i in range(11):
        tp = th.copy(); tp[i] += steps[i]
        tm = th.copy(); tm[i] -= steps[i]
        fd = (oracle_mod.loglike([D], tp, W.MODE_ALL)["logl"] - oracle_mod.loglike([D], tm, W.MODE_ALL)["logl"]) \
            / (2 * steps[i])
        assert g[i] == pytest.approx(fd, rel=2e-4, abs=1e-6 * np.abs(g).max()), W.PARAM_NAMES[i]
