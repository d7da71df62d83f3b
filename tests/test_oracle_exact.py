"""Pins of the exact references themselves (oracle/exact.py, oracle/ising.py).

Each reference is checked against an independent one: the two Onsager
integral forms against each other and against the K = 0 limit; the C
enumerator against the transfer-matrix contraction of the Ising tensor
network (which also pins the site tensor T0 of SM Sec. A); the enumerator's
beta and h derivatives against finite differences of its own ln Z.
"""
import math

import numpy as np
import pytest

from oracle import exact, ising
import synth


@pytest.mark.parametrize("beta", [0.30, 0.44, synth.BETA_C, 0.60])
def test_onsager_two_forms_agree(beta):
    a = exact.onsager_lnz(beta)
    b = exact.onsager_lnz_1d(beta)
    assert abs(a - b) < 1e-12


def test_onsager_high_temperature_limit():
    assert abs(exact.onsager_lnz(0.0) - math.log(2.0)) < 1e-14
    assert abs(exact.onsager_lnz_1d(0.0) - math.log(2.0)) < 1e-14
    # deep in the ordered phase ln Z / N -> 2 beta J (ground state, 2 bonds per site)
    b = 1.5
    assert abs(exact.onsager_lnz_1d(b) - 2 * b) < 1e-4


def test_onsager_critical_value():
    # at the critical point kappa = 1 exactly and the known closed value of
    # -beta f is ln(sqrt 2) + 2G/pi (G = Catalan's constant)
    catalan = 0.915965594177219015054603514932
    expect = 0.5 * math.log(2.0) + 2 * catalan / math.pi
    assert abs(exact.onsager_lnz_1d(synth.BETA_C) - expect) < 1e-12
    assert abs(exact.onsager_lnz(synth.BETA_C) - expect) < 1e-10


@pytest.mark.parametrize("Lx,Ly", [(2, 2), (2, 4), (4, 4), (4, 2), (6, 4)])
@pytest.mark.parametrize("beta,h", [(0.44, 0.0), (0.3, 0.1), (0.6, -0.05)])
def test_bruteforce_matches_tensor_network_torus(Lx, Ly, beta, h):
    lnz, _, _ = exact.bruteforce(Lx, Ly, beta, 1.0, h)
    tm = exact.torus_lnz(ising.ising_T0(beta, 1.0, h), Lx, Ly) / (Lx * Ly)
    assert abs(lnz - tm) < 1e-13


def test_bruteforce_small_closed_form():
    # 1 x 1 torus: two self-bonds, Z = 2 e^{2 beta J} cosh(beta h)
    b, h = 0.37, 0.2
    lnz, _, _ = exact.bruteforce(1, 1, b, 1.0, h)
    assert abs(lnz - (2 * b + math.log(2 * math.cosh(b * h)))) < 1e-14
    g = exact.density_of_states(4, 4)
    assert g.sum() == 2 ** 16


def test_bruteforce_derivatives_match_finite_differences():
    beta, h, e = 0.41, 0.07, 1e-5
    lnz, db, dh = exact.bruteforce(4, 4, beta, 1.0, h)
    fd_b = (exact.bruteforce(4, 4, beta + e, 1.0, h)[0] - exact.bruteforce(4, 4, beta - e, 1.0, h)[0]) / (2 * e)
    fd_h = (exact.bruteforce(4, 4, beta, 1.0, h + e)[0] - exact.bruteforce(4, 4, beta, 1.0, h - e)[0]) / (2 * e)
    assert abs(db - fd_b) < 1e-8
    assert abs(dh - fd_h) < 1e-8


def test_ising_T0_bond_split_and_symmetry():
    beta, h = 0.52, 0.03
    T = ising.ising_T0(beta, 1.0, h)
    # reflection and rotation symmetric
    assert np.allclose(T, T.transpose(1, 0, 2, 3), atol=0, rtol=0)
    assert np.allclose(T, T.transpose(2, 3, 0, 1), atol=0, rtol=0)
    # beta = 0: only the all-zero index survives, with weight 2 cosh(0) = 2
    T0 = ising.ising_T0(0.0, 1.0, 0.0)
    assert T0[0, 0, 0, 0] == 2.0 and np.count_nonzero(T0) == 1


def test_ising_dT0_dbeta_matches_finite_differences():
    beta, h, e = 0.44, 0.01, 1e-6
    d = ising.ising_dT0_dbeta(beta, 1.0, h)
    fd = (ising.ising_T0(beta + e, 1.0, h) - ising.ising_T0(beta - e, 1.0, h)) / (2 * e)
    assert np.max(np.abs(d - fd)) < 1e-8
