"""Quantum XY chain: exact partition functions and the Trotter density-matrix
MPO, plain FP64 on the CPU (NumPy / SciPy).

TEST INFRASTRUCTURE ONLY (see the package docstring): never called by the
product path.

Model (main text, "Infinite quantum XY chain"; SM Sec. F and G):

    H = J sum_i (S^x_i S^x_{i+1} + S^y_i S^y_{i+1}),   S^a = sigma^a / 2.

Exact solution (SM Sec. G).  The Jordan-Wigner transformation maps H to
free fermions with single-particle energies eps_q = J cos q.  On a periodic
ring of N sites the fermion-parity sectors see different boundary
conditions, and each sector keeps only the states of its parity:

    Z = 1/2 [prod_{q in P_a}(1 + e^{-beta eps_q}) + prod_{q in P_a}(1 - e^{-beta eps_q})]
      + 1/2 [prod_{q in P_p}(1 + e^{-beta eps_q}) - prod_{q in P_p}(1 - e^{-beta eps_q})],

P_a = {2 pi (n + 1/2) / N} (antiperiodic) for the even-parity sector,
P_p = {2 pi n / N} (periodic) for the odd-parity sector.  Reading: the
fermion Hamiltonian of SM Sec. G carries the boundary hop -Q c_N^+ c_1, so
the even sector (Q = 1) is antiperiodic; the sentence after it attaches the
periodic momenta to the even sector instead.  Exact diagonalisation of the
spin Hamiltonian (``lnz_ed``) decides: it agrees with the assignment above
to rounding and not with the other one (tests/test_oracle_xy.py).  In the
thermodynamic limit both sectors give

    ln Z / N = (1 / 2 pi) int_0^{2 pi} ln(1 + e^{-beta J cos q}) dq.

Density-matrix MPO (SM Sec. F).  H = H_o + H_e (bonds (1,2), (3,4), ... and
(2,3), (4,5), ...), and to second order in tau

    rho(tau) = e^{-tau/2 H_o} e^{-tau H_e} e^{-tau/2 H_o}.

The odd bonds lie inside two-site cells (sites 2c-1, 2c); the even bonds join
neighbouring cells.  Each even-bond gate is split by an operator SVD into a
left factor on site 2c and a right factor on site 2c+1, so rho(tau) is a
translation-invariant MPO with one rank-4 tensor per cell,

    T0[l, r, u, d]   (l, r: the even-bond index, dimension 4;
                      u = (s_1 s_2) the row (ket), d = the column (bra),
                      dimension 4 each),

in the layout of the HOTRG step (main text Fig. 1b: the MPO product
rho(2 tau) = rho(tau) rho(tau) is the vertical merge, contracting the upper
tensor's d with the lower tensor's u).
"""
from __future__ import annotations

import math

import numpy as np
from scipy import integrate
from scipy.linalg import expm

_SX = np.array([[0.0, 1.0], [1.0, 0.0]]) / 2.0
_SY = np.array([[0.0, -1.0j], [1.0j, 0.0]]) / 2.0


def bond_hamiltonian(J: float = 1.0) -> np.ndarray:
    """h = J (S^x S^x + S^y S^y) on two sites, 4 x 4 real, basis (s1 s2)."""
    h = J * (np.kron(_SX, _SX) + np.kron(_SY, _SY))
    return np.real_if_close(h).astype(np.float64)


def _site_op(op, i, N):
    m = np.array([[1.0]])
    for j in range(N):
        m = np.kron(m, op if j == i else np.eye(2))
    return m


def hamiltonian_dense(N: int, J: float = 1.0, bonds=None) -> np.ndarray:
    """Dense 2^N x 2^N H of the periodic ring (site 0 = most significant
    bit).  ``bonds``: the first sites i of the bonds (i, i+1 mod N) to
    include (default: all)."""
    if bonds is None:
        bonds = range(N)
    H = np.zeros((2 ** N, 2 ** N), dtype=complex)
    for i in bonds:
        j = (i + 1) % N
        H += J * (_site_op(_SX, i, N) @ _site_op(_SX, j, N) +
                  _site_op(_SY, i, N) @ _site_op(_SY, j, N))
    return np.real_if_close(H).astype(np.float64)


def lnz_ed(N: int, beta: float, J: float = 1.0) -> float:
    """ln Z of the periodic N-site ring by exact diagonalisation."""
    E = np.linalg.eigvalsh(hamiltonian_dense(N, J))
    m = -beta * E
    top = m.max()
    return float(top + math.log(np.sum(np.exp(m - top))))


def lnz_exact_finite(N: int, beta: float, J: float = 1.0) -> float:
    """ln Z of the periodic N-site ring from the fermion-parity sectors
    (SM Sec. G; the sector momenta as read in the module docstring)."""
    n = np.arange(N)
    q_anti = 2.0 * math.pi * (n + 0.5) / N
    q_per = 2.0 * math.pi * n / N
    xa = -beta * J * np.cos(q_anti)
    xp = -beta * J * np.cos(q_per)
    z_even = 0.5 * (np.prod(1.0 + np.exp(xa)) + np.prod(1.0 - np.exp(xa)))
    z_odd = 0.5 * (np.prod(1.0 + np.exp(xp)) - np.prod(1.0 - np.exp(xp)))
    return float(math.log(z_even + z_odd))


def lnz_exact_infinite(beta: float, J: float = 1.0) -> float:
    """ln Z per site of the infinite chain (thermodynamic limit of SM Sec. G)."""
    val, _ = integrate.quad(lambda q: math.log1p(math.exp(-beta * J * math.cos(q))),
                            0.0, 2.0 * math.pi, epsabs=1e-14, epsrel=1e-14, limit=200)
    return val / (2.0 * math.pi)


def free_energy_infinite(beta: float, J: float = 1.0) -> float:
    """f = -ln Z / (N beta) per site of the infinite chain."""
    return -lnz_exact_infinite(beta, J) / beta


def trotter_dense(N: int, tau: float, J: float = 1.0) -> np.ndarray:
    """e^{-tau/2 H_o} e^{-tau H_e} e^{-tau/2 H_o} on the periodic N-site ring
    (N even; H_o: bonds (0,1), (2,3), ...; H_e: bonds (1,2), ..., (N-1,0))."""
    if N % 2:
        raise ValueError("the two-site cells need an even ring")
    Ho = hamiltonian_dense(N, J, bonds=range(0, N, 2))
    He = hamiltonian_dense(N, J, bonds=range(1, N, 2))
    half = expm(-0.5 * tau * Ho)
    return half @ expm(-tau * He) @ half


def mpo_cell(tau: float, J: float = 1.0) -> np.ndarray:
    """T0[l, r, u, d] of rho(tau) for one two-site cell (SM Sec. F, second
    order Trotter), shape (4, 4, 4, 4)."""
    h = bond_hamiltonian(J)
    g_odd = expm(-0.5 * tau * h).reshape(2, 2, 2, 2)     # [s1, s2, t1, t2]
    g_even = expm(-tau * h).reshape(2, 2, 2, 2)          # [a, b, a', b']: a left, b right site
    # operator SVD across the bond: g_even[a b, a' b'] = sum_k L_k[a, a'] R_k[b, b']
    M = g_even.transpose(0, 2, 1, 3).reshape(4, 4)       # [(a a'), (b b')]
    U, s, Vt = np.linalg.svd(M)
    Lk = (U * np.sqrt(s)).reshape(2, 2, 4)               # [a, a', k]
    Rk = (np.sqrt(s)[:, None] * Vt).reshape(4, 2, 2)     # [k, b, b']
    # the cell's site 1 is the right site of the even bond on its left (index l),
    # its site 2 the left site of the even bond on its right (index r):
    # T[l, r, (s1 s2), (v1 v2)] = sum g_odd[s1 s2, t1 t2] R_l[t1, t1'] L_r[t2, t2'] g_odd[t1' t2', v1 v2]
    T = np.einsum("abcd,lce,dfr,efgh->lrabgh", g_odd, Rk, Lk, g_odd, optimize=True)
    return np.ascontiguousarray(T.reshape(4, 4, 4, 4))


def mpo_ring_trace(T: np.ndarray, L: int) -> float:
    """Tr of the MPO with L copies of the cell tensor T[l, r, u, d] on a
    ring: Tr_phys of the product operator = Tr (M^L), M[l, r] = sum_u T[l, r, u, u]."""
    M = np.einsum("lruu->lr", T)
    return float(np.trace(np.linalg.matrix_power(M, L)))


def mpo_ring_dense(T: np.ndarray, L: int) -> np.ndarray:
    """The dense operator (d^L x d^L, cell 0 most significant) of the MPO
    ring of L cells, for pins on small rings."""
    D, _, d, _ = T.shape
    # contract cell by cell, keeping the first bond open: A[l0, r, U, V]
    A = T.copy()
    for _ in range(1, L):
        A = np.einsum("lmUV,mrud->lrUuVd", A, T).reshape(D, D, A.shape[2] * d, A.shape[3] * d)
    return np.einsum("llUV->UV", A)
