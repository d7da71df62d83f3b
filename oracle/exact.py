"""Exact references used to pin the oracle (test infrastructure only).

* Onsager's free energy of the square-lattice Ising model at h = 0, in two
  independent textbook forms (the paper benchmarks against the exact Ising
  free energy, main text Fig. 2):
    (i)  ln Z/N = ln 2 + 1/(8 pi^2) int_0^{2pi} int_0^{2pi}
                  ln[cosh^2 2K - sinh 2K (cos t1 + cos t2)] dt1 dt2,
    (ii) ln Z/N = ln(2 cosh 2K) + 1/(2 pi) int_0^pi
                  ln[(1 + sqrt(1 - kappa^2 sin^2 phi)) / 2] dphi,
         kappa = 2 sinh 2K / cosh^2 2K,   K = beta J.
* Brute-force enumeration of small periodic tori (C, density of states).
* Exact contraction of a periodic torus of identical rank-4 tensors by a
  row transfer matrix -- the plain definition of Z as the trace of the
  tensor network (SM Sec. A), without any truncation.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np
from scipy import integrate

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None
_LOCK = threading.Lock()


def build_bruteforce() -> str:
    """Compile bruteforce.c into oracle/_build/ (plain gcc, no GPU)."""
    out_dir = os.path.join(_HERE, "_build")
    os.makedirs(out_dir, exist_ok=True)
    so = os.path.join(out_dir, "libbruteforce.so")
    src = os.path.join(_HERE, "bruteforce.c")
    if not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(src):
        tmp = so + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-shared", "-fPIC", "-o", tmp, src])
        os.replace(tmp, so)
    return so


def _lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            lib = ctypes.CDLL(build_bruteforce())
            lib.ising_density_of_states.argtypes = [ctypes.c_int, ctypes.c_int,
                                                    ctypes.POINTER(ctypes.c_int64)]
            lib.ising_density_of_states.restype = ctypes.c_int
            _LIB = lib
    return _LIB


def density_of_states(Lx: int, Ly: int) -> np.ndarray:
    """g[b, m]: count of configurations with bond sum b - 2n, magnetisation m - n."""
    n = Lx * Ly
    g = np.zeros((4 * n + 1, 2 * n + 1), dtype=np.int64)
    rc = _lib().ising_density_of_states(Lx, Ly, g.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
    if rc != 0:
        raise ValueError("torus too large for enumeration")
    return g


def bruteforce(Lx: int, Ly: int, beta: float, J: float = 1.0, h: float = 0.0):
    """Exact (ln Z / N, d(ln Z/N)/d beta, d(ln Z/N)/d h) of the Lx x Ly torus."""
    n = Lx * Ly
    g = density_of_states(Lx, Ly)
    b = np.arange(-2 * n, 2 * n + 1, dtype=np.float64)[:, None]
    m = np.arange(-n, n + 1, dtype=np.float64)[None, :]
    mask = g > 0
    expo = np.where(mask, beta * J * b + beta * h * m, -np.inf)
    mx = expo[mask].max()
    wgt = np.where(mask, g * np.exp(expo - mx), 0.0)
    Zs = wgt.sum()
    lnz = (math.log(Zs) + mx) / n
    dbeta = float(((J * b + h * m) * wgt).sum() / Zs) / n
    dh = float((beta * m * wgt).sum() / Zs) / n
    return lnz, dbeta, dh


def torus_lnz(T: np.ndarray, Lx: int, Ly: int) -> float:
    """ln Z (total) of an Lx x Ly periodic torus of copies of T[l, r, u, d]:
    r of each tensor meets l of its right neighbour, d meets u of the
    tensor below, both directions periodic.  Row transfer matrix
    M[(u_1..u_Lx), (d_1..d_Lx)] = sum_l prod_i T[l_i, l_{i+1}, u_i, d_i]
    (l_{Lx+1} = l_1), and Z = tr M^Ly."""
    dl, du = T.shape[0], T.shape[2]
    R = T.copy()                                   # [l_first, l_next, U, D]
    for _ in range(1, Lx):
        R = np.einsum("amUD,mbud->abUuDd", R, T).reshape(dl, dl, R.shape[2] * du, R.shape[3] * du)
    M = np.einsum("aaUD->UD", R)
    s = np.abs(M).max()
    P = np.linalg.matrix_power(M / s, Ly)
    tr = np.trace(P)
    return math.log(abs(tr)) + Ly * math.log(s)


def onsager_lnz(beta: float, J: float = 1.0) -> float:
    """Form (i): double integral."""
    K = beta * J
    c2, s2 = math.cosh(2 * K) ** 2, math.sinh(2 * K)

    def f(t1, t2):
        return math.log(c2 - s2 * (math.cos(t1) + math.cos(t2)))

    val, _ = integrate.dblquad(f, 0.0, 2 * math.pi, 0.0, 2 * math.pi,
                               epsabs=1e-14, epsrel=1e-14)
    return math.log(2.0) + val / (8 * math.pi ** 2)


def onsager_lnz_1d(beta: float, J: float = 1.0) -> float:
    """Form (ii): single integral with kappa = 2 sinh 2K / cosh^2 2K."""
    K = beta * J
    kap = 2 * math.sinh(2 * K) / math.cosh(2 * K) ** 2

    def f(p):
        return math.log(0.5 * (1.0 + math.sqrt(max(0.0, 1.0 - (kap * math.sin(p)) ** 2))))

    val, _ = integrate.quad(f, 0.0, math.pi, points=[math.pi / 2], epsabs=1e-15,
                            epsrel=1e-14, limit=500)
    return math.log(2 * math.cosh(2 * K)) + val / (2 * math.pi)
