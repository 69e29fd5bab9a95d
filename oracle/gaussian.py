"""Gaussian formalism and the iterative GSVD chain (FP64, numpy).

Sec. II A (covariance matrix, Williamson form Eq. (symDiag), Bogoliubov map
Eq. (MUV)/(bmode), Schmidt parameters Eq. (SVD1)), Sec. II B (GSVD
Eqs. (SVD2)-(bond), paired form Eq. (Q_matrix), iterative decomposition
Eq. (Am_ket)/(GMPS)), App. A (paired form Eq. (paired-form)/(matrix_Q),
regularised Q_L).

Quadrature convention: a = (x + i p)/sqrt(2), R = (x_1..x_n, p_1..p_n),
Gamma = (1/2)<{dR, dR}>, vacuum Gamma = I/2, Omega = [[0, I], [-I, 0]].
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


def omega(n: int) -> np.ndarray:
    z, i = np.zeros((n, n)), np.eye(n)
    return np.block([[z, i], [-i, z]])


# --------------------------------------------------------------------------
# moments and the paired form
# --------------------------------------------------------------------------
def complex_moments(gamma: np.ndarray):
    """N_jk = <a_j^dag a_k>, M_jk = <a_j a_k> from Gamma (Sec. II A, Eq. (GammaMat)
    with a = (x + i p)/sqrt 2 and [x_j, p_k] = i delta_jk)."""
    n = gamma.shape[0] // 2
    gxx, gxp = gamma[:n, :n], gamma[:n, n:]
    gpx, gpp = gamma[n:, :n], gamma[n:, n:]
    Nm = 0.5 * (gxx + gpp + 1j * (gxp - gpx)) - 0.5 * np.eye(n)
    Mm = 0.5 * (gxx - gpp + 1j * (gxp + gpx))
    return Nm, Mm


def q_from_gamma(gamma: np.ndarray) -> np.ndarray:
    """Paired-form matrix of a pure state, Eq. (paired-form): from a_i|psi> =
    (Q a^dag)_i |psi>, <a_k a_i> = (Q (1 + N))_ik, so Q = M (1 + N)^{-1}."""
    Nm, Mm = complex_moments(gamma)
    q = Mm @ np.linalg.inv(np.eye(Nm.shape[0]) + Nm)
    return 0.5 * (q + q.T)


def gamma_from_q(Q: np.ndarray) -> np.ndarray:
    """Inverse of q_from_gamma: N = (1 - Q*Q)^{-1} - 1, M = Q (1 + N)."""
    n = Q.shape[0]
    Nm = np.linalg.inv(np.eye(n) - Q.conj() @ Q) - np.eye(n)
    Mm = Q @ (np.eye(n) + Nm)
    gxx = Nm.real + Mm.real + 0.5 * np.eye(n)
    gpp = Nm.real - Mm.real + 0.5 * np.eye(n)
    gxp = Nm.imag + Mm.imag
    gpx = Mm.imag - Nm.imag
    g = np.block([[gxx, gxp], [gpx, gpp]])
    return 0.5 * (g + g.T)


def purity_defect(gamma: np.ndarray) -> float:
    """max |(2 Gamma Omega)^2 + 1|: zero iff every symplectic eigenvalue of
    2 Gamma is 1, i.e. the Gaussian state is pure (Sec. II A)."""
    n = gamma.shape[0] // 2
    x = 2.0 * gamma @ omega(n)
    return float(np.max(np.abs(x @ x + np.eye(2 * n))))


# --------------------------------------------------------------------------
# Williamson and the Bogoliubov matrices
# --------------------------------------------------------------------------
def williamson(gamma: np.ndarray):
    """Eq. (symDiag): Gamma = (1/2) S diag(D, D) S^T with S symplectic and D
    descending.  Textbook construction: V = 2 Gamma = L L^T (Cholesky); the
    antisymmetric K = L^{-1} Omega L^{-T} has eigenvalues +-i/D; the Hermitian
    i K has eigenvalues +-1/D.  For each positive eigenvalue 1/D with unit
    eigenvector w = (u + i v)/sqrt 2, K u = v/D and K v = -u/D; with O =
    [v_1..v_n | u_1..u_n] one gets O^T K O = [[0, D^-1], [-D^-1, 0]] and
    S = L O diag(D, D)^{-1/2}."""
    n = gamma.shape[0] // 2
    V = 2.0 * gamma
    L = np.linalg.cholesky(V)
    Li = np.linalg.inv(L)
    K = Li @ omega(n) @ Li.T
    ev, W = np.linalg.eigh(1j * K)          # ascending; positive half is 1/D ascending
    inv_d = ev[n:]
    Wp = W[:, n:]
    D = 1.0 / inv_d                          # descending
    u = np.sqrt(2.0) * Wp.real
    v = np.sqrt(2.0) * Wp.imag
    O = np.concatenate([v, u], axis=1)
    S = L @ O @ np.diag(np.concatenate([D, D]) ** -0.5)
    return D, S


def williamson_sqrt(gamma: np.ndarray):
    """A second valid FP64 route to Eq. (symDiag), used to measure how far the
    Williamson factor of a given Gamma is determined in FP64 at all.  Instead
    of the Cholesky factor it takes the symmetric square root V^{1/2} (from
    the symmetric eigendecomposition of V = 2 Gamma, the textbook
    construction): K = V^{-1/2} Omega V^{-1/2}, i K Hermitian with eigenvalues
    +-1/D, and S = V^{1/2} O diag(D, D)^{-1/2} with O built from the unit
    eigenvectors exactly as in ``williamson``.  Any other valid route gives the
    same D and the same S up to the rounding of the eigenvectors, which is
    large only for nearly degenerate D."""
    n = gamma.shape[0] // 2
    V = 2.0 * gamma
    ev, E = np.linalg.eigh(V)
    Vh = (E * np.sqrt(ev)) @ E.T
    Vmh = (E / np.sqrt(ev)) @ E.T
    K = Vmh @ omega(n) @ Vmh
    evk, W = np.linalg.eigh(1j * K)
    D = 1.0 / evk[n:]
    Wp = W[:, n:]
    O = np.concatenate([np.sqrt(2.0) * Wp.imag, np.sqrt(2.0) * Wp.real], axis=1)
    S = Vh @ O @ np.diag(np.concatenate([D, D]) ** -0.5)
    return D, S


def uv_from_s(S: np.ndarray):
    """Bogoliubov matrices of the modes b with quadratures R_b = S^{-1} R.
    From R = S R_b and a = (x + i p)/sqrt 2 one gets a = U b + V^* b^dag with
    U = [(S11 + S22) + i (S21 - S12)]/2, V = [(S11 - S22) - i (S21 + S12)]/2,
    equivalently b = U^dag a - V^dag a^dag (App. A).  This is Eq. (MUV) up to
    the per-mode phase convention of b, a gauge the method leaves free."""
    n = S.shape[0] // 2
    s11, s12, s21, s22 = S[:n, :n], S[:n, n:], S[n:, :n], S[n:, n:]
    U = 0.5 * ((s11 + s22) + 1j * (s21 - s12))
    V = 0.5 * ((s11 - s22) - 1j * (s21 + s12))
    return U, V


def sinv_rows_from_uv(U: np.ndarray, V: np.ndarray) -> np.ndarray:
    """Rows of S^{-1}: the b quadratures as combinations of the a quadratures.
    From b = U^dag a - V^dag a^dag: x_b = Re(U - V)^T x + Im(U + V)^T p and
    p_b = Im(V - U)^T x + Re(U + V)^T p.  Returns (2n, 2n) in xxpp order."""
    top = np.concatenate([(U - V).real.T, (U + V).imag.T], axis=1)
    bot = np.concatenate([(V - U).imag.T, (U + V).real.T], axis=1)
    return np.concatenate([top, bot], axis=0)


def canonical_gauge(U: np.ndarray, V: np.ndarray):
    """Fix the free phase of every Bogoliubov mode b_q (b_q -> e^{i t} b_q
    multiplies column q of U and V by e^{-i t}): the largest-modulus entry of
    each column of U is made real positive (first row on exact ties)."""
    U = U.copy()
    V = V.copy()
    for q in range(U.shape[1]):
        j = int(np.argmax(np.abs(U[:, q])))
        ph = U[j, q] / abs(U[j, q])
        U[:, q] *= np.conj(ph)
        V[:, q] *= np.conj(ph)
    return U, V


def lambda2_from_d(D: np.ndarray) -> np.ndarray:
    """Eq. (SVD1): Lambda_q^2 = (D_q - 1)/(D_q + 1)."""
    return (D - 1.0) / (D + 1.0)


def entropy_q(lam2: np.ndarray) -> np.ndarray:
    """S_q = -log(1 - L^2) - L^2/(1 - L^2) log L^2 (Sec. II A)."""
    lam2 = np.asarray(lam2, dtype=np.float64)
    return -np.log1p(-lam2) - lam2 / (1 - lam2) * np.log(lam2)


def q_left(U: np.ndarray, V: np.ndarray, n_active: int) -> np.ndarray:
    """Regularised paired form of |phi_L> = prod_q exp(b_q^dag l_q^dag)|0>
    (App. A): Q_L = [[U^-dag V^dag, U^-dag], [U^-*, -V^T U^-dag]], restricted
    to the physical rows/columns and the first n_active l modes."""
    n = U.shape[0]
    Uid = np.linalg.inv(U.conj().T)
    top = np.concatenate([Uid @ V.conj().T, Uid], axis=1)
    bot = np.concatenate([np.linalg.inv(U.conj()), -V.T @ Uid], axis=1)
    Q = np.concatenate([top, bot], axis=0)
    keep = list(range(n)) + list(range(n, n + n_active))
    Q = Q[np.ix_(keep, keep)]
    return 0.5 * (Q + Q.T)


# --------------------------------------------------------------------------
# the iterative GSVD chain
# --------------------------------------------------------------------------
@dataclass
class Cut:
    """Record of GSVD step m (1-based site m, 0-based index m-1)."""
    n_in: int            # n_e^{m-1}: incoming virtual modes r_{m-1}
    n_out: int           # n_e^m: outgoing virtual modes l_m (0 at the last site)
    D: np.ndarray        # symplectic eigenvalues of L_m (descending)
    lam2: np.ndarray     # Lambda^2 of the n_out active modes
    Q: np.ndarray        # local paired form over c_m = (r_{m-1}, a_m, l_m)
    c: float             # |det U_L|^{-1/2} (scale of the paired form)
    S: np.ndarray | None = None
    U: np.ndarray | None = None
    V: np.ndarray | None = None


def gsvd_chain(gamma: np.ndarray, lambda2_freeze: float = 1e-13,
               ne_max: int = 64, keep_matrices: bool = False, route=None):
    """Iterative GSVD (Sec. II B): at step m the residual state lives on
    (r_{m-1}, a_m..a_N).  Its reduced covariance on L_m = (r_{m-1}, a_m) is
    Williamson-diagonalised; active modes (Lambda^2 > lambda2_freeze, the D*
    tolerance of Sec. II A) become the outgoing virtual modes; the local state
    |A^m> = prod exp(b^dag l^dag)|0> has the paired form Q^m of App. A.  The
    next residual is the state of (b_active, a_{m+1..N}) with b renamed r_m
    (Eqs. (SVD3)-(bond)), whose covariance is
        [[D_active/2, S^{-1}_active Gamma_{L,R}], [..., Gamma_RR]].
    The last step converts the pure residual on (r_{N-1}, a_N) to its paired
    form directly.  ``route`` selects the Williamson construction
    (``williamson`` by default, ``williamson_sqrt`` for the second route)."""
    route = williamson if route is None else route
    N = gamma.shape[0] // 2
    cuts = []
    n_in = 0
    Dprev = np.zeros(0)
    G = np.zeros((0, 2 * N))        # cov(r_{m-1}, a_m..a_N), columns x.. then p..
    for m in range(N):              # 0-based site index
        R = N - m                   # remaining physical modes a_m..a_{N-1}
        nL = n_in + 1
        # reduced covariance of L_m in xxpp order (r's then a_m)
        gl = np.zeros((2 * nL, 2 * nL))
        gl[np.arange(n_in), np.arange(n_in)] = 0.5 * Dprev
        gl[nL + np.arange(n_in), nL + np.arange(n_in)] = 0.5 * Dprev
        # r <-> a_m
        gx, gp = G[:, 0], G[:, R]
        gl[:n_in, n_in] = gx[:n_in]
        gl[nL:nL + n_in, n_in] = gx[n_in:]
        gl[:n_in, nL + n_in] = gp[:n_in]
        gl[nL:nL + n_in, nL + n_in] = gp[n_in:]
        gl[n_in, :] = gl[:, n_in]
        gl[nL + n_in, :] = gl[:, nL + n_in]
        gl[n_in, n_in] = gamma[m, m]
        gl[n_in, nL + n_in] = gamma[m, N + m]
        gl[nL + n_in, n_in] = gamma[N + m, m]
        gl[nL + n_in, nL + n_in] = gamma[N + m, N + m]
        if m == N - 1:
            Q = q_from_gamma(gl)
            cuts.append(Cut(n_in=n_in, n_out=0, D=np.ones(nL), lam2=np.zeros(0),
                            Q=Q, c=1.0))
            break
        D, S = route(gl)
        U, V = uv_from_s(S)
        U, V = canonical_gauge(U, V)
        lam2 = lambda2_from_d(D)
        n_out = int(np.sum(lam2 > lambda2_freeze))
        if n_out > ne_max:
            raise ValueError(f"n_e={n_out} exceeds ne_max={ne_max} at cut {m + 1}")
        Q = q_left(U, V, n_out)
        c = abs(np.linalg.det(U)) ** -0.5
        # cov(L_m, a_{m+1..N}): rows xxpp of L_m, columns x then p of the rest
        Rn = R - 1
        glr = np.zeros((2 * nL, 2 * Rn))
        glr[:n_in, :Rn] = G[:n_in, 1:R]
        glr[:n_in, Rn:] = G[:n_in, R + 1:]
        glr[nL:nL + n_in, :Rn] = G[n_in:, 1:R]
        glr[nL:nL + n_in, Rn:] = G[n_in:, R + 1:]
        glr[n_in, :Rn] = gamma[m, m + 1:N]
        glr[n_in, Rn:] = gamma[m, N + m + 1:]
        glr[nL + n_in, :Rn] = gamma[N + m, m + 1:N]
        glr[nL + n_in, Rn:] = gamma[N + m, N + m + 1:]
        sinv = sinv_rows_from_uv(U, V)
        act = list(range(n_out)) + list(range(nL, nL + n_out))
        G = sinv[act, :] @ glr
        cuts.append(Cut(n_in=n_in, n_out=n_out, D=D, lam2=lam2[:n_out], Q=Q, c=c,
                        S=S if keep_matrices else None,
                        U=U if keep_matrices else None,
                        V=V if keep_matrices else None))
        Dprev = D[:n_out]
        n_in = n_out
    return cuts
