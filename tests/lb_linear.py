"""Linearised Fourier step of the D3Q19 update about the rest state, for pins
of the oracle and of the GPU path (test helper, not collected).

About rho = rho0, u = 0 the quadratic equilibrium moments m^eq_k (k >= 4)
vanish to first order, so the MRT collision of Sec. 3.4 (Eq. lco_update)
acts on a population perturbation as the linear map

    C = B diag(g) E,   E_ki = e_ki (Table 1),  B_ik = a_i e_ki / w_k
    g = (1, 1, 1, 1, gamma_b, gamma_s x 5, gamma_odd x 6, gamma_even x 3)

(conserved modes unchanged), and the pull streaming n_i(r, t+1) =
n*_i(r - c_i) multiplies the Fourier amplitude of population i at wave
vector k by exp(-i k.c_i).  The pre-collision state p(t) (streamed, before
the collision of that step) then evolves as p(t+1) = M p(t) + S xi(t) with

    M(k) = S(k) C,   S(k) = diag(exp(-i k.c_i)).

Sec. 3.4 (Eq. shearviscosity) ties the shear eigenvalue to the viscosity;
for k along z the two transverse momenta (u_x, u_y) decay with the real
eigenvalue lambda(k) of M, which tends to exp(-nu k^2) for small k.

Sec. 3.6: in equilibrium the population fluctuations are independent with
variance mu rho0 a_i per node (mu = kT / c_s^2 = 3 kT), so the Fourier
amplitude p^(k) = (1/V) sum_r p(r) e^{-i k.r} has covariance
Sigma_eq = (mu rho0 / V) diag(a), stationary under M.  From the rest state
(no fluctuation) the covariance after t steps is
Sigma(t) = Sigma_eq - M^t Sigma_eq (M^t)^H, and the transverse velocity
mode u^(k) = e . p^(k), e_i = c_ix / rho0 (linear order), has

    < Re u^(t0 + tau) conj(u^(t0)) > = Re( e^T M^tau Sigma(t0) e ),

which equals kT / (rho0 V) at tau = 0 in equilibrium.
"""
import numpy as np


def collision_matrix(tables, gamma_bulk=0.0, gamma_shear=0.0, gamma_odd=0.0, gamma_even=0.0):
    c, a, e, w, opp = tables
    g = np.array([1.0] * 4 + [gamma_bulk] + [gamma_shear] * 5 + [gamma_odd] * 6 + [gamma_even] * 3)
    B = a[:, None] * e.T / w[None, :]
    return B @ np.diag(g) @ e


def step_matrix(k, tables, **gammas):
    c = tables[0]
    S = np.diag(np.exp(-1j * (c @ np.asarray(k, dtype=np.float64))))
    return S @ collision_matrix(tables, **gammas)


def shear_eigenvalue(L, tables, **gammas):
    """The eigenvalue of M(2 pi / L z^) whose eigenvector carries the
    transverse momentum j_x (the largest share of it)."""
    c, a = tables[0], tables[1]
    M = step_matrix((0.0, 0.0, 2.0 * np.pi / L), tables, **gammas)
    lam, V = np.linalg.eig(M)
    ex = c[:, 0].astype(np.float64)
    share = np.abs(ex @ V) / np.linalg.norm(V, axis=0)
    return lam[int(np.argmax(share))]


def transverse_acf(L, tables, kT, rho0, V, taus, t_begin, t_end, **gammas):
    """Expected estimator of the transverse velocity autocorrelation for the
    mode u_x(k = 2 pi / L z^) of a run started from rest: for each tau, the
    mean over t0 in [t_begin, t_end - tau) of Re(e^T M^tau Sigma(t0) e)."""
    c, a = tables[0], tables[1]
    M = step_matrix((0.0, 0.0, 2.0 * np.pi / L), tables, **gammas)
    e = c[:, 0].astype(np.float64) / rho0
    Seq = (3.0 * kT * rho0 / V) * np.diag(a).astype(np.complex128)
    y = Seq @ e
    # Sigma(t0) e for every t0 < t_end
    se = np.empty((t_end, len(e)), dtype=np.complex128)
    P = np.eye(len(e), dtype=np.complex128)
    for t0 in range(t_end):
        se[t0] = y - P @ (Seq @ (P.conj().T @ e))
        P = M @ P
    out = []
    for tau in taus:
        r = e.astype(np.complex128)
        for _ in range(tau):
            r = r @ M
        t0 = np.arange(t_begin, t_end - tau)
        out.append(float(np.mean((se[t0] @ r).real)))
    return np.array(out)
