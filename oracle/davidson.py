"""Davidson eigensolver as the paper states it (oracle; test infrastructure only).

Follows the "Results" section: the Ritz residual r = H C - E C is computed from the
sigma vector, preconditioned, and appended as the next expansion vector; ||r|| is the
convergence measure.  Preconditioners:
  * Eq. davidsonPreconditioner (traditional): t_i = r_i / (lambda - H_ii), or 0 when
    |lambda - H_ii| is small;
  * Eq. sparsePreconditioner (compression-compatible): s_i as above with the guard
    |lambda - H_ii| >= 1e-12, then t_i = s_i if |s_i| >= eps ||s||, else 0.
eps = 0 reduces the second to the first.

Readings where the paper gives no value: the guess is the unit vector on the lowest
diagonal element (lowest address on ties); one new vector per iteration; the subspace
is collapsed to the current and previous Ritz vectors when it reaches max_sub; the new
direction is orthogonalised twice by classical Gram-Schmidt and dropped as linearly
dependent when its norm falls below 1e-10; convergence is ||r|| <= tol_r and
|dE| <= tol_e.  The log holds the columns of the paper's Tables 1-3: energy, dE,
max|dC_i| and ||r||.
"""
from __future__ import annotations

import numpy as np


def precondition(r, lam, hdiag, eps=0.0, guard=1e-12):
    den = lam - hdiag
    s = np.where(np.abs(den) >= guard, r / np.where(den == 0, 1.0, den), 0.0)
    if eps > 0.0:
        ns = np.linalg.norm(s)
        s = np.where(np.abs(s) >= eps * ns, s, 0.0)
    return s


def _orth(t, V):
    for _ in range(2):
        for v in V:
            t = t - np.vdot(v, t) * v
    return t


def davidson(matvec, hdiag, guess=None, tol_r=1e-6, tol_e=1e-10, max_iter=200,
             max_sub=32, eps=0.0, e_shift=0.0):
    """Lowest eigenpair of the Hermitian operator `matvec`.  Returns (E, c, log, converged)."""
    n = len(hdiag)
    if guess is None:
        guess = np.zeros(n)
        guess[int(np.argmin(hdiag))] = 1.0
    v = guess / np.linalg.norm(guess)
    V = [v]
    S = [matvec(v)]
    log = []
    E_prev = None
    c_prev = None
    converged = False
    for it in range(max_iter):
        k = len(V)
        Hs = np.array([[np.vdot(V[i], S[j]) for j in range(k)] for i in range(k)])
        Hs = 0.5 * (Hs + Hs.conj().T)
        w, y = np.linalg.eigh(Hs)
        lam, y0 = w[0], y[:, 0]
        c = sum(y0[i] * V[i] for i in range(k))
        sc = sum(y0[i] * S[i] for i in range(k))
        if c_prev is not None:
            ph = np.vdot(c_prev, c)
            if abs(ph) > 0:
                c = c * (abs(ph) / ph)
                sc = sc * (abs(ph) / ph)
        r = sc - lam * c
        rn = float(np.linalg.norm(r))
        dE = None if E_prev is None else float(lam - E_prev)
        dC = None if c_prev is None else float(np.max(np.abs(c - c_prev)))
        log.append(dict(iteration=it + 1, energy=float(lam) + e_shift, dE=dE, max_dC=dC, rnorm=rn))
        if rn <= tol_r and dE is not None and abs(dE) <= tol_e:
            converged = True
            break
        t = precondition(r, lam, hdiag, eps=eps)
        if k >= max_sub:
            newV, newS = [c], [sc]
            if c_prev is not None:
                # previous Ritz vector, orthogonalised against the current one; its
                # sigma vector follows by linearity from the stored ones
                ov = np.vdot(c, c_prev)
                p = c_prev - ov * c
                pn = np.linalg.norm(p)
                if pn > 1e-10:
                    newV.append(p / pn)
                    newS.append((sc_prev - ov * sc) / pn)
            V, S = newV, newS
        t = _orth(t, V)
        tn = np.linalg.norm(t)
        E_prev, c_prev, sc_prev = lam, c, sc
        if tn < 1e-10:
            break
        t = t / tn
        V.append(t)
        S.append(matvec(t))
    return float(lam) + e_shift, c, log, converged
