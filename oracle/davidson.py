"""Plain Davidson eigensolver for the lowest eigenpair (oracle side).

Appendix A (solving step, Eq. eff-eigsh) names the Davidson method without
details; this is the textbook algorithm (E. R. Davidson, J. Comput. Phys.
17, 87 (1975)) with the following fixed choices:
  * subspace of at most max_space orthonormal vectors; when full, restart
    from the two lowest Ritz vectors;
  * Ritz pair from the projected matrix V^T H V (dense symmetric eigensolver);
  * residual r = H x - theta x, converged when ||r||_2^2 < tol;
  * diagonal preconditioner: t_i = r_i / (theta - d_i), where a denominator
    of magnitude below 1e-8 is replaced by +-1e-8 (sign of the denominator,
    + for zero);
  * new direction orthogonalised twice (classical Gram-Schmidt) against the
    subspace and normalised; directions of norm below 1e-14 end the run;
  * at most max_iter matrix-vector products.

Parity status: pinned (tests/test_oracle_davidson.py) against dense eigh on
random symmetric matrices and through DMRG at full M = FCI.
"""

import numpy as np


def davidson(matvec, diag, x0, tol=1e-10, max_space=24, max_iter=200):
    """Returns (theta, x, n_matvec, converged)."""
    x = np.asarray(x0, dtype=np.float64)
    x = x / np.linalg.norm(x)
    V = [x]
    AV = [matvec(x)]
    nmv = 1
    theta = float(x @ AV[0])
    while True:
        Vm = np.array(V)
        AVm = np.array(AV)
        Hs = Vm @ AVm.T
        Hs = 0.5 * (Hs + Hs.T)
        w, Y = np.linalg.eigh(Hs)
        theta = float(w[0])
        y = Y[:, 0]
        x = y @ Vm
        Ax = y @ AVm
        r = Ax - theta * x
        rr = float(r @ r)
        if rr < tol or nmv >= max_iter:
            return theta, x, nmv, rr < tol
        den = theta - diag
        small = np.abs(den) < 1e-8
        den = np.where(small, np.where(den < 0, -1e-8, 1e-8), den)
        t = r / den
        if len(V) >= max_space:
            # thick restart from the two lowest Ritz vectors (orthonormal
            # because V is orthonormal and Y is orthogonal)
            x2 = Y[:, 1] @ Vm
            Ax2 = Y[:, 1] @ AVm
            V, AV = [x, x2], [Ax, Ax2]
        Vm = np.array(V)
        for _ in range(2):  # classical Gram-Schmidt, twice
            t = t - (Vm @ t) @ Vm
        nt = np.linalg.norm(t)
        if nt < 1e-14:
            return theta, x, nmv, rr < tol
        t = t / nt
        V.append(t)
        AV.append(matvec(t))
        nmv += 1
