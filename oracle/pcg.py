"""Preconditioned conjugate gradients on the approximate normal equation (Section 4.1).

Test infrastructure only: nothing on the product path imports this module.

Eq. 4.3:  K~^* K~ f = K~^* u, an HPD system, solved by CG preconditioned with
the ULV factorization F~ = G~^{-1} of the HSS approximation (Algorithm 1's
output used as a preconditioner, Section 4.1).  The iteration is the standard
preconditioned Hestenes-Stiefel recurrence, run independently for every
column of the right-hand side, started from f_0 = 0 and stopped when
||b - A f_k||_2 <= tol ||b||_2 (the relative residual of Section 5, where the
paper uses tol = 1e-12), with b = K~^* u:

    r_0 = b, z_0 = M r_0, p_0 = z_0
    alpha_k = <r_k, z_k> / <p_k, A p_k>
    f_{k+1} = f_k + alpha_k p_k,  r_{k+1} = r_k - alpha_k A p_k
    z_{k+1} = M r_{k+1},  beta_k = <r_{k+1}, z_{k+1}> / <r_k, z_k>
    p_{k+1} = z_{k+1} + beta_k p_k

<a, b> = a^* b.  M = I gives plain CG.
"""
import numpy as np


def pcg(apply_A, b, apply_M=None, tol=1e-12, maxit=500):
    """Solve A x = b (A HPD, columns independent).  Returns (x, iters, relres):
    iters[j] = iterations column j took, relres[j] = ||b_j - A x_j|| / ||b_j||
    (the recurrence residual, as CG monitors it)."""
    b = np.asarray(b, dtype=np.complex128)
    if b.ndim == 1:
        b = b[:, None]
    n, k = b.shape
    M = apply_M if apply_M is not None else (lambda v: v)
    x = np.zeros_like(b)
    iters = np.zeros(k, dtype=int)
    relres = np.zeros(k)
    for j in range(k):
        bj = b[:, j:j + 1]
        nb = np.linalg.norm(bj)
        if nb == 0.0:
            continue
        xj = np.zeros_like(bj)
        r = bj.copy()
        z = M(r)
        p = z.copy()
        rz = np.vdot(r, z)
        it = 0
        while np.linalg.norm(r) > tol * nb and it < maxit:
            q = apply_A(p)
            alpha = rz / np.vdot(p, q)
            xj = xj + alpha * p
            r = r - alpha * q
            it += 1
            if np.linalg.norm(r) <= tol * nb:
                break
            z = M(r)
            rz_new = np.vdot(r, z)
            p = z + (rz_new / rz) * p
            rz = rz_new
        x[:, j:j + 1] = xj
        iters[j] = it
        relres[j] = np.linalg.norm(r) / nb
    return x, iters, relres


def fio_pcg(solver, u, tol=1e-12, maxit=500, precondition=True):
    """PCG on Eq. 4.3 with the FIOSolver's BF and, when precondition is set, its ULV
    factorization as the preconditioner (Section 4.1)."""
    A = lambda v: solver.bf.adjoint(solver.bf.apply(v))
    M = solver.ulv.solve if precondition else None
    return pcg(A, solver.bf.adjoint(np.asarray(u, dtype=np.complex128).reshape(solver.bf.n, -1)), M, tol, maxit)
