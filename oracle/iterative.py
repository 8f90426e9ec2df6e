"""Iterative oracle (oracle-I) for lattices whose dense Z does not fit in memory.

It solves the ORIGINAL system Z I = V (Eq. 15) -- not the normal equations
used by the CUDA solver -- with textbook restarted GMRES (Saad and Schultz),
modified Gram-Schmidt Arnoldi and complex Givens rotations, all complex128.
The preconditioner is block Jacobi with the self block Z_0 (every diagonal
block of an MBT matrix is Z_0, Sec. II-A), applied on the right so that the
GMRES residual is the true residual V - Z I.  The product is the direct
offset sum of mbt.matvec, with no FFT.
"""
import numpy as np
import scipy.linalg

from . import mbt


def gmres(blocks, nx, ny, v, tol=1e-13, restart=60, max_iter=2000, callback=None):
    """Return (I, info) with I [nrhs][Ny][Nx][b] and info a list of per-RHS
    dicts {iters, rel_residual}."""
    v = np.asarray(v, dtype=np.complex128)
    b = v.shape[-1]
    lu0 = scipy.linalg.lu_factor(blocks[ny - 1, nx - 1].astype(np.complex128))

    def m_inv(u):
        sh = u.shape
        return scipy.linalg.lu_solve(lu0, u.reshape(-1, b).T).T.reshape(sh)

    def op(u):  # Z M^{-1} u for one RHS [Ny][Nx][b]
        return mbt.matvec(blocks, nx, ny, m_inv(u)[None])[0]

    out = np.zeros_like(v)
    infos = []
    for q in range(v.shape[0]):
        rhs = v[q]
        bnorm = np.linalg.norm(rhs)
        u = np.zeros_like(rhs)  # preconditioned unknown, I = M^{-1} u
        iters = 0
        r = rhs.copy()
        rel = 1.0
        while iters < max_iter:
            beta = np.linalg.norm(r)
            rel = beta / bnorm
            if rel <= tol:
                break
            basis = [r / beta]
            h = np.zeros((restart + 1, restart), dtype=np.complex128)
            cs = np.zeros(restart)
            sn = np.zeros(restart, dtype=np.complex128)
            g = np.zeros(restart + 1, dtype=np.complex128)
            g[0] = beta
            k = 0
            for k in range(restart):
                w = op(basis[k])
                for i in range(k + 1):  # modified Gram-Schmidt
                    h[i, k] = np.vdot(basis[i], w)
                    w = w - h[i, k] * basis[i]
                wnorm = np.linalg.norm(w)
                h[k + 1, k] = wnorm
                for i in range(k):  # previous rotations
                    t = cs[i] * h[i, k] + sn[i] * h[i + 1, k]
                    h[i + 1, k] = -np.conj(sn[i]) * h[i, k] + cs[i] * h[i + 1, k]
                    h[i, k] = t
                f, gg = h[k, k], h[k + 1, k]
                t = np.hypot(abs(f), abs(gg))
                if abs(f) == 0.0:
                    cs[k], sn[k] = 0.0, 1.0
                else:
                    cs[k] = abs(f) / t
                    sn[k] = (f / abs(f)) * np.conj(gg) / t
                h[k, k] = cs[k] * f + sn[k] * gg
                h[k + 1, k] = 0.0
                g[k + 1] = -np.conj(sn[k]) * g[k]
                g[k] = cs[k] * g[k]
                iters += 1
                if callback is not None:
                    callback(q, iters, abs(g[k + 1]) / bnorm)
                done = abs(g[k + 1]) / bnorm <= tol or iters >= max_iter
                if done or wnorm == 0.0:
                    k += 1
                    break
                basis.append(w / wnorm)
            else:
                k = restart
            y = scipy.linalg.solve_triangular(h[:k, :k], g[:k])
            for i in range(k):
                u = u + y[i] * basis[i]
            r = rhs - op(u)
        out[q] = m_inv(u)
        infos.append({"iters": iters, "rel_residual": float(np.linalg.norm(rhs - mbt.matvec(blocks, nx, ny, out[q][None])[0]) / bnorm)})
    return out, infos
