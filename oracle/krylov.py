"""Plain float64 GMRES around the iHDG sweep.  TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper (Section 4.2, closing remark; Section 6) proposes using the iHDG iteration as a
fine-scale preconditioner inside a Krylov method such as GMRES when the plain iteration does
not converge (diffusion-dominated problems on fine meshes).  It gives no algorithm.  The
reading taken here (R23): one iHDG sweep is the affine map u -> G u + c of Algorithm 1, and
its fixed point solves (I - G) u = c, the HDG system preconditioned by the iHDG splitting.
GMRES is applied to that system; each iteration costs one homogeneous sweep (zero source,
zero boundary data), which gives G v.

GMRES itself is the restarted method of Saad and Schultz (SIAM J. Sci. Stat. Comput. 7,
1986): Arnoldi with modified Gram-Schmidt, the Hessenberg least-squares problem reduced by
Givens rotations, and restart after m steps.  The iterate after j steps of a cycle minimises
||b - A x||_2 over x0 + K_j(A, r0).  Stopping test: ||b - A x_j||_2 <= tol ||b - A x_0||_2
measured at the start of the solve (x_0 = 0 gives ||b||).
"""
import numpy as np

from .ihdg import STATUS_DIVERGED, STATUS_NOT_CONVERGED, STATUS_OK


def gmres(apply_A, b, tol, restart, max_iters, x0=None):
    """Restarted GMRES(m).  Returns (x, iterations, status, history).

    `history[k]` is the residual norm after k iterations (history[0] = ||b - A x0||), taken
    from the Givens-reduced least-squares problem; the solve stops after the first
    iteration whose residual is <= tol * history[0].
    """
    b = np.asarray(b, dtype=np.float64)
    n = b.size
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    r = b - apply_A(x)
    beta = np.linalg.norm(r)
    hist = [beta]
    target = tol * beta
    if beta <= target or beta == 0.0:
        return x, 0, STATUS_OK, np.array(hist)
    its = 0
    while True:
        m = restart
        V = np.zeros((m + 1, n))
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        j_done = 0
        stop = None
        for j in range(m):
            # Arnoldi step: w = A v_j, orthogonalised against v_0..v_j one at a time
            w = apply_A(V[j])
            for i in range(j + 1):
                H[i, j] = V[i] @ w
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] > 0.0:
                V[j + 1] = w / H[j + 1, j]
            # earlier rotations applied to the new column, then the rotation that zeroes
            # its subdiagonal entry
            for i in range(j):
                a, c = H[i, j], H[i + 1, j]
                H[i, j] = cs[i] * a + sn[i] * c
                H[i + 1, j] = -sn[i] * a + cs[i] * c
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j] = H[j, j] / den if den > 0.0 else 1.0
            sn[j] = H[j + 1, j] / den if den > 0.0 else 0.0
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            its += 1
            j_done = j + 1
            res = abs(g[j + 1])
            hist.append(res)
            if not np.isfinite(res):
                stop = STATUS_DIVERGED
                break
            if res <= target:
                stop = STATUS_OK
                break
            if its >= max_iters:
                stop = STATUS_NOT_CONVERGED
                break
        # x <- x + V_j y with y solving the upper-triangular system R y = g
        y = np.zeros(j_done)
        for i in range(j_done - 1, -1, -1):
            y[i] = (g[i] - H[i, i + 1:j_done] @ y[i + 1:]) / H[i, i]
        x = x + V[:j_done].T @ y
        if stop is not None:
            return x, its, stop, np.array(hist)
        r = b - apply_A(x)
        beta = np.linalg.norm(r)
        if beta <= target:
            return x, its, STATUS_OK, np.array(hist)


def ihdg_gmres(problem, f_qp, g_qp, tol, restart=30, max_iters=2000, U_prev=None):
    """GMRES on (I - G) u = c, where u -> G u + c is one sweep of Algorithm 1 (reading R23).

    c is the sweep of the zero state with the problem's data; G v is the sweep of v with zero
    source and zero boundary data (every sweep is affine in (u, f, g)).  Returns
    (U, T, iterations, status, history) with U in the oracle's (nel, nc, nb) layout and T the
    trace of U.
    """
    shape = (problem.mesh.nel, problem.nc, problem.disc.nb)
    f0 = np.zeros_like(f_qp)
    g0 = np.zeros_like(g_qp)
    Uprev0 = None if U_prev is None else np.zeros_like(U_prev)
    c = problem.sweep(np.zeros(shape), f_qp, g_qp, U_prev).ravel()

    def apply_A(v):
        return v - problem.sweep(v.reshape(shape), f0, g0, Uprev0).ravel()

    x, its, status, hist = gmres(apply_A, c, tol, restart, max_iters)
    U = x.reshape(shape)
    return U, problem.traces(U, g_qp), its, status, hist
