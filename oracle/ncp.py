"""Coulomb-cone NCP with the De Saxce correction and its ADMM solve (oracle).  Test infrastructure.

Eq. 1: K_mu  contains lambda  perp  sigma + Gamma_mu(sigma) in K_mu^*,  sigma = G lambda + g, with
K_mu = {||l_T|| <= mu l_N} per contact, K_mu^* = K_{1/mu} and Gamma_mu(sigma) = [0, 0, mu ||sigma_T||].
Eq. 4: G = J_c M^-1 J_c^T (Delassus), g = J_c (v + dt vdot_f) (free contact velocity); lambda is an
impulse (the reading under which Eq. 4 holds).

The paper names ADMM as its solver (Sec. 2.2) without stating the iteration.  The iteration used
here is the standard one for this problem: an x-step that minimises
1/2 x^T G x + (g + s)^T x + y^T (x - z) + rho/2 ||x - z||^2 with s the De Saxce term at the current
z, a z-step that projects onto K_mu, and a dual ascent step on y.  At a fixed point x = z = lambda
and y = -(sigma + Gamma(sigma)), and lambda = Proj_K(lambda - (sigma + Gamma)/rho), which by Moreau's
decomposition is exactly Eq. 1.  It is followed by Newton steps on the equations of the identified
contact modes (Sec. 3.2, App. A).
"""
import numpy as np

from .rigid import cholesky, chol_solve

BRK, STK, SLD = 0, 1, 2


def desaxce(sigma, mu):
    """Gamma_mu(sigma) per contact: [0, 0, mu_i ||sigma_T,i||]."""
    out = np.zeros_like(sigma)
    for i in range(len(mu)):
        st = sigma[3 * i:3 * i + 2]
        out[3 * i + 2] = mu[i] * np.sqrt(st @ st)
    return out


def proj_cone(x, mu):
    """Euclidean projection onto the second-order cone {||x_T|| <= mu x_N}."""
    xt, xn = x[:2], x[2]
    nt = np.sqrt(xt @ xt)
    if nt <= mu * xn:
        return x.copy()
    if mu * nt <= -xn:
        return np.zeros(3)
    a = (mu * nt + xn) / (1.0 + mu * mu)
    return np.concatenate([mu * a * xt / nt, [a]])


def proj_K(x, mu):
    return np.concatenate([proj_cone(x[3 * i:3 * i + 3], mu[i]) for i in range(len(mu))]) if len(mu) else x.copy()


def admm_rho(G):
    """Penalty parameter: mean diagonal of G (scale of the Delassus operator)."""
    m = G.shape[0]
    return max(np.trace(G) / m, 1e-12)


def admm(G, g, mu, eps=1e-12, max_iter=20000, rho=None, lam0=None):
    """ADMM iteration for Eq. 1 (reading stated in the module docstring; the De Saxce term is taken
    at the most recent primal iterate x).  Stops when ||x - z||_inf <= eps max(1, ||z||_inf) and
    rho ||z - z_prev||_inf <= eps max(1, ||g||_inf).  Returns (lambda, iterations, converged)."""
    m = len(g)
    if m == 0:
        return np.zeros(0), 0, True
    if rho is None:
        rho = admm_rho(G)
    L = cholesky(G + rho * np.eye(m))
    z = np.zeros(m) if lam0 is None else lam0.copy()
    x = z.copy()
    y = np.zeros(m)
    gs = max(1.0, np.max(np.abs(g)))
    for k in range(1, max_iter + 1):
        s = desaxce(G @ x + g, mu)
        x = chol_solve(L, rho * z - y - g - s)
        z_prev = z
        z = proj_K(x + y / rho, mu)
        y = y + rho * (x - z)
        rp = np.max(np.abs(x - z))
        rd = rho * np.max(np.abs(z - z_prev))
        if rp <= eps * max(1.0, np.max(np.abs(z))) and rd <= eps * gs:
            return z, k, True
    return z, max_iter, False


def solve_ncp(G, g, mu, eps_sigma=1e-8, eps_lambda=1e-8, tol=1e-12, stages=(1e-4, 1e-6, 1e-9, 1e-12),
              max_iter=50000):
    """Staged solve of Eq. 1: ADMM to a loose tolerance, identification of the contact modes,
    Newton on the mode equations, and acceptance when the NCP residual is <= tol max(1, ||g||);
    otherwise ADMM continues from scratch to the next, tighter tolerance.
    Returns (lambda, admm_iterations, converged)."""
    m = len(g)
    if m == 0:
        return np.zeros(0), 0, True
    scale = max(1.0, np.max(np.abs(g)))
    best, best_r, total = None, np.inf, 0
    for eps in stages:
        lam, it, _ = admm(G, g, mu, eps=eps, max_iter=max_iter)
        total += it
        modes, _ = classify(G, g, mu, lam, max(eps_sigma, 10 * eps), max(eps_lambda, 10 * eps))
        lp = polish(G, g, mu, lam, modes)
        for cand in (lp, lam):
            r = ncp_residual(G, g, mu, cand)
            if r < best_r:
                best, best_r = cand, r
        if best_r <= tol * scale:
            return best, total, True
    return best, total, False


def ncp_residual(G, g, mu, lam):
    """max over contacts of dist(lambda_i, K_mu), dist(sigma_i + Gamma_i, K_mu^*) and
    |lambda_i . (sigma_i + Gamma_i)|  (the three conditions of Eq. 1)."""
    if len(g) == 0:
        return 0.0
    sigma = G @ lam + g
    w = sigma + desaxce(sigma, mu)
    r = 0.0
    for i in range(len(mu)):
        li, wi = lam[3 * i:3 * i + 3], w[3 * i:3 * i + 3]
        r = max(r, np.linalg.norm(li - proj_cone(li, mu[i])),
                np.linalg.norm(wi - proj_cone(wi, 1.0 / mu[i])), abs(li @ wi))
    return r


def thresholds(g, lam, eps_sigma, eps_lambda):
    es = eps_sigma * max(1.0, np.max(np.abs(g))) if len(g) else eps_sigma
    el = eps_lambda * max(1.0, np.max(np.abs(lam))) if len(lam) else eps_lambda
    return es, el


def classify(G, g, mu, lam, eps_sigma=1e-8, eps_lambda=1e-8):
    """Contact modes (Sec. 3.2): sticking if ||sigma_i|| <= eps_s; else breaking if sigma_N > eps_s
    or lambda_N <= eps_l; else sliding.  Returns (modes, margin) where margin is the smallest
    relative distance of the deciding quantities to the boundary of the identified mode."""
    sigma = G @ lam + g
    es, el = thresholds(g, lam, eps_sigma, eps_lambda)
    ss = max(1.0, np.max(np.abs(g))) if len(g) else 1.0
    sl = max(1.0, np.max(np.abs(lam))) if len(lam) else 1.0
    modes, margin = [], np.inf
    for i in range(len(mu)):
        s, l = sigma[3 * i:3 * i + 3], lam[3 * i:3 * i + 3]
        ns = np.linalg.norm(s)
        nst = np.linalg.norm(s[:2])
        if ns <= es:
            modes.append(STK)
            margin = min(margin, (es - ns) / es)
        elif s[2] > es or l[2] <= el:
            modes.append(BRK)
            margin = min(margin, (s[2] - es) / ss if s[2] > es else 0.0)
        else:
            modes.append(SLD)
            margin = min(margin, nst / ss, l[2] / sl)
    return np.array(modes, dtype=np.int32), margin


def mode_equations(lam, G, g, mu, modes):
    """Stacked equations of the identified modes at sigma = G lambda + g."""
    return mode_residual(lam, G @ lam + g, mu, modes)


def mode_residual(lam, sigma, mu, modes):
    """Stacked equations of the identified modes (Sec. 3.2, App. A): breaking lambda_i = 0;
    sticking sigma_i = 0; sliding sigma_N = 0 and lambda_T + mu lambda_N sigma_T/||sigma_T|| = 0."""
    out = []
    for i, md in enumerate(modes):
        l, s = lam[3 * i:3 * i + 3], sigma[3 * i:3 * i + 3]
        if md == BRK:
            out.append(l)
        elif md == STK:
            out.append(s)
        else:
            st = s[:2]
            out.append(np.concatenate([l[:2] + mu[i] * l[2] * st / np.sqrt(st @ st), [s[2]]]))
    return np.concatenate(out) if out else np.zeros(0)


def cs_jacobian(f, x, h=1e-30):
    """Complex-step Jacobian of f at x."""
    cols = []
    for j in range(len(x)):
        xp = np.array(x, dtype=complex)
        xp[j] += 1j * h
        cols.append(np.imag(f(xp)) / h)
    return np.stack(cols, axis=1)


def polish(G, g, mu, lam, modes, iters=20, tol=1e-15):
    """Newton on the mode equations with minimum-norm steps (the system is singular when the
    contact set is redundant).  Returns the polished lambda, or the input if it does not improve
    the NCP residual."""
    if len(g) == 0:
        return lam
    x = lam.copy()
    scale = max(1.0, np.max(np.abs(g)))
    for _ in range(iters):
        F = mode_equations(x, G, g, mu, modes)
        if np.max(np.abs(F)) <= tol * scale:
            break
        J = cs_jacobian(lambda z: mode_equations(z, G, g, mu, modes), x)
        x = x - np.linalg.lstsq(J, F, rcond=1e-13)[0]
    if ncp_residual(G, g, mu, x) <= ncp_residual(G, g, mu, lam):
        return x
    return lam


def brute_force_single(G, g, mu, n_angles=720):
    """All solutions of Eq. 1 for ONE contact by enumerating its three modes: breaking (lambda = 0
    needs g_N >= 0), sticking (lambda = -G^-1 g inside the cone) and sliding (lambda on the cone
    boundary opposite to sigma_T with sigma_N = 0: 2-D Newton on (lambda_N, angle) from a grid of
    starting angles).  Returns a list of (mode, lambda)."""
    sols = []
    if g[2] >= 0:
        sols.append((BRK, np.zeros(3)))
    lam = -np.linalg.solve(G, g)
    if np.linalg.norm(lam[:2]) <= mu * lam[2] + 1e-14:
        sols.append((STK, lam))

    def lam_of(ln, th):
        return np.array([-mu * ln * np.cos(th), -mu * ln * np.sin(th), ln])

    def res(p):
        ln, th = p
        s = G @ lam_of(ln, th) + g
        return np.array([s[2], -np.sin(th) * s[0] + np.cos(th) * s[1]])

    for th0 in np.linspace(0, 2 * np.pi, n_angles, endpoint=False):
        u = np.array([np.cos(th0), np.sin(th0)])
        a = G[2] @ np.array([-mu * u[0], -mu * u[1], 1.0])
        if abs(a) < 1e-14:
            continue
        p = np.array([-g[2] / a, th0])
        for _ in range(40):
            r = res(p)
            J = np.zeros((2, 2))
            for j in range(2):
                dp = np.zeros(2)
                dp[j] = 1e-30
                J[:, j] = np.imag(np.array(res(p + 1j * dp))) / 1e-30
            try:
                p = p - np.linalg.solve(J, r)
            except np.linalg.LinAlgError:
                break
        if np.max(np.abs(res(p))) < 1e-13 and p[0] > 0:
            l = lam_of(*p)
            s = G @ l + g
            if s[0] * np.cos(p[1]) + s[1] * np.sin(p[1]) > 1e-12:
                if not any(np.allclose(l, o, atol=1e-9) for _, o in sols):
                    sols.append((SLD, l))
    return sols
