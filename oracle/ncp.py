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
contact modes (Sec. 3.2, App. A).  A projected Gauss-Seidel solve (pgs), the other solver family
the paper cites, has the same fixed points; solve_ncp can take either one as its iteration, which
gives the tests two independent routes to a solution of Eq. 1.  A third route updates the ADMM
penalty on the way (residual balancing, balance_rho): the adaptive-penalty variant of the same
iteration, whose fixed points are again those of Eq. 1.

The iteration's parameters are the plain textbook choices (penalty rho = the mean diagonal of G,
no over-relaxation, stopping test on every iteration).  Eq. 1 can have several solutions (redundant
contacts; and Coulomb friction's non-monotone De Saxce form); where the free motion already
separates every active contact (g_N >= 0 for all of them) lambda = 0 is one of them, and it is the
one taken: no impulse acts when nothing pushes into the plane.
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


RHO_SCALE = 1.0      # rho = RHO_SCALE * mean diagonal of G
RELAX = 1.0          # relaxation of the x-step (1: none)
CHECK_EVERY = 1      # the stopping test runs on every CHECK_EVERY-th iteration
ADAPT_EVERY = 32     # route "admm_adaptive": iterations between penalty updates
ADAPT_RATIO = 10.0   # residual imbalance that changes the penalty
ADAPT_FACTOR = 2.0   # the penalty is multiplied or divided by this


def admm_rho(G):
    """Penalty parameter: RHO_SCALE x the mean diagonal of G (the scale of the Delassus operator)."""
    m = G.shape[0]
    return max(RHO_SCALE * np.trace(G) / m, 1e-12)


class AdmmState:
    def __init__(self, m, g):
        self.x = np.zeros(m)
        self.z = np.zeros(m)
        self.y = np.zeros(m)
        self.sx = np.array(g, dtype=float)     # G x + g at the current x
        self.iters = 0
        self.rho = None                        # the penalty (set on the first call)


def admm_residuals(x, z, y, sx, mu):
    """Primal and dual residuals of the ADMM iterate for the penalty update: ||x - z||_inf, and
    ||y + sigma + Gamma(sigma)||_inf at sigma = G x + g, which vanishes at a fixed point (there
    y = -(sigma + Gamma(sigma)), module docstring)."""
    return float(np.max(np.abs(x - z))), float(np.max(np.abs(y + sx + desaxce(sx, mu))))


def balance_rho(rho, r_primal, r_dual):
    """Residual balancing (Boyd et al., Distributed optimization and statistical learning via ADMM,
    2011, Sec. 3.4.1): a primal residual ADAPT_RATIO times the dual one raises the penalty by
    ADAPT_FACTOR, the reverse lowers it; otherwise it is kept.  y is the unscaled multiplier, so it
    needs no rescaling, and the fixed points do not depend on rho."""
    if r_primal > ADAPT_RATIO * r_dual:
        return rho * ADAPT_FACTOR
    if r_dual > ADAPT_RATIO * r_primal:
        return rho / ADAPT_FACTOR
    return rho


def admm(G, g, mu, eps=1e-12, max_iter=20000, state=None, adapt=False):
    """ADMM iteration for Eq. 1 (reading stated in the module docstring): the De Saxce term is taken
    at the most recent primal iterate x; with RELAX != 1 the x-step is relaxed,
    xh = RELAX x + (1 - RELAX) z, before the z-step and the dual step (the fixed points are
    unchanged).  G x is not recomputed: (G + rho I) x = rhs gives G x = rhs - rho x.  Stops when
    ||x - z||_inf <= eps max(1, ||z||_inf) and rho ||z - z_prev||_inf <= eps max(1, ||g||_inf), or
    when the state has done max_iter iterations in total; the test is evaluated when the cumulative
    iteration count is a multiple of CHECK_EVERY.  Continues from ``state`` when given.  With
    ``adapt`` the penalty is updated by balance_rho after every ADAPT_EVERY-th iteration (counted
    over the state's life) that did not stop the iteration, and G + rho I is factored again when it
    changes.  Returns (lambda, iterations, converged, state)."""
    m = len(g)
    st = state or AdmmState(m, g)
    if m == 0:
        return np.zeros(0), 0, True, st
    if st.rho is None:
        st.rho = admm_rho(G)
    rho = st.rho
    L = cholesky(G + rho * np.eye(m))
    gs = max(1.0, np.max(np.abs(g)))
    x, z, y, sx = st.x, st.z, st.y, st.sx
    conv = False
    while st.iters < max_iter:
        st.iters += 1
        rhs = rho * z - y - g - desaxce(sx, mu)
        x = chol_solve(L, rhs)
        sx = rhs - rho * x + g
        xh = RELAX * x + (1.0 - RELAX) * z
        z_prev = z
        z = proj_K(xh + y / rho, mu)
        y = y + rho * (xh - z)
        if st.iters % CHECK_EVERY:
            continue
        rp = np.max(np.abs(x - z))
        rd = rho * np.max(np.abs(z - z_prev))
        if rp <= eps * max(1.0, np.max(np.abs(z))) and rd <= eps * gs:
            conv = True
            break
        if adapt and st.iters % ADAPT_EVERY == 0:
            new = balance_rho(rho, *admm_residuals(x, z, y, sx, mu))
            if new != rho:
                rho = new
                L = cholesky(G + rho * np.eye(m))
    st.x, st.z, st.y, st.sx, st.rho = x, z, y, sx, rho
    return z.copy(), st.iters, conv, st


def pgs(G, g, mu, eps=1e-12, max_iter=20000, lam0=None):
    """Projected Gauss-Seidel on Eq. 1, the solver family the paper cites next to ADMM (Sec. 2.2):
    sweeps over the contacts in order; contact i takes the fixed-point step of Eq. 1 restricted to
    its own block, lambda_i <- Proj_K(lambda_i - (sigma_i + Gamma_i(sigma_i)) / r_i), with sigma
    = G lambda + g at the current (partly updated) lambda and r_i the largest eigenvalue of the 3x3
    diagonal block G_ii (the step that makes the local map non-expansive).  Its fixed points are
    Eq. 1 by Moreau's decomposition, as for the ADMM iteration.  Stops when a sweep moves lambda by
    at most eps max(1, ||lambda||_inf), or after max_iter sweeps.  Returns (lambda, sweeps,
    converged)."""
    m = len(g)
    nc = len(mu)
    lam = np.zeros(m) if lam0 is None else np.array(lam0, dtype=float)
    if m == 0:
        return lam, 0, True
    r = [max(np.linalg.eigvalsh(G[3 * i:3 * i + 3, 3 * i:3 * i + 3]).max(), 1e-300) for i in range(nc)]
    for it in range(1, max_iter + 1):
        delta = 0.0
        for i in range(nc):
            b = slice(3 * i, 3 * i + 3)
            si = G[b] @ lam + g[b]
            wi = si + np.array([0.0, 0.0, mu[i] * np.sqrt(si[:2] @ si[:2])])
            new = proj_cone(lam[b] - wi / r[i], mu[i])
            delta = max(delta, np.max(np.abs(new - lam[b])))
            lam[b] = new
        if delta <= eps * max(1.0, np.max(np.abs(lam))):
            return lam, it, True
    return lam, max_iter, False


def reclassify(G, g, mu, lam, modes, es, el, delta):
    """Active-set update after a Newton polish that did not give an NCP solution: a breaking
    contact that penetrates becomes sticking; a sticking or sliding contact that pulls
    (lambda_N < 0) becomes breaking; a sticking contact whose impulse leaves the cone becomes
    sliding; a sliding contact that stops (||sigma_T|| below threshold) becomes sticking."""
    sig = G @ lam + g
    new = np.array(modes).copy()
    for i, md in enumerate(modes):
        l, s = lam[3 * i:3 * i + 3], sig[3 * i:3 * i + 3]
        if md == BRK:
            if s[2] < -es:
                new[i] = STK
        elif md == STK:
            if l[2] < -el:
                new[i] = BRK
            elif mu[i] * l[2] - np.sqrt(l[:2] @ l[:2]) < -delta:
                new[i] = SLD
        else:
            if l[2] < -el:
                new[i] = BRK
            elif np.sqrt(s[:2] @ s[:2]) < es:
                new[i] = STK
    return new


def separating(g):
    """True when the free motion separates every active contact (g_N >= 0 for all): lambda = 0 then
    satisfies Eq. 1 (sigma = g, and g + Gamma(g) = (g_T, g_N + mu ||g_T||) lies in the dual cone
    exactly when g_N >= 0)."""
    return len(g) > 0 and bool(np.all(np.asarray(g)[2::3] >= 0.0))


def solve_ncp(G, g, mu, eps_sigma=1e-8, eps_lambda=1e-8, tol=1e-12, stages=(1e-4, 1e-6, 1e-9, 1e-12),
              rounds=4, max_iter=50000, route="admm"):
    """Staged solve of Eq. 1.  When the free motion separates every contact the solution with no
    impulse is returned (module docstring).  Otherwise each stage continues the iteration of the
    route ("admm"; "admm_adaptive": the same with the penalty updated by residual balancing; or
    "pgs": projected Gauss-Seidel sweeps) to a tolerance, identifies the contact
    modes, and runs up to ``rounds`` active-set rounds of Newton on the mode equations (reclassify +
    retry from the cone projection of the last iterate).  The first candidate whose NCP residual is
    <= tol max(1, ||g||_inf) is accepted.  Returns (lambda, iterations, converged)."""
    m = len(g)
    if m == 0:
        return np.zeros(0), 0, True
    if separating(g):
        return np.zeros(m), 0, True
    scale = max(1.0, np.max(np.abs(g)))
    best, best_r = None, np.inf
    state, lam, iters = None, None, 0
    for eps in stages:
        if route in ("admm", "admm_adaptive"):
            lam, iters, _, state = admm(G, g, mu, eps=eps, max_iter=max_iter, state=state,
                                        adapt=route == "admm_adaptive")
        elif route == "pgs":
            lam, sweeps, _ = pgs(G, g, mu, eps=eps, max_iter=max(1, max_iter - iters), lam0=lam)
            iters += sweeps
        else:
            raise ValueError(route)
        lscale = max(1.0, np.max(np.abs(lam)))
        es, el = max(eps_sigma, 10 * eps), max(eps_lambda, 10 * eps)
        modes, _ = classify(G, g, mu, lam, es, el)
        start = lam
        cands = [lam]
        for _ in range(rounds):
            x = newton_modes(G, g, mu, start, modes, sat_delta=10 * eps * lscale)
            cands.append(x)
            if ncp_residual(G, g, mu, x) <= tol * scale:
                break
            # the Newton iterate solves its mode equations exactly: any violation above the
            # acceptance tolerance is real and flips the mode
            new = reclassify(G, g, mu, x, modes, 10 * tol * scale, 10 * tol * lscale, 10 * tol * lscale)
            if (new == modes).all():
                break
            modes = new
            start = proj_K(x, mu)
        for c in cands:
            r = ncp_residual(G, g, mu, c)
            if r < best_r:
                best, best_r = c, r
        if best_r <= tol * scale:
            return best, iters, True
        if iters >= max_iter:
            break
    return best, iters, False


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
    or lambda_N <= eps_l; else sticking if the impulse is strictly inside the cone
    (mu lambda_N - ||lambda_T|| > eps_l: by Eq. 1 such a contact has sigma = 0, whatever the
    accuracy of the iterate); else sliding.  Thresholds are relative to max(1, ||g||_inf) and
    max(1, ||lambda||_inf).  Returns (modes, margin) where margin is the smallest relative distance
    of the deciding quantities to the boundary of the identified mode."""
    sigma = G @ lam + g
    es, el = thresholds(g, lam, eps_sigma, eps_lambda)
    ss = max(1.0, np.max(np.abs(g))) if len(g) else 1.0
    sl = max(1.0, np.max(np.abs(lam))) if len(lam) else 1.0
    modes, margin = [], np.inf
    for i in range(len(mu)):
        s, l = sigma[3 * i:3 * i + 3], lam[3 * i:3 * i + 3]
        ns = np.linalg.norm(s)
        nst = np.linalg.norm(s[:2])
        inside = mu[i] * l[2] - np.linalg.norm(l[:2])
        if ns <= es:
            modes.append(STK)
            margin = min(margin, (es - ns) / es)
        elif s[2] > es or l[2] <= el:
            modes.append(BRK)
            margin = min(margin, (s[2] - es) / ss if s[2] > es else 0.0)
        elif inside > el:
            modes.append(STK)
            margin = min(margin, inside / sl)
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


def saturated(lam, mu, modes, delta):
    """Sticking contacts whose impulse lies within delta of the cone boundary (||l_T|| = mu l_N)."""
    out = []
    for i, md in enumerate(modes):
        l = lam[3 * i:3 * i + 3]
        if md == STK and mu[i] * l[2] - np.sqrt(l[:2] @ l[:2]) <= delta:
            out.append(i)
    return out


def polish_equations(lam, G, g, mu, modes, sat):
    """Mode equations plus, for each saturated sticking contact, mu lambda_N - ||lambda_T|| = 0.
    With redundant contacts the sticking impulses are only defined up to internal forces; this
    extra equation picks the member of that family that keeps a boundary impulse on the boundary."""
    e = mode_equations(lam, G, g, mu, modes)
    extra = [mu[i] * lam[3 * i + 2] - np.sqrt(lam[3 * i:3 * i + 2] @ lam[3 * i:3 * i + 2]) for i in sat]
    return np.concatenate([e, np.array(extra)]) if extra else e


def newton_modes(G, g, mu, lam, modes, iters=20, tol=1e-15, sat_delta=0.0):
    """Newton on the mode equations (plus the saturation equations of the sticking contacts whose
    impulse is within sat_delta of the cone boundary) with minimum-norm least-squares steps (the
    system is singular when the contact set is redundant)."""
    if len(g) == 0:
        return lam
    sat = saturated(lam, mu, modes, sat_delta)
    x = lam.copy()
    scale = max(1.0, np.max(np.abs(g)))
    for _ in range(iters):
        F = polish_equations(x, G, g, mu, modes, sat)
        if np.max(np.abs(F)) <= tol * scale:
            break
        J = cs_jacobian(lambda z: polish_equations(z, G, g, mu, modes, sat), x)
        x = x - np.linalg.lstsq(J, F, rcond=1e-13)[0]
    return x


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
