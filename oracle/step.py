"""One simulation step and its derivatives dv+/d(q, v, tau) (oracle).  Test infrastructure only.

Step (Sec. 2.3, Eq. 3-4 and Eq. 5-6): M, the free velocity v_f = v + dt ABA(q, v, tau), the active
contacts and J_c, G = J_c M^-1 J_c^T, g = J_c v_f, lambda* from the NCP (Eq. 1), then
v+ = v + dt UFD(q, v, tau, lambda*) (ABA with the contact impulses as external forces) and the
symplectic-Euler position update q+ = q (+) dt v+.  lambda is an impulse, so UFD's contact term is
M^-1 J_c^T lambda / dt and G, g are exactly those of Eq. 4.

Baumgarte stabilisation (App. D): with gains K_p, K_d (options baumgarte_kp, baumgarte_kd; the
defaults K_p = 1, K_d = 0 leave g = J_c v_f for every contact with phi <= 0) the normal entry of g
gains phi/dt - K_p [phi/dt]_- - K_d (J_c v)_N, phi the contact's signed distance; sigma = G lambda +
g is then J_c v+ plus that term, and its derivatives enter the right-hand side of the implicit
solve.  Activation margin (option contact_margin, default 0): a slot is active when phi <= margin.
App. D's term with [phi/dt]_- implies that a contact can be active at phi > 0; such a contact gains
phi/dt - K_d (J_c v)_N (the proportional part acts on penetration only), so that sigma_N >= 0 lets
it approach the plane by at most phi within the step.

Derivatives (Sec. 3.1-3.3, App. B, D), w.r.t. a tangent perturbation q (+) dq of q and w.r.t. v, tau:

* D = dv+/dtheta at fixed lambda* (the second term of Eq. 7, with the collision-detection term of
  App. C included because the contact points are recomputed from q), and
  F = d(J_c v+)/dq at fixed v+ (the FKV term of App. D): complex-step derivatives of the oracle's
  own recursions.
* Route 1 (the paper's form, App. B): A = B G C + blkdiag(0, Q, ..., Q), A X = -B (J_c D + F),
  dlambda = C X, dv+/dtheta = D + M^-1 J_c^T dlambda.  A may be singular (redundant contacts) and
  is solved in the minimum-norm sense.
* The position update's adjoint (for rollouts): Jacobians of q+ = q (+) dt v+ in tangent
  coordinates by complex step (integrate_jacobians), chained in by vjp().
* Route 2 (independent check): implicit function theorem applied directly to the stacked mode
  equations E(lambda; theta) = 0 with sigma = J_c(q) v+(q, v, tau, lambda); both Jacobians of E by
  complex step; no R, P, Q, A, B or C anywhere.
"""
import numpy as np

from . import rigid
from .contact import active_slots, contact_jacobian, contact_wrenches, signed_distances
from .ncp import (BRK, SLD, STK, admm, classify, cs_jacobian, mode_residual, ncp_residual, solve_ncp)

H_CS = 1e-30


def _opt(opt, name, default):
    return getattr(opt, name, default) if opt is not None else default


def ufd_velocity(model, env, opt, slots, q, v, tau, lam):
    """v + dt * UFD(q, v, tau, lambda) with lambda (impulses) on the given contact slots (Eq. 6)."""
    dt, grav = opt.dt, np.asarray(opt.gravity, float)
    fext = contact_wrenches(model, q, env, slots, lam, scale=dt) if len(slots) else None
    return v + dt * rigid.aba(model, q, v, tau, grav, fext)


def gap_term(opt):
    """Whether g carries the signed-distance term: gains other than (1, 0), or an activation margin."""
    return not (_opt(opt, "baumgarte_kp", 1.0) == 1.0 and _opt(opt, "baumgarte_kd", 0.0) == 0.0
                and _opt(opt, "contact_margin", 0.0) == 0.0)


def baumgarte(model, env, opt, slots, q, v):
    """The Baumgarte term of g (App. D): zero on the tangent rows, and on the normal row of each
    active slot phi/dt - K_p [phi/dt]_- - K_d (J_c v)_N with [x]_- = min(x, 0) (decided on the real
    part, so that complex-step derivatives pass through).  Identically zero for K_p = 1, K_d = 0
    when no margin is set (every active contact then has phi <= 0)."""
    kp, kd, dt = _opt(opt, "baumgarte_kp", 1.0), _opt(opt, "baumgarte_kd", 0.0), opt.dt
    nc = len(slots)
    if nc == 0 or not gap_term(opt):
        return np.zeros(3 * nc)
    phi = signed_distances(model, q, env, slots) / dt
    neg = np.where(np.real(phi) < 0.0, phi, 0.0 * phi)
    jv = contact_jacobian(model, q, env, slots) @ v
    b = np.zeros(3 * nc, dtype=np.result_type(phi, jv))
    b[2::3] = phi - kp * neg - kd * jv[2::3]
    return b


def step(model, env, opt, do_polish=True):
    """One step.  Returns a dict with v_next, q_next, lambda, modes, margin and internals.  The NCP
    iteration is ADMM, or projected Gauss-Seidel when the option ``ncp_route`` is "pgs"."""
    q, v, tau = env["q"], env["v"], env["tau"]
    dt, grav = opt.dt, np.asarray(opt.gravity, float)
    M = rigid.crba(model, q)
    L = rigid.cholesky(M)
    v_f = v + dt * rigid.aba(model, q, v, tau, grav)
    slots = active_slots(model, q, env, _opt(opt, "contact_margin", 0.0))
    Jc = contact_jacobian(model, q, env, slots)
    mu = np.array([env["c_mu"][k] for k in slots])
    Y = rigid.chol_solve(L, Jc.T) if len(slots) else np.zeros((len(v), 0))
    G = Jc @ Y
    g = Jc @ v_f + baumgarte(model, env, opt, slots, q, v)
    es, el = _opt(opt, "eps_sigma", 1e-8), _opt(opt, "eps_lambda", 1e-8)
    if do_polish:
        lam, iters, conv = solve_ncp(G, g, mu, es, el, route=_opt(opt, "ncp_route", "admm"))
    else:
        lam, iters, conv, _ = admm(G, g, mu, eps=1e-12, max_iter=50000)
    modes, margin = classify(G, g, mu, lam, es, el)
    v_next = ufd_velocity(model, env, opt, slots, q, v, tau, lam)
    q_next = rigid.integrate(model, q, dt * v_next)
    return dict(v_next=v_next, q_next=q_next, lam=lam, modes=modes, margin=margin, slots=slots,
                iters=iters, converged=conv, residual=ncp_residual(G, g, mu, lam), M=M, L=L, Jc=Jc,
                Y=Y, G=G, g=g, mu=mu, v_f=v_f)


def partials(model, env, opt, st):
    """D = [dv+/dq, dv+/dv, dv+/dtau] at fixed lambda* (nv x 3nv) and F = d(J_c v+)/dq at fixed v+."""
    q, v, tau = env["q"], env["v"], env["tau"]
    nv = len(v)
    slots, lam, v_next = st["slots"], st["lam"], st["v_next"]
    Dq, Dv, Dt, F, Bq, Bv = [], [], [], [], [], []
    stab = gap_term(opt)
    for j in range(nv):
        e = np.zeros(nv, dtype=complex)
        e[j] = 1j * H_CS
        qj = rigid.integrate(model, q, e)
        Dq.append(np.imag(ufd_velocity(model, env, opt, slots, qj, v, tau, lam)) / H_CS)
        Dv.append(np.imag(ufd_velocity(model, env, opt, slots, q, v + e, tau, lam)) / H_CS)
        Dt.append(np.imag(ufd_velocity(model, env, opt, slots, q, v, tau + e, lam)) / H_CS)
        if len(slots):
            F.append(np.imag(contact_jacobian(model, qj, env, slots) @ v_next) / H_CS)
        if len(slots) and stab:
            Bq.append(np.imag(baumgarte(model, env, opt, slots, qj, v)) / H_CS)
            Bv.append(np.imag(baumgarte(model, env, opt, slots, q, v + e)) / H_CS)
    D = np.concatenate([np.stack(Dq, 1), np.stack(Dv, 1), np.stack(Dt, 1)], axis=1)
    F = np.stack(F, 1) if len(slots) else np.zeros((0, nv))
    # d(Baumgarte term)/d(q, v, tau) (App. D): the extra right-hand side of the implicit solve
    # (None with the unit gains, where the term is identically zero)
    Bt = (np.concatenate([np.stack(Bq, 1), np.stack(Bv, 1), np.zeros((3 * len(slots), nv))], axis=1)
          if len(slots) and stab else None)
    return D, F, Bt


def sliding_basis(lam_i, sigma_i, mu_i):
    """R (3x2), P (3x3), Q (2x2) of a sliding contact (Sec. 3.2, App. A):
    R = [lambda/||lambda||, e_z x u] with u = sigma_T/||sigma_T|| embedded in R^3,
    P = diag(H/alpha, 1), H = I - u u^T, alpha = ||sigma_T|| / (mu lambda_N), Q = diag(0, 1)."""
    st = sigma_i[:2]
    ns = np.sqrt(st @ st)
    u = st / ns
    r1 = lam_i / np.sqrt(lam_i @ lam_i)
    r2 = np.array([-u[1], u[0], 0.0])
    R = np.stack([r1, r2], axis=1)
    alpha = ns / (mu_i * lam_i[2])
    P = np.zeros((3, 3))
    P[:2, :2] = (np.eye(2) - np.outer(u, u)) / alpha
    P[2, 2] = 1.0
    return R, P, np.diag([0.0, 1.0])


def route1_matrices(G, g, mu, lam, modes):
    """B, C and A of App. B, formed densely (columns/rows: sticking contacts, then sliding)."""
    sigma = G @ lam + g
    nc = len(mu)
    stk = [i for i in range(nc) if modes[i] == STK]
    sld = [i for i in range(nc) if modes[i] == SLD]
    m = 3 * len(stk) + 2 * len(sld)
    B = np.zeros((m, 3 * nc))
    C = np.zeros((3 * nc, m))
    Qb = np.zeros((m, m))
    r = 0
    for i in stk:
        B[r:r + 3, 3 * i:3 * i + 3] = np.eye(3)
        C[3 * i:3 * i + 3, r:r + 3] = np.eye(3)
        r += 3
    for i in sld:
        R, P, Q = sliding_basis(lam[3 * i:3 * i + 3], sigma[3 * i:3 * i + 3], mu[i])
        B[r:r + 2, 3 * i:3 * i + 3] = R.T @ P
        C[3 * i:3 * i + 3, r:r + 2] = R
        Qb[r:r + 2, r:r + 2] = Q
        r += 2
    A = B @ G @ C + Qb
    return A, B, C


def pinv_solve(A, Bm):
    """Minimum-norm least-squares solution (SVD pseudo-inverse, cut-off 1e-12 sigma_max)."""
    if A.shape[0] == 0:
        return np.zeros((0, Bm.shape[1]))
    return np.linalg.pinv(A, rcond=1e-12) @ Bm


def jacobian_route1(model, env, opt, st, D=None, F=None, Bt=None):
    if D is None:
        D, F, Bt = partials(model, env, opt, st)
    nv = len(env["v"])
    if len(st["slots"]) == 0:
        return D, dict(D=D, F=F)
    A, Bm, C = route1_matrices(st["G"], st["g"], st["mu"], st["lam"], st["modes"])
    RHS = st["Jc"] @ D
    RHS[:, :nv] += F
    if Bt is not None:
        RHS = RHS + Bt
    X = -pinv_solve(A, Bm @ RHS)
    dlam = C @ X
    return D + st["Y"] @ dlam, dict(D=D, F=F, A=A, B=Bm, C=C, RHS=RHS, X=X, dlam=dlam)


def jacobian_route2(model, env, opt, st, D=None):
    """Direct implicit differentiation of the stacked mode equations."""
    q, v, tau = env["q"], env["v"], env["tau"]
    nv = len(v)
    if D is None:
        D = partials(model, env, opt, st)[0]
    slots, lam, mu, modes = st["slots"], st["lam"], st["mu"], st["modes"]
    if len(slots) == 0:
        return D

    def E(lam_, q_, v_, tau_):
        vn = ufd_velocity(model, env, opt, slots, q_, v_, tau_, lam_)
        sigma = contact_jacobian(model, q_, env, slots) @ vn + baumgarte(model, env, opt, slots, q_, v_)
        return mode_residual(lam_, sigma, mu, modes)

    E_lam = cs_jacobian(lambda x: E(x, q, v, tau), lam)
    cols = []
    for j in range(nv):
        e = np.zeros(nv, dtype=complex)
        e[j] = 1j * H_CS
        cols.append(np.imag(E(lam, rigid.integrate(model, q, e), v, tau)) / H_CS)
    for j in range(nv):
        e = np.zeros(nv, dtype=complex)
        e[j] = 1j * H_CS
        cols.append(np.imag(E(lam, q, v + e, tau)) / H_CS)
    for j in range(nv):
        e = np.zeros(nv, dtype=complex)
        e[j] = 1j * H_CS
        cols.append(np.imag(E(lam, q, v, tau + e)) / H_CS)
    E_th = np.stack(cols, axis=1)
    dlam = -np.linalg.pinv(E_lam, rcond=1e-12) @ E_th
    Y = cs_jacobian(lambda x: ufd_velocity(model, env, opt, slots, q, v, tau, x), lam)
    return D + Y @ dlam


def step_jac(model, env, opt, route=1):
    st = step(model, env, opt)
    if route == 1:
        J, extra = jacobian_route1(model, env, opt, st)
        st.update(extra)
    else:
        J = jacobian_route2(model, env, opt, st)
    nv = len(env["v"])
    st["dv_dq"], st["dv_dv"], st["dv_dtau"] = J[:, :nv], J[:, nv:2 * nv], J[:, 2 * nv:]
    return st


def jacobian_fd(model, env, opt, h=1e-6):
    """Central finite differences of the whole step (ADMM + polish) w.r.t. (q tangent, v, tau)."""
    q, v, tau = env["q"], env["v"], env["tau"]
    nv = len(v)
    cols = []
    for which in range(3):
        for j in range(nv):
            e = np.zeros(nv)
            e[j] = h
            outs = []
            for s in (+1, -1):
                en = dict(env)
                if which == 0:
                    en["q"] = rigid.integrate(model, q, s * e)
                elif which == 1:
                    en["v"] = v + s * e
                else:
                    en["tau"] = tau + s * e
                outs.append(step(model, en, opt)["v_next"])
            cols.append((outs[0] - outs[1]) / (2 * h))
    return np.stack(cols, axis=1)


def integrate_jacobians(model, q, dq):
    """Tangent Jacobians of the position update q+ = q (+) dq (the symplectic-Euler step of Sec. 2.3
    on the configuration manifold; dq = dt v+): with q+ (+) eta = (q (+) eps) (+) (dq + d),
    Jq = d eta / d eps and Jd = d eta / d d at eps = d = 0.  Complex step through rigid.integrate."""
    nv = len(dq)
    qp = rigid.integrate(model, q, dq)
    Jq, Jd = np.zeros((nv, nv)), np.zeros((nv, nv))
    for j in range(nv):
        e = np.zeros(nv, dtype=complex)
        e[j] = 1j * H_CS
        q_eps = rigid.integrate(model, rigid.integrate(model, q, e), dq)
        Jq[:, j] = np.imag(rigid.local_difference(model, qp, q_eps)) / H_CS
        Jd[:, j] = np.imag(rigid.local_difference(model, qp, rigid.integrate(model, q, dq + e))) / H_CS
    return Jq, Jd


def vjp(model, env, opt, v_bar, st=None, q_bar_next=None):
    """(q_bar, v_bar, tau_bar) = J^T v_bar from the route-1 Jacobian (the definition of a VJP).  With
    q_bar_next (a cotangent of q+ in its tangent coordinates) the adjoint of q+ = q (+) dt v+ is
    chained in: v_bar+ <- v_bar + dt Jd^T q_bar_next and q_bar <- q_bar + Jq^T q_bar_next."""
    if st is None or "dv_dq" not in st:
        st = step_jac(model, env, opt)
    vb = np.asarray(v_bar, float)
    qb = 0.0
    if q_bar_next is not None:
        Jq, Jd = integrate_jacobians(model, env["q"], opt.dt * st["v_next"])
        vb = vb + opt.dt * (Jd.T @ q_bar_next)
        qb = Jq.T @ q_bar_next
    return st["dv_dq"].T @ vb + qb, st["dv_dv"].T @ vb, st["dv_dtau"].T @ vb


def rollout(model, env0, taus, opt):
    """States (q_t, v_t), t = 0..T, of T steps from env0 with the joint torques taus[t]."""
    env = dict(env0)
    states = [(np.array(env["q"], float), np.array(env["v"], float))]
    for tau in taus:
        env = dict(env, tau=np.asarray(tau, float))
        st = step(model, env, opt)
        env = dict(env, q=st["q_next"], v=st["v_next"])
        states.append((st["q_next"], st["v_next"]))
    return states


def rollout_grad(model, env0, taus, opt, q_bar_T_raw):
    """Gradient w.r.t. every taus[t] of a loss whose gradient w.r.t. the final raw configuration q_T is
    q_bar_T_raw: reverse accumulation through the steps (vjp with the position-update adjoint), the
    final cotangent taken to tangent coordinates with d q_raw / d eta.  Also returns the margins of
    every step's classification (derivatives are those of the identified modes)."""
    states = rollout(model, env0, taus, opt)
    qT = states[-1][0]
    qb = rigid.tangent_to_raw_jacobian(model, qT).T @ np.asarray(q_bar_T_raw, float)
    vb = np.zeros(len(states[0][1]))
    grads, margins = [None] * len(taus), []
    for t in range(len(taus) - 1, -1, -1):
        env = dict(env0, q=states[t][0], v=states[t][1], tau=np.asarray(taus[t], float))
        st = step_jac(model, env, opt)
        margins.append(st["margin"])
        qb, vb, grads[t] = vjp(model, env, opt, vb, st=st, q_bar_next=qb)
    return np.array(grads), states, min(margins) if margins else np.inf
