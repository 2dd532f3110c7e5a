"""One step with contacts between convex shapes on two bodies (or a body and a fixed shape), and
its Jacobians by the paper's route with App. C's contact-placement terms (oracle).  Test
infrastructure only; the plane contacts of step.py are not mixed in here.

A pair is (shape_a, body_a, (E_a, r_a), shape_b, body_b, (E_b, r_b), mu): each shape sits at
placement (E, r) on its body (-1 = the fixed world).  Collision detection (collision.collide) gives
the contact frame; a pair is active when phi <= 0.  J_c v is the velocity of B's material point
relative to A's at the contact point, in the contact frame (Z along the normal from A to B), so
sigma = J_c v+ follows Eq. 1's convention (sigma_N > 0 separates).  The impulse lambda acts on B
and -lambda on A: body i receives the wrench +-X_i^T [lambda; 0] / dt in its own coordinates (X_i
the motion transform from body i to the contact frame).

The step is Eq. 3-6 with these rows: v_f = v + dt ABA(q, v, tau), G = J_c M^-1 J_c^T,
g = J_c v_f (+ App. D's Baumgarte term with the options baumgarte_kp, baumgarte_kd and the
activation margin contact_margin, as for the plane contacts), the staged NCP solve of ncp.py,
v+ = v + dt ABA(q, v, tau, f_ext(lambda)).  Its Jacobians take
App. D's route 1 (step.route1_matrices): D = dv+/d(q, v, tau) at fixed lambda and F = d(J_c v+)/dq
at fixed v+, where the q-derivatives split into the part at fixed contact placement (complex steps
through the rigid-body functions, the transforms X_i held) and App. C's placement terms
(collision.appc_dJctlam_dq, collision.appc_dJcv_dq), with dCD/dM_i by central differences of the
collision detection or, as the paper takes it, by randomized smoothing (dcd_fn)."""
import numpy as np

from . import collision as Co
from . import rigid
from .ncp import classify, solve_ncp
from .step import H_CS, pinv_solve, route1_matrices


def active_pairs(model, q, pairs, margin=0.0):
    """Indices of the pairs whose signed distance is <= margin (decided on the real part) and
    their signed distances."""
    out, phis = [], []
    for k, pr in enumerate(pairs):
        _, _, res = Co.pair_placement(model, np.real(q), pr[:6])
        if res["phi"] <= margin:
            out.append(k)
            phis.append(res["phi"])
    return out, np.array(phis)


def _gains(opt):
    kp, kd = getattr(opt, "baumgarte_kp", 1.0), getattr(opt, "baumgarte_kd", 0.0)
    margin = getattr(opt, "contact_margin", 0.0)
    return kp, kd, margin, not (kp == 1.0 and kd == 0.0 and margin == 0.0)


def baumgarte(opt, phis, Jc, v):
    """App. D's term of g on the active pairs: zero on the tangent rows, and on the normal row
    phi/dt - K_p [phi/dt]_- - K_d (J_c v)_N ([x]_- = min(x, 0)); identically zero for K_p = 1,
    K_d = 0 and no margin (every active pair then has phi <= 0)."""
    kp, kd, _, on = _gains(opt)
    b = np.zeros(Jc.shape[0])
    if not on or len(phis) == 0:
        return b
    x = phis / opt.dt
    b[2::3] = x - kp * np.minimum(x, 0.0) - kd * (Jc @ v)[2::3]
    return b


def pair_rows(model, q, pairs, act, transforms=None):
    """J_c (3 na x nv) of the active pairs; with ``transforms`` (one (cX_a, cX_b) per active pair)
    held, only the bodies' Jacobians vary with q."""
    nv = rigid.index_maps(model)[3]
    if not act:
        return np.zeros((0, nv))
    return np.concatenate([Co.pair_jc(model, q, pairs[k][:6], None if transforms is None else transforms[j])
                           for j, k in enumerate(act)], axis=0)


def pair_wrenches(model, q, pairs, act, transforms, lam, scale):
    """Body wrenches (body coordinates) of the impulses lam on the active pairs, divided by scale."""
    nb = len(model.parent)
    f = [np.zeros(6, dtype=np.result_type(q, lam, 1.0)) for _ in range(nb)]
    for j, k in enumerate(act):
        pr = pairs[k]
        lin = np.concatenate([lam[3 * j:3 * j + 3], np.zeros(3)]) / scale
        for X, body, sign in ((transforms[j][0], pr[1], -1.0), (transforms[j][1], pr[4], 1.0)):
            if body >= 0:
                f[body] = f[body] + sign * (X.T @ lin)
    return f


def ufd_velocity(model, q, v, tau, opt, fext):
    return v + opt.dt * rigid.aba(model, q, v, tau, np.asarray(opt.gravity, float), fext)


def step(model, env, pairs, opt):
    """One step with pair contacts; returns v_next, lam, modes, margin, the active pairs and the
    quantities the Jacobians need."""
    q, v, tau = env["q"], env["v"], env["tau"]
    dt = opt.dt
    M = rigid.crba(model, q)
    L = rigid.cholesky(M)
    v_f = ufd_velocity(model, q, v, tau, opt, None)
    act, phis = active_pairs(model, q, pairs, _gains(opt)[2])
    transforms = [Co.pair_transforms(model, q, pairs[k][:6]) for k in act]
    Jc = pair_rows(model, q, pairs, act, transforms)
    mu = np.array([pairs[k][6] for k in act])
    Y = rigid.chol_solve(L, Jc.T) if act else np.zeros((len(v), 0))
    G, g = Jc @ Y, Jc @ v_f + baumgarte(opt, phis, Jc, v)
    es, el = getattr(opt, "eps_sigma", 1e-8), getattr(opt, "eps_lambda", 1e-8)
    lam, iters, conv = solve_ncp(G, g, mu, es, el) if act else (np.zeros(0), 0, True)
    modes, margin = classify(G, g, mu, lam, es, el)
    fext = pair_wrenches(model, q, pairs, act, transforms, lam, dt) if act else None
    v_next = ufd_velocity(model, q, v, tau, opt, fext)
    return dict(v_next=v_next, lam=lam, modes=modes, margin=margin, act=act, transforms=transforms,
                Jc=Jc, Y=Y, G=G, g=g, mu=mu, M=M, converged=conv, phis=phis)


def partials(model, env, pairs, opt, st, dcd_fn=None):
    """D = dv+/d(q, v, tau) at fixed lambda (nv x 3 nv), F = d(J_c v+)/dq at fixed v+ and Bt, the
    derivative of the Baumgarte term (None when it is identically zero): on the normal rows
    d(phi/dt - K_p [phi/dt]_-)/dq = (1 - K_p [phi < 0]) (J_c)_N / dt, since the signed distance
    changes at the normal relative velocity of the witness points (d phi = (J_c dq)_N), and
    -K_d d(J_c v)_N/d(q, v) with the same placement terms as F.
    dcd_fn(model, q, pair, which) gives dCD/dM_i (default: central differences, Co.dcd_dbody)."""
    dcd_fn = dcd_fn or (lambda m, qq, pr, w: Co.dcd_dbody(m, qq, pr, w))
    q, v, tau = env["q"], env["v"], env["tau"]
    nv, dt = len(v), opt.dt
    act, transforms, lam, v_next = st["act"], st["transforms"], st["lam"], st["v_next"]
    fext = pair_wrenches(model, q, pairs, act, transforms, lam, dt) if act else None
    # v and tau: the contact wrenches do not move
    Dv, Dt = [], []
    for j in range(nv):
        e = np.zeros(nv, dtype=complex)
        e[j] = 1j * H_CS
        Dv.append(np.imag(ufd_velocity(model, q, v + e, tau, opt, fext)) / H_CS)
        Dt.append(np.imag(ufd_velocity(model, q, v, tau + e, opt, fext)) / H_CS)
    # q: M a* = tau - b(q, v) + J_c^T lambda / dt at the solution's a* = (v+ - v) / dt, so
    # dv+/dq = -dt M^-1 [dRNEA(q, v, a*)/dq - d(J_c^T lambda)/dq / dt]
    a_star = (v_next - v) / dt
    grav = np.asarray(opt.gravity, float)
    dRq, dJl, Fq = np.zeros((nv, nv)), np.zeros((nv, nv)), np.zeros((3 * len(act), nv))
    Kq = np.zeros((3 * len(act), nv))                             # d(J_c v)/dq at fixed v
    for j in range(nv):
        e = np.zeros(nv, dtype=complex)
        e[j] = 1j * H_CS
        qj = rigid.integrate(model, q, e)
        dRq[:, j] = np.imag(rigid.rnea(model, qj, v, a_star, grav)) / H_CS
        if act:
            Jh = pair_rows(model, qj, pairs, act, transforms)      # the transforms held
            dJl[:, j] = np.imag(Jh.T @ lam) / H_CS
            Fq[:, j] = np.imag(Jh @ v_next) / H_CS
            Kq[:, j] = np.imag(Jh @ v) / H_CS
    for jj, k in enumerate(act):
        pr = pairs[k][:6]
        dcd = (dcd_fn(model, q, pr, 0), dcd_fn(model, q, pr, 1))
        dJl += Co.appc_dJctlam_dq(model, q, lam[3 * jj:3 * jj + 3], pr, dcd)
        Fq[3 * jj:3 * jj + 3] += Co.appc_dJcv_dq(model, q, v_next, pr, dcd)
        Kq[3 * jj:3 * jj + 3] += Co.appc_dJcv_dq(model, q, v, pr, dcd)
    Dq = -dt * rigid.chol_solve(rigid.cholesky(st["M"]), dRq - dJl / dt)
    D = np.concatenate([Dq, np.stack(Dv, 1), np.stack(Dt, 1)], axis=1)
    kp, kd, _, on = _gains(opt)
    Bt = None
    if act and on:
        Bt = np.zeros((3 * len(act), 3 * nv))
        Jc = st["Jc"]
        neg = np.real(st["phis"]) < 0.0
        Bt[2::3, :nv] = (1.0 - kp * neg)[:, None] * Jc[2::3] / dt - kd * Kq[2::3]
        Bt[2::3, nv:2 * nv] = -kd * Jc[2::3]
    return D, Fq, Bt


def step_jac(model, env, pairs, opt, dcd_fn=None):
    """The step and dv+/d(q, v, tau) by route 1 (App. B, D): dv = D + Y C X with
    X = -A^- B (J_c D + [F, 0, 0]).  dcd_fn as for partials (e.g. App. C's randomized smoothing,
    Co.dcd_dbody_smoothed with the caller's samples)."""
    st = step(model, env, pairs, opt)
    D, F, Bt = partials(model, env, pairs, opt, st, dcd_fn)
    nv = len(env["v"])
    if st["act"]:
        A, Bm, C = route1_matrices(st["G"], st["g"], st["mu"], st["lam"], st["modes"])
        RHS = st["Jc"] @ D
        RHS[:, :nv] += F
        if Bt is not None:
            RHS = RHS + Bt
        X = -pinv_solve(A, Bm @ RHS)
        J = D + st["Y"] @ (C @ X)
    else:
        J = D
    st["dv_dq"], st["dv_dv"], st["dv_dtau"] = J[:, :nv], J[:, nv:2 * nv], J[:, 2 * nv:]
    return st


def jacobian_fd(model, env, pairs, opt, h=1e-6):
    """Central finite differences of the whole step w.r.t. (q tangent, v, tau)."""
    q, v, tau = env["q"], env["v"], env["tau"]
    nv = len(v)
    cols = []
    for which in range(3):
        for j in range(nv):
            e = np.zeros(nv)
            e[j] = h
            outs = []
            for s in (1.0, -1.0):
                en = dict(env)
                if which == 0:
                    en["q"] = rigid.integrate(model, q, s * e)
                elif which == 1:
                    en["v"] = v + s * e
                else:
                    en["tau"] = tau + s * e
                outs.append(step(model, en, pairs, opt)["v_next"])
            cols.append((outs[0] - outs[1]) / (2 * h))
    return np.stack(cols, axis=1)
