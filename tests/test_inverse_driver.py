"""The batched Gauss-Newton driver of paper_2409_07107_gb300.inverse on the host: fed with the
oracle's step and Jacobian (through the same [nv][nv][B] layout the library writes), it reaches the
oracle's own Gauss-Newton solution for standing quadrupeds (no GPU; the GPU run feeds it
sim_step_jac through simulator_step_jac)."""
import numpy as np
import torch

from oracle import inverse as OI
from oracle import step as S
from paper_2409_07107_gb300 import scenes
from paper_2409_07107_gb300.inverse import gauss_newton_inverse_dynamics


def test_driver_matches_oracle_loop():
    wl = scenes.quadruped_feet(3)
    wl.batch.v[:] = 0.0
    m = wl.models[0]
    nv, B = m.nv, wl.batch.B
    envs = [wl.batch.env(e, m) for e in range(B)]

    def step_jac(tau):
        tau = tau.numpy()
        vn = np.zeros((nv, B))
        jt = np.zeros((nv, nv, B))
        for e in range(B):
            st = S.step_jac(m, dict(envs[e], tau=tau[:, e]), wl.options)
            vn[:, e] = st["v_next"]
            jt[:, :, e] = st["dv_dtau"]
        return torch.from_numpy(vn), torch.from_numpy(jt)

    Sa = torch.eye(nv, dtype=torch.float64)[6:]
    ta, hist = gauss_newton_inverse_dynamics(step_jac, Sa, torch.zeros(nv, B, dtype=torch.float64),
                                             torch.zeros(nv - 6, B, dtype=torch.float64), iters=20, tol=1e-10)
    assert hist[-1] <= 1e-8 * max(1.0, hist[0]) and len(hist) <= 15
    for e in range(B):
        ref, _ = OI.inverse_dynamics(m, envs[e], wl.options, Sa.numpy(), np.zeros(nv), np.zeros(nv - 6),
                                     iters=20, tol=1e-10)
        assert np.abs(ta[:, e].numpy() - ref).max() <= 1e-7 * max(1.0, np.abs(ref).max())
