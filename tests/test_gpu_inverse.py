"""Gauss-Newton inverse dynamics through contacts (Sec. 4) driven by the library's sim_step_jac:
the actuator torques that hold standing quadrupeds at rest (v+ = 0), against the oracle's own
Gauss-Newton loop on the same envs."""
import numpy as np
import pytest

from paper_2409_07107_gb300 import scenes

pytestmark = pytest.mark.gpu


def _oracle_torques(args):
    from oracle import inverse as OI
    m, env, opt, Sa, nv = args
    ta, hist = OI.inverse_dynamics(m, env, opt, Sa, np.zeros(nv), np.zeros(Sa.shape[0]), iters=20, tol=1e-10)
    return ta, hist


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_inverse_dynamics_standing_quadrupeds(precision):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import multiprocessing as mp
    import paper_2409_07107_gb300 as ds
    from paper_2409_07107_gb300 import build
    from paper_2409_07107_gb300.inverse import gauss_newton_inverse_dynamics, simulator_step_jac
    build.build()
    B = 8
    wl = scenes.quadruped_feet(B)
    wl.batch.v[:] = 0.0
    m = wl.models[0]
    nv = m.nv
    Sa = np.eye(nv)[6:]
    with mp.get_context("spawn").Pool(B) as pool:
        refs = pool.map(_oracle_torques, [(m, wl.batch.env(e, m), wl.options, Sa, nv) for e in range(B)])
    sim = ds.Simulator(wl, precision=precision)
    f64 = dict(dtype=torch.float64, device="cuda")
    fn = simulator_step_jac(sim)
    ta, hist = gauss_newton_inverse_dynamics(fn, torch.tensor(Sa, **f64), torch.zeros(nv, B, **f64),
                                             torch.zeros(nv - 6, B, **f64), iters=20, tol=1e-10)
    ta = ta.cpu().numpy()
    if precision == "fp64":
        assert hist[-1] <= 1e-8 * max(1.0, hist[0]), hist
        for e in range(B):
            ref = refs[e][0]
            assert np.abs(ta[:, e] - ref).max() <= 1e-7 * max(1.0, np.abs(ref).max()), e
    else:
        # FP32 bulk: the residual falls to the mixed step's accuracy and the torques agree to it
        assert hist[-1] <= 1e-4 * max(1.0, hist[0]), hist
        assert max(hist[len(hist) // 2:]) <= hist[0]
        for e in range(B):
            ref = refs[e][0]
            assert np.abs(ta[:, e] - ref).max() <= 1e-3 * max(1.0, np.abs(ref).max()), e
