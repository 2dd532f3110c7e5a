"""The contact-mode mix of the arm + cube benchmark workload, measured with the oracle (no GPU).

The configuration asks for about half of the contacts sticking and half sliding.  The cube's 5 cm
face lands on the plane at 0.1-0.5 m/s; the arm's inertia couples the normal impulse to the cube's
roll and pitch, so for nearly every arm configuration the face tips onto one or two corners and
the other corners separate.  Of the corners that stay in contact, the share that sticks is set by
that same coupling more than by the initial tangential speed.  This pins the mix the generator
actually gives, so that a change to it is seen: most corners breaking, and among the persistent
ones roughly a quarter sticking."""
import multiprocessing as mp

import numpy as np
import pytest

from paper_2409_07107_gb300 import scenes


def _modes(args):
    from oracle import step as S
    m, env, opt = args
    return [int(x) for x in S.step(m, env, opt)["modes"]]


@pytest.mark.slow
def test_arm_cube_mode_mix():
    wl = scenes.arm_cube(65536)
    m = wl.models[0]
    n = 256
    with mp.get_context("spawn").Pool(8) as pool:
        res = pool.map(_modes, [(m, wl.batch.env(e, m), wl.options) for e in range(n)], chunksize=8)
    c = np.zeros(3, int)
    for md in res:
        for x in md:
            c[x] += 1
    brk, stk, sld = c
    assert c.sum() == 4 * n                          # every env has its four corners active
    assert 0.6 <= brk / c.sum() <= 0.8, c
    assert 0.15 <= stk / (stk + sld) <= 0.4, c
    even = [md for e, md in enumerate(res) if e % 2 == 0]
    odd = [md for e, md in enumerate(res) if e % 2 == 1]
    # the envs set up to stick hold nearly all sticking contacts
    assert sum(md.count(1) for md in even) > 5 * sum(md.count(1) for md in odd)
