"""The pipeline schedule index (ds_autotune / ds_set_schedule) as the binding decodes it."""
import itertools

import paper_2409_07107_gb300 as ds


def test_schedule_index_round_trip():
    radices = [len(opts) for _, opts in ds.SCHEDULE_KNOBS]
    n = 1
    for r in radices:
        n *= r
    assert n == ds.NUM_SCHEDULES
    seen = set()
    for pos in itertools.product(*[range(r) for r in radices]):
        idx = ds.schedule_index(*pos)
        assert 0 <= idx < ds.NUM_SCHEDULES
        seen.add(idx)
        d = ds.describe_schedule(idx)
        for p, (name, opts) in zip(pos, ds.SCHEDULE_KNOBS):
            assert d[name] == opts[p]
    assert len(seen) == ds.NUM_SCHEDULES


def test_default_schedule_index():
    # the library's default: default caps, row-per-lane from round 5, 4 finish CTAs per SM,
    # cooperative Newton, overlapped finish after round 5 keeping every 8th SM free, two-warp ADMM
    # rounds from round 5, no speculative Newton attempts, the single-contact presolve, the pipeline
    # (not the persistent launch)
    d = ds.describe_schedule(ds.schedule_index())
    assert d == {"round_caps": "default", "row_per_lane_admm_from_round": 5, "finish_ctas_per_sm": 4,
                 "newton": "cooperative", "overlapped_finish_after_round": 5, "two_warp_admm_from_round": 5,
                 "overlapped_finish_keeps_free_every_nth_sm": 8, "speculative_newton_from_round": None,
                 "single_contact_presolve": True, "launch": "pipeline",
                 "finish": "one kernel"}
