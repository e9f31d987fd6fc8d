"""Serving loop on the GPU: a job's result is bitwise the same alone and in a mix of concurrent jobs, and the
footprint mg_plan reports is what the console allocates."""
import numpy as np
import pytest

import workloads as W
import paper_2509_15948_gb300 as M
from paper_2509_15948_gb300.serve import Job, Server, job_footprint, latency_summary
from tests.cases import make_case

pytestmark = pytest.mark.gpu


def jobs_for(layouts, seed=5):
    jobs = []
    for i, lay in enumerate(layouts):
        case = make_case([lay], seed=seed + i)
        jobs.append(Job(i, M.Song(lay.num_tracks, lay.num_subgroups, lay.track_group, lay.num_samples),
                        case.sources[0], case.targets[0], case.noise, init_params=case.params,
                        train_steps=8, n_iter=1, finetune_steps=4, seed=i))
    return jobs


def test_job_result_is_the_same_alone_and_in_the_mix():
    jobs = jobs_for([W.SongLayout(3, 1, [0, -1, 0], 30011), W.SongLayout(2, 0, [-1, -1], 22050),
                     W.SongLayout(4, 2, [0, 1, 0, -1], 26000)])
    budget = 8 * max(job_footprint(j) for j in jobs)
    alone = [Server(budget).run([j])[0] for j in (jobs[0], jobs[2])]
    srv = Server(budget)
    mixed = srv.run(jobs)
    assert srv.peak_active == 3
    for a, m in zip(alone, (mixed[0], mixed[2])):
        assert a.error is None and m.error is None, (a.error, m.error)
        assert np.array_equal(a.params, m.params) and np.array_equal(a.present, m.present)
        assert a.la_final == m.la_final
    s = latency_summary(mixed)
    assert s["failed"] == 0 and s["track_s_per_s"] > 0


@pytest.mark.parametrize("retain", [-1, 1])
def test_plan_footprint_equals_console_allocation(retain):
    case = make_case([W.SongLayout(3, 1, [0, -1, 0], 30011)], seed=2)
    song = M.Song(3, 1, [0, -1, 0], 30011)
    cfg = M.ConsoleConfig(retain_spectra=retain)
    planned = M.plan([song], cfg)["device_bytes"]
    con = M.Console([song], case.sources, case.targets, case.noise, cfg)
    assert con.get_info()["device_bytes"] == planned > 0
    con.close()
