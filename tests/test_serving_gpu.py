"""Serving (continuous batching) through the C ABI's sfp_server_* calls.

A job's result must not depend on the other jobs it runs with: the noise is
keyed by its own id and step counter and its start by its own id, and a job
stops exactly after its steps.  Checked bit for bit (alone vs in a mix of
jobs that arrive over time) and against the oracle."""
import math
import time

import numpy as np
import pytest

import paper_1411_3487_gb300 as sfp
from golden_values import shear_tau
from oracle import oracle as O
from paper_1411_3487_gb300 import build

pytestmark = pytest.mark.gpu

DT = {64: 10.0, 128: 50.0, 256: 100.0, 512: 100.0}


@pytest.fixture(scope="module", autouse=True)
def built():
    build.build()


def rel(a, b):
    a, b = np.asarray(a)[:, 1:], np.asarray(b)[:, 1:]
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def oracle_run(M, job_id, n_steps, shear_per_s, seed=1):
    m = O.Model(M, dtau=DT[M])
    R0 = m.equilibrium_start(seed, job_id)
    return m.run_modes(R0[None], seed, [job_id], 0, n_steps, shear=shear_tau(shear_per_s))[0]


def job(M, n_steps, job_id, shear=0.0):
    return {"n_beads": M, "dtau": DT.get(M, 10.0), "n_steps": n_steps, "job_id": job_id, "shear_rate_per_s": shear}


@pytest.mark.parametrize("precision", [sfp.SFP_FP32, sfp.SFP_MIXED_BF16, sfp.SFP_FP64], ids=["fp32", "bf16", "fp64"])
def test_result_is_the_same_alone_and_in_the_mix(precision):
    probe = job(128, 301, 77, 1.0e8)
    with sfp.Server(precision=precision, slots_per_pool=64, quantum_steps=32) as s:
        t = s.submit(probe)
        s.wait_idle(120)
        alone = s.modes(t)
        assert [r["status"] for r in s.poll()] == [0]
    rng = np.random.default_rng(5)
    with sfp.Server(precision=precision, slots_per_pool=64, quantum_steps=32) as s:
        tickets = []
        for k in range(40):
            M = int(rng.choice([64, 128, 256, 512]))
            tickets.append(s.submit(job(M, int(rng.integers(20, 400)), 1000 + k,
                                        float(rng.choice([0.0, 5e7])))))
            if k == 17:
                tp = s.submit(probe)
            if k % 8 == 7:
                time.sleep(0.01)      # later jobs arrive while earlier ones run
        s.wait_idle(300)
        res = {r["ticket"]: r for r in s.poll(100)}
        assert len(res) == 41 and all(r["status"] == 0 for r in res.values())
        mixed = s.modes(tp)
        assert res[tp]["admit_s"] >= res[tp]["submit_s"]
        # a job from the mix against its own oracle run
        t5 = tickets[5]
        st = s.stats()
        assert st["finished"] == 41 and st["running"] == 0
    if precision == sfp.SFP_FP64:
        assert np.array_equal(mixed, alone)
    else:
        assert rel(mixed, alone) < 1e-6
    ref = oracle_run(128, 77, 301, 1.0e8)
    assert rel(alone, ref) < (1e-9 if precision == sfp.SFP_FP64 else 1e-5)


def test_jobs_stop_exactly_inside_a_quantum():
    with sfp.Server(slots_per_pool=16, quantum_steps=16) as s:
        short = s.submit(job(256, 37, 5))
        long_ = s.submit(job(256, 100, 6))
        s.wait_idle(60)
        r = {x["ticket"]: x for x in s.poll()}
        assert r[short]["n_steps"] == 37 and r[short]["status"] == 0
        for t, jid, n in ((short, 5, 37), (long_, 6, 100)):
            assert rel(s.modes(t), oracle_run(256, jid, n, 0.0)) < 1e-5


def test_admission_within_a_small_hbm_budget():
    """A budget that holds about one pool at a time: jobs of three lengths all
    finish, pools are released and created as the shapes change, and the
    device memory held never exceeds the budget."""
    budget = 40 << 20
    with sfp.Server(slots_per_pool=256, quantum_steps=32, hbm_budget_bytes=budget) as s:
        ts = [s.submit(job(M, 64, 300 + i)) for i, M in enumerate([512, 256, 512, 128, 256, 64])]
        peak = 0
        t0 = time.time()
        while s.stats()["finished"] < len(ts) and time.time() - t0 < 120:
            peak = max(peak, s.stats()["device_bytes"])
            time.sleep(0.005)
        s.wait_idle(60)
        assert peak <= budget
        res = {r["ticket"]: r for r in s.poll()}
        assert all(r["status"] == 0 for r in res.values()) and len(res) == len(ts)
        assert rel(s.modes(ts[3]), oracle_run(128, 303, 64, 0.0)) < 1e-5


def test_latency_statistics():
    with sfp.Server(slots_per_pool=64, quantum_steps=64, keep_results=False) as s:
        for k in range(30):
            s.submit(job(64, 200 + 10 * k, k))
        s.wait_idle(60)
        r = s.poll()
        st = s.stats()
    lat = sorted(x["latency_s"] for x in r)
    assert len(lat) == 30 and lat[0] > 0
    assert st["p50_s"] == pytest.approx(np.percentile(lat, 50), rel=1e-9)
    assert st["p99_s"] == pytest.approx(np.percentile(lat, 99), rel=1e-9)
    assert st["bead_steps"] == sum(64 * (200 + 10 * k) for k in range(30))


def test_malformed_jobs_are_refused():
    with sfp.Server() as s:
        for bad in (job(2, 10, 1), job(64, -1, 1), job(64, 10, 1 << 32)):
            with pytest.raises(sfp.SfpError):
                s.submit(bad)


def test_pools_shrink_to_fit_and_impossible_jobs_fail():
    """Pools that do not fit the budget are retried smaller; a job that cannot
    fit even a one-slot pool while nothing runs fails with SFP_ENOMEM."""
    with sfp.Server(slots_per_pool=4096, quantum_steps=32, hbm_budget_bytes=24 << 20) as s:
        t = s.submit(job(512, 40, 9))
        s.wait_idle(60)
        r = s.poll()
        assert r[0]["status"] == 0 and s.stats()["device_bytes"] <= 24 << 20
        assert rel(s.modes(t), oracle_run(512, 9, 40, 0.0)) < 1e-5
    with sfp.Server(hbm_budget_bytes=64 << 10) as s:
        s.submit(job(512, 10, 1))
        s.wait_idle(60)
        assert s.poll()[0]["status"] == sfp._lib.SFP_ENOMEM
