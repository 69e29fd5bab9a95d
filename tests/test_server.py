"""Request scheduler (gbsmps_server_*): admission by device-memory budget,
continuous refill of free slots, no starvation, latency accounting.  These run
the scheduler in its simulation mode (jobs sleep instead of using a GPU), so
they exercise the host logic on any machine."""
import time

import numpy as np
import pytest

import paper_2512_10643_gb300 as g


def test_estimate_grows_with_size():
    o = g.opts_default(d=6, chi_max=128, precision=g.PREC_MIXED)
    a = g.gbsmps_estimate_bytes(64, o, 1000)
    assert a > 0
    assert g.gbsmps_estimate_bytes(128, o, 1000) > a
    assert g.gbsmps_estimate_bytes(64, o, 100000) > a
    o2 = g.opts_default(d=6, chi_max=256, precision=g.PREC_MIXED)
    assert g.gbsmps_estimate_bytes(64, o2, 1000) > a
    bad = g.opts_default(d=0)
    assert g.gbsmps_estimate_bytes(64, bad, 1000) == 0


def _est(N, chi, S=100, d=4):
    return g.gbsmps_estimate_bytes(N, g.opts_default(d=d, chi_max=chi), S)


def test_budget_never_exceeded_and_all_complete():
    budget = 3 * _est(64, 64)
    with g.Server(slots=4, hbm_budget=budget, simulate_s_per_tensor=2e-4) as s:
        rs = np.random.default_rng(1)
        ids = [s.submit(None, 100, N=int(n), d=4, chi_max=64) for n in rs.integers(16, 65, 24)]
        infos = [s.wait(i, timeout_s=60)[1] for i in ids]
        st = s.stats()
    assert st["completed"] == 24 and st["failed"] == 0
    assert st["hbm_peak"] <= budget and st["hbm_in_use"] == 0
    # at no instant do the running jobs' estimates exceed the budget
    ev = sorted([(x["t_admit"], x["hbm_bytes"]) for x in infos] +
                [(x["t_done"], -x["hbm_bytes"]) for x in infos], key=lambda e: (e[0], e[1]))
    cur = 0
    for _, b in ev:
        cur += b
        assert cur <= budget
    # the budget admits three jobs at a time: some overlap happened
    assert max(sum(1 for y in infos if y["t_admit"] <= x["t_admit"] < y["t_done"]) for x in infos) >= 2


def test_slots_refill_as_jobs_finish():
    """Requests arriving while others run are admitted as soon as a slot
    frees up: with 2 slots and 6 equal jobs the makespan is ~3 job times."""
    with g.Server(slots=2, hbm_budget=1 << 40, simulate_s_per_tensor=1e-3) as s:
        t0 = time.time()
        ids = [s.submit(None, 10, N=50) for _ in range(2)]
        time.sleep(0.02)
        ids += [s.submit(None, 10, N=50) for _ in range(4)]
        infos = [s.wait(i, timeout_s=30)[1] for i in ids]
        wall = time.time() - t0
    assert 0.14 < wall < 0.6
    slots = [x["slot"] for x in infos]
    assert set(slots) == {0, 1}
    late = sorted(infos[2:], key=lambda x: x["t_admit"])
    first_done = min(x["t_done"] for x in infos[:2])
    assert late[0]["t_admit"] >= first_done - 1e-3    # admitted when a slot freed


def test_small_jobs_pass_a_waiting_large_one_without_starving_it():
    small, large = _est(20, 32), _est(200, 256)
    budget = large + small // 2        # the large job cannot run beside a small one
    with g.Server(slots=3, hbm_budget=budget, simulate_s_per_tensor=1e-3) as s:
        a = s.submit(None, 10, N=20, chi_max=32)          # running first
        b = s.submit(None, 10, N=200, chi_max=256)        # waits for memory
        cs = [s.submit(None, 10, N=20, chi_max=32) for _ in range(3)]
        ia, ib = s.wait(a, 30)[1], s.wait(b, 30)[1]
        ics = [s.wait(c, 30)[1] for c in cs]
    assert ib["t_admit"] >= ia["t_done"] - 1e-3
    assert any(x["t_admit"] < ib["t_admit"] for x in ics)    # small ones went past it
    assert ib["state"] == 2


def test_oversized_request_rejected_and_bad_args():
    with g.Server(slots=1, hbm_budget=_est(16, 16), simulate_s_per_tensor=1e-4) as s:
        with pytest.raises(g.GbsmpsError) as e:
            s.submit(None, 10, N=512, chi_max=512)
        assert e.value.code == g.ERR_OOM
        with pytest.raises(g.GbsmpsError):
            s.submit(None, 10, N=0)
        with pytest.raises(g.GbsmpsError) as e2:
            s.wait(12345, 1.0)
        assert e2.value.code == g.ERR_ARG


def test_latency_stats_nearest_rank():
    with g.Server(slots=1, hbm_budget=1 << 40, simulate_s_per_tensor=1e-3) as s:
        ids = [s.submit(None, 1, N=10) for _ in range(5)]
        s.drain(30)
        lat = sorted(1e3 * (x["t_done"] - x["t_submit"]) for x in (s.wait(i)[1] for i in ids))
        st = s.stats()
    assert st["completed"] == 5 and st["tensors"] == 50
    # one slot, five 10 ms jobs submitted together: latencies ~10, 20, .., 50 ms
    assert st["p50_ms"] == pytest.approx(lat[2], abs=1e-6)
    assert st["p99_ms"] == pytest.approx(lat[4], abs=1e-6)
    assert lat[4] > 4 * lat[0] * 0.8


def test_batched_admission_groups_queued_jobs():
    """With batch_max > 1 a slot that admits a job takes the admissible
    queued jobs with it (one batched build), never more than batch_max, and
    never beyond the memory budget; alone in the queue a job runs alone."""
    budget = 5 * _est(40, 64)
    with g.Server(slots=1, hbm_budget=budget, simulate_s_per_tensor=1e-3, batch_max=4) as s:
        first = s.submit(None, 10, N=40, d=4, chi_max=64)
        time.sleep(0.01)                         # the first one starts alone
        ids = [s.submit(None, 10, N=40, d=4, chi_max=64) for _ in range(9)]
        infos = [s.wait(i, timeout_s=60)[1] for i in [first] + ids]
        st = s.stats()
    assert infos[0]["batch"] == 1
    sizes = [x["batch"] for x in infos[1:]]
    assert max(sizes) == 4 and all(1 <= b <= 4 for b in sizes)
    assert st["completed"] == 10 and st["hbm_peak"] <= budget and st["hbm_in_use"] == 0
    assert sum(1 for b in sizes if b == 4) >= 4
    with pytest.raises(g.GbsmpsError):
        g.Server(slots=1, hbm_budget=budget, simulate_s_per_tensor=1e-3, batch_max=0)
