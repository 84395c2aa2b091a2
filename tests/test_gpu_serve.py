"""The request server: continuous batching of mixed 1-D / 2-D / 3-D filters.

Each filter's results through the server equal those of the same filter
served alone and of the single-filter API, and match the float64 oracle; the
full 10,000-filter workload at 200k requests/s, in the benchmarked
configuration, matches the oracle on sampled filters of each dimension."""
import numpy as np
import pytest

import workloads as w
from tests._parity import rel_l1

pytestmark = pytest.mark.gpu


def _small_workload(seed=7, duration=0.25, rate=8000.0):
    return w.c5_serving(n_filters=40, rate=rate, duration=duration, seed=seed, n1=(16, 96), n2=(16, 48),
                        n3=(16, 32))


def _server(wl, ids=None, budget=0):
    from paper_2412_07240_gb300 import Server
    s = Server(max_filters=len(wl.cfgs), hbm_budget=budget)
    ids = range(len(wl.cfgs)) if ids is None else ids
    fid = {i: s.admit(wl.cfgs[i], wl.meas[i]) for i in ids}
    return s, fid


def test_alone_equals_in_the_mix():
    wl = _small_workload()
    s, fid = _server(wl)
    lat, st = s.replay(wl.t_arrival, [fid[i] for i in wl.ids], wl.z, wl.taus)
    assert st["requests"] == wl.ids.size and np.all(lat >= 0)
    assert st["max_batch"] > 1   # requests shared batches
    for nx in (1, 2, 3):
        f = next(i for i, c in enumerate(wl.cfgs) if c.nx == nx and (wl.ids == i).sum() > 2)
        P_mix, c_mix, M_mix = s.pdf(fid[f])
        sel = wl.ids == f
        alone, afid = _server(wl, ids=[f])
        alone.replay(wl.t_arrival[sel], np.full(sel.sum(), afid[f]), wl.z[sel], wl.taus[sel])
        P_one, c_one, M_one = alone.pdf(afid[f])
        assert np.array_equal(P_mix, P_one), (nx, rel_l1(P_mix, P_one))
        assert np.array_equal(c_mix, c_one) and np.array_equal(M_mix, M_one), nx
        alone.close()
    s.close()


def test_server_matches_single_filter_api():
    from paper_2412_07240_gb300 import Filter
    wl = _small_workload(seed=8)
    s, fid = _server(wl)
    s.replay(wl.t_arrival, [fid[i] for i in wl.ids], wl.z, wl.taus)
    for nx in (1, 2, 3):
        f = next(i for i, c in enumerate(wl.cfgs) if c.nx == nx and (wl.ids == i).sum() > 2)
        sel = np.nonzero(wl.ids == f)[0]
        assert np.all(wl.taus[sel] <= 0.64)   # one time update per request
        g = Filter(wl.cfgs[f], precision="fp16x3")
        for r in sel:
            g.step(wl.meas[f], wl.z[r, :nx], wl.taus[r])
        P1, c1, M1 = g.pdf()
        P2, c2, M2 = s.pdf(fid[f])
        # 2-D requests run the batch's front and size-class kernels: the same
        # steps as the fused single-filter kernel, equal to float32 rounding
        if nx == 2:
            assert rel_l1(P2, P1) <= 2e-6, (nx, rel_l1(P2, P1))
        else:
            assert np.array_equal(P2, P1), (nx, rel_l1(P2, P1))
        assert np.array_equal(c2, c1) and np.array_equal(M2, M1), nx
        g.close()
    s.close()


def test_bf16x6_server_formats():
    """A BF16X6 server: its 2-D filters run the six-product BF16 split (equal
    to the single-filter API in that format to float32 rounding), its 3-D
    filters FP16X3 (equal to the single-filter API in FP16X3 bit for bit) and
    its 1-D filters the float32 kernel."""
    from paper_2412_07240_gb300 import Filter, Server
    wl = _small_workload(seed=8)
    s = Server(max_filters=len(wl.cfgs), precision="bf16x6")
    fid = {i: s.admit(wl.cfgs[i], wl.meas[i]) for i in range(len(wl.cfgs))}
    s.replay(wl.t_arrival, [fid[i] for i in wl.ids], wl.z, wl.taus)
    for nx, prec in ((1, "fp16x3"), (2, "bf16x6"), (3, "fp16x3")):
        f = next(i for i, c in enumerate(wl.cfgs) if c.nx == nx and (wl.ids == i).sum() > 2)
        sel = np.nonzero(wl.ids == f)[0]
        g = Filter(wl.cfgs[f], precision=prec)
        for r in sel:
            g.step(wl.meas[f], wl.z[r, :nx], wl.taus[r])
        P1, c1, M1 = g.pdf()
        P2, c2, M2 = s.pdf(fid[f])
        if nx == 2:
            assert rel_l1(P2, P1) <= 2e-6, (nx, rel_l1(P2, P1))
        else:
            assert np.array_equal(P2, P1), (nx, rel_l1(P2, P1))
        assert np.array_equal(c2, c1) and np.array_equal(M2, M1), nx
        g.close()
    s.close()


def test_server_against_oracle():
    from oracle.filter import OracleFilter
    wl = _small_workload(seed=9, duration=0.1)
    s, fid = _server(wl)
    s.replay(wl.t_arrival, [fid[i] for i in wl.ids], wl.z, wl.taus)
    for nx in (1, 2):
        f = next(i for i, c in enumerate(wl.cfgs) if c.nx == nx and (wl.ids == i).sum() > 1)
        o = OracleFilter(wl.cfgs[f])
        for r in np.nonzero(wl.ids == f)[0]:
            o.meas_update(wl.meas[f], wl.z[r, :nx])
            o.time_update(wl.taus[r])
        P, c, M = s.pdf(fid[f])
        assert rel_l1(P, o.P) < 1e-5, nx
    s.close()


def test_long_horizon_split_into_time_updates():
    # tau above PMF_MAX_SUBSTEPS * dt_sub runs as consecutive time updates
    from oracle.filter import OracleFilter
    from paper_2412_07240_gb300 import Server
    sc = w.c1_scenario(epochs=3)
    s = Server(max_filters=1)
    fid = s.admit(sc.cfg, sc.meas)
    taus = np.array([0.9, 0.3, 1.5])
    s.replay(np.zeros(3), [fid] * 3, sc.z[:3], taus)
    o = OracleFilter(sc.cfg)
    for k in range(3):
        o.meas_update(sc.meas, sc.z[k])
        left = taus[k]
        while left > 0:   # the same chunks: at most 64 sub-steps of 0.01
            t = min(left, 0.64 * (1 - 1e-12))
            o.time_update(t)
            left -= t
            if left < 1e-12 * 0.64:
                left = 0.0
    P, c, M = s.pdf(fid)
    assert rel_l1(P, o.P) < 1e-5
    s.close()


def test_admission_budget_and_eviction():
    from paper_2412_07240_gb300 import PmfError, Server
    from paper_2412_07240_gb300._binding import ERR_ADMISSION
    wl = _small_workload()
    s = Server(max_filters=len(wl.cfgs), hbm_budget=1 << 20)
    admitted = []
    with pytest.raises(PmfError) as e:
        for i in range(len(wl.cfgs)):
            admitted.append(s.admit(wl.cfgs[i], wl.meas[i]))
    assert e.value.code == ERR_ADMISSION
    assert admitted and s.bytes <= 1 << 20
    before = s.bytes
    s.evict(admitted[0])
    assert s.bytes < before
    s.admit(wl.cfgs[0], wl.meas[0])
    s.close()


def _oracle_replay(cfg, meas, zs, taus):
    """The oracle on one filter's requests, each horizon in the server's chunks
    (at most PMF_MAX_SUBSTEPS = 64 sub-steps of dt_sub per time update)."""
    from oracle.filter import OracleFilter
    o = OracleFilter(cfg)
    tmax = 64 * cfg.dt_sub * (1 - 1e-12)
    for z, tau in zip(zs, taus):
        o.meas_update(meas, z)
        left = float(tau)
        while left > 0:
            t = min(left, tmax)
            o.time_update(t)
            left -= t
            if left < 1e-12 * tmax:
                left = 0.0
    return o


def test_full_c5_workload_sampled():
    """10,000 resident filters (60% 1-D, 35% 2-D, 5% 3-D) served at 200k
    requests/s with FP16X3 and a 120 GB budget, as benchmarked; sampled filters
    of each dimension match the oracle on their own request sequences, and
    sampled moments are finite with positive definite covariances."""
    from oracle.filter import Degenerate
    from paper_2412_07240_gb300 import Server
    wl = w.c5_serving(n_filters=10000, rate=200e3, duration=0.02, seed=5)
    s = Server(max_filters=len(wl.cfgs), precision="fp16x3", hbm_budget=int(120e9))
    fid = np.array([s.admit(c, m) for c, m in zip(wl.cfgs, wl.meas)], dtype=np.int32)
    s.replay(wl.t_arrival, fid[wl.ids], wl.z, wl.taus)
    counts = np.bincount(wl.ids, minlength=len(wl.cfgs))
    rng = np.random.default_rng(0)
    order = rng.permutation(len(wl.cfgs))
    for nx, want in ((1, 3), (2, 3), (3, 1)):
        done = 0
        for i in order:
            if done == want:
                break
            if wl.cfgs[i].nx != nx or counts[i] == 0:
                continue
            r = np.nonzero(wl.ids == i)[0]
            try:
                o = _oracle_replay(wl.cfgs[i], wl.meas[i], wl.z[r, :nx], wl.taus[r])
            except Degenerate:
                continue
            P, c, M = s.pdf(fid[i])
            err = rel_l1(P, o.P)
            assert err <= 1e-5, (int(i), nx, len(r), err)
            done += 1
        assert done == want, (nx, done)
    for i in rng.choice(len(wl.cfgs), 200, replace=False):
        m, C = s.moments(fid[i])
        assert np.all(np.isfinite(m)) and np.all(np.linalg.eigvalsh(C) > 0), int(i)
    s.close()
