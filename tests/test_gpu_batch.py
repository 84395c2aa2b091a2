"""Batched filters: one launch per epoch, one CTA per filter, mixed grid sizes.

* every filter of a batch equals the same filter run alone (same kernel body),
  in FP16X3, BF16X6, BF16X3 and TF32 and with the exact-in-time multiplier;
* sampled filters equal the float64 oracle within the 1e-5 bar, in FP16X3
  and BF16X6;
* the full 4096-filter workload in the benchmarked launch configuration keeps
  unit mass, finite weights and PSD covariances, and its sampled filters match
  the oracle;
* per-item step options (shuffled subsets, measurement masks, changing taus,
  tau = 0) equal the same filters run alone;
* stepping a subset leaves the others untouched; a step rejected for a tau
  beyond the sub-step limit or an id listed twice steps nothing; admission by
  a memory budget.
"""
import numpy as np
import pytest

import workloads as w
from tests._parity import rel_l1

pytestmark = pytest.mark.gpu


def _c4(count, epochs, seed=4):
    cfgs, meas, dt, truth, z = w.c4_batch(count=count, seed=seed, epochs=epochs)
    return cfgs, meas, dt, z


# a last-bit difference of the inputs (the front kernel recomputes the
# likelihood exponents, which the compiler may contract differently) re-rounds
# the 16-bit (or TF32) operand splits; the weights far from the mass are the
# transforms' rounding noise (~1e-7 of the peak), different in the two: they
# agree to twice the precision's own resolution, each within the oracle bar
AGREE = {"fp16x3": 2e-6, "bf16x6": 2e-6, "bf16x3": 1e-4, "tf32": 3e-2}


@pytest.mark.parametrize("prec,psi", [("fp16x3", "euler"), ("bf16x6", "euler"), ("bf16x3", "euler"),
                                      ("tf32", "euler"), ("fp16x3", "exact")])
def test_batch_equals_single_filters(prec, psi):
    """The same filters run alone, in every precision and both multipliers (the
    single-filter path meets the oracle at those bars).  The batch splits the
    epoch into a front kernel (measurement update, moments, frame decision)
    and a transform kernel of the filter's size class, with the steps of the
    fused kernel; the front kernel recomputes the likelihood exponents instead
    of storing them (the compiler may contract their float32 products
    differently) and the size-64 class sums the final moments over fewer
    threads, so the two agree to the rounding of the format, on the same
    frames."""
    from paper_2412_07240_gb300 import Batch, Filter
    cfgs, meas, dt, z = _c4(10, 4)
    b = Batch(cfgs, [meas] * len(cfgs), precision=prec, psi_mode=psi)
    singles = [Filter(c, precision=prec, psi_mode=psi) for c in cfgs]
    ids = np.arange(len(cfgs))
    for k in range(4):
        b.step(ids, z[:, k], dt)
        for i, f in enumerate(singles):
            f.step(meas, z[i, k], dt)
    classes = set()
    for i, f in enumerate(singles):
        Pb, cb, Mb = b.pdf(i)
        Ps, cs, Ms = f.pdf()
        assert np.array_equal(cb, cs) and np.array_equal(Mb, Ms), i
        assert rel_l1(Pb, Ps) <= AGREE[prec], (i, rel_l1(Pb, Ps))
        m = max(cfgs[i].N)
        classes.add(64 if m <= 64 else 96 if m <= 96 else 128)
    assert classes == {64, 96, 128}


@pytest.mark.parametrize("prec", ["fp16x3", "bf16x6"])
def test_batch_matches_oracle(prec):
    from oracle.filter import OracleFilter
    from paper_2412_07240_gb300 import Batch
    cfgs, meas, dt, z = _c4(8, 4, seed=7)
    b = Batch(cfgs, [meas] * len(cfgs), precision=prec)
    orcs = [OracleFilter(c) for c in cfgs]
    ids = np.arange(len(cfgs))
    worst = 0.0
    for k in range(4):
        b.step(ids, z[:, k], dt)
        for i, o in enumerate(orcs):
            o.meas_update(meas, z[i, k])
            o.time_update(dt)
            worst = max(worst, rel_l1(b.pdf(i)[0], o.P))
    assert worst <= 1e-5, worst


def test_subset_step_leaves_others():
    from paper_2412_07240_gb300 import Batch
    cfgs, meas, dt, z = _c4(6, 2, seed=8)
    b = Batch(cfgs, [meas] * len(cfgs))
    before = [b.pdf(i)[0].copy() for i in range(6)]
    b.step([1, 4], z[[1, 4], 0], dt)
    for i in range(6):
        same = np.array_equal(b.pdf(i)[0], before[i])
        assert same == (i not in (1, 4))


def test_step_options_match_single_filters():
    """The per-item options of a batch step against the same filters run alone:
    ids in shuffled order and as changing subsets (the host places each item
    at its filter's position in the launch order by size class), measurement
    masks (a filter that skips its measurement only predicts), per-filter
    taus that change every two epochs (their time constants are recomputed
    and uploaded by the host), and tau = 0 (measurement only; with the mask
    also off, the filter is left as it was)."""
    from paper_2412_07240_gb300 import Batch, Filter
    cfgs, meas, dt, z = _c4(10, 6, seed=11)
    n = len(cfgs)
    b = Batch(cfgs, [meas] * n, precision="bf16x6")
    singles = [Filter(c, precision="bf16x6") for c in cfgs]
    rng = np.random.default_rng(5)
    untouched = 0
    for k in range(6):
        ids = rng.permutation(n)[: n - k % 3]
        taus = dt * (1.0 + 0.5 * ((ids + k // 2) % 3))
        if k == 4:
            taus[::4] = 0.0
        dm = ((ids + k) % 4 != 0).astype(np.int32)
        before = {i: b.pdf(i)[0].copy() for i, t, m in zip(ids, taus, dm) if t == 0.0 and not m}
        b.step(ids, z[ids, k], taus, do_meas=dm)
        for i, t, m in zip(ids, taus, dm):
            f = singles[i]
            if m and t > 0.0:
                f.step(meas, z[i, k], t)
            elif m:
                f.meas_update(meas, z[i, k])
            elif t > 0.0:
                f.time_update(t)
        for i, P0 in before.items():
            assert np.array_equal(b.pdf(i)[0], P0), i
            untouched += 1
    assert untouched >= 1
    classes = set()
    for i, f in enumerate(singles):
        Pb, cb, Mb = b.pdf(i)
        Ps, cs, Ms = f.pdf()
        assert np.array_equal(cb, cs) and np.array_equal(Mb, Ms), i
        assert rel_l1(Pb, Ps) <= AGREE["bf16x6"], (i, rel_l1(Pb, Ps))
        m = max(cfgs[i].N)
        classes.add(64 if m <= 64 else 96 if m <= 96 else 128)
    assert classes == {64, 96, 128}


def test_rejected_tau_steps_nothing():
    """A tau beyond the sub-step limit is rejected on the host before anything
    runs: no filter of the call is stepped, the filters listed before it keep
    their resident constants, and a retry with valid taus recomputes them (the
    filters then equal the same filters run alone)."""
    from paper_2412_07240_gb300 import Batch, Filter, PmfError
    cfgs, meas, dt, z = _c4(4, 1, seed=12)
    b = Batch(cfgs, [meas] * 4, precision="bf16x6")
    singles = [Filter(c, precision="bf16x6") for c in cfgs]
    ids = np.arange(4)
    before = [b.pdf(i)[0].copy() for i in range(4)]
    taus = np.array([2 * dt, 2 * dt, 2 * dt, 1.0])   # 1.0 needs 100 sub-steps of 0.01
    with pytest.raises(PmfError):
        b.step(ids, z[:, 0], taus)
    for i in range(4):
        assert np.array_equal(b.pdf(i)[0], before[i]), i
    taus[3] = 2 * dt
    b.step(ids, z[:, 0], taus)
    for i, f in enumerate(singles):
        f.step(meas, z[i, 0], 2 * dt)
    for i, f in enumerate(singles):
        Pb, cb, Mb = b.pdf(i)
        Ps, cs, Ms = f.pdf()
        assert np.array_equal(cb, cs) and np.array_equal(Mb, Ms), i
        assert rel_l1(Pb, Ps) <= AGREE["bf16x6"], (i, rel_l1(Pb, Ps))


def test_repeated_id_rejected():
    """An id listed twice in one step is an argument error and steps nothing."""
    from paper_2412_07240_gb300 import Batch, PmfError
    cfgs, meas, dt, z = _c4(3, 1, seed=13)
    b = Batch(cfgs, [meas] * 3, precision="bf16x6")
    before = [b.pdf(i)[0].copy() for i in range(3)]
    with pytest.raises(PmfError):
        b.step([0, 2, 0], z[[0, 2, 0], 0], dt)
    for i in range(3):
        assert np.array_equal(b.pdf(i)[0], before[i]), i
    b.step([0, 2], z[[0, 2], 0], dt)
    for i in range(3):
        assert np.array_equal(b.pdf(i)[0], before[i]) == (i == 1), i


def test_admission_by_budget():
    from paper_2412_07240_gb300 import Batch, PmfError
    from paper_2412_07240_gb300._binding import ERR_ADMISSION
    cfgs, meas, dt, z = _c4(32, 1, seed=9)
    with pytest.raises(PmfError) as e:
        Batch(cfgs, [meas] * len(cfgs), hbm_budget=1 << 20)
    assert e.value.code == ERR_ADMISSION


def _oracle_fails(cfg, meas, zs, dt, epochs):
    from oracle.filter import Degenerate, OracleFilter
    o = OracleFilter(cfg)
    try:
        for k in range(epochs):
            o.meas_update(meas, zs[k])
            m, C = o.moments()
            if not (np.all(np.isfinite(C)) and np.all(np.linalg.eigvalsh(C) > 0)):
                return True
            o.time_update(dt)
    except (Degenerate, np.linalg.LinAlgError, FloatingPointError, ValueError):
        return True
    return False


def test_full_c4_workload_sampled():
    """4096 filters, sizes from {32..128}^2, in the benchmarked launch configuration.

    A few seeded filters (strongly sheared dynamics on 32-48-node axes) are
    under-resolved after the first measurement; the oracle rings into negative
    lobes there as well.  The GPU may report them as degenerate; they must stay
    rare, and sampled healthy filters must match the oracle."""
    from oracle.filter import Degenerate, OracleFilter
    from paper_2412_07240_gb300 import Batch
    epochs = 3
    cfgs, meas, dt, z = _c4(4096, epochs)
    b = Batch(cfgs, [meas] * len(cfgs))
    ids = np.arange(len(cfgs))
    bad = np.zeros(len(cfgs), dtype=bool)
    for k in range(epochs):
        b.step(ids, z[:, k], dt)
        bad |= b.status() != 0
    assert bad.sum() <= 0.01 * len(cfgs), bad.sum()
    # a filter the GPU reports as degenerate is one the oracle cannot carry
    # either: its normaliser fails, its covariance stops being positive
    # definite, or its frame decision has no Cholesky factor
    for i in np.nonzero(bad)[0]:
        assert _oracle_fails(cfgs[i], meas, z[i], dt, epochs), i
    rng = np.random.default_rng(0)
    checked = 0
    for i in rng.permutation(len(cfgs)):
        if bad[i] or checked == 4:
            continue
        o = OracleFilter(cfgs[i])
        try:
            for k in range(epochs):
                o.meas_update(meas, z[i, k])
                assert np.all(np.linalg.eigvalsh(o.moments()[1]) > 0)
                o.time_update(dt)
        except (Degenerate, AssertionError):
            continue
        P, c, M = b.pdf(i)
        assert abs(abs(np.linalg.det(M)) * P.sum() - 1.0) < 1e-5
        assert rel_l1(P, o.P) <= 1e-5, (i, rel_l1(P, o.P))
        checked += 1
    assert checked == 4


@pytest.mark.parametrize("sigma", [0.1, 1e-3])
def test_linear_measurement_shift_paths(sigma):
    """A linear measurement's exponent shift: the box minimum of its quadratic
    (sigma = 0.1, the workload's), or the pass over the grid when the
    likelihood is sharper than a node (sigma = 1e-3: the box minimum may lie
    more than 40 below the grid's).  Measurement-only steps against the
    oracle's Bayes update (eq. filt); the shift cancels in the normalisation."""
    from oracle.filter import OracleFilter
    from paper_2412_07240_gb300 import Batch
    from workloads import MeasModel
    cfgs, _, dt, z = _c4(6, 1, seed=11)
    meas = MeasModel("linear", R=sigma ** 2 * np.eye(2), H=np.eye(2))
    b = Batch(cfgs, [meas] * len(cfgs))
    zz = np.array([c.m0 + 0.3 for c in cfgs])
    b.step(np.arange(len(cfgs)), zz, 0.0)
    for i, c in enumerate(cfgs):
        o = OracleFilter(c)
        o.meas_update(meas, zz[i])
        P, cc, M = b.pdf(i)
        assert np.allclose(cc, o.c, rtol=0, atol=1e-12) and np.allclose(M, o.M, rtol=1e-12, atol=0)
        assert rel_l1(P, o.P) <= 1e-5, (i, rel_l1(P, o.P))
