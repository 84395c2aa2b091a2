"""Shared helpers of the GPU parity tests: run the CUDA path (through the C-ABI
binding) and the float64 oracle on the same seeded inputs, update by update."""
import numpy as np

from oracle.filter import OracleFilter


def rel_l1(p, ref):
    return float(np.abs(p - ref).sum() / np.abs(ref).sum())


def compare(gpu, orc):
    """Relative L1 of the weights, frame and moment differences after one update."""
    P, c, M = gpu.pdf()
    out = {"l1": rel_l1(P, orc.P)}
    m, C = gpu.moments()
    mo, Co = orc.moments()
    # frame: centre shift relative to the spread, axis matrix relative to its size
    out["frame"] = float(max(np.abs(c - orc.c).max() / np.sqrt(abs(np.trace(Co))),
                             np.abs(M - orc.M).max() / np.abs(orc.M).max()))
    out["mean"] = float(np.abs(m - mo).max() / np.sqrt(abs(np.trace(Co))))
    out["cov"] = float(np.abs(C - Co).max() / np.abs(Co).max())
    return out


def frame_offset(orc, c, M):
    """Where the nodes of the frame (c, M) sit in the oracle's frame: the largest
    displacement |M_o^{-1}(c + M u - c_o) - u| over the nodes u, in node units."""
    n = orc.n
    Mi = np.linalg.inv(orc.M)
    B = Mi @ np.asarray(M, dtype=float).reshape(n, n) - np.eye(n)
    b = Mi @ (np.asarray(c, dtype=float) - orc.c)
    corners = np.array(np.meshgrid(*[[-(N - 1) / 2.0, (N - 1) / 2.0] for N in orc.N], indexing="ij"))
    corners = corners.reshape(n, -1)
    return float(np.abs(B @ corners + b[:, None]).max())


def displacement_bound(orc, c, M):
    """First-order change of the oracle's own relative-L1 weights if its nodes
    sat on the frame (c, M) instead: sum_j |grad_u P(u_j) . du_j| / sum_j P_j,
    du_j the node displacement in oracle node units, grad_u by centred
    differences on the oracle's grid.  Zero when the frames coincide."""
    n = orc.n
    Mi = np.linalg.inv(orc.M)
    B = Mi @ np.asarray(M, dtype=float).reshape(n, n) - np.eye(n)
    b = Mi @ (np.asarray(c, dtype=float) - orc.c)
    if not np.any(B) and not np.any(b):
        return 0.0
    u = np.stack(np.meshgrid(*[np.arange(N) - (N - 1) / 2.0 for N in orc.N], indexing="ij"))
    du = np.tensordot(B, u, axes=1) + b.reshape((n,) + (1,) * n)
    P = orc.P
    dot = np.zeros_like(P)
    for a in range(n):
        dot += 0.5 * (np.roll(P, -1, axis=a) - np.roll(P, 1, axis=a)) * du[a]
    return float(np.abs(dot).sum() / np.abs(P).sum())


def run_pair(sc, precision="fp64", epochs=None, psi_mode="euler", fused_step=False, transform="auto"):
    """Yield (stage, errors) after every update of both filters, each on its
    own regrid decisions.  Besides the weight, frame and moment differences,
    "offset" is the largest node displacement between the two frames (node
    units) and "shift_bound" the first-order change of the oracle's weights
    that this displacement alone would cause (zero when the frames coincide)."""
    from paper_2412_07240_gb300 import Filter
    gpu = Filter(sc.cfg, precision=precision, psi_mode=psi_mode, transform=transform)
    orc = OracleFilter(sc.cfg, psi_mode=psi_mode)

    def cmp():
        e = compare(gpu, orc)
        _, c, M = gpu.pdf()
        e["offset"] = frame_offset(orc, c, M)
        e["shift_bound"] = displacement_bound(orc, c, M)
        return e
    yield "prior", cmp()
    for k in range(epochs or sc.epochs):
        if fused_step:
            gpu.step(sc.meas, sc.z[k], sc.dt)
            orc.meas_update(sc.meas, sc.z[k])
            orc.time_update(sc.dt)
            yield f"step{k}", cmp()
            continue
        gpu.meas_update(sc.meas, sc.z[k])
        orc.meas_update(sc.meas, sc.z[k])
        yield f"meas{k}", cmp()
        gpu.time_update(sc.dt)
        info = orc.time_update(sc.dt)
        yield f"time{k}" + ("R" if info["realigned"] else ""), cmp()
    gpu.close()


def max_errors(sc, **kw):
    worst = {}
    log = []
    for stage, e in run_pair(sc, **kw):
        log.append((stage, e))
        for k, v in e.items():
            worst[k] = max(worst.get(k, 0.0), v)
    return worst, log


def check_own_decisions(log, bar=1e-5, cov_factor=10.0, frame_max=1e-3, start=0):
    """Parity of a float32 path against the oracle on its own regrid decisions.

    The regrid decision is a quantised function of the moments; float32
    moments can put it on a neighbouring lattice point, and both frames are
    valid grids.  Where the frames coincide the weights are held to `bar`.
    Where they differ, the sampled weights of the same density on the two
    grids differ to first order by the node displacement times the density's
    gradient (shift_bound), and that difference is carried by the later
    updates; the weights are then held to bar + 2 x the largest shift_bound
    seen so far (the factor covers the centred-difference estimate of the
    gradient on coarse grids).  The frames must stay within `frame_max` of
    each other, and the moments, which do not depend on the grid, within
    `bar` (mean) and cov_factor x bar (covariance) throughout."""
    carried = 0.0
    for k, (stage, e) in enumerate(log):
        carried = max(carried, e.get("shift_bound", 0.0))
        if k < start:
            continue
        assert e["l1"] <= bar + 2.0 * carried, (stage, e, carried)
        assert e["frame"] <= frame_max, (stage, e)
        assert e["mean"] <= bar and e["cov"] <= cov_factor * bar, (stage, e)
    return carried
