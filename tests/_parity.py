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


def frame_choice_error(orc, tau, choice):
    """Distance of a regrid decision from the oracle's own one: the branch
    (0 if equal, inf if not) or the relative difference of the new axes/scales."""
    own = orc.choose_frame(tau)
    if own["realigned"] != choice["realigned"]:
        return float("inf")
    if own["realigned"]:
        return float(np.abs(own["M"] - choice["M"]).max() / np.abs(own["M"]).max())
    return float(np.abs(own["D"] - choice["D"]).max() / np.abs(own["D"]).max())


def run_pair(sc, precision="fp64", epochs=None, psi_mode="euler", fused_step=False, follow_frame=False,
             transform="auto"):
    """Yield (stage, errors) after every update of both filters.

    follow_frame: the oracle takes each regrid decision (centre shift, scales
    or re-aligned axes, all on their quantisation lattices) from the CUDA path
    instead of from its own moments, and the distance between the two
    decisions is reported as "choice".  The decision is a discrete function of
    the moments; on a float32 path whose moments differ from the oracle's in
    the sixth digit it can land on a neighbouring lattice point, and both
    frames are then valid grids for the method."""
    from paper_2412_07240_gb300 import Filter
    gpu = Filter(sc.cfg, precision=precision, psi_mode=psi_mode, transform=transform)
    orc = OracleFilter(sc.cfg, psi_mode=psi_mode)
    yield "prior", compare(gpu, orc)
    for k in range(epochs or sc.epochs):
        if fused_step:
            gpu.step(sc.meas, sc.z[k], sc.dt)
            orc.meas_update(sc.meas, sc.z[k])
            orc.time_update(sc.dt)
            yield f"step{k}", compare(gpu, orc)
            continue
        gpu.meas_update(sc.meas, sc.z[k])
        orc.meas_update(sc.meas, sc.z[k])
        yield f"meas{k}", compare(gpu, orc)
        gpu.time_update(sc.dt)
        choice, extra = None, {}
        if follow_frame:
            _, c, M = gpu.pdf()
            choice = orc.frame_from_target(sc.dt, c, M)
            extra["choice"] = frame_choice_error(orc, sc.dt, choice)
        info = orc.time_update(sc.dt, choice)
        yield f"time{k}" + ("R" if info["realigned"] else ""), {**compare(gpu, orc), **extra}
    gpu.close()


def max_errors(sc, **kw):
    worst = {}
    log = []
    for stage, e in run_pair(sc, **kw):
        log.append((stage, e))
        for k, v in e.items():
            worst[k] = max(worst.get(k, 0.0), v)
    return worst, log
