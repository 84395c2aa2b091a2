"""The spectral point-mass filter, step by step in float64 (oracle).

State: weights P on an equidistant grid (eq. PDF_pm) held in an affine frame
x = c + M u, with u_m = j_m - (N_m - 1)/2 (index units, unit spacing, so the
periodic box length along axis m is L_m = N_m).  The frame moves with the
dynamics (eq. gridMov): over a time update of length tau, c <- e^{A tau} c and
M <- e^{A tau} M.  In u-coordinates the moved-frame Fokker-Planck equation
(eq. easyFPE) reads

    dP/dt = -trace(A) P + 1/2 sum_ab Q_u,ab(t) d_a d_b P,
    Q_u(t) = M(t)^{-1} Q M(t)^{-T},

which for a diagonal M is the paper's per-axis form with L_m = N_m delta_m.

Readings where the paper is silent or inconsistent (each listed in the design
notes of the repository):
  * trace factor (1 - dt trace(A))^l (sign that conserves mass, eq. easyFPE);
  * l diffusion factors evaluated at the sub-step ends t_k + n dt, n = 1..l;
  * cross terms of a non-diagonal Q_u use the first-derivative coefficients
    (Nyquist = 0), diagonal terms the second-derivative ones (Nyquist kept);
  * regridding at the head of each time update: the box covers +-span
    standard deviations of the predicted covariance pulled back by
    e^{-A tau}; per-axis rescale + recentre by the trigonometric interpolant
    (eq. interFreq), or, when the whitened correlation of the frame exceeds
    ``realign_rho``, a re-aligned frame filled by multilinear interpolation
    (default) or, in the band-limited mode, by n_x line-wise passes of the
    trigonometric interpolant (shear_realign, shear_realign_nd); points
    outside the old box get weight 0;
  * the separable regrid is quantised: the centre moves by a multiple of 1/64
    of a node towards the mean and each axis scale by a factor with an 8-bit
    mantissa, so the grid geometry is exact in any precision and does not
    random-walk with the rounding of the moments; a re-aligned frame has its
    centre on the same 1/64-node lattice and its axis entries rounded to a
    12-bit mantissa;
  * weights normalised so that |det M| sum P = 1 (eq. PDF_pm, c = delta sum P);
  * moments are point sums (no cell-variance term).
"""
from __future__ import annotations

import itertools
import math

import numpy as np

from . import model, spectral


class Degenerate(RuntimeError):
    """Normaliser zero or non-finite (state left unchanged)."""


def grid_u(N: int) -> np.ndarray:
    """Centred node coordinates u_j = j - (N-1)/2."""
    return np.arange(N) - (N - 1) / 2.0


def frame_points(c: np.ndarray, M: np.ndarray, N) -> np.ndarray:
    """All grid points x = c + M u in C order (last axis fastest); shape (P, n)."""
    us = np.meshgrid(*[grid_u(n) for n in N], indexing="ij")
    U = np.stack([u.ravel() for u in us], axis=1)
    return c[None, :] + U @ M.T


def _first_interp_axis(P: np.ndarray, axis: int, pos: np.ndarray, N: int) -> np.ndarray:
    """Trig-interpolate P along ``axis`` at node-relative positions ``pos``; 0 outside the box."""
    u_old = pos - (N - 1) / 2.0
    E = spectral.interp_matrix(N, pos)
    E[np.abs(u_old) > N / 2.0, :] = 0.0
    return spectral.apply_along_axis(E, P, axis)


def multilinear(P: np.ndarray, z: np.ndarray) -> np.ndarray:
    """Multilinear interpolation of the node array P at index coordinates z (Q, n).

    Nodes outside 0..N_m-1 contribute zero.
    """
    n = P.ndim
    f = np.floor(z)
    w = z - f
    f = f.astype(np.int64)
    out = np.zeros(z.shape[0])
    for corner in range(1 << n):
        idx = []
        wt = np.ones(z.shape[0])
        ok = np.ones(z.shape[0], dtype=bool)
        for m in range(n):
            b = (corner >> m) & 1
            i = f[:, m] + b
            wt = wt * (w[:, m] if b else 1.0 - w[:, m])
            ok &= (i >= 0) & (i < P.shape[m])
            idx.append(np.clip(i, 0, P.shape[m] - 1))
        out += np.where(ok, wt * P[tuple(idx)], 0.0)
    return out


def shear_realign(P: np.ndarray, B: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Band-limited re-alignment of a 2-D grid: the trigonometric interpolant
    (eq. interFreq) of the old weights P evaluated at u_old = B u_new + b, as
    two line-wise passes (the affine map factored into a per-line 1-D affine
    map along one axis, then one along the other):

      pass 1, along axis q for each old node i of axis p:
        h(i, v) = f(u_p = i, u_q = c_i + d v),
        c_i = (B_qp / B_pp) (i - b_p) + b_q,   d = det(B) / B_pp;
      pass 2, along axis p for each new node v of axis q:
        P'(w, v) = h(u_p = B_pp w + B_pq v + b_p, v),

    with (p, q) chosen to make the line-dependent shift of pass 1 the smaller
    one: (0, 1) when |B_10 / B_00| <= |B_01 / B_11|, else (1, 0).  Each pass is
    the 1-D interpolant at per-line positions, so it is exact for
    trigonometric polynomials along its axis, and the whole map is exact on
    them when B is triangular; positions outside the old box get weight 0.
    """
    N = P.shape
    p, q = (0, 1) if abs(B[1, 0]) * abs(B[1, 1]) <= abs(B[0, 1]) * abs(B[0, 0]) else (1, 0)
    Bpp, Bpq, Bqp, Bqq = B[p, p], B[p, q], B[q, p], B[q, q]
    d = (Bpp * Bqq - Bpq * Bqp) / Bpp
    Pp = np.moveaxis(P, p, 0)                     # [i (axis p), j (axis q)]
    Np, Nq = Pp.shape
    up, uq = grid_u(Np), grid_u(Nq)
    H = np.empty((Np, Nq))
    for i in range(Np):
        pos = (Bqp / Bpp) * (up[i] - b[p]) + b[q] + d * uq      # u_q positions on line i
        E = spectral.interp_matrix(Nq, pos + (Nq - 1) / 2.0)
        E[np.abs(pos) > Nq / 2.0, :] = 0.0
        H[i] = E @ Pp[i]
    out = np.empty((Np, Nq))
    for v in range(Nq):
        pos = Bpp * up + Bpq * uq[v] + b[p]                      # u_p positions on column v
        E = spectral.interp_matrix(Np, pos + (Np - 1) / 2.0)
        E[np.abs(pos) > Np / 2.0, :] = 0.0
        out[:, v] = E @ H[:, v]
    return np.moveaxis(out, 0, p)


def shear_orders(n: int) -> tuple:
    """Axis orders of the n-pass factorisation, in lexicographic order (the
    order in which ties are broken)."""
    return tuple(itertools.permutations(range(n)))


SHEAR_ORDERS_3D = shear_orders(3)


def shear_passes(B: np.ndarray, b: np.ndarray):
    """Factor u_old = B w + b into n line-wise passes (n = 2, 3 or 4).

    With an axis order (a_1, ..., a_n), pass k (applied to the data in the
    order k = n, ..., 1) resamples along axis a_k; on its array the axes
    S = {a_1..a_{k-1}} still carry old coordinates u_S and T = {a_k..a_n} new
    ones w_T, and the old coordinate a_k sits at
        u_{a_k} = alpha . u_S + beta . w_T + gamma,
        alpha = B[a_k, S] B[S, S]^{-1},  beta = B[a_k, T] - alpha B[S, T],
        gamma = b[a_k] - alpha b[S]
    (eliminating w_S from the rows S of the map).  The order minimises the
    largest |alpha| (the line-dependent shifts); orders within a relative
    1e-9 of the minimum count as tied (orders that share their alpha sets tie
    exactly in real arithmetic, so the choice must not depend on rounding)
    and the first tied one in lexicographic order (shear_orders) is taken; for
    n = 2 this is the rule of shear_realign.  Returns
    [(axis, coefficient per axis (n-vector over all axes), gamma)] in data
    order (k = n first)."""
    n = B.shape[0]
    orders = shear_orders(n)
    cands = []
    for order in orders:
        val, ok, passes = 0.0, True, []
        for k in range(n, 0, -1):
            a, S, T = order[k - 1], list(order[:k - 1]), list(order[k - 1:])
            if S:
                BSS = B[np.ix_(S, S)]
                if abs(np.linalg.det(BSS)) <= 1e-12 * max(1.0, np.abs(BSS).max()) ** len(S):
                    ok = False
                    break
                alpha = B[a, S] @ np.linalg.inv(BSS)
                val = max(val, np.abs(alpha).max())
            else:
                alpha = np.zeros(0)
            beta = B[a, T] - (alpha @ B[np.ix_(S, T)] if S else 0.0)
            gamma = b[a] - (alpha @ b[S] if S else 0.0)
            coef = np.zeros(n)
            coef[S] = alpha
            coef[T] = beta
            passes.append((a, coef, float(gamma)))
        if ok:
            cands.append((val, passes))
    if not cands:
        raise Degenerate("re-alignment map has a singular leading block in every order")
    vmin = min(v for v, _ in cands)
    return next(p for v, p in cands if v <= vmin * (1.0 + 1e-9))


def shear_realign_nd(P: np.ndarray, B: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Band-limited re-alignment in n = 2, 3 or 4 dimensions: the passes of
    shear_passes, each the 1-D trigonometric interpolant (eq. interFreq) of
    every line along its axis at that line's positions (coordinate value of
    the other axes times their coefficients, plus gamma, plus the running
    coefficient times the new node); positions outside the old box get 0."""
    G = np.array(P, dtype=float)
    N = G.shape
    for a, coef, gamma in shear_passes(np.asarray(B, float), np.asarray(b, float)):
        Ga = np.moveaxis(G, a, -1)                    # lines along a, other axes in order
        others = [m for m in range(G.ndim) if m != a]
        grids = np.meshgrid(*[grid_u(N[m]) for m in others], indexing="ij")
        offset = gamma + sum(coef[m] * g for m, g in zip(others, grids))
        ua = grid_u(N[a])
        out = np.empty_like(Ga)
        for idx in np.ndindex(*Ga.shape[:-1]):
            pos = offset[idx] + coef[a] * ua
            E = spectral.interp_matrix(N[a], pos + (N[a] - 1) / 2.0)
            E[np.abs(pos) > N[a] / 2.0, :] = 0.0
            out[idx] = E @ Ga[idx]
        G = np.moveaxis(out, -1, a)
    return G


SHIFT_QUANTUM = 1.0 / 64.0
SCALE_MANTISSA_BITS = 8


def quantize_shift(s: np.ndarray) -> np.ndarray:
    """Frame-centre shift in old-node units, rounded to a multiple of 1/64 node."""
    return np.rint(np.asarray(s) / SHIFT_QUANTUM) * SHIFT_QUANTUM


def quantize_scale(d: float) -> float:
    """Axis rescale factor rounded to an 8-bit mantissa (relative step 2^-8)."""
    f, e = math.frexp(d)
    return math.ldexp(round(math.ldexp(f, SCALE_MANTISSA_BITS)), e - SCALE_MANTISSA_BITS)


MATRIX_MANTISSA_BITS = 12


def quantize_matrix(M: np.ndarray) -> np.ndarray:
    """Re-aligned frame axes, each entry rounded to a 12-bit mantissa."""
    f, e = np.frexp(np.asarray(M, dtype=float))
    return np.ldexp(np.rint(np.ldexp(f, MATRIX_MANTISSA_BITS)), e - MATRIX_MANTISSA_BITS)


class OracleFilter:
    """Float64 spectral point-mass filter for one model (one state dimension n_x <= 4)."""

    def __init__(self, cfg, psi_mode: str = "euler", realign_mode: str = None):
        self.cfg = cfg
        self.n = cfg.nx
        if realign_mode is None:
            realign_mode = getattr(cfg, "realign_mode", "multilinear")
        if realign_mode not in ("multilinear", "shear") or (realign_mode == "shear" and cfg.nx == 1):
            raise ValueError("realign_mode: 'multilinear', or 'shear' for n_x = 2, 3 or 4")
        self.realign_mode = realign_mode
        self.N = tuple(int(v) for v in cfg.N)
        self.A = np.asarray(cfg.A, dtype=float)
        self.Q = np.asarray(cfg.Q, dtype=float)
        self.psi_mode = psi_mode
        # Initial frame: centred on m0, spanning +-span sigma of P0 per whitened axis.
        L0 = np.linalg.cholesky(cfg.P0)
        self.c = np.asarray(cfg.m0, dtype=float).copy()
        self.M = L0 @ np.diag([2.0 * cfg.span / n for n in self.N])
        x = frame_points(self.c, self.M, self.N)
        d = x - cfg.m0[None, :]
        q = np.einsum("pi,ij,pj->p", d, np.linalg.inv(cfg.P0), d)
        self.P = np.exp(-0.5 * q).reshape(self.N)
        self.normalise()
        self.last_regrid = None

    # --- density bookkeeping (eq. PDF_pm) ---------------------------------
    @property
    def cell_volume(self) -> float:
        return abs(np.linalg.det(self.M))

    def normalise(self) -> float:
        s = self.P.sum()
        cst = self.cell_volume * s
        if not np.isfinite(cst) or cst <= 0.0:
            raise Degenerate("normalisation constant is zero or not finite")
        self.P = self.P / cst
        return cst

    def points(self) -> np.ndarray:
        return frame_points(self.c, self.M, self.N)

    def moments(self):
        """Mean and covariance as point sums: m = V sum P x, C = V sum P (x-m)(x-m)^T."""
        x = self.points()
        w = self.P.ravel() * self.cell_volume
        m = w @ x
        d = x - m[None, :]
        C = (d * w[:, None]).T @ d
        return m, 0.5 * (C + C.T)

    def pdf(self) -> np.ndarray:
        return self.P.copy()

    # --- measurement update (eq. filt) -------------------------------------
    def meas_update(self, meas, z) -> None:
        """Posterior weights: predictive weights times the likelihood, normalised.

        The likelihood exp(-1/2 r^T R^{-1} r) (or, for the terrain measurement,
        the Gaussian-mixture density of Sec. VI) is shifted by its smallest
        exponent over the grid (a constant factor, removed by normalisation).
        """
        x = self.points()
        params = getattr(meas, "params", None)
        r = model.residual(meas.kind, np.atleast_1d(z), x, meas.H, params)
        if meas.kind == "terrain_gm":
            e = model.gm_neg_log_lik(r[:, 0], params)     # -log of the mixture likelihood
        else:
            Ri = np.linalg.inv(meas.R)
            e = 0.5 * np.einsum("pi,ij,pj->p", r, Ri, r)
        lik = np.exp(-(e - e.min()))
        old = self.P
        self.P = self.P * lik.reshape(self.N)
        try:
            self.normalise()
        except Degenerate:
            self.P = old
            raise

    # --- time update ---------------------------------------------------------
    def substeps(self, tau: float) -> int:
        return max(1, int(math.ceil(tau / self.cfg.dt_sub - 1e-9)))

    def choose_frame(self, tau: float) -> dict:
        """The regrid decision of the time update over tau (reading of Sec. V):
        re-aligned frame (Mnew, centre m) when the whitened correlation of the
        pulled-back predicted covariance exceeds realign_rho, otherwise the
        per-axis scales D and the centre shift s (both quantised)."""
        n = self.n
        m, C = self.moments()
        Phi, Qd = model.van_loan(self.A, self.Q, tau)
        Ppred = Phi @ C @ Phi.T + Qd
        Phinv = np.linalg.inv(Phi)
        S = Phinv @ Ppred @ Phinv.T
        Minv = np.linalg.inv(self.M)
        Su = Minv @ S @ Minv.T
        sd = np.sqrt(np.diag(Su))
        rho = 0.0
        for a in range(n):
            for b in range(a + 1, n):
                rho = max(rho, abs(Su[a, b]) / (sd[a] * sd[b]))
        span = self.cfg.span
        if n >= 2 and rho > self.cfg.realign_rho:
            Lp = np.linalg.cholesky(0.5 * (Ppred + Ppred.T))
            Mnew = quantize_matrix(Phinv @ Lp @ np.diag([2.0 * span / Nm for Nm in self.N]))
            s = quantize_shift(Minv @ (m - self.c))
            return {"realigned": True, "rho": rho, "M": Mnew, "s": s}
        D = np.array([quantize_scale(2.0 * span * sd[a] / self.N[a]) for a in range(n)])
        s = quantize_shift(Minv @ (m - self.c))
        return {"realigned": False, "rho": rho, "D": D, "s": s}

    def regrid(self, tau: float, choice: dict = None) -> dict:
        """Re-centre and re-size the grid for the prediction over tau (head of the
        time update), with the decision of choose_frame (or the one given)."""
        n = self.n
        ch = self.choose_frame(tau) if choice is None else choice
        Minv = np.linalg.inv(self.M)
        m = self.c + self.M @ ch["s"]
        if ch["realigned"]:
            Mnew = ch["M"]
            if self.realign_mode == "shear":
                # u_old = Minv (c' + M' u_new - c) = B u_new + b
                shear = shear_realign if n == 2 else shear_realign_nd
                self.P = shear(self.P, Minv @ Mnew, Minv @ (m - self.c))
            else:
                x = frame_points(m, Mnew, self.N)
                u_old = (x - self.c[None, :]) @ Minv.T
                zidx = u_old + (np.array(self.N) - 1) / 2.0
                self.P = multilinear(self.P, zidx).reshape(self.N)
        else:
            D = ch["D"]
            Mnew = self.M @ np.diag(D)
            P = self.P
            for a in range(n):
                pos = ch["s"][a] + D[a] * grid_u(self.N[a]) + (self.N[a] - 1) / 2.0
                P = _first_interp_axis(P, a, pos, self.N[a])
            self.P = P
        self.c = m.copy()
        self.M = Mnew
        self.normalise()
        self.last_regrid = {"realigned": ch["realigned"], "rho": ch["rho"]}
        return self.last_regrid

    def diffusion_multiplier(self, tau: float):
        """Psi on the DFT index grid and the trace factor (Sec. V-B algorithm, steps 2-4)."""
        n = self.n
        c2 = [spectral.c2_coeffs(Nm, float(Nm)) for Nm in self.N]
        c1 = [spectral.c1_coeffs(Nm, float(Nm)) for Nm in self.N]
        C2 = np.meshgrid(*c2, indexing="ij")
        C1 = np.meshgrid(*c1, indexing="ij")
        trA = np.trace(self.A)
        if self.psi_mode == "exact":
            Qb = model.backward_diffusion_integral(self.A, self.Q, tau)
            Mi = np.linalg.inv(self.M)
            Qu = Mi @ Qb @ Mi.T
            expo = np.zeros(self.N)
            for a in range(n):
                for b in range(n):
                    term = C2[a] if a == b else (C1[a] * C1[b]).real
                    expo = expo + 0.5 * Qu[a, b] * term
            return np.exp(expo), math.exp(-trA * tau)
        l = self.substeps(tau)
        dt = tau / l
        Psi = np.ones(self.N)
        for step in range(1, l + 1):
            Mt = model.expm(self.A * (step * dt)) @ self.M
            Mi = np.linalg.inv(Mt)
            Qu = Mi @ self.Q @ Mi.T
            psi = np.ones(self.N)
            for a in range(n):
                for b in range(n):
                    term = C2[a] if a == b else (C1[a] * C1[b]).real
                    psi = psi - 0.5 * dt * Qu[a, b] * term
            Psi = Psi / psi
        return Psi, (1.0 - dt * trA) ** l

    def spectral_step(self, tau: float) -> None:
        """Algorithm of Sec. V-B on the current frame, then the frame moves by e^{A tau}."""
        mass0 = self.cell_volume * self.P.sum()
        Pc = self.P.astype(complex)
        for a in range(self.n):                      # step 1: DFT per dimension
            Pc = spectral.apply_along_axis(spectral.dft_matrix(self.N[a]), Pc, a)
        Psi, g = self.diffusion_multiplier(tau)      # steps 2-3
        Pc = Psi * Pc * g                            # step 4
        for a in range(self.n):                      # step 5: inverse per dimension
            Pc = spectral.apply_along_axis(spectral.synthesis_matrix(self.N[a]), Pc, a)
        scale = max(1e-300, np.abs(Pc.real).max())
        if np.abs(Pc.imag).max() > 1e-10 * scale:
            raise AssertionError("spectral update produced a non-real density")
        self.P = Pc.real
        Phi = model.expm(self.A * tau)               # grid movement (eq. gridMov)
        self.c = Phi @ self.c
        self.M = Phi @ self.M
        self.last_mass_ratio = self.cell_volume * self.P.sum() / mass0
        self.normalise()                             # step 6

    def time_update(self, tau: float, choice: dict = None) -> dict:
        info = self.regrid(tau, choice)
        self.spectral_step(tau)
        return info
