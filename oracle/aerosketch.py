"""AeroSketch, plain FP64 (oracle; test infrastructure only).

Only tests/, the smoke check and the bench's CPU-baseline leg may import this
package.  It shares no code with the CUDA path; the two meet only in the seeded
input generators (synth/) and in the published Philox definition that each
side implements on its own.

What it follows, step by step and in the paper's notation:

* Algorithm 1 (power iteration), with A = C'^T, so A^T A x = C' (C'^T x).
* Algorithm 2 (simultaneous iteration), with A = C'^T: K = A Pi, q products
  by A A^T, QR, M = Q^T A A^T Q, eigendecomposition of M, Z = Q U.
* Algorithm 3 (Initialize): l = ceil(2/eps) or given, C_0 = 0 (2l x d), queue S.
* Algorithm 4 (Update): insert, FD shrink when the buffer is full, the
  power-iteration gate, the doubling loop over k = 2, 4, ..., the selection of
  xi components, the snapshot (Z, Z^T C'^T C') and the residual C' - C' Z Z^T.
* Algorithm 5 (Query(lb, ub)): B = C^T C + the snapshot terms, eigendecomposition,
  shrink by lambda_l, top l rows.
* Algorithm 8 (ATTP): ||A_t||_F^2 += ||a_i||^2 and theta = eps ||A_t||_F^2
  before every Update.

Readings where the paper is silent or inconsistent (each one also listed in
the design notes of the repository):

 R1  The power-iteration vector lives in R^{2l} (Algorithm 1 applied to C'^T),
     including empty rows; k_PI = ceil(log2 d) + 1.
 R2  q = ceil(ln d / eps_SI) for the Theta(log d / eps_SI) of Algorithm 2.
 R3  K = (A A^T)^q A Pi is re-orthonormalised (Householder QR) after every
     product; the span, and so the Ritz pairs, are unchanged in exact arithmetic.
 R4  Pi is 2l x k and is drawn afresh for each doubling step j.
 R5  SVD(M) of the symmetric PSD M is its eigendecomposition, descending.
 R6  The gate is sigma^2 >= theta/2 (Algorithm 4); the loop stops when
     sigma_k^2 < theta; xi = #{sigma^2 >= theta}.  A gate or a selected
     component also needs sigma^2 > 0 (nothing to dump in a zero residual; this
     only matters when theta = 0, i.e. before any non-zero row).
 R7  xi = 0 (gate passed, nothing above theta): no snapshot, C = C'.
 R8  The trailing C_i <- C'_i of Algorithm 4 applies only when the doubling
     loop ends without a break.
 R9  After a shrink the kept rows are the singular directions in descending
     order at indices 0..l-2; the row counter is always l-1 and the next row is
     inserted at index l-1.
 R10 The sign of each singular pair (u_j, v_j) is fixed so that the entry of
     largest magnitude of u_j (the left singular vector, a 2l-vector) is
     positive, the lowest index winning exact ties.
 R11 The current-time query (lb = 0, ub = T) includes C_T (Algorithm 5).
 R17 Probability amplification (Algorithm 7, optional: delta): r and s are
     rounded up; SI h of the r draws its test matrix at sub-index
     j + 64 (h - 1) (h = 1 is the plain draw), estimate g of SI h its start
     vector at sub-index 64 h + g; the first minimum of the estimates wins.
     Estimates below tie_rel * theta are rounding noise of a zero residual:
     when replaying another run, any SI among them is a valid minimiser.
 R12 A historical query ub = t < T (Algorithm 8's Query(t) = Query(0, t)) has
     no residual C_t to add (it is not stored); B is the sum of the snapshot
     terms with t_j <= t, as in B_i of the ATTP error analysis.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import philox


def default_k_pi(d: int) -> int:
    """Corollary 1: k = ceil(log2 d) + 1."""
    return int(math.ceil(math.log2(d))) + 1


def default_q(d: int, eps_si: float) -> int:
    """Algorithm 2, q = Theta(log d / eps_SI), read as ceil(ln d / eps_SI)."""
    return int(math.ceil(math.log(d) / eps_si))


def power_iteration(A: np.ndarray, k: int, x0: np.ndarray) -> tuple[float, np.ndarray]:
    """Algorithm 1 on A (d x m) from the start vector x0 (m,)."""
    x = x0 / np.linalg.norm(x0)
    for _ in range(k):
        y = A.T @ (A @ x)
        nrm = np.linalg.norm(y)
        if nrm == 0.0:
            return 0.0, x
        x = y / nrm
    sig2 = float(x @ (A.T @ (A @ x)))
    return sig2, x


def simul_iter(A: np.ndarray, q: int, Pi: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Algorithm 2 on A (d x m) with test matrix Pi (m x k).

    Returns (Z, sigma2) with sigma2 descending (reading R5) and Z = Q U.
    The q products by A A^T are each followed by a Householder QR (R3)."""
    Q, _ = np.linalg.qr(A @ Pi)
    for _ in range(q):
        Q, _ = np.linalg.qr(A @ (A.T @ Q))
    AtQ = A.T @ Q
    M = AtQ.T @ AtQ
    M = 0.5 * (M + M.T)
    w, U = np.linalg.eigh(M)
    order = np.argsort(w)[::-1]
    return Q @ U[:, order], w[order]


@dataclass
class Snapshot:
    Z: np.ndarray   # d x xi
    Y: np.ndarray   # xi x d, = Z^T C'^T C'
    s: int
    t: int


@dataclass
class Event:
    """Decision record of one row whose gate passed (or was replayed)."""
    i: int
    sig2_pi: float
    theta: float
    j_stop: int = 0          # doubling step that broke the loop (0: none)
    xi: int = 0
    ritz: list = field(default_factory=list)   # sigma^2 per doubling step


class AeroSketch:
    """ATTP AeroSketch (Algorithm 8 over Algorithms 3-5), FP64.

    theta_mode 'attp' sets theta = eps ||A_t||_F^2 before each update;
    'fixed' keeps theta = theta_fixed (Algorithm 3's dump threshold)."""

    def __init__(self, d: int, ell: int, eps: float | None = None, *, seed: int = 0,
                 stream_id: int = 0, eps_si: float = 0.4, k_pi: int | None = None,
                 q: int | None = None, theta_mode: str = "attp",
                 theta_fixed: float | None = None, replay: dict | None = None,
                 tie_rel: float = 1e-4, track_delta: bool = False,
                 check_restore: bool = False, delta: float | None = None):
        if not (1 <= ell and 2 * ell <= d):
            raise ValueError("needs 1 <= l <= d/2")
        self.d, self.ell = d, ell
        self.eps = 2.0 / ell if eps is None else float(eps)
        self.seed, self.stream_id = seed, stream_id
        self.k_pi = default_k_pi(d) if k_pi is None else k_pi
        self.q = default_q(d, eps_si) if q is None else q
        self.theta_mode = theta_mode
        self.theta = 0.0 if theta_mode == "attp" else float(theta_fixed)
        self.C = np.zeros((2 * ell, d), dtype=np.float64)
        self.r = 0
        self.F = 0.0
        self.T = 0
        self.S: list[Snapshot] = []
        self.events: list[Event] = []
        self.shrink_rows: list[int] = []
        self.replay = replay
        self.tie_rel = tie_rel
        self.replayed = 0
        self.mismatches: list[tuple] = []
        self.sign_ties = 0
        self.track_delta = track_delta
        self.delta_sum = np.zeros((d, d)) if track_delta else None
        self.check_restore = check_restore
        self.restore_err = 0.0
        # Algorithm 7 (probability amplification), R17: r = ceil(log_100(2/delta))
        # simultaneous iterations with eps_SI = 0.2, s = ceil(2 log_3(2/delta))
        # power-iteration estimates of each residual's top eigenvalue
        self.delta = delta
        if delta is not None:
            self.amp_r = max(1, int(math.ceil(math.log(2.0 / delta) / math.log(100.0))))
            self.amp_s = max(1, int(math.ceil(2.0 * math.log(2.0 / delta) / math.log(3.0))))
            self.q_amp = default_q(d, 0.2)
        self.amp_choices: list[tuple[int, int, list[float], int]] = []   # (i, j, c_h, chosen h)

    # -- decisions, with optional replay of another run's choices at ties -----
    def _decide(self, own: bool, value: float, thr: float, kind: str, i: int, other):
        tied = abs(value - thr) <= self.tie_rel * abs(thr)
        if self.replay is None or other is None:
            return own
        if tied:
            if other != own:
                self.replayed += 1
            return other
        if other != own:
            self.mismatches.append((kind, i, value, thr))
        return own

    def _replay_gate(self, i):
        if self.replay is None:
            return None
        return i in self.replay.get("fired", ())

    def _replay_si(self, i):
        if self.replay is None:
            return None
        return self.replay.get("si", {}).get(i)

    # -- Algorithm 4 ------------------------------------------------------------
    def _shrink(self, i: int) -> None:
        ell = self.ell
        U, s, Vt = np.linalg.svd(self.C, full_matrices=False)
        s2 = s * s
        s2_ell = s2[ell - 1]
        for j in range(ell - 1):               # R10: canonical sign
            col = np.abs(U[:, j])
            p = int(np.argmax(col))
            srt = np.sort(col)
            if srt.size > 1 and srt[-1] - srt[-2] <= 1e-9 * srt[-1]:
                self.sign_ties += 1
            if U[p, j] < 0:
                U[:, j] = -U[:, j]
                Vt[j] = -Vt[j]
        if self.track_delta:
            loss = np.minimum(s2, s2_ell)
            self.delta_sum += (Vt.T * loss) @ Vt
        kept = np.sqrt(np.maximum(s2 - s2_ell, 0.0))
        self.C = kept[:, None] * Vt
        self.C[ell - 1:] = 0.0
        self.r = ell - 1                        # R9
        self.shrink_rows.append(i)

    def update(self, a: np.ndarray) -> None:
        a = np.asarray(a, dtype=np.float64)
        self.T += 1
        i = self.T
        if self.theta_mode == "attp":          # Algorithm 8
            self.F += float(a @ a)
            self.theta = self.eps * self.F
        theta = self.theta
        ell = self.ell
        self.C[self.r] = a                      # insert into the first empty row
        self.r += 1
        if self.r == 2 * ell:                   # full buffer: FD shrink
            self._shrink(i)
        Cp = self.C                             # C'_i
        x0 = philox.gaussians(self.seed, self.stream_id, philox.PURPOSE_PI_START, i, 0, 2 * ell)
        sig2, _ = power_iteration(Cp.T, self.k_pi, x0)          # Algorithm 1 on C'^T
        own_gate = sig2 >= theta / 2.0 and sig2 > 0.0            # the gate (R6)
        gate = self._decide(own_gate, sig2, theta / 2.0, "gate", i, self._replay_gate(i))
        if not gate:
            return
        ev = Event(i=i, sig2_pi=sig2, theta=theta)
        self.events.append(ev)
        other = self._replay_si(i)
        jmax = int(math.ceil(math.log2(min(ell, self.d)))) if min(ell, self.d) > 1 else 0
        for j in range(1, jmax + 1):                              # doubling loop
            k = min(2 ** j, ell, self.d)
            if self.delta is None:
                Pi = philox.gaussians(self.seed, self.stream_id, philox.PURPOSE_SI_TEST,
                                      i, j, 2 * ell * k).reshape(2 * ell, k)
                Zp, s2 = simul_iter(Cp.T, self.q, Pi)             # Algorithm 2 on C'^T
            else:
                Zp, s2 = self._amplified_si(Cp, k, i, j, theta)   # Algorithm 7 in place of Algorithm 2
            ev.ritz.append(s2.copy())
            own_stop = s2[k - 1] < theta                          # stop test
            stop = self._decide(own_stop, s2[k - 1], theta, "stop", i,
                                None if other is None else (other[0] == j))
            if not stop:
                continue
            own_xi = int(np.sum((s2 >= theta) & (s2 > 0.0)))     # xi
            xi = own_xi
            if other is not None and other[0] == j:
                near = np.any(np.abs(s2 - theta) <= self.tie_rel * theta)
                if near:
                    if other[1] != own_xi:
                        self.replayed += 1
                    xi = int(other[1])
                elif other[1] != own_xi:
                    self.mismatches.append(("xi", i, own_xi, other[1]))
            ev.j_stop, ev.xi = j, xi
            if xi >= 1:                                           # R7
                Z = Zp[:, :xi]
                CZ = Cp @ Z
                Y = CZ.T @ Cp                                     # Z^T C'^T C'
                s_prev = self.S[-1].t + 1 if self.S else 1
                self.S.append(Snapshot(Z=Z, Y=Y, s=s_prev, t=i))  # snapshot
                Cnew = Cp - CZ @ Z.T                              # residual C' - C' Z Z^T
                if self.check_restore:
                    lhs = Cnew.T @ Cnew + snapshot_term(Z, Y)
                    rhs = Cp.T @ Cp
                    den = max(np.linalg.norm(rhs), 1e-300)
                    self.restore_err = max(self.restore_err, float(np.linalg.norm(lhs - rhs) / den))
                self.C = Cnew
            return                                                # break
        # loop ended without break: C_i <- C'_i (R8)

    def _amplified_si(self, Cp: np.ndarray, k: int, i: int, j: int, theta: float):
        """Algorithm 7: r simultaneous iterations; keep the one whose residual
        C' - C' Z_h Z_h^T has the smallest estimated top eigenvalue (the
        maximum of s power iterations).  R17: SI h draws Pi at sub-index
        j + 64 (h-1); estimate g of SI h draws x^(0) at sub-index 64 h + g."""
        ell = self.ell
        best = None
        cs = []
        for h in range(1, self.amp_r + 1):
            Pi = philox.gaussians(self.seed, self.stream_id, philox.PURPOSE_SI_TEST,
                                  i, j + 64 * (h - 1), 2 * ell * k).reshape(2 * ell, k)
            Zh, s2h = simul_iter(Cp.T, self.q_amp, Pi)
            xi_h = int(np.sum((s2h >= theta) & (s2h > 0.0)))
            Zx = Zh[:, :xi_h]
            R = Cp - (Cp @ Zx) @ Zx.T
            ch = 0.0
            for g in range(1, self.amp_s + 1):
                x0 = philox.gaussians(self.seed, self.stream_id, philox.PURPOSE_PI_START, i, 64 * h + g, 2 * ell)
                c2, _ = power_iteration(R.T, self.k_pi, x0)
                ch = max(ch, c2)
            cs.append(ch)
            if best is None or ch < best[0]:
                best = (ch, h, Zh, s2h)
        h_star = best[1]
        other = None if self.replay is None else self.replay.get(("amp", i, j))
        if other is not None and other != h_star:
            # adopt the other run's choice only when the two estimates tie:
            # within tie_rel of the larger, or both at the rounding level of
            # a residual that is zero (below tie_rel * theta, every such SI
            # is a minimiser)
            c_o, c_b = cs[other - 1], cs[h_star - 1]
            if abs(c_o - c_b) <= self.tie_rel * max(c_o, c_b, theta):
                self.replayed += 1
                h_star = other
            else:
                self.mismatches.append(("amp", i, j, h_star, other))
        self.amp_choices.append((i, j, cs, h_star))
        Pi = philox.gaussians(self.seed, self.stream_id, philox.PURPOSE_SI_TEST,
                              i, j + 64 * (h_star - 1), 2 * ell * k).reshape(2 * ell, k)
        return simul_iter(Cp.T, self.q_amp, Pi)

    def load_state(self, C: np.ndarray, r: int, F: float, T: int) -> "AeroSketch":
        """Start from a given buffer (rows >= r zero), ||A_T||_F^2 and time T,
        with an empty snapshot queue: lets a test continue another
        implementation's stream for a window of rows."""
        self.C = np.array(C, dtype=np.float64, copy=True)
        self.C[r:] = 0.0
        self.r, self.F, self.T = int(r), float(F), int(T)
        if self.theta_mode == "attp":
            self.theta = self.eps * self.F
        return self

    def run(self, A: np.ndarray) -> "AeroSketch":
        for a in np.asarray(A, dtype=np.float64):
            self.update(a)
        return self

    # -- Algorithm 5 ------------------------------------------------------------
    def pre_query(self, lb: int = 0, ub: int | None = None) -> np.ndarray:
        """B of Algorithm 5 (before the eigendecomposition).

        At the current time (ub = T) B = C_T^T C_T plus the snapshot terms
        with lb < t <= T.  For a historical time ub < T (the ATTP Query(t) of
        Algorithm 8 asks for Query(0, t)) the residual C_ub is no longer
        stored, and B is the sum of the snapshot terms with lb < t <= ub, the
        B_i of the ATTP error analysis (reading R12)."""
        ub = self.T if ub is None else ub
        if not (0 <= ub <= self.T):
            raise ValueError("ub must lie in [0, T]")
        B = self.C.T @ self.C if ub == self.T else np.zeros((self.d, self.d))
        for sn in self.S:
            if lb < sn.t <= ub:
                B += snapshot_term(sn.Z, sn.Y)
        return 0.5 * (B + B.T)

    def query(self, lb: int = 0, ub: int | None = None) -> np.ndarray:
        """The eigen-shrink of Algorithm 5: the l x d sketch B_hat."""
        B = self.pre_query(lb, ub)
        lam, V = np.linalg.eigh(B)
        lam, V = lam[::-1], V[:, ::-1]
        scale = np.sqrt(np.maximum(lam - lam[self.ell - 1], 0.0))
        return (scale[:, None] * V.T)[: self.ell]

    def snapshot_rank(self) -> int:
        return int(sum(sn.Z.shape[1] for sn in self.S))


def snapshot_term(Z: np.ndarray, Y: np.ndarray) -> np.ndarray:
    """Z Z^T C'^T C' + C'^T C' Z Z^T - Z Z^T C'^T C' Z Z^T, from Z and Y = Z^T C'^T C'."""
    ZY = Z @ Y
    return ZY + ZY.T - Z @ (Y @ Z) @ Z.T
