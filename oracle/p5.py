"""P5: AeroSketch for the tracking distributed matrix sketch (Algorithm 10),
plain FP64 (oracle; test infrastructure only).

m sites each run AeroSketch (Algorithms 3-5) with a threshold theta that
the coordinator controls; the coordinator sums the sites' snapshot terms into
B and answers queries from B (the eigen-shrink of Algorithm 5 on B).

Site j, for each row a (Algorithm 10, site Update):
  F_j += ||a||^2; if F_j >= (eps/m) F_hat: send F_j, F_j = 0;
  AeroSketch.Update(a); every snapshot taken is sent to the coordinator and
  removed from the site's queue.
Coordinator:
  on F_j: F_hat += F_j, msgs += 1; when msgs >= m: msgs = 0, broadcast F_hat;
  on a snapshot (Z, Y = Z^T C'^T C'): B += Z Y + Y^T Z^T - Z (Y Z) Z^T;
  Query: eigendecomposition of B, shrink by lambda_l, top l rows.

Readings (also in the design notes):
  R13 A site's dump threshold after a broadcast is theta = (eps/m) F_hat: the
      per-site error eps/m of the proof (the algorithm text prints eps F_hat).
      Algorithm 10 leaves the threshold a site starts with open (Algorithm 3
      takes it as an input); it is +inf: no snapshot is sent before the
      coordinator's first broadcast.  (theta = 0 would make the stop test
      sigma_k^2 < theta of Algorithm 2 hinge on the rounding sign of
      numerically zero Ritz values.)
  R14 Synchronous rounds: every site ingests its rows of a round; the F
      messages of the round reach the coordinator at the round's end, in
      site order, and a broadcast made then applies from the next round on.
      A site compares F_j with the F_hat of the last broadcast it received.
"""
from __future__ import annotations

import numpy as np

from .aerosketch import AeroSketch, snapshot_term


class P5:
    def __init__(self, d: int, ell: int, m: int, eps: float | None = None, *, seed: int = 0,
                 replay: list | None = None, tie_rel: float = 1e-4, track_delta: bool = False):
        self.d, self.ell, self.m = d, ell, m
        self.eps = 2.0 / ell if eps is None else float(eps)
        self.sites = [AeroSketch(d, ell, self.eps, seed=seed, stream_id=j, theta_mode="fixed", theta_fixed=np.inf,
                                 replay=None if replay is None else replay[j], tie_rel=tie_rel,
                                 track_delta=track_delta)
                      for j in range(m)]
        self.F = [0.0] * m            # F_j, unsent row mass of site j
        self.F_site = 0.0             # F_hat as the sites know it (last broadcast)
        self.F_hat = 0.0              # the coordinator's running F_hat
        self.msgs = 0
        self.messages = 0
        self.broadcasts = 0
        self.B = np.zeros((d, d))
        self.sent_snapshots = 0

    def round(self, blocks: list[np.ndarray]) -> None:
        """One synchronous round: blocks[j] holds site j's rows (R14)."""
        assert len(blocks) == self.m
        pending = []
        for j, rows in enumerate(blocks):
            s = self.sites[j]
            for a in np.asarray(rows, dtype=np.float64):
                self.F[j] += float(a @ a)
                if self.F[j] >= (self.eps / self.m) * self.F_site:
                    pending.append(self.F[j])
                    self.F[j] = 0.0
                s.update(a)
                while s.S:                                   # send S[0], delete it
                    sn = s.S.pop(0)
                    self.B += snapshot_term(sn.Z, sn.Y)
                    self.sent_snapshots += 1
        for f in pending:                                    # coordinator, Receive_Update
            self.F_hat += f
            self.messages += 1
            self.msgs += 1
            if self.msgs >= self.m:
                self.msgs = 0
                self.broadcasts += 1
                self.F_site = self.F_hat
                for s in self.sites:                         # R13
                    s.theta = (self.eps / self.m) * self.F_hat

    def query(self) -> np.ndarray:
        """Coordinator Query: the l x d sketch from B."""
        B = 0.5 * (self.B + self.B.T)
        lam, V = np.linalg.eigh(B)
        lam, V = lam[::-1], V[:, ::-1]
        scale = np.sqrt(np.maximum(lam - lam[self.ell - 1], 0.0))
        return (scale[:, None] * V.T)[: self.ell]

    def residual_gram(self) -> np.ndarray:
        """sum_j C_j^T C_j: what the sites still hold (never sent)."""
        return sum(s.C.T @ s.C for s in self.sites)
