"""ML-AeroSketch for sliding windows (Algorithm 6), plain FP64 (oracle; test
infrastructure only).

Levels j = 0 .. L-1, each an AeroSketch (Algorithms 3-5) with the fixed
threshold theta_j = 2^j eps N, and a queue S_j of items (s, t, payload): the
level's snapshots (Z, Z^T C'^T C') and raw heavy rows.  For each row a_i
(i = 1, 2, ...) and each level j:
  pop the queue's front while len(S_j) > 8/eps or S_j[0].t <= i - N;
  if ||a_i||^2 >= theta_j: append the raw row (s, t = i);
  else: update the level's AeroSketch with a_i; a snapshot it takes is moved
  to S_j with (s, t = i).
Query at time T: the lowest level j whose queue is empty or starts at
S_j[0].s <= T - N + 1; B = C_j^T C_j + the snapshot terms and the raw rows
a^T a of S_j with t in (T-N, T]; eigendecomposition, shrink by lambda_l, top
l rows (the eigen-shrink of Algorithm 5).

Readings (also in the design notes):
  R15 s = S[-1].t + 1 for every item (Algorithm 4 prints +1, Algorithm 6's raw
      row does not), and s = 1 when the queue is empty.  The raw rows are
      added to B as a^T a before the eigendecomposition (one shrink instead of
      an FD pass over the query sketch and the raw rows).  A level's
      AeroSketch numbers its own rows (the light rows it received) for its
      random draws; queue items carry the stream time i.
  R16 L = ceil(log2 R) + 1 levels, so that the level floor(log2(||A_w||^2 / N))
      of Fact 1 exists for every window mass in [N, N R]; if no level
      qualifies at a query, the top level answers.  Before the window is
      full (T < N) it starts at row 1: the level test is S[0].s <= max(1,
      T - N + 1).
"""
from __future__ import annotations

import math
from collections import deque
from dataclasses import dataclass

import numpy as np

from .aerosketch import AeroSketch, snapshot_term


@dataclass
class Item:
    s: int
    t: int
    Z: np.ndarray | None = None   # snapshot: Z and Y = Z^T C'^T C'
    Y: np.ndarray | None = None
    a: np.ndarray | None = None   # raw heavy row


def levels_for(R: float) -> int:
    return int(math.ceil(math.log2(max(R, 1.0)))) + 1   # R16


class SlidingAeroSketch:
    def __init__(self, d: int, ell: int, N: int, R: float, eps: float | None = None, *, seed: int = 0,
                 replay: list | None = None, tie_rel: float = 1e-4):
        self.d, self.ell, self.N = d, ell, int(N)
        self.eps = 2.0 / ell if eps is None else float(eps)
        self.cap = int(math.floor(8.0 / self.eps))
        self.L = levels_for(R)
        self.theta = [(2.0 ** j) * self.eps * self.N for j in range(self.L)]
        self.levels = [AeroSketch(d, ell, self.eps, seed=seed, stream_id=j, theta_mode="fixed",
                                  theta_fixed=self.theta[j], replay=None if replay is None else replay[j],
                                  tie_rel=tie_rel)
                       for j in range(self.L)]
        self.S: list[deque] = [deque() for _ in range(self.L)]
        self.T = 0
        self.popped_cap = [0] * self.L

    def _append(self, j: int, item: Item) -> None:
        Q = self.S[j]
        item.s = Q[-1].t + 1 if Q else 1                    # R15
        Q.append(item)

    def update(self, a: np.ndarray) -> None:
        a = np.asarray(a, dtype=np.float64)
        self.T += 1
        i = self.T
        na = float(a @ a)
        for j in range(self.L):
            Q = self.S[j]
            while Q and (len(Q) > self.cap or Q[0].t <= i - self.N):
                if len(Q) > self.cap and Q[0].t > i - self.N:
                    self.popped_cap[j] += 1
                Q.popleft()
            if na >= self.theta[j]:
                self._append(j, Item(0, i, a=a.copy()))
            else:
                lv = self.levels[j]
                lv.update(a)
                while lv.S:
                    sn = lv.S.pop(0)
                    self._append(j, Item(0, i, Z=sn.Z, Y=sn.Y))

    def run(self, A: np.ndarray) -> "SlidingAeroSketch":
        for a in np.asarray(A, dtype=np.float64):
            self.update(a)
        return self

    def level_for_query(self) -> int:
        lo = max(1, self.T - self.N + 1)                    # R16: the window starts at row 1 at the latest
        for j in range(self.L):
            Q = self.S[j]
            if not Q or 1 <= Q[0].s <= lo:
                return j
        return self.L - 1                                   # R16

    def pre_query(self, j: int | None = None) -> np.ndarray:
        j = self.level_for_query() if j is None else j
        lv = self.levels[j]
        B = lv.C.T @ lv.C
        lb = self.T - self.N
        for it in self.S[j]:
            if it.t > lb:
                B += snapshot_term(it.Z, it.Y) if it.a is None else np.outer(it.a, it.a)
        return 0.5 * (B + B.T)

    def query(self, j: int | None = None) -> np.ndarray:
        B = self.pre_query(j)
        lam, V = np.linalg.eigh(B)
        lam, V = lam[::-1], V[:, ::-1]
        scale = np.sqrt(np.maximum(lam - lam[self.ell - 1], 0.0))
        return (scale[:, None] * V.T)[: self.ell]
