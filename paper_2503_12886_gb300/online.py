"""Online reconstruction's data pools (RGBAvatar Sec. 3.3 "Online Reconstruction Process",
Supp. "Online Frame Processing", Alg. 2): a local FIFO pool of recent frames and a global
reservoir of past frames, and the training batches drawn from both.

Alg. 2, per incoming frame D_i: if the local pool M_l is full, its oldest sample D_j (j = the
frame's position in the stream, 0-based) leaves it; if the global pool M_g is full, D_j replaces
M_g[k] for k = randint(0, j) when k < |M_g| (reservoir sampling, Vitter 1985, so every frame
that left M_l is in M_g with the same probability |M_g| / (j + 1)), otherwise it is appended.
Then D_i joins M_l. A batch of B takes round(eta B) (half to even) samples from M_l and the
rest from M_g, uniformly without replacement within each pool; while a pool is short, the other
one fills in.
The paper uses eta = 0.7, |M_l| = 150, |M_g| = 1000.

Random numbers come from a counter-based splitmix64 stream (synth.Stream), so a run is a pure
function of its seed. The pools hold whatever the caller passes as a sample (an index into a
device-resident frame store, in the benchmark).
"""
from __future__ import annotations

from collections import deque

import numpy as np

from . import synth


class LocalGlobalSampler:
    def __init__(self, local_cap: int = 150, global_cap: int = 1000, eta: float = 0.7,
                 seed: int = 0):
        if local_cap < 1 or global_cap < 0 or not (0.0 <= eta <= 1.0):
            raise ValueError("need local_cap >= 1, global_cap >= 0, 0 <= eta <= 1")
        self.local_cap, self.global_cap, self.eta = local_cap, global_cap, eta
        self.local: deque = deque()
        self.glob: list = []
        self.n_seen = 0                    # frames pushed so far (the next frame's index)
        self._pos = deque()                # stream index of each local sample
        self._rng = synth.Stream(seed, 60)

    def _randint(self, hi: int) -> int:
        """Uniform integer in [0, hi] (inclusive): one 64-bit draw reduced modulo hi + 1 (the
        modulo bias is below 2^-40 for any pool or stream length under 2^24)."""
        return int(self._rng.u64(1)[0] % np.uint64(hi + 1))

    def push(self, sample) -> None:
        """Alg. 2 for one incoming frame."""
        if len(self.local) == self.local_cap:
            d = self.local.popleft()
            j = self._pos.popleft()
            if len(self.glob) == self.global_cap:
                if self.global_cap > 0:
                    k = self._randint(j)
                    if k < self.global_cap:
                        self.glob[k] = d
            else:
                self.glob.append(d)
        self.local.append(sample)
        self._pos.append(self.n_seen)
        self.n_seen += 1

    def _choose(self, pool, m: int) -> list:
        """m distinct elements of pool, uniformly (partial Fisher-Yates on an index list)."""
        idx = list(range(len(pool)))
        for t in range(m):
            r = t + self._randint(len(idx) - 1 - t)
            idx[t], idx[r] = idx[r], idx[t]
        return [pool[i] for i in idx[:m]]

    def sample(self, batch: int) -> list:
        """A training batch: round(eta B) from the local pool, the rest from the global pool."""
        nl, ng = len(self.local), len(self.glob)
        want_l = int(round(self.eta * batch))
        take_l = min(want_l, nl)
        take_g = min(batch - take_l, ng)
        take_l = min(nl, batch - take_g)          # the local pool fills in for a short global one
        local = list(self.local)
        return self._choose(local, take_l) + self._choose(self.glob, take_g)
