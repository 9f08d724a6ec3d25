"""Fault tolerance of the distributed shot loop and of the FWI iterations.

The paper's FWI (Sec. 2; Algorithm 3) relies on a dependability library for
three things: detecting that a process failed, conserving the data needed to
go on, and failing over so that the inversion continues from a state before
the interruption.  This module provides the same three on the host, around
the GPU gradient:

* Failure detection.  Ranks share a key-value store (the torch.distributed
  Store the process group was created from, e.g. the launcher's TCPStore).
  A rank that leaves between gradient calls writes a `left` marker; a rank
  that dies without one is noticed when the next reduction of results fails
  (gloo closes the connection; other backends end the collective at the
  process group's timeout).  Only the host learns of it, between steps: no
  kernel waits on another rank.
* Failover.  The survivors agree on the new membership through one atomic
  compare-and-set on the store (the first proposal wins, so every survivor
  adopts the same member list), rebuild the process group among themselves
  under a fresh store prefix, and split the shots of the ranks that left
  over the survivors with the same cost-balanced partition as the initial
  split.  Shots a survivor already finished are not recomputed.
* Data conservation.  `Checkpoint` writes the optimizer state (model, misfit,
  gradient, L-BFGS pairs, iteration, history) atomically after every
  iteration; a restarted run resumes from it (fwi.run(checkpoint=...)).

Failure model: crash-stop ranks, and a store that stays up (hosted by the
launcher, not by a worker).  Results are the same shot sums as without a
failure, grouped differently, so they agree to rounding.
"""
from __future__ import annotations

import datetime
import json
import os
import time

import numpy as np

from .sharding import partition


class RankLost(RuntimeError):
    """This rank is not in the membership the survivors agreed on."""


class FaultTolerantGroup:
    """Membership, failure detection and failover for ranks that share a
    torch.distributed Store.

    store    a torch.distributed Store reachable by every rank (TCPStore)
    rank     this process's rank in the initial world
    world    initial number of ranks
    backend  process-group backend of the result reductions ("gloo", "nccl")
    timeout  seconds before a collective with a silent peer gives up
    grace    seconds the survivors wait for each other when agreeing on the
             new membership
    """

    def __init__(self, store, rank: int, world: int, backend: str = "gloo", timeout: float = 10.0,
                 grace: float = 2.0, prefix: str = "mamute-ft"):
        self.store, self.rank, self.backend = store, rank, backend
        self.timeout, self.grace, self.prefix = timeout, grace, prefix
        self.members = list(range(world))
        self.epoch = 0
        self.failovers = 0
        self._init_group()

    # ------------------------------------------------------------ membership
    def _key(self, *parts) -> str:
        return "/".join((self.prefix,) + tuple(str(p) for p in parts))

    def _has(self, key: str) -> bool:
        return bool(self.store.check([key]))

    def _init_group(self):
        import torch.distributed as dist
        if dist.is_initialized():
            dist.destroy_process_group()
        ps = dist.PrefixStore(self._key("pg", self.epoch), self.store)
        dist.init_process_group(self.backend, store=ps, rank=self.members.index(self.rank),
                                world_size=len(self.members),
                                timeout=datetime.timedelta(seconds=self.timeout))

    def leave(self):
        """Leaves the computation between steps: the others fail over before
        their next reduction."""
        import torch.distributed as dist
        self.store.set(self._key("left", self.rank), "1")
        if dist.is_initialized():
            dist.destroy_process_group()

    def departed(self):
        """Members that announced they left."""
        return [r for r in self.members if r != self.rank and self._has(self._key("left", r))]

    def failover(self):
        """Agrees with the other survivors on the new member list and rebuilds
        the process group among them.  Raises RankLost if the survivors did
        not count this rank in."""
        e = self.epoch + 1
        self.store.set(self._key("ready", e, self.rank), "1")
        deadline = time.monotonic() + self.grace
        while time.monotonic() < deadline:
            ready = [r for r in self.members if self._has(self._key("ready", e, r))]
            if len(ready) == len(self.members):
                break
            time.sleep(0.02)
        ready = [r for r in self.members if self._has(self._key("ready", e, r))
                 and not self._has(self._key("left", r))]
        # First proposal wins: every survivor adopts the same list.
        agreed = self.store.compare_set(self._key("members", e), "", json.dumps(ready))
        members = json.loads(agreed.decode() if isinstance(agreed, bytes) else agreed)
        if self.rank not in members:
            raise RankLost(f"rank {self.rank} was left out of epoch {e}")
        self.members, self.epoch = members, e
        self.failovers += 1
        self._init_group()

    # ------------------------------------------------------------ reductions
    def ordered_sum(self, J: float, grad):
        """(sum of J, sum of grad) over the members, added in ascending rank
        order on every member (all-gather, then a fixed-order sum)."""
        import torch
        import torch.distributed as dist
        world = dist.get_world_size()
        Jt = torch.tensor([float(J)], dtype=torch.float64, device=grad.device)
        Js = [torch.zeros_like(Jt) for _ in range(world)]
        gs = [torch.zeros_like(grad) for _ in range(world)]
        dist.all_gather(Js, Jt)
        dist.all_gather(gs, grad.contiguous())
        tot = gs[0].clone()
        for r in range(1, world):
            tot += gs[r]
        Jtot = 0.0
        for r in range(world):
            Jtot += float(Js[r].item())
        return Jtot, tot

    def sharded(self, compute, costs):
        """One sharded gradient: compute(shot_indices) -> (J, grad tensor) on
        this rank's shots, summed over the members.  If members leave or die
        before the sum completes, the survivors fail over, take over the lost
        shots (balanced by cost) and sum again."""
        parts = partition(costs, len(self.members))
        assign = {r: list(parts[i]) for i, r in enumerate(self.members)}
        J, grad = compute(assign[self.rank])
        while True:
            if not self.departed():
                try:
                    return self.ordered_sum(J, grad)
                except RuntimeError:
                    pass  # a peer failed inside the collective
            old = list(self.members)
            self.failover()
            lost = sorted(s for r in old if r not in self.members for s in assign.pop(r))
            if not lost:
                continue
            extra = partition([costs[s] for s in lost], len(self.members))
            for i, r in enumerate(self.members):
                assign[r] = assign[r] + [lost[k] for k in extra[i]]
            mine = [lost[k] for k in extra[self.members.index(self.rank)]]
            if mine:
                J2, g2 = compute(sorted(mine))
                J, grad = J + J2, grad + g2


class Checkpoint:
    """Atomic save / load of an optimizer state: numpy arrays and a JSON
    header in one .npz file, written to a temporary name and renamed, so a
    crash during the write leaves the previous checkpoint intact."""

    def __init__(self, path: str):
        self.path = path

    def save(self, arrays: dict, meta: dict):
        tmp = f"{self.path}.tmp{os.getpid()}"
        with open(tmp, "wb") as f:
            np.savez(f, __meta__=np.frombuffer(json.dumps(meta).encode(), np.uint8), **arrays)
            f.flush()
            os.fsync(f.fileno())
        os.replace(tmp, self.path)

    def load(self):
        """(arrays, meta) of the last completed save, or None."""
        if not os.path.exists(self.path):
            return None
        with np.load(self.path) as z:
            meta = json.loads(bytes(z["__meta__"]).decode())
            arrays = {k: z[k].copy() for k in z.files if k != "__meta__"}
        return arrays, meta
