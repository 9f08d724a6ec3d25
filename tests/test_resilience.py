"""Fault tolerance of the shot loop and of the FWI iterations, on CPU.

Failures are made on the host only: a gloo rank that announces it leaves
between gradient calls, and a rank that dies inside its shot computation
without notice (its process exits).  The survivors must agree on the new
membership, take over the lost shots and return the same sums as a run
without failure.  The L-BFGS driver must resume from its checkpoint and end
with the same model as an uninterrupted run.
"""
import datetime
import json
import multiprocessing as mp
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2502_12350_gb300 import resilience  # noqa: E402

SHAPE = (3, 4, 5)
N_SHOTS = 11


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _shot(s, call):
    """A shot's (misfit, gradient): small integers, so sums are exact in any order."""
    g = np.arange(np.prod(SHAPE), dtype=np.float64).reshape(SHAPE) % 7 + (s + 1) * (call + 1)
    return float((s + 1) * (call + 2)), torch.from_numpy(g)


def _expected(call):
    J = sum(_shot(s, call)[0] for s in range(N_SHOTS))
    g = sum(_shot(s, call)[1] for s in range(N_SHOTS))
    return J, g.numpy()


def _worker(rank, world, port, out_dir, scenario):
    import torch.distributed as dist
    store = dist.TCPStore("127.0.0.1", port, None, False, timeout=datetime.timedelta(seconds=60))
    grp = resilience.FaultTolerantGroup(store, rank, world, timeout=20.0, grace=1.5)
    costs = [1.0 + (s % 4) for s in range(N_SHOTS)]
    out = {"calls": [], "members": []}
    for call in range(3):
        if scenario == "leave" and rank == 2 and call == 1:
            grp.leave()  # between gradient calls, nothing in flight
            out["left"] = True
            break
        done = []

        def compute(idx):
            if scenario == "crash" and rank == 1 and call == 1:
                os._exit(3)  # dies inside its shard, without notice
            done.extend(idx)
            J, g = 0.0, torch.zeros(SHAPE, dtype=torch.float64)
            for s in idx:
                Js, gs = _shot(s, call)
                J, g = J + Js, g + gs
            return J, g

        J, g = grp.sharded(compute, costs)
        out["calls"].append({"J": J, "g": g.numpy().tolist(), "shots": sorted(done)})
        out["members"].append(list(grp.members))
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump(out, f)
    if dist.is_initialized() and not out.get("left"):
        dist.destroy_process_group()


def _run(scenario, world, tmp_path):
    import torch.distributed as dist
    port = _free_port()
    master = dist.TCPStore("127.0.0.1", port, None, True, timeout=datetime.timedelta(seconds=60),
                           wait_for_workers=False)
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_worker, args=(r, world, port, str(tmp_path), scenario))
             for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=180)
    codes = [p.exitcode for p in procs]
    for p in procs:
        if p.is_alive():
            p.kill()
    del master
    return codes


def _check_calls(out, calls):
    for call, rec in zip(calls, out["calls"]):
        J, g = _expected(call)
        assert rec["J"] == J
        np.testing.assert_array_equal(np.array(rec["g"]), g)


def test_rank_leaves_between_gradient_calls(tmp_path):
    codes = _run("leave", 3, tmp_path)
    assert codes == [0, 0, 0], codes
    r0 = json.load(open(tmp_path / "r0.json"))
    r1 = json.load(open(tmp_path / "r1.json"))
    assert json.load(open(tmp_path / "r2.json"))["left"]
    for out in (r0, r1):
        assert len(out["calls"]) == 3
        _check_calls(out, [0, 1, 2])
        assert out["members"] == [[0, 1, 2], [0, 1], [0, 1]]
    # after the departure every shot is computed exactly once per call
    for call in (1, 2):
        shots = sorted(r0["calls"][call]["shots"] + r1["calls"][call]["shots"])
        assert shots == list(range(N_SHOTS))


def test_rank_dies_inside_its_shard(tmp_path):
    codes = _run("crash", 3, tmp_path)
    assert codes[0] == 0 and codes[2] == 0 and codes[1] == 3, codes
    r0 = json.load(open(tmp_path / "r0.json"))
    r2 = json.load(open(tmp_path / "r2.json"))
    for out in (r0, r2):
        assert len(out["calls"]) == 3
        _check_calls(out, [0, 1, 2])
        assert out["members"][1] == [0, 2] and out["members"][2] == [0, 2]
    # in the failed call the survivors computed their own shards and the lost one
    shots = sorted(r0["calls"][1]["shots"] + r2["calls"][1]["shots"])
    assert shots == list(range(N_SHOTS))


def test_checkpoint_is_atomic(tmp_path):
    path = str(tmp_path / "state.npz")
    ck = resilience.Checkpoint(path)
    assert ck.load() is None
    ck.save({"x": np.arange(5.0)}, {"iteration": 3, "J": 0.1})
    # a write that died half way leaves only its temporary file behind
    with open(path + ".tmp999", "wb") as f:
        f.write(b"partial")
    arrays, meta = ck.load()
    np.testing.assert_array_equal(arrays["x"], np.arange(5.0))
    assert meta == {"iteration": 3, "J": 0.1}


class _Quadratic:
    """A bound-constrained, badly scaled least-squares problem standing in for
    the FWI misfit on CPU (the driver only sees misfit, gradient and a
    positive diagonal)."""

    def __init__(self, n=40, seed=0):
        rng = np.random.default_rng(seed)
        self.M = rng.standard_normal((2 * n, n)) * np.logspace(0, 1.5, n)
        self.b = rng.standard_normal(2 * n) * 30
        self.dev = torch.device("cpu")
        self.n_grad = self.n_fwd = 0
        self.vmin, self.vmax = -5.0, 5.0

    def misfit(self, v):
        self.n_fwd += 1
        r = self.M @ v.ravel() - self.b
        return 0.5 * float(r @ r)

    def gradient(self, v):
        self.n_grad += 1
        r = self.M @ v.ravel() - self.b
        diag = torch.from_numpy(np.sum(self.M ** 2, axis=0))
        return 0.5 * float(r @ r), self.M.T @ r, diag

    def project(self, v):
        return np.clip(v, self.vmin, self.vmax)


def test_fwi_resumes_from_checkpoint(tmp_path):
    from paper_2502_12350_gb300 import fwi
    v0 = np.zeros((5, 8))
    ref = fwi.run(_Quadratic(), v0, 7, precond="pseudo", first_step=0.5)
    path = str(tmp_path / "fwi.npz")

    class Crash(Exception):
        pass

    def crash_at_3(it, x, J):
        if it == 3:
            raise Crash()

    with pytest.raises(Crash):
        fwi.run(_Quadratic(), v0, 7, precond="pseudo", first_step=0.5, checkpoint=path,
                on_iteration=crash_at_3)
    prob = _Quadratic()
    got = fwi.run(prob, v0, 7, precond="pseudo", first_step=0.5, checkpoint=path)
    np.testing.assert_array_equal(got.vel, ref.vel)
    assert [h[1] for h in got.history] == [h[1] for h in ref.history]
    assert prob.n_grad == 4  # iterations 4..7 only: nothing before the crash is redone
