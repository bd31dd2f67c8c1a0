"""The sharded loop's collective step on CPU ranks (gloo, world size 2): each rank owns
rows of the pupil and computes its partial Theta and its phase rows with the FP64 oracle;
the partial Theta is all-reduced through torch.distributed.  The joined phase, the
weights and the xi history must equal the unsharded oracle run; a rank delayed before
its partial changes nothing; a rank that is lost makes the other's collective raise
after the group's timeout instead of hanging."""
import datetime
import multiprocessing as mp
import os
import socket
import time

import numpy as np
import pytest

import oracle as O
from paper_2206_12661_gb300 import shard as SH

torch = pytest.importorskip("torch")

NX, NY, K, N_ITER = 40, 36, 6, 5


def workload():
    rng = np.random.default_rng(17)
    p, lam, f = 8e-6, 532e-9, 0.2
    half = lam * f / (2 * p)
    xy = rng.uniform(-0.8 * half, 0.8 * half, (K, 2))
    t = rng.uniform(0.5, 1.0, K)
    A = O.default_amplitude(NX, NY, p, p)
    phi0 = rng.uniform(-np.pi, np.pi, (NY, NX))
    fx, fy = O.plan_matrices(NX, NY, p, p, lam, f, xy)
    return A, phi0, fx, fy, t


class OracleShard:
    """Rows [row0, row0 + rows) of the pupil, with the oracle's operators on them."""

    def __init__(self, row0, rows, delay_at=None):
        A, phi0, fx, fy, t = workload()
        sl = slice(row0, row0 + rows)
        self.A, self.phi, self.fx, self.fy, self.t = A[sl], phi0[sl].copy(), fx, fy[:, sl], t
        self.w = np.ones(K)
        self.xi = []
        self.it = 0
        self.delay_at = delay_at

    def forward(self):
        if self.delay_at is not None and self.it == self.delay_at:
            time.sleep(0.5)
        theta = O.forward(O.pupil_field(self.A, self.phi), self.fx, self.fy)
        return torch.tensor(np.stack([theta.real, theta.imag], 1), dtype=torch.float64)

    def update(self, total):
        tt = total.numpy()
        theta = tt[:, 0] + 1j * tt[:, 1]
        inten = np.abs(theta) ** 2
        self.xi.append(O.intensity_accuracy(self.t, inten))
        self.w = O.generalized_weights(self.w, self.t, inten)
        back = O.adjoint(O.focused_field(self.w, self.t, theta), self.fx, self.fy)
        self.phi = O.phase_projection(back)
        self.it += 1


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def worker(rank, world, port, mode, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=10))
    r0, rows = SH.row_ranges(NY, world)[rank]
    shard = OracleShard(r0, rows, delay_at=2 if (mode == "delay" and rank == 1) else None)
    loop = SH.ShardedLoop([shard], SH.DistributedSum())
    try:
        for it in range(N_ITER):
            if mode == "lost" and rank == 1 and it == 2:
                os._exit(0)                   # leaves between steps, nothing in flight
            loop.step()
        out.put((rank, "ok", shard.phi, shard.w, shard.xi))
    except Exception as e:                    # the surviving rank of "lost"
        out.put((rank, "error", type(e).__name__, str(e)[:200], shard.it))
    finally:
        try:
            dist.destroy_process_group()
        except Exception:
            pass


def run(mode, world=2):
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=worker, args=(r, world, port, mode, out)) for r in range(world)]
    for p in procs:
        p.start()
    results = []
    deadline = time.time() + 120
    expected = world if mode != "lost" else 1
    while len(results) < expected and time.time() < deadline:
        try:
            results.append(out.get(timeout=5))
        except Exception:
            pass
    for p in procs:
        p.join(timeout=30)
        if p.is_alive():
            p.kill()
    return sorted(results, key=lambda r: r[0])


@pytest.mark.parametrize("mode", ["plain", "delay"])
def test_gloo_sharded_loop_equals_unsharded_oracle(mode):
    res = run(mode)
    assert [r[1] for r in res] == ["ok", "ok"], res
    A, phi0, fx, fy, t = workload()
    ref = O.gsw(A, phi0, fx, fy, t, N_ITER)
    phi = np.concatenate([r[2] for r in res], axis=0)
    assert np.max(np.abs(np.exp(1j * phi) - np.exp(1j * ref["phi"]))) < 1e-9
    for r in res:
        assert np.allclose(r[3], ref["w"], rtol=1e-12, atol=0)
        assert np.allclose(r[4], ref["xi_hist"], rtol=0, atol=1e-12)


def test_gloo_lost_rank_raises_on_the_survivor():
    res = run("lost")
    assert len(res) == 1 and res[0][0] == 0, res
    assert res[0][1] == "error" and res[0][4] == 2, res
