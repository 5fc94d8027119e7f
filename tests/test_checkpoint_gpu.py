"""Checkpoint / resume of a chunked run and the reduction of shards (the sums of
Sec. 2.3 are additive over points).

* Kill and restart: a child process spreads the first chunks of the device-generated
  1-D sweep sample, writes the accumulator's state to a file and dies without cleaning
  up; this process loads the state, adds the remaining chunks and must get the same
  bits as an uninterrupted run (the 1-D fixed-point path adds each chunk's sums in
  chunk order).
* Shards: two accumulators over halves of the points, combined by loading one state
  and adding the other, equal a single accumulator over both (bit for bit in 1-D; in
  2-D within the NUFFT tolerance of the oracle, since the register sums of one shard
  do not add in a fixed order).
* Two processes, one shard each, exchange their states through torch.distributed
  (gloo) and reduce them with fk_accum_add_state: both ranks end with the sums of the
  whole sample, divided by the total point count.
"""
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

import oracle as O
import synthetic as S

pytestmark = pytest.mark.gpu

fk = pytest.importorskip("paper_2509_02649_b300")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
M, NT, EPS, CHUNK, K = 60, 4, 1e-6, 1 << 20, 4


def sweep_chunk(i):
    x, y, amax = fk.generate_sweep_1d(i * CHUNK, CHUNK, NT)
    return x, y, amax


CHILD = r"""
import sys, torch
sys.path.insert(0, {root!r})
import paper_2509_02649_b300 as fk
acc = fk.Accumulator(1, {m}, {nt}, {eps}, "mixed")
for i in range({k0}):
    x, y, a = fk.generate_sweep_1d(i * {chunk}, {chunk}, {nt})
    acc.add(x, y, a)
open({path!r}, "wb").write(acc.state())
import os
os._exit(9)  # dies here: no destructor, no synchronisation, no cleanup
"""


def test_kill_and_restart_is_bit_identical(tmp_path):
    # uninterrupted run
    full = fk.Accumulator(1, M, NT, EPS, "mixed")
    for i in range(K):
        full.add(*sweep_chunk(i))
    T_ref, b_ref, n_ref = full.system()
    th_ref = full.fit_sobolev(1.0, [1e-6, 1e-3])
    full.close()
    # the first half in a child process that dies after writing its checkpoint
    path = str(tmp_path / "acc.state")
    code = CHILD.format(root=ROOT, m=M, nt=NT, eps=EPS, k0=K // 2, chunk=CHUNK, path=path)
    rc = subprocess.run([sys.executable, "-c", code], cwd=ROOT, timeout=600).returncode
    assert rc == 9 and os.path.getsize(path) > 64
    # restart from the checkpoint
    acc = fk.Accumulator(1, M, NT, EPS, "mixed")
    acc.load_state(open(path, "rb").read())
    for i in range(K // 2, K):
        acc.add(*sweep_chunk(i))
    T, b, n = acc.system()
    th = acc.fit_sobolev(1.0, [1e-6, 1e-3])
    acc.close()
    assert n == n_ref == K * CHUNK
    assert torch.equal(T, T_ref) and torch.equal(b, b_ref)  # the sums: the same bits
    # the solve on the same sums (its reductions may add in another order)
    assert float((th - th_ref).abs().max() / th_ref.abs().max()) <= 1e-13


def test_shards_reduce_to_the_single_accumulator_1d():
    xa, ya, aa = sweep_chunk(0)
    xb, yb, ab = sweep_chunk(1)
    single = fk.Accumulator(1, M, NT, EPS, "mixed")
    single.add(xa, ya, aa)
    single.add(xb, yb, ab)
    sa = fk.Accumulator(1, M, NT, EPS, "mixed")
    sb = fk.Accumulator(1, M, NT, EPS, "mixed")
    sa.add(xa, ya, aa)
    sb.add(xb, yb, ab)
    merged = fk.Accumulator(1, M, NT, EPS, "mixed")
    merged.load_state(sa.state())
    merged.add_state(sb.state())
    T1, b1, n1 = single.system()
    T2, b2, n2 = merged.system()
    assert n1 == n2 == 2 * CHUNK
    assert torch.equal(T1, T2) and torch.equal(b1, b2)
    for a in (single, sa, sb, merged):
        a.close()


def test_shards_reduce_2d_against_oracle():
    n, m = 60000, 12
    x, y = S.wl2_sobolev_2d(n, dtype=np.float32)
    xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    h = n // 2
    sa = fk.Accumulator(2, m, 1, EPS, "mixed")
    sb = fk.Accumulator(2, m, 1, EPS, "mixed")
    sa.add(xd[:, :h].contiguous(), yd[:h].contiguous())
    sb.add(xd[:, h:].contiguous(), yd[h:].contiguous())
    merged = fk.Accumulator(2, m, 1, EPS, "mixed")
    merged.load_state(sa.state())
    merged.add_state(sb.state())
    T, b, nt = merged.system()
    assert nt == n
    x64, y64 = x.astype(np.float64), y.astype(np.float64)
    To, bo = O.moments(x64, m), O.rhs(x64, y64, m)
    assert float(np.linalg.norm(T.cpu().numpy() - To) / np.linalg.norm(To)) <= 10 * EPS
    assert float(np.linalg.norm(b.cpu().numpy().ravel() - bo.ravel()) / np.linalg.norm(bo)) <= 10 * EPS
    for a in (sa, sb, merged):
        a.close()


def test_state_of_another_shape_is_rejected():
    a = fk.Accumulator(1, M, NT, EPS, "mixed")
    b = fk.Accumulator(1, M + 1, NT, EPS, "mixed")
    with pytest.raises(fk.FkError) as e:
        b.load_state(a.state())
    assert e.value.name == "FK_EINVAL"
    with pytest.raises(fk.FkError):
        b.add_state(b"not a state" * 10)
    a.close()
    b.close()


def _rank(rank, world, port, out_path):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import paper_2509_02649_b300 as fkr
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    acc = fkr.Accumulator(1, M, NT, EPS, "mixed")
    x, y, a = fkr.generate_sweep_1d(rank * CHUNK, CHUNK, NT)  # this rank's shard
    acc.add(x, y, a)
    states = [None] * world
    dist.all_gather_object(states, acc.state())
    total = fkr.Accumulator(1, M, NT, EPS, "mixed")
    total.load_state(states[0])
    for s in states[1:]:
        total.add_state(s)
    T, b, n = total.system()
    torch.save({"T": T.cpu(), "b": b.cpu(), "n": n}, out_path % rank)
    acc.close()
    total.close()
    dist.destroy_process_group()


def test_two_processes_reduce_their_shards(tmp_path):
    import socket
    import torch.multiprocessing as mp
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    out = str(tmp_path / "rank%d.pt")
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=600)
        assert p.exitcode == 0
    single = fk.Accumulator(1, M, NT, EPS, "mixed")
    for r in range(2):
        single.add(*sweep_chunk(r))
    T, b, n = single.system()
    single.close()
    for r in range(2):
        got = torch.load(out % r)
        assert got["n"] == n == 2 * CHUNK
        assert torch.equal(got["T"], T.cpu()) and torch.equal(got["b"], b.cpu())
