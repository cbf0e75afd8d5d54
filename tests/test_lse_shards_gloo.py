"""The per-frame log-sum-exp over rotations splits into rotation shards that
exchange only (max, sum) pairs (Sec. 3.2-3.3: the nodes exchange per-frame
maxima and sums, not probabilities; the tile merge of pass 1 uses the same
identity across rotation tiles).

Two gloo ranks on CPU each hold half of the rotations' FP64 oracle scores. An
all-reduce MAX of the shard maxima followed by an all-reduce SUM of the rescaled
shard sums reproduces the oracle's lse over all rotations, and with it every
responsibility P_jk = exp(S_jk - lse_k) a shard computes locally.
"""
import json
import os
import socket

import numpy as np
import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, path, out_dir):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    S = np.load(path)  # [n_rot, n_frames] scores of every rotation
    lo, hi = rank * S.shape[0] // world, (rank + 1) * S.shape[0] // world
    Sr = S[lo:hi]
    m = torch.as_tensor(Sr.max(0))
    M = m.clone()
    dist.all_reduce(M, op=dist.ReduceOp.MAX)
    s = torch.as_tensor(np.exp(Sr - M.numpy()[None, :]).sum(0))
    dist.all_reduce(s, op=dist.ReduceOp.SUM)
    lse = M.numpy() + np.log(s.numpy())
    P = np.exp(Sr - lse[None, :])
    dist.destroy_process_group()
    np.save(os.path.join(out_dir, f"lse{rank}.npy"), lse)
    np.save(os.path.join(out_dir, f"P{rank}.npy"), P)
    with open(os.path.join(out_dir, f"rows{rank}.json"), "w") as f:
        json.dump([lo, hi], f)


def test_lse_over_rotation_shards(tmp_path, small_problem, oracle):
    pytest.importorskip("torch")
    import torch.multiprocessing as mp
    p = small_problem
    quat, w = p["quat"][:400], p["w"][:400] / p["w"][:400].sum()
    K = p["K"][:60].astype(np.float64)
    W = oracle.expand(p["grid"], quat, p["q"], p["w_floor"])
    S = oracle.scores(W, w, K)
    P, lse, _ = oracle.estep(S)
    np.save(tmp_path / "S.npy", S)
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path / "S.npy"),
                                         str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    for rank in range(world):
        got = np.load(tmp_path / f"lse{rank}.npy")
        assert np.max(np.abs(got - lse)) <= 1e-9 * np.max(np.abs(lse))
        lo, hi = json.loads((tmp_path / f"rows{rank}.json").read_text())
        Pr = np.load(tmp_path / f"P{rank}.npy")
        assert np.max(np.abs(Pr - P[lo:hi])) <= 1e-12
