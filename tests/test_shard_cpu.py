"""Multi-rank path on CPU: the LPT slice planner and the sharded solve with
its gather, as two gloo ranks on 127.0.0.1.

The per-slice work here is the oracle's initialisation of Alg. 1 on tiny
slices (host code); on a GPU machine each rank would run its share through the
library instead.  The sharded result must equal the single-process result
item for item, whatever the plan."""
import itertools
import os
import socket
import tempfile

import numpy as np
import pytest

from paper_2308_01290_gb300.shard import lpt_plan, slice_cost


def test_lpt_plan_covers_every_item_once():
    rng = np.random.default_rng(0)
    for world in (1, 2, 3, 5):
        costs = rng.uniform(1, 10, size=23)
        plan = lpt_plan(costs, world)
        assert len(plan) == world
        assert sorted(i for p in plan for i in p) == list(range(23))


def test_lpt_plan_within_graham_bound_of_optimum():
    """LPT's makespan is at most (4/3 - 1/(3m)) times the optimum (Graham);
    the optimum comes from brute force over all assignments."""
    rng = np.random.default_rng(1)
    for world in (2, 3):
        for _ in range(20):
            n = int(rng.integers(2, 8))
            costs = rng.integers(1, 20, size=n).astype(float)
            plan = lpt_plan(costs, world)
            span = max(sum(costs[i] for i in p) for p in plan)
            best = min(max(sum(costs[i] for i in range(n) if a[i] == r) for r in range(world))
                       for a in itertools.product(range(world), repeat=n))
            assert span <= (4.0 / 3.0 - 1.0 / (3 * world)) * best + 1e-9


def test_lpt_plan_balances_uneven_slices():
    sizes = [256, 320, 384, 448, 512] * 4
    costs = [slice_cost(n, n, 100) for n in sizes]
    plan = lpt_plan(costs, 4)
    loads = [sum(costs[i] for i in p) for p in plan]
    assert max(loads) / min(loads) < 1.1


def _slices():
    from synthetic import phantoms as ph
    out = []
    for k, n in enumerate([12, 16, 8, 20, 10]):
        P = ph.small_phantom(50 + k, n=n)
        out.append((n, P["Z"], P["rhoe"]))
    return out


def _solve(items):
    from oracle import alg1, model
    from synthetic import phantoms as ph
    acq = ph.acquisition("small", n=8)
    tab = model.Tables(acq.low, acq.high)
    res = []
    for n, Z, rho in items:
        uL = model.mu_hat(rho, Z, 60.0)
        uH = model.mu_hat(rho, Z, 90.0)
        st = alg1.init_state(uL, uH, tab)
        res.append(np.stack([st["rhoe"], st["zt"]]))
    return res


def _rank(rank, world, port, out_path):
    import pickle

    import torch.distributed as dist

    from paper_2308_01290_gb300.shard import solve_sharded

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        items = _slices()
        got = solve_sharded(items, lambda x: slice_cost(x[0], x[0], 1), _solve)
        if rank == 0:
            with open(out_path, "wb") as f:
                pickle.dump(got, f)
        else:
            assert got is None
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_sharded_solve_two_gloo_ranks_equals_single_process():
    import pickle

    import torch.multiprocessing as mp

    pytest.importorskip("torch.distributed")
    with tempfile.TemporaryDirectory() as d:
        out = os.path.join(d, "res.pkl")
        mp.start_processes(_rank, args=(2, _free_port(), out), nprocs=2, join=True, start_method="spawn")
        with open(out, "rb") as f:
            got = pickle.load(f)
    ref = _solve(_slices())
    assert len(got) == len(ref)
    for a, b in zip(got, ref):
        assert np.array_equal(a, b)
