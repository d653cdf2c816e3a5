"""Sharding a population over ranks (host logic; gloo ranks on the CPU)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2502_11129_b300 import population as P
from paper_2502_11129_b300 import shard as SH


def test_shards_cover_every_robot_once_and_are_contiguous():
    rng = np.random.default_rng(0)
    for n, world in ((1, 1), (5, 8), (8, 8), (9, 8), (4096, 2), (4096, 3), (1000, 7)):
        c = rng.uniform(1, 400, size=n)
        sh = SH.balanced_shards(c, world)
        assert len(sh) == world
        allidx = np.concatenate(sh)
        assert np.array_equal(np.sort(allidx), np.arange(n))
        for s in sh:
            if s.size:
                assert np.array_equal(s, np.arange(s[0], s[-1] + 1))
        if n >= world:
            assert all(s.size > 0 for s in sh)


def test_shard_costs_balance_within_one_robot():
    rng = np.random.default_rng(1)
    for world in (2, 3, 4, 8):
        c = rng.uniform(9, 441, size=4096)
        sh = SH.balanced_shards(c, world)
        share = c.sum() / world
        for s in sh:
            assert abs(c[s].sum() - share) <= c.max() + 1e-9


def test_equal_costs_split_evenly_and_bad_input_is_rejected():
    sh = SH.balanced_shards(np.ones(12), 4)
    assert [s.size for s in sh] == [3, 3, 3, 3]
    with pytest.raises(ValueError):
        SH.balanced_shards([1.0, -1.0], 2)
    with pytest.raises(ValueError):
        SH.balanced_shards([1.0], 0)


STEPS = 100


def engine_fitness(pop):
    """Fitness after STEPS steps from the population's start, simulated by the
    host engine (libb3cpu): the real simulator a rank would run on its shard."""
    from paper_2502_11129_b300 import cpu as CP
    from paper_2502_11129_b300 import sim as S
    Q, V, Sx = S.state_rows(pop, pop.q0, pop.v0, P.cpg_initial(pop))
    cs = CP.CpuSim(threads=1)
    cs.set_population(pop)
    cs.set_state(Q, V, Sx)
    cs.step(STEPS)
    f = cs.fitness()
    cs.close()
    return f


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    pop = P.grammar(37, seed=11).as_float32()
    seen = []

    def sim(sub):
        seen.append(sub.n)
        return engine_fitness(sub)

    f = SH.run_sharded(pop, sim, dist)
    np.save(os.path.join(out_dir, f"r{rank}.npy"), np.concatenate([[seen[0]], f]))
    dist.barrier()
    dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("world", [2, 3])
def test_run_sharded_gathers_every_result_on_every_rank(tmp_path, world):
    """Every rank simulates its shard with the host engine for 100 steps; the
    gathered fitness equals, bitwise and on every rank, one process
    simulating the whole population (robots are independent)."""
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    pop = P.grammar(37, seed=11).as_float32()
    ref = engine_fitness(pop).astype(np.float64)
    assert np.abs(ref).max() > 0  # the robots moved
    sizes = []
    for r in range(world):
        a = np.load(tmp_path / f"r{r}.npy")
        sizes.append(int(a[0]))
        assert np.array_equal(a[1:], ref)
    assert sum(sizes) == pop.n and all(s > 0 for s in sizes)


def test_single_rank_runs_everything_locally():
    pop = P.grammar(5, seed=2).as_float32()
    f = SH.run_sharded(pop, engine_fitness, None)
    assert np.array_equal(f, engine_fitness(pop))
