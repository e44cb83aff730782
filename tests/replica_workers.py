"""Worker for the multi-process replica test (a module of its own so that
spawned processes can import it)."""
import os


def replica_rank(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    env = bench.dist_env()
    ms = bench.max_over_ranks(1.0 + 0.5 * rank, ws, torch.device("cpu"))
    rate = bench.job_rate(1000.0, ws, ms)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, env, ms, rate))
