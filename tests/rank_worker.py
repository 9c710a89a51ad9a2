"""Worker of the multi-process CPU tests (one gloo rank per process)."""
import os


def replica_rank(rank, world, port, queue):
    import torch.distributed as dist

    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # each replica times its own steps; the slowest sets the job's time
        ms = bench.slowest_rank(10.0 + rank, "cpu")
        rate = bench.whole_job_rate(world, 200, 50, ms / 1e3)
        dist.barrier()
        queue.put((rank, ms, rate))
    finally:
        dist.destroy_process_group()
