"""Oracle runs in worker processes (test infrastructure): independent long
runs of the FP64 oracle go to a pool of spawned processes, one per host core
at most, so that several beds settle at once.  The workers load the oracle's
library (built by the caller beforehand) and touch no GPU."""
import multiprocessing as mp
import os


def _run(job):
    import oracle

    sc, margin, K, n_steps = job
    sim = oracle.OracleSim(sc, margin, K)
    sim.step(n_steps)
    pos, quat, vel, angvel = sim.state()
    sim.close()
    return pos, quat, vel, angvel


def run_many(jobs):
    """[(scene, margin, rebuild interval, steps)] -> [(pos, quat, vel, angvel)]
    of each run's end state, in the order given."""
    n = max(1, min(len(jobs), os.cpu_count() or 1))
    with mp.get_context("spawn").Pool(n) as pool:
        return pool.map(_run, jobs, chunksize=1)
