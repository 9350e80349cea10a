"""Runs the oracle on instances of the 256-instance batched workload in a
pool of processes (test infrastructure, used by the full-size batch test).

The pool starts with the spawn method (no process is forked after the GPU
was used) and gives each worker one OpenMP thread, so that the instances run
side by side on every host core.  A worker regenerates its instance from the
seeded generator and returns the oracle's results for it."""
import os

import numpy as np


def _init():
    os.environ["OMP_NUM_THREADS"] = "1"


def sample_rows(i, n, m=512):
    return np.sort(np.random.default_rng(1000 + i).choice(n, min(m, n), replace=False))


def instance_oracle(i):
    import oracle
    import synth
    I = synth.batch_instances(only=[i])[0]
    cfg = I["cfg"]
    ref = oracle.run_workload(dict(cfg=cfg, x=I["x"], a=I["a"], b=I["b"], w=I["w"], silk=I["silk"]),
                              assign_rows=sample_rows(i, cfg.n))
    return dict(i=i, codes=ref["codes"].astype(np.int32), obj_bucket=ref["buckets"].obj_bucket,
                seeds=ref["seeds"].sets(), centres=ref.get("centres"), labels=ref["labels"], rows=ref["rows"])


def run(indices, workers=None):
    """Yields the oracle's result of every instance in ``indices`` (in any order)."""
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor, as_completed
    workers = workers or max(1, (os.cpu_count() or 1))
    with ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn"), initializer=_init) as ex:
        futs = [ex.submit(instance_oracle, int(i)) for i in indices]
        for f in as_completed(futs):
            yield f.result()
