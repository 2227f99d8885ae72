"""Process-pool helpers that run the FP64 oracle on many sampled probes of a
large case (test infrastructure).  Workers are started with the 'spawn'
method (safe after CUDA has been initialised in the parent) and read the
transmission stack from a memory-mapped .npy file, so the stack is written
once and shared through the page cache.  A worker that dies makes the call
raise (BrokenProcessPool) instead of waiting."""
import concurrent.futures as cf
import multiprocessing as mp
import os

import numpy as np


def _rings_chunk(args):
    from oracle import stem as O
    params, t_path, xy = args
    t = np.load(t_path, mmap_mode="r")
    return O.multislice_rings(params, t, xy)


def multislice_rings_pool(params, t: np.ndarray, xy: np.ndarray, scratch: str, workers: int = 0,
                          timeout: float = 1800.0) -> np.ndarray:
    """oracle.multislice_rings(params, t, xy) computed by a pool of processes."""
    t_path = os.path.join(scratch, "trans.npy")
    np.save(t_path, t)
    try:
        workers = workers or max(1, min(len(xy), os.cpu_count() or 1))
        parts = [c for c in np.array_split(np.arange(len(xy)), workers) if len(c)]
        with cf.ProcessPoolExecutor(len(parts), mp_context=mp.get_context("spawn")) as ex:
            futs = [ex.submit(_rings_chunk, (params, t_path, xy[c])) for c in parts]
            out = [f.result(timeout=timeout) for f in futs]
    finally:
        os.remove(t_path)
    return np.concatenate(out, axis=0)
