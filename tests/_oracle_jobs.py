"""Oracle runs for the full-size parity tests, executed in worker processes.

Each job regenerates its seeded input, sorts it with the CPU oracle and returns a
BLAKE2b-256 digest of the sorted bytes (for key-value sorts, of the keys and of the
payloads).  The tests compare it with the digest of the GPU's output for the same
input: equal digests mean byte-for-byte equal outputs (a collision has probability
2^-256).  The workers are started with the "spawn" method and import only numpy,
the oracle and the input generators, never CUDA.
"""
import hashlib

import numpy as np


def digest(*arrays) -> str:
    h = hashlib.blake2b(digest_size=32)
    for a in arrays:
        h.update(np.ascontiguousarray(a).view(np.uint8))
    return h.hexdigest()


def sort_job(n: int, dtype: str, dist: str, seed: int, pivot: str) -> str:
    import oracle
    from paper_1604_06697_gb300 import inputs
    a = inputs.make_keys(n, dtype, dist, seed)
    oracle.sort_inplace(a, pivot=pivot)
    return digest(a)


def pairs_job(n: int, seed: int, pivot: str) -> str:
    import oracle
    from paper_1604_06697_gb300 import inputs
    k, v = inputs.make_pairs(n, seed=seed)
    k, v = oracle.sort_pairs(k, v, pivot=pivot)
    return digest(k, v)


def segmented_job(nseg: int, seed: int, pivot: str) -> str:
    import oracle
    from paper_1604_06697_gb300 import inputs
    keys, off = inputs.make_segments(nseg, seed=seed)
    return digest(oracle.sort_segmented(keys, off, pivot=pivot))
