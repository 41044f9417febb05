"""On-disk cache of oracle coefficient tensors for the test session (keyed by the
model's defining data).  The files are written by the oracle only."""
import hashlib
import os
import pickle

import numpy as np

from oracle import coefficients

CACHE_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), ".oracle_cache")


def _key(model, tag):
    h = hashlib.sha1()
    h.update(repr((tag, model.grid, model.layers, model.freqs)).encode())
    return h.hexdigest()[:16]


def _cached(model, tag, fn):
    os.makedirs(CACHE_DIR, exist_ok=True)
    path = os.path.join(CACHE_DIR, f"{tag}_{model.name}_{_key(model, tag)}.npy")
    if os.path.exists(path):
        return np.load(path)
    arr = fn()
    np.save(path + ".tmp.npy", arr)
    os.replace(path + ".tmp.npy", path)
    return arr


def all_offsets_cached(model, freq=None):
    f = model.freqs[0] if freq is None else freq
    return _cached(model, f"all{f:g}", lambda: coefficients.all_offsets(model.grid, model.layers, f))


def compressed_cached(model, freq=None):
    f = model.freqs[0] if freq is None else freq
    return _cached(model, f"cq{f:g}", lambda: coefficients.compressed_q(model.grid, model.layers, f))
