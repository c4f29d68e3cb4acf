"""The depth-bucket map that orders tile lists (hard raster and soft renderer), evaluated in FP32 on the CPU.

Both kernels place a tile's 32-bit depth keys k in [lo, hi] into NB = 256 buckets by
b = min(NB - 1, int(float32(k - lo) * float32(NB / (float32(hi - lo) + 1)))).  Their early exit and exact
order rest on one property: every key of a bucket is <= every key of a later bucket (the map is monotone,
ties included).  This checks it with the same FP32 operations (round-to-nearest conversion, one rounded
product, truncation) on random, clustered and extreme key sets.
"""
import numpy as np
import pytest

NB = 256


def bucket(keys, lo, hi):
    k = np.asarray(keys, np.uint64)
    scale = np.float32(NB) / (np.float32(np.uint32(hi - lo)) + np.float32(1.0))
    x = (k - np.uint64(lo)).astype(np.uint32).astype(np.float32) * scale
    return np.minimum(NB - 1, x.astype(np.int64))


def key_sets():
    rng = np.random.default_rng(7)
    yield rng.integers(0, 2 ** 32, 2048, dtype=np.uint64)                       # full range
    yield np.concatenate([rng.integers(1000, 1100, 2000, dtype=np.uint64), [2 ** 32 - 1]])  # cluster + outlier
    yield np.arange(2 ** 32 - 3000, 2 ** 32, dtype=np.uint64)                   # top of the range, dense
    yield np.array([5, 5, 5, 5], np.uint64)                                     # one key
    yield np.array([0, 2 ** 32 - 1], np.uint64)                                 # the two extremes
    yield (rng.normal(2 ** 31, 2 ** 20, 4096).astype(np.int64)).astype(np.uint64)  # narrow Gaussian


@pytest.mark.parametrize("idx", range(6))
def test_buckets_are_ordered_by_key(idx):
    keys = list(key_sets())[idx]
    lo, hi = int(keys.min()), int(keys.max())
    b = bucket(keys, lo, hi)
    assert b.min() >= 0 and b.max() <= NB - 1
    order = np.argsort(keys, kind="stable")
    # monotone: sorting by key never decreases the bucket
    assert (np.diff(b[order]) >= 0).all()
    # hence each bucket's smallest key is a lower bound for every later entry of the bucket-ordered list
    present = np.unique(b)
    mins = np.array([keys[b == v].min() for v in present])
    maxs = np.array([keys[b == v].max() for v in present])
    assert (maxs[:-1] <= mins[1:]).all()
    # equal keys always share a bucket (the exact soft order sorts ties by id inside one bucket)
    for v in np.unique(keys)[:64]:
        assert len(np.unique(b[keys == v])) == 1
