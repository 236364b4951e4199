"""Cache of tuned batched-sweep schedules.

su2_batch_tune times candidate (block size, group count) pairs on a scratch
copy of a batch's links and keeps the fastest.  The choice depends only on the GPU, the link
precision and the multiset of lattice shapes (couplings change acceptance
rates, not the work per sweep), so it is stored under that key in a JSON
file and reused by later batches of the same composition instead of being
timed again.  The file is $SU2_TUNE_CACHE, or ~/.cache/su2_gb300/batch_tune.json.
"""
import json
import os
from collections import Counter


def cache_path():
    p = os.environ.get("SU2_TUNE_CACHE")
    if p:
        return p
    return os.path.join(os.path.expanduser("~"), ".cache", "su2_gb300", "batch_tune.json")


def key(gpu, prec, dims_list):
    """GPU name | precision | shapes with their counts, in a fixed order."""
    shapes = Counter("x".join(str(int(d)) for d in dims) for dims in dims_list)
    return "%s|%s|%s" % (gpu, prec, ",".join("%s*%d" % (s, n) for s, n in sorted(shapes.items())))


def load(path=None):
    p = path or cache_path()
    try:
        with open(p) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def lookup(k, path=None):
    return load(path).get(k)


def store(k, value, path=None):
    """Record value under key k (the file is rewritten atomically)."""
    p = path or cache_path()
    d = load(p)
    d[k] = value
    os.makedirs(os.path.dirname(os.path.abspath(p)), exist_ok=True)
    tmp = "%s.tmp%d" % (p, os.getpid())
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
    os.replace(tmp, p)
