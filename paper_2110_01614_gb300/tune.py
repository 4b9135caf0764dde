"""Persistent cache of the grouped launch's autotuned configuration.

nsdf_autotune_grouped (C ABI) times every tile shape / occupancy pair on the
actual problem.  This module remembers the winner per (GPU, SM count, network
shape, precision, problem-size bucket) in a JSON file so that later processes
apply it with nsdf_set_grouped_config instead of re-timing.
"""

import json
import os

import torch

from . import nsdf_autotune_grouped, nsdf_set_grouped_config

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "nsdf", "tune.json")


def _key(net, max_total):
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    bucket = max(1, int(max_total)).bit_length()          # power-of-two size bucket
    a = net.arch
    return (f"{props.name}|sm{props.multi_processor_count}|w{a.width}|L{a.n_hidden}|"
            f"s{a.skip_layer}|b{a.beta:g}|p{net.precision}|n{net.n_nets}|2^{bucket}")


def load(path=DEFAULT_CACHE):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def tuned_grouped(net, pts, offsets, counts, max_total, eps, out_pts, out_n_sdf=None,
                  path=DEFAULT_CACHE, retune=False):
    """Apply the cached configuration for this problem, tuning (and caching) it if absent.

    Returns (points per thread, CTAs per SM).  Tuning runs the problem a few
    times and synchronises; call it outside CUDA-graph capture.
    """
    cache = load(path)
    key = _key(net, max_total)
    if key in cache and not retune:
        pt, cps = cache[key]
        nsdf_set_grouped_config(net.ctx, pt, cps)
        return pt, cps
    pt, cps = nsdf_autotune_grouped(net.ctx, pts, offsets, counts, max_total, eps, out_pts,
                                    out_n_sdf)
    cache[key] = [pt, cps]
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)
    return pt, cps
