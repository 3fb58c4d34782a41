"""Distribution of a batched ensemble over ranks, one GPU each: replicas only.

The replicas of an ensemble are independent Monte Carlo runs (each with its own
Philox replica word), so a multi-GPU job gives every rank a subset of them and no
data crosses between ranks; the job's time is that of the slowest rank, and each
replica's results are those it has in a single-GPU batch.  ``balance_replicas``
assigns the replicas largest first, each to the rank with the fewest sites so far
(the longest-processing-time rule), so that the ranks' site counts differ by at
most the size of one replica.
"""
from __future__ import annotations


def balance_replicas(sites, nranks):
    """Replica indices per rank (ascending within a rank) for replicas of ``sites``
    sites each; every replica goes to exactly one rank."""
    if nranks < 1:
        raise ValueError("nranks must be >= 1")
    order = sorted(range(len(sites)), key=lambda r: (-int(sites[r]), r))
    load = [0] * nranks
    parts = [[] for _ in range(nranks)]
    for r in order:
        k = min(range(nranks), key=lambda i: (load[i], i))
        parts[k].append(r)
        load[k] += int(sites[r])
    return [sorted(p) for p in parts]
