"""Test helpers: random hierarchical constraint families and tiny instances."""
import numpy as np


def random_laminar(M, rng, max_nodes=6):
    """Random hierarchical family of item sets over M items (Sec. 2.1, Definition 1):
    built by recursively splitting random subsets; caps between 1 and |S|."""
    S, C = [], []
    items = list(range(M))

    def rec(sub, depth):
        if len(S) >= max_nodes or len(sub) == 0:
            return
        mask = sum(1 << j for j in sub)
        S.append(mask)
        C.append(int(rng.integers(1, len(sub) + 1)))
        if depth >= 3 or len(sub) < 2:
            return
        parts = rng.integers(1, 4)
        perm = list(rng.permutation(sub))
        cuts = sorted(rng.choice(range(1, len(sub)), size=min(parts, len(sub) - 1), replace=False))
        prev = 0
        for c in list(cuts) + [len(sub)]:
            piece = perm[prev:c]
            prev = c
            if rng.random() < 0.7:
                rec(piece, depth + 1)

    # a forest: maybe several disjoint roots, maybe some items uncovered
    if rng.random() < 0.5:
        rec(items, 0)
    else:
        perm = list(rng.permutation(items))
        h = int(rng.integers(1, M)) if M > 1 else 1
        rec(perm[:h], 1)
        rec(perm[h:], 1)
    return S, C


def feasible_local(mask, S, C):
    return all(bin(mask & s).count("1") <= c for s, c in zip(S, C))
