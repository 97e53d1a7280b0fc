"""Sequential model of the level-synchronous maxId traversal (Section 4, Fig. 5/6).

Test helper only: it replays, one iteration at a time, the rule that the
paper's parallel traversal applies to every frontier vertex, so the tests can
compare the intermediate state with the worked example the paper prints
(Fig. 6) and check the final state against the oracle.  ``visit_once=True``
plants the mistake the paper warns about in Section 4 (plain fill2 run with
several thresholds in parallel, where a vertex is claimed the first time it is
seen): on the worked example it loses the fill (8, 4).
"""
from __future__ import annotations

import numpy as np

INF = 1 << 40


def maxid_levels(A, src: int, order=None, visit_once: bool = False):
    """Return (labels dict, frontier list per iteration, labels after iteration 1, L, U)."""
    adj = {v: [int(w) for w in A.row(v)] for v in range(A.n)}
    lab = {}
    frontier = []
    for w in adj[src]:
        if w == src:
            continue
        lab[w] = 0            # the paper initialises direct neighbours to 0
        if w < src:
            frontier.append(w)
    fills_L = {w for w in adj[src] if w < src}
    U = {src} | {w for w in adj[src] if w > src}
    seen = set(frontier)
    history = [sorted(frontier)]
    after1 = None
    it = 0
    while frontier:
        it += 1
        nxt = []
        fr = list(frontier) if order is None else sorted(frontier, key=order)
        for f in fr:
            nm = max(lab[f], f)
            for w in adj[f]:
                if w == src or w == f:
                    continue
                if w > src:
                    U.add(w)
                    continue
                if visit_once:
                    # plain fill2 with parallel thresholds: first visitor claims w
                    if w in seen:
                        continue
                    seen.add(w)
                    lab[w] = nm
                    if nm < w:
                        fills_L.add(w)
                    nxt.append(w)
                    continue
                old = lab.get(w, INF)
                if nm < old:
                    lab[w] = nm
                    if nm < w:
                        fills_L.add(w)
                    if old > w:           # proposal max(lab, w) changed
                        if w not in nxt:
                            nxt.append(w)
        if it == 1:
            after1 = dict(lab)
        frontier = nxt
        if frontier:
            history.append(sorted(frontier))
    return lab, history, after1, sorted(fills_L), sorted(U)
