"""Plain tree searches over the Monotone Scene Generation Tree -- TEST
INFRASTRUCTURE ONLY.

The MSGT (Sec. IV-A): the root is the empty assignment; a child adds one
more object O_{j+1} = (type, x, y, yaw) that does not occlude the parent's
render (Eq. (3)); the edge cost is dJ_r + dJ_o (+ residual at level K)
(Eq. (4)); every state with all K objects is a goal and the answer is the
cheapest root-to-goal path.

Readings where the paper is silent:
  - level j branches over the distinct types still unplaced times every pose
    (the paper's d^{K-i} count for the no-repetition case);
  - a state is keyed by the sorted multiset of its objects: the same set
    reached in another order has the same render and hence the same cost-to-go
    (the paper keeps one ordering, a tree instead of a DAG); the search keeps
    the cheapest g per key;
  - among minimum-cost goals the lexicographically smallest sorted key wins;
    the search keeps popping while the smallest open g does not exceed the
    best goal's g, because zero-cost edges exist.
"""
from __future__ import annotations

import heapq
import math
import itertools
from collections import Counter

import numpy as np

from . import eval_batch


def key_of(objs) -> tuple:
    return tuple(sorted((int(o["mesh"]), int(o["ix"]), int(o["iy"]), int(o["iyaw"])) for o in objs))


def symmetric_yaws(grid, syms):
    """Per mesh, the yaw indices a search over a symmetric mesh keeps: yaw k
    is dropped when a smaller index j has theta_k - theta_j a multiple of
    2 pi / sym (Sec. IV-E: a rotationally symmetric object needs only (x, y));
    angles from the pose table's (cos, sin) in double, to 1e-6 of a period."""
    th = [math.atan2(float(s), float(c)) for c, s in grid.cos_sin]
    out = {}
    for m, sym in enumerate(syms):
        keep = []
        for k in range(len(th)):
            if not any(abs(t - round(t)) < 1e-6 for t in ((th[k] - th[j]) * max(int(sym), 1) / (2 * math.pi)
                                                           for j in keep)):
                keep.append(k)
        out[m] = keep
    return out


def _children(grid, remaining_types, yaws=None):
    """Every pose of every remaining type (yaws: per mesh the yaw indices to
    keep, None = all)."""
    from paper_1510_05613_gb300.synth import all_hypotheses
    h = all_hypotheses(grid, sorted(set(remaining_types)))
    if yaws is None:
        return h
    keep = np.zeros(len(h), bool)
    for m, ks in yaws.items():
        keep |= (h["mesh"] == m) & np.isin(h["iyaw"], ks)
    return h[keep]


def _remaining(multiset, placed):
    c = Counter(multiset)
    c.subtract(int(o["mesh"]) for o in placed)
    return [m for m, n in c.items() for _ in range(n) if n > 0]


def uniform_cost_search(world, depth, grid, multiset, threads: int = 0, max_expansions: int = 10 ** 7,
                        yaws=None):
    """Dijkstra (A* with h = 0) over set-keyed MSGT states. yaws: per mesh
    the yaw indices the tree places it at (symmetric_yaws), None = all.

    Returns (cost, goal_key, expansions)."""
    from paper_1510_05613_gb300.synth import OBJ_DTYPE
    K = len(multiset)
    root = np.zeros(0, OBJ_DTYPE)
    heap = [(0, (), 0)]
    states = {(): root}
    best_g = {(): 0}
    closed = set()
    best_goal = None  # (g, key)
    expansions = 0
    tie = itertools.count(1)
    while heap:
        g, key, _ = heapq.heappop(heap)
        if best_goal is not None and g > best_goal[0]:
            break
        if key in closed or g > best_g[key]:
            continue
        closed.add(key)
        s = states[key]
        if len(s) == K:
            if best_goal is None or (g, key) < best_goal:
                best_goal = (g, key)
            continue
        expansions += 1
        if expansions > max_expansions:
            raise RuntimeError("expansion limit")
        hyps = _children(grid, _remaining(multiset, s), yaws)
        recs = eval_batch(world, depth, [s], np.zeros(len(hyps), np.int32), hyps, K, threads)
        for h, r in zip(hyps, recs):
            if r[3] > 0:
                continue  # occludes the parent: not a successor (Eq. (3))
            c = int(r[0]) + int(r[1]) + int(r[2])
            child = np.concatenate([s, np.array([h], OBJ_DTYPE)])
            ck = key_of(child)
            if ck in closed:
                continue
            ng = g + c
            if ng < best_g.get(ck, 1 << 62):
                best_g[ck] = ng
                states[ck] = child
                heapq.heappush(heap, (ng, ck, next(tie)))
    if best_goal is None:
        return None, None, expansions
    return best_goal[0], best_goal[1], expansions


def exhaustive(world, depth, grid, multiset, threads: int = 0):
    """Every valid ordered sequence of K placements, summed edge costs; the
    minimum cost and, among ties, the smallest sorted key. Tiny inputs only."""
    from paper_1510_05613_gb300.synth import OBJ_DTYPE
    K = len(multiset)
    frontier = [(np.zeros(0, OBJ_DTYPE), 0)]
    for level in range(K):
        parents = [s for s, _ in frontier]
        hyp_parent, hyps = [], []
        for i, s in enumerate(parents):
            hs = _children(grid, _remaining(multiset, s))
            hyps.append(hs)
            hyp_parent.append(np.full(len(hs), i, np.int32))
        hyps = np.concatenate(hyps) if hyps else np.zeros(0, OBJ_DTYPE)
        hyp_parent = np.concatenate(hyp_parent) if hyp_parent else np.zeros(0, np.int32)
        recs = eval_batch(world, depth, parents, hyp_parent, hyps, K, threads)
        nxt = []
        for h, p, r in zip(hyps, hyp_parent, recs):
            if r[3] > 0:
                continue
            g = frontier[p][1] + int(r[0]) + int(r[1]) + int(r[2])
            nxt.append((np.concatenate([parents[p], np.array([h], OBJ_DTYPE)]), g))
        frontier = nxt
    if not frontier:
        return None, None
    best = min((g, key_of(s)) for s, g in frontier)
    return best[0], best[1]


def focal_mha(world, depth, grid, multiset, w: float, heuristics=("depth", "overlap"), n_obs: int = 0,
              threads: int = 0, max_expansions: int = 10 ** 6):
    """Focal-MHA* as Sec. IV-B describes it, one expansion per iteration:
    the anchor orders the open states by g + h0 (h0 = 0); the focal set holds
    the open states with g <= w * (smallest anchor key); the queues take turns
    (anchor, then each inadmissible heuristic picking its minimum over the
    focal set). h_depth(s) = K - |s|; h_overlap(s) = |I| - |I n V_j|, kept per
    state from the records' n_vol; any other entry of `heuristics` is a
    callable h(sorted key) (Theorem 2 holds for every inadmissible heuristic).
    Stops when the best goal has g <= w * (smallest anchor key). Returns
    (cost, goal_key, expansions)."""
    from paper_1510_05613_gb300.synth import OBJ_DTYPE
    K = len(multiset)
    states = {(): (np.zeros(0, OBJ_DTYPE), 0, n_obs)}  # key -> (objects, g, h_overlap)
    open_set = {()}
    closed = set()
    best = None
    expansions = 0
    queues = ["anchor"] + list(heuristics)
    turn = 0
    while open_set:
        f0 = min(states[k][1] for k in open_set)
        if best is not None and best[0] <= w * f0:
            break
        q = queues[turn % len(queues)]
        turn += 1
        if q == "anchor":
            key = min(open_set, key=lambda k: (states[k][1], k))
        else:
            focal = [k for k in open_set if states[k][1] <= w * f0]
            if callable(q):
                h = q
            else:
                h = (lambda k: K - len(k)) if q == "depth" else (lambda k: states[k][2])
            key = min(focal, key=lambda k: (h(k), states[k][1], k))
        open_set.discard(key)
        closed.add(key)
        s, g, hov = states[key]
        expansions += 1
        if expansions > max_expansions:
            raise RuntimeError("expansion limit")
        hyps = _children(grid, _remaining(multiset, s))
        recs = eval_batch(world, depth, [s], np.zeros(len(hyps), np.int32), hyps, K, threads)
        for hh, r in zip(hyps, recs):
            if r[3] > 0:
                continue
            child = np.concatenate([s, np.array([hh], OBJ_DTYPE)])
            ck = key_of(child)
            ng = g + int(r[0]) + int(r[1]) + int(r[2])
            if len(child) == K:
                if best is None or (ng, ck) < best:
                    best = (ng, ck)
                continue
            if ck not in states or ng < states[ck][1]:
                states[ck] = (child, ng, hov - int(r[6]))
                closed.discard(ck)
                open_set.add(ck)
    if best is None:
        return None, None, expansions
    return best[0], best[1], expansions
