"""Small graph utilities for the tests: independent restatements of textbook
definitions (Newman's pairwise modularity, BFS components) in plain Python."""
from __future__ import annotations

from collections import deque

import numpy as np


def csr_from_edges(n, edges, weights=None):
    """Symmetric CSR (int64 off, int32 col, int64 w) from undirected edges;
    an edge (i, i) becomes one self-loop arc."""
    rows = [[] for _ in range(n)]
    for k, (u, v) in enumerate(edges):
        w = 1 if weights is None else int(weights[k])
        rows[u].append((v, w))
        if u != v:
            rows[v].append((u, w))
    off = np.zeros(n + 1, np.int64)
    col, wt = [], []
    for i in range(n):
        r = sorted(rows[i])
        off[i + 1] = off[i] + len(r)
        col += [c for c, _ in r]
        wt += [x for _, x in r]
    return off, np.array(col, np.int32), np.array(wt, np.int64)


def newman_numerator(off, col, w, C) -> int:
    """Q * (2m)^2 from Newman's pairwise form
    Q = 1/(2m) sum_ij [A_ij - k_i k_j / 2m] delta(c_i, c_j), in exact integers."""
    n = len(off) - 1
    k = [int(w[off[i]:off[i + 1]].sum()) for i in range(n)]
    m2 = sum(k)
    a_in = 0
    for i in range(n):
        for a in range(off[i], off[i + 1]):
            if C[i] == C[col[a]]:
                a_in += int(w[a])
    kk = 0
    groups = {}
    for i in range(n):
        groups.setdefault(int(C[i]), []).append(k[i])
    for ks in groups.values():
        s = sum(ks)
        kk += s * s  # sum_{i,j in c} k_i k_j
    return m2 * a_in - kk


def components(off, col, members):
    """Connected components of the subgraph induced by `members` (a set)."""
    seen, comps = set(), []
    for r in sorted(members):
        if r in seen:
            continue
        comp, q = [], deque([r])
        seen.add(r)
        while q:
            u = q.popleft()
            comp.append(u)
            for a in range(off[u], off[u + 1]):
                v = int(col[a])
                if v in members and v not in seen:
                    seen.add(v)
                    q.append(v)
        comps.append(sorted(comp))
    return comps


def disconnected_communities(off, col, C) -> int:
    """Number of communities of C that are not connected (BFS per community)."""
    off = np.asarray(off)
    col = np.asarray(col)
    C = np.asarray(C)
    order = np.argsort(C, kind="stable")
    bounds = np.flatnonzero(np.diff(C[order])) + 1
    bad = 0
    n = len(C)
    label = np.full(n, -1, np.int64)
    for grp in np.split(order, bounds):
        if len(grp) <= 1:
            continue
        c = C[grp[0]]
        r = int(grp[0])
        label[r] = r
        q = deque([r])
        cnt = 1
        while q:
            u = q.popleft()
            for a in range(off[u], off[u + 1]):
                v = int(col[a])
                if C[v] == c and label[v] != r:
                    label[v] = r
                    cnt += 1
                    q.append(v)
        if cnt != len(grp):
            bad += 1
    return bad


def set_partitions(n):
    """All set partitions of range(n) as restricted growth strings."""
    a = [0] * n

    def rec(i, mx):
        if i == n:
            yield list(a)
            return
        for v in range(mx + 2):
            a[i] = v
            yield from rec(i + 1, max(mx, v))

    if n == 0:
        yield []
        return
    yield from rec(1, 0)
