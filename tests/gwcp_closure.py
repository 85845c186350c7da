"""Independent brute-force closure of the GWCP relation on tiny traces.

This pins the oracle to the paper's Definition of GWCP (section "Extending WCP to GPU
Programs", rules (i)-(iv)) rather than to its Algorithms: the relation is computed as a
fixpoint of boolean matrices over event pairs, with no vector clocks, epochs, queues
or per-location state. It shares no code with the oracle or the CUDA path.

Two modes:

* ``definition``: rules (i)-(iv) as stated. Rule (iii) is composed with scoped HB on
  both sides (rule iv), rule (ii) applies to any two releases.
* ``algorithm``: the same rules with the two places where Algorithm 1 computes a
  narrower relation than the Definition made explicit:
    D1  rule (ii) only relates releases of different threads (the acquire and release
        queues of Algorithm 1 are filled only for threads t' != t);
    D2  a barrier passes on C_t, the GWCP knowledge of each thread in its scope
        (section "Tracking GWCP", barrier paragraph), so rule (iii) is composed on its
        left with the GWCP relation and program order, not with scoped HB.
  On traces where any two critical sections on one lock overlap in scope, this mode
  must equal the vector-clock oracle exactly; elsewhere the oracle may order fewer
  pairs (its release loop stops at the first record not yet ordered, and pops
  records whose release has not happened).

Races: conflicting accesses by different threads, not both atomics with overlapping
scopes, not ordered by the relation. Shared-memory locations are per block.
"""
from __future__ import annotations

import numpy as np

READ, WRITE, ATOMIC, ACQ, REL, BARRIER, FENCE = range(7)
CTA, DEVICE, WARP = 0, 1, 2


def _closure(m: np.ndarray) -> np.ndarray:
    """Reflexive-transitive closure (Warshall)."""
    r = m.copy()
    n = len(r)
    np.fill_diagonal(r, True)
    for k in range(n):
        r |= np.outer(r[:, k], r[k, :])
    return r


def _compose(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    return (a.astype(np.int32) @ b.astype(np.int32)) > 0


class Trace:
    def __init__(self, events, num_agents, agents_per_block, granularity):
        self.ev = [tuple(int(v) for v in (e["agent"], e["op"], e["scope"], e["space"], e["addr"])) for e in events]
        self.n = len(self.ev)
        self.W, self.apb, self.gran = num_agents, agents_per_block, granularity
        self.threads = [self._threads(i) for i in range(self.n)]

    def block(self, t):
        return t // self.apb

    def _threads(self, i):
        agent, op, scope, space, addr = self.ev[i]
        if op != BARRIER:
            return [agent]
        if scope == CTA:
            return list(range(addr * self.apb, (addr + 1) * self.apb))
        if self.gran == 1:
            return [agent]
        blk = self.block(agent)
        base = blk * self.apb + ((agent - blk * self.apb) // 32) * 32
        return [base + lane for lane in range(32) if (addr >> lane) & 1]

    def is_access(self, i):
        return self.ev[i][1] in (READ, WRITE, ATOMIC)

    def key(self, i):
        agent, op, scope, space, addr = self.ev[i]
        return (1, self.block(agent), addr) if space == 1 else (0, 0, addr)

    def is_write(self, i):
        return self.ev[i][1] in (WRITE, ATOMIC)

    def lock_scope(self, i):
        agent, op, scope, space, addr = self.ev[i]
        return ("dev",) if scope == DEVICE else ("blk", self.block(agent))


def _scopes_overlap(s1, s2):
    # two scoped uses overlap iff one is device-scoped or both belong to one block
    return s1[0] == "dev" or s2[0] == "dev" or s1 == s2


def _atomics_exempt(tr: Trace, a, b, lesser=False):
    if tr.ev[a][1] != ATOMIC or tr.ev[b][1] != ATOMIC:
        return False
    da, db = tr.ev[a][2] == DEVICE, tr.ev[b][2] == DEVICE
    same_block = tr.block(tr.ev[a][0]) == tr.block(tr.ev[b][0])
    if lesser:
        return (da and db) or same_block
    return da or db or same_block


def conflicting(tr: Trace, a, b, lesser=False):
    return (tr.is_access(a) and tr.is_access(b) and tr.ev[a][0] != tr.ev[b][0] and tr.key(a) == tr.key(b)
            and (tr.is_write(a) or tr.is_write(b)) and not _atomics_exempt(tr, a, b, lesser))


def analyze(events, num_agents, agents_per_block, granularity, mode="definition", lesser=False):
    """Returns (racing pairs as a set of (a, b) with a < b, relation matrix, HB matrix)."""
    tr = Trace(events, num_agents, agents_per_block, granularity)
    n = tr.n
    # program order: pairs i <= j that share a thread (a barrier belongs to each member)
    seq = {}
    for i in range(n):
        for t in tr.threads[i]:
            seq.setdefault(t, []).append(i)
    TO = np.zeros((n, n), dtype=bool)
    for t, s in seq.items():
        for x in range(len(s)):
            for y in range(x, len(s)):
                TO[s[x], s[y]] = True
    # critical sections: for each release, its acquire (innermost matching) and the
    # events of that thread from the acquire to the release
    cs_of_rel = {}
    open_stack = {t: [] for t in range(tr.W)}
    for i in range(n):
        agent, op, scope, space, addr = tr.ev[i]
        if op == ACQ:
            open_stack[agent].append(i)
        elif op == REL:
            a = open_stack[agent].pop()
            cs_of_rel[i] = a
    cs_members = {}
    for r, a in cs_of_rel.items():
        t = tr.ev[r][0]
        cs_members[r] = [i for i in seq[t] if a <= i <= r]
    # critical sections an event lies in: (lock, scope) of every acquire of its
    # thread that is open at the event
    inside = [[] for _ in range(n)]
    for i in range(n):
        if not tr.is_access(i):
            continue
        t = tr.ev[i][0]
        for j in seq[t]:
            if j >= i:
                break
            if tr.ev[j][1] == ACQ:
                rel = next((r for r, a in cs_of_rel.items() if a == j), None)
                if rel is None or rel > i:
                    inside[i].append(j)
    # scoped HB: program order, release -> later acquire of the same lock when the
    # scopes overlap, barrier (through the shared barrier event in program order)
    E = TO.copy()
    for r in range(n):
        if tr.ev[r][1] != REL:
            continue
        for a in range(r + 1, n):
            if tr.ev[a][1] == ACQ and tr.ev[a][4] == tr.ev[r][4] and _scopes_overlap(tr.lock_scope(r), tr.lock_scope(a)):
                E[r, a] = True
    HB = _closure(E)
    # rule (i): release r of a section on lock l, access e inside a section on l with
    # r before e, scopes overlap, r's section holds an access conflicting with e
    # (same location, at least one write; atomics count as writes)
    rule_i = np.zeros((n, n), dtype=bool)
    for r, members in cs_members.items():
        lock = tr.ev[r][4]
        s1 = tr.lock_scope(r)
        accs = [m for m in members if tr.is_access(m)]
        for e in range(r + 1, n):
            if not tr.is_access(e):
                continue
            held = [j for j in inside[e] if tr.ev[j][4] == lock and _scopes_overlap(s1, tr.lock_scope(j))]
            if not held:
                continue
            if any(tr.key(m) == tr.key(e) and (tr.is_write(m) or tr.is_write(e)) for m in accs):
                rule_i[r, e] = True
    # rule (iii): barrier b over threads S; e1 on t1 in S before b, e2 on t2 in S after b
    rule_iii = np.zeros((n, n), dtype=bool)
    for bi in range(n):
        if tr.ev[bi][1] != BARRIER:
            continue
        members = tr.threads[bi]
        before = [i for t in members for i in seq[t] if i < bi]
        after = [i for t in members for i in seq[t] if i > bi]
        for e1 in before:
            for e2 in after:
                rule_iii[e1, e2] = True
    rels = sorted(cs_members)
    R = np.zeros((n, n), dtype=bool)
    while True:
        rule_ii = np.zeros((n, n), dtype=bool)
        for x, r1 in enumerate(rels):
            for r2 in rels[x + 1:]:
                if tr.ev[r1][4] != tr.ev[r2][4]:
                    continue
                if not _scopes_overlap(tr.lock_scope(r1), tr.lock_scope(r2)):
                    continue
                if mode == "algorithm" and tr.ev[r1][0] == tr.ev[r2][0]:
                    continue  # D1
                if R[np.ix_(cs_members[r1], cs_members[r2])].any():
                    rule_ii[r1, r2] = True
        if mode == "definition":
            new = _compose(_compose(HB, R | rule_i | rule_ii | rule_iii), HB)
        else:
            left = R | TO  # D2: GWCP knowledge and program order, reflexive through TO
            new = (_compose(_compose(HB, rule_i | rule_ii), HB) | _compose(_compose(left, rule_iii), HB)
                   | _compose(R, HB))
        new |= R
        if (new == R).all():
            break
        R = new
    races = set()
    for a in range(n):
        for b in range(a + 1, n):
            if conflicting(tr, a, b, lesser) and not R[a, b]:
                races.add((a, b))
    return races, R, HB


def hb_races(events, num_agents, agents_per_block, granularity, lesser=False):
    tr = Trace(events, num_agents, agents_per_block, granularity)
    _, _, HB = analyze(events, num_agents, agents_per_block, granularity)
    return {(a, b) for a in range(tr.n) for b in range(a + 1, tr.n) if conflicting(tr, a, b, lesser) and not HB[a, b]}


def project(events, num_agents, agents_per_block, granularity, pairs, lesser=False):
    """Maps all racing pairs to one pair per (later access b, other thread v): the
    latest access a* by v before b that conflicts with b and is not exempt."""
    tr = Trace(events, num_agents, agents_per_block, granularity)
    out = set()
    for a, b in pairs:
        v = tr.ev[a][0]
        best = max(i for i in range(b) if tr.ev[i][0] == v and conflicting(tr, i, b, lesser))
        out.add((best, b))
    return out


def all_conflicting(events, num_agents, agents_per_block, granularity, lesser=False):
    tr = Trace(events, num_agents, agents_per_block, granularity)
    return {(a, b) for a in range(tr.n) for b in range(a + 1, tr.n) if conflicting(tr, a, b, lesser)}
