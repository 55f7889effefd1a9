"""The paper's storage model of the failure-less trie, written plainly.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Section 3.1 (Storage Model): the patterns are sorted alphabetically and
inserted breadth-first into one contiguous array of node structures; node 0
is the root.  A node holds a bitmap with one bit per alphabet symbol (bit c
set when the node has a child on symbol c) and the offset of its first child,
0 when it has no child.  Siblings are contiguous and ordered by symbol, so
the child on symbol c is found with Eq. 1:

    child = node.offset + i,   i = number of bitmap bits set below c.

The record costs |Sigma|/8 bytes of bitmap plus a 4-byte offset: 36 bytes at
|Sigma| = 256 and 8 bytes at |Sigma| = 32 (Section 3.1).  A dense state-
transition table instead keeps one 4-byte next state per symbol per node.

Section 3.2, Eq. 2: every pattern's last node has no children, so all those
leaves can share one global final node; with |P| patterns that each end in a
leaf the node count drops to Q - (|P| - 1).  When some patterns are prefixes of
others only the childless final nodes are leaves, and the count is
Q - (L - 1) for L leaves (see ``leaf_merged_count``).
"""
from __future__ import annotations

from dataclasses import dataclass


@dataclass
class PaperTrie:
    sigma: int
    offset: list      # first-child index per node, 0 when childless
    bitmap: list      # int bitmap per node, bit c = child on symbol c
    final_id: list    # pattern id ending at the node, or -1
    depth: list

    @property
    def n_nodes(self) -> int:
        return len(self.offset)

    def child(self, node: int, c: int):
        """Eq. 1: offset of the first child plus the rank of c's bit."""
        bm = self.bitmap[node]
        if not (bm >> c) & 1:
            return None
        i = bin(bm & ((1 << c) - 1)).count("1")
        return self.offset[node] + i

    @property
    def n_leaves(self) -> int:
        return sum(1 for bm in self.bitmap if bm == 0) if self.n_nodes > 1 else 0


def build_paper_trie(patterns, sigma: int) -> PaperTrie:
    """Breadth-first construction over the alphabetically sorted patterns.

    Each node is a contiguous range of the sorted pattern list sharing the
    node's prefix; the node's children are the distinct symbols at the next
    position among the range's longer patterns, taken in symbol order.  The
    queue of ranges is processed first-in first-out, so nodes are numbered
    level by level and siblings are contiguous.
    """
    order = sorted(range(len(patterns)), key=lambda j: patterns[j])
    srt = [patterns[j] for j in order]
    offset, bitmap, final_id, depth = [0], [0], [-1], [0]
    queue = [(0, 0, len(srt), 0)]   # (node, lo, hi, depth)
    head = 0
    while head < len(queue):
        node, lo, hi, d = queue[head]
        head += 1
        # a pattern equal to the node's prefix ends here (it sorts first)
        i = lo
        if i < hi and len(srt[i]) == d:
            final_id[node] = order[i]
            i += 1
        first = True
        while i < hi:
            c = srt[i][d]
            k = i
            while k < hi and srt[k][d] == c:
                k += 1
            idx = len(offset)
            offset.append(0)
            bitmap.append(0)
            final_id.append(-1)
            depth.append(d + 1)
            if first:
                offset[node] = idx
                first = False
            bitmap[node] |= 1 << c
            queue.append((idx, i, k, d + 1))
            i = k
    return PaperTrie(sigma, offset, bitmap, final_id, depth)


def walk_matches(trie: PaperTrie, text, seg_offsets):
    """Failure-less matching over the storage model: a walk from the root at
    every start position, following Eq. 1 until a symbol has no child or the
    segment ends, reporting every final node passed (Section 2.3)."""
    text = bytes(text)
    seg = [int(x) for x in seg_offsets]
    out = []
    for k in range(len(seg) - 1):
        a, b = seg[k], seg[k + 1]
        for p in range(a, b):
            node = 0
            q = p
            while q < b:
                c = text[q]
                if c >= trie.sigma:
                    break
                nxt = trie.child(node, c)
                if nxt is None:
                    break
                node = nxt
                q += 1
                if trie.final_id[node] >= 0:
                    out.append((p, trie.final_id[node]))
    out.sort()
    return out


def prefix_set_count(patterns) -> int:
    """Closed form of the trie size: one root plus one node per distinct
    non-empty prefix of the pattern set."""
    return 1 + len({p[:k] for p in patterns for k in range(1, len(p) + 1)})


def leaf_count(patterns) -> int:
    """Number of childless nodes: patterns that are not a proper prefix of
    another pattern."""
    s = set(patterns)
    proper = {p[:k] for p in s for k in range(1, len(p))}
    return sum(1 for p in s if p not in proper)


def leaf_merged_count(q: int, leaves: int) -> int:
    """Eq. 2 generalised: all leaves merged into one global final node."""
    return q - (leaves - 1) if leaves else q


def paper_bytes_per_node(sigma: int) -> int:
    """Bitmap of |Sigma| bits rounded to bytes plus the 4-byte offset."""
    return (sigma + 7) // 8 + 4


def paper_layout_bytes(q: int, sigma: int) -> int:
    return q * paper_bytes_per_node(sigma)


def dense_stt_bytes(q: int, sigma: int) -> int:
    """One 4-byte next state per (node, symbol)."""
    return q * 4 * sigma


# --------------------------------------------------------------------------
# Section 3.2, step 2: merging the last levels of the trie
# --------------------------------------------------------------------------
#
# Reading: a node's subtree is "in the last three levels" when it is at most
# three levels tall (height 0 = a leaf, height <= 2).  Two such nodes merge
# when their subtrees are equal: same finality and the same children on the
# same symbols, the children compared after merging (bottom up).  With
# ``levels = 1`` only leaves merge, which is step 1 (Eq. 2).  The merged
# structure is a DAG; a merged final node stands for several patterns, so it
# no longer names one: a walk reports (start, length) and the id comes from
# a side channel keyed by the matched bytes (one table per pattern length).
#
# Node counts follow the paper's accounting (nodes x bytes per node).  Shared
# children are not contiguous for every parent, so the Eq. 1 layout would need
# an indirection for them; the counts ignore that, as the paper does.


@dataclass
class DagTrie:
    sigma: int
    children: list    # per node: dict symbol -> node
    final: list       # per node: bool

    @property
    def n_nodes(self) -> int:
        return len(self.children)


def heights(trie: PaperTrie) -> list:
    """Height of every node (0 for a leaf), children before parents: nodes
    are numbered breadth-first, so a reverse scan sees children first."""
    h = [0] * trie.n_nodes
    for v in range(trie.n_nodes - 1, -1, -1):
        bm, o = trie.bitmap[v], trie.offset[v]
        k = bin(bm).count("1")
        if k:
            h[v] = 1 + max(h[o + i] for i in range(k))
    return h


def suffix_merge(trie: PaperTrie, levels: int = 3) -> DagTrie:
    """Merge equal subtrees at most ``levels`` levels tall (Section 3.2)."""
    h = heights(trie)
    n = trie.n_nodes
    new_id = [-1] * n
    sig_to_id = {}
    children, final = [], []

    def kids(v):
        bm, o = trie.bitmap[v], trie.offset[v]
        syms = [c for c in range(trie.sigma) if (bm >> c) & 1]
        return [(c, o + i) for i, c in enumerate(syms)]

    # bottom up: a node's children get their ids first
    for v in sorted(range(n), key=lambda x: h[x]):
        ks = tuple((c, new_id[u]) for c, u in kids(v))
        fin = trie.final_id[v] >= 0
        if h[v] < levels and v != 0:
            key = (fin, ks)
            if key in sig_to_id:
                new_id[v] = sig_to_id[key]
                continue
            sig_to_id[key] = len(children)
        new_id[v] = len(children)
        children.append(dict(ks))
        final.append(fin)
    # the root first, as in the breadth-first array
    root = new_id[0]
    order = [root] + [i for i in range(len(children)) if i != root]
    pos = {old: i for i, old in enumerate(order)}
    return DagTrie(trie.sigma, [{c: pos[u] for c, u in children[old].items()} for old in order],
                   [final[old] for old in order])


def dag_strings(dag: DagTrie) -> set:
    """Every string the DAG accepts (paths from the root to a final node)."""
    out = set()
    stack = [(0, b"")]
    while stack:
        v, s = stack.pop()
        if dag.final[v] and s:
            out.add(s)
        for c, u in dag.children[v].items():
            stack.append((u, s + bytes([c])))
    return out


def side_channel(patterns) -> dict:
    """Pattern id by length and bytes: the id a merged final node cannot
    hold."""
    t = {}
    for j, p in enumerate(patterns):
        t.setdefault(len(p), {})[bytes(p)] = j
    return t


def dag_walk_matches(dag: DagTrie, side: dict, text, seg_offsets):
    """Failure-less matching over the merged DAG: a walk from the root at
    every start position; a final node reached after L symbols reports the
    pattern the side channel names for the L matched bytes."""
    text = bytes(text)
    seg = [int(x) for x in seg_offsets]
    out = []
    for k in range(len(seg) - 1):
        a, b = seg[k], seg[k + 1]
        for p in range(a, b):
            v, q = 0, p
            while q < b:
                nxt = dag.children[v].get(text[q])
                if nxt is None:
                    break
                v = nxt
                q += 1
                if dag.final[v]:
                    out.append((p, side[q - p][text[p:q]]))
    out.sort()
    return out
