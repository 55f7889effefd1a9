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
