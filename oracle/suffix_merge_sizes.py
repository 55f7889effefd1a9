"""Node counts of the storage model before and after the two reduction steps
of Section 3.2 (step 1: one global final node, Eq. 2; step 2: equal subtrees
of the last three levels merged), for the trie-size experiments' pattern
shape (Section 4: 20-symbol patterns over 4 and 52 symbols).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``): a measurement of the
storage model, run as ``python -m oracle.suffix_merge_sizes`` from the
repository root.
"""
import numpy as np

import workloads
from oracle import trie as T


def rows(sigmas=(4, 52), counts=(10, 100, 1000, 10000), length=20):
    for sigma in sigmas:
        for n in counts:
            pats = workloads.uniform_patterns(np.random.RandomState(1704 + sigma * 100000 + n),
                                              n, sigma, length, length)
            t = T.build_paper_trie(pats, sigma)
            q = t.n_nodes
            s1 = T.suffix_merge(t, 1).n_nodes
            s2 = T.suffix_merge(t, 3).n_nodes
            yield sigma, len(pats), q, s1, s2, T.paper_bytes_per_node(sigma)


def main():
    print("| alphabet | patterns | trie nodes | after step 1 (Eq. 2) | after step 2 | step 2 vs trie | "
          "bytes (trie -> step 2) |")
    print("|---|---|---|---|---|---|---|")
    for sigma, n, q, s1, s2, b in rows():
        print(f"| {sigma} | {n:,} | {q:,} | {s1:,} | {s2:,} | -{100 * (1 - s2 / q):.1f}% | "
              f"{q * b:,} -> {s2 * b:,} |")


if __name__ == "__main__":
    main()
