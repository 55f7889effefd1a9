"""Pure-Python statement of the match set, for exhaustive small cases.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Section 2.2 states the problem (find every occurrence of patterns P in a text
T); Section 2.3 gives the failure-less semantics: one walk starts at each
input position and reports every pattern it completes.  With segments (packets)
no occurrence may cross a segment end.  The result is sorted by start position
and then by pattern id (the caller's index into the pattern list).
"""


def matches(patterns, text, seg_offsets):
    text = bytes(text)
    out = []
    seg = [int(x) for x in seg_offsets]
    for k in range(len(seg) - 1):
        a, b = seg[k], seg[k + 1]
        for p in range(a, b):
            for j, pat in enumerate(patterns):
                if p + len(pat) <= b and text[p:p + len(pat)] == pat:
                    out.append((p, j))
    out.sort()
    return out
