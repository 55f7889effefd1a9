"""GB300-native failure-less Aho-Corasick (PFAC) matching over a compressed
state-transition table.

The matcher lives in ``libpfac.so`` (C ABI in include/pfac.h): a host C++
builder of the bitmap trie and hand-written sm_103a kernels.  This package is
its thin Python binding; importing it fails when the library is not built.
"""
from .binding import (ID_BITS, LAYOUT_COMPRESSED, LAYOUT_DENSE, VARIANT_DEFAULT,  # noqa: F401
                      VARIANT_DSMEM, VARIANT_FILTER, PfacError, Server, Table, autotune,
                      match, match_async, match_host, match_into, match_noalloc, plan, single_segment, unpack, verify,
                      verify_into,
                      version,
                      workspace_bytes)
