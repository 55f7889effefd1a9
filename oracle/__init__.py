"""CPU oracle for exact multi-pattern matching (PFAC semantics).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The GPU library
never imports it and it never imports the GPU library.

Contents
--------
``match_bf``      O1, brute force in C (definition of the result written out).
``ACOracle``      O2, Aho-Corasick with failure links in C (Section 2.2).
``pyref``         the same definition as a tiny pure-Python loop for
                  exhaustive small cases.
``trie``          the paper's storage model (Section 3.1) and node-count
                  closed forms (Eq. 1, Eq. 2), used to pin table statistics;
                  reduction step 2 (Section 3.2) as a DAG with an id side
                  channel, and a walker over it.

The result all matchers compute: distinct non-empty patterns P_j, text T and
segment offsets o_0 = 0 <= ... <= o_S = N; the sorted list of (p, j) with
o_k <= p, p + |P_j| <= o_{k+1} and T[p : p + |P_j|] == P_j (Section 2.3: one
walk per start position, every final state passed is reported).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SRC = os.path.join(_HERE, "pfac_oracle.c")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compiles the C oracle with gcc into oracle/_build/liboracle.so."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread",
                               "-o", tmp, _SRC])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            u8p = ctypes.POINTER(ctypes.c_uint8)
            u64p = ctypes.POINTER(ctypes.c_uint64)
            u32p = ctypes.POINTER(ctypes.c_uint32)
            lib.obf_match.restype = ctypes.c_int64
            lib.obf_match.argtypes = [u8p, u64p, ctypes.c_uint32, u8p, ctypes.c_uint64, u64p,
                                      ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint64,
                                      ctypes.c_int, u64p, u32p, ctypes.c_uint64]
            lib.oac_build.restype = ctypes.c_void_p
            lib.oac_build.argtypes = [u8p, u64p, ctypes.c_uint32]
            lib.oac_free.restype = None
            lib.oac_free.argtypes = [ctypes.c_void_p]
            lib.oac_nodes.restype = ctypes.c_uint32
            lib.oac_nodes.argtypes = [ctypes.c_void_p]
            lib.oac_match.restype = ctypes.c_int64
            lib.oac_match.argtypes = [ctypes.c_void_p, u8p, ctypes.c_uint64, u64p,
                                      ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint64,
                                      ctypes.c_int, u64p, u32p, ctypes.c_uint64]
            _lib = lib
    return _lib


def _ptr(a, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


def _flatten(patterns):
    lens = np.array([len(p) for p in patterns], dtype=np.uint64)
    off = np.zeros(len(patterns) + 1, dtype=np.uint64)
    np.cumsum(lens, out=off[1:])
    flat = np.frombuffer(b"".join(patterns) or b"\0", dtype=np.uint8).copy()
    return flat, off


def _prep(text, seg):
    text = np.ascontiguousarray(np.asarray(text, dtype=np.uint8))
    if text.size == 0:
        text = np.zeros(1, np.uint8)[:0]
    seg = np.ascontiguousarray(np.asarray(seg, dtype=np.uint64))
    return text, seg


def default_threads() -> int:
    return max(1, len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count() or 1)


def _run(fn, args_front, text, seg, lo, hi, threads):
    text, seg = _prep(text, seg)
    n_bytes = text.shape[0]
    hi = n_bytes if hi is None else min(hi, n_bytes)
    threads = default_threads() if threads is None else threads
    tbuf = text if n_bytes else np.zeros(1, np.uint8)
    n_seg = max(0, seg.shape[0] - 1)
    cap = 0
    dummy_p = np.zeros(1, np.uint64)
    dummy_i = np.zeros(1, np.uint32)
    total = fn(*args_front, _ptr(tbuf, ctypes.c_uint8), n_bytes, _ptr(seg, ctypes.c_uint64),
               n_seg, lo, hi, threads, _ptr(dummy_p, ctypes.c_uint64),
               _ptr(dummy_i, ctypes.c_uint32), cap)
    if total < 0:
        raise ValueError(f"oracle rejected its input (status {total})")
    pos = np.zeros(max(total, 1), np.uint64)
    ids = np.zeros(max(total, 1), np.uint32)
    if total:
        t2 = fn(*args_front, _ptr(tbuf, ctypes.c_uint8), n_bytes, _ptr(seg, ctypes.c_uint64),
                n_seg, lo, hi, threads, _ptr(pos, ctypes.c_uint64), _ptr(ids, ctypes.c_uint32),
                total)
        assert t2 == total
    return pos[:total], ids[:total]


def match_bf(patterns, text, seg, lo=0, hi=None, threads=None):
    """O1 brute force: sorted (positions uint64[], ids uint32[]) of the
    matches whose start lies in [lo, hi)."""
    lib = _load()
    flat, off = _flatten(patterns)
    return _run(lib.obf_match, (_ptr(flat, ctypes.c_uint8), _ptr(off, ctypes.c_uint64),
                                len(patterns)), text, seg, lo, hi, threads)


class ACOracle:
    """O2: Aho-Corasick automaton with failure links, built once."""

    def __init__(self, patterns):
        lib = _load()
        flat, off = _flatten(patterns)
        self._lib = lib
        self._h = lib.oac_build(_ptr(flat, ctypes.c_uint8), _ptr(off, ctypes.c_uint64),
                                len(patterns))
        if not self._h:
            raise ValueError("oracle: empty or duplicate pattern")
        self.max_len = max((len(p) for p in patterns), default=0)

    @property
    def n_nodes(self) -> int:
        return int(self._lib.oac_nodes(self._h))

    def match(self, text, seg, lo=0, hi=None, threads=None):
        return _run(self._lib.oac_match, (ctypes.c_void_p(self._h),), text, seg, lo, hi, threads)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.oac_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def match_ac(patterns, text, seg, lo=0, hi=None, threads=None):
    ac = ACOracle(patterns)
    try:
        return ac.match(text, seg, lo, hi, threads)
    finally:
        ac.close()


def pack_keys(pos, ids, id_bits=24):
    """(position, id) pairs as the packed uint64 keys position << id_bits | id,
    whose numeric order is the (position, id) order."""
    return (np.asarray(pos, np.uint64) << np.uint64(id_bits)) | np.asarray(ids, np.uint64)
