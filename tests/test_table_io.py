"""pfac_table_save / pfac_table_load on the host (no GPU): host-only tables of
every record format and layout survive a save and a load unchanged (the same
statistics, the same scan plans, byte-identical files when saved again), the
stored checksum is FNV-1a over 64-bit words (recomputed here from its
published definition), and damaged or foreign files are refused with
PFAC_EFORMAT / PFAC_EIO before anything is allocated."""
import ctypes
import os
import struct

import pytest

import workloads

pfac = pytest.importorskip("paper_1704_02272_gb300")

EINVAL, EIO, EFORMAT = -1, -9, -10
HEADER = 48

TABLES = {
    "sigma4-packed": dict(sigma=4, n=500),
    "sigma20": dict(sigma=20, n=500),
    "sigma64": dict(sigma=64, n=500),
    "sigma256-wide": dict(sigma=256, n=300),
    "sigma20-wide-records": dict(sigma=20, n=300, wide_records=True),
    "sigma20-dense": dict(sigma=20, n=300, layout=pfac.LAYOUT_DENSE),
    "sigma4-suffix-merge": dict(sigma=4, n=500, suffix_merge=True),
    "sigma20-truncated": dict(sigma=20, n=300, truncate_depth=4),
    "empty": dict(sigma=8, n=0),
}


def host_table(sigma, n, **kw):
    w = workloads.config4(sigma, max(n, 1), n_bytes=1 << 12)
    pats = w.patterns[:n]
    return pfac.Table(pats, sigma, host_only=True, **kw)


def fnv1a_words(data: bytes) -> int:
    """FNV-1a with the 64-bit offset basis and prime, one step per
    little-endian 64-bit word (the tail zero-padded)."""
    h = 0xcbf29ce484222325
    if len(data) % 8:
        data = data + bytes(8 - len(data) % 8)
    for (w,) in struct.iter_unpack("<Q", data):
        h = ((h ^ w) * 0x100000001b3) & 0xFFFFFFFFFFFFFFFF
    return h


PLAN_OPTS = [{}, dict(variant=1), dict(variant=2), dict(warps_per_cta=24), dict(records_per_slice=512)]


def plans(t):
    out = []
    for o in PLAN_OPTS:
        try:
            out.append(pfac.plan(t, **o))
        except pfac.PfacError as e:
            out.append(e.status)
    return out


@pytest.mark.parametrize("name", list(TABLES))
def test_round_trip(tmp_path, name):
    kw = dict(TABLES[name])
    with host_table(**kw) as t:
        p1 = tmp_path / "a.pfac"
        t.save(p1)
        info, pl = t.info(), plans(t)
    with pfac.Table.load(p1, host_only=True) as u:
        assert u.info() == info
        assert plans(u) == pl
        p2 = tmp_path / "b.pfac"
        u.save(p2)
    a, b = p1.read_bytes(), p2.read_bytes()
    assert a == b
    # header: magic, format 1, sizes, then the blob's bytes and the checksum
    assert a[:8] == b"PFACTBL\0"
    version, endian, dt, ib, mb, _, blob, csum = struct.unpack_from("<IIIIIIQQ", a, 8)
    assert (version, endian) == (1, 0x01020304)
    assert blob == info["device_bytes"]
    assert len(a) == HEADER + mb + blob
    assert csum == fnv1a_words(a[HEADER:])
    assert not [f for f in os.listdir(tmp_path) if ".tmp." in f]


def damaged(tmp_path, src: bytes, at: int, new: bytes, fix_checksum: bool) -> str:
    d = bytearray(src)
    d[at:at + len(new)] = new
    if fix_checksum:
        struct.pack_into("<Q", d, 40, fnv1a_words(bytes(d[HEADER:])))
    p = tmp_path / "bad.pfac"
    p.write_bytes(bytes(d))
    return str(p)


def refused(path, status):
    with pytest.raises(pfac.PfacError) as ei:
        pfac.Table.load(path, host_only=True)
    assert ei.value.status == status, str(ei.value)
    return str(ei.value)


def test_damaged_files_are_refused(tmp_path):
    with host_table(20, 300) as t:
        good = tmp_path / "good.pfac"
        t.save(good)
    src = good.read_bytes()
    _, _, _, _, mb, _, blob, _ = struct.unpack_from("<IIIIIIQQ", src, 8)
    # one flipped bit in the blob, and in the description
    assert "checksum" in refused(damaged(tmp_path, src, HEADER + mb + blob // 2,
                                         bytes([src[HEADER + mb + blob // 2] ^ 1]), False), EFORMAT)
    assert "checksum" in refused(damaged(tmp_path, src, HEADER + 4, bytes([src[HEADER + 4] ^ 0x10]),
                                         False), EFORMAT)
    # a valid checksum over a description that does not hold: the alphabet
    # size (first field), the record format (second), the records' offset
    # (the first pointer, after twelve 32-bit fields) past the blob
    assert "alphabet" in refused(damaged(tmp_path, src, HEADER, struct.pack("<I", 0), True), EFORMAT)
    assert "record format" in refused(damaged(tmp_path, src, HEADER + 4, struct.pack("<I", 5), True),
                                      EFORMAT)
    assert "section" in refused(damaged(tmp_path, src, HEADER + 48, struct.pack("<Q", blob + 64), True),
                                EFORMAT)
    # truncated file, another format version, not a table file at all
    short = tmp_path / "short.pfac"
    short.write_bytes(src[:-100])
    refused(str(short), EFORMAT)
    assert "format version" in refused(damaged(tmp_path, src, 8, struct.pack("<I", 2), False), EFORMAT)
    other = tmp_path / "other.pfac"
    other.write_bytes(b"\x7fELF" + bytes(200))
    assert "not a table file" in refused(str(other), EFORMAT)
    tiny = tmp_path / "tiny.pfac"
    tiny.write_bytes(b"PFAC")
    refused(str(tiny), EFORMAT)
    refused(str(tmp_path / "missing.pfac"), EIO)


def test_bad_arguments(tmp_path):
    with host_table(4, 50) as t:
        with pytest.raises(pfac.PfacError) as ei:
            t.save(tmp_path / "no-such-dir" / "t.pfac")
        assert ei.value.status == EIO
        p = tmp_path / "t.pfac"
        t.save(p)
    h = pfac.binding.LIB
    out = ctypes.c_void_p()
    assert h.pfac_table_load(os.fsencode(p), 0x80, None, ctypes.byref(out)) == EINVAL
    assert h.pfac_table_load(None, pfac.binding.BUILD_HOST_ONLY, None, ctypes.byref(out)) == EINVAL
    assert h.pfac_table_save(None, os.fsencode(p)) == EINVAL



# every alphabet size class the builder distinguishes (record formats, packed
# shifts, bits per symbol), in both layouts, over sets of patterns of 1 to 12
# symbols (many of them prefixes of others)
SIGMAS = [1, 2, 3, 4, 5, 8, 9, 16, 17, 32, 33, 64, 128, 129, 200, 256]


@pytest.mark.parametrize("sigma", SIGMAS)
def test_round_trip_every_alphabet_class(tmp_path, sigma):
    w = workloads.tiny_case(900 + sigma, sigma, 150, 1, 12, 64)
    for kw in ({}, {"layout": pfac.LAYOUT_DENSE}):
        with pfac.Table(w.patterns, sigma, host_only=True, **kw) as t:
            t.save(tmp_path / "a.pfac")
            info = t.info()
        with pfac.Table.load(tmp_path / "a.pfac", host_only=True) as u:
            assert u.info() == info
            u.save(tmp_path / "b.pfac")
        assert (tmp_path / "a.pfac").read_bytes() == (tmp_path / "b.pfac").read_bytes()


def test_misaligned_section_is_refused(tmp_path):
    with host_table(20, 300) as t:
        t.save(tmp_path / "good.pfac")
    src = (tmp_path / "good.pfac").read_bytes()
    # the records' offset (the first pointer of the description) moved off
    # its 4-byte alignment, checksum made valid again
    assert "section offset" in refused(damaged(tmp_path, src, HEADER + 48, struct.pack("<Q", 2), True),
                                       EFORMAT)
