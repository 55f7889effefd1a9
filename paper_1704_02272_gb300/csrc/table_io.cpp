// pfac_table_save / pfac_table_load: a built table written to a file and
// read back (checkpoint and resume; the paper builds the compressed table of
// Section 3.1 once and only reads it afterwards).
//
// File: FileHeader, FileMeta (the DevTable with each pointer replaced by its
// offset into the blob, NO_SECTION for none; the table statistics, the
// prefix depths held, the tuned defaults), then the blob bytes.
#include <cuda_runtime.h>
#include <stdio.h>
#include <string.h>
#include <unistd.h>

#include <new>
#include <string>
#include <type_traits>
#include <vector>

#include "internal.h"

using namespace pfac;

namespace {

constexpr char MAGIC[8] = {'P', 'F', 'A', 'C', 'T', 'B', 'L', 0};
constexpr uint32_t FORMAT_VERSION = 1;
constexpr uint32_t ENDIAN_MARK = 0x01020304u;
constexpr uint64_t NO_SECTION = ~0ull;

struct FileHeader {
    char magic[8];
    uint32_t version;
    uint32_t endian;          // ENDIAN_MARK as the writer stored it
    uint32_t devtable_bytes;  // sizeof(DevTable)
    uint32_t info_bytes;      // sizeof(pfac_table_info_t)
    uint32_t meta_bytes;      // sizeof(FileMeta)
    uint32_t reserved;
    uint64_t blob_bytes;
    uint64_t checksum;        // over FileMeta and the blob
};
static_assert(sizeof(FileHeader) == 48, "header is 48 bytes");

struct FileMeta {
    DevTable dev;  // pointers hold offsets into the blob (NO_SECTION: none)
    pfac_table_info_t info;
    uint32_t kmin, kmax;
    uint32_t tuned[10];
    uint32_t pad;
    double match_density;
};

// Calls fn(p) with a reference to every pointer field p of a DevTable.
template <class Fn>
void for_each_section(DevTable &d, Fn &&fn) {
    fn(d.rec);
    fn(d.fin);
    fn(d.fbc);
    fn(d.fvals);
    fn(d.leaf_fin);
    fn(d.pool);
    for (int k = 0; k <= KMAX; k++) {
        fn(d.F[k]);
        fn(d.C[k]);
        fn(d.E[k]);
        fn(d.M[k]);
        fn(d.B[k]);
    }
    fn(d.G);
    fn(d.pat);
    fn(d.pat_off);
    fn(d.stt);
    fn(d.dfin);
    fn(d.ind);
    fn(d.side_keys);
    fn(d.side_vals);
}

template <class T>
uint64_t as_offset(T *p, const uint8_t *base) {
    return p ? (uint64_t)((const uint8_t *)p - base) : NO_SECTION;
}

// FNV-1a (Fowler, Noll, Vo) with its 64-bit offset basis and prime, applied
// to little-endian 64-bit words instead of bytes; a tail shorter than a word
// is zero-padded.
struct Fnv64 {
    uint64_t h = 0xcbf29ce484222325ull;
    void add(const void *p, uint64_t n) {
        const uint8_t *b = (const uint8_t *)p;
        uint64_t i = 0;
        for (; i + 8 <= n; i += 8) {
            uint64_t w;
            memcpy(&w, b + i, 8);
            h = (h ^ w) * 0x100000001b3ull;
        }
        if (i < n) {
            uint64_t w = 0;
            memcpy(&w, b + i, n - i);
            h = (h ^ w) * 0x100000001b3ull;
        }
    }
};

uint64_t checksum(const FileMeta &m, const uint8_t *blob, uint64_t n) {
    Fnv64 f;
    f.add(&m, sizeof m);
    f.add(blob, n);
    return f.h;
}

int io_error(const char *who, const char *what, const std::string &path) {
    return set_error(PFAC_EIO, "%s: %s %s", who, what, path.c_str());
}

// Section extents and field ranges of a loaded description (offsets not yet
// rebased) against its blob.  Returns PFAC_OK or PFAC_EFORMAT with the field
// named.
int check_meta(FileMeta &m, const uint8_t *blob, uint64_t blob_bytes) {
    DevTable &d = m.dev;
    const char *who = "pfac_table_load";
    auto bad = [&](const char *what) { return set_error(PFAC_EFORMAT, "%s: %s", who, what); };
    if (d.sigma < 1 || d.sigma > 256) return bad("alphabet size out of range");
    if (!(d.W == 0 || d.W == 1 || d.W == 2 || d.W == 3 || d.W == 8)) return bad("record format");
    if (d.bps < 1 || d.bps > 8) return bad("bits per symbol");
    if (m.kmin < 1 || m.kmin > m.kmax || m.kmax > (uint32_t)KMAX || m.kmax * d.bps > 32)
        return bad("prefix depths");
    if (d.kmin != m.kmin || d.kdef < m.kmin || d.kdef > m.kmax) return bad("default prefix depth");
    if (d.dag > 1 || d.g_bits > 32) return bad("flags");
    if (d.layout > PFAC_LAYOUT_DENSE || d.layout != m.info.layout || (d.layout == PFAC_LAYOUT_DENSE) != (d.W == 3))
        return bad("layout");
    if (d.W == 0 && d.pk_shift != pk_shift(d.sigma)) return bad("packed record shift");

    // every section: inside the blob, aligned for its elements, and long
    // enough for the elements the description counts
    int rc = PFAC_OK;
    auto span = [&](auto &p, uint64_t elems, bool required) {
        using E = std::remove_cv_t<std::remove_pointer_t<std::remove_reference_t<decltype(p)>>>;
        const uint64_t off = (uint64_t)(uintptr_t)p;
        if (off == NO_SECTION) {
            if (required && rc == PFAC_OK) rc = bad("a required section is missing");
            return;
        }
        if (rc != PFAC_OK) return;
        if (off > blob_bytes || off % alignof(E) != 0) rc = bad("section offset");
        else if (elems > (blob_bytes - off) / sizeof(E)) rc = bad("section extends past the blob");
    };
    const bool dense = d.W == 3;
    const uint64_t nr = d.n_rec;
    span(d.rec, dense ? (uint64_t)d.n_nodes * d.sigma : nr * rec_words((int)d.W), true);
    span(d.fin, d.W == 1 ? nr : 0, true);
    span(d.fbc, d.W == 0 ? 2 * (nr / 32 + 1) : 0, d.W == 0);
    span(d.fvals, d.n_fvals, d.W == 0);
    span(d.leaf_fin, d.leaf_words, true);
    span(d.pool, d.pool_words, true);
    for (uint32_t k = 0; k <= (uint32_t)KMAX; k++) {
        const bool held = k >= m.kmin && k <= m.kmax;
        if (!held) {
            if ((uint64_t)(uintptr_t)d.F[k] != NO_SECTION || (uint64_t)(uintptr_t)d.C[k] != NO_SECTION ||
                (uint64_t)(uintptr_t)d.E[k] != NO_SECTION || (uint64_t)(uintptr_t)d.M[k] != NO_SECTION ||
                (uint64_t)(uintptr_t)d.B[k] != NO_SECTION)
                return bad("prefix node outside the depths held");
            continue;
        }
        if (d.c_shift[k] != 0 && d.c_shift[k] != 3) return bad("count stride");
        const uint64_t ent = 1ull << (k * d.bps);
        const uint64_t fw = ent >= 32 ? ent / 32 : 1;
        span(d.F[k], fw, true);
        span(d.C[k], (fw + (1ull << d.c_shift[k]) - 1) >> d.c_shift[k], true);
        span(d.E[k], d.n_e[k], true);
        span(d.M[k], d.m_words[k], false);
        span(d.B[k], ent < 4 ? 4 : ent, false);
    }
    span(d.G, (1ull << d.g_bits) / 32, false);
    span(d.pat_off, (uint64_t)d.n_pat + 1, false);
    span(d.pat, 0, false);
    span(d.stt, dense ? (uint64_t)d.n_nodes * d.sigma : 0, dense);
    span(d.dfin, dense ? (uint64_t)d.n_nodes : 0, dense);
    span(d.ind, d.ind_words, true);
    span(d.side_keys, d.dag ? (uint64_t)d.side_slots : 0, d.dag != 0);
    span(d.side_vals, d.dag ? (uint64_t)d.side_slots : 0, d.dag != 0);
    if (rc != PFAC_OK) return rc;
    // truncated tables: pattern j is pat[pat_off[j] .. pat_off[j + 1])
    const uint64_t o_po = (uint64_t)(uintptr_t)d.pat_off, o_pb = (uint64_t)(uintptr_t)d.pat;
    if (o_po != NO_SECTION) {
        if (o_pb == NO_SECTION) return bad("pattern offsets without pattern bytes");
        uint32_t prev = 0;
        for (uint64_t j = 0; j <= d.n_pat; j++) {
            uint32_t v;
            memcpy(&v, blob + o_po + 4 * j, 4);
            if (v < prev) return bad("pattern offsets not ascending");
            prev = v;
        }
        if (prev > blob_bytes - o_pb) return bad("pattern bytes extend past the blob");
    }
    return PFAC_OK;
}

}  // namespace

extern "C" int pfac_table_save(const pfac_table *t, const char *path) {
    if (!t || !path) return set_error(PFAC_EINVAL, "pfac_table_save: NULL argument");
    clear_error();
    try {
        // the blob as the kernels see it
        std::vector<uint8_t> devcopy;
        const uint8_t *blob = nullptr;
        const uint8_t *base = nullptr;
        if (t->d_blob) {
            devcopy.resize(t->blob_bytes);
            int cur = 0;
            cudaGetDevice(&cur);
            if (cur != t->device) cudaSetDevice(t->device);
            cudaError_t ce = cudaMemcpy(devcopy.data(), t->d_blob, t->blob_bytes, cudaMemcpyDeviceToHost);
            if (cur != t->device) cudaSetDevice(cur);
            if (ce != cudaSuccess)
                return set_error(PFAC_ECUDA, "pfac_table_save: read-back: %s", cudaGetErrorString(ce));
            blob = devcopy.data();
            base = (const uint8_t *)t->d_blob;
        } else {
            if (t->h_blob.size() != t->blob_bytes)
                return set_error(PFAC_EINVAL, "pfac_table_save: table holds no blob");
            blob = t->h_blob.data();
            base = blob;
        }

        FileMeta m;
        memset(&m, 0, sizeof m);
        memcpy(&m.dev, &t->dev, sizeof m.dev);
        for_each_section(m.dev, [&](auto &p) {
            using P = std::remove_reference_t<decltype(p)>;
            p = (P)(uintptr_t)as_offset(p, base);
        });
        m.info = t->info;
        m.kmin = t->kmin;
        m.kmax = t->kmax;
        const uint32_t tuned[10] = {t->tuned_variant, t->tuned_k,     t->tuned_copies, t->tuned_masks,
                                    t->tuned_gram,    t->tuned_bytes, t->tuned_nw,     t->tuned_kernel,
                                    t->tuned_records, t->tuned_resolver};
        memcpy(m.tuned, tuned, sizeof tuned);
        m.match_density = t->match_density;

        FileHeader h;
        memset(&h, 0, sizeof h);
        memcpy(h.magic, MAGIC, sizeof MAGIC);
        h.version = FORMAT_VERSION;
        h.endian = ENDIAN_MARK;
        h.devtable_bytes = sizeof(DevTable);
        h.info_bytes = sizeof(pfac_table_info_t);
        h.meta_bytes = sizeof(FileMeta);
        h.blob_bytes = t->blob_bytes;
        h.checksum = checksum(m, blob, t->blob_bytes);

        const std::string dst(path);
        const std::string tmp = dst + ".tmp." + std::to_string((long)getpid());
        FILE *f = fopen(tmp.c_str(), "wb");
        if (!f) return io_error("pfac_table_save", "cannot create", tmp);
        bool ok = fwrite(&h, sizeof h, 1, f) == 1 && fwrite(&m, sizeof m, 1, f) == 1 &&
                  (t->blob_bytes == 0 || fwrite(blob, t->blob_bytes, 1, f) == 1);
        ok = (fflush(f) == 0) && ok;
        ok = (fclose(f) == 0) && ok;
        if (!ok) {
            unlink(tmp.c_str());
            return io_error("pfac_table_save", "write failed:", tmp);
        }
        if (rename(tmp.c_str(), dst.c_str()) != 0) {
            unlink(tmp.c_str());
            return io_error("pfac_table_save", "cannot rename onto", dst);
        }
        return PFAC_OK;
    } catch (const std::bad_alloc &) {
        return set_error(PFAC_ENOMEM, "pfac_table_save: host allocation failed");
    }
}

extern "C" int pfac_table_load(const char *path, uint32_t flags, void *cuda_stream, pfac_table **out) {
    if (!path || !out) return set_error(PFAC_EINVAL, "pfac_table_load: NULL argument");
    *out = nullptr;
    if (flags & ~PFAC_BUILD_HOST_ONLY)
        return set_error(PFAC_EINVAL, "pfac_table_load: only PFAC_BUILD_HOST_ONLY is accepted");
    clear_error();
    const std::string src(path);
    try {
        FILE *f = fopen(path, "rb");
        if (!f) return io_error("pfac_table_load", "cannot open", src);
        FileHeader h;
        FileMeta m;
        std::vector<uint8_t> blob;
        int rc = PFAC_OK;
        long long fsize = -1;
        if (fseek(f, 0, SEEK_END) == 0) fsize = ftell(f);
        if (fsize < 0 || fseek(f, 0, SEEK_SET) != 0) {
            rc = io_error("pfac_table_load", "cannot seek", src);
        } else if (fread(&h, sizeof h, 1, f) != 1) {
            rc = set_error(PFAC_EFORMAT, "pfac_table_load: %s is shorter than a header", path);
        } else if (memcmp(h.magic, MAGIC, sizeof MAGIC) != 0 || h.endian != ENDIAN_MARK) {
            rc = set_error(PFAC_EFORMAT, "pfac_table_load: %s is not a table file", path);
        } else if (h.version != FORMAT_VERSION || h.devtable_bytes != sizeof(DevTable) ||
                   h.info_bytes != sizeof(pfac_table_info_t) || h.meta_bytes != sizeof(FileMeta)) {
            rc = set_error(PFAC_EFORMAT,
                           "pfac_table_load: %s was written by another format version (%u; this "
                           "library reads %u)", path, h.version, FORMAT_VERSION);
        } else if ((uint64_t)fsize != sizeof h + sizeof m + h.blob_bytes) {
            rc = set_error(PFAC_EFORMAT, "pfac_table_load: %s has %lld bytes, its header says %llu",
                           path, fsize, (unsigned long long)(sizeof h + sizeof m + h.blob_bytes));
        } else if (fread(&m, sizeof m, 1, f) != 1) {
            rc = io_error("pfac_table_load", "cannot read", src);
        } else {
            blob.resize(h.blob_bytes);
            if (h.blob_bytes && fread(blob.data(), h.blob_bytes, 1, f) != 1)
                rc = io_error("pfac_table_load", "cannot read", src);
        }
        fclose(f);
        if (rc != PFAC_OK) return rc;
        if (checksum(m, blob.data(), h.blob_bytes) != h.checksum)
            return set_error(PFAC_EFORMAT, "pfac_table_load: %s: checksum mismatch", path);
        rc = check_meta(m, blob.data(), h.blob_bytes);
        if (rc != PFAC_OK) return rc;

        pfac_table *t = new (std::nothrow) pfac_table();
        if (!t) return set_error(PFAC_ENOMEM, "pfac_table_load: host allocation failed");
        const bool host_only = (flags & PFAC_BUILD_HOST_ONLY) != 0;
        if (!host_only) {
            cudaStream_t st = (cudaStream_t)cuda_stream;
            cudaGetDevice(&t->device);
            cudaError_t ce = cudaMalloc(&t->d_blob, h.blob_bytes);
            if (ce != cudaSuccess) {
                delete t;
                cudaGetLastError();
                return set_error(ce == cudaErrorMemoryAllocation ? PFAC_ENOMEM : PFAC_ECUDA,
                                 "pfac_table_load: cudaMalloc(%llu): %s",
                                 (unsigned long long)h.blob_bytes, cudaGetErrorString(ce));
            }
            ce = cudaMemcpyAsync(t->d_blob, blob.data(), h.blob_bytes, cudaMemcpyHostToDevice, st);
            if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
            if (ce != cudaSuccess) {
                cudaFree(t->d_blob);
                delete t;
                return set_error(PFAC_ECUDA, "pfac_table_load: upload: %s", cudaGetErrorString(ce));
            }
        } else {
            t->h_blob = std::move(blob);
        }
        uint8_t *B = host_only ? t->h_blob.data() : (uint8_t *)t->d_blob;
        t->blob_bytes = h.blob_bytes;
        memcpy(&t->dev, &m.dev, sizeof m.dev);
        for_each_section(t->dev, [&](auto &p) {
            using P = std::remove_reference_t<decltype(p)>;
            const uint64_t off = (uint64_t)(uintptr_t)p;
            p = off == NO_SECTION ? nullptr : (P)(B + off);
        });
        t->info = m.info;
        t->kmin = m.kmin;
        t->kmax = m.kmax;
        t->tuned_variant = m.tuned[0];
        t->tuned_k = m.tuned[1];
        t->tuned_copies = m.tuned[2];
        t->tuned_masks = m.tuned[3];
        t->tuned_gram = m.tuned[4];
        t->tuned_bytes = m.tuned[5];
        t->tuned_nw = m.tuned[6];
        t->tuned_kernel = m.tuned[7];
        t->tuned_records = m.tuned[8];
        t->tuned_resolver = m.tuned[9];
        t->match_density = m.match_density;
        *out = t;
        return PFAC_OK;
    } catch (const std::bad_alloc &) {
        return set_error(PFAC_ENOMEM, "pfac_table_load: host allocation failed");
    }
}
