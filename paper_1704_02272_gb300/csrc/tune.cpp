// Autotuner of the scan configuration (pfac_autotune).  For a built table
// and a device-resident sample it times the scan kernel for each candidate
// (the scan kernel: queued or register-staged x prefix depth resolved in
// shared memory x entries in shared memory or not x child masks on or off x
// the first stage (prefix bitmap, gram filter or prefix bytes) x copies of
// that bitmap over the banks x CTA width), keeps the fastest as the
// table's default, and can remember the choice in a small text cache keyed by
// the table's shape and the GPU.
#include <cuda_runtime.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "internal.h"

using namespace pfac;

namespace {

std::string cache_key(const pfac_table *t, uint64_t n_bytes, uint32_t n_segments) {
    cudaDeviceProp prop;
    int dev = 0;
    cudaGetDevice(&dev);
    std::string gpu = "unknown";
    if (cudaGetDeviceProperties(&prop, dev) == cudaSuccess) gpu = prop.name;
    for (char &c : gpu)
        if (c == ' ' || c == ',') c = '_';
    uint32_t lg = 0;
    while ((1ull << (lg + 1)) <= n_bytes) lg++;
    char buf[256];
    // the record format (packed, wide, dense rows ...) and the merge are part
    // of the key: each makes its own plans
    snprintf(buf, sizeof buf, "sigma=%u,n=%u,maxlen=%u,rec=%u%s,segs=%s,bytes=2^%u,gpu=%s",
             t->info.alphabet_size, t->info.n_patterns, t->info.max_len, t->dev.W,
             t->dev.dag ? "m" : "", n_segments > 1 ? "many" : "one", lg, gpu.c_str());
    return buf;
}

// A cache line: key, variant, depth, copies, masks, gram filter, prefix
// bytes, warps per CTA, scan kernel, records per slice, resolver, time.
// Lines without the scan kernel (written before the register-staged kernel
// existed) name the queued one; lines without the records or the resolver
// leave them to the library.
bool cache_lookup(const char *path, const std::string &key, uint32_t *v, uint32_t *k,
                  uint32_t *c, uint32_t *mk, uint32_t *gf, uint32_t *pb, uint32_t *nw,
                  uint32_t *kind, uint32_t *recs, uint32_t *resv, float *ms) {
    FILE *f = fopen(path, "r");
    if (!f) return false;
    char line[512];
    bool found = false;
    while (fgets(line, sizeof line, f)) {
        // whitespace-separated tokens: the key, 7 to 10 fields, the time
        char *tok[13], *save = nullptr;
        int nt = 0;
        for (char *p = strtok_r(line, " \t\r\n", &save); p && nt < 13;
             p = strtok_r(nullptr, " \t\r\n", &save))
            tok[nt++] = p;
        if (nt < 9 || nt > 12 || key != tok[0]) continue;
        uint32_t u[10];
        bool ok = true;
        for (int i = 0; i < nt - 2; i++) {
            char *end = nullptr;
            const unsigned long x = strtoul(tok[1 + i], &end, 10);
            if (!end || *end || x > 0xFFFFFFFFul) ok = false;
            u[i] = (uint32_t)x;
        }
        char *end = nullptr;
        const float e = strtof(tok[nt - 1], &end);
        if (!ok || !end || *end) continue;
        {
            const uint32_t q = nt >= 10 ? u[7] : 1u;
            *recs = nt >= 11 ? u[8] : 0u;
            *resv = nt == 12 ? u[9] : 0u;
            *v = u[0];
            *k = u[1];
            *c = u[2];
            *mk = u[3];
            *gf = u[4];
            *pb = u[5];
            *nw = u[6];
            *kind = q;
            *ms = e;
            found = true;  // the last line for a key wins
        }
    }
    fclose(f);
    return found;
}

}  // namespace

extern "C" int pfac_autotune(pfac_table *t, const uint8_t *d_sample, uint64_t n_bytes,
                             const uint64_t *d_seg_offsets, uint32_t n_segments,
                             const char *cache_path, void *cuda_stream, pfac_tune_result *out) {
    clear_error();
    if (!t) return set_error(PFAC_EINVAL, "pfac_autotune: NULL table");
    pfac_tune_result res;
    memset(&res, 0, sizeof res);
    const std::string key = cache_key(t, n_bytes, n_segments);
    if (cache_path) {
        uint32_t v, k, c, mk, gf, pb, nw, kind, rp, rsv;
        float ms;
        if (cache_lookup(cache_path, key, &v, &k, &c, &mk, &gf, &pb, &nw, &kind, &rp, &rsv, &ms) &&
            rsv <= 2 &&
            k >= t->kmin && k <= t->kmax && (gf != 2 || t->dev.g_len) &&
            (pb != 2 || t->dev.B[k])) {
            t->tuned_bytes = pb;
            t->tuned_nw = nw;
            t->tuned_kernel = kind;
            t->tuned_records = rp;
            t->tuned_resolver = rsv;
            res.records_per_slice = rp;
            res.resolver = rsv;
            res.prefix_bytes = pb;
            res.warps_per_cta = nw;
            res.scan_kernel = kind;
            t->tuned_variant = v;
            t->tuned_k = k;
            t->tuned_copies = c;
            t->tuned_masks = mk;
            t->tuned_gram = gf;
            res.variant = v;
            res.prefix_depth = k;
            res.bitmap_copies = c;
            res.child_masks = mk;
            res.gram_filter = gf;
            res.scan_ms = ms;
            res.from_cache = 1;
            // a cached choice that no longer makes a plan (an edited or
            // foreign cache line) is dropped and the table tuned afresh
            pfac_plan_info pi;
            const bool sane = (kind == 1 || kind == 2) && (nw == 0 || nw == 16 || nw == 24) &&
                              (rp == 0 || rp == 32 || rp == 512) &&
                              v <= 2 && mk <= 2 && gf <= 2 && pb <= 2 && c <= 32 &&
                              (c & (c - 1)) == 0;
            if (sane && pfac_match_plan(t, nullptr, &pi) == PFAC_OK) {
                if (out) *out = res;
                return PFAC_OK;
            }
            clear_error();
            memset(&res, 0, sizeof res);
        }
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    // forget an earlier choice so the default is measured as the library's own
    t->tuned_variant = t->tuned_k = t->tuned_copies = t->tuned_masks = t->tuned_gram = 0;
    t->tuned_bytes = 0;
    t->tuned_nw = 0;
    t->tuned_kernel = 0;
    t->tuned_records = 0;
    t->tuned_resolver = 0;
    if (!t->d_blob) return set_error(PFAC_EINVAL, "pfac_autotune: table was built host-only");
    {
        const int drc = check_table_device(t, cuda_stream, "pfac_autotune");
        if (drc) return drc;
    }

    struct Cand {
        uint32_t var, k, copies, masks, gram, bytes, nw, kernel;
        float ms;
        uint32_t recs = 0;  // records per slice (0: the library's choice)
        uint32_t resolver = 0;  // who resolves the queues (0: the library's choice)
    };
    auto opts_of = [](const Cand &c) {
        pfac_match_opts o;
        memset(&o, 0, sizeof o);
        o.variant = c.var;
        o.prefix_depth = c.k;
        o.bitmap_copies = c.copies;
        o.child_masks = c.masks;
        o.gram_filter = c.gram;
        o.prefix_bytes = c.bytes;
        o.warps_per_cta = c.nw;
        o.scan_kernel = c.kernel;
        o.records_per_slice = c.recs;
        o.resolver = c.resolver;
        return o;
    };
    std::vector<Cand> cands;
    cands.push_back({0, 0, 0, 0, 0, 0, 0, 0, 0.f});  // library default
    const uint32_t gmax = t->dev.g_len ? 2u : 1u;
    for (uint32_t nw : {16u, 24u})
        for (uint32_t k = t->kmin; k <= t->kmax; k++)
            for (uint32_t var = 1; var <= 2; var++)
                for (uint32_t masks = 1; masks <= 2; masks++) {
                    for (uint32_t gram = 1; gram <= gmax; gram++)
                        for (uint32_t copies = 32; copies >= 1; copies >>= 1)
                            cands.push_back({var, k, copies, masks, gram, 1, nw, 1, 0.f});
                    if (t->dev.B[k]) cands.push_back({var, k, 1, masks, 1, 2, nw, 1, 0.f});
                }
    // the register-staged kernel (8-bit and 2-bit symbols)
    if (t->dev.bps == 8 || t->dev.bps == 2)
        for (uint32_t nw : {16u})
            for (uint32_t k = t->kmin; k <= t->kmax; k++)
                for (uint32_t var = 1; var <= 2; var++)
                    for (uint32_t masks = 1; masks <= 2; masks++)
                        for (uint32_t gram = 1; gram <= gmax; gram++)
                            for (uint32_t copies = 16; copies >= 1; copies >>= 1)
                                cands.push_back({var, k, copies, masks, gram, 1, nw, 2, 0.f});

    uint64_t ws_max = 0;
    std::vector<Cand> ok;
    for (const Cand &c : cands) {
        pfac_match_opts o = opts_of(c);
        uint64_t b = 0;
        if (pfac_workspace_bytes(t, n_bytes, n_segments, &o, &b) != PFAC_OK) continue;
        ws_max = std::max(ws_max, b);
        // room for the same plan with a record per position (tried last)
        o.records_per_slice = 512;
        if (pfac_workspace_bytes(t, n_bytes, n_segments, &o, &b) == PFAC_OK)
            ws_max = std::max(ws_max, b);
        ok.push_back(c);
    }
    clear_error();
    void *ws = nullptr, *small = nullptr;
    cudaError_t e = cudaMalloc(&ws, ws_max ? ws_max : 256);
    if (e == cudaSuccess) e = cudaMalloc(&small, 256);
    cudaEvent_t e0 = nullptr, e1 = nullptr, e2 = nullptr, e3 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaEventCreate(&e2);
    if (e == cudaSuccess) e = cudaEventCreate(&e3);
    if (e != cudaSuccess) {
        cudaFree(ws);
        cudaFree(small);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (e2) cudaEventDestroy(e2);
        cudaGetLastError();
        return set_error(PFAC_ENOMEM, "pfac_autotune: %s", cudaGetErrorString(e));
    }
    uint64_t *d_cnt = (uint64_t *)small;
    int32_t *d_st = (int32_t *)((uint8_t *)small + 128);
    // the scan kernel's time for one candidate (both launches: the scan pass
    // and the emit pass), median of three after a warm-up; false when it
    // does not run
    auto time_cand = [&](Cand &c) -> bool {
        pfac_match_opts o = opts_of(c);
        uint64_t b = 0;
        pfac_workspace_bytes(t, n_bytes, n_segments, &o, &b);
        int rc = pfac_match_async(t, d_sample, n_bytes, d_seg_offsets, n_segments, nullptr, 0,
                                  d_cnt, d_st, ws, b, &o, st);
        if (rc != PFAC_OK) {
            clear_error();
            return false;
        }
        o.ev_scan_begin = e0;
        o.ev_scan_end = e1;
        o.ev_emit_begin = e2;
        o.ev_emit_end = e3;
        float t3[3];
        for (int r = 0; r < 3; r++) {
            rc = pfac_match_async(t, d_sample, n_bytes, d_seg_offsets, n_segments, nullptr, 0,
                                  d_cnt, d_st, ws, b, &o, st);
            float ms_scan = 0.f, ms_emit = 0.f;
            if (rc == PFAC_OK && cudaEventSynchronize(e3) == cudaSuccess &&
                cudaEventElapsedTime(&ms_scan, e0, e1) == cudaSuccess &&
                cudaEventElapsedTime(&ms_emit, e2, e3) == cudaSuccess) {
                t3[r] = ms_scan + ms_emit;
            } else {
                clear_error();
                return false;
            }
        }
        std::sort(t3, t3 + 3);
        c.ms = t3[1];
        return true;
    };
    std::vector<Cand> timed;
    for (Cand c : ok)
        if (time_cand(c)) timed.push_back(c);
    // the best plan with the other record space per slice
    if (!timed.empty()) {
        Cand best0 = timed[0];
        for (const Cand &c : timed)
            if (c.var && c.ms < best0.ms) best0 = c;
        pfac_plan_info pi;
        pfac_match_opts o = opts_of(best0);
        if (best0.var && pfac_match_plan(t, &o, &pi) == PFAC_OK) {
            Cand alt = best0;
            alt.recs = pi.records_per_slice == 512 ? 32u : 512u;
            if (time_cand(alt)) timed.push_back(alt);
        }
        clear_error();
        // the best of those with the other resolution of the queues
        Cand best1 = best0;
        for (const Cand &c : timed)
            if (c.var && c.ms < best1.ms) best1 = c;
        o = opts_of(best1);
        if (best1.var && pfac_match_plan(t, &o, &pi) == PFAC_OK && pi.resolver) {
            Cand alt = best1;
            alt.resolver = pi.resolver == 2 ? 1u : 2u;
            if (time_cand(alt)) timed.push_back(alt);
        }
        clear_error();
    }
    int32_t h_st = 0;
    e = cudaMemcpyAsync(&h_st, d_st, 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaEventDestroy(e2);
    cudaEventDestroy(e3);
    cudaFree(ws);
    cudaFree(small);
    if (e != cudaSuccess) return set_error(PFAC_ECUDA, "pfac_autotune: %s", cudaGetErrorString(e));
    if (h_st != PFAC_OK) return set_error(h_st, "pfac_autotune: device reported %d", h_st);
    if (timed.empty()) return set_error(PFAC_EINVAL, "pfac_autotune: no candidate ran");
    const Cand &def = timed[0];
    Cand best = def;
    for (const Cand &c : timed)
        if (c.var && c.ms < best.ms) best = c;
    res.default_ms = def.var == 0 ? def.ms : 0.f;
    res.n_tried = (uint32_t)timed.size();
    if (best.var) {
        t->tuned_variant = best.var;
        t->tuned_k = best.k;
        t->tuned_copies = best.copies;
        t->tuned_masks = best.masks;
        t->tuned_gram = best.gram;
        t->tuned_bytes = best.bytes;
        t->tuned_nw = best.nw;
        t->tuned_kernel = best.kernel;
        t->tuned_records = best.recs;
        t->tuned_resolver = best.resolver;
    }
    res.variant = best.var;
    res.prefix_depth = best.k;
    res.bitmap_copies = best.copies;
    res.child_masks = best.masks;
    res.gram_filter = best.gram;
    res.prefix_bytes = best.bytes;
    res.warps_per_cta = best.nw;
    res.scan_kernel = best.kernel;
    res.records_per_slice = best.recs;
    res.resolver = best.resolver;
    res.scan_ms = best.ms;
    if (cache_path && best.var) {
        FILE *f = fopen(cache_path, "a");
        if (f) {
            fprintf(f, "%s %u %u %u %u %u %u %u %u %u %u %.6f\n", key.c_str(), best.var, best.k,
                    best.copies, best.masks, best.gram, best.bytes, best.nw, best.kernel,
                    best.recs, best.resolver, best.ms);
            fclose(f);
        }
    }
    if (out) *out = res;
    return PFAC_OK;
}
