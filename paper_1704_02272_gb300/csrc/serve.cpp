// Serving loop over a resident table (pfac_server_*): continuous batching of
// packet batches.
//
// Requests (a host text plus its segment offsets) queue in arrival order.  A
// dispatcher thread admits the oldest waiting request as soon as a slot (a
// CUDA stream) is free and the device-memory pool has room for its input,
// offsets, workspace and output; admitted requests run concurrently on their
// own streams, so a request that arrives while others are on the GPU starts
// as soon as a slot and memory free up, and copies of one request overlap the
// matching of another.  Each request completes in two stream-ordered phases:
// H2D of its input, pfac_match_async, D2H of its count; then D2H of its keys
// (in the rare case the first estimate was too small, re-matched into a
// buffer of exactly its count first, asynchronously on its slot with its own
// status check).  The keys land in a block of a pinned result arena, taken
// when the count is known and handed out in place until the request is
// released, so the dispatcher neither allocates nor copies host memory per
// request (fresh host pages cost milliseconds while the process grows); when
// the arena is full they land in the slot's staging buffer and are copied
// into the request's own vector.  Latency is stamped at submit, admission,
// issue, count and completion.
//
// Threads: submitters, pollers and waiters share one lock over the request
// queue and the completed list; the dispatcher owns the slots and the pool
// and takes the lock only to pick up new requests and to publish finished
// ones, so no copy, launch or host copy of keys happens under it.
#include <cuda_runtime.h>
#include <string.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "internal.h"

using namespace pfac;

namespace {

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

// First-fit allocator over one device allocation (offsets, 256-byte units).
struct Pool {
    uint8_t *base = nullptr;
    uint64_t size = 0;
    std::map<uint64_t, uint64_t> free_;  // offset -> length
    void init(uint8_t *b, uint64_t n) {
        base = b;
        size = n;
        free_.clear();
        free_[0] = n;
    }
    bool alloc(uint64_t n, uint64_t *off) {
        n = (n + 255) & ~255ull;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= n) {
                *off = it->first;
                const uint64_t rest = it->second - n, at = it->first + n;
                free_.erase(it);
                if (rest) free_[at] = rest;
                return true;
            }
        }
        return false;
    }
    void release(uint64_t off, uint64_t n) {
        n = (n + 255) & ~255ull;
        auto it = free_.emplace(off, n).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
};

struct Request {
    uint64_t id;
    const uint8_t *h_in;
    uint64_t n;
    const uint64_t *h_seg;
    uint32_t nseg;
    double t_submit = 0, t_admit = 0, t_done = 0, t_issued = 0, t_counted = 0;
    int status = PFAC_OK;
    std::vector<uint64_t> keys;  // keys outside the arena
    bool in_arena = false;       // keys at arena_off of the result arena
    uint64_t arena_off = 0, n_arena = 0;
    bool done = false;
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t ev = nullptr;
    Request *req = nullptr;
    int phase = 0;  // 0 idle, 1 matching, 2 copying keys out, 3 failed, 4 re-matching
    uint64_t off = 0, bytes = 0;
    uint64_t *d_out = nullptr;
    uint64_t cap = 0;
    uint64_t *h_small = nullptr;  // pinned: [count, status]
    uint64_t *h_keys = nullptr;   // pinned staging of the keys
    uint64_t h_cap = 0;
    uint64_t count = 0;
    uint64_t *d_big = nullptr;    // re-match buffer (phase 4)
    bool big_in_pool = false;
    uint64_t big_off = 0;
};

}  // namespace

struct pfac_server {
    const pfac_table *t = nullptr;
    int device = 0;
    uint8_t *d_pool = nullptr;
    Pool pool;
    uint8_t *h_arena = nullptr;  // pinned result arena
    Pool hpool;                  // its blocks (under mu: release runs on callers' threads)
    std::vector<Slot> slots;
    uint64_t max_req = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request *> pending;
    std::unordered_map<uint64_t, Request *> reqs;
    std::deque<uint64_t> completed;
    uint64_t next_id = 1;
    bool stop = false;
    std::thread th;
    int fatal = 0;
};

namespace {

// Bytes of one request's device block: input, offsets, workspace, count and
// status, output keys.
uint64_t request_bytes(const pfac_table *t, uint64_t n, uint32_t nseg, uint64_t cap,
                       uint64_t *ws_out) {
    uint64_t ws = 0;
    if (pfac_workspace_bytes(t, n, nseg, nullptr, &ws) != PFAC_OK) return 0;
    *ws_out = ws;
    auto a = [](uint64_t x) { return (x + 255) & ~255ull; };
    return a(n) + a(8ull * (nseg + 1)) + a(ws) + 256 + a(8 * cap);
}

uint64_t first_capacity(uint64_t n) { return n / 8 > 4096 ? n / 8 : 4096; }

// Issues phase 1 of a request on its slot (the dispatcher's thread; the slots
// and the pool are the dispatcher's, so no lock is held).
bool admit(pfac_server *s, Slot &sl, Request *r) {
    const uint64_t cap = first_capacity(r->n);
    uint64_t ws = 0;
    const uint64_t need = request_bytes(s->t, r->n, r->nseg, cap, &ws);
    uint64_t off = 0;
    if (!need || !s->pool.alloc(need, &off)) return false;
    auto a = [](uint64_t x) { return (x + 255) & ~255ull; };
    uint8_t *p = s->pool.base + off;
    uint8_t *d_in = p;
    uint64_t *d_seg = (uint64_t *)(p + a(r->n));
    uint8_t *d_ws = (uint8_t *)d_seg + a(8ull * (r->nseg + 1));
    uint64_t *d_small = (uint64_t *)(d_ws + a(ws));
    uint64_t *d_out = (uint64_t *)((uint8_t *)d_small + 256);
    sl.req = r;
    sl.off = off;
    sl.bytes = need;
    sl.d_out = d_out;
    sl.cap = cap;
    sl.phase = 1;
    r->t_admit = now_s();
    cudaError_t e = cudaSuccess;
    if (r->n) e = cudaMemcpyAsync(d_in, r->h_in, r->n, cudaMemcpyHostToDevice, sl.stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_seg, r->h_seg, 8ull * (r->nseg + 1), cudaMemcpyHostToDevice,
                            sl.stream);
    int rc = e == cudaSuccess ? PFAC_OK : PFAC_ECUDA;
    if (rc == PFAC_OK)
        rc = pfac_match_async(s->t, d_in, r->n, d_seg, r->nseg, d_out, cap, d_small,
                              (int32_t *)(d_small + 1), d_ws, ws, nullptr, sl.stream);
    if (rc == PFAC_OK)
        e = cudaMemcpyAsync(sl.h_small, d_small, 16, cudaMemcpyDeviceToHost, sl.stream);
    if (rc == PFAC_OK && e == cudaSuccess) e = cudaEventRecord(sl.ev, sl.stream);
    if (rc != PFAC_OK || e != cudaSuccess) {
        r->status = rc != PFAC_OK ? rc : PFAC_ECUDA;
        sl.phase = 3;  // complete with an error once the stream drains
        cudaEventRecord(sl.ev, sl.stream);
    }
    r->t_issued = now_s();
    return true;
}

// Publishes a finished request (its keys already in place) and frees its
// slot and memory.
void finish(pfac_server *s, Slot &sl) {
    Request *r = sl.req;
    s->pool.release(sl.off, sl.bytes);
    if (sl.d_big) {
        if (sl.big_in_pool) s->pool.release(sl.big_off, 8 * sl.count);
        else cudaFreeAsync(sl.d_big, sl.stream);
        sl.d_big = nullptr;
    }
    sl.req = nullptr;
    sl.phase = 0;
    std::lock_guard<std::mutex> lk(s->mu);
    r->t_done = now_s();
    r->done = true;
    s->completed.push_back(r->id);
}

// The device block of a slot's request: input, offsets, workspace, count
// and status words.
struct Block {
    uint8_t *in;
    uint64_t *seg, *small;
    uint8_t *ws;
    uint64_t ws_bytes;
};
Block block_of(pfac_server *s, const Slot &sl, const Request *r) {
    auto a = [](uint64_t x) { return (x + 255) & ~255ull; };
    Block b;
    b.in = s->pool.base + sl.off;
    b.seg = (uint64_t *)(b.in + a(r->n));
    b.ws_bytes = 0;
    pfac_workspace_bytes(s->t, r->n, r->nseg, nullptr, &b.ws_bytes);
    b.ws = (uint8_t *)b.seg + a(8ull * (r->nseg + 1));
    b.small = (uint64_t *)(b.ws + a(b.ws_bytes));
    return b;
}

// Host destination of a request's cnt keys: a block of the result arena when
// it has room (recorded in the request), else nullptr (the slot's staging).
uint64_t *arena_block(pfac_server *s, Request *r, uint64_t cnt) {
    if (!cnt || !s->h_arena) return nullptr;
    std::lock_guard<std::mutex> lk(s->mu);
    uint64_t off = 0;
    if (!s->hpool.alloc(8 * cnt, &off)) return nullptr;
    r->in_arena = true;
    r->arena_off = off;
    r->n_arena = cnt;
    return (uint64_t *)(s->h_arena + off);
}

// Phase 1 done with more keys than the output buffer holds: match again into
// a buffer of exactly cnt keys (from the pool when it has room), copy count,
// status and keys back to dst (the arena block) or to the slot's staging,
// grown first when too small; the slot moves to phase 4.  Returns false on
// failure (status set).
bool rematch(pfac_server *s, Slot &sl, Request *r, uint64_t cnt, uint64_t *dst) {
    if (!dst && cnt > sl.h_cap) {
        cudaStreamSynchronize(sl.stream);
        cudaFreeHost(sl.h_keys);
        sl.h_keys = nullptr;
        if (cudaHostAlloc((void **)&sl.h_keys, 8 * cnt, cudaHostAllocDefault) != cudaSuccess) {
            cudaGetLastError();
            sl.h_cap = 0;
            r->status = PFAC_ENOMEM;
            return false;
        }
        sl.h_cap = cnt;
    }
    const Block b = block_of(s, sl, r);
    sl.count = cnt;
    sl.big_in_pool = s->pool.alloc(8 * cnt, &sl.big_off);
    if (sl.big_in_pool) {
        sl.d_big = (uint64_t *)(s->pool.base + sl.big_off);
    } else if (cudaMallocAsync((void **)&sl.d_big, 8 * cnt, sl.stream) != cudaSuccess) {
        cudaGetLastError();
        sl.d_big = nullptr;
        r->status = PFAC_ENOMEM;
        return false;
    }
    const int rc = pfac_match_async(s->t, b.in, r->n, b.seg, r->nseg, sl.d_big, cnt, b.small,
                                    (int32_t *)(b.small + 1), b.ws, b.ws_bytes, nullptr, sl.stream);
    cudaError_t e = cudaSuccess;
    if (rc == PFAC_OK)
        e = cudaMemcpyAsync(sl.h_small, b.small, 16, cudaMemcpyDeviceToHost, sl.stream);
    if (rc == PFAC_OK && e == cudaSuccess)
        e = cudaMemcpyAsync(dst ? dst : sl.h_keys, sl.d_big, 8 * cnt, cudaMemcpyDeviceToHost,
                            sl.stream);
    if (rc == PFAC_OK && e == cudaSuccess) e = cudaEventRecord(sl.ev, sl.stream);
    if (rc != PFAC_OK || e != cudaSuccess) {
        cudaGetLastError();
        r->status = rc != PFAC_OK ? rc : PFAC_ECUDA;
        cudaStreamSynchronize(sl.stream);
        return false;
    }
    sl.phase = 4;
    return true;
}

void dispatcher(pfac_server *s) {
    cudaSetDevice(s->device);
    std::deque<Request *> local;  // requests picked up, not yet admitted (oldest first)
    for (;;) {
        {
            std::lock_guard<std::mutex> lk(s->mu);
            if (s->stop) break;
            while (!s->pending.empty()) {
                local.push_back(s->pending.front());
                s->pending.pop_front();
            }
        }
        bool progressed = false;
        // admissions, oldest first, while a slot and memory are free
        while (!local.empty()) {
            Slot *free_slot = nullptr;
            for (Slot &sl : s->slots)
                if (sl.phase == 0) {
                    free_slot = &sl;
                    break;
                }
            if (!free_slot) break;
            if (!admit(s, *free_slot, local.front())) break;
            local.pop_front();
            progressed = true;
        }
        // completions
        for (Slot &sl : s->slots) {
            if (sl.phase == 0) continue;
            const cudaError_t q = cudaEventQuery(sl.ev);
            if (q == cudaErrorNotReady) continue;
            progressed = true;
            Request *r = sl.req;
            if (q != cudaSuccess || sl.phase == 3) {
                if (q != cudaSuccess) r->status = PFAC_ECUDA;
                finish(s, sl);
                continue;
            }
            if (sl.phase == 1) {
                r->t_counted = now_s();
                const uint64_t cnt = sl.h_small[0];
                const int32_t st = (int32_t)(uint32_t)sl.h_small[1];
                if (st != PFAC_OK) {
                    r->status = st;
                    finish(s, sl);
                    continue;
                }
                sl.count = cnt;
                uint64_t *dst = arena_block(s, r, cnt);
                if (cnt > sl.cap || (!dst && cnt > sl.h_cap)) {
                    if (!rematch(s, sl, r, cnt, dst)) finish(s, sl);
                    continue;
                }
                cudaError_t e = cudaSuccess;
                if (cnt)
                    e = cudaMemcpyAsync(dst ? dst : sl.h_keys, sl.d_out, 8 * cnt,
                                        cudaMemcpyDeviceToHost, sl.stream);
                if (e == cudaSuccess) e = cudaEventRecord(sl.ev, sl.stream);
                if (e != cudaSuccess) {
                    r->status = PFAC_ECUDA;
                    finish(s, sl);
                    continue;
                }
                sl.phase = 2;
            } else if (sl.phase == 2 || sl.phase == 4) {
                const int32_t st = (int32_t)(uint32_t)sl.h_small[1];
                if (sl.phase == 4 && (st != PFAC_OK || sl.h_small[0] != sl.count))
                    r->status = st != PFAC_OK ? st : PFAC_EDEVICE;
                else if (!r->in_arena)
                    r->keys.assign(sl.h_keys, sl.h_keys + sl.count);
                finish(s, sl);
            }
        }
        if (progressed) {
            s->cv_done.notify_all();
        } else {
            // nothing moved: wait briefly for a submit or a completion
            std::unique_lock<std::mutex> lk(s->mu);
            if (!s->stop && s->pending.empty())
                s->cv_work.wait_for(lk, std::chrono::microseconds(20));
        }
    }
}

}  // namespace

extern "C" int pfac_server_create(const pfac_table *t, const pfac_server_opts *o,
                                  pfac_server **out) {
    clear_error();
    if (!t || !out) return set_error(PFAC_EINVAL, "pfac_server_create: NULL argument");
    if (!t->d_blob) return set_error(PFAC_EINVAL, "pfac_server_create: host-only table");
    {
        const int drc = check_table_device(t, nullptr, "pfac_server_create");
        if (drc) return drc;
    }
    pfac_server_opts opt{};
    if (o) opt = *o;
    const uint32_t n_slots = opt.n_slots ? opt.n_slots : 4;
    const uint64_t pool = opt.device_bytes ? opt.device_bytes : (1ull << 30);
    pfac_server *s = new (std::nothrow) pfac_server();
    if (!s) return set_error(PFAC_ENOMEM, "pfac_server_create: host allocation");
    cudaGetDevice(&s->device);
    s->t = t;
    s->max_req = opt.max_request_bytes ? opt.max_request_bytes : pool / 4;
    cudaError_t e = cudaMalloc((void **)&s->d_pool, pool);
    if (e != cudaSuccess) {
        delete s;
        cudaGetLastError();
        return set_error(PFAC_ENOMEM, "pfac_server_create: pool of %llu bytes: %s",
                         (unsigned long long)pool, cudaGetErrorString(e));
    }
    s->pool.init(s->d_pool, pool);
    const uint64_t hbytes = opt.host_bytes ? opt.host_bytes : (256ull << 20);
    e = cudaHostAlloc((void **)&s->h_arena, hbytes, cudaHostAllocDefault);
    if (e != cudaSuccess) {
        cudaGetLastError();
        cudaFree(s->d_pool);
        delete s;
        return set_error(PFAC_ENOMEM, "pfac_server_create: result arena of %llu bytes: %s",
                         (unsigned long long)hbytes, cudaGetErrorString(e));
    }
    s->hpool.init(s->h_arena, hbytes);
    s->slots.resize(n_slots);
    for (Slot &sl : s->slots) {
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaMallocHost((void **)&sl.h_small, 64);
        sl.h_cap = first_capacity(s->max_req);
        if (e == cudaSuccess) e = cudaMallocHost((void **)&sl.h_keys, 8 * sl.h_cap);
    }
    if (e != cudaSuccess) {
        pfac_server_destroy(s);
        return set_error(PFAC_ECUDA, "pfac_server_create: %s", cudaGetErrorString(e));
    }
    s->th = std::thread(dispatcher, s);
    *out = s;
    return PFAC_OK;
}

extern "C" int pfac_server_submit(pfac_server *s, const uint8_t *h_input, uint64_t n_bytes,
                                  const uint64_t *h_seg_offsets, uint32_t n_segments,
                                  uint64_t *id) {
    clear_error();
    if (!s || !id || !h_seg_offsets || (n_bytes && !h_input))
        return set_error(PFAC_EINVAL, "pfac_server_submit: NULL argument");
    if (n_bytes && n_segments == 0)
        return set_error(PFAC_EINVAL, "pfac_server_submit: a non-empty input needs a segment");
    uint64_t ws = 0;
    const uint64_t need = request_bytes(s->t, n_bytes, n_segments, first_capacity(n_bytes), &ws);
    if (n_bytes > s->max_req || need > s->pool.size)
        return set_error(PFAC_ENOMEM, "pfac_server_submit: request of %llu bytes exceeds the "
                         "server's limits", (unsigned long long)n_bytes);
    Request *r = new (std::nothrow) Request();
    if (!r) return set_error(PFAC_ENOMEM, "pfac_server_submit: host allocation");
    r->h_in = h_input;
    r->n = n_bytes;
    r->h_seg = h_seg_offsets;
    r->nseg = n_segments;
    r->t_submit = now_s();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->fatal) {
            delete r;
            return set_error(PFAC_ECUDA, "pfac_server_submit: server failed");
        }
        r->id = s->next_id++;
        s->reqs[r->id] = r;
        s->pending.push_back(r);
        *id = r->id;
    }
    s->cv_work.notify_one();
    return PFAC_OK;
}

static void fill(const pfac_server *s, const Request *r, pfac_result *res) {
    res->id = r->id;
    res->status = r->status;
    res->in_arena = r->in_arena ? 1 : 0;
    if (r->in_arena) {
        res->n_keys = r->status == PFAC_OK ? r->n_arena : 0;
        res->keys = (const uint64_t *)(s->h_arena + r->arena_off);
    } else {
        res->n_keys = r->keys.size();
        res->keys = r->keys.data();
    }
    res->t_submit = r->t_submit;
    res->t_admit = r->t_admit;
    res->t_done = r->t_done;
    res->t_issued = r->t_issued;
    res->t_counted = r->t_counted;
}

extern "C" int pfac_server_wait(pfac_server *s, uint64_t id, double timeout_s,
                                pfac_result *res) {
    if (!s || !res) return set_error(PFAC_EINVAL, "pfac_server_wait: NULL argument");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return set_error(PFAC_EINVAL, "pfac_server_wait: unknown id");
    Request *r = it->second;
    const auto until = std::chrono::steady_clock::now() +
                       std::chrono::duration_cast<std::chrono::steady_clock::duration>(
                           std::chrono::duration<double>(timeout_s > 0 ? timeout_s : 1e9));
    while (!r->done)
        if (s->cv_done.wait_until(lk, until) == std::cv_status::timeout && !r->done)
            return set_error(PFAC_ETIMEOUT, "pfac_server_wait: request %llu not done",
                             (unsigned long long)id);
    fill(s, r, res);
    return PFAC_OK;
}

extern "C" int pfac_server_poll(pfac_server *s, pfac_result *res) {
    if (!s || !res) return set_error(PFAC_EINVAL, "pfac_server_poll: NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    while (!s->completed.empty()) {
        const uint64_t id = s->completed.front();
        s->completed.pop_front();
        auto it = s->reqs.find(id);
        if (it == s->reqs.end()) continue;  // already released
        fill(s, it->second, res);
        return PFAC_OK;
    }
    return 1;
}

extern "C" int pfac_server_release(pfac_server *s, uint64_t id) {
    if (!s) return set_error(PFAC_EINVAL, "pfac_server_release: NULL server");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end() || !it->second->done)
        return set_error(PFAC_EINVAL, "pfac_server_release: unknown or unfinished request");
    Request *r = it->second;
    if (r->in_arena) s->hpool.release(r->arena_off, 8 * r->n_arena);
    delete r;
    s->reqs.erase(it);
    return PFAC_OK;
}

extern "C" void pfac_server_destroy(pfac_server *s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->th.joinable()) s->th.join();
    for (Slot &sl : s->slots) {
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        if (sl.ev) cudaEventDestroy(sl.ev);
        if (sl.stream) cudaStreamDestroy(sl.stream);
        if (sl.h_small) cudaFreeHost(sl.h_small);
        if (sl.h_keys) cudaFreeHost(sl.h_keys);
    }
    if (s->d_pool) cudaFree(s->d_pool);
    if (s->h_arena) cudaFreeHost(s->h_arena);
    for (auto &kv : s->reqs) delete kv.second;  // pending requests are in reqs too
    delete s;
}
