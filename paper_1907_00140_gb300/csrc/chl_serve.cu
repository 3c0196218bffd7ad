// Serving loop of libchl.so (declared in include/chl.h): resident label sets,
// continuous batching of PPSD queries across label sets, and builds admitted by
// device memory beside them.
//
// Threads. One batcher thread owns the query path: whenever a batch slot is
// free it takes every request that has arrived (submitted ones and, during a
// replay, scheduled ones whose arrival time has passed), in arrival order, up
// to max_batch pairs, packs them into the slot's pinned staging, and issues
// copy-in, one query launch (pairs may belong to different label sets) and
// copy-out on the slot's high-priority stream; it then keeps polling the slots'
// events, scatters finished answers to their requests and records latencies.
// With query_slots > 1 a batch is formed and launched while earlier ones are on
// the GPU. Build workers each take the oldest queued build whose memory
// estimate fits, run chl_build on their own stream with fewer tree slots than
// SMs (so query batches keep SMs), and complete its ticket.
//
// Every wait in this file is on the host (condition variables with timeouts,
// event queries); no kernel here waits on another.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "chl_common.cuh"

namespace {

using Clock = std::chrono::steady_clock;
constexpr uint32_t MAX_SETS = 4096;
constexpr uint64_t ZERO_COPY_MAX = 4096;  // batches this small run on host-mapped staging

struct Req {
    uint64_t id = 0;
    int kind = 0;  // 0 query, 1 build
    uint32_t set = 0;
    const uint32_t *pairs = nullptr;
    uint64_t count = 0;
    uint32_t *out = nullptr;
    Clock::time_point t_arrive, t_done;
    bool done = false;
    chl_status st = CHL_OK;
    std::string err;
    // build
    chl_csr g{};
    const uint32_t *rank = nullptr;
    chl_build_opts bo{};
    chl_labels *result = nullptr;
    uint64_t est = 0;
};

// one request's share of a batch
struct Part {
    uint32_t *out;
    uint64_t count, off;
    Req *req;         // submitted request, or null for a replayed one
    double *lat;      // replayed: where its latency goes
    Clock::time_point arrive;
};

// A batch slot. A batch of up to B pairs (B a bucket size) travels as one
// pinned block [pairs B x 8 bytes][set ids B x 2 bytes] copied in, and one
// block [answers B x 4][bad flag] copied out; unused set ids are 0xFFFF
// (skipped). Per bucket size the memset of the flag, the two copies and the
// query launch are captured once as a CUDA graph, so a batch costs one graph
// launch and one event record.
struct Slot {
    cudaStream_t s = nullptr;
    cudaEvent_t ev = nullptr;
    uint8_t *h_in = nullptr;   // pinned: pairs, then set ids
    uint32_t *h_out = nullptr; // pinned: answers, then the flag
    uint16_t *h_set = nullptr; // host scratch of set ids while a batch forms
    uint8_t *d_in = nullptr;
    uint32_t *d_out = nullptr;
    uint32_t *d_perm = nullptr;     // grouped order of the batch (query_order 1)
    uint32_t *d_scratch = nullptr;  // its key counters
    std::vector<uint64_t> bucket;            // batch sizes with a captured graph
    std::vector<cudaGraphExec_t> graph;      // one per bucket size
    std::vector<Part> parts;
    uint64_t count = 0, cap = 0;             // pairs in the batch, its bucket size
    bool busy = false;
    cudaError_t err = cudaSuccess;           // the batch's launch failed with this
};

struct Replay {
    bool active = false;
    uint64_t n = 0, next = 0;
    std::atomic<uint64_t> finished{0};
    std::atomic<int> failed{0};  // some batch of the replay failed on the device
    Clock::time_point start;
    const double *arrival = nullptr;
    const uint32_t *set_of = nullptr;
    const uint64_t *off = nullptr;
    const uint32_t *pairs = nullptr;
    uint32_t *out = nullptr;
    double *lat = nullptr;
    Clock::time_point last_done;
    Clock::time_point at(uint64_t i) const {
        return start + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(arrival[i]));
    }
};

double secs(Clock::duration d) { return std::chrono::duration<double>(d).count(); }

}  // namespace

struct chl_server {
    chl_server_opts o{};
    int device = 0, sms = 0;
    std::mutex mu;
    std::condition_variable cv_q, cv_b, cv_done;
    bool stop = false;
    std::deque<Req *> qq, bq;
    std::unordered_map<uint64_t, Req *> reqs;
    uint64_t next_id = 1;
    std::vector<chl::QuerySet> sets;
    std::vector<chl::QuerySet *> part_arrays;  // device arrays of partitioned sets
    chl::QuerySet *d_sets = nullptr;
    uint32_t *d_nsets = nullptr;  // set count read by the (captured) query launches
    std::vector<Slot> slots;
    Replay rp;
    std::mutex replay_mu;  // one replay at a time
    uint64_t running_est = 0;
    chl_server_stats st{};
    // fault injection on the host (tests): the batch launched as number
    // fail_batch (1-based; CHL_FAULT_QUERY_BATCH in the environment at
    // creation) is not launched and reports a launch failure instead
    uint64_t fail_batch = 0;
    std::thread batcher;
    std::vector<std::thread> builders;

    void run_batcher();
    void run_builder();
    bool retire(Slot &sl, bool block);
    bool launch(Slot &sl);
};

// scatter a finished slot's answers; returns true if it was busy and is now
// free. A batch whose launch or event reports an error (anything but "not
// ready") is finished as failed: its requests get CHL_ECUDA, its replayed
// answers UINT32_MAX, and the slot is free again.
bool chl_server::retire(Slot &sl, bool block) {
    if (!sl.busy) return false;
    cudaError_t e = sl.err;
    if (e == cudaSuccess) {
        e = block ? cudaEventSynchronize(sl.ev) : cudaEventQuery(sl.ev);
        if (e == cudaErrorNotReady) return false;
    }
    const bool failed = e != cudaSuccess;
    const Clock::time_point now = Clock::now();
    int bad = 0;
    // the flag was copied out with the answers (4 bytes after the bucket)
    if (!failed) std::memcpy(&bad, sl.h_out + sl.cap, sizeof(int));
    std::vector<Req *> finished;
    uint64_t replayed = 0;
    for (const Part &pt : sl.parts) {
        if (failed) std::memset(pt.out, 0xFF, pt.count * 4);
        else std::memcpy(pt.out, sl.h_out + pt.off, pt.count * 4);
        if (pt.req) {
            finished.push_back(pt.req);
        } else {
            *pt.lat = secs(now - pt.arrive);
            ++replayed;
        }
    }
    if (failed && replayed) rp.failed.store(1, std::memory_order_relaxed);
    {
        std::lock_guard<std::mutex> lk(mu);
        if (replayed) rp.last_done = now;
        for (Req *r : finished) {
            r->t_done = now;
            r->done = true;
            if (failed) {
                r->st = CHL_ECUDA;
                r->err = std::string("query batch failed: ") + cudaGetErrorString(e);
            } else if (bad) {
                r->st = CHL_EINVAL;
                r->err = "a query vertex id is out of range";
            }
        }
    }
    // counted after last_done is stored, so a finished replay reads it complete
    if (replayed) rp.finished.fetch_add(replayed, std::memory_order_release);
    if (!finished.empty()) cv_done.notify_all();
    sl.parts.clear();
    sl.count = 0;
    sl.busy = false;
    sl.err = cudaSuccess;
    return true;
}

// fill a free slot with arrived requests in arrival order and start it;
// returns false when nothing had arrived
bool chl_server::launch(Slot &sl) {
    const uint64_t cap = o.max_batch;
    const bool plain = o.batching == 1;
    const Clock::time_point now = Clock::now();
    uint64_t used = 0;
    uint32_t nsets = 0;
    {
        std::lock_guard<std::mutex> lk(mu);
        nsets = uint32_t(sets.size());
        for (;;) {
            if (plain && !sl.parts.empty()) break;
            // the earlier of the next submitted and the next replayed arrival
            Req *r = qq.empty() ? nullptr : qq.front();
            const bool have_rp = rp.active && rp.next < rp.n && rp.at(rp.next) <= now;
            if (!r && !have_rp) break;
            const bool take_rp = have_rp && (!r || rp.at(rp.next) <= r->t_arrive);
            if (take_rp) {
                const uint64_t i = rp.next;
                const uint64_t c = rp.off[i + 1] - rp.off[i];
                if (used + c > cap && used) break;
                Part pt{rp.out + rp.off[i], c, used, nullptr, rp.lat + i, rp.at(i)};
                std::memcpy(sl.h_in + 8 * used, rp.pairs + 2 * rp.off[i], c * 8);
                std::fill(sl.h_set + used, sl.h_set + used + c, uint16_t(rp.set_of[i]));
                sl.parts.push_back(pt);
                used += c;
                rp.next++;
            } else {
                if (used + r->count > cap && used) break;
                Part pt{r->out, r->count, used, r, nullptr, r->t_arrive};
                std::memcpy(sl.h_in + 8 * used, r->pairs, r->count * 8);
                std::fill(sl.h_set + used, sl.h_set + used + r->count, uint16_t(r->set));
                sl.parts.push_back(pt);
                used += r->count;
                qq.pop_front();
            }
        }
    }
    if (sl.parts.empty()) return false;
    (void)nsets;
    // the smallest captured bucket that holds the batch
    size_t b = 0;
    while (sl.bucket[b] < used) ++b;
    const uint64_t B = sl.bucket[b];
    uint16_t *set_in = reinterpret_cast<uint16_t *>(sl.h_in + 8 * B);
    std::memcpy(set_in, sl.h_set, used * 2);
    std::fill(set_in + used, set_in + B, uint16_t(0xFFFF));
    sl.count = used;
    sl.cap = B;
    if (B <= ZERO_COPY_MAX) sl.h_out[B] = 0;  // the kernel sets it on a bad id
    uint64_t nth = 0;
    {
        std::lock_guard<std::mutex> lk(mu);
        nth = st.batches + 1;
    }
    cudaError_t e = nth == fail_batch ? cudaErrorLaunchFailure : cudaGraphLaunch(sl.graph[b], sl.s);
    if (e == cudaSuccess) e = cudaEventRecord(sl.ev, sl.s);
    if (e != cudaSuccess) (void)cudaGetLastError();  // not left for a later check to find
    sl.err = e;  // retire() finishes a failed batch as failed
    sl.busy = true;
    {
        std::lock_guard<std::mutex> lk(mu);
        st.batches++;
        st.pairs += used;
        if (used > st.max_batch_seen) st.max_batch_seen = used;
    }
    return true;
}

void chl_server::run_batcher() {
    cudaSetDevice(device);
    size_t rr = 0;
    for (;;) {
        bool progress = false;
        for (Slot &sl : slots) progress |= retire(sl, false);
        // a free slot gets the next batch; plain mode also waits for it
        Slot *free_sl = nullptr;
        for (size_t k = 0; k < slots.size() && !free_sl; ++k) {
            Slot &sl = slots[(rr + k) % slots.size()];
            if (!sl.busy) free_sl = &sl;
        }
        if (free_sl && launch(*free_sl)) {
            rr++;
            if (o.batching == 1) retire(*free_sl, true);
            continue;
        }
        if (progress) continue;
        bool busy = false;
        for (Slot &sl : slots) busy |= sl.busy;
        std::unique_lock<std::mutex> lk(mu);
        const bool pending = !qq.empty() || (rp.active && rp.next < rp.n);
        if (stop && !busy && qq.empty() && !(rp.active && rp.next < rp.n)) break;
        if (busy || pending) {
            // results or arrivals are due soon: poll
            lk.unlock();
            std::this_thread::yield();
        } else {
            cv_q.wait_for(lk, std::chrono::milliseconds(1));
        }
    }
}

void chl_server::run_builder() {
    cudaSetDevice(device);
    cudaStream_t s = nullptr;
    cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    for (;;) {
        Req *r = nullptr;
        {
            // free memory is read outside the lock: cudaMemGetInfo must not
            // hold up the batcher
            size_t fr = 0, tot = 0;
            cudaMemGetInfo(&fr, &tot);
            std::unique_lock<std::mutex> lk(mu);
            for (;;) {
                if (!bq.empty()) {
                    Req *h = bq.front();
                    const bool fits_budget = running_est + h->est <= o.build_budget || running_est == 0;
                    const bool fits_free = h->est + (uint64_t(1) << 30) <= fr || running_est == 0;
                    if (fits_budget && fits_free) {
                        r = h;
                        bq.pop_front();
                        running_est += r->est;
                        if (running_est > st.build_bytes_peak) st.build_bytes_peak = running_est;
                        break;
                    }
                } else if (stop) {
                    break;
                }
                cv_b.wait_for(lk, std::chrono::milliseconds(1));
                lk.unlock();
                cudaMemGetInfo(&fr, &tot);
                lk.lock();
            }
        }
        if (!r) break;
        chl_labels *L = nullptr;
        const chl_status bs = chl_build(&r->g, r->rank, &r->bo, s, &L);
        {
            std::lock_guard<std::mutex> lk(mu);
            running_est -= r->est;
            r->st = bs;
            if (bs != CHL_OK) r->err = chl_last_error();
            r->result = L;
            r->t_done = Clock::now();
            r->done = true;
            if (bs == CHL_OK) st.builds_done++; else st.builds_failed++;
        }
        cv_done.notify_all();
        cv_b.notify_all();
    }
    cudaStreamDestroy(s);
}

using namespace chl;

extern "C" chl_status chl_server_create(const chl_server_opts *opts, chl_server **out) {
    if (!out) return set_error(CHL_EINVAL, "out is NULL");
    *out = nullptr;
    chl_server_opts o{};
    if (opts) o = *opts;
    if (o.query_slots < 0 || o.query_slots > 16 || o.build_workers < 0 || o.build_workers > 16 ||
        o.batching < 0 || o.batching > 1 || o.build_slots < 0 || o.query_order < 0 || o.query_order > 1)
        return set_error(CHL_EINVAL, "bad server options");
    if (!o.query_slots) o.query_slots = 3;
    if (o.batching == 1) o.query_slots = 1;
    if (!o.max_batch) o.max_batch = uint64_t(1) << 20;
    if (o.max_batch > (uint64_t(1) << 26)) return set_error(CHL_EINVAL, "max_batch above 2^26");
    if (!o.build_workers) o.build_workers = 2;
    chl_server *S = new (std::nothrow) chl_server;
    if (!S) return set_error(CHL_ENOMEM, "host allocation failed");
    if (const char *f = std::getenv("CHL_FAULT_QUERY_BATCH")) S->fail_batch = std::strtoull(f, nullptr, 10);
    cudaError_t e = cudaGetDevice(&S->device);
    if (!e) e = cudaDeviceGetAttribute(&S->sms, cudaDevAttrMultiProcessorCount, S->device);
    if (!o.build_slots) o.build_slots = S->sms > 32 ? S->sms - 16 : S->sms;
    if (!o.build_budget && !e) {
        size_t fr = 0, tot = 0;
        e = cudaMemGetInfo(&fr, &tot);
        o.build_budget = fr > (uint64_t(4) << 30) ? fr - (uint64_t(4) << 30) : fr / 2;
    }
    S->o = o;
    if (!e) e = cudaMalloc(&S->d_sets, MAX_SETS * sizeof(QuerySet));
    if (!e) e = cudaMalloc(&S->d_nsets, sizeof(uint32_t));
    if (!e) e = cudaMemset(S->d_nsets, 0, sizeof(uint32_t));
    int lo = 0, hi = 0;
    if (!e) e = cudaDeviceGetStreamPriorityRange(&lo, &hi);
    S->slots.resize(o.query_slots);
    for (Slot &sl : S->slots) {
        if (e) break;
        const uint64_t mb = o.max_batch;
        e = cudaStreamCreateWithPriority(&sl.s, cudaStreamNonBlocking, hi);
        if (!e) e = cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming);
        if (!e) e = cudaMallocHost(&sl.h_in, mb * 10 + 16);
        if (!e) e = cudaMallocHost(&sl.h_out, mb * 4 + 16);
        if (!e) sl.h_set = static_cast<uint16_t *>(std::malloc(mb * 2));
        if (!e && !sl.h_set) e = cudaErrorMemoryAllocation;
        if (!e) e = cudaMalloc(&sl.d_in, mb * 10 + 16);
        if (!e) e = cudaMalloc(&sl.d_out, mb * 4 + 16);
        if (!e && o.query_order == 1) e = cudaMalloc(&sl.d_perm, mb * 4);
        if (!e && o.query_order == 1) e = cudaMalloc(&sl.d_scratch, GROUP_SCRATCH_WORDS * 4);
        // bucket sizes 32, 64, ... up to max_batch, each captured as a graph
        for (uint64_t B = 32; !e; B *= 2) {
            if (B > mb) B = mb;
            cudaGraph_t gph = nullptr;
            cudaGraphExec_t ex = nullptr;
            e = cudaStreamBeginCapture(sl.s, cudaStreamCaptureModeThreadLocal);
            if (!e && B <= ZERO_COPY_MAX) {
                // small batches: the kernel reads the pinned staging and writes
                // the answers straight to host memory (no copies to wait for)
                uint32_t *flag = sl.h_out + B;
                launch_query_sets(S->d_sets, S->d_nsets, reinterpret_cast<const uint32_t *>(sl.h_in),
                                  reinterpret_cast<const uint16_t *>(sl.h_in + 8 * B), nullptr, B,
                                  sl.h_out, reinterpret_cast<int *>(flag), S->sms * 64, sl.s);
                e = cudaStreamEndCapture(sl.s, &gph);
            } else if (!e) {
                uint32_t *flag = sl.d_out + B;
                cudaMemsetAsync(flag, 0, sizeof(int), sl.s);
                cudaMemcpyAsync(sl.d_in, sl.h_in, B * 10, cudaMemcpyHostToDevice, sl.s);
                const uint32_t *pairs_d = reinterpret_cast<const uint32_t *>(sl.d_in);
                const uint16_t *set_d = reinterpret_cast<const uint16_t *>(sl.d_in + 8 * B);
                // grouped order: the batch sorted by the vertex blocks its pairs read
                if (o.query_order == 1)
                    launch_group_order(S->d_sets, S->d_nsets, pairs_d, set_d, B, sl.d_scratch, sl.d_perm, sl.s);
                launch_query_sets(S->d_sets, S->d_nsets, pairs_d, set_d,
                                  o.query_order == 1 ? sl.d_perm : nullptr, B, sl.d_out,
                                  reinterpret_cast<int *>(flag), S->sms * 64, sl.s);
                cudaMemcpyAsync(sl.h_out, sl.d_out, B * 4 + 4, cudaMemcpyDeviceToHost, sl.s);
                e = cudaStreamEndCapture(sl.s, &gph);
            }
            if (!e) e = cudaGraphInstantiate(&ex, gph, 0);
            if (gph) cudaGraphDestroy(gph);
            if (!e) {
                sl.bucket.push_back(B);
                sl.graph.push_back(ex);
            }
            if (B == mb) break;
        }
    }
    if (e) {
        chl_server_destroy(S);
        return cuda_status(e, "server setup");
    }
    S->batcher = std::thread([S] { S->run_batcher(); });
    for (int k = 0; k < o.build_workers; ++k) S->builders.emplace_back([S] { S->run_builder(); });
    *out = S;
    return CHL_OK;
}

extern "C" chl_status chl_server_add_set(chl_server *S, const chl_labels *L, uint32_t *set_id) {
    if (!S || !L || !set_id) return set_error(CHL_EINVAL, "server, labels or set_id is NULL");
    if (L->device != S->device)
        return set_error(CHL_EINVAL, "labels live on device %d, the server on device %d", L->device,
                         S->device);
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->sets.size() >= MAX_SETS) return set_error(CHL_EINVAL, "too many label sets");
    QuerySet q{L->n, L->offsets, L->hubpos, L->dist, 0, nullptr};
    const uint32_t k = uint32_t(S->sets.size());
    const uint32_t k1 = k + 1;
    // published before any query on it can be submitted (the id is returned after)
    cudaError_t e = cudaMemcpy(S->d_sets + k, &q, sizeof(q), cudaMemcpyHostToDevice);
    if (!e) e = cudaMemcpy(S->d_nsets, &k1, sizeof(k1), cudaMemcpyHostToDevice);
    if (e) return cuda_status(e, "cudaMemcpy");
    S->sets.push_back(q);
    *set_id = k;
    return CHL_OK;
}

extern "C" chl_status chl_server_add_partitioned_set(chl_server *S, const chl_labels *const *parts,
                                                     uint32_t nparts, uint32_t *set_id) {
    if (!S || !parts || !set_id) return set_error(CHL_EINVAL, "server, parts or set_id is NULL");
    if (nparts < 1 || nparts > CHL_MAX_PARTS)
        return set_error(CHL_EINVAL, "nparts must be in [1, %d]", CHL_MAX_PARTS);
    std::vector<QuerySet> h(nparts);
    for (uint32_t k = 0; k < nparts; ++k) {
        const chl_labels *L = parts[k];
        if (!L) return set_error(CHL_EINVAL, "part %u is NULL", k);
        if (L->device != S->device)
            return set_error(CHL_EINVAL, "part %u lives on device %d, the server on device %d", k,
                             L->device, S->device);
        if (L->n != parts[0]->n) return set_error(CHL_EINVAL, "parts cover different vertex counts");
        h[k] = QuerySet{L->n, L->offsets, L->hubpos, L->dist, 0, nullptr};
    }
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->sets.size() >= MAX_SETS) return set_error(CHL_EINVAL, "too many label sets");
    QuerySet *d_parts = nullptr;
    cudaError_t e = cudaMalloc(&d_parts, nparts * sizeof(QuerySet));
    if (!e) e = cudaMemcpy(d_parts, h.data(), nparts * sizeof(QuerySet), cudaMemcpyHostToDevice);
    const QuerySet q{parts[0]->n, nullptr, nullptr, nullptr, nparts, d_parts};
    const uint32_t k = uint32_t(S->sets.size());
    const uint32_t k1 = k + 1;
    if (!e) e = cudaMemcpy(S->d_sets + k, &q, sizeof(q), cudaMemcpyHostToDevice);
    if (!e) e = cudaMemcpy(S->d_nsets, &k1, sizeof(k1), cudaMemcpyHostToDevice);
    if (e) {
        if (d_parts) cudaFree(d_parts);
        return cuda_status(e, "partitioned set");
    }
    S->part_arrays.push_back(d_parts);
    S->sets.push_back(q);
    *set_id = k;
    return CHL_OK;
}

extern "C" chl_status chl_server_submit_query(chl_server *S, uint32_t set_id, const uint32_t *pairs,
                                              uint64_t count, uint32_t *out, uint64_t *ticket) {
    if (!S || !ticket || (count && (!pairs || !out))) return set_error(CHL_EINVAL, "NULL argument");
    uint32_t n = 0;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (set_id >= S->sets.size()) return set_error(CHL_EINVAL, "unknown label set %u", set_id);
        n = S->sets[set_id].n;
    }
    if (count > S->o.max_batch) return set_error(CHL_EINVAL, "request larger than max_batch");
    for (uint64_t i = 0; i < 2 * count; ++i)
        if (pairs[i] >= n) return set_error(CHL_EINVAL, "a query vertex id is >= n");
    Req *r = new (std::nothrow) Req;
    if (!r) return set_error(CHL_ENOMEM, "host allocation failed");
    r->kind = 0;
    r->set = set_id;
    r->pairs = pairs;
    r->count = count;
    r->out = out;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        r->id = S->next_id++;
        r->t_arrive = Clock::now();
        S->reqs[r->id] = r;
        S->qq.push_back(r);
        *ticket = r->id;
    }
    S->cv_q.notify_one();
    return CHL_OK;
}

extern "C" chl_status chl_server_submit_build(chl_server *S, const chl_csr *g, const uint32_t *rank,
                                              const chl_build_opts *opts, uint64_t *ticket) {
    if (!S || !g || !rank || !ticket) return set_error(CHL_EINVAL, "NULL argument");
    Req *r = new (std::nothrow) Req;
    if (!r) return set_error(CHL_ENOMEM, "host allocation failed");
    r->kind = 1;
    r->g = *g;
    r->rank = rank;
    if (opts) r->bo = *opts;
    // one 1024-thread tree slot per SM; the build workers share build_slots
    // SMs so that running builds never hold every SM and query batches keep
    // the rest (tree CTAs are persistent: an SM they hold stays theirs)
    if (!r->bo.threads_per_tree && !r->bo.slots) r->bo.threads_per_tree = 1024;
    if (!r->bo.slots) {
        r->bo.slots = S->o.build_slots / S->o.build_workers;
        if (r->bo.slots < 1) r->bo.slots = 1;
    }
    // estimate: inputs and rank-ordered copy, slot state at 32 window buckets,
    // 256 labels per vertex in the build buffer and in the final CSR
    const double n = g->n, m = double(g->num_arcs);
    const double slots = r->bo.slots;
    r->est = uint64_t(2 * (8 * (n + 1) + 8 * m + 4 * n) + slots * n * 152.0 + n * 256 * 24.0);
    {
        std::lock_guard<std::mutex> lk(S->mu);
        r->id = S->next_id++;
        r->t_arrive = Clock::now();
        S->reqs[r->id] = r;
        S->bq.push_back(r);
        *ticket = r->id;
    }
    S->cv_b.notify_all();
    return CHL_OK;
}

extern "C" chl_status chl_server_wait(chl_server *S, uint64_t ticket, double timeout_s,
                                      chl_labels **built, double *latency_s) {
    if (built) *built = nullptr;
    if (!S) return set_error(CHL_EINVAL, "server is NULL");
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return set_error(CHL_EINVAL, "unknown ticket");
    Req *r = it->second;
    const auto pred = [r] { return r->done; };
    if (timeout_s < 0) {
        S->cv_done.wait(lk, pred);
    } else if (!S->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), pred)) {
        return set_error(CHL_ETIMEOUT, "ticket not finished");
    }
    S->reqs.erase(it);
    lk.unlock();
    const chl_status st = r->st;
    if (latency_s) *latency_s = secs(r->t_done - r->t_arrive);
    if (r->result) {
        if (built) *built = r->result; else chl_labels_free(r->result);
    }
    if (st != CHL_OK) set_error(st, "%s", r->err.c_str());
    delete r;
    return st;
}

extern "C" chl_status chl_server_replay(chl_server *S, uint64_t nreq, const double *arrival_s,
                                        const uint32_t *set_of, const uint64_t *pair_off,
                                        const uint32_t *pairs, uint32_t *out, double *latency_s,
                                        double *wall_s) {
    if (!S || (nreq && (!arrival_s || !set_of || !pair_off || !pairs || !out || !latency_s)))
        return set_error(CHL_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> one(S->replay_mu);
    {
        std::lock_guard<std::mutex> lk(S->mu);
        for (uint64_t i = 0; i < nreq; ++i) {
            if (set_of[i] >= S->sets.size()) return set_error(CHL_EINVAL, "unknown label set");
            if (pair_off[i + 1] < pair_off[i] || pair_off[i + 1] - pair_off[i] > S->o.max_batch)
                return set_error(CHL_EINVAL, "request %llu: bad size", (unsigned long long)i);
            if (i && arrival_s[i] < arrival_s[i - 1]) return set_error(CHL_EINVAL, "arrivals not sorted");
            const uint32_t n = S->sets[set_of[i]].n;
            for (uint64_t j = 2 * pair_off[i]; j < 2 * pair_off[i + 1]; ++j)
                if (pairs[j] >= n) return set_error(CHL_EINVAL, "a query vertex id is >= n");
        }
        S->rp.n = nreq;
        S->rp.next = 0;
        S->rp.finished.store(0);
        S->rp.arrival = arrival_s;
        S->rp.set_of = set_of;
        S->rp.off = pair_off;
        S->rp.pairs = pairs;
        S->rp.out = out;
        S->rp.lat = latency_s;
        S->rp.start = Clock::now();
        S->rp.last_done = S->rp.start;
        S->rp.failed.store(0);
        S->rp.active = true;
    }
    S->cv_q.notify_one();
    while (S->rp.finished.load(std::memory_order_acquire) < nreq) std::this_thread::yield();
    std::lock_guard<std::mutex> lk(S->mu);
    S->rp.active = false;
    if (wall_s) *wall_s = secs(S->rp.last_done - S->rp.start);
    if (S->rp.failed.load()) return set_error(CHL_ECUDA, "a query batch of the replay failed on the device");
    return CHL_OK;
}

extern "C" chl_status chl_server_stats_get(const chl_server *S, chl_server_stats *stats) {
    if (!S || !stats) return set_error(CHL_EINVAL, "NULL argument");
    chl_server *M = const_cast<chl_server *>(S);
    std::lock_guard<std::mutex> lk(M->mu);
    *stats = S->st;
    return CHL_OK;
}

extern "C" void chl_server_destroy(chl_server *S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_q.notify_all();
    S->cv_b.notify_all();
    if (S->batcher.joinable()) S->batcher.join();
    for (std::thread &t : S->builders)
        if (t.joinable()) t.join();
    for (auto &kv : S->reqs) {
        if (kv.second->result) chl_labels_free(kv.second->result);
        delete kv.second;
    }
    for (Slot &sl : S->slots) {
        if (sl.s) cudaStreamSynchronize(sl.s);
        for (cudaGraphExec_t ex : sl.graph) cudaGraphExecDestroy(ex);
        cudaFreeHost(sl.h_in);
        cudaFreeHost(sl.h_out);
        std::free(sl.h_set);
        cudaFree(sl.d_in);
        cudaFree(sl.d_out);
        cudaFree(sl.d_perm);
        cudaFree(sl.d_scratch);
        if (sl.ev) cudaEventDestroy(sl.ev);
        if (sl.s) cudaStreamDestroy(sl.s);
    }
    cudaFree(S->d_sets);
    cudaFree(S->d_nsets);
    for (QuerySet *p : S->part_arrays) cudaFree(p);
    delete S;
}
