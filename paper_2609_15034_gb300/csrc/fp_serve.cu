// Served decode: a request loop with continuous batching.
//
// Clients submit decode requests (a column already on the device plus the
// key of a registered dictionary) from any thread.  A scheduler thread owns
// the GPU side:
//   - admission: a request enters the device only while the bytes in flight
//     (its output and string offsets, held until the client releases them,
//     plus its inputs until its decode completes) stay within the HBM
//     budget; outputs are carved from one device arena allocated up front;
//   - dictionary cache: registered dictionaries are repacked once on the
//     host (pinned); a fixed number of device slots holds the resident ones,
//     replaced least-recently-used among slots no in-flight request uses;
//   - waves: whenever one of the launch lanes (a stream with its own batch
//     buffers) is free, the admitted requests at the head of the queue, up
//     to the wave size, are decoded together by one persistent batched
//     launch; lanes run concurrently, so requests that arrive while others
//     are on the GPU start as soon as a lane and memory free up;
//   - completion: an event per wave; each request gets its own status and
//     decoded size and the host times of submission, admission and
//     completion.
// Requests are admitted in arrival order (no overtaking).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "fp_internal.h"

using namespace fp;

namespace {

int64_t now_ns() {
    return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

uint64_t al256(uint64_t x) { return (x + 255) & ~(uint64_t)255; }

// First-fit allocator over [0, size) with coalescing free blocks.
class Arena {
public:
    void reset(uint64_t size) {
        free_.clear();
        if (size) free_[0] = size;
    }
    bool alloc(uint64_t need, uint64_t* off) {
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= need) {
                *off = it->first;
                const uint64_t rest = it->second - need, at = it->first + need;
                free_.erase(it);
                if (rest) free_[at] = rest;
                return true;
            }
        }
        return false;
    }
    void release(uint64_t off, uint64_t size) {
        auto it = free_.emplace(off, size).first;
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

private:
    std::map<uint64_t, uint64_t> free_;
};

struct HostDict {
    fp_codec codec;
    uint32_t n_entries = 0;
    uint8_t* h_table = nullptr;   // pinned, repacked
    uint8_t* h_lens = nullptr;    // pinned
    size_t table_bytes = 0, lens_bytes = 0;
    int slot = -1;                // device slot while resident
};

struct Slot {
    uint64_t key = 0;
    bool used = false;
    uint32_t refs = 0;            // admitted requests not yet completed
    uint64_t lru = 0;
    cudaEvent_t ready = nullptr;  // recorded after the upload into the slot
    fp_dict view{};
};

struct Req {
    uint64_t ticket = 0;
    fp_request r{};
    int64_t t_submit = 0, t_admit = 0, t_done = 0;
    uint64_t out_off = 0, block = 0;   // arena block: output bytes then string offsets
    uint64_t in_bytes = 0;
    uint32_t status = 0;
    uint64_t total = 0;
    bool done = false;
    int slot = -1;
};

struct Lane {
    cudaStream_t s = nullptr;
    cudaEvent_t ev = nullptr;
    WaveBuffers W;
    std::vector<Req*> reqs;
    bool busy = false;
};

}  // namespace

struct fp_server {
    fp_serve_config cfg{};
    int device = 0;
    int config = 0;
    char* d_arena = nullptr;
    Arena arena;
    char* d_dicts = nullptr;
    size_t slot_bytes = 0;
    std::vector<Slot> slots;
    uint64_t lru_clock = 0;
    std::unordered_map<uint64_t, HostDict> dicts;
    std::vector<Lane> lanes;

    std::mutex mu;
    std::condition_variable cv_sched, cv_done;
    std::deque<Req*> inbox;                      // submitted, not yet taken by the scheduler
    std::deque<Req*> pending;                    // scheduler's FIFO
    std::unordered_map<uint64_t, Req*> live;     // every request not yet released
    std::deque<Req*> finished;                   // completed, not yet polled
    uint64_t next_ticket = 0;
    uint64_t inflight_bytes = 0;                 // under mu
    uint32_t inflight_reqs = 0;                  // admitted, not completed
    bool stopping = false;
    std::thread th;
    fp_serve_stats_t st{};
    std::string sched_error;
};

namespace {

void lane_complete(fp_server* S, Lane& L) {
    const int64_t t = now_ns();
    const uint32_t ws_bits = *L.W.h_ws_status;
    std::lock_guard<std::mutex> lk(S->mu);
    for (size_t i = 0; i < L.reqs.size(); ++i) {
        Req* q = L.reqs[i];
        const uint32_t bits = L.W.h_status[i] | (ws_bits & ERRB_TIMEOUT);
        q->status = (uint32_t)status_code(bits);
        q->total = L.W.h_total[i];
        q->t_done = t;
        q->done = true;
        Slot& sl = S->slots[q->slot];
        --sl.refs;
        S->inflight_bytes -= q->in_bytes;
        --S->inflight_reqs;
        S->st.completed++;
        if (q->status != FP_OK) S->st.failed++;
        S->st.bytes_decoded += q->total;
        S->finished.push_back(q);
    }
    L.reqs.clear();
    L.busy = false;
    S->cv_done.notify_all();
}

// Find (or make) the device slot of dictionary `key`; false if every slot
// is in use.  `upload` is set when the slot must be (re)filled.
bool dict_slot(fp_server* S, uint64_t key, int* slot, bool* upload) {
    HostDict& hd = S->dicts.at(key);
    if (hd.slot >= 0) {
        *slot = hd.slot;
        *upload = false;
        S->st.dict_hits++;
        return true;
    }
    int best = -1;
    for (int i = 0; i < (int)S->slots.size(); ++i) {
        const Slot& sl = S->slots[i];
        if (!sl.used) { best = i; break; }
        if (sl.refs == 0 && (best < 0 || sl.lru < S->slots[best].lru)) best = i;
    }
    if (best < 0) return false;
    Slot& sl = S->slots[best];
    if (sl.used) {
        S->dicts.at(sl.key).slot = -1;
        S->st.dict_evictions++;
    }
    sl.used = true;
    sl.key = key;
    sl.view.codec = hd.codec;
    sl.view.n_entries = hd.n_entries;
    hd.slot = best;
    *slot = best;
    *upload = true;
    S->st.dict_misses++;
    return true;
}

// Admit requests from the head of the queue into a wave on lane L.
void lane_launch(fp_server* S, Lane& L) {
    std::vector<fp_chunk> chunks;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        while (!S->pending.empty() && L.reqs.size() < S->cfg.max_wave) {
            Req* q = S->pending.front();
            const uint64_t out_b = al256(q->r.decoded_size), offs_b = al256(((uint64_t)q->r.n_strings + 1) * 4);
            const uint64_t need = out_b + offs_b;
            if (S->inflight_reqs >= S->cfg.max_inflight) break;
            if (S->inflight_bytes + need + q->in_bytes > S->cfg.hbm_budget) break;
            uint64_t off = 0;
            if (!S->arena.alloc(need, &off)) break;
            int slot = -1;
            bool upload = false;
            if (!dict_slot(S, q->r.dict_key, &slot, &upload)) {
                S->arena.release(off, need);
                break;
            }
            Slot& sl = S->slots[slot];
            HostDict& hd = S->dicts.at(q->r.dict_key);
            cudaError_t e;
            if (upload) {
                e = cudaMemcpyAsync(sl.view.d_table, hd.h_table, hd.table_bytes, cudaMemcpyHostToDevice, L.s);
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(sl.view.d_lens, hd.h_lens, hd.lens_bytes, cudaMemcpyHostToDevice, L.s);
                if (e == cudaSuccess) e = cudaEventRecord(sl.ready, L.s);
            } else {
                e = cudaStreamWaitEvent(L.s, sl.ready, 0);
            }
            if (e != cudaSuccess) {
                // the device refused the dictionary's upload: fail this request (a dead context
                // fails every later one the same way instead of leaving them queued)
                S->sched_error = cudaGetErrorString(e);
                S->dicts.at(q->r.dict_key).slot = -1;
                sl.used = false;
                S->arena.release(off, need);
                S->pending.pop_front();
                q->status = (uint32_t)FP_ERR_CUDA;
                q->t_admit = q->t_done = now_ns();
                q->done = true;
                q->block = 0;
                S->st.completed++;
                S->st.failed++;
                S->finished.push_back(q);
                S->cv_done.notify_all();
                continue;
            }
            sl.refs++;
            sl.lru = ++S->lru_clock;
            S->pending.pop_front();
            q->slot = slot;
            q->out_off = off;
            q->block = need;
            q->t_admit = now_ns();
            S->inflight_bytes += need + q->in_bytes;
            S->inflight_reqs++;
            S->st.admitted++;
            if (S->inflight_bytes > S->st.peak_inflight_bytes) S->st.peak_inflight_bytes = S->inflight_bytes;
            fp_chunk c;
            c.codec = hd.codec;
            c.dict = &sl.view;
            c.d_codes = q->r.d_codes;
            c.codes_bytes = q->r.codes_bytes;
            c.d_code_offsets = q->r.d_code_offsets;
            c.n_strings = q->r.n_strings;
            c.d_out_bytes = reinterpret_cast<uint8_t*>(S->d_arena + off);
            c.out_capacity = q->r.decoded_size;
            c.d_out_offsets = reinterpret_cast<uint32_t*>(S->d_arena + off + out_b);
            chunks.push_back(c);
            L.reqs.push_back(q);
        }
    }
    if (L.reqs.empty()) return;
    fp_status stt = wave_launch(L.W, chunks.data(), (uint32_t)chunks.size(), S->config, L.s);
    cudaError_t e = cudaSuccess;
    if (stt == FP_OK) e = cudaEventRecord(L.ev, L.s);
    if (stt != FP_OK || e != cudaSuccess) {
        // the launch failed on the host: fail the wave's requests
        std::lock_guard<std::mutex> lk(S->mu);
        S->sched_error = fp_last_error();
        for (Req* q : L.reqs) {
            q->status = stt != FP_OK ? (uint32_t)stt : (uint32_t)FP_ERR_CUDA;
            q->t_done = now_ns();
            q->done = true;
            S->slots[q->slot].refs--;
            S->inflight_bytes -= q->in_bytes;
            S->inflight_reqs--;
            S->st.completed++;
            S->st.failed++;
            S->finished.push_back(q);
        }
        L.reqs.clear();
        S->cv_done.notify_all();
        return;
    }
    L.busy = true;
    S->st.waves++;
    if (L.reqs.size() > S->st.max_wave_seen) S->st.max_wave_seen = (uint32_t)L.reqs.size();
}

// A wave whose completion event reports an error (not "not ready"): its
// requests fail with FP_ERR_CUDA.
void lane_fail(fp_server* S, Lane& L, cudaError_t e) {
    std::lock_guard<std::mutex> lk(S->mu);
    S->sched_error = cudaGetErrorString(e);
    const int64_t t = now_ns();
    for (Req* q : L.reqs) {
        q->status = (uint32_t)FP_ERR_CUDA;
        q->t_done = t;
        q->done = true;
        S->slots[q->slot].refs--;
        S->inflight_bytes -= q->in_bytes;
        S->inflight_reqs--;
        S->st.completed++;
        S->st.failed++;
        S->finished.push_back(q);
    }
    L.reqs.clear();
    L.busy = false;
    S->cv_done.notify_all();
}

void scheduler(fp_server* S) {
    cudaSetDevice(S->device);
    for (;;) {
        bool stopping = false;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            while (!S->inbox.empty()) {
                S->pending.push_back(S->inbox.front());
                S->inbox.pop_front();
            }
            bool busy = false;
            for (const Lane& L : S->lanes) busy |= L.busy;
            stopping = S->stopping;
            // on shutdown: finish the waves on the GPU, admit nothing new
            if (!busy && (S->pending.empty() || stopping)) {
                if (stopping) break;
                S->cv_sched.wait_for(lk, std::chrono::milliseconds(2));
                continue;
            }
        }
        bool progress = false;
        for (Lane& L : S->lanes) {
            if (!L.busy) continue;
            const cudaError_t e = cudaEventQuery(L.ev);
            if (e == cudaSuccess) {
                lane_complete(S, L);
                progress = true;
            } else if (e != cudaErrorNotReady) {
                lane_fail(S, L, e);
                progress = true;
            }
        }
        if (!stopping) {
            for (Lane& L : S->lanes) {
                if (!L.busy) {
                    lane_launch(S, L);
                    progress |= L.busy;
                }
            }
        }
        if (!progress) std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
}

void server_free(fp_server* S) {
    cudaSetDevice(S->device);
    cudaDeviceSynchronize();
    for (Lane& L : S->lanes) {
        if (L.ev) cudaEventDestroy(L.ev);
        if (L.s) cudaStreamDestroy(L.s);
        wave_free(L.W);
    }
    for (Slot& sl : S->slots)
        if (sl.ready) cudaEventDestroy(sl.ready);
    for (auto& kv : S->dicts) {
        if (kv.second.h_table) cudaFreeHost(kv.second.h_table);
        if (kv.second.h_lens) cudaFreeHost(kv.second.h_lens);
    }
    for (auto& kv : S->live) delete kv.second;
    if (S->d_arena) cudaFree(S->d_arena);
    if (S->d_dicts) cudaFree(S->d_dicts);
    delete S;
}

}  // namespace

extern "C" {

fp_status fp_serve_create(const fp_serve_config* cfg_in, fp_server** out) {
    if (!out) return fail(FP_ERR_ARG, "out is NULL");
    *out = nullptr;
    fp_serve_config cfg{};
    if (cfg_in) cfg = *cfg_in;
    if (cfg.hbm_budget == 0) return fail(FP_ERR_ARG, "hbm_budget must be > 0");
    if (cfg.dict_cache_slots == 0) cfg.dict_cache_slots = 512;
    if (cfg.max_inflight == 0) cfg.max_inflight = 4096;
    if (cfg.n_streams == 0) cfg.n_streams = 4;
    if (cfg.max_wave == 0) cfg.max_wave = 256;
    if (cfg.n_streams > 64 || cfg.max_wave > (1u << 20) || cfg.dict_cache_slots > (1u << 16))
        return fail(FP_ERR_ARG, "serve configuration out of range");
    fp_server* S = new fp_server();
    S->cfg = cfg;
    S->config = cfg.batch_config >= 0 ? cfg.batch_config : batch_config_default();
    if (S->config >= fp_batch_config_count()) {
        delete S;
        return fail(FP_ERR_ARG, "batch configuration %d out of range", cfg.batch_config);
    }
    cudaError_t e = cudaGetDevice(&S->device);
    S->slot_bytes = 65536 * 16 + 65536;   // the largest table (OnPair-16) and its lengths
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&S->d_arena), cfg.hbm_budget);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&S->d_dicts), S->slot_bytes * cfg.dict_cache_slots);
    if (e != cudaSuccess) {
        server_free(S);
        return cuda_fail(e, "server memory");
    }
    S->arena.reset(cfg.hbm_budget);
    S->slots.resize(cfg.dict_cache_slots);
    for (uint32_t i = 0; i < cfg.dict_cache_slots && e == cudaSuccess; ++i) {
        Slot& sl = S->slots[i];
        e = cudaEventCreateWithFlags(&sl.ready, cudaEventDisableTiming);
        sl.view.device = S->device;
        sl.view.d_table = S->d_dicts + i * S->slot_bytes;
        sl.view.d_lens = reinterpret_cast<uint8_t*>(S->d_dicts + i * S->slot_bytes + 65536 * 16);
    }
    S->lanes.resize(cfg.n_streams);
    for (Lane& L : S->lanes) {
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&L.s, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&L.ev, cudaEventDisableTiming);
        if (e == cudaSuccess) {
            fp_status st = wave_init(L.W, cfg.max_wave);
            if (st != FP_OK) {
                const std::string m = fp_last_error();
                server_free(S);
                return fail(st, "%s", m.c_str());
            }
        }
    }
    if (e != cudaSuccess) {
        server_free(S);
        return cuda_fail(e, "server streams");
    }
    S->th = std::thread(scheduler, S);
    *out = S;
    return FP_OK;
}

fp_status fp_serve_dict_put(fp_server* S, uint64_t key, fp_codec codec, const uint8_t* h_bytes,
                            const uint32_t* h_offsets, uint32_t n_entries) {
    if (!S) return fail(FP_ERR_ARG, "server is NULL");
    std::vector<uint8_t> table, lens;
    std::vector<uint32_t> offs;
    fp_status st = repack_dictionary(codec, h_bytes, h_offsets, n_entries, table, lens, offs);
    if (st != FP_OK) return st;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->dicts.count(key)) return fail(FP_ERR_ARG, "dictionary key %llu is already registered",
                                             (unsigned long long)key);
    }
    HostDict hd;
    hd.codec = codec;
    hd.n_entries = n_entries;
    hd.table_bytes = table.size();
    hd.lens_bytes = lens.size();
    cudaError_t e = cudaHostAlloc(reinterpret_cast<void**>(&hd.h_table), hd.table_bytes, 0);
    if (e == cudaSuccess) e = cudaHostAlloc(reinterpret_cast<void**>(&hd.h_lens), hd.lens_bytes, 0);
    if (e != cudaSuccess) {
        if (hd.h_table) cudaFreeHost(hd.h_table);
        return cuda_fail(e, "cudaHostAlloc(dictionary)");
    }
    memcpy(hd.h_table, table.data(), hd.table_bytes);
    memcpy(hd.h_lens, lens.data(), hd.lens_bytes);
    std::lock_guard<std::mutex> lk(S->mu);
    S->dicts.emplace(key, hd);
    S->st.dicts_registered++;
    return FP_OK;
}

fp_status fp_serve_submit(fp_server* S, const fp_request* r, uint64_t* ticket) {
    if (!S || !r || !ticket) return fail(FP_ERR_ARG, "server/request/ticket is NULL");
    const int64_t t = now_ns();
    fp_codec codec;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        auto it = S->dicts.find(r->dict_key);
        if (it == S->dicts.end()) return fail(FP_ERR_ARG, "dictionary key %llu is not registered",
                                              (unsigned long long)r->dict_key);
        codec = it->second.codec;
    }
    if (!r->d_code_offsets || reinterpret_cast<uintptr_t>(r->d_code_offsets) % 4)
        return fail(FP_ERR_ARG, "d_code_offsets is NULL or not 4-byte aligned");
    if (r->codes_bytes && !r->d_codes) return fail(FP_ERR_ARG, "d_codes is NULL");
    if (reinterpret_cast<uintptr_t>(r->d_codes) % 16) return fail(FP_ERR_ARG, "d_codes not 16-byte aligned");
    if (r->n_strings == 0xffffffffu) return fail(FP_ERR_ARG, "n_strings must be below 2^32-1");
    if (r->decoded_size > 0x7fffffffull) return fail(FP_ERR_ARG, "decoded_size above 2^31-1");
    (void)codec;
    Req* q = new Req();
    q->r = *r;
    q->t_submit = t;
    q->in_bytes = r->codes_bytes + ((uint64_t)r->n_strings + 1) * 4;
    const uint64_t need = al256(r->decoded_size) + al256(((uint64_t)r->n_strings + 1) * 4) + q->in_bytes;
    if (need > S->cfg.hbm_budget) {
        delete q;
        return fail(FP_ERR_BUSY, "request needs %llu bytes, above the HBM budget of %llu",
                    (unsigned long long)need, (unsigned long long)S->cfg.hbm_budget);
    }
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->stopping) {
            delete q;
            return fail(FP_ERR_BUSY, "server is shutting down");
        }
        q->ticket = ++S->next_ticket;
        S->live[q->ticket] = q;
        S->inbox.push_back(q);
        S->st.submitted++;
    }
    S->cv_sched.notify_one();
    *ticket = q->ticket;
    return FP_OK;
}

fp_status fp_serve_poll(fp_server* S, fp_result* out, uint32_t max, uint32_t* n, int64_t timeout_ns) {
    if (!S || !n || (max && !out)) return fail(FP_ERR_ARG, "server/out/n is NULL");
    *n = 0;
    std::unique_lock<std::mutex> lk(S->mu);
    if (S->finished.empty() && timeout_ns > 0)
        S->cv_done.wait_for(lk, std::chrono::nanoseconds(timeout_ns), [&] { return !S->finished.empty(); });
    while (*n < max && !S->finished.empty()) {
        Req* q = S->finished.front();
        S->finished.pop_front();
        fp_result& o = out[(*n)++];
        memset(&o, 0, sizeof(o));
        o.ticket = q->ticket;
        o.status = q->status;
        o.user_tag = q->r.user_tag;
        o.bytes = q->total;
        o.n_strings = q->r.n_strings;
        o.d_out_bytes = reinterpret_cast<uint8_t*>(S->d_arena + q->out_off);
        o.d_out_offsets = reinterpret_cast<uint32_t*>(S->d_arena + q->out_off + al256(q->r.decoded_size));
        o.t_submit_ns = q->t_submit;
        o.t_admit_ns = q->t_admit;
        o.t_done_ns = q->t_done;
    }
    return FP_OK;
}

fp_status fp_serve_release(fp_server* S, uint64_t ticket) {
    if (!S) return fail(FP_ERR_ARG, "server is NULL");
    {
        std::lock_guard<std::mutex> lk(S->mu);
        auto it = S->live.find(ticket);
        if (it == S->live.end()) return fail(FP_ERR_ARG, "unknown ticket %llu", (unsigned long long)ticket);
        Req* q = it->second;
        if (!q->done) return fail(FP_ERR_NOT_READY, "ticket %llu is still in flight", (unsigned long long)ticket);
        if (std::find(S->finished.begin(), S->finished.end(), q) != S->finished.end())
            return fail(FP_ERR_NOT_READY, "ticket %llu has not been polled", (unsigned long long)ticket);
        if (q->block) {
            S->arena.release(q->out_off, q->block);
            S->inflight_bytes -= q->block;
        }
        S->live.erase(it);
        S->st.released++;
        delete q;
    }
    S->cv_sched.notify_one();
    return FP_OK;
}

fp_status fp_serve_stats(fp_server* S, fp_serve_stats_t* out) {
    if (!S || !out) return fail(FP_ERR_ARG, "server/out is NULL");
    std::lock_guard<std::mutex> lk(S->mu);
    *out = S->st;
    out->inflight_bytes = S->inflight_bytes;
    out->inflight_requests = S->inflight_reqs;
    out->queued = (uint32_t)(S->inbox.size() + S->pending.size());
    return FP_OK;
}

fp_status fp_serve_destroy(fp_server* S) {
    if (!S) return FP_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stopping = true;
    }
    S->cv_sched.notify_all();
    if (S->th.joinable()) S->th.join();
    server_free(S);
    return FP_OK;
}

}  // extern "C"
