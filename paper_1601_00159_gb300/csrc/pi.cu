// Host side of the C ABI (include/pi.h): owns the device state of an index and
// enqueues the batch pipeline of Algorithm 1 on the caller's stream:
//   K0/K1 pack + radix sort  ->  K2/K3 descent + locate  ->  K4/K5 ownership + apply
//   ->  K6 merge + level layout + rebuild  ->  async copy of the small device meta to
//   a pinned mailbox (used only to tighten capacity bounds; never waited on, except
//   when a bound could be exceeded).

#include <cstdio>
#include <cstddef>
#include <cstring>
#include <mutex>
#include <string>
#include <new>
#include <algorithm>
#include <type_traits>
#include <vector>

#include "common.cuh"

namespace pi {
thread_local uint64_t g_launches = 0;
thread_local KernelTimer* g_ktimer = nullptr;
}  // namespace pi

using namespace pi;

namespace {

thread_local int g_last_error = PI_OK;

constexpr uint64_t kMinStorage = 1u << 16;

struct Scratch {
    uint64_t cap = 0;  // queries
    uint64_t* in_k = nullptr;
    uint32_t* in_p = nullptr;
    uint64_t* a_k = nullptr;
    uint32_t* a_p = nullptr;
    uint64_t* b_k = nullptr;
    uint32_t* b_p = nullptr;
    uint32_t* loc = nullptr;
    uint8_t* flags = nullptr;
    uint64_t* val0 = nullptr;
    NewNodes nn{};
    NewNodes stage{};
    uint32_t* tile_pref = nullptr;
    uint32_t* tile_new = nullptr;
    uint32_t* tcnt = nullptr;  // radix sort: per-tile digit counts
    uint32_t* toff = nullptr;  // radix sort: per-tile digit offsets
    uint32_t* gsum = nullptr;  // radix sort: per-group digit totals / offsets
    uint32_t* gctr = nullptr;  // radix sort: the count kernels' arrival counters
    uint8_t* ndig = nullptr;   // radix sort: next pass's digits
    uint32_t* fixmap = nullptr;  // radix sort: segment marks of the prefix fix-up
    LevelChanges cstage{};       // apply: per-tile staging of level membership changes
    LevelChanges chg{};          // apply: the changes, packed in key order
    uint32_t* tile_chg = nullptr;
    uint32_t* tile_chg_pref = nullptr;
    uint64_t* lst_keys = nullptr;  // incremental rebuild: per-level change lists
    uint32_t* lst_pos = nullptr;
    int32_t* lst_pref = nullptr;
    uint8_t* lst_ins = nullptr;
    uint64_t lst_cap = 0;
    uint32_t* sub_pref = nullptr;
    uint64_t* dq = nullptr;    // descent: dense distinct keys
    uint32_t* dlo = nullptr;   // descent: per-key start position
};

// pi_profile level 2: the two events around every kernel launch of the batch entry
// points, folded into per-kernel sums when read (or when the event pool is full).
struct KernelTimes final : KernelTimer {
    struct Rec {
        const void* f;
        cudaEvent_t a, b;
    };
    std::vector<cudaEvent_t> pool;
    size_t used = 0;
    cudaEvent_t pending = nullptr;
    std::vector<Rec> recs;
    std::vector<std::pair<const void*, std::pair<double, uint64_t>>> acc;  // kernel -> (ms, launches)
    cudaEvent_t take() {
        if (used == pool.size()) {
            cudaEvent_t e = nullptr;
            if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
            pool.push_back(e);
        }
        return pool[used++];
    }
    void before(cudaStream_t s) override {
        if (used + 2 > 8192) fold();
        pending = take();
        if (pending) cudaEventRecord(pending, s);
    }
    void after(const void* f, cudaStream_t s) override {
        cudaEvent_t e = take();
        if (!e || !pending) return;
        cudaEventRecord(e, s);
        recs.push_back({f, pending, e});
    }
    void fold() {
        for (const Rec& r : recs) {
            float ms = 0.f;
            cudaEventSynchronize(r.b);
            if (cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) continue;
            size_t k = 0;
            while (k < acc.size() && acc[k].first != r.f) ++k;
            if (k == acc.size()) acc.push_back({r.f, {0.0, 0}});
            acc[k].second.first += ms;
            acc[k].second.second += 1;
        }
        recs.clear();
        used = 0;
    }
    ~KernelTimes() {
        for (cudaEvent_t e : pool) cudaEventDestroy(e);
    }
};

struct Staging {
    uint64_t cap = 0;
    uint8_t* ops = nullptr;
    uint64_t* keys = nullptr;
    uint64_t* vals = nullptr;
    pi_result_t* res = nullptr;
};

}  // namespace

struct pi_index {
    int device = 0;
    int num_sms = 0;
    HashParams hp{};
    uint32_t rebuild_policy = 0, threshold_pct = 15;
    uint32_t smem_top = kSmemTopMax;  // pinned-entry cap
    uint32_t min_lb = 2;              // lowest index level built
    uint32_t test_flags = 0;
    uint32_t sort_cfg = 0;            // pi_config_t.sort_passes
    uint64_t launches = 0;            // kernels launched by the batch entry points
    uint32_t full_sort_left = 0;      // batches still sorted with all eight passes
    // range search: both bounds back to back, per-query storage slices and counts
    uint64_t* r_bounds = nullptr;
    uint32_t* r_start = nullptr;
    uint32_t* r_end = nullptr;
    uint32_t* r_cnt = nullptr;
    uint64_t* r_bsum = nullptr;
    uint64_t r_cap = 0;
    DevMeta* d_meta = nullptr;
    BatchMeta* d_bm = nullptr;  // two per-batch counter blocks, alternating between batches
    uint32_t* d_dofs = nullptr;
    uint32_t* d_count = nullptr;
    Storage st{};
    uint64_t st_cap = 0;  // nodes per buffer, padding excluded
    uint64_t* lkeys = nullptr;   // index-layer buffer 0
    uint32_t* ldown = nullptr;
    uint64_t* lkeys1 = nullptr;  // buffer 1 (DevMeta::lcur picks the one in use)
    uint32_t* ldown1 = nullptr;
    uint64_t idx_cap = 0;  // entries, padding excluded
    Scratch sc;
    // pi_execute_batch_host's pipeline: two staging slots, copies in on `hs`, the batch on
    // `cs`, copies out on `ds`; per slot, events for inputs copied, batch done, results
    // copied out (created on the first host-buffer call)
    Staging stg[2];
    cudaStream_t hs = nullptr, cs = nullptr, ds = nullptr;
    cudaEvent_t ev_in[2] = {}, ev_comp[2] = {}, ev_out[2] = {};
    uint64_t host_calls = 0;
    uint64_t* desc = nullptr;
    uint64_t desc_words = 0;
    uint32_t* lcnt = nullptr;  // per-level per-tile live counts: 32 rows x lstride
    uint32_t* mcnt = nullptr;  // merge: per-tile live counts and their prefix, 2 x lstride
    uint32_t* wcount = nullptr;  // PI_TEST_OWNER_CHECK: writes per storage node in a batch
    uint64_t wcap = 0;
    uint32_t* loff = nullptr;  // rebuild offsets, same shape
    uint32_t lstride = 0;
    uint32_t epoch = 1;
    // Ring of mailboxes: batch b copies the device meta to slot b % kRing and records
    // ev[b % kRing]; the newest completed slot bounds the host's view of the sizes.
    DevMeta* h_mbox = nullptr;  // pinned, kRing slots
    cudaEvent_t ev[64] = {};
    uint64_t ring_n[64] = {};   // queries of the batch in each slot
    uint64_t issued = 0;        // batches issued
    uint64_t seen = 0;          // batches whose mailbox has been read (a prefix)
    DevMeta known{};       // last mailbox snapshot
    uint64_t pending_n = 0;  // queries issued after that snapshot
    uint64_t extra_n = 0;    // queries of batching-form calls since the last full sync
    bool force_rebuild = false;
    // With small_mode 1, small batches (Q <= kSmallBatch on at most kSmallIndex nodes) run
    // through a one-index batching set whose batch takes a thread-block cluster: one
    // launch instead of the level-synchronous pipeline's tens. Created on first use.
    pi_multi* small = nullptr;
    uint32_t small_mode = 0;
    uint64_t routed = 0;  // batches that took the route
    // stage timing (pi_profile): events recorded between the pipeline's kernels
    bool prof = false;
    KernelTimes* kt = nullptr;   // pi_profile level 2
    cudaEvent_t* pev = nullptr;  // kProfSlots batches x kProfEvents events
    uint32_t pused = 0;          // batches recorded but not folded yet
    double pms[PI_NUM_STAGES] = {};
    uint64_t pbatches = 0;
    // Background rebuild (Section 4.4.4): the index-layer rebuild of a batch runs on its
    // own stream, overlapping the next batch's sort; the next batch's descent waits for
    // it (ev_rebuilt), and so does every other use of the index state.
    cudaStream_t rs = nullptr;
    cudaEvent_t ev_applied = nullptr, ev_rebuilt = nullptr;
    bool rebuild_pending = false;
    // The index's last operation (a batch, a range search or a batching-form call) ends
    // at last_ev on last_stream; an entry point on another stream first waits for it.
    // last_ev is the index's own ev_last, or the batching set's event for its calls.
    cudaEvent_t ev_last = nullptr;
    cudaEvent_t last_ev = nullptr;
    cudaStream_t last_stream = nullptr;
    bool has_last = false;
};

namespace {

// pi_test_fail_allocations: device allocations of this host thread still to fail.
thread_local uint32_t g_fail_allocs = 0;

template <typename T>
cudaError_t dalloc(T** p, uint64_t count) {
    *p = nullptr;
    if (g_fail_allocs > 0) {  // injected failure, as if the device were out of memory
        --g_fail_allocs;
        return cudaErrorMemoryAllocation;
    }
    if (count == 0) count = 1;
    return cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(T));
}

template <typename T>
void dfree(T*& p) {
    if (p) cudaFree(p);
    p = nullptr;
}

uint64_t host_splitmix64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

int shift_of(double p) {
    for (int b = 1; b <= 4; ++b)
        if (p == 1.0 / (double)(1u << b)) return b;
    return 0;
}

int map_cuda(cudaError_t e) {
    if (e == cudaSuccess) return PI_OK;
    if (e == cudaErrorMemoryAllocation) return PI_ERR_OOM;
    return PI_ERR_CUDA;
}

// Look-back descriptors needed for q queries and a storage capacity of s nodes.
uint64_t desc_need(uint64_t q, uint64_t s) {
    uint64_t a = 0;                                    // (the sort needs none)
    uint64_t b = 2 * ((q + 2047) / 2048);    // apply
    uint64_t c = (s / 4096 + 2) * 32;        // merge, export
    if (c < 32 * 64) c = 32 * 64;            // rebuild level scan: 64 chunks x 32 levels
    uint64_t m = a > b ? a : b;
    return (m > c ? m : c) + 64;
}

cudaError_t ensure_desc(pi_index* x, uint64_t words) {
    if (words <= x->desc_words) return cudaSuccess;
    dfree(x->desc);
    cudaError_t e = dalloc(&x->desc, words);
    if (e != cudaSuccess) {
        x->desc_words = 0;
        return e;
    }
    e = cudaMemset(x->desc, 0, words * sizeof(uint64_t));
    x->desc_words = words;
    return e;
}

// Per-level per-tile counts are rows of (storage capacity / 4096 + 2) tiles; a new
// capacity reallocates them and the next rebuild recounts (force_rebuild).
cudaError_t ensure_tile_cnt(pi_index* x, uint64_t st_cap) {
    const uint64_t stride = st_cap / 4096 + 2;
    if (stride <= x->lstride) return cudaSuccess;
    dfree(x->lcnt);
    dfree(x->loff);
    dfree(x->mcnt);
    cudaError_t e = dalloc(&x->lcnt, 32 * stride);
    if (e == cudaSuccess) e = dalloc(&x->loff, 32 * stride);
    if (e == cudaSuccess) e = dalloc(&x->mcnt, 2 * stride);
    if (e == cudaSuccess) e = cudaMemset(x->lcnt, 0, 32 * stride * sizeof(uint32_t));
    x->lstride = (e == cudaSuccess) ? (uint32_t)stride : 0u;
    x->force_rebuild = true;
    return e;
}

// PI_TEST_OWNER_CHECK: one zeroed write counter per storage node.
cudaError_t ensure_wcount(pi_index* x, uint64_t st_cap) {
    if (!(x->test_flags & PI_TEST_OWNER_CHECK) || x->wcap >= st_cap) return cudaSuccess;
    dfree(x->wcount);
    x->wcap = 0;
    cudaError_t e = dalloc(&x->wcount, st_cap + 1);
    if (e == cudaSuccess) e = cudaMemset(x->wcount, 0, (st_cap + 1) * sizeof(uint32_t));
    if (e == cudaSuccess) x->wcap = st_cap;
    return e;
}

uint32_t next_epochs(pi_index* x, uint32_t count, cudaStream_t s) {
    // Epochs tag look-back descriptors; on wrap-around clear them so no stale word can
    // carry a reused epoch.
    if (x->epoch > 0xFFFFFFFFu - count - 64u) {
        cudaMemsetAsync(x->desc, 0, x->desc_words * sizeof(uint64_t), s);
        x->epoch = 1;
    }
    return x->epoch;
}

void free_scratch(Scratch& s) {
    dfree(s.in_k); dfree(s.in_p); dfree(s.a_k); dfree(s.a_p); dfree(s.b_k); dfree(s.b_p);
    dfree(s.loc); dfree(s.flags); dfree(s.val0);
    dfree(s.nn.keys); dfree(s.nn.vals); dfree(s.nn.loc); dfree(s.nn.height);
    dfree(s.stage.keys); dfree(s.stage.vals); dfree(s.stage.loc); dfree(s.stage.height);
    dfree(s.tile_pref); dfree(s.tile_new);
    dfree(s.tcnt); dfree(s.toff); dfree(s.ndig); dfree(s.fixmap); dfree(s.gsum); dfree(s.gctr);
    dfree(s.cstage.keys); dfree(s.cstage.pos); dfree(s.cstage.hl); dfree(s.chg.keys); dfree(s.chg.pos); dfree(s.chg.hl);
    dfree(s.tile_chg); dfree(s.tile_chg_pref);
    dfree(s.lst_keys); dfree(s.lst_pos); dfree(s.lst_pref); dfree(s.lst_ins);
    dfree(s.sub_pref); dfree(s.dq); dfree(s.dlo);
    s.cap = 0;
}

cudaError_t alloc_scratch(Scratch& s, uint64_t q) {
    cudaError_t e = cudaSuccess;
    const uint64_t c = q + kPad;
#define PI_TRY(expr) do { e = (expr); if (e != cudaSuccess) { free_scratch(s); return e; } } while (0)
    PI_TRY(dalloc(&s.in_k, c)); PI_TRY(dalloc(&s.in_p, c));
    PI_TRY(dalloc(&s.a_k, c)); PI_TRY(dalloc(&s.a_p, c));
    PI_TRY(dalloc(&s.b_k, c)); PI_TRY(dalloc(&s.b_p, c));
    PI_TRY(dalloc(&s.loc, c)); PI_TRY(dalloc(&s.flags, c)); PI_TRY(dalloc(&s.val0, c));
    PI_TRY(dalloc(&s.nn.keys, c)); PI_TRY(dalloc(&s.nn.vals, c));
    PI_TRY(dalloc(&s.nn.loc, c)); PI_TRY(dalloc(&s.nn.height, c));
    const uint64_t tiles = (q + kApplyTile - 1) / kApplyTile + 1;
    const uint64_t cs = tiles * kApplyTile;
    PI_TRY(dalloc(&s.stage.keys, cs)); PI_TRY(dalloc(&s.stage.vals, cs));
    PI_TRY(dalloc(&s.stage.loc, cs)); PI_TRY(dalloc(&s.stage.height, cs));
    PI_TRY(dalloc(&s.tile_pref, tiles)); PI_TRY(dalloc(&s.tile_new, tiles));
    const uint64_t stiles = (q + kSortTile - 1) / kSortTile + 1;
    PI_TRY(dalloc(&s.tcnt, stiles * 256)); PI_TRY(dalloc(&s.toff, stiles * 256));
    const uint64_t sgroups = stiles / kScanGroup + 1;
    PI_TRY(dalloc(&s.gsum, sgroups * 256)); PI_TRY(dalloc(&s.gctr, 8 * (sgroups + 1)));
    PI_TRY(dalloc(&s.ndig, stiles * kSortTile + 16));
    PI_TRY(dalloc(&s.fixmap, c / 32 + 1));
    PI_TRY(dalloc(&s.cstage.keys, cs)); PI_TRY(dalloc(&s.cstage.pos, cs)); PI_TRY(dalloc(&s.cstage.hl, cs));
    PI_TRY(dalloc(&s.chg.keys, c)); PI_TRY(dalloc(&s.chg.pos, c)); PI_TRY(dalloc(&s.chg.hl, c));
    PI_TRY(dalloc(&s.tile_chg, tiles)); PI_TRY(dalloc(&s.tile_chg_pref, tiles));
    s.lst_cap = 2 * c + 64;
    PI_TRY(dalloc(&s.lst_keys, s.lst_cap)); PI_TRY(dalloc(&s.lst_pos, s.lst_cap));
    PI_TRY(dalloc(&s.lst_pref, s.lst_cap)); PI_TRY(dalloc(&s.lst_ins, s.lst_cap));
    const uint64_t nsub = (q + kSubTile - 1) / kSubTile + 1;
    PI_TRY(dalloc(&s.sub_pref, nsub));
    PI_TRY(dalloc(&s.dq, c)); PI_TRY(dalloc(&s.dlo, c));
#undef PI_TRY
    s.cap = q;
    return cudaSuccess;
}

void free_storage(Storage& st) {
    for (int i = 0; i < 2; ++i) {
        dfree(st.keys[i]); dfree(st.vals[i]); dfree(st.meta[i]);
    }
}

// Storage arrays are padded by a whole 4096-node tile plus kPad entries, so that tile
// loads of the last (partial) tile and read-ahead past the sentinel stay in bounds.
uint64_t storage_alloc(uint64_t cap) { return cap + 4096 + kPad; }

cudaError_t alloc_storage(Storage& st, uint64_t cap) {
    cudaError_t e;
    const uint64_t c = storage_alloc(cap);
    for (int i = 0; i < 2; ++i) {
        if ((e = dalloc(&st.keys[i], c)) != cudaSuccess) break;
        if ((e = dalloc(&st.vals[i], c)) != cudaSuccess) break;
        if ((e = dalloc(&st.meta[i], c)) != cudaSuccess) break;
        cudaMemset(st.meta[i], 0, c);
    }
    if (e != cudaSuccess) free_storage(st);
    return e;
}

constexpr uint32_t kProfSlots = 2048;
// Per batch: 0 start, 1 after sort, 2 after waiting for the previous rebuild, 3 after
// descent, 4 after apply, 5 after merge, 6 after layout, 7 rebuild start, 8 before the
// rebuild's writer kernel, 9 rebuild end, 10 before the storage locate.
constexpr int kProfEvents = 11;

void prof_fold(pi_index* x) {
    static const int from[PI_NUM_STAGES] = {0, 2, 3, 4, 5, 7, 8, 10};
    static const int to[PI_NUM_STAGES] = {1, 3, 4, 5, 6, 9, 9, 3};
    for (uint32_t b = 0; b < x->pused; ++b) {
        cudaEvent_t* e = x->pev + (size_t)b * kProfEvents;
        cudaEventSynchronize(e[9]);
        cudaEventSynchronize(e[6]);
        for (int st = 0; st < PI_NUM_STAGES; ++st) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, e[from[st]], e[to[st]]) == cudaSuccess) x->pms[st] += ms;
        }
        x->pbatches++;
    }
    x->pused = 0;
}

// Event for stage boundary k of the batch being enqueued (nullptr when not profiling).
cudaEvent_t prof_event(pi_index* x, int k) {
    if (!x->prof) return nullptr;
    return x->pev[(size_t)x->pused * kProfEvents + k];
}

void prof_mark(pi_index* x, int k, cudaStream_t s) {
    if (cudaEvent_t e = prof_event(x, k)) cudaEventRecord(e, s);
}

void multi_destroy(pi_multi* mx);
bool small_route(const pi_index* x, uint64_t n, uint64_t size_ub);
int execute_small(pi_index* x, const uint8_t* ops, const uint64_t* keys, const uint64_t* values, uint64_t n,
                  pi_result_t* results, cudaStream_t s);
constexpr int kNoRoute = 1;  // execute_small: no cluster fits; the caller takes the plain path

void destroy(pi_index* x) {
    if (!x) return;
    cudaSetDevice(x->device);
    cudaDeviceSynchronize();
    if (x->small) multi_destroy(x->small);
    if (x->pev) {
        for (size_t i = 0; i < (size_t)kProfSlots * kProfEvents; ++i) cudaEventDestroy(x->pev[i]);
        delete[] x->pev;
    }
    delete x->kt;
    free_scratch(x->sc);
    dfree(x->r_bounds); dfree(x->r_start); dfree(x->r_end); dfree(x->r_cnt); dfree(x->r_bsum);
    for (auto& g : x->stg) {
        dfree(g.ops); dfree(g.keys); dfree(g.vals); dfree(g.res);
    }
    for (int k = 0; k < 2; ++k) {
        if (x->ev_in[k]) cudaEventDestroy(x->ev_in[k]);
        if (x->ev_comp[k]) cudaEventDestroy(x->ev_comp[k]);
        if (x->ev_out[k]) cudaEventDestroy(x->ev_out[k]);
    }
    if (x->hs) cudaStreamDestroy(x->hs);
    if (x->cs) cudaStreamDestroy(x->cs);
    if (x->ds) cudaStreamDestroy(x->ds);
    if (x->ev_last) cudaEventDestroy(x->ev_last);
    free_storage(x->st);
    dfree(x->lkeys); dfree(x->ldown); dfree(x->lkeys1); dfree(x->ldown1);
    dfree(x->desc); dfree(x->lcnt); dfree(x->loff); dfree(x->mcnt); dfree(x->wcount); dfree(x->d_meta); dfree(x->d_bm); dfree(x->d_dofs); dfree(x->d_count);
    if (x->h_mbox) cudaFreeHost(x->h_mbox);
    if (x->ev_applied) cudaEventDestroy(x->ev_applied);
    if (x->ev_rebuilt) cudaEventDestroy(x->ev_rebuilt);
    if (x->rs) cudaStreamDestroy(x->rs);
    for (auto& e : x->ev)
        if (e) cudaEventDestroy(e);
    delete x;
}

SortBuffers sort_buffers(pi_index* x, const Scratch& s) {
    SortBuffers sb;
    sb.in_k = s.in_k; sb.in_p = s.in_p; sb.a_k = s.a_k; sb.a_p = s.a_p; sb.b_k = s.b_k; sb.b_p = s.b_p;
    sb.dofs = x->d_dofs;
    sb.desc = x->desc;
    sb.tcnt = s.tcnt;
    sb.toff = s.toff;
    sb.gsum = s.gsum;
    sb.gctr = s.gctr;
    sb.ndig = s.ndig;
    sb.fixmap = s.fixmap;
    return sb;
}

// Read the device meta synchronously (after a stream sync).
cudaError_t read_meta(pi_index* x, cudaStream_t s, DevMeta* out) {
    cudaError_t e = cudaMemcpyAsync(out, x->d_meta, sizeof(DevMeta), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e;
}

constexpr uint64_t kRing = 64;

// Non-blocking: adopt the newest completed batch's mailbox.
void refresh_known(pi_index* x) {
    uint64_t newest = x->seen;
    for (uint64_t b = x->issued; b > x->seen; --b) {
        if (cudaEventQuery(x->ev[(b - 1) % kRing]) == cudaSuccess) {
            newest = b;
            break;
        }
    }
    if (newest == x->seen) return;
    x->known = x->h_mbox[(newest - 1) % kRing];
    x->seen = newest;
    uint64_t p = 0;
    for (uint64_t b = newest; b < x->issued; ++b) p += x->ring_n[b % kRing];
    x->pending_n = p;
}

// Makes `s` wait for the background rebuild still in flight, if any (no host sync).
void wait_rebuild(pi_index* x, cudaStream_t s) {
    if (x->rebuild_pending) cudaStreamWaitEvent(s, x->ev_rebuilt, 0);
}

// Makes `s` wait for the index's last operation when that ran on another stream.
void order_after_last(pi_index* x, cudaStream_t s) {
    if (x->has_last && x->last_stream != s) cudaStreamWaitEvent(s, x->last_ev, 0);
}

void mark_last(pi_index* x, cudaStream_t s) {
    cudaEventRecord(x->ev_last, s);
    x->last_ev = x->ev_last;
    x->last_stream = s;
    x->has_last = true;
}

cudaError_t sync_known(pi_index* x, cudaStream_t s) {
    order_after_last(x, s);
    wait_rebuild(x, s);
    cudaError_t e = read_meta(x, s, &x->known);
    if (e == cudaSuccess) x->rebuild_pending = false;
    if (e == cudaSuccess) {
        for (uint64_t b = x->seen; b < x->issued; ++b) cudaEventSynchronize(x->ev[b % kRing]);
        x->seen = x->issued;
        x->pending_n = 0;
        x->extra_n = 0;
    }
    return e;
}

int sticky_error(const DevMeta& m) {
    if (m.error & kErrTimeout) return PI_ERR_TIMEOUT;
    if (m.error) return PI_ERR_CUDA;
    return PI_OK;
}

cudaError_t grow_storage(pi_index* x, uint64_t need, cudaStream_t s) {
    uint64_t cap = need + need / 2 + kMinStorage;
    if (cap > PI_MAX_KEYS) cap = PI_MAX_KEYS;
    Storage ns{};
    cudaError_t e = alloc_storage(ns, cap);
    if (e != cudaSuccess) return e;
    const uint32_t cur = x->known.cur;
    const uint64_t cnt = (uint64_t)x->known.size + 1;  // with the sentinel
    cudaMemcpyAsync(ns.keys[0], x->st.keys[cur], cnt * 8, cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(ns.vals[0], x->st.vals[cur], cnt * 8, cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(ns.meta[0], x->st.meta[cur], cnt, cudaMemcpyDeviceToDevice, s);
    cudaMemsetAsync(&x->d_meta->cur, 0, sizeof(uint32_t), s);
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        free_storage(ns);
        return e;
    }
    free_storage(x->st);
    x->st = ns;
    x->st_cap = cap;
    x->known.cur = 0;
    if ((e = ensure_tile_cnt(x, cap)) != cudaSuccess) return e;
    if ((e = ensure_wcount(x, cap)) != cudaSuccess) return e;
    return ensure_desc(x, desc_need(x->sc.cap, cap));
}

cudaError_t grow_index(pi_index* x, uint64_t need, cudaStream_t s) {
    uint64_t cap = need + need / 4 + 4096;
    uint64_t *nk = nullptr, *nk1 = nullptr;
    uint32_t *nd = nullptr, *nd1 = nullptr;
    cudaError_t e = dalloc(&nk, cap + kPad);
    if (e == cudaSuccess) e = dalloc(&nd, cap + kPad);
    if (e == cudaSuccess) e = dalloc(&nk1, cap + kPad);
    if (e == cudaSuccess) e = dalloc(&nd1, cap + kPad);
    if (e != cudaSuccess) {
        dfree(nk); dfree(nd); dfree(nk1); dfree(nd1);
        return e;
    }
    // the levels in use move to buffer 0 of the new arrays (called with `known` current)
    const uint64_t used = x->known.index_total;
    const uint64_t* ok = x->known.lcur ? x->lkeys1 : x->lkeys;
    const uint32_t* od = x->known.lcur ? x->ldown1 : x->ldown;
    if (ok && used) {
        cudaMemcpyAsync(nk, ok, used * 8, cudaMemcpyDeviceToDevice, s);
        cudaMemcpyAsync(nd, od, used * 4, cudaMemcpyDeviceToDevice, s);
    }
    const uint32_t zero = 0;
    cudaMemcpyAsync(&x->d_meta->lcur, &zero, sizeof(zero), cudaMemcpyHostToDevice, s);
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        dfree(nk); dfree(nd); dfree(nk1); dfree(nd1);
        return e;
    }
    dfree(x->lkeys); dfree(x->ldown); dfree(x->lkeys1); dfree(x->ldown1);
    x->lkeys = nk;
    x->ldown = nd;
    x->lkeys1 = nk1;
    x->ldown1 = nd1;
    x->known.lcur = 0;
    x->idx_cap = cap;
    x->force_rebuild = true;
    return cudaSuccess;
}

// Per-batch scratch for at least n queries (synchronises `s`: the scratch is in use until
// the batches before have finished). It grows to 1.5 times the old capacity at least, so
// a stream of growing batches reallocates a few times, not once per batch.
cudaError_t grow_scratch(pi_index* x, uint64_t n, cudaStream_t s) {
    wait_rebuild(x, s);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    x->rebuild_pending = false;
    uint64_t q = std::max<uint64_t>(n, x->sc.cap + x->sc.cap / 2);
    q = std::min<uint64_t>(std::max<uint64_t>(q, 4096), std::max<uint64_t>(n, PI_MAX_BATCH));
    free_scratch(x->sc);
    if ((e = alloc_scratch(x->sc, q)) != cudaSuccess) return e;
    return ensure_desc(x, desc_need(q, x->st_cap));
}

// The descent walks the levels below the pinned ones inside its top kernel, one key
// per thread, as long as they are small (about 24 MB of entries: L2-resident); the
// levels below get one launch each. Taken from the host's last view of the index; any
// split gives the same result.
constexpr uint64_t kWalkEntries = 2u << 20;

int top_launched_for(const pi_index* x) {
    const DevMeta& k = x->known;
    if (x->test_flags & PI_TEST_WALK_LEVELS) return 2;
    if (k.Ls < 3 || k.Ls > (uint32_t)x->hp.hmax + 1) return x->hp.hmax;
    uint64_t cum = 0;
    int l = (int)k.Ls - 1;
    while (l >= 2 && cum + k.n[l] <= kWalkEntries) {
        cum += k.n[l];
        --l;
    }
    return l < 2 ? 2 : l;
}

RebuildArgs rebuild_args(pi_index* x, BatchMeta* bm, uint32_t size_ub, uint32_t force) {
    RebuildArgs r{};
    r.st = x->st;
    r.nn = x->sc.nn;
    r.m = x->d_meta;
    r.bm = bm;
    r.lkeys = x->lkeys;
    r.ldown = x->ldown;
    r.lkeys1 = x->lkeys1;
    r.ldown1 = x->ldown1;
    r.desc = x->desc;
    r.lcnt = x->lcnt;
    r.loff = x->loff;
    r.mcnt = x->mcnt;
    r.lstride = x->lstride;
    r.index_cap = (uint32_t)(x->idx_cap > 0xFFFFFFF0ull ? 0xFFFFFFF0ull : x->idx_cap);
    r.size_ub = size_ub;
    r.rebuild_policy = x->rebuild_policy;
    r.threshold_pct = x->threshold_pct;
    r.force_rebuild = force;
    r.st_cap = (uint32_t)x->st_cap;
    r.smem_top = x->smem_top;
    r.min_lb = x->min_lb;
    r.err = &x->d_meta->error;
    return r;
}

// ---------------------------------------------------------------------------------
// Allocation-free batches (pi_execute_batch_noalloc): the per-batch scratch of up to
// PI_NOALLOC_MAX_BATCH queries lives in one file-scope device array, carved into the
// same buffers alloc_scratch() would allocate, in this order.
constexpr uint64_t al256(uint64_t b) { return (b + 255) & ~uint64_t(255); }

constexpr uint64_t noalloc_bytes(uint64_t q) {
    const uint64_t c = q + kPad;
    const uint64_t tiles = (q + kApplyTile - 1) / kApplyTile + 1, cs = tiles * kApplyTile;
    const uint64_t stiles = (q + kSortTile - 1) / kSortTile + 1;
    const uint64_t nsub = (q + kSubTile - 1) / kSubTile + 1;
    return 3 * al256(c * 8) + 3 * al256(c * 4)                    // in, a, b (keys, payload)
           + al256(c * 4) + al256(c) + al256(c * 8)               // loc, flags, val0
           + 2 * al256(c * 8) + al256(c * 4) + al256(c)           // new nodes
           + 2 * al256(cs * 8) + al256(cs * 4) + al256(cs)        // new-node staging
           + 2 * al256(tiles * 4)                                 // tile prefix / new
           + 2 * al256(stiles * 256 * 4) + al256(stiles * kSortTile + 16)  // tcnt, toff, ndig
           + al256((stiles / kScanGroup + 1) * 256 * 4) + al256(8 * (stiles / kScanGroup + 2) * 4)  // gsum, gctr
           + al256((c / 32 + 1) * 4)                              // fixmap
           + al256(cs * 8) + al256(cs * 4) + al256(cs)            // level-change staging
           + al256(c * 8) + al256(c * 4) + al256(c)               // level changes
           + 2 * al256(tiles * 4)                                 // per-tile change counts
           + al256((2 * c + 64) * 8) + 2 * al256((2 * c + 64) * 4) + al256(2 * c + 64)  // lists
           + al256(nsub * 4)                                      // sub_pref
           + al256(c * 8) + al256(c * 4);                         // dq, dlo
}

constexpr uint64_t kNoAllocBytes = noalloc_bytes(PI_NOALLOC_MAX_BATCH);

// Shared by every call on a device; each GPU that loads the library holds it until exit.
static __device__ __align__(256) uint8_t g_noalloc_scratch[kNoAllocBytes];

// Carves `base` like noalloc_bytes(q); returns the bytes used.
uint64_t carve_scratch(uint8_t* base, uint64_t q, Scratch& s) {
    uint64_t off = 0;
    auto take = [&](auto*& ptr, uint64_t bytes) {
        ptr = reinterpret_cast<std::remove_reference_t<decltype(ptr)>>(base + off);
        off += al256(bytes);
    };
    const uint64_t c = q + kPad;
    const uint64_t tiles = (q + kApplyTile - 1) / kApplyTile + 1, cs = tiles * kApplyTile;
    const uint64_t stiles = (q + kSortTile - 1) / kSortTile + 1;
    const uint64_t nsub = (q + kSubTile - 1) / kSubTile + 1;
    take(s.in_k, c * 8); take(s.a_k, c * 8); take(s.b_k, c * 8);
    take(s.in_p, c * 4); take(s.a_p, c * 4); take(s.b_p, c * 4);
    take(s.loc, c * 4); take(s.flags, c); take(s.val0, c * 8);
    take(s.nn.keys, c * 8); take(s.nn.vals, c * 8); take(s.nn.loc, c * 4); take(s.nn.height, c);
    take(s.stage.keys, cs * 8); take(s.stage.vals, cs * 8); take(s.stage.loc, cs * 4); take(s.stage.height, cs);
    take(s.tile_pref, tiles * 4); take(s.tile_new, tiles * 4);
    take(s.tcnt, stiles * 256 * 4); take(s.toff, stiles * 256 * 4); take(s.ndig, stiles * kSortTile + 16);
    take(s.gsum, (stiles / kScanGroup + 1) * 256 * 4); take(s.gctr, 8 * (stiles / kScanGroup + 2) * 4);
    take(s.fixmap, (c / 32 + 1) * 4);
    take(s.cstage.keys, cs * 8); take(s.cstage.pos, cs * 4); take(s.cstage.hl, cs);
    take(s.chg.keys, c * 8); take(s.chg.pos, c * 4); take(s.chg.hl, c);
    take(s.tile_chg, tiles * 4); take(s.tile_chg_pref, tiles * 4);
    s.lst_cap = 2 * c + 64;
    take(s.lst_keys, s.lst_cap * 8); take(s.lst_pos, s.lst_cap * 4); take(s.lst_pref, s.lst_cap * 4);
    take(s.lst_ins, s.lst_cap);
    take(s.sub_pref, nsub * 4);
    take(s.dq, c * 8); take(s.dlo, c * 4);
    s.cap = q;
    return off;
}

// Per device: the array's device address, looked up once with that device current, and
// the hand-over between calls on different indices. A batch's index-layer rebuild runs
// on its index's own stream and reads its part of the array (new nodes, level changes,
// change lists) after the caller's stream has moved on. A call on another index would
// overwrite those parts from its first kernels, so its stream first waits for the last
// call's rebuild (`rebuilt`, recorded after it). Calls on one index need no such wait:
// only the sort runs before a batch waits for the previous rebuild, and the sort's
// buffers are not among the parts the rebuild reads.
struct NoAllocDevice {
    uint8_t* ptr = nullptr;
    cudaEvent_t rebuilt = nullptr;
    const pi_index* last = nullptr;  // index of the last call on this device
};
std::mutex g_noalloc_mu;
NoAllocDevice g_noalloc[64];

cudaError_t noalloc_scratch_for(int device, NoAllocDevice** out) {
    if (device < 0 || device >= 64) return cudaErrorInvalidDevice;
    NoAllocDevice& d = g_noalloc[device];
    if (!d.ptr) {
        int prev = -1;
        cudaError_t e = cudaGetDevice(&prev);
        if (e != cudaSuccess) return e;
        if (prev != device && (e = cudaSetDevice(device)) != cudaSuccess) return e;
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e == cudaSuccess && !d.rebuilt) e = cudaEventCreateWithFlags(&d.rebuilt, cudaEventDisableTiming);
        if (prev != device) cudaSetDevice(prev);
        if (e != cudaSuccess) return e;
        d.ptr = static_cast<uint8_t*>(p);
    }
    *out = &d;
    return cudaSuccess;
}

// Radix passes for a batch of n queries. Four passes on the most significant varying
// key bytes leave only prefix collisions to the fix-up; when the last batch the host
// knows of had more than n/16 queries in long colliding segments (keys whose leading
// bytes carry little spread), the next 64 batches take all eight passes instead.
int sort_passes(pi_index* x, uint64_t n) {
    const uint32_t forced = (x->test_flags / PI_TEST_SORT_PREFIX(1)) & 7u;
    if (forced >= 1 && forced <= 4) return (int)forced;
    if (x->test_flags & PI_TEST_SORT_FULL) return 8;
    if (x->sort_cfg == 8) return 8;
    const int prefix = x->sort_cfg ? (int)x->sort_cfg : 4;
    if ((uint64_t)x->known.sort_fix_big * 16u > n) {
        x->full_sort_left = 64;
        x->known.sort_fix_big = 0;  // one trigger per snapshot
    }
    if (x->full_sort_left > 0) {
        --x->full_sort_left;
        return 8;
    }
    return prefix;
}

// Enqueues one batch (Algorithm 1) with the given per-batch scratch:
//   stream s:  pack + sort -> [wait for the previous batch's rebuild] -> descent ->
//              ownership + apply -> merge -> layout -> meta to the mailbox ring
//   stream rs: [wait for this batch's layout] -> index-layer rebuild
// The rebuild thus overlaps the next batch's sort (the paper's background rebuild,
// Section 4.4.4). Results are complete when `s` completes.
int enqueue_batch_body(pi_index* x, const Scratch& sc, const uint8_t* ops, const uint64_t* keys,
                       const uint64_t* values, uint64_t n, pi_result_t* results, uint64_t size_ub,
                       cudaStream_t s) {
    cudaError_t e;
    BatchMeta* bm = x->d_bm + (x->issued & 1u);  // the other block may still be read by the rebuild
    uint32_t ep = next_epochs(x, 16, s);
    if (x->prof && x->pused == kProfSlots) prof_fold(x);
    prof_mark(x, 0, s);
    cudaMemsetAsync(bm, 0, sizeof(BatchMeta), s);
    SortBuffers sb = sort_buffers(x, sc);
    if ((e = launch_sort(ops, keys, (uint32_t)n, sb, bm, &x->d_meta->error, s, x->num_sms, sort_passes(x, n))) !=
        cudaSuccess)
        return map_cuda(e);
    prof_mark(x, 1, s);
    wait_rebuild(x, s);
    prof_mark(x, 2, s);
    DescendArgs da{};
    da.sk = sc.a_k;
    da.sp = sc.a_p;
    da.tile_pref = sc.tile_pref;
    da.sub_pref = sc.sub_pref;
    da.desc = x->desc;
    da.dq = sc.dq;
    da.dlo = sc.dlo;
    // the lowest buildable level is never walked by the prologue: the storage locate
    // searches it itself (it needs that level's gap ends)
    da.top_launched = std::max(top_launched_for(x), (int)x->min_lb);
    da.bottom_launched = (int)x->min_lb;
    da.m = x->d_meta;
    da.bm = bm;
    da.lkeys = x->lkeys;
    da.ldown = x->ldown;
    da.lkeys1 = x->lkeys1;
    da.ldown1 = x->ldown1;
    da.st = x->st;
    da.loc = sc.loc;
    da.flags = sc.flags;
    da.val0 = sc.val0;
    da.n = (uint32_t)n;
    da.err = &x->d_meta->error;
    if ((e = launch_descend(da, ep, s, x->num_sms, prof_event(x, 10))) != cudaSuccess) return map_cuda(e);
    prof_mark(x, 3, s);
    ApplyArgs aa{};
    aa.sk = sc.a_k;
    aa.sp = sc.a_p;
    aa.loc = sc.loc;
    aa.flags = sc.flags;
    aa.val0 = sc.val0;
    aa.uvals = values;
    aa.results = results;
    aa.st = x->st;
    aa.nn = sc.nn;
    aa.m = x->d_meta;
    aa.bm = bm;
    aa.desc = x->desc;
    aa.tile_pref = sc.tile_pref;
    aa.tile_new = sc.tile_new;
    aa.sub_pref = sc.sub_pref;
    aa.stage = sc.stage;
    aa.cstage = sc.cstage;
    aa.chg = sc.chg;
    aa.tile_chg = sc.tile_chg;
    aa.tile_chg_pref = sc.tile_chg_pref;
    aa.lcnt = x->lcnt;
    aa.lstride = x->lstride;
    aa.n = (uint32_t)n;
    aa.hp = x->hp;
    aa.err = &x->d_meta->error;
    aa.wcount = x->wcount;
    if ((e = launch_apply(aa, ep, s, x->num_sms)) != cudaSuccess) return map_cuda(e);
    if ((e = launch_owner_check(aa, s, x->num_sms)) != cudaSuccess) return map_cuda(e);
    prof_mark(x, 4, s);
    RebuildArgs ra = rebuild_args(x, bm, (uint32_t)size_ub, x->force_rebuild ? 1u : 0u);
    ra.nn = sc.nn;
    ra.chg = sc.chg;
    ra.lst_keys = sc.lst_keys;
    ra.lst_pos = sc.lst_pos;
    ra.lst_pref = sc.lst_pref;
    ra.lst_ins = sc.lst_ins;
    ra.lst_cap = (uint32_t)(sc.lst_cap > 0xFFFFFFF0ull ? 0xFFFFFFF0ull : sc.lst_cap);
    if ((e = launch_merge(ra, ep, s, x->num_sms)) != cudaSuccess) return map_cuda(e);
    prof_mark(x, 5, s);
    if ((e = launch_level_bases(ra, s)) != cudaSuccess) return map_cuda(e);
    prof_mark(x, 6, s);
    const uint64_t slot = x->issued % kRing;
    if (x->issued - x->seen >= kRing) {  // the slot is still unread: wait for its batch
        cudaEventSynchronize(x->ev[slot]);
        refresh_known(x);
    }
    cudaMemcpyAsync(&x->h_mbox[slot], x->d_meta, sizeof(DevMeta), cudaMemcpyDeviceToHost, s);
    cudaEventRecord(x->ev[slot], s);
    // the rebuild, in the background
    cudaEventRecord(x->ev_applied, s);
    cudaStreamWaitEvent(x->rs, x->ev_applied, 0);
    prof_mark(x, 7, x->rs);
    if ((e = launch_rebuild_prep(ra, ep, x->rs, x->num_sms)) != cudaSuccess) return map_cuda(e);
    prof_mark(x, 8, x->rs);
    if ((e = launch_rebuild_write(ra, x->rs, x->num_sms)) != cudaSuccess) return map_cuda(e);
    if ((e = launch_relevel(ra, x->rs, x->num_sms)) != cudaSuccess) return map_cuda(e);
    prof_mark(x, 9, x->rs);
    cudaEventRecord(x->ev_rebuilt, x->rs);
    x->rebuild_pending = true;
    if (x->prof) x->pused++;
    x->epoch = ep;
    x->force_rebuild = false;
    x->ring_n[slot] = n;
    x->issued++;
    x->pending_n += n;
    return map_cuda(cudaGetLastError());
}

int enqueue_batch(pi_index* x, const Scratch& sc, const uint8_t* ops, const uint64_t* keys,
                  const uint64_t* values, uint64_t n, pi_result_t* results, uint64_t size_ub, cudaStream_t s) {
    const uint64_t l0 = g_launches;
    g_ktimer = x->kt;
    const int r = enqueue_batch_body(x, sc, ops, keys, values, n, results, size_ub, s);
    g_ktimer = nullptr;
    if (r == PI_OK) mark_last(x, s);
    x->launches += g_launches - l0;
    return r;
}

}  // namespace

extern "C" {

int pi_last_error(void) { return g_last_error; }

pi_index_t* pi_create_ex(const uint64_t* keys, const uint64_t* values, uint64_t n, double promote_p,
                         uint64_t seed, const pi_config_t* cfg) {
    g_last_error = PI_OK;
    const int b = shift_of(promote_p);
    if (b == 0 || n > PI_MAX_KEYS || (n > 0 && (!keys || !values))) {
        g_last_error = PI_ERR_INVALID_ARG;
        return nullptr;
    }
    // the fields up to lowest_level are required; later ones read as 0 when struct_size
    // does not reach them (callers built against an older header)
    constexpr size_t kCfgBase = offsetof(pi_config_t, sort_passes);
    if (cfg && cfg->struct_size != 0 && cfg->struct_size < kCfgBase) {
        g_last_error = PI_ERR_INVALID_ARG;
        return nullptr;
    }
    const bool cfg_full = cfg && (cfg->struct_size == 0 || cfg->struct_size >= sizeof(pi_config_t));
    pi_index* x = new (std::nothrow) pi_index();
    if (!x) {
        g_last_error = PI_ERR_OOM;
        return nullptr;
    }
    cudaError_t e = cudaGetDevice(&x->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&x->num_sms, cudaDevAttrMultiProcessorCount, x->device);
    if (e != cudaSuccess) {
        g_last_error = PI_ERR_CUDA;
        delete x;
        return nullptr;
    }
    x->hp.b = b;
    x->hp.hmax = (64 / b) < 32 ? (64 / b) : 32;
    x->hp.seed_mix = host_splitmix64(seed);
    if (cfg) {
        x->rebuild_policy = cfg->rebuild_policy;
        if (cfg->rebuild_threshold_pct) x->threshold_pct = cfg->rebuild_threshold_pct;
        if (cfg->smem_top_entries && cfg->smem_top_entries < kSmemTopMax) x->smem_top = cfg->smem_top_entries;
        x->test_flags = cfg->test_flags;
        if (cfg_full) {
            const uint32_t sp = cfg->sort_passes;
            if (sp > 8 || (sp > 4 && sp < 8)) {
                g_last_error = PI_ERR_INVALID_ARG;
                delete x;
                return nullptr;
            }
            x->sort_cfg = sp;
            if (cfg->small_batches > 1) {
                g_last_error = PI_ERR_INVALID_ARG;
                delete x;
                return nullptr;
            }
            x->small_mode = cfg->small_batches;
        }
    }
    // Lowest index level: the lowest l whose expected storage gap 2^(b (l - 1)) is at
    // least 32 nodes, unless the caller picks one. The storage search interpolates within
    // the gap, so a wide gap costs about one 64-byte line, while every built level costs
    // rebuild work and a descent step; the autotuner measured level 4 fastest at P = 1/4
    // (64-node gaps) for indices of 2^24 to 2^27 keys.
    x->min_lb = 2;
    while ((uint32_t)b * (x->min_lb - 1) < 5u) ++x->min_lb;
    if (cfg && cfg->lowest_level) {
        if (cfg->lowest_level < 2 || cfg->lowest_level > 16) {
            g_last_error = PI_ERR_INVALID_ARG;
            delete x;
            return nullptr;
        }
        x->min_lb = cfg->lowest_level;
    }
    uint64_t st_cap = n + (n / 2 > kMinStorage ? n / 2 : kMinStorage);
    if (cfg && cfg->storage_capacity > st_cap) st_cap = cfg->storage_capacity;
    if (st_cap > PI_MAX_KEYS) st_cap = PI_MAX_KEYS;

    cudaStream_t s = nullptr;
    Scratch tmp{};
    int rc = PI_OK;
    do {
        if ((e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)) != cudaSuccess) break;
        for (auto& ev : x->ev)
            if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) break;
        if (e != cudaSuccess) break;
        if ((e = cudaMallocHost(reinterpret_cast<void**>(&x->h_mbox), kRing * sizeof(DevMeta))) != cudaSuccess) break;
        if ((e = dalloc(&x->d_meta, 1)) != cudaSuccess) break;
        if ((e = dalloc(&x->d_bm, 2)) != cudaSuccess) break;
        if ((e = cudaStreamCreateWithFlags(&x->rs, cudaStreamNonBlocking)) != cudaSuccess) break;
        if ((e = cudaEventCreateWithFlags(&x->ev_applied, cudaEventDisableTiming)) != cudaSuccess) break;
        if ((e = cudaEventCreateWithFlags(&x->ev_rebuilt, cudaEventDisableTiming)) != cudaSuccess) break;
        if ((e = cudaEventCreateWithFlags(&x->ev_last, cudaEventDisableTiming)) != cudaSuccess) break;
        if ((e = dalloc(&x->d_dofs, 8 * 256)) != cudaSuccess) break;
        if ((e = dalloc(&x->d_count, 1)) != cudaSuccess) break;
        cudaMemsetAsync(x->d_meta, 0, sizeof(DevMeta), s);
        cudaMemsetAsync(x->d_bm, 0, 2 * sizeof(BatchMeta), s);
        if ((e = alloc_storage(x->st, st_cap)) != cudaSuccess) break;
        x->st_cap = st_cap;
        if ((e = ensure_tile_cnt(x, st_cap)) != cudaSuccess) break;
        if ((e = ensure_wcount(x, st_cap)) != cudaSuccess) break;
        if ((e = ensure_desc(x, desc_need(n, st_cap))) != cudaSuccess) break;
        // 1. sort (key, arrival) and keep the last of every key run
        if (n > 0) {
            if ((e = alloc_scratch(tmp, n)) != cudaSuccess) break;
            SortBuffers sb = sort_buffers(x, tmp);
            uint32_t ep = next_epochs(x, 16, s);
            if ((e = launch_sort(nullptr, keys, (uint32_t)n, sb, x->d_bm, &x->d_meta->error, s, x->num_sms, 8)) !=
                cudaSuccess)
                break;
            x->epoch = ep;
            BatchMeta hbm;
            if ((e = cudaMemcpyAsync(&hbm, x->d_bm, sizeof(BatchMeta), cudaMemcpyDeviceToHost, s)) != cudaSuccess) break;
            if ((e = cudaStreamSynchronize(s)) != cudaSuccess) break;
            if (hbm.invalid) {
                rc = PI_ERR_INVALID_ARG;
                break;
            }
            CreateArgs ca{};
            ca.sk = tmp.a_k;
            ca.sp = tmp.a_p;
            ca.uvals = values;
            ca.n = (uint32_t)n;
            ca.st = x->st;
            ca.m = x->d_meta;
            ca.bm = x->d_bm;
            ca.desc = x->desc;
            ca.hp = x->hp;
            ca.st_cap = (uint32_t)x->st_cap;
            ca.err = &x->d_meta->error;
            ep = next_epochs(x, 4, s);
            if ((e = launch_create_storage(ca, ep, s, x->num_sms)) != cudaSuccess) break;
            x->epoch = ep;
        }
        DevMeta hm;
        if ((e = read_meta(x, s, &hm)) != cudaSuccess) break;
        uint64_t need = 0;
        for (int l = 2; l < kLevelSlots; ++l)
            if (hm.cnt[l]) need += (uint64_t)hm.cnt[l] + 1;
        uint64_t icap = need + need / 4 + 4096;
        if (cfg && cfg->index_capacity) icap = cfg->index_capacity;
        if ((e = dalloc(&x->lkeys, icap + kPad)) != cudaSuccess) break;
        if ((e = dalloc(&x->ldown, icap + kPad)) != cudaSuccess) break;
        if ((e = dalloc(&x->lkeys1, icap + kPad)) != cudaSuccess) break;
        if ((e = dalloc(&x->ldown1, icap + kPad)) != cudaSuccess) break;
        x->idx_cap = icap;
        // 2. lay out and build the index layer
        cudaMemsetAsync(x->d_bm, 0, sizeof(BatchMeta), s);
        RebuildArgs ra = rebuild_args(x, x->d_bm, (uint32_t)hm.size, 2u);
        uint32_t ep = next_epochs(x, 4, s);
        if ((e = launch_merge(ra, ep, s, x->num_sms)) != cudaSuccess) break;
        if ((e = launch_level_bases(ra, s)) != cudaSuccess) break;
        if ((e = launch_rebuild(ra, ep, s, x->num_sms)) != cudaSuccess) break;
        x->epoch = ep;
        if ((e = read_meta(x, s, &x->known)) != cudaSuccess) break;
        x->force_rebuild = false;
        if (x->known.error) {
            rc = sticky_error(x->known);
            break;
        }
    } while (0);
    free_scratch(tmp);
    if (s) {
        cudaStreamSynchronize(s);
        cudaStreamDestroy(s);
    }
    if (rc == PI_OK && e != cudaSuccess) rc = map_cuda(e);
    if (rc != PI_OK) {
        g_last_error = rc;
        destroy(x);
        return nullptr;
    }
    return x;
}

pi_index_t* pi_create(const uint64_t* keys, const uint64_t* values, uint64_t n, double promote_p,
                      uint64_t seed) {
    return pi_create_ex(keys, values, n, promote_p, seed, nullptr);
}

int pi_execute_batch(pi_index_t* x, const uint8_t* ops, const uint64_t* keys, const uint64_t* values,
                     uint64_t n, pi_result_t* results, pi_stream_t stream) {
    if (!x) return PI_ERR_INVALID_ARG;
    if (n == 0) return PI_OK;
    if (!ops || !keys || !values || !results || n > PI_MAX_BATCH) return PI_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e;
    order_after_last(x, s);
    refresh_known(x);
    if (int rc = sticky_error(x->known)) return rc;
    // capacities (grow rarely; growing synchronises the stream)
    if (n > x->sc.cap && (e = grow_scratch(x, n, s)) != cudaSuccess) return map_cuda(e);
    uint64_t size_ub = (uint64_t)x->known.size + x->pending_n + x->extra_n + n;
    if (size_ub > x->st_cap) {
        if ((e = sync_known(x, s)) != cudaSuccess) return map_cuda(e);
        if (int rc = sticky_error(x->known)) return rc;
        size_ub = (uint64_t)x->known.size + n;
        if (size_ub > PI_MAX_KEYS) return PI_ERR_INVALID_ARG;
        if (size_ub > x->st_cap && (e = grow_storage(x, size_ub, s)) != cudaSuccess) return map_cuda(e);
    }
    if (x->known.grow_request) {
        if ((e = sync_known(x, s)) != cudaSuccess) return map_cuda(e);
        if (x->known.grow_request && x->known.index_need + 64ull > x->idx_cap) {
            if ((e = grow_index(x, x->known.index_need, s)) != cudaSuccess) return map_cuda(e);
        }
        x->known.grow_request = 0;
    }
    if (small_route(x, n, size_ub)) {
        const int rc = execute_small(x, ops, keys, values, n, results, s);
        if (rc != kNoRoute) return rc;
        x->small_mode = 0;  // no cluster of the needed size fits this device: plain path
    }
    return enqueue_batch(x, x->sc, ops, keys, values, n, results, size_ub, s);
}

int pi_execute_batch_host(pi_index_t* x, const uint8_t* ops_host, const uint64_t* keys_host,
                          const uint64_t* values_host, uint64_t n, pi_result_t* results_host,
                          pi_stream_t stream) {
    if (!x) return PI_ERR_INVALID_ARG;
    if (n == 0) return PI_OK;
    if (!ops_host || !keys_host || !values_host || !results_host || n > PI_MAX_BATCH) return PI_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaSuccess;
    if (!x->hs) {  // first host-buffer call: the pipeline's streams and events
        for (cudaStream_t* p : {&x->hs, &x->cs, &x->ds})
            if (e == cudaSuccess) e = cudaStreamCreateWithFlags(p, cudaStreamNonBlocking);
        for (int k = 0; k < 2 && e == cudaSuccess; ++k)
            for (cudaEvent_t* p : {&x->ev_in[k], &x->ev_comp[k], &x->ev_out[k]})
                if (e == cudaSuccess) e = cudaEventCreateWithFlags(p, cudaEventDisableTiming);
        if (e != cudaSuccess) return map_cuda(e);
    }
    const int k = (int)(x->host_calls & 1u);
    Staging& g = x->stg[k];
    if (n > g.cap) {  // grow the slot (rare): wait until nothing uses it
        if ((e = cudaEventSynchronize(x->ev_comp[k])) != cudaSuccess ||
            (e = cudaEventSynchronize(x->ev_out[k])) != cudaSuccess)
            return map_cuda(e);
        dfree(g.ops); dfree(g.keys); dfree(g.vals); dfree(g.res);
        g.cap = 0;
        if ((e = dalloc(&g.ops, n)) != cudaSuccess || (e = dalloc(&g.keys, n)) != cudaSuccess ||
            (e = dalloc(&g.vals, n)) != cudaSuccess || (e = dalloc(&g.res, n)) != cudaSuccess) {
            dfree(g.ops); dfree(g.keys); dfree(g.vals); dfree(g.res);
            return map_cuda(e);
        }
        g.cap = n;
    }
    // copy in, once the batch that last read this slot's inputs has finished
    cudaStreamWaitEvent(x->hs, x->ev_comp[k], 0);
    cudaMemcpyAsync(g.ops, ops_host, n, cudaMemcpyHostToDevice, x->hs);
    cudaMemcpyAsync(g.keys, keys_host, n * 8, cudaMemcpyHostToDevice, x->hs);
    cudaMemcpyAsync(g.vals, values_host, n * 8, cudaMemcpyHostToDevice, x->hs);
    cudaEventRecord(x->ev_in[k], x->hs);
    // the batch, after the index's previous operation, its inputs, and the copy out of
    // the slot's previous results
    cudaStreamWaitEvent(x->cs, x->ev_in[k], 0);
    cudaStreamWaitEvent(x->cs, x->ev_out[k], 0);
    const int rc = pi_execute_batch(x, g.ops, g.keys, g.vals, n, g.res, reinterpret_cast<pi_stream_t>(x->cs));
    if (rc != PI_OK) return rc;
    cudaEventRecord(x->ev_comp[k], x->cs);
    // copy out; the caller's stream completes after it
    cudaStreamWaitEvent(x->ds, x->ev_comp[k], 0);
    cudaMemcpyAsync(results_host, g.res, n * sizeof(pi_result_t), cudaMemcpyDeviceToHost, x->ds);
    cudaEventRecord(x->ev_out[k], x->ds);
    e = cudaStreamWaitEvent(s, x->ev_out[k], 0);
    x->host_calls++;
    return map_cuda(e);
}

int pi_range_search(pi_index_t* x, const uint64_t* lo, const uint64_t* hi, uint64_t n, uint64_t* offsets,
                    uint64_t* keys_out, uint64_t* vals_out, uint64_t cap, pi_stream_t stream) {
    if (!x || !offsets) return PI_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (n == 0) return map_cuda(cudaMemsetAsync(offsets, 0, sizeof(uint64_t), s));
    if (!lo || !hi || n > PI_MAX_BATCH / 2 || (cap && (!keys_out || !vals_out))) return PI_ERR_INVALID_ARG;
    cudaError_t e;
    refresh_known(x);
    if (int rc = sticky_error(x->known)) return rc;
    order_after_last(x, s);
    const uint64_t nb = 2 * n;
    // sort and descent scratch for the 2n bounds (grows like a batch's)
    if (nb > x->sc.cap && (e = grow_scratch(x, nb, s)) != cudaSuccess) return map_cuda(e);
    if (n > x->r_cap) {
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return map_cuda(e);
        dfree(x->r_bounds); dfree(x->r_start); dfree(x->r_end); dfree(x->r_cnt); dfree(x->r_bsum);
        x->r_cap = 0;
        if ((e = dalloc(&x->r_bounds, nb)) != cudaSuccess || (e = dalloc(&x->r_start, n)) != cudaSuccess ||
            (e = dalloc(&x->r_end, n)) != cudaSuccess || (e = dalloc(&x->r_cnt, n)) != cudaSuccess ||
            (e = dalloc(&x->r_bsum, n / 256 + 2)) != cudaSuccess)
            return map_cuda(e);
        x->r_cap = n;
    }
    const uint64_t l0 = g_launches;
    cudaMemcpyAsync(x->r_bounds, lo, n * 8, cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(x->r_bounds + n, hi, n * 8, cudaMemcpyDeviceToDevice, s);
    BatchMeta* bm = x->d_bm + (x->issued & 1u);  // the other block may still be read by the rebuild
    cudaMemsetAsync(bm, 0, sizeof(BatchMeta), s);
    const Scratch& sc = x->sc;
    SortBuffers sb = sort_buffers(x, sc);
    if ((e = launch_sort(nullptr, x->r_bounds, (uint32_t)nb, sb, bm, &x->d_meta->error, s, x->num_sms,
                         sort_passes(x, nb))) != cudaSuccess)
        return map_cuda(e);
    wait_rebuild(x, s);
    DescendArgs da{};
    da.sk = sc.a_k;
    da.sp = sc.a_p;
    da.tile_pref = sc.tile_pref;
    da.sub_pref = sc.sub_pref;
    da.desc = x->desc;
    da.dq = sc.dq;
    da.dlo = sc.dlo;
    // the lowest buildable level is never walked by the prologue: the storage locate
    // searches it itself (it needs that level's gap ends)
    da.top_launched = std::max(top_launched_for(x), (int)x->min_lb);
    da.bottom_launched = (int)x->min_lb;
    da.m = x->d_meta;
    da.bm = bm;
    da.lkeys = x->lkeys;
    da.ldown = x->ldown;
    da.lkeys1 = x->lkeys1;
    da.ldown1 = x->ldown1;
    da.st = x->st;
    da.loc = sc.loc;
    da.flags = sc.flags;
    da.val0 = sc.val0;
    da.n = (uint32_t)nb;
    da.err = &x->d_meta->error;
    uint32_t ep = next_epochs(x, 4, s);
    e = launch_descend(da, ep, s, x->num_sms);
    x->epoch = ep;
    if (e != cudaSuccess) return map_cuda(e);
    RangeArgs ra{};
    ra.sk = sc.a_k;
    ra.sp = sc.a_p;
    ra.loc = sc.loc;
    ra.flags = sc.flags;
    ra.sub_pref = sc.sub_pref;
    ra.m = x->d_meta;
    ra.bm = bm;
    ra.st = x->st;
    ra.start = x->r_start;
    ra.end = x->r_end;
    ra.cnt = x->r_cnt;
    ra.bsum = x->r_bsum;
    ra.offsets = offsets;
    ra.keys_out = keys_out;
    ra.vals_out = vals_out;
    ra.cap = cap;
    ra.n = (uint32_t)n;
    ra.err = &x->d_meta->error;
    e = launch_range(ra, s);
    x->launches += g_launches - l0;
    if (e == cudaSuccess) mark_last(x, s);
    return map_cuda(e);
}

int pi_execute_batch_noalloc(pi_index_t* x, const uint8_t* ops, const uint64_t* keys, const uint64_t* values,
                             uint64_t n, pi_result_t* results, pi_stream_t stream) {
    if (!x) return PI_ERR_INVALID_ARG;
    if (n == 0) return PI_OK;
    if (!ops || !keys || !values || !results) return PI_ERR_INVALID_ARG;
    if (n > PI_NOALLOC_MAX_BATCH) return PI_ERR_INVALID_ARG;  // beyond the static scratch
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    NoAllocDevice* nd = nullptr;
    if ((e = noalloc_scratch_for(x->device, &nd)) != cudaSuccess) return map_cuda(e);
    Scratch sc{};
    if (carve_scratch(nd->ptr, PI_NOALLOC_MAX_BATCH, sc) != kNoAllocBytes) return PI_ERR_CUDA;
    order_after_last(x, s);
    refresh_known(x);
    if (int rc = sticky_error(x->known)) return rc;
    uint64_t size_ub = (uint64_t)x->known.size + x->pending_n + x->extra_n + n;
    if (size_ub > x->st_cap) {
        if ((e = sync_known(x, s)) != cudaSuccess) return map_cuda(e);
        if (int rc = sticky_error(x->known)) return rc;
        size_ub = (uint64_t)x->known.size + n;
        if (size_ub > x->st_cap) return PI_ERR_OOM;  // the storage layer would have to grow
    }
    // the previous call was on another index: its rebuild may still read the array
    if (nd->last && nd->last != x && (e = cudaStreamWaitEvent(s, nd->rebuilt, 0)) != cudaSuccess) return map_cuda(e);
    // An index layer that outgrew its capacity is not grown here: the rebuild then drops
    // its lowest levels and results stay exact.
    const int rc = enqueue_batch(x, sc, ops, keys, values, n, results, size_ub, s);
    if (rc == PI_OK) {
        if ((e = cudaEventRecord(nd->rebuilt, x->rs)) != cudaSuccess) return map_cuda(e);
        nd->last = x;
    }
    return rc;
}

void pi_destroy(pi_index_t* x) { destroy(x); }

int pi_flush(pi_index_t* x, pi_stream_t stream) {
    if (!x) return PI_ERR_INVALID_ARG;
    order_after_last(x, reinterpret_cast<cudaStream_t>(stream));
    wait_rebuild(x, reinterpret_cast<cudaStream_t>(stream));
    return map_cuda(cudaGetLastError());
}

int pi_profile(pi_index_t* x, int enable) {
    if (!x) return PI_ERR_INVALID_ARG;
    if (enable && !x->pev) {
        const size_t cnt = (size_t)kProfSlots * kProfEvents;
        x->pev = new (std::nothrow) cudaEvent_t[cnt];
        if (!x->pev) return PI_ERR_OOM;
        for (size_t i = 0; i < cnt; ++i) {
            if (cudaEventCreate(&x->pev[i]) != cudaSuccess) {
                for (size_t j = 0; j < i; ++j) cudaEventDestroy(x->pev[j]);
                delete[] x->pev;
                x->pev = nullptr;
                return PI_ERR_CUDA;
            }
        }
    }
    if (x->pused) prof_fold(x);
    x->prof = enable != 0;
    delete x->kt;  // level 2: per-kernel times as well
    x->kt = nullptr;
    if (enable == 2) {
        x->kt = new (std::nothrow) KernelTimes();
        if (!x->kt) return PI_ERR_OOM;
    }
    for (int st = 0; st < PI_NUM_STAGES; ++st) x->pms[st] = 0.0;
    x->pbatches = 0;
    return PI_OK;
}

int pi_profile_read(pi_index_t* x, double* stage_ms_host, uint64_t* batches_host, pi_stream_t stream) {
    if (!x || !stage_ms_host || !batches_host) return PI_ERR_INVALID_ARG;
    order_after_last(x, reinterpret_cast<cudaStream_t>(stream));
    wait_rebuild(x, reinterpret_cast<cudaStream_t>(stream));
    cudaError_t e = cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return map_cuda(e);
    prof_fold(x);
    for (int st = 0; st < PI_NUM_STAGES; ++st) stage_ms_host[st] = x->pms[st];
    *batches_host = x->pbatches;
    return PI_OK;
}

int pi_profile_kernels(pi_index_t* x, char* buf, uint64_t cap, pi_stream_t stream) {
    if (!x || (cap && !buf)) return PI_ERR_INVALID_ARG;
    if (!x->kt) return PI_ERR_INVALID_ARG;
    order_after_last(x, reinterpret_cast<cudaStream_t>(stream));
    wait_rebuild(x, reinterpret_cast<cudaStream_t>(stream));
    cudaError_t e = cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return map_cuda(e);
    x->kt->fold();
    std::string out;
    for (const auto& k : x->kt->acc) {
        const char* name = nullptr;
        if (cudaFuncGetName(&name, k.first) != cudaSuccess || !name) name = "?";
        char line[64];
        std::snprintf(line, sizeof(line), "\t%llu\t%.6f\n", (unsigned long long)k.second.second, k.second.first);
        out += name;
        out += line;
    }
    if (cap) {
        const size_t c = std::min<size_t>(out.size(), cap - 1);
        std::memcpy(buf, out.data(), c);
        buf[c] = 0;
    }
    return (int)std::min<size_t>(out.size() + 1, 0x7FFFFFFF);
}

int pi_status(pi_index_t* x, pi_stream_t stream) {
    if (!x) return PI_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = sync_known(x, s);
    if (e != cudaSuccess) return map_cuda(e);
    return sticky_error(x->known);
}

int pi_info(pi_index_t* x, pi_info_t* out, pi_stream_t stream) {
    if (!x || !out) return PI_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = sync_known(x, s);
    if (e != cudaSuccess) return map_cuda(e);
    const DevMeta& m = x->known;
    std::memset(out, 0, sizeof(*out));
    out->size = m.size;
    out->live = m.cnt[1];
    out->tombstones = m.tombs;
    out->top_level = m.H;
    out->bottom_built = m.Lb;
    out->smem_low_level = m.Ls;
    out->promote_shift = (uint32_t)x->hp.b;
    for (int l = 1; l < kLevelSlots; ++l) out->level_size[l] = m.cnt[l];
    out->storage_capacity = x->st_cap;
    out->index_capacity = x->idx_cap;
    out->batches = m.batches;
    out->rebuilds = m.rebuilds;
    out->kernel_launches = x->launches;
    out->incremental_rebuilds = m.inc_rebuilds;
    out->owner_checked_writes = m.owner_writes;
    out->routed_batches = x->routed;
    return sticky_error(m);
}

void pi_test_fail_allocations(uint32_t count) { g_fail_allocs = count; }

int pi_selftest_wait(uint32_t* err_word_host, pi_stream_t stream) {
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    uint64_t* desc = nullptr;
    uint32_t* err = nullptr;
    cudaError_t e = dalloc(&desc, 64);
    if (e == cudaSuccess) e = dalloc(&err, 1);
    uint32_t w = 0;
    if (e == cudaSuccess) e = cudaMemsetAsync(desc, 0, 64 * sizeof(uint64_t), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(uint32_t), s);
    if (e == cudaSuccess) e = launch_wait_selftest(desc, err, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&w, err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    dfree(desc);
    dfree(err);
    if (e != cudaSuccess) return map_cuda(e);
    if (err_word_host) *err_word_host = w;
    if (w & kErrTimeout) return PI_ERR_TIMEOUT;
    return w ? PI_ERR_CUDA : PI_OK;
}

int pi_size(pi_index_t* x, uint64_t* out, pi_stream_t stream) {
    if (!x || !out) return PI_ERR_INVALID_ARG;
    cudaError_t e = sync_known(x, reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return map_cuda(e);
    *out = x->known.cnt[1];
    return sticky_error(x->known);
}

int pi_num_levels(pi_index_t* x, pi_stream_t stream) {
    if (!x) return PI_ERR_INVALID_ARG;
    cudaError_t e = sync_known(x, reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return map_cuda(e);
    if (int rc = sticky_error(x->known)) return rc;
    return (int)x->known.H;
}

int pi_export(pi_index_t* x, uint64_t* keys_out, uint64_t* vals_out, uint64_t cap, uint64_t* n_out_host,
              pi_stream_t stream) {
    if (!x || !n_out_host || (cap > 0 && (!keys_out || !vals_out))) return PI_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = sync_known(x, s);
    if (e != cudaSuccess) return map_cuda(e);
    if (int rc = sticky_error(x->known)) return rc;
    cudaMemsetAsync(x->d_count, 0, sizeof(uint32_t), s);
    cudaMemsetAsync(&x->d_bm->tile_ctr[12], 0, sizeof(uint32_t), s);
    uint32_t ep = next_epochs(x, 2, s);
    e = launch_export_live(x->st, x->d_meta, keys_out, vals_out, cap, x->d_count, x->desc, &x->d_bm->tile_ctr[12], ep,
                           &x->d_meta->error, s, x->num_sms, x->known.size);
    x->epoch = ep;
    if (e != cudaSuccess) return map_cuda(e);
    uint32_t c = 0;
    e = cudaMemcpyAsync(&c, x->d_count, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return map_cuda(e);
    *n_out_host = c;
    return PI_OK;
}

int pi_export_storage(pi_index_t* x, uint64_t* keys_out, uint8_t* meta_out, uint64_t cap, uint64_t* n_out_host,
                      pi_stream_t stream) {
    if (!x || !n_out_host || (cap > 0 && !keys_out)) return PI_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = sync_known(x, s);
    if (e != cudaSuccess) return map_cuda(e);
    if (int rc = sticky_error(x->known)) return rc;
    const DevMeta& m = x->known;
    *n_out_host = m.size;
    const uint64_t c = m.size < cap ? m.size : cap;
    if (c) {
        cudaMemcpyAsync(keys_out, x->st.keys[m.cur], c * 8, cudaMemcpyDeviceToDevice, s);
        if (meta_out) cudaMemcpyAsync(meta_out, x->st.meta[m.cur], c, cudaMemcpyDeviceToDevice, s);
    }
    return map_cuda(cudaStreamSynchronize(s));
}

int pi_export_level(pi_index_t* x, int level, uint64_t* keys_out, uint32_t* down_out, uint64_t cap,
                    uint64_t* n_out_host, pi_stream_t stream) {
    if (!x || !n_out_host || level < 2 || level >= kLevelSlots || (cap > 0 && !keys_out)) return PI_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = sync_known(x, s);
    if (e != cudaSuccess) return map_cuda(e);
    const DevMeta& m = x->known;
    if ((uint32_t)level > m.H) {
        *n_out_host = 0;
        return PI_OK;
    }
    if ((uint32_t)level < m.Lb) {
        *n_out_host = 0;
        return PI_ERR_NOT_BUILT;
    }
    const uint64_t cnt = m.n[level];
    *n_out_host = cnt;
    const uint64_t c = cnt < cap ? cnt : cap;
    if (c) {
        const uint64_t* lk = m.lcur ? x->lkeys1 : x->lkeys;
        const uint32_t* ld = m.lcur ? x->ldown1 : x->ldown;
        cudaMemcpyAsync(keys_out, lk + m.base[level], c * 8, cudaMemcpyDeviceToDevice, s);
        if (down_out) cudaMemcpyAsync(down_out, ld + m.base[level], c * 4, cudaMemcpyDeviceToDevice, s);
    }
    e = cudaStreamSynchronize(s);
    return map_cuda(e);
}


// ---------------------------------------------------------------------------------
// Batching form (host side). The queue buffer holds, per class, the number of items
// and the next-item counter, then one slice of `count` items per class; it is filled
// on the host (pinned, one buffer per call parity) and copied in by the graph's first
// node. One CUDA graph per parity: copy -> one persistent kernel per size class on
// parallel branches.

}  // extern "C"

struct pi_multi {
    int device = 0;
    int num_sms = 0;
    std::vector<pi_index*> idx;
    std::vector<MIndex> h_idx;
    pi_multi_config_t cfg{};
    MIndex* d_idx = nullptr;
    DevMeta* d_mirror = nullptr;
    uint8_t* d_q = nullptr;
    uint8_t* h_q[2] = {};
    uint64_t q_bytes = 0;
    cudaEvent_t q_free[2] = {};
    uint64_t calls = 0;
    uint64_t launches = 0;  // kernels per graph launch
    uint32_t grid[PI_MULTI_MAX_CLASSES] = {};
    uint32_t qcap[PI_MULTI_MAX_CLASSES] = {};
    uint8_t* scratch[PI_MULTI_MAX_CLASSES] = {};
    uint64_t stride[PI_MULTI_MAX_CLASSES] = {};
    cudaStream_t cs = nullptr;
    cudaStream_t ls[PI_MULTI_MAX_CLASSES] = {};
    cudaEvent_t evf = nullptr;
    cudaEvent_t evj[PI_MULTI_MAX_CLASSES] = {};
    cudaEvent_t ev_done = nullptr;  // end of the last call: the indices' last operation
    cudaGraphExec_t gx[2] = {};
    bool graph_valid = false;
};

namespace {

constexpr uint64_t kQHeader = 64;  // counts[PI_MULTI_MAX_CLASSES], heads[PI_MULTI_MAX_CLASSES], pad

MIndex mindex_of(const pi_index* x) {
    MIndex mi{};
    mi.m = x->d_meta;
    mi.st = x->st;
    mi.lkeys = x->lkeys;
    mi.ldown = x->ldown;
    mi.lkeys1 = x->lkeys1;
    mi.ldown1 = x->ldown1;
    mi.st_cap = (uint32_t)x->st_cap;
    mi.idx_cap = (uint32_t)(x->idx_cap > 0xFFFFFFF0ull ? 0xFFFFFFF0ull : x->idx_cap);
    mi.smem_top = x->smem_top;
    mi.min_lb = x->min_lb;
    mi.hp = x->hp;
    return mi;
}

void multi_free_graphs(pi_multi* mx) {
    for (auto& g : mx->gx)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
    mx->graph_valid = false;
}

void multi_destroy(pi_multi* mx) {
    if (!mx) return;
    cudaSetDevice(mx->device);
    for (int p = 0; p < 2; ++p)
        if (mx->q_free[p]) cudaEventSynchronize(mx->q_free[p]);
    for (pi_index* x : mx->idx)  // the calls are complete: forget the set's event
        if (x->last_ev == mx->ev_done) x->has_last = false;
    if (mx->ev_done) cudaEventDestroy(mx->ev_done);
    multi_free_graphs(mx);
    dfree(mx->d_idx);
    dfree(mx->d_mirror);
    dfree(mx->d_q);
    for (auto& h : mx->h_q)
        if (h) cudaFreeHost(h);
    for (auto& sc : mx->scratch) dfree(sc);
    for (auto& e : mx->q_free)
        if (e) cudaEventDestroy(e);
    for (auto& e : mx->evj)
        if (e) cudaEventDestroy(e);
    if (mx->evf) cudaEventDestroy(mx->evf);
    for (auto& st : mx->ls)
        if (st) cudaStreamDestroy(st);
    if (mx->cs) cudaStreamDestroy(mx->cs);
    delete mx;
}

int class_of(const pi_multi* mx, uint64_t nodes) {
    uint32_t lg = 0;
    while (lg < 63 && (1ull << lg) < nodes) ++lg;
    for (uint32_t c = 0; c + 1 < mx->cfg.num_classes; ++c)
        if (lg <= mx->cfg.cls[c].max_log2_size) return (int)c;
    return (int)mx->cfg.num_classes - 1;
}

cudaError_t multi_build_graphs(pi_multi* mx) {
    multi_free_graphs(mx);
    const uint32_t count = (uint32_t)mx->idx.size();
    uint64_t launches = 0;
    for (int p = 0; p < 2; ++p) {
        const uint64_t l0 = g_launches;
        cudaError_t e = cudaStreamBeginCapture(mx->cs, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return e;
        cudaMemcpyAsync(mx->d_q, mx->h_q[p], mx->q_bytes, cudaMemcpyHostToDevice, mx->cs);
        cudaEventRecord(mx->evf, mx->cs);
        const uint32_t* counts = reinterpret_cast<const uint32_t*>(mx->d_q);
        uint32_t* heads = reinterpret_cast<uint32_t*>(mx->d_q) + PI_MULTI_MAX_CLASSES;
        const MItem* items = reinterpret_cast<const MItem*>(mx->d_q + kQHeader);
        cudaError_t le = cudaSuccess;
        for (uint32_t c = 0; c < mx->cfg.num_classes; ++c) {
            if (!mx->grid[c] || !mx->qcap[c]) continue;
            cudaStreamWaitEvent(mx->ls[c], mx->evf, 0);
            MultiArgs a{};
            a.idx = mx->d_idx;
            a.items = items + (uint64_t)c * count;  // class c's slice of the queue
            a.nitems = counts + c;
            a.head = heads + c;
            a.scratch = mx->scratch[c];
            a.stride = mx->stride[c];
            a.qcap = mx->qcap[c];
            a.mirror = mx->d_mirror;
            const pi_multi_class_t& q = mx->cfg.cls[c];
            cudaError_t r =
                launch_multi(a, (int)q.warps, (int)q.radix_bits, (int)q.cluster, mx->grid[c], mx->ls[c]);
            if (r != cudaSuccess && le == cudaSuccess) le = r;
            cudaEventRecord(mx->evj[c], mx->ls[c]);
            cudaStreamWaitEvent(mx->cs, mx->evj[c], 0);
        }
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(mx->cs, &g);
        if (e == cudaSuccess && le != cudaSuccess) e = le;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&mx->gx[p], g, 0);
        if (g) cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            multi_free_graphs(mx);
            return e;
        }
        launches = g_launches - l0;
    }
    g_launches -= 2 * launches;  // counted per graph launch instead
    mx->launches = launches;
    mx->graph_valid = true;
    return cudaSuccess;
}

}  // namespace

extern "C" {

pi_multi_t* pi_multi_create(pi_index_t* const* indices, uint32_t count, const pi_multi_config_t* cfg) {
    g_last_error = PI_OK;
    if (!indices || count == 0) {
        g_last_error = PI_ERR_INVALID_ARG;
        return nullptr;
    }
    pi_multi_config_t c{};
    if (cfg) {
        if (cfg->struct_size != sizeof(pi_multi_config_t) || cfg->num_classes < 1 ||
            cfg->num_classes > PI_MULTI_MAX_CLASSES) {
            g_last_error = PI_ERR_INVALID_ARG;
            return nullptr;
        }
        c = *cfg;
        for (uint32_t k = 0; k < c.num_classes; ++k) {
            const pi_multi_class_t& q = c.cls[k];
            const bool ok = multi_variant_ok((int)q.warps, (int)q.radix_bits, (int)q.cluster) &&
                            (k == 0 || q.max_log2_size > c.cls[k - 1].max_log2_size);
            if (!ok) {
                g_last_error = PI_ERR_INVALID_ARG;
                return nullptr;
            }
        }
    } else {
        c.struct_size = sizeof(c);
        c.num_classes = 3;
        c.cls[0] = {14, 8, 4, 0};
        c.cls[1] = {17, 16, 8, 0};
        c.cls[2] = {32, 32, 8, 0};
    }
    std::vector<pi_index*> v(indices, indices + count);
    {
        std::vector<pi_index*> sorted = v;
        std::sort(sorted.begin(), sorted.end());
        if (sorted[0] == nullptr || std::adjacent_find(sorted.begin(), sorted.end()) != sorted.end()) {
            g_last_error = PI_ERR_INVALID_ARG;
            return nullptr;
        }
    }
    for (auto* x : v)
        if (x->device != v[0]->device) {
            g_last_error = PI_ERR_INVALID_ARG;
            return nullptr;
        }
    pi_multi* mx = new (std::nothrow) pi_multi();
    if (!mx) {
        g_last_error = PI_ERR_OOM;
        return nullptr;
    }
    mx->device = v[0]->device;
    mx->num_sms = v[0]->num_sms;
    mx->idx = v;
    mx->cfg = c;
    cudaSetDevice(mx->device);
    cudaError_t e = cudaSuccess;
    do {
        for (auto* x : v) mx->h_idx.push_back(mindex_of(x));
        if ((e = dalloc(&mx->d_idx, count)) != cudaSuccess) break;
        if ((e = cudaMemcpy(mx->d_idx, mx->h_idx.data(), count * sizeof(MIndex), cudaMemcpyHostToDevice)) !=
            cudaSuccess)
            break;
        if ((e = dalloc(&mx->d_mirror, count)) != cudaSuccess) break;
        mx->q_bytes = kQHeader + (uint64_t)PI_MULTI_MAX_CLASSES * count * sizeof(MItem);
        if ((e = dalloc(&mx->d_q, mx->q_bytes)) != cudaSuccess) break;
        for (int p = 0; p < 2; ++p) {
            if ((e = cudaMallocHost(reinterpret_cast<void**>(&mx->h_q[p]), mx->q_bytes)) != cudaSuccess) break;
            std::memset(mx->h_q[p], 0, mx->q_bytes);
            if ((e = cudaEventCreateWithFlags(&mx->q_free[p], cudaEventDisableTiming)) != cudaSuccess) break;
        }
        if (e != cudaSuccess) break;
        if ((e = cudaStreamCreateWithFlags(&mx->cs, cudaStreamNonBlocking)) != cudaSuccess) break;
        if ((e = cudaEventCreateWithFlags(&mx->evf, cudaEventDisableTiming)) != cudaSuccess) break;
        if ((e = cudaEventCreateWithFlags(&mx->ev_done, cudaEventDisableTiming)) != cudaSuccess) break;
        for (uint32_t k = 0; k < c.num_classes && e == cudaSuccess; ++k) {
            e = cudaStreamCreateWithFlags(&mx->ls[k], cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&mx->evj[k], cudaEventDisableTiming);
            const pi_multi_class_t& q = c.cls[k];
            const uint32_t per = q.cluster > 1 ? q.cluster : 1u;  // CTAs per batch
            uint32_t slots = 0;
            if (e == cudaSuccess) e = multi_grid((int)q.warps, (int)q.radix_bits, (int)q.cluster, mx->num_sms, &slots);
            if (e == cudaSuccess && slots < per) e = cudaErrorInvalidConfiguration;
            // no more batch slots (CTAs or clusters) than indices in the set
            const uint64_t units = std::min<uint64_t>(slots / per, count);
            mx->grid[k] = (uint32_t)(units * per);
        }
    } while (0);
    if (e != cudaSuccess) {
        g_last_error = map_cuda(e);
        multi_destroy(mx);
        return nullptr;
    }
    return mx;
}

}  // extern "C"

namespace {
int multi_execute(pi_multi* mx, const pi_multi_batch_t* b, uint32_t nb, cudaStream_t s, pi_index* single);
}  // namespace

extern "C" {

int pi_multi_execute(pi_multi_t* mx, const pi_multi_batch_t* b, uint32_t nb, pi_stream_t stream) {
    if (!mx) return PI_ERR_INVALID_ARG;
    return multi_execute(mx, b, nb, reinterpret_cast<cudaStream_t>(stream), nullptr);
}

uint64_t pi_multi_kernels_per_call(const pi_multi_t* mx) { return mx ? mx->launches : 0; }

void pi_multi_destroy(pi_multi_t* mx) { multi_destroy(mx); }

}  // extern "C"

namespace {

// One call of a batching set. `single`: the set is an index's small-batch route, and the
// call is that index's batch for pi_execute_batch, which has already checked the
// capacities; its bookkeeping is then a plain batch's (the mailbox ring and the index's
// last-operation event) so the host's view of the sizes stays current without a sync.
int multi_execute(pi_multi* mx, const pi_multi_batch_t* b, uint32_t nb, cudaStream_t s, pi_index* single) {
    if (nb == 0) return PI_OK;
    const uint32_t count = (uint32_t)mx->idx.size();
    if (!b || nb > count) return PI_ERR_INVALID_ARG;
    cudaSetDevice(mx->device);
    std::vector<uint8_t> seen(count, 0);
    for (uint32_t i = 0; i < nb; ++i) {
        const pi_multi_batch_t& q = b[i];
        if (q.index >= count || seen[q.index] || q.n > PI_MULTI_MAX_BATCH) return PI_ERR_INVALID_ARG;
        if (q.n && (!q.ops || !q.keys || !q.values || !q.results)) return PI_ERR_INVALID_ARG;
        seen[q.index] = 1;
    }
    cudaError_t e;
    // Capacities: every index must hold its batch's new keys without growing in the
    // kernel. Growing (rare) synchronises the stream, as in pi_execute_batch.
    bool idx_changed = false;
    for (uint32_t i = 0; i < nb; ++i) {
        pi_index* x = mx->idx[b[i].index];
        refresh_known(x);
        if (int rc = sticky_error(x->known)) return rc;
        const uint64_t n = b[i].n;
        uint64_t size_ub = (uint64_t)x->known.size + x->pending_n + x->extra_n + n;
        bool grew = false;
        if (size_ub > x->st_cap || x->known.grow_request) {
            if ((e = sync_known(x, s)) != cudaSuccess) return map_cuda(e);
            if (int rc = sticky_error(x->known)) return rc;
            size_ub = (uint64_t)x->known.size + n;
            if (size_ub > PI_MAX_KEYS) return PI_ERR_INVALID_ARG;
            if (size_ub > x->st_cap) {
                if ((e = grow_storage(x, size_ub, s)) != cudaSuccess) return map_cuda(e);
                grew = true;
            }
            if (x->known.grow_request && x->known.index_need + 64ull > x->idx_cap) {
                if ((e = grow_index(x, x->known.index_need, s)) != cudaSuccess) return map_cuda(e);
                grew = true;
            }
            x->known.grow_request = 0;
        }
        (void)grew;
        // The single-index path may have grown this index's arrays since the set last
        // looked (a plain batch with new keys): the device table must hold the arrays in
        // use, never freed ones.
        order_after_last(x, s);
        const MIndex now = mindex_of(x);
        if (std::memcmp(&now, &mx->h_idx[b[i].index], sizeof(MIndex)) != 0) {
            mx->h_idx[b[i].index] = now;
            idx_changed = true;
        }
        wait_rebuild(x, s);
    }
    if (idx_changed &&
        (e = cudaMemcpyAsync(mx->d_idx, mx->h_idx.data(), mx->h_idx.size() * sizeof(MIndex),
                             cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return map_cuda(e);
    // the queue: per class, largest estimated work first (longest-processing-time order)
    std::vector<std::vector<std::pair<uint64_t, uint32_t>>> per(mx->cfg.num_classes);
    uint32_t need_q[PI_MULTI_MAX_CLASSES] = {};
    for (uint32_t i = 0; i < nb; ++i) {
        if (b[i].n == 0) continue;
        const pi_index* x = mx->idx[b[i].index];
        const uint64_t nodes = (uint64_t)x->known.size + x->pending_n + x->extra_n;
        const int c = class_of(mx, nodes);
        per[c].push_back({nodes + 8 * b[i].n, i});
        if (b[i].n > need_q[c]) need_q[c] = (uint32_t)b[i].n;
    }
    bool rebuild_graphs = !mx->graph_valid;
    for (uint32_t c = 0; c < mx->cfg.num_classes; ++c) {
        if (need_q[c] <= mx->qcap[c] || !mx->grid[c]) continue;
        // grow the class's scratch (rare): wait for the calls that may still use it
        for (int p = 0; p < 2; ++p) cudaEventSynchronize(mx->q_free[p]);
        uint32_t q = mx->qcap[c] ? mx->qcap[c] : 4096u;
        while (q < need_q[c]) q *= 2;
        dfree(mx->scratch[c]);
        mx->qcap[c] = 0;
        mx->stride[c] = multi_scratch_bytes(q);
        const uint32_t units = mx->grid[c] / (mx->cfg.cls[c].cluster > 1 ? mx->cfg.cls[c].cluster : 1u);
        if ((e = dalloc(&mx->scratch[c], mx->stride[c] * units)) != cudaSuccess) {
            mx->graph_valid = false;
            return map_cuda(e);
        }
        mx->qcap[c] = q;
        rebuild_graphs = true;
    }
    if (rebuild_graphs && (e = multi_build_graphs(mx)) != cudaSuccess) return map_cuda(e);
    const int p = (int)(mx->calls & 1u);
    if ((e = cudaEventSynchronize(mx->q_free[p])) != cudaSuccess) return map_cuda(e);
    uint32_t* hdr = reinterpret_cast<uint32_t*>(mx->h_q[p]);
    MItem* items = reinterpret_cast<MItem*>(mx->h_q[p] + kQHeader);
    for (uint32_t c = 0; c < PI_MULTI_MAX_CLASSES; ++c) {
        hdr[c] = 0;                         // items of class c
        hdr[PI_MULTI_MAX_CLASSES + c] = 0;  // its next-item counter
    }
    for (uint32_t c = 0; c < mx->cfg.num_classes; ++c) {
        auto& L = per[c];
        std::sort(L.begin(), L.end(), [](const auto& u, const auto& w) { return u.first > w.first; });
        hdr[c] = (uint32_t)L.size();
        MItem* slice = items + (uint64_t)c * count;
        for (size_t k = 0; k < L.size(); ++k) {
            const pi_multi_batch_t& q = b[L[k].second];
            MItem& it = slice[k];
            it.ops = q.ops;
            it.keys = q.keys;
            it.vals = q.values;
            it.results = q.results;
            it.n = (uint32_t)q.n;
            it.index = q.index;
        }
    }
    if ((e = cudaGraphLaunch(mx->gx[p], s)) != cudaSuccess) return map_cuda(e);
    if ((e = cudaEventRecord(mx->q_free[p], s)) != cudaSuccess) return map_cuda(e);
    mx->calls++;
    g_launches += mx->launches;
    if (single) {
        pi_index* x = single;
        const uint64_t slot = x->issued % kRing;
        if (x->issued - x->seen >= kRing) {  // the slot is still unread: wait for its batch
            cudaEventSynchronize(x->ev[slot]);
            refresh_known(x);
        }
        cudaMemcpyAsync(&x->h_mbox[slot], x->d_meta, sizeof(DevMeta), cudaMemcpyDeviceToHost, s);
        cudaEventRecord(x->ev[slot], s);
        x->ring_n[slot] = b[0].n;
        x->issued++;
        x->pending_n += b[0].n;
        x->force_rebuild = true;  // the plain path recounts its per-tile level counts
        x->launches += mx->launches;
        x->routed++;
        mark_last(x, s);
        return map_cuda(cudaGetLastError());
    }
    for (uint32_t i = 0; i < nb; ++i) {
        pi_index* x = mx->idx[b[i].index];
        x->extra_n += b[i].n;
        x->force_rebuild = true;  // the plain path recounts its per-tile level counts
        x->last_ev = mx->ev_done;  // recorded once for the call, below
        x->last_stream = s;
        x->has_last = true;
    }
    cudaEventRecord(mx->ev_done, s);
    return PI_OK;
}

constexpr uint64_t kSmallBatch = 1ull << 16;  // queries
constexpr uint64_t kSmallIndex = 1ull << 20;  // storage nodes, the batch's new keys included

bool small_route(const pi_index* x, uint64_t n, uint64_t size_ub) {
    return x->small_mode == 1 && n <= kSmallBatch && size_ub <= kSmallIndex && !x->prof && !x->kt &&
           x->test_flags == 0 && x->rebuild_policy == 0;
}

// A small batch as a one-item batching-form call on a thread-block cluster of 16 CTAs of
// 16 warps (8 CTAs where 16 do not fit; 16-warp CTAs keep the pipeline's registers
// unspilled). Returns kNoRoute when no cluster size fits this device.
int execute_small(pi_index* x, const uint8_t* ops, const uint64_t* keys, const uint64_t* values, uint64_t n,
                  pi_result_t* results, cudaStream_t s) {
    if (!x->small) {
        const int saved = g_last_error;  // an internal set: pi_last_error stays the caller's
        for (uint32_t cl : {16u, 8u}) {
            pi_multi_config_t c{};
            c.struct_size = sizeof(c);
            c.num_classes = 1;
            c.cls[0] = {32, 16, 8, cl};
            pi_index_t* one = x;
            x->small = pi_multi_create(&one, 1, &c);
            if (x->small) break;
        }
        g_last_error = saved;
        if (!x->small) return kNoRoute;
    }
    pi_multi_batch_t b{};
    b.index = 0;
    b.ops = ops;
    b.keys = keys;
    b.values = values;
    b.n = n;
    b.results = results;
    return multi_execute(x->small, &b, 1, s, x);
}

}  // namespace

namespace pi {
void set_last_error(int code) { g_last_error = code; }

// Makes the index's per-batch scratch hold batches of n queries (the serving runtime
// sizes it for its largest coalesced batch up front). Synchronises `s`.
int reserve_batch(pi_index* x, uint64_t n, cudaStream_t s) {
    if (!x || n > PI_MAX_BATCH) return PI_ERR_INVALID_ARG;
    order_after_last(x, s);
    if (n <= x->sc.cap) return PI_OK;
    return map_cuda(grow_scratch(x, n, s));
}
}  // namespace pi
