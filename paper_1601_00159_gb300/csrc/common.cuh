// Shared device-side definitions of the PI batch path (sm_103a).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/pi.h"

namespace pi {

constexpr uint64_t kMaxKey = ~0ull;  // reserved key: level and storage sentinel
constexpr int kLevelSlots = 34;      // per-level arrays are indexed by level 0..33
constexpr uint8_t kTomb = 0x80;      // meta bit 7: the delete flag F_del (Algorithm 4)
constexpr uint8_t kHeightMask = 0x3F;
constexpr uint32_t kSmemTopMax = 12288;  // index entries staged in shared memory (148 KB with their downs)
constexpr uint32_t kPad = 64;           // readable entries past every array's end
constexpr uint32_t kSortTile = 2048;    // elements per radix-sort tile
constexpr uint32_t kScanGroup = 64;     // radix-sort tiles per group of the count kernel's scan
constexpr uint32_t kCtrDistinct = 14;   // BatchMeta::tile_ctr slot: the descent prologue's tile counter
constexpr uint32_t kApplyTile = 2048;   // sorted queries per apply tile
constexpr uint32_t kSubTile = 256;      // sorted queries per descent warp step (one apply warp)

// Sticky error bits in DevMeta::error.
constexpr uint32_t kErrTimeout = 1u;  // a bounded wait gave up
constexpr uint32_t kErrBounds = 2u;   // an internal bound check refused an access
constexpr uint32_t kErrOwner = 4u;    // debug check: a storage node had two writers in one batch

// Bounded spins: a look-back or barrier wait gives up after this many polls (about
// 1.4 s on a GB300 with the back-off below) and records kErrTimeout instead of hanging.
constexpr uint32_t kSpinLimit = 1u << 22;

// Persistent device state of one index (one allocation, lives with the index).
struct DevMeta {
    uint32_t cur;          // which of the two storage buffers is current
    uint32_t size;         // storage-layer nodes (delete-flagged ones included)
    uint32_t tombs;        // delete-flagged nodes
    uint32_t error;        // sticky kErr* bits
    // layout of the index layer as last built
    uint32_t H;            // top built level (1: no index level)
    uint32_t Lb;           // lowest materialised index level
    uint32_t Ls;           // lowest level staged in shared memory (> H: none)
    uint32_t smem_entries; // entries [0, smem_entries) are staged
    uint32_t index_total;  // entries in use (sentinels included)
    uint32_t index_need;   // entries a full build needs
    uint32_t grow_request; // 1 when levels were dropped for lack of capacity
    uint32_t updates;      // node changes since the last rebuild
    uint32_t rebuilds;     // rebuilds run
    uint32_t batches;      // batches run
    uint32_t sort_fix_big; // last batch: queries in key-prefix segments sorted by one CTA
    uint32_t lcur;         // which of the two index-layer buffers holds the built levels
    uint32_t levels_exact; // 1: the built levels hold exactly the live keys of their heights
    uint32_t inc_rebuilds; // rebuilds that updated the previous levels instead of scanning
    uint32_t owner_writes; // debug check: storage-node writes counted so far
    uint32_t cnt[kLevelSlots];   // live keys with height >= l, kept current every batch
    uint32_t n[kLevelSlots];     // n[l]: size of built level l
    uint32_t base[kLevelSlots];  // built level l occupies [base[l], base[l] + n[l]] (+ sentinel)
};

struct SortPlan {
    uint64_t pmask;   // the key bytes the passes sort
    uint32_t npass;
    uint32_t digit[8];
    uint32_t src[8];  // 0 = packed input, 1 = buffer A, 2 = buffer B
    uint32_t dst[8];
    uint32_t fix;     // 1: segments of equal pmask bytes still need ordering by the full key
    uint32_t nr;      // the other bytes that can differ inside a segment, ascending in rdig
    uint32_t rdig[8];
};

// Digit plan of a radix sort of n keys (see the sort's description): bmax / bnmin are
// the per-byte maxima and (255 - minima) over the valid keys, invalid the number of
// invalid keys (sort key 2^64-1), max_passes the pass budget (1..8).
__device__ __forceinline__ void plan_digits(const uint32_t* bmax, const uint32_t* bnmin, uint32_t invalid,
                                            uint32_t n, uint32_t max_passes, SortPlan& P) {
    const bool any_valid = invalid < n;
    uint32_t r = 0;
    uint32_t dig[8];
    bool varies[8], differs[8];  // among valid keys; between valid and invalid keys
    int p = -1;                  // highest byte where every valid key is below 0xFF
    for (int d = 0; d < 8; ++d) {
        const uint32_t hi = bmax[d], lo = 255u - bnmin[d];
        varies[d] = any_valid && hi != lo;
        differs[d] = invalid && any_valid && lo < 255u;
        if (varies[d]) dig[r++] = (uint32_t)d;
        if (!any_valid || hi < 255u) p = d;
    }
    if (invalid) {
        bool have = false;
        for (uint32_t j = 0; j < r; ++j) have |= dig[j] == (uint32_t)p;
        if (p < 0) {  // no single byte separates the invalid key: sort every byte
            r = 0;
            for (int d = 0; d < 8; ++d) dig[r++] = (uint32_t)d;
        } else if (!have) {  // insert p, keeping dig ascending
            uint32_t j = r++;
            while (j > 0 && dig[j - 1] > (uint32_t)p) {
                dig[j] = dig[j - 1];
                --j;
            }
            dig[j] = (uint32_t)p;
        }
    }
    if (r == 0) dig[r++] = 0;  // all keys equal: one pass (identity order)
    const uint32_t skip = r > max_passes ? r - max_passes : 0u;  // D bytes below the prefix
    P.npass = r - skip;
    P.pmask = 0;
    for (uint32_t j = 0; j < P.npass; ++j) {
        P.digit[j] = dig[skip + j];
        P.src[j] = (j == 0) ? 0u : P.dst[j - 1];
        P.dst[j] = ((P.npass - 1 - j) % 2 == 0) ? 1u : 2u;  // the last pass writes buffer A
        P.pmask |= 0xFFull << (8 * dig[skip + j]);
    }
    P.fix = skip ? 1u : 0u;
    P.nr = 0;
    if (skip)
        for (int d = 0; d < 8; ++d)
            if (!((P.pmask >> (8 * d)) & 1u) && (varies[d] || differs[d])) P.rdig[P.nr++] = (uint32_t)d;
}

// Per-batch scratch counters, cleared by one memset at the start of every batch.
struct BatchMeta {
    uint32_t tile_ctr[24];       // dynamic tile counters, one per look-back kernel
    int32_t delta[kLevelSlots];  // change of n[l] in this batch
    int32_t tomb_delta;
    uint32_t invalid;            // invalid queries
    uint32_t new_count;          // new storage nodes
    uint32_t merged;             // storage layer re-laid-out
    uint32_t index_dirty;        // level membership changed
    uint32_t rebuild;            // the rebuild runs in this batch
    uint32_t changes;            // storage nodes whose liveness changed or that were added
    uint32_t distinct;           // distinct keys of the batch (local run heads)
    uint32_t bmax[8];            // per key byte: its maximum over the batch
    uint32_t bnmin[8];           // per key byte: 255 - its minimum over the batch
    uint32_t fix_big;            // queries in key-prefix segments longer than one warp
    SortPlan plan;
    // incremental level rebuild (no storage re-layout): the levels are updated from the
    // previous buffer and the batch's membership changes
    uint32_t nchg;                    // packed membership changes
    uint32_t chg_hist[kLevelSlots];   // changes by height
    uint32_t inc;                     // 1: this batch's rebuild is incremental
    uint32_t old_H, old_total;
    uint32_t old_n[kLevelSlots], old_base[kLevelSlots];
    uint32_t lst_off[kLevelSlots], lst_n[kLevelSlots];  // per-level change lists
};

// Storage layer, double buffered: [0] and [1]; DevMeta::cur picks the current one.
struct Storage {
    uint64_t* keys[2];
    uint64_t* vals[2];
    uint8_t* meta[2];
};

struct NewNodes {
    uint64_t* keys;
    uint64_t* vals;
    uint32_t* loc;  // storage position + 1 of the largest stored key below it (0: front)
    uint8_t* height;
};

// Membership changes of the built index levels in one batch, in key order: nodes of
// height >= the lowest built level whose liveness changed (no storage re-layout).
struct LevelChanges {
    uint64_t* keys;
    uint32_t* pos;  // storage position
    uint8_t* hl;    // height | 0x80 when the node became live (else it became delete-flagged)
};

struct HashParams {
    uint64_t seed_mix;  // splitmix64(seed)
    int b;              // P = 2^-b
    int hmax;           // min(32, 64 / b)
};

// ---------------------------------------------------------------------------------
// Tower height (Definition 1 with the geometric draw replaced by a seeded key hash).
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ uint32_t tower_height(uint64_t key, const HashParams& hp) {
    uint64_t h = splitmix64(key ^ hp.seed_mix);
    int tz = h ? (__ffsll((long long)h) - 1) : 64;
    int lvl = tz / hp.b;
    if (lvl > hp.hmax - 1) lvl = hp.hmax - 1;
    return 1u + (uint32_t)lvl;
}

// ---------------------------------------------------------------------------------
// Memory helpers.
__device__ __forceinline__ uint64_t ld_relaxed(const uint64_t* p) {
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
// Publishes a look-back descriptor. An atomic exchange is performed at L2, where the
// readers' relaxed loads look; a plain relaxed store was measured to take several
// microseconds to become visible to them (a decoupled look-back waited 7.9 us per tile
// on average with stores, 3.1 us with exchanges).
__device__ __forceinline__ void publish(uint64_t* p, uint64_t v) {
    atomicExch(reinterpret_cast<unsigned long long*>(p), (unsigned long long)v);
}
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
// Programmatic dependent launch. Kernels of the batch path are launched with
// launch_dep, which lets the next kernel on the stream be scheduled while this one
// drains. Every such kernel calls pdl_wait() before it touches memory: it returns once
// the previous kernel on the stream has completed and its writes are visible (at once
// when there is none). pdl_trigger() then lets the next kernel's CTAs be placed as SMs
// free up; they wait in their own pdl_wait().
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}
__device__ __forceinline__ uint32_t lanemask_le() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_le;" : "=r"(m));
    return m;
}

// ---------------------------------------------------------------------------------
// Decoupled look-back (Merrill and Garland, "Single-pass parallel prefix scan with
// decoupled look-back", 2016). Descriptor word: epoch (32) | flag (2) | value (30).
// The epoch is unique per launch, so descriptors never need clearing between
// launches: a word from an older launch reads as "not yet published".
constexpr uint64_t kFlagAgg = 1ull << 30;
constexpr uint64_t kFlagPrefix = 2ull << 30;
constexpr uint32_t kValMask = (1u << 30) - 1u;

template <bool kMax>
__device__ __forceinline__ uint32_t lb_op(uint32_t a, uint32_t b) {
    return kMax ? (a > b ? a : b) : a + b;
}

// Publishes `agg` for tile `tile` and returns the exclusive prefix of the tiles before
// it (identity 0 for both sum and max). Sets *ok = false and records kErrTimeout if a
// predecessor never published within the spin bound.
template <bool kMax>
__device__ uint32_t lookback(uint64_t* desc, size_t stride, uint32_t tile, uint32_t epoch,
                             uint32_t agg, uint32_t* err, bool* ok) {
    const uint64_t tag = (uint64_t)epoch << 32;
    *ok = true;
    if (tile == 0) {
        publish(desc, tag | kFlagPrefix | (agg & kValMask));
        return 0;
    }
    publish(desc + (size_t)tile * stride, tag | kFlagAgg | (agg & kValMask));
    uint32_t excl = 0;
    int64_t t = (int64_t)tile - 1;
    uint32_t spins = 0;
    while (t >= 0) {
        uint64_t d = ld_relaxed(desc + (size_t)t * stride);
        uint64_t flag = d & (3ull << 30);
        if ((uint32_t)(d >> 32) != epoch || flag == 0) {
            ++spins;
            if (spins > kSpinLimit) {
                atomicOr(err, kErrTimeout);
                *ok = false;
                return 0;
            }
            if ((spins & 1023u) == 0 && *(volatile uint32_t*)err) {  // another wait gave up
                *ok = false;
                return 0;
            }
            if (spins > 32) __nanosleep(100);
            continue;
        }
        excl = lb_op<kMax>(excl, (uint32_t)(d & kValMask));
        if (flag == kFlagPrefix) break;
        --t;
    }
    publish(desc + (size_t)tile * stride, tag | kFlagPrefix | (lb_op<kMax>(excl, agg) & kValMask));
    return excl;
}

// Per-thread variant that keeps kWin predecessor reads in flight per round trip
// (one thread per digit in the radix sort, descriptors strided by `stride`).
template <int kWin>
__device__ __forceinline__ uint32_t lookback_sum_win(uint64_t* desc, size_t stride, uint32_t tile, uint32_t epoch, uint32_t agg,
                                  uint32_t* err, bool* ok) {
    const uint64_t tag = (uint64_t)epoch << 32;
    *ok = true;
    if (tile == 0) {
        publish(desc, tag | kFlagPrefix | (agg & kValMask));
        return 0;
    }
    publish(desc + (size_t)tile * stride, tag | kFlagAgg | (agg & kValMask));
    uint32_t excl = 0, spins = 0;
    int64_t t = (int64_t)tile - 1;
    while (t >= 0) {
        uint64_t d[kWin];
#pragma unroll
        for (int i = 0; i < kWin; ++i) d[i] = (t - i >= 0) ? ld_relaxed(desc + (size_t)(t - i) * stride) : (tag | kFlagPrefix);
        int used = 0;
        bool stop = false, stall = false;
        uint32_t add = 0;
#pragma unroll
        for (int i = 0; i < kWin; ++i) {
            if (stop || stall) continue;
            const uint64_t flag = d[i] & (3ull << 30);
            if ((uint32_t)(d[i] >> 32) != epoch || flag == 0) {
                stall = true;
                continue;
            }
            add += (uint32_t)(d[i] & kValMask);
            ++used;
            if (flag == kFlagPrefix) stop = true;
        }
        excl += add;
        t -= used;
        if (stop) break;
        if (stall) {
            ++spins;
            if (spins > kSpinLimit) {
                atomicOr(err, kErrTimeout);
                *ok = false;
                return 0;
            }
            if ((spins & 1023u) == 0 && *(volatile uint32_t*)err) {
                *ok = false;
                return 0;
            }
            if (spins > 32) __nanosleep(100);
        }
    }
    publish(desc + (size_t)tile * stride, tag | kFlagPrefix | ((excl + agg) & kValMask));
    return excl;
}

// First half of a look-back, for callers that publish their aggregate early and do
// other work before waiting on their predecessors: tile 0 publishes its inclusive
// prefix at once, every other tile its aggregate. One thread calls it.
__device__ __forceinline__ void lookback_publish(uint64_t* desc, uint32_t tile, uint32_t epoch, uint32_t agg) {
    const uint64_t tag = (uint64_t)epoch << 32;
    publish(desc + tile, tag | (tile == 0 ? kFlagPrefix : kFlagAgg) | (agg & kValMask));
}

// Warp-wide variant, called by all 32 lanes of one warp: each round reads the
// descriptors of 32 predecessors at once (lane i reads tile base - 1 - i), so a run of
// predecessors that have published only their aggregates is crossed 32 tiles per
// memory round trip instead of one. Returns the exclusive prefix in every lane.
// With `published`, lookback_publish has already stored this tile's aggregate; `agg` must
// still be that aggregate, since the inclusive prefix published at the end adds it.
template <bool kMax>
__device__ uint32_t lookback_warp(uint64_t* desc, uint32_t tile, uint32_t epoch, uint32_t agg, uint32_t* err,
                                  bool* ok, bool published = false) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t tag = (uint64_t)epoch << 32;
    *ok = true;
    if (tile == 0) {
        if (lane == 0 && !published) publish(desc, tag | kFlagPrefix | (agg & kValMask));
        return 0;
    }
    if (lane == 0 && !published) publish(desc + tile, tag | kFlagAgg | (agg & kValMask));
    uint32_t excl = 0;
    int64_t base = (int64_t)tile;
    uint32_t spins = 0;
    for (;;) {
        const int64_t t = base - 1 - (int64_t)lane;
        uint64_t d = (t >= 0) ? ld_relaxed(desc + t) : (tag | kFlagPrefix);  // before tile 0: prefix 0
        const uint64_t flag = d & (3ull << 30);
        const bool valid = (uint32_t)(d >> 32) == epoch && flag != 0;
        const uint32_t pref = __ballot_sync(0xffffffffu, valid && flag == kFlagPrefix);
        const uint32_t inval = __ballot_sync(0xffffffffu, !valid);
        const uint32_t stop = pref ? (uint32_t)(__ffs(pref) - 1) : 32u;
        const uint32_t need = (stop >= 31u) ? 0xffffffffu : ((2u << stop) - 1u);  // lanes 0..stop
        if (inval & need) {
            ++spins;
            if (spins > kSpinLimit) {
                if (lane == 0) atomicOr(err, kErrTimeout);
                *ok = false;
                return 0;
            }
            if ((spins & 1023u) == 0 && *(volatile uint32_t*)err) {
                *ok = false;
                return 0;
            }
            if (spins > 32) __nanosleep(100);
            continue;
        }
        uint32_t v = (lane <= stop) ? (uint32_t)(d & kValMask) : 0u;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const uint32_t y = __shfl_xor_sync(0xffffffffu, v, o);
            v = lb_op<kMax>(v, y);
        }
        excl = lb_op<kMax>(excl, v);
        if (stop < 32u) break;
        base -= 32;
    }
    if (lane == 0) publish(desc + tile, tag | kFlagPrefix | (lb_op<kMax>(excl, agg) & kValMask));
    return excl;
}

// Wider warp-wide variant: each lane reads kPer predecessors per round (lane i reads tile
// base - 1 - i - 32 k), so 32 kPer tiles are crossed per memory round trip. Kernels whose
// first wave holds hundreds of tiles that all publish their aggregates at once use it:
// the last tile of such a wave finds the nearest inclusive prefix in a few rounds.
template <bool kMax, int kPer>
__device__ uint32_t lookback_warp_wide(uint64_t* desc, uint32_t tile, uint32_t epoch, uint32_t agg, uint32_t* err,
                                       bool* ok) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t tag = (uint64_t)epoch << 32;
    *ok = true;
    if (tile == 0) {
        if (lane == 0) publish(desc, tag | kFlagPrefix | (agg & kValMask));
        return 0;
    }
    if (lane == 0) publish(desc + tile, tag | kFlagAgg | (agg & kValMask));
    uint32_t excl = 0;
    int64_t base = (int64_t)tile;
    uint32_t spins = 0;
    for (;;) {
        uint64_t d[kPer];
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            const int64_t t = base - 1 - (int64_t)lane - 32 * k;
            d[k] = (t >= 0) ? ld_relaxed(desc + t) : (tag | kFlagPrefix);  // before tile 0: prefix 0
        }
        // distance (lane + 32 k) of the nearest predecessor that published its prefix
        uint32_t mine = 0xffffffffu;
#pragma unroll
        for (int k = kPer - 1; k >= 0; --k) {
            const bool valid = (uint32_t)(d[k] >> 32) == epoch && (d[k] & (3ull << 30)) != 0;
            if (valid && (d[k] & (3ull << 30)) == kFlagPrefix) mine = lane + 32u * (uint32_t)k;
        }
        const uint32_t stop = __reduce_min_sync(0xffffffffu, mine);
        const uint32_t lim = (stop == 0xffffffffu) ? 32u * kPer - 1u : stop;
        bool bad = false;
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            const bool valid = (uint32_t)(d[k] >> 32) == epoch && (d[k] & (3ull << 30)) != 0;
            if (lane + 32u * (uint32_t)k <= lim && !valid) bad = true;
        }
        if (__any_sync(0xffffffffu, bad)) {
            ++spins;
            if (spins > kSpinLimit) {
                if (lane == 0) atomicOr(err, kErrTimeout);
                *ok = false;
                return 0;
            }
            if ((spins & 1023u) == 0 && *(volatile uint32_t*)err) {
                *ok = false;
                return 0;
            }
            if (spins > 32) __nanosleep(100);
            continue;
        }
        uint32_t v = 0;
#pragma unroll
        for (int k = 0; k < kPer; ++k)
            if (lane + 32u * (uint32_t)k <= lim) v = lb_op<kMax>(v, (uint32_t)(d[k] & kValMask));
        v = kMax ? __reduce_max_sync(0xffffffffu, v) : __reduce_add_sync(0xffffffffu, v);
        excl = lb_op<kMax>(excl, v);
        if (stop != 0xffffffffu) break;
        base -= 32 * kPer;
    }
    if (lane == 0) publish(desc + tile, tag | kFlagPrefix | (lb_op<kMax>(excl, agg) & kValMask));
    return excl;
}

// ---------------------------------------------------------------------------------
// TMA bulk copies (cp.async.bulk, global -> shared) completing on an mbarrier.
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
// Requires 16-byte aligned addresses and a size that is a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t phase) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}
// Bounded wait for one phase. On timeout records kErrTimeout and returns false.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t phase, uint32_t* err) {
    for (uint32_t i = 0; i < (1u << 20); ++i) {
        if (mbar_try_wait(bar, phase)) return true;
        if (i > 16) __nanosleep(64);
    }
    atomicOr(err, kErrTimeout);
    return false;
}

// Block-uniform test of the sticky error word (every thread gets the same answer).
__device__ __forceinline__ bool block_sees_error(const uint32_t* err) {
    return __syncthreads_or(threadIdx.x == 0 && *(volatile const uint32_t*)err) != 0;
}

// ---------------------------------------------------------------------------------
// Block-wide exclusive sum over one value per thread (blockDim.x a multiple of 32).
template <int kThreads>
__device__ __forceinline__ uint32_t block_excl_sum(uint32_t v, uint32_t* warp_tmp, uint32_t* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tmp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = (lane < kThreads / 32) ? warp_tmp[lane] : 0;
        uint32_t s = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < kThreads / 32) warp_tmp[lane] = s - w;
        if (lane == kThreads / 32 - 1) warp_tmp[32] = s;
    }
    __syncthreads();
    uint32_t r = warp_tmp[warp] + x - v;
    if (total) *total = warp_tmp[32];
    __syncthreads();
    return r;
}

// Stable rank within a warp of kI x 32 elements visited in index order (k, then lane),
// by a kBits-bit digit; dig = 1 << kBits marks an empty slot. The lanes holding the
// same digit are found with kBits + 1 ballots (validity + digit bits); the lowest of
// them adds the group's size to the warp's counter for that digit (whist) with one
// shared-memory atomic, whose old value is the group's base. The __syncwarp orders the
// atomics of consecutive items, so equal digits keep index order; the bases are
// gathered only after the loop. On return rank[k] counts the warp's earlier elements
// with the same digit, and whist[d] has grown by the warp's elements with digit d.
template <int kI, int kBits>
__device__ __forceinline__ void warp_digit_ranks(const uint32_t (&dig)[kI], uint32_t (&rank)[kI], uint32_t* whist) {
    constexpr uint32_t kEmpty = 1u << kBits;
    const uint32_t lt = lanemask_lt();
    uint32_t lower[kI], old[kI], lead[kI];
#pragma unroll
    for (int k = 0; k < kI; ++k) {
        const uint32_t d = dig[k];
        uint32_t peers = __ballot_sync(0xffffffffu, d < kEmpty);
        if (d >= kEmpty) peers = ~peers;
#pragma unroll
        for (int b = 0; b < kBits; ++b) {
            const uint32_t m = __ballot_sync(0xffffffffu, (d >> b) & 1u);
            peers &= ((d >> b) & 1u) ? m : ~m;
        }
        lead[k] = (uint32_t)(__ffs(peers) - 1);
        lower[k] = __popc(peers & lt);
        old[k] = 0;
        if (lower[k] == 0 && d < kEmpty) old[k] = atomicAdd(&whist[d], (uint32_t)__popc(peers));
        __syncwarp();
    }
#pragma unroll
    for (int k = 0; k < kI; ++k) rank[k] = __shfl_sync(0xffffffffu, old[k], (int)lead[k]) + lower[k];
}

// Block-wide inclusive max over one value per thread; returns the exclusive max.
template <int kThreads>
__device__ __forceinline__ uint32_t block_excl_max(uint32_t v, uint32_t* warp_tmp, uint32_t* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x = max(x, y);
    }
    uint32_t ex = __shfl_up_sync(0xffffffffu, x, 1);
    if (lane == 0) ex = 0;
    if (lane == 31) warp_tmp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = (lane < kThreads / 32) ? warp_tmp[lane] : 0;
        uint32_t s = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s = max(s, y);
        }
        uint32_t e = __shfl_up_sync(0xffffffffu, s, 1);
        if (lane == 0) e = 0;
        if (lane < kThreads / 32) warp_tmp[lane] = e;
        if (lane == kThreads / 32 - 1) warp_tmp[32] = s;
    }
    __syncthreads();
    uint32_t r = max(warp_tmp[warp], ex);
    if (total) *total = warp_tmp[32];
    __syncthreads();
    return r;
}

// ---------------------------------------------------------------------------------
// Host-side launch wrappers (defined in the .cu files).
struct SortBuffers {
    uint64_t* in_k;  // packed keys (written by the pack kernel)
    uint32_t* in_p;  // packed payload: op << 30 | arrival index
    uint64_t* a_k;
    uint32_t* a_p;
    uint64_t* b_k;
    uint32_t* b_p;
    uint32_t* dofs;  // [256] digit bases (first output slot of each digit) of the current pass
    uint64_t* desc;  // [tiles][256] look-back descriptors
    uint32_t* tcnt;      // [tiles][256] per-tile digit counts of the current pass
    uint32_t* toff;      // [tiles][256] per-tile digit offsets within the tile's group
    uint32_t* gsum;      // [groups][256] per-group digit totals, then the groups' offsets
    uint32_t* gctr;      // [8][groups + 1] arrival counters of the count kernel's CTAs
    uint8_t* ndig;       // next pass's digit of every element, in the current pass's output order
    uint32_t* fixmap;    // [ceil(n / 32)] bit per position: start of a segment to reorder
};

// Radix sort of (key, payload) pairs: result in a_k / a_p, stable, by key.
// ops may be NULL (all searches). Counts invalid queries into bm->invalid.
// At most max_passes (1..8) digit passes run, on the most significant bytes that vary;
// when more bytes vary, runs of equal sorted bytes are then ordered by the rest.
cudaError_t launch_sort(const uint8_t* ops, const uint64_t* keys, uint32_t n, const SortBuffers& sb,
                        BatchMeta* bm, uint32_t* err, cudaStream_t s, int num_sms, int max_passes);

struct DescendArgs {
    const uint64_t* sk;  // sorted keys
    const uint32_t* sp;  // sorted payload (op << 30 | arrival index)
    uint32_t* tile_pref; // per-apply-tile exclusive max prefix of the run markers e_i
    uint32_t* sub_pref;  // dense index of each sub-tile's first distinct key
    uint64_t* desc;      // look-back descriptors: 2 words per apply tile
    uint64_t* dq;        // dense distinct keys
    uint32_t* dlo;       // their current start position on the level being searched
    int top_launched;    // highest index level given its own launch (see launch_descend);
                         // at least bottom_launched
    int bottom_launched; // lowest level that can be built: searched by the storage locate
    const DevMeta* m;
    BatchMeta* bm;
    const uint64_t* lkeys;   // index-layer buffer 0 (DevMeta::lcur picks the one in use)
    const uint32_t* ldown;
    const uint64_t* lkeys1;  // buffer 1
    const uint32_t* ldown1;
    Storage st;
    uint32_t* loc;
    uint8_t* flags;
    uint64_t* val0;
    uint32_t n;
    uint32_t* err;
};
// before_locate (may be null) is recorded on s just before the storage-locate kernel.
// The look-back of the first kernel takes ++epoch; a.desc needs 2 words per apply tile.
cudaError_t launch_descend(const DescendArgs& a, uint32_t& epoch, cudaStream_t s, int num_sms,
                           cudaEvent_t before_locate = nullptr);

struct ApplyArgs {
    const uint64_t* sk;
    const uint32_t* sp;
    const uint32_t* loc;
    const uint8_t* flags;
    const uint64_t* val0;
    const uint64_t* uvals;
    pi_result_t* results;
    Storage st;
    NewNodes nn;
    DevMeta* m;
    BatchMeta* bm;
    uint64_t* desc;  // unused
    uint32_t* tile_pref;  // per-tile exclusive prefix (max, then reused for new-node sums)
    uint32_t* tile_new;   // per-tile new-node count
    const uint32_t* sub_pref;  // dense index of each 256-query sub-tile's first distinct key
    NewNodes stage;       // per-tile staging of new nodes (kApplyTile slots per tile)
    LevelChanges cstage;  // per-tile staging of level membership changes
    LevelChanges chg;     // the changes, packed in key order
    uint32_t* tile_chg;   // per-tile change count
    uint32_t* tile_chg_pref;
    uint32_t* lcnt;  // per-level per-tile live counts (see RebuildArgs)
    uint32_t lstride;
    uint32_t n;
    HashParams hp;
    uint32_t* err;
    uint32_t* wcount;  // debug check (null when off): writes per storage node in this batch
};
cudaError_t launch_apply(const ApplyArgs& a, uint32_t& epoch, cudaStream_t s, int num_sms);
// Debug check of single ownership: every storage node written at most once by the
// batch's apply (sets kErrOwner otherwise); adds the writes to DevMeta::owner_writes and
// clears the counts.
cudaError_t launch_owner_check(const ApplyArgs& a, cudaStream_t s, int num_sms);
// Failure-path self-test: one CTA waits, by the batch kernels' bounded look-back, for a
// predecessor that never publishes (desc: 64 zeroed words; err: zeroed word).
cudaError_t launch_wait_selftest(uint64_t* desc, uint32_t* err, cudaStream_t s);

struct RebuildArgs {
    Storage st;
    NewNodes nn;
    DevMeta* m;
    BatchMeta* bm;
    uint64_t* lkeys;      // index-layer buffer 0 (DevMeta::lcur picks the one in use)
    uint32_t* ldown;
    uint64_t* lkeys1;     // buffer 1
    uint32_t* ldown1;
    uint64_t* desc;       // look-back descriptors: max(tiles_merge, tiles_rebuild * 32)
    uint32_t* lcnt;       // per-level per-tile live counts, level-major, row stride lstride
    uint32_t* loff;       // rebuild: per-level per-tile offsets (scan output)
    uint32_t* mcnt;       // merge: live old nodes per tile [0, lstride), their prefix [lstride, 2 lstride)
    uint32_t lstride;     // tiles per row of lcnt (storage capacity / 4096 + 2)
    uint32_t index_cap;   // entries (without padding)
    uint32_t size_ub;     // upper bound of the storage size after the batch
    uint32_t rebuild_policy;
    uint32_t threshold_pct;
    uint32_t force_rebuild;  // 1: rebuild regardless; 2: initial build (not a batch)
    uint32_t st_cap;         // storage capacity (nodes, padding excluded)
    uint32_t smem_top;       // cap on pinned entries (<= kSmemTopMax)
    uint32_t min_lb;         // lowest index level to build (>= 2)
    uint32_t* err;
    LevelChanges chg;        // the batch's level membership changes (key order)
    uint64_t* lst_keys;      // per-level change lists (level l at bm->lst_off[l])
    uint32_t* lst_pos;
    int32_t* lst_pref;       // entries' running (inserts - deletes) before them; one extra at the end
    uint8_t* lst_ins;
    uint32_t lst_cap;        // entries the lists hold (an incremental rebuild needs them all)
};
cudaError_t launch_relevel(const RebuildArgs& a, cudaStream_t s, int num_sms);
cudaError_t launch_merge(const RebuildArgs& a, uint32_t& epoch, cudaStream_t s, int num_sms);
cudaError_t launch_level_bases(const RebuildArgs& a, cudaStream_t s);
// ---------------------------------------------------------------------------------
// Batching form: a set of indices, one batch each, in one persistent launch.
struct MIndex {           // one index of the set: its own arrays and device meta
    DevMeta* m;
    Storage st;
    uint64_t* lkeys;      // index-layer buffer 0 (DevMeta::lcur picks the one in use)
    uint32_t* ldown;
    uint64_t* lkeys1;     // buffer 1
    uint32_t* ldown1;
    uint32_t st_cap;      // storage nodes per buffer
    uint32_t idx_cap;     // index-layer entries
    uint32_t smem_top;    // the plain descent's pinned-entry cap (kept in DevMeta::Ls)
    uint32_t min_lb;      // lowest index level to build (>= 2)
    HashParams hp;
};

struct MItem {            // one queued batch
    const uint8_t* ops;
    const uint64_t* keys;
    const uint64_t* vals;
    pi_result_t* results;
    uint32_t n;
    uint32_t index;
};

struct MultiArgs {
    const MIndex* idx;
    const MItem* items;       // the queue, largest work first
    const uint32_t* nitems;   // queue length (device)
    uint32_t* head;           // next queue slot (device, 0 at launch)
    uint8_t* scratch;         // per-CTA scratch, stride bytes each
    uint64_t stride;
    uint32_t qcap;            // queries per batch the scratch holds
    uint32_t pad_;
    DevMeta* mirror;          // copy of every processed index's meta, by index (may be null)
};

// Range search: both bounds of n queries, sorted and descended as 2n point lookups.
struct RangeArgs {
    const uint64_t* sk;       // sorted bounds
    const uint32_t* sp;       // their payload: bound index (lo of query b, or hi of query b - n)
    const uint32_t* loc;      // per distinct bound: storage nodes with key <= it
    const uint8_t* flags;     // per distinct bound: bit 0 = a node with this key exists
    const uint32_t* sub_pref; // descent sub-tile prefixes of the distinct bounds
    const DevMeta* m;
    const BatchMeta* bm;
    Storage st;
    uint32_t* start;          // [n] first node with key >= lo
    uint32_t* end;            // [n] first node with key > hi
    uint32_t* cnt;            // [n] live nodes in [start, end)
    uint64_t* bsum;           // [n / 256 + 1] per-CTA sums, then their prefix
    uint64_t* offsets;        // [n + 1] output (caller's)
    uint64_t* keys_out;       // [cap] output (caller's)
    uint64_t* vals_out;
    uint64_t cap;
    uint32_t n;
    uint32_t* err;
};
cudaError_t launch_range(const RangeArgs& a, cudaStream_t s);

uint64_t multi_scratch_bytes(uint32_t qcap);
// A kernel variant: warps per CTA, radix digit bits, CTAs per batch (cluster; <= 1: one).
bool multi_variant_ok(int warps, int radix_bits, int cluster);
cudaError_t launch_multi(const MultiArgs& a, int warps, int radix_bits, int cluster, uint32_t grid, cudaStream_t s);
// The variant's largest resident grid in CTAs (sets its shared-memory limit first).
cudaError_t multi_grid(int warps, int radix_bits, int cluster, int num_sms, uint32_t* grid);

// Sets the error code pi_last_error reports on this host thread.
void set_last_error(int code);
// Sizes an index's per-batch scratch for batches of n queries (serving runtime).
int reserve_batch(pi_index_t* idx, uint64_t n, cudaStream_t s);

// Kernels launched by this host thread (every launcher adds the launches it issues); the
// batch entry points fold the difference into the index's own count.
extern thread_local uint64_t g_launches;

template <typename... KP, typename... A>
inline cudaError_t launch_dep_raw(void (*kernel)(KP...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                                  A... args) {
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KP>(args)...);
}

// Per-kernel timing (pi_profile level 2): while a recorder is installed on the host
// thread, launch_dep brackets every launch with two events on the launch's stream.
struct KernelTimer {
    virtual void before(cudaStream_t s) = 0;
    virtual void after(const void* func, cudaStream_t s) = 0;
};
extern thread_local KernelTimer* g_ktimer;

// kernel<<<grid, block, smem, s>>>(args...) with programmatic dependent launch allowed
// (the kernel must begin with pdl_wait()).
template <typename... KP, typename... A>
inline cudaError_t launch_dep(void (*kernel)(KP...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              A... args) {
    if (g_ktimer) g_ktimer->before(s);
    const cudaError_t e = launch_dep_raw(kernel, grid, block, smem, s, args...);
    if (g_ktimer) g_ktimer->after(reinterpret_cast<const void*>(kernel), s);
    return e;
}

cudaError_t launch_rebuild(const RebuildArgs& a, uint32_t& epoch, cudaStream_t s, int num_sms);
cudaError_t launch_rebuild_prep(const RebuildArgs& a, uint32_t& epoch, cudaStream_t s, int num_sms);
cudaError_t launch_rebuild_write(const RebuildArgs& a, cudaStream_t s, int num_sms);

// Bulk build: sorted (key, payload) -> storage layer (last duplicate wins) + counts.
struct CreateArgs {
    const uint64_t* sk;
    const uint32_t* sp;
    const uint64_t* uvals;
    uint32_t n;
    Storage st;
    DevMeta* m;
    BatchMeta* bm;
    uint64_t* desc;
    HashParams hp;
    uint32_t st_cap;
    uint32_t* err;
};
cudaError_t launch_create_storage(const CreateArgs& a, uint32_t& epoch, cudaStream_t s, int num_sms);

// Test-support compactions.
cudaError_t launch_export_live(const Storage& st, const DevMeta* m, uint64_t* keys_out,
                               uint64_t* vals_out, uint64_t cap, uint32_t* count, uint64_t* desc,
                               uint32_t* tile_ctr, uint32_t& epoch, uint32_t* err, cudaStream_t s,
                               int num_sms, uint32_t size_ub);

}  // namespace pi
