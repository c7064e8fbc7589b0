// Batching form: many independent indices, each with its own query batch, in one
// persistent launch (Algorithm 1 applied to every index of a set at once).
//
// Small indices and small batches leave the level-synchronous whole-GPU pipeline of a
// single index (tens of launches, each spread over all SMs) launch-bound. Here a CTA
// runs the whole pipeline of one index's batch by itself, and the CTAs of a persistent
// launch take batches from a device-side work queue, largest first:
//   sort        stable LSD radix sort of (key, arrival) over the varying key bytes,
//               chunks of kT x kMI queries ranked by warp ballots (kBits-bit digits);
//   distinct    the run heads of the sorted batch, compacted;
//   descent     each thread walks kMK distinct keys down the index together (one
//               independent gather per key per step); the top levels are staged in
//               shared memory and resolved by a binary search of the lowest staged one;
//   locate      the storage node with the largest key <= q;
//   apply       one chunked pass with running carries: a max-scan of write markers
//               gives every query the state of its key just before it (arrival order),
//               the last query of each key run owns the node and writes the final state;
//               keys that are new become a sorted list of new nodes;
//   merge       live old nodes and new nodes into the other storage buffer, by the
//               insertion points the descent found;
//   rebuild     the lowest built level from the storage layer, each higher level from
//               the one below it (heights recomputed from the seeded key hash).
// A size class of large indices can instead give each batch to a thread-block cluster
// (k_multi_cl): the same stages, each split into one span per CTA of the cluster, so a
// large index no longer bounds the launch at the speed of one SM.
// All state lives in the indices' own device arrays and DevMeta blocks, so the single-
// index entry points (export, info, the plain batch path) see the same index after it.
// The queue is filled before the launch, so taking an item is one atomicAdd and no CTA
// ever waits on a CTA outside its own cluster.

#include <cooperative_groups.h>

#include "common.cuh"

namespace cg = cooperative_groups;

namespace pi {
namespace {

constexpr uint32_t kMSeqMask = (1u << 30) - 1u;
constexpr int kMI = 4;             // queries or nodes per thread in a chunked pass
constexpr int kMK = 8;             // distinct keys per thread walked down together
constexpr uint32_t kMTop = 2048;   // index entries staged in shared memory
constexpr uint32_t kMSeg = 256;    // colliding segments one CTA orders after the prefix passes
constexpr int kXMax = 40;          // values one cluster exchange carries
constexpr uint32_t kJbWin = 256;   // merge chunks whose new-node bounds are found together
// The radix scatter's chunk staging starts after the digit counters of the largest
// variant (32 warps x 256 digits + three 256-entry arrays, 4 B each).
constexpr uint32_t kSortStage = (32u * 256u + 3u * 256u) * 4u;

__device__ __forceinline__ void mstore_result(pi_result_t* res, uint32_t seq, uint64_t v, uint32_t st) {
    uint4 w;
    w.x = (uint32_t)v;
    w.y = (uint32_t)(v >> 32);
    w.z = st;
    w.w = 0u;
    *reinterpret_cast<uint4*>(res + seq) = w;
}

struct MShared {
    uint32_t tmp[33];
    uint64_t tmp64[33];
    uint32_t bmax[8], bnmin[8];
    uint32_t invalid;
    uint32_t item;
    uint32_t D, newc, dirty, changes, j1;
    uint32_t nseg, overflow;
    uint32_t seg[kMSeg];  // starts of segments the prefix fix-up orders
    int32_t tomb_delta;
    int32_t delta[kLevelSlots];
    uint32_t xs[kXMax];   // staging of values a cluster exchange publishes
    uint32_t jb[kJbWin + 1];  // merge: new nodes placed before each chunk of a window
    SortPlan plan;
    DevMeta m;
};

struct MScratchPtrs {
    uint64_t *ka, *kb;
    uint32_t *pa, *pb;
    uint64_t* dq;   // distinct keys
    uint32_t* dr;   // storage position + 1 of the largest key <= q
    uint8_t* df;    // bit 0: exists, bit 1: live
    uint64_t* dv;   // value when live
    uint64_t *nk, *nv;
    uint8_t* nh;
    uint32_t* ni;   // insertion point (old node the new node precedes)
};

__device__ __forceinline__ uint64_t al256(uint64_t b) { return (b + 255u) & ~255ull; }

__device__ MScratchPtrs carve(uint8_t* base, uint32_t q) {
    MScratchPtrs p;
    uint64_t off = 0;
    const uint64_t c = (uint64_t)q + kPad;
    auto take = [&](uint64_t bytes) {
        uint8_t* r = base + off;
        off += al256(bytes);
        return r;
    };
    p.ka = reinterpret_cast<uint64_t*>(take(c * 8));
    p.kb = reinterpret_cast<uint64_t*>(take(c * 8));
    p.pa = reinterpret_cast<uint32_t*>(take(c * 4));
    p.pb = reinterpret_cast<uint32_t*>(take(c * 4));
    p.dq = reinterpret_cast<uint64_t*>(take(c * 8));
    p.dr = reinterpret_cast<uint32_t*>(take(c * 4));
    p.df = take(c);
    p.dv = reinterpret_cast<uint64_t*>(take(c * 8));
    p.nk = reinterpret_cast<uint64_t*>(take(c * 8));
    p.nv = reinterpret_cast<uint64_t*>(take(c * 8));
    p.nh = take(c);
    p.ni = reinterpret_cast<uint32_t*>(take(c * 4));
    return p;
}

// In-place exclusive scan of cnt[0, kR) by kT threads.
template <int kT, int kR>
__device__ __forceinline__ void small_excl_scan(uint32_t* cnt, uint32_t* tmp) {
    constexpr int per = (kR + kT - 1) / kT;
    uint32_t v[per];
    uint32_t sum = 0;
#pragma unroll
    for (int k = 0; k < per; ++k) {
        const int d = threadIdx.x * per + k;
        v[k] = d < kR ? cnt[d] : 0u;
        sum += v[k];
    }
    uint32_t run = block_excl_sum<kT>(sum, tmp, nullptr);
#pragma unroll
    for (int k = 0; k < per; ++k) {
        const int d = threadIdx.x * per + k;
        if (d < kR) cnt[d] = run;
        run += v[k];
    }
    __syncthreads();
}

// TMA bulk prefetch of [p, p + bytes) into L2 (p 16-byte aligned, bytes a multiple of 16).
__device__ __forceinline__ void l2_prefetch(const void* p, uint32_t bytes) {
    if (bytes) asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// Block-wide exclusive sum of 64-bit values over kT threads; total in *total.
template <int kT>
__device__ __forceinline__ uint64_t block_excl_sum64(uint64_t v, uint64_t* tmp, uint64_t* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) tmp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        const uint64_t w = lane < kT / 32 ? tmp[lane] : 0ull;
        uint64_t t = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint64_t y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < kT / 32) tmp[lane] = t - w;
        if (lane == kT / 32 - 1) tmp[32] = t;
    }
    __syncthreads();
    const uint64_t r = tmp[warp] + x - v;
    if (total) *total = tmp[32];
    __syncthreads();
    return r;
}

// Entries of the sorted a[0, n) below x, by a whole warp: each round probes 32 evenly
// spaced entries of the remaining interval, about log32(n) rounds of one load per lane.
__device__ __forceinline__ uint32_t warp_count_below(const uint32_t* a, uint32_t n, uint32_t x) {
    const uint32_t lane = threadIdx.x & 31u;
    uint32_t lo = 0, hi = n;  // the count lies in [lo, hi]
    while (hi - lo > 32u) {
        const uint32_t step = (hi - lo + 31u) / 32u;
        const uint32_t p = lo + lane * step;
        const uint32_t c = (uint32_t)__popc(__ballot_sync(0xffffffffu, p < hi && a[p] < x));
        if (c == 0) return lo;
        const uint32_t pc = lo + c * step;
        hi = (c < 32u && pc < hi) ? pc : hi;
        lo = lo + (c - 1u) * step + 1u;
    }
    const uint32_t p = lo + lane;
    return lo + (uint32_t)__popc(__ballot_sync(0xffffffffu, p < hi && a[p] < x));
}

// For up to kMK keys at once (bit k of act): narrows [lo[k], hi[k]] of the sorted array K
// to the first index whose key is above q[k], given that K[hi[k]] is above q[k] (the
// next entry of the level above, or a sentinel) and K[lo[k] - 1] is not. Each step
// issues one probe per key before comparing any, so the keys' loads are in flight
// together. hi beyond lim (a bad down pointer) records kErrBounds and is clamped.
__device__ __forceinline__ void multi_bsearch(const uint64_t* K, const uint64_t (&q)[kMK], uint32_t (&lo)[kMK],
                                              uint32_t (&hi)[kMK], uint32_t act, uint32_t lim, uint32_t* err) {
#pragma unroll
    for (int k = 0; k < kMK; ++k) {
        if (!((act >> k) & 1u)) {
            lo[k] = hi[k] = 0;
            continue;
        }
        if (hi[k] > lim || lo[k] > hi[k]) {
            atomicOr(err, kErrBounds);
            hi[k] = min(hi[k], lim);
            lo[k] = min(lo[k], hi[k]);
        }
    }
    for (;;) {
        uint32_t more = 0;
#pragma unroll
        for (int k = 0; k < kMK; ++k) more |= lo[k] < hi[k] ? 1u : 0u;
        if (!more) break;
        uint64_t v[kMK];
#pragma unroll
        for (int k = 0; k < kMK; ++k) v[k] = K[(lo[k] + hi[k]) >> 1];  // <= hi <= lim: in bounds
#pragma unroll
        for (int k = 0; k < kMK; ++k) {
            const uint32_t mid = (lo[k] + hi[k]) >> 1;
            if (lo[k] < hi[k]) {
                if (v[k] <= q[k]) lo[k] = mid + 1;
                else hi[k] = mid;
            }
        }
    }
}

// Scatter of [lo, hi) of (src_k, src_p) by the kBits-bit digit at `shift`. On entry
// sbase[d] (after the per-warp counters in dsm) holds the first destination of digit d
// for this range. Chunks of kT x kMI elements are ranked by warp ballots (elements in
// index order within a chunk), so the scatter is stable; each chunk is first placed in
// shared memory in digit order and then written out in runs, so consecutive threads
// store consecutive addresses of one digit's run (a chunk scattered straight to global
// memory costs one L2 request per element). Destinations at or past dlim are refused
// (kErrBounds).
template <int kT, int kBits>
__device__ void m_scatter(const uint64_t* src_k, const uint32_t* src_p, uint64_t* dst_k, uint32_t* dst_p,
                          uint32_t lo, uint32_t hi, uint32_t shift, uint32_t dlim, uint8_t* dsm, uint32_t* tmp,
                          uint32_t* err) {
    constexpr int kW = kT / 32;
    constexpr int kR = 1 << kBits;
    constexpr uint32_t kC = (uint32_t)kT * kMI;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint32_t* whist = reinterpret_cast<uint32_t*>(dsm);  // [kW][kR]
    uint32_t* sbase = whist + kW * kR;                   // [kR]
    uint32_t* stot = sbase + kR;                         // [kR] the chunk's count per digit
    uint32_t* loff = stot + kR;                          // [kR] the chunk's first slot per digit
    uint64_t* sk = reinterpret_cast<uint64_t*>(dsm + kSortStage);  // [kC] the chunk in digit order
    uint32_t* sp = reinterpret_cast<uint32_t*>(sk + kC);           // [kC]
    for (int d = tid; d < kW * kR; d += kT) whist[d] = 0;
    __syncthreads();
    for (uint32_t c0 = lo; c0 < hi; c0 += kC) {
        uint64_t key[kMI];
        uint32_t pay[kMI], dig[kMI], rank[kMI];
#pragma unroll
        for (int k = 0; k < kMI; ++k) {
            const uint32_t i = c0 + (uint32_t)warp * 32u * kMI + (uint32_t)k * 32u + (uint32_t)lane;
            const bool v = i < hi;
            key[k] = v ? src_k[i] : 0ull;
            pay[k] = v ? src_p[i] : 0u;
            dig[k] = v ? (uint32_t)(key[k] >> shift) & (kR - 1) : (uint32_t)kR;
        }
        warp_digit_ranks<kMI, kBits>(dig, rank, whist + warp * kR);
        __syncthreads();
        for (int d = tid; d < kR; d += kT) {
            uint32_t total = 0;
#pragma unroll 4
            for (int w = 0; w < kW; ++w) {
                const uint32_t cc = whist[w * kR + d];
                whist[w * kR + d] = total;
                total += cc;
            }
            stot[d] = total;
            loff[d] = total;
        }
        __syncthreads();
        small_excl_scan<kT, kR>(loff, tmp);
#pragma unroll
        for (int k = 0; k < kMI; ++k) {
            const uint32_t d = dig[k];
            if (d < (uint32_t)kR) {
                const uint32_t l = loff[d] + whist[warp * kR + d] + rank[k];
                sk[l] = key[k];
                sp[l] = pay[k];
            }
        }
        __syncthreads();
        const uint32_t cnt = hi - c0 < kC ? hi - c0 : kC;
        for (uint32_t i = tid; i < cnt; i += kT) {
            const uint64_t k = sk[i];
            const uint32_t d = (uint32_t)(k >> shift) & (kR - 1);
            const uint32_t pos = sbase[d] + (i - loff[d]);
            if (pos < dlim) {
                dst_k[pos] = k;
                dst_p[pos] = sp[i];
            } else {
                atomicOr(err, kErrBounds);
            }
        }
        __syncthreads();
        for (int d = tid; d < kR; d += kT) {
            sbase[d] += stot[d];
#pragma unroll 4
            for (int w = 0; w < kW; ++w) whist[w * kR + d] = 0;
        }
        __syncthreads();
    }
}

// Adds the kBits-bit digits at `shift` of src_k[lo, hi) to the counters h. Each thread
// loads kMI keys before its first atomic, so the loads are in flight together.
template <int kT, int kBits>
__device__ __forceinline__ void m_histogram(const uint64_t* src_k, uint32_t lo, uint32_t hi, uint32_t shift,
                                            uint32_t* h) {
    constexpr uint32_t kR = 1u << kBits;
    for (uint32_t b0 = lo; b0 < hi; b0 += (uint32_t)kT * kMI) {
        uint32_t dg[kMI];
#pragma unroll
        for (int u = 0; u < kMI; ++u) {
            const uint32_t i = b0 + (uint32_t)u * kT + threadIdx.x;
            dg[u] = i < hi ? (uint32_t)(src_k[i] >> shift) & (kR - 1u) : kR;
        }
#pragma unroll
        for (int u = 0; u < kMI; ++u)
            if (dg[u] < kR) atomicAdd(&h[dg[u]], 1u);
    }
}

// One stable LSD pass over [lo, hi) of (src_k, src_p) by the kBits-bit digit at `shift`,
// into the same range of (dst_k, dst_p): a histogram, its exclusive scan, the scatter.
template <int kT, int kBits>
__device__ void m_lsd_pass(const uint64_t* src_k, const uint32_t* src_p, uint64_t* dst_k, uint32_t* dst_p,
                           uint32_t lo, uint32_t hi, uint32_t shift, uint8_t* dsm, uint32_t* tmp, uint32_t* err) {
    constexpr int kW = kT / 32;
    constexpr int kR = 1 << kBits;
    const int tid = threadIdx.x;
    uint32_t* sbase = reinterpret_cast<uint32_t*>(dsm) + kW * kR;
    for (int d = tid; d < kR; d += kT) sbase[d] = 0;
    __syncthreads();
    m_histogram<kT, kBits>(src_k, lo, hi, shift, sbase);
    __syncthreads();
    small_excl_scan<kT, kR>(sbase, tmp);
    for (int d = tid; d < kR; d += kT) sbase[d] += lo;
    m_scatter<kT, kBits>(src_k, src_p, dst_k, dst_p, lo, hi, shift, hi, dsm, tmp, err);
}

// ---------------------------------------------------------------------------------
// Stages of one batch over a span of its work. The one-CTA pipeline runs each over the
// whole batch; the cluster pipeline gives each CTA of a cluster one span, with carries
// (the values of the spans before it) exchanged through distributed shared memory.

// Run heads of the sorted valid prefix [0, qv) that lie in [lo, hi), compacted into dq
// from position carry on. Returns carry + the heads of the span.
template <int kT>
__device__ uint32_t m_distinct_span(const uint64_t* K, uint32_t qv, uint32_t lo, uint32_t hi, uint32_t carry,
                                    uint64_t* dq, MShared& sh) {
    constexpr uint32_t kC = (uint32_t)kT * kMI;
    const int tid = threadIdx.x;
    for (uint32_t c0 = lo; c0 < hi; c0 += kC) {
        const uint32_t j0 = c0 + (uint32_t)tid * kMI;
        uint64_t prev = (j0 > 0 && j0 - 1 < qv) ? K[j0 - 1] : 0ull;
        uint32_t hm = 0;
#pragma unroll
        for (int k = 0; k < kMI; ++k) {
            const uint32_t j = j0 + k;
            const uint64_t kk = j < qv ? K[j] : 0ull;
            if (j < hi && (j == 0 || kk != prev)) hm |= 1u << k;
            prev = kk;
        }
        uint32_t tot;
        uint32_t o = carry + block_excl_sum<kT>((uint32_t)__popc(hm), sh.tmp, &tot);
#pragma unroll
        for (int k = 0; k < kMI; ++k)
            if ((hm >> k) & 1u) dq[o++] = K[j0 + k];
        carry += tot;
    }
    return carry;
}

// Descent + locate of the distinct keys d0 = first, first + step, ... (kT x kMK keys each):
// the storage node with the largest key <= q, whether q exists and is live, its value.
template <int kT>
__device__ void m_descend(const MIndex& X, const MScratchPtrs& s, const DevMeta& m, const uint64_t* LK,
                          const uint32_t* LD, const uint64_t* SK, const uint64_t* SV, const uint8_t* SM, uint32_t D,
                          uint32_t first, uint32_t step, uint8_t* dsm, uint32_t* err) {
    const int tid = threadIdx.x;
    const uint32_t H = m.H, Lb = m.Lb, size = m.size;
    const bool built = Lb <= H && H >= 2;
    uint32_t Lp = H + 1;  // lowest level staged in shared memory (> H: none)
    if (built)
        for (int l = (int)H; l >= (int)Lb; --l) {
            if (m.base[l] + m.n[l] + 1u <= kMTop) Lp = (uint32_t)l;
            else break;
        }
    uint64_t* tk = reinterpret_cast<uint64_t*>(dsm);
    uint32_t* td = reinterpret_cast<uint32_t*>(dsm + kMTop * sizeof(uint64_t));
    const uint32_t nst = (built && Lp <= H) ? m.base[Lp] + m.n[Lp] + 1u : 0u;
    for (uint32_t i = tid; i < nst; i += kT) {
        tk[i] = LK[i];
        td[i] = LD[i];
    }
    __syncthreads();
    for (uint32_t d0 = first; d0 < D; d0 += step) {
        uint64_t q[kMK];
        uint32_t lo[kMK], hi[kMK];  // the key's predecessor at the level searched lies in [lo - 1, hi)
        uint32_t act = 0;
#pragma unroll
        for (int k = 0; k < kMK; ++k) {
            const uint32_t d = d0 + (uint32_t)k * kT + (uint32_t)tid;
            q[k] = d < D ? s.dq[d] : kMaxKey;
            lo[k] = 0;
            hi[k] = 0;
            if (d < D) act |= 1u << k;
        }
        int l = built ? (int)H : 0;
        if (built && Lp <= H) {
            // the staged level Lp holds every key of the levels above it
            const uint32_t b = m.base[Lp], cnt = m.n[Lp];
#pragma unroll
            for (int k = 0; k < kMK; ++k) {
                uint32_t a = 0, e = cnt;  // first index with key > q
                while (a < e) {
                    const uint32_t mid = (a + e) >> 1;
                    if (tk[b + mid] <= q[k]) a = mid + 1;
                    else e = mid;
                }
                // the gap of level Lp - 1 under the predecessor: [its down, the next entry's down)
                lo[k] = a ? td[b + a - 1] : 0u;
                hi[k] = td[b + a];
            }
            l = (int)Lp - 1;
        } else if (built) {
            // no staged level: the whole top built level
#pragma unroll
            for (int k = 0; k < kMK; ++k) hi[k] = m.n[H];
        } else {
#pragma unroll
            for (int k = 0; k < kMK; ++k) hi[k] = size;  // no index level: the storage layer
        }
        if (built)
            for (; l >= (int)Lb; --l) {
                const uint32_t b = m.base[l];
                multi_bsearch(LK + b, q, lo, hi, act, m.n[l], err);
                // lo = first entry above q (at most the sentinel, n[l]); the gap below its
                // predecessor in the next level down ends at lo's own down pointer
#pragma unroll
                for (int k = 0; k < kMK; ++k) {
                    const uint32_t a = lo[k];
                    const uint32_t dn = LD[b + a];
                    lo[k] = a ? LD[b + a - 1] : 0u;
                    hi[k] = dn;
                }
            }
        multi_bsearch(SK, q, lo, hi, act, size, err);
#pragma unroll
        for (int k = 0; k < kMK; ++k) {
            if (!((act >> k) & 1u)) continue;
            const int32_t r = (int32_t)lo[k] - 1;  // storage node with the largest key <= q
            const uint32_t d = d0 + (uint32_t)k * kT + (uint32_t)tid;
            const bool exists = r >= 0 && SK[r] == q[k];
            const bool live = exists && !(SM[r] & kTomb);
            s.dr[d] = (uint32_t)(r + 1);
            s.df[d] = (uint8_t)((exists ? 1u : 0u) | (live ? 2u : 0u));
            s.dv[d] = live ? SV[r] : 0ull;
        }
    }
    (void)X;
}

// Carries of the apply pass for the queries before a span: the largest write or head
// marker (2j + 3 for a write at j, 2j + 2 for a run head at j), the run heads, and the
// new nodes.
struct ApplyCarry {
    uint32_t cmax, cheads, cnew;
};

// Results, ownership and apply over [lo, hi) of the valid sorted prefix [0, qv), one
// chunked pass with running carries: a max-scan of write markers gives every query the
// state of its key just before it (arrival order), the last query of each key run owns
// the node and writes the final state; keys that are new become the sorted list of new
// nodes from slot c.cnew on. kFull = false only counts the new nodes (no store). Returns
// c.cnew + the span's new nodes. Node changes are counted in sh (delta, tomb_delta,
// changes, dirty).
template <int kT, bool kFull>
__device__ uint32_t m_apply_span(const MItem& it, const MIndex& X, const MScratchPtrs& s, const uint64_t* K,
                                 const uint32_t* P, uint32_t qv, uint32_t lo, uint32_t hi, ApplyCarry c,
                                 uint64_t* SV, uint8_t* SM, MShared& sh) {
    constexpr uint32_t kC = (uint32_t)kT * kMI;
    const int tid = threadIdx.x;
    uint32_t cmax = c.cmax, cheads = c.cheads, cnew = c.cnew;
    for (uint32_t c0 = lo; c0 < hi; c0 += kC) {
        const uint32_t j0 = c0 + (uint32_t)tid * kMI;
        uint64_t key[kMI];
        uint32_t pay[kMI];
#pragma unroll
        for (int k = 0; k < kMI; ++k) {
            const uint32_t j = j0 + k;
            key[k] = j < qv ? K[j] : kMaxKey;
            pay[k] = j < hi ? P[j] : 0u;
        }
        const uint64_t kprev = (j0 > 0 && j0 - 1 < qv) ? K[j0 - 1] : kMaxKey;
        const uint64_t knext = (j0 + kMI < qv) ? K[j0 + kMI] : kMaxKey;
        uint32_t agg = 0, hm = 0, om = 0;
#pragma unroll
        for (int k = 0; k < kMI; ++k) {
            const uint32_t j = j0 + k;
            const bool valid = j < hi;
            const uint64_t prev = k ? key[k - 1] : kprev;
            const uint64_t next = k + 1 < kMI ? key[k + 1] : knext;
            const bool head = valid && (j == 0 || key[k] != prev);
            const bool last = valid && (j + 1 == qv || key[k] != next);
            const uint32_t op = pay[k] >> 30;
            const uint32_t e = (valid && (op == 1u || op == 2u)) ? 2u * j + 3u : (head ? 2u * j + 2u : 0u);
            agg = max(agg, e);
            hm |= (head ? 1u : 0u) << k;
            om |= (last ? 1u : 0u) << k;
        }
        uint32_t tmax;
        uint32_t M = max(cmax, block_excl_max<kT>(agg, sh.tmp, &tmax));
        uint32_t htot;
        uint32_t hidx = cheads + block_excl_sum<kT>((uint32_t)__popc(hm), sh.tmp, &htot);
        // First walk: every query's result; the owners' final states.
        uint32_t nm = 0, wm = 0, lm = 0;  // new node; run wrote; final live
        uint64_t fval[kMI];
        uint32_t djs[kMI];
#pragma unroll
        for (int k = 0; k < kMI; ++k) {
            const uint32_t j = j0 + k;
            fval[k] = 0;
            djs[k] = 0;
            if (j >= hi) continue;
            const bool head = (hm >> k) & 1u;
            hidx += head ? 1u : 0u;
            const uint32_t dj = hidx - 1u;
            djs[k] = dj;
            const uint32_t op = pay[k] >> 30;
            const uint32_t e = (op == 1u || op == 2u) ? 2u * j + 3u : (head ? 2u * j + 2u : 0u);
            const uint32_t mex = M;
            M = max(M, e);
            const uint8_t fl = s.df[dj];
            bool pl;
            uint64_t pv;
            bool wrote = false;
            if (!head && (mex & 1u)) {  // the last write before j lies in j's key run
                const uint32_t pw = P[(mex - 3u) >> 1];
                pl = (pw >> 30) == 1u;
                pv = pl ? it.vals[pw & kMSeqMask] : 0ull;
                wrote = true;
            } else {
                pl = (fl & 2u) != 0;
                pv = s.dv[dj];
            }
            if constexpr (kFull)
                mstore_result(it.results, pay[k] & kMSeqMask, pl ? pv : 0ull, pl ? PI_R_PRESENT : PI_R_ABSENT);
            if (!((om >> k) & 1u)) continue;
            bool flive = pl;
            uint64_t fv = pv;
            if (op == 1u) {
                flive = true;
                fv = it.vals[pay[k] & kMSeqMask];
                wrote = true;
            } else if (op == 2u) {
                flive = false;
                fv = 0;
                wrote = true;
            }
            fval[k] = fv;
            if (wrote) wm |= 1u << k;
            if (flive) lm |= 1u << k;
            if (wrote && !(fl & 1u) && flive) nm |= 1u << k;
        }
        uint32_t ntot;
        uint32_t slot = cnew + block_excl_sum<kT>((uint32_t)__popc(nm), sh.tmp, &ntot);
        if constexpr (kFull) {
            // Second walk: the owners whose run wrote update their node or add a new one.
            int32_t tomb_d = 0;
            uint32_t chg = 0, dirty = 0;
#pragma unroll
            for (int k = 0; k < kMI; ++k) {
                if (!((wm >> k) & 1u)) continue;
                const uint32_t dj = djs[k];
                const uint8_t fl = s.df[dj];
                const bool flive = (lm >> k) & 1u;
                const bool live0 = (fl & 2u) != 0;
                if (fl & 1u) {
                    const uint32_t r = s.dr[dj] - 1u;
                    const uint8_t meta = SM[r];
                    const uint32_t h = meta & 0x3Fu;
                    if (flive) SV[r] = fval[k];
                    SM[r] = (uint8_t)(h | (flive ? 0u : kTomb));
                    if (flive != live0) {
                        tomb_d += flive ? -1 : 1;
                        ++chg;
                        if (h >= 2u) dirty = 1;
                        for (uint32_t l = 1; l <= h && l < (uint32_t)kLevelSlots; ++l)
                            atomicAdd(&sh.delta[l], flive ? 1 : -1);
                    }
                } else if (flive) {
                    const uint32_t h = tower_height(key[k], X.hp);
                    s.nk[slot] = key[k];
                    s.nv[slot] = fval[k];
                    s.nh[slot] = (uint8_t)h;
                    s.ni[slot] = s.dr[dj];
                    ++slot;
                    ++chg;
                    dirty = 1;
                    for (uint32_t l = 1; l <= h && l < (uint32_t)kLevelSlots; ++l) atomicAdd(&sh.delta[l], 1);
                }
            }
            if (tomb_d) atomicAdd(&sh.tomb_delta, tomb_d);
            if (chg) atomicAdd(&sh.changes, chg);
            if (dirty) sh.dirty = 1;
        }
        cmax = max(cmax, tmax);
        cheads += htot;
        cnew += ntot;
    }
    return cnew;
}

// The new level layout from the live counts (one thread; before the merge, which may
// write the lowest level): levels that do not fit the index layer's capacity are
// dropped from the bottom, and the pinned-entry prefix is recomputed.
__device__ void m_layout(const MIndex& X, DevMeta& m) {
    uint32_t H = 1;
    for (int l = 2; l < kLevelSlots; ++l)
        if (m.cnt[l] > 0) H = (uint32_t)l;
    const uint32_t Lb0 = X.min_lb > 2u ? X.min_lb : 2u;
    uint64_t need = 0;
    for (uint32_t l = Lb0; l <= H; ++l) need += (uint64_t)m.cnt[l] + 1u;
    uint32_t Lb = Lb0;
    uint64_t fit = need;
    while (Lb <= H && fit > X.idx_cap) {
        fit -= (uint64_t)m.cnt[Lb] + 1u;
        ++Lb;
    }
    m.index_need = (uint32_t)need;
    m.grow_request = (Lb > Lb0) ? 1u : 0u;
    for (int l = 0; l < kLevelSlots; ++l) {
        m.n[l] = 0;
        m.base[l] = 0;
    }
    uint32_t off = 0;
    for (int l = (int)H; l >= (int)Lb; --l) {
        m.base[l] = off;
        m.n[l] = m.cnt[l];
        off += m.cnt[l] + 1u;
    }
    m.H = H;
    m.Lb = Lb;
    m.index_total = off;
    uint32_t Ls = H + 1;
    for (int l = (int)H; l >= (int)Lb; --l) {
        if (m.base[l] + m.n[l] + 1u <= X.smem_top) Ls = (uint32_t)l;
        else break;
    }
    m.Ls = Ls;
    m.smem_entries = (Ls <= H) ? m.base[Ls] + m.n[Ls] + 1u : 0u;
    m.updates = 0;
    m.rebuilds += 1;
    m.levels_exact = 1;  // rebuilt in place from the storage layer
}

// nmp[j] = new nodes of height >= Lb among the first j (j = 0..M), for the merge that
// also writes the lowest built level.
template <int kT>
__device__ void m_member_prefix(const MScratchPtrs& s, uint32_t* nmp, uint32_t M, uint32_t Lb, MShared& sh) {
    constexpr uint32_t kC = (uint32_t)kT * kMI;
    const int tid = threadIdx.x;
    uint32_t run = 0;
    for (uint32_t g0 = 0; g0 < M; g0 += kC) {
        const uint32_t i0 = g0 + (uint32_t)tid * kMI;
        uint32_t mm = 0;
#pragma unroll
        for (int k = 0; k < kMI; ++k)
            if (i0 + k < M && s.nh[i0 + k] >= Lb) mm |= 1u << k;
        uint32_t tot;
        uint32_t r = run + block_excl_sum<kT>((uint32_t)__popc(mm), sh.tmp, &tot);
#pragma unroll
        for (int k = 0; k < kMI; ++k) {
            if (i0 + k < M) nmp[i0 + k] = r;
            r += (mm >> k) & 1u;
        }
        run += tot;
    }
    if (tid == 0) nmp[M] = run;
    __syncthreads();
}

// Where the merge writes: the destination storage buffer and, when fused, the lowest
// built level (its base, size and the new nodes' member prefix).
struct MergeOut {
    uint64_t* DK;
    uint64_t* DV;
    uint8_t* DM;
    uint64_t* LK;
    uint32_t* LD;
    const uint32_t* nmp;
    uint32_t lbase, nLb, Lb;
    bool fused;
};

// Merge of the old nodes [lo, hi) (lo a multiple of the chunk) and the new nodes placed
// before them, into the other storage buffer. carry: live old nodes before lo; cmem: old
// members of level Lb before lo; both advance. Returns in j0 the new nodes placed before
// hi. The new nodes of each chunk (those placed before one of its old nodes) are found
// for a window of chunks at once, one warp per chunk bound.
template <int kT>
__device__ void m_merge_span(const MScratchPtrs& s, const uint64_t* SK, const uint64_t* SV, const uint8_t* SM,
                             const MergeOut& o, uint32_t lo, uint32_t hi, uint32_t size, uint32_t M,
                             uint32_t& carry, uint32_t& cmem, uint32_t& j0, uint8_t* dsm, MShared& sh) {
    constexpr uint32_t kC = (uint32_t)kT * kMI;
    constexpr uint32_t kW = (uint32_t)kT / 32u;
    const int tid = threadIdx.x;
    const bool fused = o.fused;
    const uint32_t Lb = o.Lb;
    uint32_t* lp = reinterpret_cast<uint32_t*>(dsm);  // live old nodes before each chunk position
    uint32_t* nl = lp + kC;                             // new nodes at or before each chunk position
    uint32_t* ob = nl + kC;                             // old members of level Lb before each position
    if (lo >= hi) {  // an empty span: the new nodes before it
        if (tid < 32) {
            const uint32_t r = warp_count_below(s.ni, M, lo);
            if (tid == 0) sh.j1 = r;
        }
        __syncthreads();
        j0 = sh.j1;
        __syncthreads();
        return;
    }
    for (uint32_t w0 = lo; w0 < hi; w0 += kJbWin * kC) {
    const uint32_t wend = hi - w0 > kJbWin * kC ? w0 + kJbWin * kC : hi;
    const uint32_t nch = (wend - w0 + kC - 1u) / kC;
    for (uint32_t c = (uint32_t)tid >> 5; c <= nch; c += kW) {  // jb[c]: new nodes before chunk c
        const uint32_t bnd = c < nch ? w0 + c * kC : wend;
        const uint32_t r = warp_count_below(s.ni, M, bnd);
        if ((tid & 31) == 0) sh.jb[c] = r;
    }
    __syncthreads();
    for (uint32_t ci = 0; ci < nch; ++ci) {
        const uint32_t c0 = w0 + ci * kC;
        const uint32_t lim = c0 + kC < hi ? c0 + kC : hi;
        if (tid == 0 && lim < hi) {  // the next chunk's nodes into L2 while this one is copied
            const uint32_t nx = lim, nn = (hi - nx < kC ? hi - nx : kC);
            // nx is a multiple of the chunk, so every start is 16-byte aligned; sizes
            // round up to 16 bytes (the storage arrays are padded past their end)
            l2_prefetch(SK + nx, (nn * 8u + 15u) & ~15u);
            l2_prefetch(SV + nx, (nn * 8u + 15u) & ~15u);
            l2_prefetch(SM + nx, (nn + 15u) & ~15u);
        }
        j0 = sh.jb[ci];
        const uint32_t j1 = sh.jb[ci + 1];  // new nodes placed before an old node of this chunk: [j0, j1)
        for (uint32_t x = tid; x < kC; x += kT) nl[x] = 0u;
        __syncthreads();
        for (uint32_t j = j0 + tid; j < j1; j += kT) atomicAdd(&nl[s.ni[j] - c0], 1u);
        __syncthreads();
        // blocked: positions [kMI tid, kMI tid + kMI) of the chunk
        const uint32_t b0 = (uint32_t)tid * kMI, i0 = c0 + b0;
        uint32_t lmask = 0, omask = 0, nsum = 0;
        uint32_t nat[kMI];
        uint32_t hb[kMI];
        if (i0 + kMI <= size) {
            static_assert(kMI == 4 || kMI == 8, "one 4- or 8-byte load of a thread's meta bytes");
            uint32_t w[2];
            if constexpr (kMI == 8) {
                const uint2 w8 = *reinterpret_cast<const uint2*>(SM + i0);  // i0 is a multiple of 8
                w[0] = w8.x;
                w[1] = w8.y;
            } else {
                w[0] = *reinterpret_cast<const uint32_t*>(SM + i0);  // i0 is a multiple of 4
                w[1] = 0;
            }
#pragma unroll
            for (int k = 0; k < kMI; ++k) hb[k] = (w[k >> 2] >> (8 * (k & 3))) & 0xFFu;
        } else {
#pragma unroll
            for (int k = 0; k < kMI; ++k) hb[k] = i0 + k < size ? (uint32_t)SM[i0 + k] : (uint32_t)kTomb;
        }
#pragma unroll
        for (int k = 0; k < kMI; ++k) {
            if (i0 + k >= lim) hb[k] = kTomb;  // past the span: another span's node
            if (!(hb[k] & kTomb)) {
                lmask |= 1u << k;
                if (fused && (hb[k] & 0x3Fu) >= Lb) omask |= 1u << k;
            }
            nat[k] = nl[b0 + k];
            nsum += nat[k];
        }
        // one scan of three counts: live (bits 0-15), old members (16-31), new (32-63)
        uint64_t tot;
        const uint64_t ex = block_excl_sum64<kT>(
            (uint64_t)__popc(lmask) | ((uint64_t)__popc(omask) << 16) | ((uint64_t)nsum << 32), sh.tmp64, &tot);
        {
            uint32_t rl = carry + (uint32_t)(ex & 0xFFFFu), ro = cmem + (uint32_t)((ex >> 16) & 0xFFFFu);
            uint32_t rn = j0 + (uint32_t)(ex >> 32);
#pragma unroll
            for (int k = 0; k < kMI; ++k) {
                lp[b0 + k] = rl;
                ob[b0 + k] = ro;
                rl += (lmask >> k) & 1u;
                ro += (omask >> k) & 1u;
                rn += nat[k];
                nl[b0 + k] = rn;
            }
        }
        __syncthreads();
        // striped: the chunk's live old nodes, coalesced, four positions per round
        const uint32_t cnt = lim - c0;
        for (uint32_t x0 = tid; x0 < cnt; x0 += 4u * kT) {
            uint32_t mt[4];
            uint64_t kv[4], vv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const uint32_t x = x0 + (uint32_t)u * kT;
                const bool in = x < cnt;
                mt[u] = in ? (uint32_t)SM[c0 + x] : (uint32_t)kTomb;
                kv[u] = in ? SK[c0 + x] : 0ull;
                vv[u] = in ? SV[c0 + x] : 0ull;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (mt[u] & kTomb) continue;
                const uint32_t x = x0 + (uint32_t)u * kT;
                const uint32_t d = lp[x] + nl[x];
                o.DK[d] = kv[u];
                o.DV[d] = vv[u];
                o.DM[d] = (uint8_t)(mt[u] & 0x3Fu);
                if (fused && (mt[u] & 0x3Fu) >= Lb) {
                    const uint32_t r = ob[x] + o.nmp[nl[x]];
                    if (r < o.nLb) {
                        o.LK[o.lbase + r] = kv[u];
                        o.LD[o.lbase + r] = d;
                    }
                }
            }
        }
        for (uint32_t j = j0 + tid; j < j1; j += kT) {
            const uint32_t x = s.ni[j] - c0;
            const uint32_t d = j + lp[x];
            o.DK[d] = s.nk[j];
            o.DV[d] = s.nv[j];
            o.DM[d] = s.nh[j];
            if (fused && s.nh[j] >= Lb) {
                const uint32_t r = ob[x] + o.nmp[j];
                if (r < o.nLb) {
                    o.LK[o.lbase + r] = s.nk[j];
                    o.LD[o.lbase + r] = d;
                }
            }
        }
        carry += (uint32_t)(tot & 0xFFFFu);
        cmem += (uint32_t)((tot >> 16) & 0xFFFFu);
        j0 = j1;
        __syncthreads();
    }
    }
}

// The new nodes placed after the last old node: [j0, M), after `carry` live old nodes.
template <int kT>
__device__ void m_merge_tail(const MScratchPtrs& s, const MergeOut& o, uint32_t j0, uint32_t M, uint32_t carry,
                             uint32_t cmem) {
    for (uint32_t j = j0 + threadIdx.x; j < M; j += kT) {
        const uint32_t d = j + carry;
        o.DK[d] = s.nk[j];
        o.DV[d] = s.nv[j];
        o.DM[d] = s.nh[j];
        if (o.fused && s.nh[j] >= o.Lb) {
            const uint32_t r = cmem + o.nmp[j];
            if (r < o.nLb) {
                o.LK[o.lbase + r] = s.nk[j];
                o.LD[o.lbase + r] = d;
            }
        }
    }
}

// Live nodes and old members of level Lb (live, height >= Lb) in storage [lo, hi) (lo a
// multiple of 16), summed over the block: (live, members).
template <int kT>
__device__ uint2 m_count_nodes(const uint8_t* SM, uint32_t lo, uint32_t hi, uint32_t Lb, MShared& sh) {
    const int tid = threadIdx.x;
    uint32_t live = 0, mem = 0;
    for (uint32_t i0 = lo + (uint32_t)tid * 16u; i0 < hi; i0 += kT * 16u) {
        uint32_t w[4];
        if (i0 + 16u <= hi) {
            const uint4 v = *reinterpret_cast<const uint4*>(SM + i0);
            w[0] = v.x;
            w[1] = v.y;
            w[2] = v.z;
            w[3] = v.w;
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                w[q] = 0;
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    const uint32_t i = i0 + 4u * q + b;
                    w[q] |= (i < hi ? (uint32_t)SM[i] : (uint32_t)kTomb) << (8 * b);
                }
            }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const uint32_t mt = (w[q] >> (8 * b)) & 0xFFu;
                if (!(mt & kTomb)) {
                    ++live;
                    if ((mt & 0x3Fu) >= Lb) ++mem;
                }
            }
    }
    live = __reduce_add_sync(0xffffffffu, live);
    mem = __reduce_add_sync(0xffffffffu, mem);
    if (tid == 0) {
        sh.xs[0] = 0;
        sh.xs[1] = 0;
    }
    __syncthreads();
    if ((tid & 31) == 0) {
        atomicAdd(&sh.xs[0], live);
        atomicAdd(&sh.xs[1], mem);
    }
    __syncthreads();
    const uint2 r = make_uint2(sh.xs[0], sh.xs[1]);
    __syncthreads();
    return r;
}

// Level Lb from the storage layer: the live nodes of height >= Lb in [lo, hi), written
// from rank `carry` on (kWrite), or only counted. Returns carry + the span's members.
template <int kT, bool kWrite>
__device__ uint32_t m_level_from_storage(const uint64_t* RK, const uint8_t* RM, uint32_t Lb, uint32_t lo, uint32_t hi,
                                         uint32_t carry, uint64_t* LKb, uint32_t* LDb, uint32_t nLb, MShared& sh) {
    constexpr uint32_t kC = (uint32_t)kT * kMI;
    const int tid = threadIdx.x;
    for (uint32_t c0 = lo; c0 < hi; c0 += kC) {
        const uint32_t i0 = c0 + (uint32_t)tid * kMI;
        uint32_t mm = 0;
#pragma unroll
        for (int k = 0; k < kMI; ++k) {
            const uint32_t i = i0 + k;
            if (i < hi) {
                const uint8_t mt = RM[i];
                if (!(mt & kTomb) && (mt & 0x3Fu) >= Lb) mm |= 1u << k;
            }
        }
        uint32_t tot;
        uint32_t o = carry + block_excl_sum<kT>((uint32_t)__popc(mm), sh.tmp, &tot);
        if constexpr (kWrite) {
#pragma unroll
            for (int k = 0; k < kMI; ++k) {
                if (!((mm >> k) & 1u)) continue;
                if (o < nLb) {
                    LKb[o] = RK[i0 + k];
                    LDb[o] = i0 + k;
                }
                ++o;
            }
        }
        carry += tot;
    }
    return carry;
}

// Level l + 1 from level l: the entries of [lo, hi) of level l whose tower reaches l + 1,
// written from rank `carry` on (kWrite), or only counted. Returns carry + the span's.
template <int kT, bool kWrite>
__device__ uint32_t m_level_up(const uint64_t* LKl, uint64_t* LKu, uint32_t* LDu, uint32_t nu, uint32_t l,
                               uint32_t lo, uint32_t hi, uint32_t carry, const HashParams& hp, MShared& sh) {
    constexpr uint32_t kC = (uint32_t)kT * kMI;
    const int tid = threadIdx.x;
    for (uint32_t c0 = lo; c0 < hi; c0 += kC) {
        const uint32_t i0 = c0 + (uint32_t)tid * kMI;
        uint32_t mm = 0;
        uint64_t kk[kMI];
#pragma unroll
        for (int k = 0; k < kMI; ++k) {
            const uint32_t i = i0 + k;
            kk[k] = i < hi ? LKl[i] : 0ull;
            if (i < hi && tower_height(kk[k], hp) >= l + 1u) mm |= 1u << k;
        }
        uint32_t tot;
        uint32_t o = carry + block_excl_sum<kT>((uint32_t)__popc(mm), sh.tmp, &tot);
        if constexpr (kWrite) {
#pragma unroll
            for (int k = 0; k < kMI; ++k) {
                if (!((mm >> k) & 1u)) continue;
                if (o < nu) {
                    LKu[o] = kk[k];
                    LDu[o] = i0 + k;
                }
                ++o;
            }
        }
        carry += tot;
    }
    return carry;
}

// The sentinels of the built levels Lb..H (key 2^64-1; down = the size of the level
// below, the storage size for level Lb).
template <int kT>
__device__ void m_sentinels(const DevMeta& m, uint64_t* LK, uint32_t* LD) {
    for (uint32_t l = m.Lb + threadIdx.x; l <= m.H; l += kT) {
        const uint32_t sidx = m.base[l] + m.n[l];
        LK[sidx] = kMaxKey;
        LD[sidx] = (l > m.Lb) ? m.n[l - 1] : m.size;
    }
}

// Publishes the index's new state (one thread).
__device__ void m_publish(const MultiArgs& a, const MItem& it, const MIndex& X, const DevMeta& m) {
    DevMeta* gm = X.m;
    gm->cur = m.cur;
    gm->size = m.size;
    gm->tombs = m.tombs;
    gm->H = m.H;
    gm->Lb = m.Lb;
    gm->Ls = m.Ls;
    gm->smem_entries = m.smem_entries;
    gm->index_total = m.index_total;
    gm->index_need = m.index_need;
    gm->grow_request = m.grow_request;
    gm->updates = m.updates;
    gm->rebuilds = m.rebuilds;
    gm->levels_exact = m.levels_exact;
    gm->batches = m.batches;
    for (int l = 0; l < kLevelSlots; ++l) {
        gm->cnt[l] = m.cnt[l];
        gm->n[l] = m.n[l];
        gm->base[l] = m.base[l];
    }
    if (a.mirror) a.mirror[it.index] = *gm;  // the host reads the set's sizes from one copy
}

// Per-item shared state reset (every CTA that works on the item).
template <int kT>
__device__ void m_begin(const MIndex& X, MShared& sh) {
    const int tid = threadIdx.x;
    if (tid == 0) {
        sh.m = *X.m;
        sh.invalid = 0;
        sh.newc = 0;
        sh.dirty = 0;
        sh.changes = 0;
        sh.tomb_delta = 0;
    }
    if (tid < 8) {
        sh.bmax[tid] = 0;
        sh.bnmin[tid] = 0;
    }
    if (tid < kLevelSlots) sh.delta[tid] = 0;
    __syncthreads();
}

// Packs queries [lo, hi) of the batch into (key, op << 30 | arrival) and folds their
// byte-wise key extremes and invalid count into sh.bmax / sh.bnmin / sh.invalid (which
// the caller zeroed). An invalid query (op > 2 or the reserved key) sorts last.
template <int kT>
__device__ void m_pack(const MItem& it, const MScratchPtrs& s, uint32_t lo, uint32_t hi, MShared& sh) {
    const int lane = threadIdx.x & 31;
    uint32_t mx[8], mn[8], inv = 0;
#pragma unroll
    for (int d = 0; d < 8; ++d) mx[d] = mn[d] = 0;
    constexpr int kU = 4;  // queries a thread loads before it stores any
    for (uint32_t b0 = lo; b0 < hi; b0 += (uint32_t)kT * kU) {
        uint32_t op[kU];
        uint64_t kk[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const uint32_t i = b0 + (uint32_t)u * kT + threadIdx.x;
            op[u] = i < hi ? (uint32_t)it.ops[i] : 0xFFu;
            kk[u] = i < hi ? it.keys[i] : 0ull;
        }
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const uint32_t i = b0 + (uint32_t)u * kT + threadIdx.x;
            if (i >= hi) continue;
            const uint64_t k = kk[u];
            const bool valid = op[u] <= 2u && k != kMaxKey;
            s.ka[i] = valid ? k : kMaxKey;
            s.pa[i] = ((op[u] & 3u) << 30) | i;
            inv += valid ? 0u : 1u;
            if (valid) {
#pragma unroll
                for (int d = 0; d < 8; ++d) {
                    const uint32_t b = (uint32_t)(k >> (8 * d)) & 255u;
                    mx[d] = max(mx[d], b);
                    mn[d] = max(mn[d], 255u - b);
                }
            }
        }
    }
#pragma unroll
    for (int d = 0; d < 8; ++d) {
        mx[d] = __reduce_max_sync(0xffffffffu, mx[d]);
        mn[d] = __reduce_max_sync(0xffffffffu, mn[d]);
    }
    inv = __reduce_add_sync(0xffffffffu, inv);
    if (lane == 0) {
        if (inv) atomicAdd(&sh.invalid, inv);
#pragma unroll
        for (int d = 0; d < 8; ++d) {
            atomicMax(&sh.bmax[d], mx[d]);
            atomicMax(&sh.bnmin[d], mn[d]);
        }
    }
    __syncthreads();
}

// Segments of equal leading (pmask) bytes that hold two different keys, found from every
// key change i in [lo, hi) inside one (galloping back, then bisecting to its start): the
// starts are appended to seg through the counter nseg (a CTA's own shared memory, or rank
// 0's in a cluster); past kMSeg entries *overflow is set.
template <int kT>
__device__ void m_find_segments(const uint64_t* K, uint64_t pm, uint32_t lo, uint32_t hi, uint32_t* nseg,
                                uint32_t* seg, uint32_t* overflow) {
    for (uint32_t i = (lo ? lo : 1u) + threadIdx.x; i < hi; i += kT) {
        const uint64_t k0 = K[i - 1], k1 = K[i];
        if (k0 == k1 || ((k0 ^ k1) & pm) != 0) continue;
        const uint64_t mk = k1 & pm;
        uint32_t in = i - 1;
        uint64_t d = 1;
        while (d <= in && (K[in - d] & pm) == mk) {
            in -= (uint32_t)d;
            d <<= 1;
        }
        uint32_t a = d <= in ? in - (uint32_t)d + 1 : 0u, b = in;
        while (a < b) {
            const uint32_t mid = a + (b - a) / 2;
            if ((K[mid] & pm) == mk) b = mid;
            else a = mid + 1;
        }
        const uint32_t slot = atomicAdd(nseg, 1u);
        if (slot < kMSeg) seg[slot] = a;
        else *overflow = 1;
    }
}

// Orders the segments listed in sh.seg (sh.nseg of them, at most kMSeg) by the key bytes
// the prefix passes skipped, with stable one-CTA passes over each segment through the
// other buffer (K2, P2), so (K, P) ends sorted by the full key.
template <int kT, int kBits>
__device__ void m_fix_segments(uint64_t* K, uint32_t* P, uint64_t* K2, uint32_t* P2, uint32_t n, uint8_t* dsm,
                               MShared& sh, uint32_t* err) {
    const int tid = threadIdx.x;
    const uint64_t pm = sh.plan.pmask;
    if (tid == 0) {  // ascending and unique (several key changes share a segment)
        uint32_t m = sh.nseg, u = 0;
        for (uint32_t a = 1; a < m; ++a) {
            const uint32_t v = sh.seg[a];
            uint32_t b = a;
            while (b > 0 && sh.seg[b - 1] > v) {
                sh.seg[b] = sh.seg[b - 1];
                --b;
            }
            sh.seg[b] = v;
        }
        for (uint32_t a = 0; a < m; ++a)
            if (a == 0 || sh.seg[a] != sh.seg[u - 1]) sh.seg[u++] = sh.seg[a];
        sh.nseg = u;
    }
    __syncthreads();
    const uint32_t nseg = sh.nseg;
    for (uint32_t x = 0; x < nseg; ++x) {
        const uint32_t s0 = sh.seg[x];
        if (tid == 0) {  // the segment's end: gallop forward, then bisect
            const uint64_t mk = K[s0] & pm;
            uint32_t in = s0;
            uint64_t d = 1;
            while (d < n - in && (K[in + d] & pm) == mk) {
                in += (uint32_t)d;
                d <<= 1;
            }
            uint32_t lo = in + 1, hi = (d < n - in) ? in + (uint32_t)d : n;
            while (lo < hi) {
                const uint32_t mid = lo + (hi - lo) / 2;
                if ((K[mid] & pm) == mk) lo = mid + 1;
                else hi = mid;
            }
            sh.j1 = lo;
        }
        __syncthreads();
        const uint32_t e = sh.j1;
        // stable passes over the other bytes, ping-ponging through the other buffer
        uint64_t* A = K;
        uint32_t* AP = P;
        uint64_t* B = K2;
        uint32_t* BP = P2;
        for (uint32_t r = 0; r < sh.plan.nr; ++r)
            for (int sub = 0; sub < 8 / kBits; ++sub) {
                m_lsd_pass<kT, kBits>(A, AP, B, BP, s0, e, 8u * sh.plan.rdig[r] + (uint32_t)(sub * kBits), dsm,
                                      sh.tmp, err);
                uint64_t* tk = A; A = B; B = tk;
                uint32_t* tp = AP; AP = BP; BP = tp;
            }
        if (A != K)
            for (uint32_t i = s0 + tid; i < e; i += kT) {
                K[i] = A[i];
                P[i] = AP[i];
            }
        __syncthreads();
    }
}

// The plan's radix passes over one chunk (n <= kT x kMI) held in registers and shared
// memory: the chunk is read from (K, P) once, every pass ranks it by warp ballots and
// places it in digit order in shared memory, the next pass reads it back from there, and
// the result is written to (K, P) once. Stable, like the passes through global memory.
template <int kT, int kBits>
__device__ void m_sort_chunk_smem(uint64_t* K, uint32_t* P, uint32_t n, const SortPlan& plan, uint8_t* dsm,
                                  uint32_t* tmp) {
    constexpr int kW = kT / 32;
    constexpr int kR = 1 << kBits;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint32_t* whist = reinterpret_cast<uint32_t*>(dsm);  // [kW][kR]
    uint32_t* stot = whist + kW * kR + kR;               // [kR] (the layout of m_scatter)
    uint32_t* loff = stot + kR;                          // [kR]
    uint64_t* sk = reinterpret_cast<uint64_t*>(dsm + kSortStage);
    uint32_t* sp = reinterpret_cast<uint32_t*>(sk + (uint32_t)kT * kMI);
    uint64_t key[kMI];
    uint32_t pay[kMI];
#pragma unroll
    for (int k = 0; k < kMI; ++k) {
        const uint32_t i = (uint32_t)warp * 32u * kMI + (uint32_t)k * 32u + (uint32_t)lane;
        key[k] = i < n ? K[i] : 0ull;
        pay[k] = i < n ? P[i] : 0u;
    }
    for (int d = tid; d < kW * kR; d += kT) whist[d] = 0;
    __syncthreads();
    for (uint32_t j = 0; j < plan.npass; ++j)
        for (int sub = 0; sub < 8 / kBits; ++sub) {
            const uint32_t shift = 8u * plan.digit[j] + (uint32_t)(sub * kBits);
            uint32_t dig[kMI], rank[kMI];
#pragma unroll
            for (int k = 0; k < kMI; ++k) {
                const uint32_t i = (uint32_t)warp * 32u * kMI + (uint32_t)k * 32u + (uint32_t)lane;
                dig[k] = i < n ? (uint32_t)(key[k] >> shift) & (kR - 1) : (uint32_t)kR;
            }
            warp_digit_ranks<kMI, kBits>(dig, rank, whist + warp * kR);
            __syncthreads();
            for (int d = tid; d < kR; d += kT) {
                uint32_t total = 0;
#pragma unroll 4
                for (int w = 0; w < kW; ++w) {
                    const uint32_t cc = whist[w * kR + d];
                    whist[w * kR + d] = total;
                    total += cc;
                }
                stot[d] = total;
                loff[d] = total;
            }
            __syncthreads();
            small_excl_scan<kT, kR>(loff, tmp);
#pragma unroll
            for (int k = 0; k < kMI; ++k) {
                const uint32_t d = dig[k];
                if (d < (uint32_t)kR) {
                    const uint32_t l = loff[d] + whist[warp * kR + d] + rank[k];
                    sk[l] = key[k];
                    sp[l] = pay[k];
                }
            }
            __syncthreads();
#pragma unroll
            for (int k = 0; k < kMI; ++k) {
                const uint32_t i = (uint32_t)warp * 32u * kMI + (uint32_t)k * 32u + (uint32_t)lane;
                if (i < n) {
                    key[k] = sk[i];
                    pay[k] = sp[i];
                }
            }
            for (int d = tid; d < kW * kR; d += kT) whist[d] = 0;
            __syncthreads();
        }
#pragma unroll
    for (int k = 0; k < kMI; ++k) {
        const uint32_t i = (uint32_t)warp * 32u * kMI + (uint32_t)k * 32u + (uint32_t)lane;
        if (i < n) {
            K[i] = key[k];
            P[i] = pay[k];
        }
    }
    __syncthreads();
}

// Pack + sort of a whole batch by one CTA. Four passes on the most significant varying
// bytes, then the segments of equal leading bytes that hold different keys are ordered
// by the rest (as in the single-index sort). With more such segments than the list
// holds, the batch is packed again and sorted with every pass. Returns the buffer that
// holds the sorted (key, payload) pairs (K and P); sh.invalid counts the invalid queries.
template <int kT, int kBits>
__device__ void m_sort_cta(const MItem& it, const MScratchPtrs& s, uint8_t* dsm, MShared& sh, uint32_t* err,
                           uint64_t*& Kout, uint32_t*& Pout) {
    const int tid = threadIdx.x;
    const uint32_t n = it.n;
    uint64_t* K = s.ka;
    uint32_t* P = s.pa;
    for (uint32_t budget = 4; budget <= 8; budget += 4) {
        if (tid < 8) {
            sh.bmax[tid] = 0;
            sh.bnmin[tid] = 0;
        }
        if (tid == 0) {
            sh.invalid = 0;
            sh.nseg = 0;
            sh.overflow = 0;
        }
        __syncthreads();
        m_pack<kT>(it, s, 0, n, sh);
        if (tid == 0) plan_digits(sh.bmax, sh.bnmin, sh.invalid, n, budget, sh.plan);
        __syncthreads();
        K = s.ka;
        P = s.pa;
        uint64_t* K2 = s.kb;
        uint32_t* P2 = s.pb;
        if (n <= (uint32_t)kT * kMI) {
            m_sort_chunk_smem<kT, kBits>(K, P, n, sh.plan, dsm, sh.tmp);  // sorted in place
        } else {
            for (uint32_t j = 0; j < sh.plan.npass; ++j)
                for (int sub = 0; sub < 8 / kBits; ++sub) {
                    m_lsd_pass<kT, kBits>(K, P, K2, P2, 0u, n, 8u * sh.plan.digit[j] + (uint32_t)(sub * kBits),
                                          dsm, sh.tmp, err);
                    uint64_t* tk = K; K = K2; K2 = tk;
                    uint32_t* tp = P; P = P2; P2 = tp;
                }
        }
        if (!sh.plan.fix) break;
        m_find_segments<kT>(K, sh.plan.pmask, 1u, n, &sh.nseg, sh.seg, &sh.overflow);
        __syncthreads();
        if (sh.overflow) continue;  // pack again and sort with every pass
        m_fix_segments<kT, kBits>(K, P, K2, P2, n, dsm, sh, err);
        break;
    }
    Kout = K;
    Pout = P;
}

// ---------------------------------------------------------------------------------
// One CTA runs the whole pipeline of one batch.
template <int kT, int kBits>
__device__ void m_item(const MultiArgs& a, const MItem& it, const MScratchPtrs& s, uint8_t* dsm, MShared& sh) {
    const int tid = threadIdx.x;
    const MIndex& X = a.idx[it.index];
    const uint32_t n = it.n;
    uint32_t* err = &X.m->error;

    m_begin<kT>(X, sh);
    if (sh.m.error || n == 0) return;
    const uint32_t cur = sh.m.cur;
    uint64_t* SK = X.st.keys[cur];
    uint64_t* SV = X.st.vals[cur];
    uint8_t* SM = X.st.meta[cur];
    uint64_t* LK = sh.m.lcur ? X.lkeys1 : X.lkeys;  // the index layer's buffer in use
    uint32_t* LD = sh.m.lcur ? X.ldown1 : X.ldown;

    // ---- pack + sort
    uint64_t* K;
    uint32_t* P;
    m_sort_cta<kT, kBits>(it, s, dsm, sh, err, K, P);
    const uint32_t qv = n - sh.invalid;

    // ---- distinct keys of the valid prefix [0, qv); descent + locate for each
    const uint32_t D = m_distinct_span<kT>(K, qv, 0, qv, 0, s.dq, sh);
    __syncthreads();
    m_descend<kT>(X, s, sh.m, LK, LD, SK, SV, SM, D, 0, (uint32_t)kT * kMK, dsm, err);
    __syncthreads();

    // ---- results, ownership and apply
    const uint32_t M = m_apply_span<kT, true>(it, X, s, K, P, qv, 0, qv, ApplyCarry{0, 0, 0}, SV, SM, sh);
    for (uint32_t j = qv + tid; j < n; j += kT) mstore_result(it.results, P[j] & kMSeqMask, 0ull, PI_R_INVALID);
    if (tid == 0) sh.newc = M;
    __syncthreads();
    if (tid == 0) {
        DevMeta& m = sh.m;
        m.tombs = (uint32_t)((int32_t)m.tombs + sh.tomb_delta);
        for (int l = 1; l < kLevelSlots; ++l) m.cnt[l] = (uint32_t)((int32_t)m.cnt[l] + sh.delta[l]);
        m.updates += sh.changes;
        m.batches += 1;
    }
    __syncthreads();

    // ---- the new level layout (before the merge, which may write the lowest level)
    const bool merged = M > 0 || (sh.m.tombs > 0 && (uint64_t)sh.m.tombs * 8u > sh.m.size);
    const bool relevel = merged || sh.dirty;
    if (relevel) {
        if (tid == 0) m_layout(X, sh.m);
        __syncthreads();
    }
    // A merge rewrites the storage layer in key order, so it also writes the lowest built
    // level: each member's key and new storage position, at its rank among the members.
    const bool fused = merged && sh.m.Lb <= sh.m.H;

    // ---- merge: live old nodes and the new nodes into the other storage buffer
    if (merged) {
        const uint32_t size = sh.m.size;
        const uint32_t dst = cur ^ 1u;
        const uint32_t Lb = sh.m.Lb;
        uint32_t* nmp = s.dr;  // members among the first j new nodes (the descent's output is dead)
        if (fused) m_member_prefix<kT>(s, nmp, M, Lb, sh);
        const MergeOut o{X.st.keys[dst], X.st.vals[dst], X.st.meta[dst], LK, LD, nmp,
                         sh.m.base[Lb], sh.m.n[Lb], Lb, fused};
        uint32_t carry = 0, cmem = 0, j0 = 0;
        m_merge_span<kT>(s, SK, SV, SM, o, 0, size, size, M, carry, cmem, j0, dsm, sh);
        m_merge_tail<kT>(s, o, j0, M, carry, cmem);
        const uint32_t nsize = carry + M;
        if (tid == 0) {
            if (nsize > X.st_cap) atomicOr(err, kErrBounds);
            if (fused && cmem + nmp[M] != sh.m.n[Lb]) atomicOr(err, kErrBounds);
            o.DK[nsize] = kMaxKey;
            o.DV[nsize] = 0;
            o.DM[nsize] = 0;
            sh.m.size = nsize;
            sh.m.tombs = 0;
            sh.m.cur = dst;
        }
        __syncthreads();
    }

    // ---- rebuild the index layer when the membership of any level changed
    if (relevel) {
        __syncthreads();
        const DevMeta& m = sh.m;
        const uint32_t H = m.H, Lb = m.Lb, size = m.size;
        const uint32_t ncur = m.cur;
        if (Lb <= H) {
            // level Lb from the storage layer: live nodes of height >= Lb (a merge wrote it)
            if (!fused) {
                const uint32_t c = m_level_from_storage<kT, true>(X.st.keys[ncur], X.st.meta[ncur], Lb, 0, size, 0,
                                                                  LK + m.base[Lb], LD + m.base[Lb], m.n[Lb], sh);
                if (tid == 0 && c != m.n[Lb]) atomicOr(err, kErrBounds);
            }
            __syncthreads();
            // level l + 1 from level l: its members of height >= l + 1
            for (uint32_t l = Lb; l < H; ++l) {
                const uint32_t c = m_level_up<kT, true>(LK + m.base[l], LK + m.base[l + 1], LD + m.base[l + 1],
                                                        m.n[l + 1], l, 0, m.n[l], 0, X.hp, sh);
                if (tid == 0 && c != m.n[l + 1]) atomicOr(err, kErrBounds);
                __syncthreads();
            }
            m_sentinels<kT>(m, LK, LD);
        }
        __syncthreads();
    }

    // ---- publish the index's new state
    if (tid == 0) m_publish(a, it, X, sh.m);
    __syncthreads();
}

// ---------------------------------------------------------------------------------
// A thread-block cluster runs the pipeline of one large batch: each CTA takes one span
// of every stage (queries for the sort, distinct keys and apply; storage chunks for the
// merge and the level rebuild), and the carries between spans (prefix counts, the
// largest write marker) go through distributed shared memory at cluster barriers.
// Every CTA keeps the same copy of the index's meta, updated from the cluster totals.
// All decisions that pick a code path depend only on values every CTA shares, so all
// CTAs reach the same barriers.
struct CXShared {
    uint32_t hist[2][256];      // per-CTA digit counts of a sort pass (alternating)
    uint32_t v[2][kXMax];       // per-CTA values of an exchange (alternating)
    uint32_t pre[kXMax];        // exchange results: over the lower ranks
    uint32_t tot[kXMax];        //   and over the whole cluster
    uint32_t item;              // rank 0's queue slot
};

// Exchange of nv values per CTA (sh-resident, uniform within the CTA): afterwards
// cx.pre[k] holds the sum (the maximum, for bit k of maxmask) over the lower ranks and
// cx.tot[k] over the cluster. The cluster barrier inside also orders every global and
// shared write before it for all CTAs of the cluster.
__device__ void cl_exchange(const cg::cluster_group& cl, CXShared& cx, uint32_t& ph, const uint32_t* v, int nv,
                            uint64_t maxmask) {
    uint32_t* slot = cx.v[ph & 1u];
    ++ph;
    const int tid = threadIdx.x;
    if (tid < nv) slot[tid] = v[tid];
    cl.sync();
    if (tid < nv) {
        const uint32_t me = cl.block_rank(), C = cl.num_blocks();
        const bool mx = (maxmask >> tid) & 1u;
        uint32_t x[16];
#pragma unroll
        for (uint32_t r = 0; r < 16; ++r) x[r] = r < C ? cl.map_shared_rank(slot, r)[tid] : 0u;  // loads in flight together
        uint32_t p = 0, t = 0;
#pragma unroll
        for (uint32_t r = 0; r < 16; ++r) {
            t = mx ? max(t, x[r]) : t + x[r];
            if (r < me) p = mx ? max(p, x[r]) : p + x[r];
        }
        cx.pre[tid] = p;
        cx.tot[tid] = t;
    }
    __syncthreads();
}

// First element of rank r's share of [0, n) split in C parts, in whole chunks of `al`.
__device__ __forceinline__ uint32_t cl_split(uint32_t n, uint32_t r, uint32_t C, uint32_t al) {
    const uint32_t nch = (n + al - 1u) / al;
    const uint32_t c = (uint32_t)((uint64_t)nch * r / C);
    return min(n, c * al);
}

// One stable LSD pass of the cluster over [0, n): every CTA histograms its span, the
// bases of its digits are the counts of all smaller digits plus those of its digit in
// the lower ranks, then it scatters its span.
template <int kT, int kBits>
__device__ void cl_lsd_pass(const cg::cluster_group& cl, CXShared& cx, uint32_t& hph, const uint64_t* src_k,
                            const uint32_t* src_p, uint64_t* dst_k, uint32_t* dst_p, uint32_t lo, uint32_t hi,
                            uint32_t n, uint32_t shift, uint8_t* dsm, uint32_t* tmp, uint32_t* err) {
    constexpr int kW = kT / 32;
    constexpr int kR = 1 << kBits;
    const int tid = threadIdx.x;
    uint32_t* sbase = reinterpret_cast<uint32_t*>(dsm) + kW * kR;
    uint32_t* stot = sbase + kR;
    uint32_t* h = cx.hist[hph & 1u];
    ++hph;
    for (int d = tid; d < kR; d += kT) h[d] = 0;
    __syncthreads();
    m_histogram<kT, kBits>(src_k, lo, hi, shift, h);
    cl.sync();
    uint32_t pre = 0;
    if (tid < kR) {
        const uint32_t me = cl.block_rank(), C = cl.num_blocks();
        uint32_t x[16];
#pragma unroll
        for (uint32_t r = 0; r < 16; ++r) x[r] = r < C ? cl.map_shared_rank(h, r)[tid] : 0u;  // loads in flight together
        uint32_t t = 0;
#pragma unroll
        for (uint32_t r = 0; r < 16; ++r) {
            t += x[r];
            if (r < me) pre += x[r];
        }
        stot[tid] = t;
    }
    __syncthreads();
    small_excl_scan<kT, kR>(stot, tmp);
    if (tid < kR) sbase[tid] = stot[tid] + pre;
    m_scatter<kT, kBits>(src_k, src_p, dst_k, dst_p, lo, hi, shift, n, dsm, tmp, err);
    cl.sync();
}

template <int kT, int kBits>
__device__ void m_item_cl(const cg::cluster_group& cl, const MultiArgs& a, const MItem& it, const MScratchPtrs& s,
                          uint8_t* dsm, MShared& sh, CXShared& cx) {
    constexpr uint32_t kC = (uint32_t)kT * kMI;
    const int tid = threadIdx.x;
    const uint32_t me = cl.block_rank(), C = cl.num_blocks();
    const MIndex& X = a.idx[it.index];
    const uint32_t n = it.n;
    uint32_t* err = &X.m->error;
    uint32_t ph = 0, hph = 0;

    // Every CTA reads the index's meta before the first cluster barrier; no CTA of the
    // cluster writes it before that barrier, so all start from the same copy.
    m_begin<kT>(X, sh);
    if (sh.m.error || n == 0) return;
    const uint32_t cur = sh.m.cur;
    uint64_t* SK = X.st.keys[cur];
    uint64_t* SV = X.st.vals[cur];
    uint8_t* SM = X.st.meta[cur];
    uint64_t* LK = sh.m.lcur ? X.lkeys1 : X.lkeys;
    uint32_t* LD = sh.m.lcur ? X.ldown1 : X.ldown;

    // ---- pack + sort. A batch of at most two chunks is sorted by rank 0 alone (a cluster
    // pass costs two cluster barriers and an exchange, more than a chunk's ranking); a
    // larger one by the cluster.
    uint64_t* K = s.ka;
    uint32_t* P = s.pa;
    if (n <= 2 * kC) {
        if (me == 0) m_sort_cta<kT, kBits>(it, s, dsm, sh, err, K, P);
        if (tid == 0) {
            sh.xs[0] = (me == 0 && K != s.ka) ? 1u : 0u;  // rank 0's result buffer
            sh.xs[1] = me == 0 ? sh.invalid : 0u;
        }
        __syncthreads();
        cl_exchange(cl, cx, ph, sh.xs, 2, 0ull);
        K = cx.tot[0] ? s.kb : s.ka;
        P = cx.tot[0] ? s.pb : s.pa;
        if (tid == 0) sh.invalid = cx.tot[1];
        __syncthreads();
    } else {
        // four cluster passes on the most significant varying bytes; the key-prefix
        // segments they leave are collected on rank 0 and ordered there (with more than
        // its list holds, the batch is packed again and sorted with every byte)
        const uint32_t plo = (uint32_t)((uint64_t)n * me / C), phi = (uint32_t)((uint64_t)n * (me + 1) / C);
        uint32_t* rnseg = cl.map_shared_rank(&sh.nseg, 0);
        uint32_t* rseg = cl.map_shared_rank(sh.seg, 0);
        uint32_t* rover = cl.map_shared_rank(&sh.overflow, 0);
        for (uint32_t budget = 4; budget <= 8; budget += 4) {
            if (tid < 8) {
                sh.bmax[tid] = 0;
                sh.bnmin[tid] = 0;
            }
            if (tid == 0) {
                sh.invalid = 0;
                sh.nseg = 0;  // rank 0's list: the others append only after the exchange below
                sh.overflow = 0;
            }
            __syncthreads();
            m_pack<kT>(it, s, plo, phi, sh);
            if (tid == 0) {
                for (int d = 0; d < 8; ++d) {
                    sh.xs[d] = sh.bmax[d];
                    sh.xs[8 + d] = sh.bnmin[d];
                }
                sh.xs[16] = sh.invalid;
            }
            __syncthreads();
            cl_exchange(cl, cx, ph, sh.xs, 17, 0xFFFFull);
            if (tid == 0) {
                for (int d = 0; d < 8; ++d) {
                    sh.bmax[d] = cx.tot[d];
                    sh.bnmin[d] = cx.tot[8 + d];
                }
                sh.invalid = cx.tot[16];
                plan_digits(sh.bmax, sh.bnmin, sh.invalid, n, budget, sh.plan);
            }
            __syncthreads();
            K = s.ka;
            P = s.pa;
            uint64_t* K2 = s.kb;
            uint32_t* P2 = s.pb;
            for (uint32_t j = 0; j < sh.plan.npass; ++j)
                for (int sub = 0; sub < 8 / kBits; ++sub) {
                    cl_lsd_pass<kT, kBits>(cl, cx, hph, K, P, K2, P2, plo, phi, n,
                                           8u * sh.plan.digit[j] + (uint32_t)(sub * kBits), dsm, sh.tmp, err);
                    uint64_t* tk = K; K = K2; K2 = tk;
                    uint32_t* tp = P; P = P2; P2 = tp;
                }
            if (!sh.plan.fix) break;
            m_find_segments<kT>(K, sh.plan.pmask, plo, phi, rnseg, rseg, rover);
            cl.sync();  // rank 0's list complete
            if (tid == 0) sh.xs[0] = me == 0 ? sh.overflow : 0u;
            __syncthreads();
            cl_exchange(cl, cx, ph, sh.xs, 1, 0ull);
            if (cx.tot[0]) continue;  // pack again and sort with every byte
            if (me == 0) m_fix_segments<kT, kBits>(K, P, K2, P2, n, dsm, sh, err);
            cl.sync();  // the segments ordered
            break;
        }
    }
    const uint32_t qv = n - sh.invalid;

    // ---- per span of [0, qv): the largest write/head marker and the run heads
    const uint32_t alo = (uint32_t)((uint64_t)qv * me / C), ahi = (uint32_t)((uint64_t)qv * (me + 1) / C);
    {
        uint32_t mx = 0, hc = 0;
        for (uint32_t j = alo + tid; j < ahi; j += kT) {
            const uint64_t kk = K[j];
            const bool head = j == 0 || K[j - 1] != kk;
            const uint32_t op = P[j] >> 30;
            const uint32_t e = (op == 1u || op == 2u) ? 2u * j + 3u : (head ? 2u * j + 2u : 0u);
            mx = max(mx, e);
            hc += head ? 1u : 0u;
        }
        mx = __reduce_max_sync(0xffffffffu, mx);
        hc = __reduce_add_sync(0xffffffffu, hc);
        if (tid == 0) {
            sh.xs[0] = 0;
            sh.xs[1] = 0;
        }
        __syncthreads();
        if ((tid & 31) == 0) {
            atomicMax(&sh.xs[0], mx);
            atomicAdd(&sh.xs[1], hc);
        }
        __syncthreads();
    }
    cl_exchange(cl, cx, ph, sh.xs, 2, 0x1ull);
    const ApplyCarry c0{cx.pre[0], cx.pre[1], 0u};
    const uint32_t D = cx.tot[1];
    m_distinct_span<kT>(K, qv, alo, ahi, c0.cheads, s.dq, sh);
    cl.sync();  // every distinct key written

    // ---- descent: the CTAs take interleaved groups of kT x kMK distinct keys
    m_descend<kT>(X, s, sh.m, LK, LD, SK, SV, SM, D, me * (uint32_t)kT * kMK, C * (uint32_t)kT * kMK, dsm, err);
    cl.sync();  // every distinct key located

    // ---- apply: count the span's new nodes, exchange, then the full pass
    {
        const uint32_t cnt = m_apply_span<kT, false>(it, X, s, K, P, qv, alo, ahi, c0, SV, SM, sh);
        if (tid == 0) sh.xs[0] = cnt;
        __syncthreads();
    }
    cl_exchange(cl, cx, ph, sh.xs, 1, 0ull);
    const uint32_t M = cx.tot[0];
    m_apply_span<kT, true>(it, X, s, K, P, qv, alo, ahi, ApplyCarry{c0.cmax, c0.cheads, cx.pre[0]}, SV, SM, sh);
    for (uint32_t j = qv + me * (uint32_t)kT + tid; j < n; j += C * (uint32_t)kT)
        mstore_result(it.results, P[j] & kMSeqMask, 0ull, PI_R_INVALID);
    __syncthreads();
    // the node changes of every span: dirty, changes, tomb delta, per-level deltas
    if (tid == 0) {
        sh.xs[0] = sh.dirty;
        sh.xs[1] = sh.changes;
        sh.xs[2] = (uint32_t)sh.tomb_delta;
    }
    if (tid < kLevelSlots) sh.xs[3 + tid] = (uint32_t)sh.delta[tid];
    __syncthreads();
    cl_exchange(cl, cx, ph, sh.xs, 3 + kLevelSlots, 0x1ull);
    const bool dirty = cx.tot[0] != 0;
    if (tid == 0) {
        DevMeta& m = sh.m;
        m.tombs = (uint32_t)((int32_t)m.tombs + (int32_t)cx.tot[2]);
        for (int l = 1; l < kLevelSlots; ++l) m.cnt[l] = (uint32_t)((int32_t)m.cnt[l] + (int32_t)cx.tot[3 + l]);
        m.updates += cx.tot[1];
        m.batches += 1;
        sh.newc = M;
    }
    __syncthreads();
    const bool merged = M > 0 || (sh.m.tombs > 0 && (uint64_t)sh.m.tombs * 8u > sh.m.size);
    const bool relevel = merged || dirty;
    if (relevel) {
        if (tid == 0) m_layout(X, sh.m);
        __syncthreads();
    }
    const bool fused = merged && sh.m.Lb <= sh.m.H;

    // ---- merge over chunk-aligned spans of the old storage layer
    if (merged) {
        const uint32_t size = sh.m.size;
        const uint32_t dst = cur ^ 1u;
        const uint32_t Lb = sh.m.Lb;
        uint32_t* nmp = s.dr;  // every CTA has read the descent's output (exchange above)
        if (fused && me == 0) m_member_prefix<kT>(s, nmp, M, Lb, sh);
        const uint32_t slo = cl_split(size, me, C, kC), shi = cl_split(size, me + 1, C, kC);
        const uint2 cnt = m_count_nodes<kT>(SM, slo, shi, fused ? Lb : 64u, sh);
        if (tid == 0) {
            sh.xs[0] = cnt.x;
            sh.xs[1] = cnt.y;
        }
        __syncthreads();
        cl_exchange(cl, cx, ph, sh.xs, 2, 0ull);  // also publishes rank 0's member prefix
        uint32_t carry = cx.pre[0], cmem = cx.pre[1];
        const uint32_t live_tot = cx.tot[0], mem_tot = cx.tot[1];
        uint32_t j0 = 0;  // set by the span: the new nodes placed before its end
        const MergeOut o{X.st.keys[dst], X.st.vals[dst], X.st.meta[dst], LK, LD, nmp,
                         sh.m.base[Lb], sh.m.n[Lb], Lb, fused};
        m_merge_span<kT>(s, SK, SV, SM, o, slo, shi, size, M, carry, cmem, j0, dsm, sh);
        const uint32_t nsize = live_tot + M;
        if (me == C - 1) {
            m_merge_tail<kT>(s, o, j0, M, live_tot, mem_tot);
            if (tid == 0) {
                if (nsize > X.st_cap) atomicOr(err, kErrBounds);
                if (fused && mem_tot + nmp[M] != sh.m.n[Lb]) atomicOr(err, kErrBounds);
                o.DK[nsize] = kMaxKey;
                o.DV[nsize] = 0;
                o.DM[nsize] = 0;
            }
        }
        if (tid == 0) {
            sh.m.size = nsize;
            sh.m.tombs = 0;
            sh.m.cur = dst;
        }
        cl.sync();  // the new storage layer (and level Lb) complete
    }

    // ---- rebuild: level Lb and the large levels above it by spans, the rest by rank 0
    if (relevel) {
        const DevMeta& m = sh.m;
        const uint32_t H = m.H, Lb = m.Lb, size = m.size;
        const uint32_t ncur = m.cur;
        if (Lb <= H) {
            if (!fused) {
                const uint64_t* RK = X.st.keys[ncur];
                const uint8_t* RM = X.st.meta[ncur];
                const uint32_t slo = cl_split(size, me, C, kC), shi = cl_split(size, me + 1, C, kC);
                const uint32_t c = m_level_from_storage<kT, false>(RK, RM, Lb, slo, shi, 0, nullptr, nullptr, 0, sh);
                if (tid == 0) sh.xs[0] = c;
                __syncthreads();
                cl_exchange(cl, cx, ph, sh.xs, 1, 0ull);
                const uint32_t pre = cx.pre[0], tot = cx.tot[0];
                m_level_from_storage<kT, true>(RK, RM, Lb, slo, shi, pre, LK + m.base[Lb], LD + m.base[Lb], m.n[Lb],
                                               sh);
                if (me == 0 && tid == 0 && tot != m.n[Lb]) atomicOr(err, kErrBounds);
                cl.sync();  // level Lb complete
            }
            uint32_t l = Lb;
            for (; l < H; ++l) {
                const uint32_t nl = m.n[l];
                if (nl < C * kC) break;  // the remaining levels are small: rank 0 alone
                const uint32_t slo = cl_split(nl, me, C, kC), shi = cl_split(nl, me + 1, C, kC);
                const uint32_t c = m_level_up<kT, false>(LK + m.base[l], nullptr, nullptr, 0, l, slo, shi, 0, X.hp, sh);
                if (tid == 0) sh.xs[0] = c;
                __syncthreads();
                cl_exchange(cl, cx, ph, sh.xs, 1, 0ull);
                const uint32_t pre = cx.pre[0], tot = cx.tot[0];
                m_level_up<kT, true>(LK + m.base[l], LK + m.base[l + 1], LD + m.base[l + 1], m.n[l + 1], l, slo, shi,
                                     pre, X.hp, sh);
                if (me == 0 && tid == 0 && tot != m.n[l + 1]) atomicOr(err, kErrBounds);
                cl.sync();  // level l + 1 complete
            }
            if (me == 0) {
                for (; l < H; ++l) {
                    const uint32_t c = m_level_up<kT, true>(LK + m.base[l], LK + m.base[l + 1], LD + m.base[l + 1],
                                                            m.n[l + 1], l, 0, m.n[l], 0, X.hp, sh);
                    if (tid == 0 && c != m.n[l + 1]) atomicOr(err, kErrBounds);
                    __syncthreads();
                }
                m_sentinels<kT>(m, LK, LD);
            }
        }
    }
    if (me == 0) {
        __syncthreads();
        if (tid == 0) m_publish(a, it, X, sh.m);
    }
    __syncthreads();
}

template <int kW, int kBits>
__global__ void __launch_bounds__(kW * 32) k_multi(MultiArgs a) {
    constexpr int kT = kW * 32;
    extern __shared__ __align__(16) uint8_t dsm[];
    __shared__ MShared sh;
    const MScratchPtrs s = carve(a.scratch + (uint64_t)blockIdx.x * a.stride, a.qcap);
    const uint32_t nitems = *a.nitems;
    for (;;) {
        if (threadIdx.x == 0) sh.item = atomicAdd(a.head, 1u);
        __syncthreads();
        const uint32_t item = sh.item;
        __syncthreads();
        if (item >= nitems) break;
        const MItem it = a.items[item];
        if (it.n <= a.qcap) m_item<kT, kBits>(a, it, s, dsm, sh);
        else if (threadIdx.x == 0) atomicOr(&a.idx[it.index].m->error, kErrBounds);
        __syncthreads();
    }
}

// Clusters of CTAs take batches from the queue; the scratch is per cluster.
template <int kW, int kBits>
__global__ void __launch_bounds__(kW * 32) k_multi_cl(MultiArgs a) {
    constexpr int kT = kW * 32;
    extern __shared__ __align__(16) uint8_t dsm[];
    __shared__ MShared sh;
    __shared__ CXShared cx;
    const cg::cluster_group cl = cg::this_cluster();
    const uint32_t me = cl.block_rank(), C = cl.num_blocks();
    const MScratchPtrs s = carve(a.scratch + (uint64_t)(blockIdx.x / C) * a.stride, a.qcap);
    const uint32_t nitems = *a.nitems;
    cl.sync();  // every CTA of the cluster runs before any reads another's shared memory
    for (;;) {
        if (me == 0 && threadIdx.x == 0) cx.item = atomicAdd(a.head, 1u);
        cl.sync();
        const uint32_t item = *cl.map_shared_rank(&cx.item, 0);
        if (item >= nitems) break;
        const MItem it = a.items[item];
        if (it.n <= a.qcap) m_item_cl<kT, kBits>(cl, a, it, s, dsm, sh, cx);
        else if (me == 0 && threadIdx.x == 0) atomicOr(&a.idx[it.index].m->error, kErrBounds);
        cl.sync();  // rank 0 takes the next slot only after every CTA has read this one
    }
    cl.sync();  // no CTA leaves while another may still read its shared memory
}

template <int kW, int kBits>
constexpr int multi_smem() {
    constexpr int kT = kW * 32;
    constexpr int sort = (int)kSortStage + kT * kMI * 12;  // counters, then the staged chunk
    constexpr int top = (int)kMTop * 12;
    constexpr int merge = kT * kMI * 12;  // live, new-node and member prefixes per chunk position
    return sort > top ? (sort > merge ? sort : merge) : (top > merge ? top : merge);
}

// Sets the kernels' dynamic shared-memory limit (before any capture) and returns the
// largest grid (CTAs) that is resident at once: CTAs per SM x SMs, or for clusters of
// `cluster` CTAs the resident clusters x cluster.
template <int kW, int kBits>
cudaError_t grid_t(int cluster, int num_sms, uint32_t* grid) {
    constexpr int dyn = multi_smem<kW, kBits>();
    if (cluster <= 1) {
        cudaError_t e = cudaFuncSetAttribute(k_multi<kW, kBits>, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
        if (e != cudaSuccess) return e;
        int blocks = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_multi<kW, kBits>, kW * 32, dyn);
        *grid = (uint32_t)(blocks > 0 ? blocks : 0) * (uint32_t)num_sms;
        return e;
    }
    if constexpr ((kW != 16 && kW != 32) || kBits != 8) {
        return cudaErrorInvalidValue;  // clusters run the 16- and 32-warp, 8-bit variants only
    } else {
    cudaError_t e = cudaFuncSetAttribute(k_multi_cl<kW, kBits>, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
    if (e == cudaSuccess && cluster > 8)
        e = cudaFuncSetAttribute(k_multi_cl<kW, kBits>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)cluster;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3((unsigned)(cluster * num_sms));
    cfg.blockDim = dim3(kW * 32);
    cfg.dynamicSmemBytes = dyn;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int clusters = 0;
    e = cudaOccupancyMaxActiveClusters(&clusters, k_multi_cl<kW, kBits>, &cfg);
    *grid = (uint32_t)(clusters > 0 ? clusters : 0) * (uint32_t)cluster;
    return e;
    }
}

template <int kW, int kBits>
cudaError_t launch_t(const MultiArgs& a, int cluster, uint32_t grid, cudaStream_t s) {
    if (cluster <= 1) {
        k_multi<kW, kBits><<<grid, kW * 32, multi_smem<kW, kBits>(), s>>>(a);
    } else if constexpr ((kW != 16 && kW != 32) || kBits != 8) {
        return cudaErrorInvalidValue;
    } else {
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = (unsigned)cluster;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(grid);
        cfg.blockDim = dim3(kW * 32);
        cfg.dynamicSmemBytes = multi_smem<kW, kBits>();
        cfg.stream = s;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        cudaError_t e = cudaLaunchKernelEx(&cfg, k_multi_cl<kW, kBits>, a);
        if (e != cudaSuccess) return e;
    }
    ++g_launches;
    return cudaGetLastError();
}

}  // namespace

uint64_t multi_scratch_bytes(uint32_t qcap) {
    const uint64_t c = (uint64_t)qcap + kPad;
    auto al = [](uint64_t b) { return (b + 255u) & ~255ull; };
    return 2 * al(c * 8) + 2 * al(c * 4) + al(c * 8) + al(c * 4) + al(c) + al(c * 8) + 2 * al(c * 8) + al(c) +
           al(c * 4);
}

bool multi_variant_ok(int warps, int radix_bits, int cluster) {
    const bool base = (warps == 8 || warps == 16 || warps == 32) && (radix_bits == 4 || radix_bits == 8);
    if (cluster <= 1) return base;
    return (warps == 16 || warps == 32) && radix_bits == 8 &&
           (cluster == 2 || cluster == 4 || cluster == 8 || cluster == 16);
}

// multi_grid must have run for the variant first (it sets the shared-memory limit).
cudaError_t launch_multi(const MultiArgs& a, int warps, int radix_bits, int cluster, uint32_t grid, cudaStream_t s) {
    if (grid == 0) return cudaSuccess;
    if (!multi_variant_ok(warps, radix_bits, cluster)) return cudaErrorInvalidValue;
    if (cluster > 1) return warps == 16 ? launch_t<16, 8>(a, cluster, grid, s) : launch_t<32, 8>(a, cluster, grid, s);
    if (radix_bits == 8) {
        if (warps == 8) return launch_t<8, 8>(a, 1, grid, s);
        if (warps == 16) return launch_t<16, 8>(a, 1, grid, s);
        return launch_t<32, 8>(a, 1, grid, s);
    }
    if (warps == 8) return launch_t<8, 4>(a, 1, grid, s);
    if (warps == 16) return launch_t<16, 4>(a, 1, grid, s);
    return launch_t<32, 4>(a, 1, grid, s);
}

cudaError_t multi_grid(int warps, int radix_bits, int cluster, int num_sms, uint32_t* grid) {
    *grid = 0;
    if (!multi_variant_ok(warps, radix_bits, cluster)) return cudaErrorInvalidValue;
    if (cluster > 1) return warps == 16 ? grid_t<16, 8>(cluster, num_sms, grid) : grid_t<32, 8>(cluster, num_sms, grid);
    if (radix_bits == 8) {
        if (warps == 8) return grid_t<8, 8>(1, num_sms, grid);
        if (warps == 16) return grid_t<16, 8>(1, num_sms, grid);
        return grid_t<32, 8>(1, num_sms, grid);
    }
    if (warps == 8) return grid_t<8, 4>(1, num_sms, grid);
    if (warps == 16) return grid_t<16, 4>(1, num_sms, grid);
    return grid_t<32, 4>(1, num_sms, grid);
}

}  // namespace pi
