// K2 + K3: descend the index layer to each query's interception (Algorithm 2,
// Definition 4), then locate the query's key in the storage layer (Algorithm 4's
// getNode), for every distinct key of the sorted batch.
//
// Layout (built by the rebuild): all index levels live in one key array and one down
// array, top level first; level l is [base[l], base[l] + n[l]) followed by a sentinel
// entry with key 2^64-1. down[i] is the position of the same key in the level below
// (for the lowest built level: its storage-layer position), so the keys of level l-1
// that lie between two consecutive keys of level l are exactly
// [down[r], down[r + 1]).
//
// The descent is level-synchronous over the whole batch -- the paper's group query
// processing (Section 4.4.3) with the group being every distinct key of the batch:
//  k_heads      one persistent kernel: the distinct keys (local run heads: a query
//               whose key differs from the previous one, or the first query of a
//               256-query sub-tile), their dense index by a decoupled look-back over
//               the apply tiles, the tiles' ownership-marker prefixes for k_apply, and
//               each key's start position below the levels pinned in shared memory
//               (staged once per CTA by TMA bulk copies): one binary search of the
//               lowest pinned level, which holds every key of the levels above it;
//  k_level      one launch per remaining index level: every key scans its gap;
//  k_locate     the storage layer: the node with the largest key <= q, and its state.
// Each launch is one independent gather per key, so hundreds of thousands of keys are
// in flight at once. Within a warp, when the 32 keys' start positions lie within 8
// entries (upper levels: the keys are sorted), the warp loads one 32-key segment with
// one coalesced access and each lane ranks its key in it by a binary search over the
// lanes (the SIMD-compare analogue of Section 3.2.1); otherwise each lane scans its own
// gap four keys (and downs) per round. Both end at the level's sentinel.

#include "common.cuh"

namespace pi {
namespace {

constexpr int kThreads = 256;
constexpr uint32_t kFull = 0xffffffffu;

// r = largest index >= lo-1 with K[r] <= q (K[lo] <= q unless lo is the head, 0).
// Also returns D[r] (0 if r < 0 or no down array) and K[r], and the next entry's
// K[r + 1] and D[r + 1] (the first key above q; at the level's sentinel, key 2^64-1 and
// for the lowest built level the storage size). Each round reads kWide
// consecutive entries with 16-byte loads (keys) and 8-byte loads (downs): 4 on index
// levels, 16 (one 128-byte line) on the storage layer, whose gaps below the lowest built level span
// (1/P)^(Lb-1) nodes. The loads need &K[i] 16-byte aligned (K and D come from arrays
// whose bases are, and a level may start at any entry), so an odd start steps back one
// entry, which is <= q, or, at the head of a level, tests the head on its own.
template <bool kDown, int kWide>
__device__ __forceinline__ void lane_scan(const uint64_t* K, const uint32_t* D, uint32_t lo, uint32_t lim,
                                          uint64_t q, int32_t& r_out, uint32_t& d_out, uint64_t& k_out,
                                          uint64_t& kn_out, uint32_t& dn_out, uint32_t* err) {
    static_assert(kWide % 2 == 0, "whole 16-byte key pairs and 8-byte down pairs");
    uint32_t i = lo, dprev = 0;
    uint64_t kprev = 0;
    if ((reinterpret_cast<uintptr_t>(K + i) & 15u) != 0) {
        if (i > 0) {
            --i;
        } else {
            const uint64_t k0 = K[0];
            if (k0 > q) {
                r_out = -1;
                d_out = 0;
                k_out = 0;
                kn_out = k0;
                dn_out = kDown ? D[0] : 0u;
                return;
            }
            kprev = k0;
            dprev = kDown ? D[0] : 0u;
            i = 1;
        }
    }
    for (;;) {
        if (i > lim) {
            atomicOr(err, kErrBounds);
            r_out = -1;
            d_out = 0;
            k_out = 0;
            kn_out = kMaxKey;
            dn_out = 0;
            return;
        }
        uint64_t kk[kWide];
        uint32_t dd[kWide];
        const ulonglong2* kp = reinterpret_cast<const ulonglong2*>(K + i);
#pragma unroll
        for (int j = 0; j < kWide / 2; ++j) {
            const ulonglong2 v = kp[j];
            kk[2 * j] = v.x;
            kk[2 * j + 1] = v.y;
        }
        if (kDown) {
            const uint2* dp = reinterpret_cast<const uint2*>(D + i);
#pragma unroll
            for (int j = 0; j < kWide / 2; ++j) {
                const uint2 v = dp[j];
                dd[2 * j] = v.x;
                dd[2 * j + 1] = v.y;
            }
        } else {
#pragma unroll
            for (int j = 0; j < kWide; ++j) dd[j] = 0u;
        }
        uint32_t gt = 0;  // bit j: kk[j] > q (the keys are sorted, so the bits are a suffix)
#pragma unroll
        for (int j = 0; j < kWide; ++j) gt |= (kk[j] > q ? 1u : 0u) << j;
        if (gt) {
            const int f = __ffs(gt) - 1;
            uint32_t dsel = dprev, dnext = dd[0];
            uint64_t ksel = kprev, knext = kk[0];
#pragma unroll
            for (int j = 1; j < kWide; ++j) {
                if (j == f) {
                    dsel = dd[j - 1];
                    ksel = kk[j - 1];
                    dnext = dd[j];
                    knext = kk[j];
                }
            }
            r_out = (int32_t)(i + (uint32_t)f) - 1;
            d_out = dsel;
            k_out = ksel;
            kn_out = knext;
            dn_out = dnext;
            return;
        }
        dprev = dd[kWide - 1];
        kprev = kk[kWide - 1];
        i += kWide;
    }
}

// Called by all 32 lanes. Lanes with `want` search level (K, D) from their `lo`.
// When the searching lanes start within 24 entries of each other (the usual case on
// the upper levels, since the batch is sorted), the warp loads one 32-key segment
// from the lowest start with one coalesced access and each lane finds its rank in it by
// a five-step binary search over the lanes (every key before a lane's start is <= its
// q, so the rank is right from any start inside the segment); a lane whose answer lies
// past the segment, and every lane when the starts are spread out (the lower levels),
// scans on its own.
template <bool kDown>
__device__ __forceinline__ void warp_search(const uint64_t* K, const uint32_t* D, uint32_t& lo, uint32_t lim,
                                            uint64_t q, bool want, int32_t& r, uint32_t& dn, uint64_t& kr,
                                            uint64_t& kn, uint32_t& dnn, uint32_t* err) {
    const int lane = threadIdx.x & 31;
    const uint32_t lo_min = __reduce_min_sync(kFull, want ? lo : 0xffffffffu);
    if (lo_min == 0xffffffffu) return;  // no lane searches this level
    const uint32_t lo_max = __reduce_max_sync(kFull, want ? lo : 0u);
    bool scan = want;
    if (lo_max - lo_min < 24u && lo_min <= lim) {
        const uint32_t s = lo_min;
        uint64_t seg_k = K[s + lane];
        const uint32_t seg_d = kDown ? D[s + lane] : 0u;
        // Past the level's sentinel the array holds the next level: clamp so the
        // segment stays sorted.
        const uint32_t sent = __ballot_sync(kFull, seg_k == kMaxKey);
        if (sent && lane > __ffs(sent) - 1) seg_k = kMaxKey;
        uint32_t c = 0;  // segment keys <= q (keys before lo are <= q as well)
#pragma unroll
        for (uint32_t step = 16; step >= 1; step >>= 1) {
            const uint64_t kk = __shfl_sync(kFull, seg_k, (int)(c + step - 1));
            if (kk <= q) c += step;
        }
        const uint64_t k31 = __shfl_sync(kFull, seg_k, 31);
        if (c == 31 && k31 <= q) c = 32;
        const int pick = c ? (int)c - 1 : 0;
        const uint32_t dsel = __shfl_sync(kFull, seg_d, pick & 31);
        const uint64_t ksel = __shfl_sync(kFull, seg_k, pick & 31);
        const uint32_t dnx = __shfl_sync(kFull, seg_d, (int)(c & 31u));
        const uint64_t knx = __shfl_sync(kFull, seg_k, (int)(c & 31u));
        if (want) {
            if (c < 32u) {
                r = (int32_t)s + (int32_t)c - 1;
                dn = c ? dsel : 0u;
                kr = c ? ksel : 0ull;
                kn = knx;
                dnn = dnx;
                scan = false;
            } else {
                lo = s + 31u;  // every segment key is <= q: continue from its end
            }
        }
    }
    if (scan) lane_scan<kDown, kDown ? 4 : 16>(K, D, lo, lim, q, r, dn, kr, kn, dnn, err);
}

// Local run heads of one 256-query sub-tile (a run head, or the sub-tile's first query),
// by one warp: their keys go to `heads` in order, and the largest ownership marker e_i of
// the sub-tile (see apply.cu) to *emax_out. Returns their count. The sub-tile's keys and
// payloads are all loaded before any is used, so the warp waits for memory once.
__device__ __forceinline__ uint32_t subtile_heads(const DescendArgs& a, uint32_t sub, uint32_t qv,
                                                  uint64_t* heads, uint32_t* emax_out) {
    constexpr int kR = kSubTile / 32;
    const int lane = threadIdx.x & 31;
    const uint32_t sb = sub * kSubTile;
    const uint32_t lt = lanemask_lt();
    uint64_t kk[kR];
    uint32_t op[kR];
#pragma unroll
    for (int k = 0; k < kR; ++k) {
        const uint32_t i = sb + (uint32_t)k * 32u + (uint32_t)lane;
        kk[k] = i < qv ? a.sk[i] : kMaxKey;
        op[k] = i < qv ? (a.sp[i] >> 30) : 0u;
    }
    uint64_t carry = (sb > 0 && sb - 1 < qv) ? a.sk[sb - 1] : kMaxKey;  // key before the element
    uint32_t nq = 0, emax = 0;
#pragma unroll
    for (int k = 0; k < kR; ++k) {
        const uint32_t i = sb + (uint32_t)k * 32u + (uint32_t)lane;
        const bool valid = i < qv;
        const uint64_t q = kk[k];
        uint64_t prev = __shfl_up_sync(0xffffffffu, q, 1);
        if (lane == 0) prev = carry;
        carry = __shfl_sync(0xffffffffu, q, 31);
        const bool head = valid && (i == 0 || q != prev);
        const bool local = valid && (head || (k == 0 && lane == 0));
        const uint32_t e = (valid && (op[k] == 1u || op[k] == 2u)) ? 2u * i + 3u : (head ? 2u * i + 2u : 0u);
        emax = max(emax, e);
        const uint32_t b = __ballot_sync(0xffffffffu, local);
        if (local) heads[nq + __popc(b & lt)] = q;
        nq += __popc(b);
    }
    *emax_out = __reduce_max_sync(0xffffffffu, emax);
    return nq;
}

constexpr int kWarps = kThreads / 32;

// The distinct keys of the sorted batch, one CTA per 2048-query apply tile, in the order
// CTAs start (a tile counter), so that a decoupled look-back (Merrill and Garland 2016)
// waits only on tiles that running CTAs hold. One warp per 256-query sub-tile collects
// its local run heads (in shared memory) and its largest ownership marker; the tile's
// head count (a sum) and marker maximum (a max) go through the look-back, which gives
// the tile's first dense index and the exclusive max prefix of the markers that k_apply
// starts from. The heads are then written densely (dq).
__global__ void __launch_bounds__(kThreads) k_heads(DescendArgs a, uint32_t epoch) {
    pdl_wait();
    pdl_trigger();
    __shared__ uint64_t s_hk[kWarps][kSubTile];  // each sub-tile's local heads
    __shared__ uint32_t s_cnt[kWarps], s_max[kWarps], s_off[kWarps + 1];
    __shared__ uint32_t s_tile, s_base, s_pref;
    __shared__ int s_fail;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (block_sees_error(&a.m->error)) return;
    if (tid == 0) {
        s_tile = atomicAdd(&a.bm->tile_ctr[kCtrDistinct], 1u);
        s_fail = 0;
    }
    __syncthreads();
    const uint32_t tile = s_tile, ntiles = gridDim.x;
    const uint32_t n = a.n, qv = n - a.bm->invalid;
    const uint32_t nsub = (n + kSubTile - 1) / kSubTile;
    const uint32_t sub = tile * kWarps + (uint32_t)warp;
    uint32_t nq = 0, emax = 0;
    if (sub < nsub) nq = subtile_heads(a, sub, qv, s_hk[warp], &emax);
    if (lane == 0) {
        s_cnt[warp] = nq;
        s_max[warp] = emax;
    }
    __syncthreads();
    if (warp < 2) {
        uint32_t c = 0, mx = 0;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) {
            if (warp == 0 && lane == 0) s_off[w] = c;
            c += s_cnt[w];
            mx = max(mx, s_max[w]);
        }
        if (warp == 0 && lane == 0) s_off[kWarps] = c;
        bool ok = true;
        const uint32_t ex = warp == 0 ? lookback_warp_wide<false, 8>(a.desc, tile, epoch, c, a.err, &ok)
                                      : lookback_warp_wide<true, 8>(a.desc + ntiles, tile, epoch, mx, a.err, &ok);
        if (lane == 0) {
            if (warp == 0) s_base = ex;
            else s_pref = ex;
            if (!ok) s_fail = 1;
        }
    }
    __syncthreads();
    if (s_fail) return;
    const uint32_t base = s_base, tot = s_off[kWarps];
    if (tid == 0) a.tile_pref[tile] = s_pref;
    if (lane == 0 && sub < nsub) a.sub_pref[sub] = base + s_off[warp];
    if (tile == ntiles - 1 && tid == 0) a.bm->distinct = base + tot;
    for (uint32_t g = (uint32_t)tid; g < tot; g += kThreads) {
        int w = 0;
#pragma unroll
        for (int k = 1; k < kWarps; ++k) w = (g >= s_off[k]) ? k : w;
        a.dq[base + g] = s_hk[w][g - s_off[w]];
    }
}

constexpr int kTopThreads = 1024;  // one CTA per SM: the staged levels take most of its shared memory

// Start position below the pinned levels for every distinct key: a persistent grid, one
// CTA per SM, whose CTAs stage the pinned top levels (up to kSmemTopMax entries) in
// shared memory once (TMA bulk copies, one mbarrier) and then take one key per thread at
// a time: the count of keys <= q in the lowest pinned
// level (it holds every key of the levels above it) by binary lifting, then one
// warp_search per walked level. The dense keys are sorted, so on the upper walked levels
// a warp's 32 keys usually start within a few entries and share one coalesced segment.
__global__ void __launch_bounds__(kTopThreads, 1) k_top(DescendArgs a) {
    pdl_wait();
    pdl_trigger();
    extern __shared__ __align__(16) uint8_t s_dyn[];
    uint64_t* s_k = reinterpret_cast<uint64_t*>(s_dyn);
    uint32_t* s_d = reinterpret_cast<uint32_t*>(s_dyn + (kSmemTopMax + kPad) * sizeof(uint64_t));
    __shared__ __align__(8) uint64_t s_bar;
    __shared__ int s_fail;
    const int tid = threadIdx.x;
    const DevMeta* m = a.m;
    if (block_sees_error(&m->error)) return;
    const uint32_t H = m->H, Ls = m->Ls, Lb = m->Lb, E = m->smem_entries;
    const uint32_t D = a.bm->distinct;
    if (blockIdx.x * kTopThreads >= D) return;
    if (tid == 0) s_fail = 0;
    if (E > 0) {
        if (tid == 0) {
            mbar_init(&s_bar, 1);
            const uint32_t bk = ((E * 8u + 15u) / 16u) * 16u;
            const uint32_t bd = ((E * 4u + 15u) / 16u) * 16u;
            mbar_arrive_expect_tx(&s_bar, bk + bd);
            bulk_g2s(s_k, m->lcur ? a.lkeys1 : a.lkeys, bk, &s_bar);
            bulk_g2s(s_d, m->lcur ? a.ldown1 : a.ldown, bd, &s_bar);
        }
        __syncthreads();
        if (!mbar_wait_bounded(&s_bar, 0, a.err)) s_fail = 1;
        __syncthreads();
        if (s_fail) {
            if (tid == 0) mbar_wait_bounded(&s_bar, 0, a.err);  // let the copy land
            return;
        }
    }
    const bool pinned = Ls <= H;
    const uint32_t bL = m->base[Ls], nL = pinned ? m->n[Ls] : 0u;
    const uint32_t step0 = nL ? 1u << (31 - __clz(nL)) : 0u;
    const uint64_t* LK = m->lcur ? a.lkeys1 : a.lkeys;
    const uint32_t* LD = m->lcur ? a.ldown1 : a.ldown;
    // levels between the pinned ones and the top launched level are walked here
    const int l_hi = pinned ? (int)Ls - 1 : (int)H;
    const int l_lo = max(a.top_launched + 1, (int)Lb);
    for (uint32_t d0 = blockIdx.x * kTopThreads; d0 < D; d0 += gridDim.x * kTopThreads) {
        const uint32_t d = d0 + (uint32_t)tid;
        const bool active = d < D;
        const uint64_t q = active ? a.dq[d] : kMaxKey;
        uint32_t c = 0;  // keys <= q in the lowest pinned level
        for (uint32_t step = step0; step > 0; step >>= 1)
            if (c + step <= nL && s_k[bL + c + step - 1] <= q) c += step;
        uint32_t lo = c ? s_d[bL + c - 1] : 0u;
        for (int l = l_hi; l >= l_lo; --l) {
            int32_t r = -1;
            uint32_t dn = 0, dnn = 0;
            uint64_t kr = 0, kn = 0;
            warp_search<true>(LK + m->base[l], LD + m->base[l], lo, m->n[l], q, active, r, dn, kr, kn, dnn, a.err);
            lo = (r >= 0) ? dn : 0u;
        }
        if (active) a.dlo[d] = lo;
    }
}

// One global index level: every distinct key scans its gap from its start position.
__global__ void __launch_bounds__(kThreads) k_level(DescendArgs a, int l) {
    pdl_wait();
    pdl_trigger();
    const DevMeta* m = a.m;
    if (*(volatile const uint32_t*)&m->error) return;  // no barrier in this kernel
    const uint32_t H = m->H, Lb = m->Lb, Ls = m->Ls;
    const int top = (Ls <= H) ? (int)Ls - 1 : (int)H;
    if (l > top || l < (int)Lb) return;  // this level is pinned or not built
    const uint32_t D = a.bm->distinct;
    const uint32_t base = m->base[l], lim = m->n[l];
    const uint64_t* K = (m->lcur ? a.lkeys1 : a.lkeys) + base;
    const uint32_t* Dn = (m->lcur ? a.ldown1 : a.ldown) + base;
    for (uint32_t d0 = blockIdx.x * kThreads; d0 < D; d0 += gridDim.x * kThreads) {
        const uint32_t d = d0 + threadIdx.x;
        const bool active = d < D;
        const uint64_t q = active ? a.dq[d] : kMaxKey;
        uint32_t lo = active ? a.dlo[d] : 0u;
        int32_t r = -1;
        uint32_t dn = 0, dnn = 0;
        uint64_t kr = 0, kn = 0;
        warp_search<true>(K, Dn, lo, lim, q, active, r, dn, kr, kn, dnn, a.err);
        if (active) a.dlo[d] = (r >= 0) ? dn : 0u;
    }
}

// Largest p in [slo - 1, shi) with K[p] <= q, for a storage gap with K[shi] > q and,
// when slo > 0 or has_lo, K[slo] <= q; -1 when q is below every key. The gap's keys
// lie between klo = K[slo] and khi = K[shi], so the answer is looked for first in the
// 64-byte line of 8 keys around the linear estimate slo + (q - klo) / (khi - klo) *
// (shi - slo): for keys spread evenly over the gap that line usually holds it. From
// there the search moves line by line towards the answer, so it stays exact for any
// key distribution.
__device__ __forceinline__ int32_t gap_search(const uint64_t* K, uint32_t slo, uint32_t shi, uint64_t klo,
                                              uint64_t khi, uint64_t q, uint32_t lim, uint64_t& k_out, uint32_t* err) {
    uint32_t est = slo;
    if (shi > slo + 1u && khi != kMaxKey && khi > klo) {
        const float f = __ull2float_rz(q - klo) / __ull2float_rn(khi - klo);  // in [0, 1]
        est = slo + (uint32_t)(f * (float)(shi - slo));
        if (est >= shi) est = shi - 1u;
    }
    uint32_t c = est & ~7u;
    int dir = 0;
    const uint32_t max_lines = (shi - slo) / 8u + 3u;
    for (uint32_t it = 0;; ++it) {
        if (c > lim || it > max_lines) {
            atomicOr(err, kErrBounds);
            return -1;
        }
        const ulonglong2* kp = reinterpret_cast<const ulonglong2*>(K + c);
        uint64_t kk[8];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const ulonglong2 v = kp[j];
            kk[2 * j] = v.x;
            kk[2 * j + 1] = v.y;
        }
        uint32_t gt = 0;  // bit j: K[c + j] > q (a suffix of the line, the keys being sorted)
#pragma unroll
        for (int j = 0; j < 8; ++j) gt |= (kk[j] > q ? 1u : 0u) << j;
        if (gt == 0xFFu) {  // the answer is before this line
            if (dir > 0) return (int32_t)c - 1;  // (k_out was set on the previous line)
            if (c == 0) return -1;
            dir = -1;
            c -= 8u;
        } else if (gt == 0u) {  // the answer is at the end of this line or after it
            k_out = kk[7];
            if (dir < 0) return (int32_t)c + 7;
            dir = 1;
            c += 8u;
        } else {
            const int f = __ffs(gt) - 1;  // >= 1
#pragma unroll
            for (int j = 1; j < 8; ++j)
                if (j == f) k_out = kk[j - 1];
            return (int32_t)c + f - 1;
        }
    }
}

// The storage layer: the node with the largest key <= q (exists if equal) and its state.
// `lvl` is the lowest index level that can be built. When it is built and not pinned in
// shared memory (the usual case), it has no launch of its own: it is searched here, which
// gives the storage gap of q between the down pointers of two consecutive entries of that
// level, D[r] and D[r + 1], and their keys K[r] <= q < K[r + 1]; gap_search then finds the
// node. Otherwise the node is scanned for from the start position the descent left.
__global__ void __launch_bounds__(kThreads) k_locate(DescendArgs a, int lvl) {
    pdl_wait();
    pdl_trigger();
    const DevMeta* m = a.m;
    if (*(volatile const uint32_t*)&m->error) return;  // no barrier in this kernel
    const uint32_t size = m->size, cur = m->cur;
    const uint64_t* SK = a.st.keys[cur];
    const uint8_t* SM = a.st.meta[cur];
    const uint64_t* SV = a.st.vals[cur];
    const uint32_t H = m->H, Lb = m->Lb, Ls = m->Ls;
    const int top = (Ls <= H) ? (int)Ls - 1 : (int)H;
    const bool fused = lvl <= top && lvl >= (int)Lb;  // then lvl == Lb: its downs are storage positions
    const uint64_t* LK = (m->lcur ? a.lkeys1 : a.lkeys) + (fused ? m->base[lvl] : 0u);
    const uint32_t* LD = (m->lcur ? a.ldown1 : a.ldown) + (fused ? m->base[lvl] : 0u);
    const uint32_t lim = fused ? m->n[lvl] : 0u;
    const uint32_t D = a.bm->distinct;
    for (uint32_t d0 = blockIdx.x * kThreads; d0 < D; d0 += gridDim.x * kThreads) {
        const uint32_t d = d0 + threadIdx.x;
        const bool active = d < D;
        const uint64_t q = active ? a.dq[d] : kMaxKey;
        uint32_t lo = active ? a.dlo[d] : 0u;
        int32_t r = -1;
        uint32_t dn = 0, dnn = 0;
        uint64_t kr = 0, kn = 0;
        if (fused) {
            warp_search<true>(LK, LD, lo, lim, q, active, r, dn, kr, kn, dnn, a.err);
            if (active) {
                r = gap_search(SK, r >= 0 ? dn : 0u, dnn, r >= 0 ? kr : 0ull, kn, q, size, kr, a.err);
            }
        } else {
            warp_search<false>(SK, nullptr, lo, size, q, active, r, dn, kr, kn, dnn, a.err);
        }
        if (active) {
            const bool exists = r >= 0 && kr == q;
            // the value is read with the meta byte, not after it, so both requests are in
            // flight together (a delete-flagged node's value is read and dropped)
            const uint8_t meta = exists ? SM[r] : (uint8_t)0;
            const uint64_t v = exists ? SV[r] : 0ull;
            const bool live = exists && !(meta & kTomb);
            a.loc[d] = (uint32_t)(r + 1);
            a.flags[d] = (uint8_t)((exists ? 1u : 0u) | (live ? 2u : 0u));
            a.val0[d] = live ? v : 0ull;
        }
    }
}

}  // namespace

cudaError_t launch_descend(const DescendArgs& a, uint32_t& epoch, cudaStream_t s, int num_sms,
                           cudaEvent_t before_locate) {
    static bool attr_set = false;
    const int dyn = (int)((kSmemTopMax + kPad) * (sizeof(uint64_t) + sizeof(uint32_t)));
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_top, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    if (a.n == 0) return cudaSuccess;
    const uint32_t ntiles = (a.n + kApplyTile - 1) / kApplyTile;
    launch_dep(k_heads, ntiles, kThreads, 0, s, a, ++epoch);
    ++g_launches;
    // CTAs past the distinct keys exit at once
    const uint32_t tcap = (uint32_t)num_sms, tneed = (a.n + kTopThreads - 1) / kTopThreads;
    launch_dep(k_top, tneed < tcap ? tneed : tcap, kTopThreads, dyn, s, a);
    ++g_launches;
    const uint32_t need = (a.n + kThreads - 1) / kThreads;
    // one launch per index level from top_launched down to bottom_launched + 1; a launch
    // whose level is pinned or not built exits at once, levels above top_launched that
    // are neither are walked by k_heads, and level bottom_launched by k_locate
    const uint32_t capg = (uint32_t)num_sms * 16u;
    const uint32_t gblocks = need < capg ? need : capg;  // grid-stride over the distinct keys
    for (int l = a.top_launched; l > a.bottom_launched; --l) {
        launch_dep(k_level, gblocks, kThreads, 0, s, a, l);
        ++g_launches;
    }
    if (before_locate) cudaEventRecord(before_locate, s);
    launch_dep(k_locate, gblocks, kThreads, 0, s, a, a.bottom_launched);  // searches that level itself
    ++g_launches;
    return cudaGetLastError();
}

}  // namespace pi
