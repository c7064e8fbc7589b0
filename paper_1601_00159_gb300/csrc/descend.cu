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
//  k_distinct   per 256-query sub-tile, one warp counts the distinct keys (run heads,
//               plus the sub-tile's first query); the last CTA to finish scans the
//               apply tiles' counts (dense index) and ownership-marker maxima;
//  k_dpack      each warp writes its sub-tile's distinct keys densely;
//  k_top        the levels pinned in shared memory (copied once per CTA by TMA bulk
//               copies) are resolved by one binary search of the lowest pinned level,
//               which holds every key of the levels above it; writes the dense key and
//               its start position on the next level;
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
// Also returns D[r] (0 if r < 0 or no down array) and K[r]. Each round reads kWide
// consecutive entries with 16-byte loads (keys) and 8-byte loads (downs): 4 on index
// levels, 16 (one 128-byte line) on the storage layer, whose gaps below the lowest built level span
// (1/P)^(Lb-1) nodes. The loads need &K[i] 16-byte aligned (K and D come from arrays
// whose bases are, and a level may start at any entry), so an odd start steps back one
// entry, which is <= q, or, at the head of a level, tests the head on its own.
template <bool kDown, int kWide>
__device__ __forceinline__ void lane_scan(const uint64_t* K, const uint32_t* D, uint32_t lo, uint32_t lim,
                                          uint64_t q, int32_t& r_out, uint32_t& d_out, uint64_t& k_out,
                                          uint32_t* err) {
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
            uint32_t dsel = dprev;
            uint64_t ksel = kprev;
#pragma unroll
            for (int j = 1; j < kWide; ++j) {
                if (j == f) {
                    dsel = dd[j - 1];
                    ksel = kk[j - 1];
                }
            }
            r_out = (int32_t)(i + (uint32_t)f) - 1;
            d_out = dsel;
            k_out = ksel;
            return;
        }
        dprev = dd[kWide - 1];
        kprev = kk[kWide - 1];
        i += kWide;
    }
}

// Called by all 32 lanes. Lanes with `want` search level (K, D) from their `lo`.
// When the searching lanes start within 8 entries of each other (the usual case on
// the upper levels, since the batch is sorted), the warp loads one 32-key segment
// with one coalesced access and each lane finds its rank in it by a five-step binary
// search over the lanes; a lane whose answer lies past the segment, and every lane
// when the starts are spread out (the lower levels), scans on its own.
template <bool kDown>
__device__ __forceinline__ void warp_search(const uint64_t* K, const uint32_t* D, uint32_t& lo, uint32_t lim,
                                            uint64_t q, bool want, int32_t& r, uint32_t& dn, uint64_t& kr,
                                            uint32_t* err) {
    const int lane = threadIdx.x & 31;
    const uint32_t lo_min = __reduce_min_sync(kFull, want ? lo : 0xffffffffu);
    if (lo_min == 0xffffffffu) return;  // no lane searches this level
    const uint32_t lo_max = __reduce_max_sync(kFull, want ? lo : 0u);
    bool scan = want;
    if (lo_max - lo_min < 8u && lo_min <= lim) {
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
        if (want) {
            if (c < 32u) {
                r = (int32_t)s + (int32_t)c - 1;
                dn = c ? dsel : 0u;
                kr = c ? ksel : 0ull;
                scan = false;
            } else {
                lo = s + 31u;  // every segment key is <= q: continue from its end
            }
        }
    }
    if (scan) lane_scan<kDown, kDown ? 4 : 16>(K, D, lo, lim, q, r, dn, kr, err);
}

// Largest index of K[0..n) (sorted, in shared memory) with key <= q, or -1.
__device__ __forceinline__ int32_t smem_rank(const uint64_t* K, uint32_t n, uint64_t q) {
    uint32_t lo = 0, len = n;
    while (len > 0) {
        const uint32_t half = len >> 1;
        if (K[lo + half] <= q) {
            lo += half + 1;
            len -= half + 1;
        } else {
            len = half;
        }
    }
    return (int32_t)lo - 1;
}

// Local run heads of one 256-query sub-tile (a run head, or the sub-tile's first query),
// by one warp. Pass 0 returns their count and the largest ownership marker e_i (see
// apply.cu); pass 1 writes the heads' keys to dq from dense index d0 on.
__device__ __forceinline__ uint32_t subtile_heads(const DescendArgs& a, uint32_t sub, uint32_t qv, bool write,
                                                  uint32_t d0, uint32_t* emax_out) {
    const int lane = threadIdx.x & 31;
    const uint32_t sb = sub * kSubTile;
    const uint32_t lt = lanemask_lt();
    uint32_t nq = 0, emax = 0;
    uint64_t carry = (sb > 0 && sb - 1 < qv) ? a.sk[sb - 1] : kMaxKey;  // key before the element
#pragma unroll 2
    for (int k = 0; k < kSubTile / 32; ++k) {
        const uint32_t i = sb + (uint32_t)k * 32u + (uint32_t)lane;
        const bool valid = i < qv;
        const uint64_t q = valid ? a.sk[i] : kMaxKey;
        uint64_t prev = __shfl_up_sync(0xffffffffu, q, 1);
        if (lane == 0) prev = carry;
        carry = __shfl_sync(0xffffffffu, q, 31);
        const bool head = valid && (i == 0 || q != prev);
        const bool local = valid && (head || (k == 0 && lane == 0));
        if (!write) {
            const uint32_t op = valid ? (a.sp[i] >> 30) : 0u;
            const uint32_t e = (valid && (op == 1u || op == 2u)) ? 2u * i + 3u : (head ? 2u * i + 2u : 0u);
            emax = max(emax, e);
        }
        const uint32_t b = __ballot_sync(0xffffffffu, local);
        if (write && local) a.dq[d0 + nq + __popc(b & lt)] = q;
        nq += __popc(b);
    }
    if (emax_out) *emax_out = __reduce_max_sync(0xffffffffu, emax);
    return nq;
}

// The distinct keys of the sorted batch, in two launches with no CTA waiting for
// another. k_distinct: one CTA per 2048-query apply tile, one warp per 256-query
// sub-tile, counts the local run heads and the largest ownership marker e_i; the last
// CTA to finish scans the tiles' totals into each tile's first dense index (sum) and
// its exclusive prefix of markers (max), so k_apply never waits. k_dpack: each warp
// writes its sub-tile's heads densely from the tile's index on.
__global__ void __launch_bounds__(kThreads) k_distinct(DescendArgs a) {
    pdl_wait();
    pdl_trigger();
    constexpr uint32_t kPer = 8;  // tiles per thread in the final scan
    __shared__ uint32_t s_cnt[kThreads / 32], s_max[kThreads / 32];
    __shared__ uint32_t s_tmp[33], s_last;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (block_sees_error(&a.m->error)) return;
    const uint32_t tile = blockIdx.x, ntiles = gridDim.x;
    const uint32_t n = a.n, qv = n - a.bm->invalid;
    const uint32_t nsub = (n + kSubTile - 1) / kSubTile;
    const uint32_t sub = tile * (kApplyTile / kSubTile) + (uint32_t)warp;
    uint32_t emax = 0, nq = 0;
    if (sub < nsub) nq = subtile_heads(a, sub, qv, false, 0u, &emax);
    if (lane == 0) {
        s_cnt[warp] = nq;
        s_max[warp] = emax;
        if (sub < nsub) a.sub_cnt[sub] = nq;
    }
    __syncthreads();
    if (tid == 0) {
        uint32_t c = 0, mx = 0;
#pragma unroll
        for (int w = 0; w < kThreads / 32; ++w) {
            c += s_cnt[w];
            mx = max(mx, s_max[w]);
        }
        a.tile_heads[tile] = c;
        a.tile_emax[tile] = mx;
        __threadfence();  // the totals, before this CTA's arrival is counted
        s_last = atomicAdd(&a.bm->tile_ctr[kCtrDistinct], 1u) == ntiles - 1u;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();  // every tile has arrived: their totals are visible
    uint32_t csum = 0, cmax = 0;
    for (uint32_t g0 = 0; g0 < ntiles; g0 += kThreads * kPer) {
        const uint32_t t0 = g0 + (uint32_t)tid * kPer;
        uint32_t c[kPer], m[kPer], sum = 0, mx = 0;
#pragma unroll
        for (uint32_t k = 0; k < kPer; ++k) {
            c[k] = t0 + k < ntiles ? __ldcg(&a.tile_heads[t0 + k]) : 0u;
            m[k] = t0 + k < ntiles ? __ldcg(&a.tile_emax[t0 + k]) : 0u;
            sum += c[k];
            mx = max(mx, m[k]);
        }
        uint32_t tsum, tmax;
        uint32_t rs = csum + block_excl_sum<kThreads>(sum, s_tmp, &tsum);
        uint32_t rm = max(cmax, block_excl_max<kThreads>(mx, s_tmp, &tmax));
#pragma unroll
        for (uint32_t k = 0; k < kPer; ++k) {
            if (t0 + k < ntiles) {
                a.tile_base[t0 + k] = rs;
                a.tile_pref[t0 + k] = rm;
            }
            rs += c[k];
            rm = max(rm, m[k]);
        }
        csum += tsum;
        cmax = max(cmax, tmax);
    }
    if (tid == 0) a.bm->distinct = csum;
}

__global__ void __launch_bounds__(kThreads) k_dpack(DescendArgs a) {
    pdl_wait();
    pdl_trigger();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (*(volatile const uint32_t*)&a.m->error) return;  // no barrier in this kernel
    const uint32_t n = a.n, qv = n - a.bm->invalid;
    const uint32_t nsub = (n + kSubTile - 1) / kSubTile;
    const uint32_t tile = blockIdx.x;
    const uint32_t s0 = tile * (kApplyTile / kSubTile), sub = s0 + (uint32_t)warp;
    if (sub >= nsub) return;
    uint32_t d0 = a.tile_base[tile];
    for (uint32_t t = s0; t < sub; ++t) d0 += a.sub_cnt[t];
    if (lane == 0) a.sub_pref[sub] = d0;
    subtile_heads(a, sub, qv, true, d0, nullptr);
}

// Start position below the pinned levels for every distinct key (one per thread): one
// binary search of the lowest pinned level (in shared memory, copied per CTA by TMA
// bulk copies), then a walk of the levels down to top_launched + 1.
__global__ void __launch_bounds__(kThreads) k_top(DescendArgs a) {
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
    if (blockIdx.x * kThreads >= D) return;
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
    const uint32_t bL = m->base[Ls], nL = m->n[Ls];
    for (uint32_t d = blockIdx.x * kThreads + tid; d < D; d += gridDim.x * kThreads) {
        const uint64_t q = a.dq[d];
        uint32_t lo = 0;
        if (Ls <= H) {
            const int32_t r = smem_rank(s_k + bL, nL, q);
            lo = (r >= 0) ? s_d[bL + r] : 0u;
        }
        // levels between the pinned ones and the top launched level: walked here
        for (int l = (Ls <= H ? (int)Ls - 1 : (int)H); l > a.top_launched && l >= (int)Lb; --l) {
            int32_t r = -1;
            uint32_t dn = 0;
            uint64_t kr = 0;
            lane_scan<true, 4>((m->lcur ? a.lkeys1 : a.lkeys) + m->base[l], (m->lcur ? a.ldown1 : a.ldown) + m->base[l],
                               lo, m->n[l], q, r, dn, kr, a.err);
            lo = (r >= 0) ? dn : 0u;
        }
        a.dlo[d] = lo;
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
        uint32_t dn = 0;
        uint64_t kr = 0;
        warp_search<true>(K, Dn, lo, lim, q, active, r, dn, kr, a.err);
        if (active) a.dlo[d] = (r >= 0) ? dn : 0u;
    }
}

// The storage layer: node with the largest key <= q (exists if equal) and its state.
__global__ void __launch_bounds__(kThreads) k_locate(DescendArgs a) {
    pdl_wait();
    pdl_trigger();
    const DevMeta* m = a.m;
    if (*(volatile const uint32_t*)&m->error) return;  // no barrier in this kernel
    const uint32_t size = m->size, cur = m->cur;
    const uint64_t* SK = a.st.keys[cur];
    const uint8_t* SM = a.st.meta[cur];
    const uint64_t* SV = a.st.vals[cur];
    const uint32_t D = a.bm->distinct;
    for (uint32_t d0 = blockIdx.x * kThreads; d0 < D; d0 += gridDim.x * kThreads) {
        const uint32_t d = d0 + threadIdx.x;
        const bool active = d < D;
        const uint64_t q = active ? a.dq[d] : kMaxKey;
        uint32_t lo = active ? a.dlo[d] : 0u;
        int32_t r = -1;
        uint32_t dn = 0;
        uint64_t kr = 0;
        warp_search<false>(SK, nullptr, lo, size, q, active, r, dn, kr, a.err);
        if (active) {
            const bool exists = r >= 0 && kr == q;
            const uint8_t meta = exists ? SM[r] : (uint8_t)0;
            const bool live = exists && !(meta & kTomb);
            a.loc[d] = (uint32_t)(r + 1);
            a.flags[d] = (uint8_t)((exists ? 1u : 0u) | (live ? 2u : 0u));
            a.val0[d] = live ? SV[r] : 0ull;
        }
    }
}

}  // namespace

cudaError_t launch_descend(const DescendArgs& a, cudaStream_t s, int num_sms, cudaEvent_t before_locate) {
    static bool attr_set = false;
    const int dyn = (int)((kSmemTopMax + kPad) * (sizeof(uint64_t) + sizeof(uint32_t)));
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_top, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    if (a.n == 0) return cudaSuccess;
    const uint32_t ntiles = (a.n + kApplyTile - 1) / kApplyTile;
    launch_dep(k_distinct, ntiles, kThreads, 0, s, a);
    ++g_launches;
    launch_dep(k_dpack, ntiles, kThreads, 0, s, a);
    ++g_launches;
    const uint32_t need = (a.n + kThreads - 1) / kThreads;
    launch_dep(k_top, need, kThreads, dyn, s, a);  // CTAs past the distinct keys exit at once
    ++g_launches;
    // one launch per index level from top_launched down to 2; a launch whose level is
    // pinned or not built exits at once, and levels above top_launched that are
    // neither (the index grew) are walked by k_top
    const uint32_t capg = (uint32_t)num_sms * 16u;
    const uint32_t gblocks = need < capg ? need : capg;  // grid-stride over the distinct keys
    for (int l = a.top_launched; l >= a.bottom_launched; --l) {
        launch_dep(k_level, gblocks, kThreads, 0, s, a, l);
        ++g_launches;
    }
    if (before_locate) cudaEventRecord(before_locate, s);
    launch_dep(k_locate, gblocks, kThreads, 0, s, a);
    ++g_launches;
    return cudaGetLastError();
}

}  // namespace pi
