// Range search (Section 3.2.5): for every query [lo, hi], the live pairs with
// lo <= key <= hi in key order, packed query after query (offsets in CSR form).
//
// The paper sorts range queries by their lower bound, finds the interceptions like
// point queries, splits a range that crosses into the next thread's part and walks the
// storage layer up to the upper bound. Here both bounds of every query go through the
// batch path's own sort and descent (2n point lookups), which gives each bound's
// storage position; a query's range is then the slice [start, end) of the storage
// layer, and a warp per query walks its meta bytes 16 per lane per step:
//   k_range_ends   per sorted bound: start = first node with key >= lo,
//                  end = first node with key > hi;
//   k_range_count  live nodes in [start, end) per query, and per-CTA sums;
//   k_range_scan   one CTA prefixes the CTA sums (64-bit);
//   k_range_write  offsets[i] and, when the query's pairs fit in the caller's capacity,
//                  its keys and values.
// A warp per query replaces the paper's hand-over of range pieces between threads: the
// CSR offsets fix every query's output place, so no query waits for another.

#include "common.cuh"

namespace pi {
namespace {

constexpr int kThreads = 256;
constexpr int kItems = 8;  // sorted bounds per thread in k_range_ends (a warp = one 256-bound sub-tile)
constexpr uint32_t kSeqMask = (1u << 30) - 1u;
constexpr int kQ = kThreads;  // queries per CTA in count / write

// Block-wide exclusive sum of 64-bit values (kThreads threads); total in *total.
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
        const uint64_t w = lane < kThreads / 32 ? tmp[lane] : 0ull;
        uint64_t s = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint64_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < kThreads / 32) tmp[lane] = s - w;
        if (lane == kThreads / 32 - 1) tmp[32] = s;
    }
    __syncthreads();
    const uint64_t r = tmp[warp] + x - v;
    if (total) *total = tmp[32];
    __syncthreads();
    return r;
}

// Bytes of the 16-byte meta chunk c that lie in [s, e) and are live, as a bit mask.
__device__ __forceinline__ uint32_t live_mask(const uint8_t* meta, uint64_t c, uint32_t s, uint32_t e) {
    const uint4 w = *reinterpret_cast<const uint4*>(meta + c * 16u);
    const uint32_t words[4] = {w.x, w.y, w.z, w.w};
    uint32_t m = 0;
#pragma unroll
    for (int b = 0; b < 16; ++b) {
        const uint64_t p = c * 16u + (uint64_t)b;
        const uint32_t byte = (words[b >> 2] >> (8 * (b & 3))) & 0xFFu;
        if (p >= s && p < e && !(byte & kTomb)) m |= 1u << b;
    }
    return m;
}

// Storage slice of every query from the descent of its two bounds. Each thread takes
// kItems consecutive sorted bounds, so a warp covers one descent sub-tile and the
// dense index of a bound's key is its sub-tile's prefix plus the warp's local heads.
__global__ void __launch_bounds__(kThreads) k_range_ends(RangeArgs a) {
    pdl_wait();
    pdl_trigger();
    const DevMeta* m = a.m;
    if (*(volatile const uint32_t*)&m->error) return;
    const uint32_t nb = 2u * a.n, qv = nb - a.bm->invalid, size = m->size;
    const uint32_t base = (blockIdx.x * kThreads + threadIdx.x) * kItems;
    const int lane = threadIdx.x & 31;
    uint64_t key[kItems];
    uint32_t lh = 0, nh = 0;
    const uint64_t kprev = (base > 0 && base - 1 < qv) ? a.sk[base - 1] : kMaxKey;
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        const uint32_t i = base + k;
        key[k] = i < qv ? a.sk[i] : kMaxKey;
        const uint64_t prev = k ? key[k - 1] : kprev;
        const bool local = i < qv && (i == 0 || key[k] != prev || (i % kSubTile) == 0);
        lh |= (local ? 1u : 0u) << k;
        nh += local ? 1u : 0u;
    }
    uint32_t incl = nh;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    uint32_t hidx = base < nb ? incl - nh + a.sub_pref[base / kSubTile] : 0u;
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        const uint32_t i = base + k;
        hidx += (lh >> k) & 1u;
        if (i >= nb) continue;
        const uint32_t b = a.sp[i] & kSeqMask;  // bound index: lo of query b, or hi of query b - n
        uint32_t pos;
        if (i >= qv) {
            pos = size;  // the bound 2^64-1 lies past every stored key
        } else {
            const uint32_t dj = hidx - 1u;
            const uint32_t L = a.loc[dj];  // nodes with key <= the bound
            pos = (b < a.n && (a.flags[dj] & 1u)) ? L - 1u : L;
        }
        if (b < a.n) a.start[b] = pos;
        else if (b < nb) a.end[b - a.n] = pos;
        else atomicOr(a.err, kErrBounds);
    }
}

// Live nodes per query (a warp per query) and per-CTA totals.
__global__ void __launch_bounds__(kThreads) k_range_count(RangeArgs a) {
    pdl_wait();
    pdl_trigger();
    __shared__ uint64_t s_sum[kThreads / 32];
    const DevMeta* m = a.m;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint8_t* SM = a.st.meta[m->cur];
    const uint32_t q0 = blockIdx.x * kQ;
    uint64_t wsum = 0;
    for (uint32_t j = warp; j < (uint32_t)kQ; j += kThreads / 32) {
        const uint32_t i = q0 + j;
        if (i >= a.n) break;
        const uint32_t s = a.start[i], e = a.end[i];
        uint32_t cnt = 0;
        if (e > s) {
            const uint64_t c0 = s / 16u, c1 = (e - 1u) / 16u;
            for (uint64_t c = c0 + (uint64_t)lane; c <= c1; c += 32u) cnt += __popc(live_mask(SM, c, s, e));
        }
        cnt = __reduce_add_sync(0xffffffffu, cnt);
        if (lane == 0) a.cnt[i] = cnt;
        wsum += cnt;
    }
    if (lane == 0) s_sum[warp] = wsum;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint64_t t = 0;
        for (int w = 0; w < kThreads / 32; ++w) t += s_sum[w];
        a.bsum[blockIdx.x] = t;
    }
}

// Exclusive prefix of the CTA sums in place (one CTA), the grand total in offsets[n].
__global__ void __launch_bounds__(kThreads) k_range_scan(RangeArgs a) {
    pdl_wait();
    pdl_trigger();
    __shared__ uint64_t s_tmp[33];
    const uint32_t nblk = (a.n + kQ - 1) / kQ;
    uint64_t carry = 0;
    for (uint32_t b0 = 0; b0 < nblk; b0 += kThreads) {
        const uint32_t b = b0 + threadIdx.x;
        const uint64_t v = b < nblk ? a.bsum[b] : 0ull;
        uint64_t tot;
        const uint64_t ex = block_excl_sum64(v, s_tmp, &tot);
        if (b < nblk) a.bsum[b] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) a.offsets[a.n] = carry;
}

// Offsets and pairs. A query whose pairs do not fit below cap gets its offset only.
__global__ void __launch_bounds__(kThreads) k_range_write(RangeArgs a) {
    pdl_wait();
    pdl_trigger();
    __shared__ uint64_t s_tmp[33];
    __shared__ uint64_t s_off[kQ];
    const DevMeta* m = a.m;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t cur = m->cur;
    const uint8_t* SM = a.st.meta[cur];
    const uint64_t* SK = a.st.keys[cur];
    const uint64_t* SV = a.st.vals[cur];
    const uint32_t q0 = blockIdx.x * kQ;
    {
        const uint32_t i = q0 + threadIdx.x;
        const uint64_t c = i < a.n ? a.cnt[i] : 0ull;
        const uint64_t o = a.bsum[blockIdx.x] + block_excl_sum64(c, s_tmp, nullptr);
        s_off[threadIdx.x] = o;
        if (i < a.n) a.offsets[i] = o;
    }
    __syncthreads();
    for (uint32_t j = warp; j < (uint32_t)kQ; j += kThreads / 32) {
        const uint32_t i = q0 + j;
        if (i >= a.n) break;
        const uint64_t off = s_off[j];
        const uint32_t s = a.start[i], e = a.end[i];
        if (e <= s || off + a.cnt[i] > a.cap) continue;
        const uint64_t c0 = s / 16u, c1 = (e - 1u) / 16u;
        uint64_t run = off;
        for (uint64_t cb = c0; cb <= c1; cb += 32u) {
            const uint64_t c = cb + (uint64_t)lane;
            const uint32_t lm = c <= c1 ? live_mask(SM, c, s, e) : 0u;
            const uint32_t cnt = __popc(lm);
            uint32_t incl = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            uint64_t w = run + (incl - cnt);
            uint32_t mm = lm;
            while (mm) {
                const uint32_t b = (uint32_t)(__ffs(mm) - 1);
                mm &= mm - 1;
                const uint64_t p = c * 16u + b;
                a.keys_out[w] = SK[p];
                a.vals_out[w] = SV[p];
                ++w;
            }
            run += __shfl_sync(0xffffffffu, incl, 31);
        }
    }
}

}  // namespace

cudaError_t launch_range(const RangeArgs& a, cudaStream_t s) {
    if (a.n == 0) return cudaSuccess;
    const uint32_t nb = 2u * a.n;
    const uint32_t ends_blocks = (nb + kThreads * kItems - 1) / (kThreads * kItems);
    launch_dep(k_range_ends, ends_blocks, kThreads, 0, s, a);
    ++g_launches;
    const uint32_t qblocks = (a.n + kQ - 1) / kQ;
    launch_dep(k_range_count, qblocks, kThreads, 0, s, a);
    ++g_launches;
    launch_dep(k_range_scan, 1, kThreads, 0, s, a);
    ++g_launches;
    launch_dep(k_range_write, qblocks, kThreads, 0, s, a);
    ++g_launches;
    return cudaGetLastError();
}

}  // namespace pi
