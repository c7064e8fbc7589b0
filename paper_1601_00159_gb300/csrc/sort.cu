// K0 + K1: validate/pack the query set and sort it by key (Definition 3: the queries
// of a query set are ordered by key; Section 4.2: the sort can use data parallelism).
//
// LSD radix sort with 8-bit digits. Every pass is three launches over tiles of 2048
// elements, so no tile ever waits for another:
//   count:   the tile's digit histogram (tile-major rows of 256 counters);
//   scan:    one CTA per digit turns that digit's column into global offsets
//            (digit base from the up-front histograms + prefix over tiles);
//   scatter: ranks the tile's elements stably within the tile and writes them to
//            offset + rank, staged in shared memory so each digit's run is written
//            contiguously.
// A pass whose byte is the same in every key is skipped (byte-wise min/max in the pack
// kernel). The sort is stable, so equal keys stay in arrival order: the order is
// (key, arrival index), the reading of Definition 3 for duplicate keys.
//
// Prefix passes. When more bytes vary than the caller's pass budget (4 for batches),
// only the most significant varying bytes get passes. Keys that agree on those bytes
// then form contiguous segments, still in arrival order. Distinct keys share a segment
// only when they collide on those bytes: about D^2 / 2^33 pairs for D distinct uniform
// keys under 4 bytes, a few hundred at D = 1.2 M. Two kernels finish the order:
//   find: marks the start of every segment that holds two different keys;
//   fix:  orders each marked segment by (key, position). A warp does segments of up to
//         32 queries by counting ranks. A CTA does longer ones (a hot key that collides)
//         with a stable LSD pass per remaining byte, through buffer B.
//
// Payload word: op << 30 | arrival index. Invalid queries (op > 2 or the reserved key)
// get the sort key 2^64-1 and so gather at the end of the sorted batch.

#include "common.cuh"

namespace pi {
namespace {

constexpr int kThreads = 256;
constexpr int kItems = 8;
constexpr int kTile = kThreads * kItems;  // kSortTile
constexpr int kWarps = kThreads / 32;
constexpr int kWarpSpan = 32 * kItems;    // 256 consecutive elements per warp
static_assert(kTile == kSortTile, "tile size shared with the host's descriptor sizing");

// K0: validate and pack. Also finds, per key byte, whether it is the same in every
// valid key (byte-wise min and max), which decides the radix passes that can be skipped.
// Four consecutive queries per thread and step (16-byte key loads, one 4-byte load of
// their op codes, vector stores) when the caller's arrays are aligned for it, so that
// every thread keeps several loads in flight; the byte-wise extremes are kept four bytes
// to a word with SIMD min/max.
struct PackAcc {
    uint32_t invalid = 0;
    uint32_t mxl = 0, mxh = 0;                  // byte-wise max of the valid keys (low, high word)
    uint32_t mnl = 0xFFFFFFFFu, mnh = 0xFFFFFFFFu;  // byte-wise min
    __device__ __forceinline__ uint64_t take(uint64_t k, uint32_t op) {
        const bool valid = op <= 2u && k != kMaxKey;
        invalid += valid ? 0u : 1u;
        if (!valid) return kMaxKey;
        mxl = __vmaxu4(mxl, (uint32_t)k);
        mxh = __vmaxu4(mxh, (uint32_t)(k >> 32));
        mnl = __vminu4(mnl, (uint32_t)k);
        mnh = __vminu4(mnh, (uint32_t)(k >> 32));
        return k;
    }
};

__global__ void __launch_bounds__(256) k_pack(const uint8_t* __restrict__ ops, const uint64_t* __restrict__ keys,
                                              uint32_t n, uint64_t* __restrict__ sk, uint32_t* __restrict__ sp,
                                              uint32_t* __restrict__ fixmap, BatchMeta* bm) {
    pdl_wait();
    pdl_trigger();
    const uint32_t gt = blockIdx.x * blockDim.x + threadIdx.x, gs = gridDim.x * blockDim.x;
    for (uint32_t w = gt; w < (n + 31u) / 32u; w += gs) fixmap[w] = 0;  // segment marks of the prefix fix-up
    PackAcc acc;
    const bool vec = ((reinterpret_cast<uintptr_t>(keys) & 15u) | (reinterpret_cast<uintptr_t>(ops) & 3u)) == 0;
    uint32_t tail = 0;  // first query left to the scalar loop
    if (vec) {
        const uint32_t n4 = n / 4u;
        for (uint32_t g = gt; g < n4; g += gs) {
            const uint32_t i = 4u * g;
            const ulonglong2 k01 = reinterpret_cast<const ulonglong2*>(keys + i)[0];
            const ulonglong2 k23 = reinterpret_cast<const ulonglong2*>(keys + i)[1];
            const uint32_t o4 = ops ? *reinterpret_cast<const uint32_t*>(ops + i) : 0u;
            const uint32_t o0 = o4 & 255u, o1 = (o4 >> 8) & 255u, o2 = (o4 >> 16) & 255u, o3 = o4 >> 24;
            ulonglong2 s01, s23;
            s01.x = acc.take(k01.x, o0);
            s01.y = acc.take(k01.y, o1);
            s23.x = acc.take(k23.x, o2);
            s23.y = acc.take(k23.y, o3);
            reinterpret_cast<ulonglong2*>(sk + i)[0] = s01;
            reinterpret_cast<ulonglong2*>(sk + i)[1] = s23;
            uint4 p;
            p.x = ((o0 & 3u) << 30) | i;
            p.y = ((o1 & 3u) << 30) | (i + 1u);
            p.z = ((o2 & 3u) << 30) | (i + 2u);
            p.w = ((o3 & 3u) << 30) | (i + 3u);
            *reinterpret_cast<uint4*>(sp + i) = p;
        }
        tail = 4u * n4;
    }
    for (uint32_t i = tail + gt; i < n; i += gs) {
        const uint32_t op = ops ? ops[i] : 0u;
        sk[i] = acc.take(keys[i], op);
        sp[i] = ((op & 3u) << 30) | i;
    }
    uint32_t invalid = acc.invalid;
    uint32_t mx[8], mn[8];  // mn holds max of (255 - byte), so zero is the identity
#pragma unroll
    for (int d = 0; d < 4; ++d) {
        mx[d] = (acc.mxl >> (8 * d)) & 255u;
        mx[4 + d] = (acc.mxh >> (8 * d)) & 255u;
        mn[d] = 255u - ((acc.mnl >> (8 * d)) & 255u);
        mn[4 + d] = 255u - ((acc.mnh >> (8 * d)) & 255u);
    }
    __shared__ uint32_t s_red[17];
    if (threadIdx.x < 17) s_red[threadIdx.x] = 0;
    __syncthreads();
#pragma unroll
    for (int d = 0; d < 8; ++d) {
        mx[d] = __reduce_max_sync(0xffffffffu, mx[d]);
        mn[d] = __reduce_max_sync(0xffffffffu, mn[d]);
    }
    invalid = __reduce_add_sync(0xffffffffu, invalid);
    if ((threadIdx.x & 31) == 0) {
        if (invalid) atomicAdd(&s_red[16], invalid);
#pragma unroll
        for (int d = 0; d < 8; ++d) {
            atomicMax(&s_red[d], mx[d]);
            atomicMax(&s_red[8 + d], mn[d]);
        }
    }
    __syncthreads();
    // one global atomic per byte per CTA
    if (threadIdx.x < 8) atomicMax(&bm->bmax[threadIdx.x], s_red[threadIdx.x]);
    else if (threadIdx.x < 16) atomicMax(&bm->bnmin[threadIdx.x - 8], s_red[threadIdx.x]);
    else if (threadIdx.x == 16 && s_red[16]) atomicAdd(&bm->invalid, s_red[16]);
}

// Pass plan. The digit bytes D are the bytes that vary among the valid keys. Invalid
// queries carry the sort key 2^64-1 and must follow every valid key: when there are
// some, D also holds the highest byte p whose maximum over the valid keys is below 0xFF
// (every invalid key is larger there; with no such byte D is every byte). Passes
// ping-pong so that the last one writes buffer A.
// With more than max_passes bytes in D, the passes take the most significant
// max_passes of them (the prefix). The fix-up then orders each segment of equal prefix
// bytes by the full key; its long-segment path sorts by every other byte that can
// differ inside a segment (rdig).
__global__ void __launch_bounds__(256) k_sort_plan(uint32_t n, BatchMeta* bm, uint32_t* gctr, uint32_t max_passes) {
    pdl_wait();
    pdl_trigger();
    const int b = threadIdx.x;
    const uint32_t ngroups = ((n + kTile - 1) / kTile + kScanGroup - 1) / kScanGroup;
    for (uint32_t i = b; i < 8u * (ngroups + 1u); i += 256) gctr[i] = 0;  // the count kernels' arrivals
    if (b == 0) plan_digits(bm->bmax, bm->bnmin, bm->invalid, n, max_passes, bm->plan);
}

__device__ __forceinline__ const uint64_t* pass_src_keys(const SortPlan& P, uint32_t j, const SortBuffers& sb) {
    return P.src[j] == 0 ? sb.in_k : (P.src[j] == 1 ? sb.a_k : sb.b_k);
}

// Digit histogram of every tile for pass j, then its scan, by the CTAs that finish
// last (no CTA waits for another): the last CTA of each group of kScanGroup tiles turns
// the group's counts into offsets within the group (toff) and the group's digit totals
// (gsum); the last group to finish turns those totals into the groups' offsets, in
// place, and the digit totals into digit bases (dofs). A tile's first output slot for
// digit d is then dofs[d] + gsum[group][d] + toff[tile][d]. Pass 0 reads the packed
// keys; later passes read the digit bytes the previous scatter wrote beside its output.
// Each thread counts 8 consecutive elements and adds each run of equal digits with one
// shared-memory atomic (one per warp when the whole warp holds one digit), so a run of a
// hot key costs no atomic contention. The scans load 16 rows per round trip.
__device__ __forceinline__ void count_digits(const uint32_t (&d)[8], uint32_t nv, uint32_t* h) {
    const uint32_t lane = threadIdx.x & 31u;
    uint32_t cur = d[0], run = nv ? 1u : 0u;
    bool single = true;
#pragma unroll
    for (int k = 1; k < 8; ++k) {
        if ((uint32_t)k >= nv) break;
        if (d[k] == cur) {
            ++run;
        } else {
            single = false;
            atomicAdd(&h[cur], run);
            cur = d[k];
            run = 1;
        }
    }
    const uint32_t d0 = __shfl_sync(0xffffffffu, cur, 0);
    if (__all_sync(0xffffffffu, single && cur == d0)) {  // the warp holds one digit
        const uint32_t tot = __reduce_add_sync(0xffffffffu, run);
        if (lane == 0 && tot) atomicAdd(&h[d0], tot);
    } else if (run) {
        atomicAdd(&h[cur], run);
    }
}

// Exclusive running sum, per digit (thread d), over `rows` rows of 256 counters starting
// at `in`: writes each row's prefix to `out` (may equal `in`) and returns the total.
__device__ __forceinline__ uint32_t scan_rows(const uint32_t* in, uint32_t* out, uint32_t rows) {
    const uint32_t d = threadIdx.x;
    uint32_t run = 0;
    for (uint32_t t = 0; t < rows; t += 16) {
        uint32_t c[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) c[k] = (t + k < rows) ? __ldcg(&in[(size_t)(t + k) * 256 + d]) : 0u;
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            if (t + k < rows) {
                out[(size_t)(t + k) * 256 + d] = run;
                run += c[k];
            }
        }
    }
    return run;
}

__global__ void __launch_bounds__(kThreads, 6) k_sort_count(uint32_t j, uint32_t n, SortBuffers sb, BatchMeta* bm) {
    pdl_wait();
    pdl_trigger();
    __shared__ uint32_t h[256];
    __shared__ uint32_t s_tmp[33];
    __shared__ uint32_t s_last;
    const SortPlan& P = bm->plan;
    if (j >= P.npass) return;
    h[threadIdx.x] = 0;
    __syncthreads();
    const uint32_t tbase = blockIdx.x * kTile;
    const uint32_t i0 = tbase + threadIdx.x * 8u;
    const uint32_t nv = i0 < n ? min(8u, n - i0) : 0u;
    uint32_t dg[8];
    if (j == 0) {
        const uint32_t shift = 8u * P.digit[0];
        const uint64_t* src = pass_src_keys(P, 0, sb);
        if (nv == 8u) {
            const ulonglong2* p = reinterpret_cast<const ulonglong2*>(src + i0);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const ulonglong2 v = p[k];
                dg[2 * k] = (uint32_t)(v.x >> shift) & 255u;
                dg[2 * k + 1] = (uint32_t)(v.y >> shift) & 255u;
            }
        } else {
#pragma unroll
            for (int k = 0; k < 8; ++k) dg[k] = (uint32_t)k < nv ? (uint32_t)(src[i0 + k] >> shift) & 255u : 0u;
        }
    } else {
        if (nv == 8u) {  // 8 digit bytes per thread: one 8-byte load
            const uint2 v = *reinterpret_cast<const uint2*>(sb.ndig + i0);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                dg[k] = (v.x >> (8 * k)) & 255u;
                dg[4 + k] = (v.y >> (8 * k)) & 255u;
            }
        } else {
#pragma unroll
            for (int k = 0; k < 8; ++k) dg[k] = (uint32_t)k < nv ? sb.ndig[i0 + k] : 0u;
        }
    }
    count_digits(dg, nv, h);
    __syncthreads();
    const uint32_t d = threadIdx.x;
    const uint32_t tile = blockIdx.x, ntiles = gridDim.x;
    sb.tcnt[(size_t)tile * 256 + d] = h[d];
    const uint32_t g = tile / kScanGroup, ngroups = (ntiles + kScanGroup - 1) / kScanGroup;
    const uint32_t t0 = g * kScanGroup, t1 = min(t0 + kScanGroup, ntiles);
    uint32_t* ctr = sb.gctr + (size_t)j * (ngroups + 1);
    // Arrival: the block barrier orders every thread's counts before thread 0's fence,
    // which (being cumulative) releases them all before its atomic; the last CTA's
    // thread 0 fences after the atomic and the barrier passes that on to its threads.
    __syncthreads();
    if (d == 0) {
        __threadfence();
        s_last = atomicAdd(&ctr[g], 1u) == t1 - t0 - 1u;
        if (s_last) __threadfence();  // every CTA of the group has arrived: their counts are visible
    }
    __syncthreads();
    if (!s_last) return;
    sb.gsum[(size_t)g * 256 + d] = scan_rows(sb.tcnt + (size_t)t0 * 256, sb.toff + (size_t)t0 * 256, t1 - t0);
    __syncthreads();
    if (d == 0) {
        __threadfence();
        s_last = atomicAdd(&ctr[ngroups], 1u) == ngroups - 1u;
        if (s_last) __threadfence();
    }
    __syncthreads();
    if (!s_last) return;
    const uint32_t run = scan_rows(sb.gsum, sb.gsum, ngroups);
    sb.dofs[d] = block_excl_sum<kThreads>(run, s_tmp, nullptr);  // digit bases of this pass
}


__global__ void __launch_bounds__(kThreads, 4) k_sort_pass(uint32_t j, uint32_t n, SortBuffers sb,
                                                           BatchMeta* bm, uint32_t* err) {
    pdl_wait();
    pdl_trigger();
    const SortPlan& P = bm->plan;
    if (j >= P.npass) return;
    const uint32_t shift = 8u * P.digit[j];
    const uint64_t* src_k = P.src[j] == 0 ? sb.in_k : (P.src[j] == 1 ? sb.a_k : sb.b_k);
    const uint32_t* src_p = P.src[j] == 0 ? sb.in_p : (P.src[j] == 1 ? sb.a_p : sb.b_p);
    uint64_t* dst_k = P.dst[j] == 1 ? sb.a_k : sb.b_k;
    uint32_t* dst_p = P.dst[j] == 1 ? sb.a_p : sb.b_p;

    extern __shared__ __align__(16) uint8_t s_dyn[];
    uint64_t* s_key = reinterpret_cast<uint64_t*>(s_dyn);
    uint32_t* s_pay = reinterpret_cast<uint32_t*>(s_dyn + kTile * sizeof(uint64_t));
    __shared__ uint32_t s_whist[kWarps][256];
    __shared__ uint32_t s_gbase[256];
    __shared__ uint32_t s_tstart[256];
    __shared__ uint32_t s_tmp[33];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < kWarps * 256; i += kThreads) (&s_whist[0][0])[i] = 0;
    __syncthreads();
    const uint32_t tile = blockIdx.x;
    const uint32_t tbase = tile * kTile;
    const uint32_t tn = min((uint32_t)kTile, n - tbase);

    uint64_t key[kItems];
    uint32_t pay[kItems];
    uint32_t dig[kItems];
    uint32_t rank[kItems];
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        uint32_t li = warp * kWarpSpan + k * 32 + lane;
        bool v = li < tn;
        key[k] = v ? src_k[tbase + li] : 0ull;
        pay[k] = v ? src_p[tbase + li] : 0u;
        dig[k] = v ? (uint32_t)((key[k] >> shift) & 255u) : 256u;
    }
    warp_digit_ranks<kItems, 8>(dig, rank, s_whist[warp]);
    __syncthreads();
    // Thread tid owns digit tid: tile total and per-warp exclusive prefix.
    uint32_t total = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
        uint32_t c = s_whist[w][tid];
        s_whist[w][tid] = total;
        total += c;
    }
    s_gbase[tid] = sb.dofs[tid] + sb.gsum[(size_t)(tile / kScanGroup) * 256 + tid] +
                   sb.toff[(size_t)tile * 256 + tid];
    s_tstart[tid] = block_excl_sum<kThreads>(total, s_tmp, nullptr);
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        uint32_t d = dig[k];
        if (d < 256u) {
            uint32_t pos = s_tstart[d] + s_whist[warp][d] + rank[k];
            s_key[pos] = key[k];
            s_pay[pos] = pay[k];
        }
    }
    __syncthreads();
    const bool next = j + 1 < P.npass;
    const uint32_t nshift = next ? 8u * P.digit[j + 1] : 0u;
    for (uint32_t s = tid; s < tn; s += kThreads) {
        uint64_t k = s_key[s];
        uint32_t d = (uint32_t)((k >> shift) & 255u);
        uint32_t g = s_gbase[d] + (s - s_tstart[d]);
        if (g < n) {
            dst_k[g] = k;
            dst_p[g] = s_pay[s];
            if (next) sb.ndig[g] = (uint8_t)(k >> nshift);  // the next pass's digit
        } else {
            atomicOr(err, kErrBounds);
        }
    }
}

// ---------------------------------------------------------------------------------
// Prefix fix-up. After the prefix passes buffer A is sorted by key & pmask ("the
// prefix"), and positions with equal prefix hold their queries in arrival order.

// Marks (in fixmap) the first position of every segment of equal prefix that holds two
// different keys. A position i whose key differs from key i-1 but whose prefix does not
// lies inside such a segment; the segment's start is found by a galloping search back
// from i followed by a binary search, both over the prefix order.
__global__ void __launch_bounds__(256) k_sort_find(uint32_t n, SortBuffers sb, const BatchMeta* bm) {
    pdl_wait();
    pdl_trigger();
    const SortPlan& P = bm->plan;
    if (!P.fix) return;
    const uint64_t pm = P.pmask;
    const uint64_t* __restrict__ ak = sb.a_k;
    const uint32_t lane = threadIdx.x & 31u;
    constexpr int kU = 4;  // positions per thread and step, loaded together
    for (uint32_t base = blockIdx.x * 256u * kU; base < n; base += gridDim.x * 256u * kU) {
        uint64_t k1[kU], k0[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const uint32_t i = base + (uint32_t)u * 256u + threadIdx.x;
            k1[u] = i < n ? ak[i] : 0ull;
            k0[u] = (lane == 0 && i > 0 && i < n) ? ak[i - 1] : 0ull;
        }
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const uint32_t i = base + (uint32_t)u * 256u + threadIdx.x;
            uint64_t kp = __shfl_up_sync(0xffffffffu, k1[u], 1);
            if (lane == 0) kp = k0[u];
            if (i == 0 || i >= n || kp == k1[u] || ((kp ^ k1[u]) & pm) != 0) continue;
            const uint64_t mk = k1[u] & pm;
            uint32_t in = i - 1;  // ak[in] is in the segment
            uint64_t d = 1;
            while (d <= in && (ak[in - d] & pm) == mk) {
                in -= (uint32_t)d;
                d <<= 1;
            }
            uint32_t lo = d <= in ? in - (uint32_t)d + 1 : 0u, hi = in;  // the start lies in [lo, hi]
            while (lo < hi) {
                const uint32_t mid = lo + (hi - lo) / 2;
                if ((ak[mid] & pm) == mk) hi = mid;
                else lo = mid + 1;
            }
            atomicOr(&sb.fixmap[lo >> 5], 1u << (lo & 31u));
        }
    }
}

constexpr int kFixSlice = kThreads * 32;  // positions per fix-up CTA: one fixmap word per thread

// Stable LSD sort of the segment [s, e) of buffer A by the bytes P.rdig (ascending),
// by the whole CTA, through the same range of buffer B. The segment is in arrival
// order, so the result is in (key, arrival) order.
__device__ void cta_segment_lsd(uint32_t s, uint32_t e, const SortPlan& P, const SortBuffers& sb,
                                uint32_t (*s_whist)[256], uint32_t* s_base, uint32_t* s_tmp) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint64_t* src_k = sb.a_k;
    uint32_t* src_p = sb.a_p;
    uint64_t* dst_k = sb.b_k;
    uint32_t* dst_p = sb.b_p;
    for (uint32_t r = 0; r < P.nr; ++r) {
        const uint32_t shift = 8u * P.rdig[r];
        for (int w = 0; w < kWarps; ++w) s_whist[w][tid] = 0;
        s_base[tid] = 0;
        __syncthreads();
        for (uint32_t i = s + tid; i < e; i += kThreads) atomicAdd(&s_base[(uint32_t)(src_k[i] >> shift) & 255u], 1u);
        __syncthreads();
        const uint32_t cnt = s_base[tid];
        __syncthreads();
        s_base[tid] = s + block_excl_sum<kThreads>(cnt, s_tmp, nullptr);
        __syncthreads();
        for (uint32_t c = s; c < e; c += kTile) {
            uint64_t key[kItems];
            uint32_t pay[kItems], dig[kItems], rank[kItems];
#pragma unroll
            for (int k = 0; k < kItems; ++k) {
                const uint32_t i = c + warp * kWarpSpan + k * 32 + lane;
                const bool v = i < e;
                key[k] = v ? src_k[i] : 0ull;
                pay[k] = v ? src_p[i] : 0u;
                dig[k] = v ? (uint32_t)((key[k] >> shift) & 255u) : 256u;
            }
            warp_digit_ranks<kItems, 8>(dig, rank, s_whist[warp]);
            __syncthreads();
            uint32_t total = 0;  // thread tid owns digit tid: per-warp exclusive prefix
#pragma unroll
            for (int w = 0; w < kWarps; ++w) {
                const uint32_t cc = s_whist[w][tid];
                s_whist[w][tid] = total;
                total += cc;
            }
            __syncthreads();
#pragma unroll
            for (int k = 0; k < kItems; ++k) {
                const uint32_t d = dig[k];
                if (d < 256u) {
                    const uint32_t pos = s_base[d] + s_whist[warp][d] + rank[k];
                    if (pos >= s && pos < e) {
                        dst_k[pos] = key[k];
                        dst_p[pos] = pay[k];
                    }
                }
            }
            __syncthreads();
            s_base[tid] += total;
#pragma unroll
            for (int w = 0; w < kWarps; ++w) s_whist[w][tid] = 0;
            __syncthreads();
        }
        uint64_t* tk = src_k; src_k = dst_k; dst_k = tk;
        uint32_t* tp = src_p; src_p = dst_p; dst_p = tp;
    }
    if (src_k != sb.a_k) {  // an odd number of passes left the result in B
        for (uint32_t i = s + tid; i < e; i += kThreads) {
            sb.a_k[i] = src_k[i];
            sb.a_p[i] = src_p[i];
        }
    }
    __syncthreads();
}

// Orders the segment [s, e) of buffer A by the bytes the prefix passes skipped, for a
// segment of at most one tile: it is read into registers once, every pass ranks it and
// places it in shared memory (s_k, s_p: kTile entries) in digit order, the next pass
// reads it back from there, and the result is written to A once. Stable.
__device__ void cta_segment_smem(uint32_t s, uint32_t e, const SortPlan& P, const SortBuffers& sb,
                                 uint64_t* s_k, uint32_t* s_p, uint32_t (*s_whist)[256], uint32_t* s_base,
                                 uint32_t* s_tmp) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t L = e - s;
    uint64_t key[kItems];
    uint32_t pay[kItems];
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        const uint32_t li = (uint32_t)(warp * kWarpSpan + k * 32 + lane);
        key[k] = li < L ? sb.a_k[s + li] : 0ull;
        pay[k] = li < L ? sb.a_p[s + li] : 0u;
    }
    for (int w = 0; w < kWarps; ++w) s_whist[w][tid] = 0;
    __syncthreads();
    for (uint32_t r = 0; r < P.nr; ++r) {
        const uint32_t shift = 8u * P.rdig[r];
        uint32_t dig[kItems], rank[kItems];
#pragma unroll
        for (int k = 0; k < kItems; ++k) {
            const uint32_t li = (uint32_t)(warp * kWarpSpan + k * 32 + lane);
            dig[k] = li < L ? (uint32_t)((key[k] >> shift) & 255u) : 256u;
        }
        warp_digit_ranks<kItems, 8>(dig, rank, s_whist[warp]);
        __syncthreads();
        uint32_t total = 0;  // thread tid owns digit tid: per-warp exclusive prefix
#pragma unroll
        for (int w = 0; w < kWarps; ++w) {
            const uint32_t cc = s_whist[w][tid];
            s_whist[w][tid] = total;
            total += cc;
        }
        s_base[tid] = block_excl_sum<kThreads>(total, s_tmp, nullptr);  // the digit's first slot
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kItems; ++k) {
            const uint32_t d = dig[k];
            if (d < 256u) {
                const uint32_t pos = s_base[d] + s_whist[warp][d] + rank[k];
                s_k[pos] = key[k];
                s_p[pos] = pay[k];
            }
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kItems; ++k) {
            const uint32_t li = (uint32_t)(warp * kWarpSpan + k * 32 + lane);
            if (li < L) {
                key[k] = s_k[li];
                pay[k] = s_p[li];
            }
        }
        for (int w = 0; w < kWarps; ++w) s_whist[w][tid] = 0;
        __syncthreads();
    }
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        const uint32_t li = (uint32_t)(warp * kWarpSpan + k * 32 + lane);
        if (li < L) {
            sb.a_k[s + li] = key[k];
            sb.a_p[s + li] = pay[k];
        }
    }
    __syncthreads();
}

// Orders every marked segment. Each CTA reads kThreads fixmap words (kFixSlice
// positions) and takes the segments that start there. A warp orders a segment of at
// most 32 queries: rank = queries with a smaller key, or the same key and an earlier
// position. Longer segments are queued for the whole CTA.
__global__ void __launch_bounds__(kThreads) k_sort_fix(uint32_t n, SortBuffers sb, BatchMeta* bm) {
    pdl_wait();
    pdl_trigger();
    const SortPlan& P = bm->plan;
    if (!P.fix) return;
    // segment starts (a segment holds >= 2 queries); then the keys of a long segment
    // ordered in shared memory
    __shared__ __align__(16) uint32_t s_list[kFixSlice / 2];
    __shared__ uint32_t s_pay[kTile];
    static_assert(kFixSlice / 2 * sizeof(uint32_t) >= kTile * sizeof(uint64_t), "a tile's keys fit s_list");
    __shared__ uint32_t s_big[kFixSlice / 32 + 1];  // starts of segments of more than 32
    __shared__ uint32_t s_nbig, s_end;
    __shared__ uint32_t s_tmp[33];
    __shared__ uint32_t s_whist[kWarps][256];
    __shared__ uint32_t s_base[256];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t nwords = (n + 31u) / 32u;
    const uint32_t wi = blockIdx.x * kThreads + tid;
    uint32_t w = wi < nwords ? sb.fixmap[wi] : 0u;
    uint32_t total;
    uint32_t off = block_excl_sum<kThreads>((uint32_t)__popc(w), s_tmp, &total);
    while (w) {
        const uint32_t b = (uint32_t)(__ffs(w) - 1);
        w &= w - 1;
        if (off < kFixSlice / 2) s_list[off] = wi * 32u + b;  // starts are >= 2 apart: always true
        ++off;
    }
    if (tid == 0) s_nbig = 0;
    __syncthreads();
    if (total == 0) return;
    if (total > kFixSlice / 2) total = kFixSlice / 2;
    const uint64_t pm = P.pmask;
    const uint64_t* ak = sb.a_k;
    for (uint32_t x = warp; x < total; x += kWarps) {
        const uint32_t s = s_list[x];
        const uint64_t mk = ak[s] & pm;
        const uint32_t i = s + lane;
        // The segment's queries are the lanes of a prefix of the warp (prefix order).
        const uint64_t key = i < n ? ak[i] : 0ull;
        const bool in = i < n && (key & pm) == mk;
        const uint32_t m = (uint32_t)__popc(__ballot_sync(0xffffffffu, in));
        const bool longer = m == 32u && s + 32u < n && (ak[s + 32u] & pm) == mk;
        if (longer) {
            if (lane == 0) {
                const uint32_t slot = atomicAdd(&s_nbig, 1u);
                if (slot < kFixSlice / 32 + 1) s_big[slot] = s;  // starts are > 32 apart: always true
            }
            continue;
        }
        const uint32_t pay = in ? sb.a_p[i] : 0u;
        uint32_t rank = 0;
#pragma unroll 8
        for (int j = 0; j < 32; ++j) {
            const uint64_t kj = __shfl_sync(0xffffffffu, key, j);
            rank += ((uint32_t)j < m && (kj < key || (kj == key && j < lane))) ? 1u : 0u;
        }
        __syncwarp();
        if (in) {
            sb.a_k[s + rank] = key;
            sb.a_p[s + rank] = pay;
        }
    }
    __syncthreads();
    const uint32_t nbig = min(s_nbig, (uint32_t)(kFixSlice / 32 + 1));
    for (uint32_t x = 0; x < nbig; ++x) {
        const uint32_t s = s_big[x];
        if (warp == 0) {
            // End of the segment, by the first warp: lane l probes s + 32 + 2^l - 1 (a
            // gallop in one round), then 32-way rounds narrow the bracket. The segment's
            // positions are a prefix of [s + 32, n), so each round's hits are a prefix.
            const uint64_t mk = ak[s] & pm;
            const uint32_t base = s + 32u;  // in the segment
            const uint64_t off = (1ull << lane) - 1ull;
            const bool hit = base + off < n && (ak[base + off] & pm) == mk;
            const uint32_t hm = __ballot_sync(0xffffffffu, hit);  // lane 0 always hits
            const int top = 31 - __clz(hm);
            uint32_t lo = base + ((1u << top) - 1u) + 1u;  // past the last position known in it
            const uint64_t qn = (uint64_t)base + (2ull << top) - 1ull;  // the first probe past it
            uint32_t hi = (top < 31 && qn < (uint64_t)n) ? (uint32_t)qn : n;  // not in it (or n)
            while (hi > lo) {  // the end lies in [lo, hi]
                const uint32_t step = (hi - lo + 31u) / 32u;
                const uint32_t p = lo + lane * step;
                const bool in = p < hi && (ak[p] & pm) == mk;
                const uint32_t c = (uint32_t)__popc(__ballot_sync(0xffffffffu, in));
                if (c == 0) break;  // lo itself is past the segment
                const uint32_t nlo = lo + (c - 1u) * step + 1u;
                const uint32_t nhi = lo + c * step;
                lo = nlo;
                hi = nhi < hi ? nhi : hi;
            }
            if (lane == 0) {
                s_end = lo;
                atomicAdd(&bm->fix_big, lo - s);
            }
        }
        __syncthreads();
        if (s_end - s <= (uint32_t)kTile)
            cta_segment_smem(s, s_end, P, sb, reinterpret_cast<uint64_t*>(s_list), s_pay, s_whist, s_base, s_tmp);
        else
            cta_segment_lsd(s, s_end, P, sb, s_whist, s_base, s_tmp);
    }
}

}  // namespace

cudaError_t launch_sort(const uint8_t* ops, const uint64_t* keys, uint32_t n, const SortBuffers& sb,
                        BatchMeta* bm, uint32_t* err, cudaStream_t s, int num_sms, int max_passes) {
    if (n == 0) return cudaSuccess;
    if (max_passes < 1 || max_passes > 8) return cudaErrorInvalidValue;
    int grid = min((int)((n + 255) / 256), num_sms * 8);
    launch_dep(k_pack, grid, 256, 0, s, ops, keys, n, sb.in_k, sb.in_p, sb.fixmap, bm);
    ++g_launches;
    launch_dep(k_sort_plan, 1, 256, 0, s, n, bm, sb.gctr, (uint32_t)max_passes);
    ++g_launches;
    static bool attr_set = false;
    const int dyn = kTile * (int)(sizeof(uint64_t) + sizeof(uint32_t));
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_sort_pass, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    const uint32_t tiles = (n + kTile - 1) / kTile;
    launch_dep(k_sort_count, tiles, kThreads, 0, s, 0, n, sb, bm);
    ++g_launches;
    for (uint32_t j = 0; j < (uint32_t)max_passes; ++j) {
        launch_dep(k_sort_pass, tiles, kThreads, dyn, s, j, n, sb, bm, err);
        ++g_launches;
        if (j + 1 < (uint32_t)max_passes) {
            launch_dep(k_sort_count, tiles, kThreads, 0, s, j + 1, n, sb, bm);
            ++g_launches;
        }
    }
    if (max_passes < 8) {  // with eight passes every byte is sorted: nothing to fix
        const int fgrid = min((int)((n + 1023) / 1024), num_sms * 8);
        launch_dep(k_sort_find, fgrid, 256, 0, s, n, sb, bm);
        ++g_launches;
        launch_dep(k_sort_fix, (n + kFixSlice - 1) / kFixSlice, kThreads, 0, s, n, sb, bm);
        ++g_launches;
    }
    return cudaGetLastError();
}

}  // namespace pi
