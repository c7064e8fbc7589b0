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
// The up-front histograms of all eight digits (one read of the keys) give the digit
// bases and let a pass whose digit is the same for every key be skipped. The sort is
// stable, so equal keys stay in arrival order: the order is (key, arrival index), the
// reading of Definition 3 for duplicate keys.
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
// key (byte-wise min and max), which decides the radix passes that can be skipped.
__global__ void __launch_bounds__(256) k_pack(const uint8_t* __restrict__ ops, const uint64_t* __restrict__ keys,
                                              uint32_t n, uint64_t* __restrict__ sk, uint32_t* __restrict__ sp,
                                              BatchMeta* bm) {
    uint32_t invalid = 0;
    uint32_t mx[8], mn[8];  // mn holds max of (255 - byte), so zero is the identity
#pragma unroll
    for (int d = 0; d < 8; ++d) {
        mx[d] = 0;
        mn[d] = 0;
    }
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint64_t k = keys[i];
        const uint32_t op = ops ? ops[i] : 0u;
        const bool valid = op <= 2u && k != kMaxKey;
        const uint64_t s = valid ? k : kMaxKey;
        invalid += valid ? 0u : 1u;
        sk[i] = s;
        sp[i] = ((op & 3u) << 30) | i;
#pragma unroll
        for (int d = 0; d < 8; ++d) {
            const uint32_t b = (uint32_t)(s >> (8 * d)) & 255u;
            mx[d] = max(mx[d], b);
            mn[d] = max(mn[d], 255u - b);
        }
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

// Pass plan: the passes whose byte varies (at least one), ping-ponging so the last
// pass writes buffer A.
__global__ void __launch_bounds__(256) k_sort_plan(uint32_t n, BatchMeta* bm, uint32_t* tile_max) {
    const int b = threadIdx.x;
    if (tile_max)
        for (uint32_t t = b; t < (n + kApplyTile - 1) / kApplyTile; t += 256) tile_max[t] = 0;
    if (b == 0) {
        SortPlan& P = bm->plan;
        uint32_t r = 0;
        uint32_t dig[8];
        for (int d = 0; d < 8; ++d)
            if (bm->bmax[d] != 255u - bm->bnmin[d]) dig[r++] = d;  // max byte != min byte
        if (r == 0) dig[r++] = 0;  // all keys equal: one pass (identity order)
        P.npass = r;
        for (uint32_t j = 0; j < r; ++j) {
            P.digit[j] = dig[j];
            P.src[j] = (j == 0) ? 0u : P.dst[j - 1];
            P.dst[j] = ((r - 1 - j) % 2 == 0) ? 1u : 2u;  // the last pass writes buffer A
        }
    }
}

__device__ __forceinline__ const uint64_t* pass_src_keys(const SortPlan& P, uint32_t j, const SortBuffers& sb) {
    return P.src[j] == 0 ? sb.in_k : (P.src[j] == 1 ? sb.a_k : sb.b_k);
}

// Digit histogram of every tile for pass j. Pass 0 reads the packed keys; later
// passes read the digit bytes the previous scatter wrote beside its output.
__global__ void __launch_bounds__(kThreads) k_sort_count(uint32_t j, uint32_t n, SortBuffers sb, BatchMeta* bm) {
    __shared__ uint32_t h[256];
    const SortPlan& P = bm->plan;
    if (j >= P.npass) return;
    h[threadIdx.x] = 0;
    __syncthreads();
    const uint32_t tbase = blockIdx.x * kTile;
    if (j == 0) {
        const uint32_t shift = 8u * P.digit[0];
        const uint64_t* src = pass_src_keys(P, 0, sb);
#pragma unroll
        for (int k = 0; k < kItems; ++k) {
            const uint32_t i = tbase + k * kThreads + threadIdx.x;
            if (i < n) atomicAdd(&h[(uint32_t)(src[i] >> shift) & 255u], 1u);
        }
    } else {
        // 8 digit bytes per thread: one 8-byte load
        const uint32_t i0 = tbase + threadIdx.x * 8u;
        if (i0 + 8u <= n) {
            const uint2 v = *reinterpret_cast<const uint2*>(sb.ndig + i0);
#pragma unroll
            for (int k = 0; k < 4; ++k) atomicAdd(&h[(v.x >> (8 * k)) & 255u], 1u);
#pragma unroll
            for (int k = 0; k < 4; ++k) atomicAdd(&h[(v.y >> (8 * k)) & 255u], 1u);
        } else {
            for (uint32_t i = i0; i < n && i < i0 + 8u; ++i) atomicAdd(&h[sb.ndig[i]], 1u);
        }
    }
    __syncthreads();
    sb.tcnt[(size_t)blockIdx.x * 256 + threadIdx.x] = h[threadIdx.x];
}

// One CTA per digit: that digit's offset in every tile for pass j, relative to the
// digit's first slot, and the digit's total (the scatter adds the digit bases).
__global__ void __launch_bounds__(1024) k_sort_scan(uint32_t j, uint32_t n, SortBuffers sb, BatchMeta* bm) {
    __shared__ uint32_t s_tmp[33];
    const SortPlan& P = bm->plan;
    if (j >= P.npass) return;
    const uint32_t d = blockIdx.x;
    const uint32_t ntiles = (n + kTile - 1) / kTile;
    const uint32_t per = (ntiles + 1023u) / 1024u;
    const uint32_t t0 = min(threadIdx.x * per, ntiles), t1 = min(t0 + per, ntiles);
    uint32_t c[4];
    uint32_t sum = 0;
    if (per <= 4) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            c[k] = (t0 + k < t1) ? sb.tcnt[(size_t)(t0 + k) * 256 + d] : 0u;
            sum += c[k];
        }
    } else {
        for (uint32_t t = t0; t < t1; ++t) sum += sb.tcnt[(size_t)t * 256 + d];
    }
    uint32_t total;
    uint32_t run = block_excl_sum<1024>(sum, s_tmp, &total);
    if (threadIdx.x == 0) sb.dofs[d] = total;  // digit total of this pass
    if (per <= 4) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (t0 + k < t1) {
                sb.toff[(size_t)(t0 + k) * 256 + d] = run;
                run += c[k];
            }
        }
    } else {
        for (uint32_t t = t0; t < t1; ++t) {
            const uint32_t cc = sb.tcnt[(size_t)t * 256 + d];
            sb.toff[(size_t)t * 256 + d] = run;
            run += cc;
        }
    }
}

__global__ void __launch_bounds__(kThreads, 4) k_sort_pass(uint32_t j, uint32_t n, SortBuffers sb,
                                                           BatchMeta* bm, uint32_t* err) {
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
    // Rank within the warp: elements are visited in index order (k, then lane). The
    // lanes holding the same digit are found with nine ballots (validity + 8 bits);
    // the lowest of them adds the group's size to the warp's counter for that digit
    // with one shared-memory atomic, whose old value is the group's base. The
    // __syncwarp orders the atomics of consecutive items, so equal digits keep index
    // order (stability); the bases are gathered only after the loop.
    const uint32_t lt = lanemask_lt();
    uint32_t lower[kItems], old[kItems], lead[kItems];
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        const uint32_t d = dig[k];
        uint32_t peers = __ballot_sync(0xffffffffu, d < 256u);
        if (d >= 256u) peers = ~peers;
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            const uint32_t m = __ballot_sync(0xffffffffu, (d >> b) & 1u);
            peers &= ((d >> b) & 1u) ? m : ~m;
        }
        lead[k] = (uint32_t)(__ffs(peers) - 1);
        lower[k] = __popc(peers & lt);
        old[k] = 0;
        if (lower[k] == 0 && d < 256u) old[k] = atomicAdd(&s_whist[warp][d], (uint32_t)__popc(peers));
        __syncwarp();
    }
#pragma unroll
    for (int k = 0; k < kItems; ++k) rank[k] = __shfl_sync(0xffffffffu, old[k], (int)lead[k]) + lower[k];
    __syncthreads();
    // Thread tid owns digit tid: tile total and per-warp exclusive prefix.
    uint32_t total = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
        uint32_t c = s_whist[w][tid];
        s_whist[w][tid] = total;
        total += c;
    }
    const uint32_t dbase = block_excl_sum<kThreads>(sb.dofs[tid], s_tmp, nullptr);  // digit bases
    s_gbase[tid] = dbase + sb.toff[(size_t)tile * 256 + tid];
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

}  // namespace

cudaError_t launch_sort(const uint8_t* ops, const uint64_t* keys, uint32_t n, const SortBuffers& sb,
                        BatchMeta* bm, uint32_t* err, uint32_t& epoch, cudaStream_t s, int num_sms) {
    if (n == 0) return cudaSuccess;
    int grid = min((int)((n + 255) / 256), num_sms * 8);
    k_pack<<<grid, 256, 0, s>>>(ops, keys, n, sb.in_k, sb.in_p, bm);
    k_sort_plan<<<1, 256, 0, s>>>(n, bm, sb.tile_max);
    static bool attr_set = false;
    const int dyn = kTile * (int)(sizeof(uint64_t) + sizeof(uint32_t));
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_sort_pass, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    const uint32_t tiles = (n + kTile - 1) / kTile;
    k_sort_count<<<tiles, kThreads, 0, s>>>(0, n, sb, bm);
    for (uint32_t j = 0; j < 8; ++j) {
        k_sort_scan<<<256, 1024, 0, s>>>(j, n, sb, bm);
        k_sort_pass<<<tiles, kThreads, dyn, s>>>(j, n, sb, bm, err);
        if (j + 1 < 8) k_sort_count<<<tiles, kThreads, 0, s>>>(j + 1, n, sb, bm);
    }
    (void)epoch;
    return cudaGetLastError();
}

}  // namespace pi
