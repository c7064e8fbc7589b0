// K2 + K3: descend the index layer to each query's interception (Algorithm 2,
// Definition 4), then locate the query's key in the storage layer (Algorithm 4's
// getNode), for every query of the sorted batch.
//
// Layout (built by the rebuild): all index levels live in one key array and one down
// array, top level first; level l is [base[l], base[l] + n[l]) followed by a sentinel
// entry with key 2^64-1. down[i] is the position of the same key in the level below
// (for the lowest built level: its storage-layer position), so the keys of level l-1
// that lie between two consecutive keys of level l are exactly
// [down[r], down[r + 1]). The top levels are copied once per CTA into shared memory
// with one TMA bulk copy each for keys and downs.
//
// Per level, a warp holds 32 consecutive sorted queries (the paper's query group,
// Section 4.4.3, processed level by level). Lanes whose key equals the previous lane's
// key do not search: they take their leader's result at the end. Two search forms:
//  * warp-cooperative (the SIMD-compare analogue of Section 3.2.1): when the leaders'
//    start positions lie within 16 entries, the warp loads one 32-key segment with one
//    coalesced access, and every lane finds the rank of the largest segment key <= its
//    query by a five-step binary search over the lanes (shuffles); __ballot_sync
//    locates the level's sentinel inside the segment;
//  * per lane: when the leaders are spread out (the lower levels), each lane scans its
//    own gap from its start position, four keys (and their downs) per round.
// Both end at the sentinel, so no bound check is needed on a well-formed level; a
// defensive bound records kErrBounds instead of reading past it.

#include "common.cuh"

namespace pi {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr uint32_t kFull = 0xffffffffu;

// r = largest index >= lo-1 with K[r] <= q (K[lo] <= q unless lo is the head, 0).
// Also returns D[r] (0 if r < 0 or no down array) and K[r].
template <bool kDown>
__device__ __forceinline__ void lane_scan(const uint64_t* K, const uint32_t* D, uint32_t lo, uint32_t lim,
                                          uint64_t q, int32_t& r_out, uint32_t& d_out, uint64_t& k_out,
                                          uint32_t* err) {
    uint32_t i = lo, dprev = 0;
    uint64_t kprev = 0;
    for (;;) {
        if (i > lim) {
            atomicOr(err, kErrBounds);
            r_out = -1;
            d_out = 0;
            k_out = 0;
            return;
        }
        const uint64_t k0 = K[i], k1 = K[i + 1], k2 = K[i + 2], k3 = K[i + 3];
        uint32_t d0 = 0, d1 = 0, d2 = 0, d3 = 0;
        if (kDown) {
            d0 = D[i];
            d1 = D[i + 1];
            d2 = D[i + 2];
            d3 = D[i + 3];
        }
        if (k0 > q) { r_out = (int32_t)i - 1; d_out = dprev; k_out = kprev; return; }
        if (k1 > q) { r_out = (int32_t)i;     d_out = d0;    k_out = k0;    return; }
        if (k2 > q) { r_out = (int32_t)i + 1; d_out = d1;    k_out = k1;    return; }
        if (k3 > q) { r_out = (int32_t)i + 2; d_out = d2;    k_out = k2;    return; }
        dprev = d3;
        kprev = k3;
        i += 4;
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
    if (scan) lane_scan<kDown>(K, D, lo, lim, q, r, dn, kr, err);
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

__global__ void __launch_bounds__(kThreads, 6) k_descend(DescendArgs a) {
    extern __shared__ __align__(16) uint8_t s_dyn[];
    uint64_t* s_k = reinterpret_cast<uint64_t*>(s_dyn);
    uint32_t* s_d = reinterpret_cast<uint32_t*>(s_dyn + (kSmemTopMax + kPad) * sizeof(uint64_t));
    __shared__ __align__(8) uint64_t s_bar;
    __shared__ uint32_t s_base[kLevelSlots], s_n[kLevelSlots];
    __shared__ int s_fail;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const DevMeta* m = a.m;
    if (block_sees_error(&m->error)) return;
    const uint32_t H = m->H, Lb = m->Lb, Ls = m->Ls, E = m->smem_entries;
    const uint32_t size = m->size, cur = m->cur;
    const uint32_t qv = a.n - a.bm->invalid;
    if (tid < kLevelSlots) {
        s_base[tid] = m->base[tid];
        s_n[tid] = m->n[tid];
    }
    if (tid == 0) s_fail = 0;
    if (E > 0) {
        if (tid == 0) {
            mbar_init(&s_bar, 1);
            const uint32_t bk = ((E * 8u + 15u) / 16u) * 16u;
            const uint32_t bd = ((E * 4u + 15u) / 16u) * 16u;
            mbar_arrive_expect_tx(&s_bar, bk + bd);
            bulk_g2s(s_k, a.lkeys, bk, &s_bar);
            bulk_g2s(s_d, a.ldown, bd, &s_bar);
        }
        __syncthreads();
        if (!mbar_wait_bounded(&s_bar, 0, a.err)) s_fail = 1;
        __syncthreads();
        if (s_fail) {
            if (tid == 0) mbar_wait_bounded(&s_bar, 0, a.err);  // let the copy land
            return;
        }
    } else {
        __syncthreads();
    }

    const uint64_t* SK = a.st.keys[cur];
    const uint8_t* SM = a.st.meta[cur];
    const uint64_t* SV = a.st.vals[cur];
    for (uint32_t chunk = blockIdx.x * kWarps + warp; chunk * 32u < qv; chunk += gridDim.x * kWarps) {
        const uint32_t i = chunk * 32u + lane;
        const bool active = i < qv;
        const uint64_t q = active ? a.sk[i] : kMaxKey;
        const uint64_t qp = __shfl_up_sync(kFull, q, 1);
        const bool leader = active && (lane == 0 || qp != q);
        const uint32_t lead = __ballot_sync(kFull, leader);
        {
            // run markers for the ownership scan: e = 2i+3 for a write, 2i+2 for a run
            // head, else 0; the tile's maximum feeds the scan across apply tiles
            const uint32_t op = active ? (a.sp[i] >> 30) : 0u;
            const uint64_t before = (lane == 0) ? (i > 0 ? a.sk[i - 1] : kMaxKey) : qp;
            const bool head = active && (i == 0 || before != q);
            const uint32_t e = (active && (op == 1u || op == 2u)) ? 2u * i + 3u : (head ? 2u * i + 2u : 0u);
            const uint32_t wmax = __reduce_max_sync(kFull, e);
            if (lane == 0 && wmax) atomicMax(&a.tile_max[i / kApplyTile], wmax);
        }
        uint32_t lo = 0;
        int32_t r = -1;
        uint32_t dn = 0;
        uint64_t kr = 0;
        int top = (int)H;
        if (Ls <= H) {
            // The pinned levels Ls..H are in shared memory. Level Ls holds every key of
            // the levels above it, so the entry the walk down those levels would reach
            // on level Ls -- its largest key <= q -- is found by one binary search.
            if (leader) {
                r = smem_rank(s_k + s_base[Ls], s_n[Ls], q);
                lo = (r >= 0) ? s_d[s_base[Ls] + r] : 0u;
            }
            top = (int)Ls - 1;
        }
        for (int l = top; l >= (int)Lb; --l) {
            const uint64_t* K = a.lkeys + s_base[l];
            const uint32_t* D = a.ldown + s_base[l];
            r = -1;
            dn = 0;
            warp_search<true>(K, D, lo, s_n[l], q, leader, r, dn, kr, a.err);
            if (leader) lo = (r >= 0) ? dn : 0u;
        }
        r = -1;
        kr = 0;
        warp_search<false>(SK, nullptr, lo, size, q, leader, r, dn, kr, a.err);
        const bool exists = leader && r >= 0 && kr == q;
        const uint8_t meta = exists ? SM[r] : (uint8_t)0;
        const bool live = exists && !(meta & kTomb);
        const uint64_t v = live ? SV[r] : 0ull;
        const int src = 31 - __clz(lead & lanemask_le());
        const int32_t r_l = __shfl_sync(kFull, r, src);
        const uint32_t f_l = __shfl_sync(kFull, (exists ? 1u : 0u) | (live ? 2u : 0u), src);
        const uint64_t v_l = __shfl_sync(kFull, v, src);
        if (active) {
            a.loc[i] = (uint32_t)(r_l + 1);
            a.flags[i] = (uint8_t)f_l;
            a.val0[i] = v_l;
        }
    }
}

}  // namespace

cudaError_t launch_descend(const DescendArgs& a, cudaStream_t s, int num_sms) {
    static bool attr_set = false;
    const int dyn = (int)((kSmemTopMax + kPad) * (sizeof(uint64_t) + sizeof(uint32_t)));
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_descend, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    if (a.n == 0) return cudaSuccess;
    uint32_t warps_needed = (a.n + 31) / 32;
    uint32_t blocks = (warps_needed + kWarps - 1) / kWarps, cap = (uint32_t)num_sms * 6u;
    int grid = (int)(blocks < cap ? blocks : cap);
    k_descend<<<grid, kThreads, dyn, s>>>(a);
    return cudaGetLastError();
}

}  // namespace pi
