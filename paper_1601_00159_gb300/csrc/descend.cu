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

// Persistent warps over sub-tiles of kSubTile (256) sorted queries; warp-global index
// gw = blockIdx.x * 8 + warp takes sub-tiles gw, gw + 8 * gridDim.x, ... Per sub-tile
// the warp, without block barriers,
//  1. marks the local run heads (a query whose key differs from the previous query's,
//     and the sub-tile's first query) and compacts their keys, in order, into its own
//     shared-memory list -- equal keys are searched once;
//  2. folds the sub-tile's ownership markers e (see the apply kernel) into its apply
//     tile's maximum;
//  3. descends the list with full warps (32 keys per step) and writes one result per
//     local head at sub_base + its index among the sub-tile's local heads.
__global__ void __launch_bounds__(kThreads, 5) k_descend(DescendArgs a) {
    extern __shared__ __align__(16) uint8_t s_dyn[];
    uint64_t* s_k = reinterpret_cast<uint64_t*>(s_dyn);
    uint32_t* s_d = reinterpret_cast<uint32_t*>(s_dyn + (kSmemTopMax + kPad) * sizeof(uint64_t));
    uint64_t* s_qall = reinterpret_cast<uint64_t*>(s_dyn + (kSmemTopMax + kPad) * 12);  // 8 x kSubTile keys
    __shared__ __align__(8) uint64_t s_bar;
    __shared__ uint32_t s_base[kLevelSlots], s_n[kLevelSlots];
    __shared__ int s_fail;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const DevMeta* m = a.m;
    if (block_sees_error(&m->error)) return;
    const uint32_t H = m->H, Lb = m->Lb, Ls = m->Ls, E = m->smem_entries;
    const uint32_t size = m->size, cur = m->cur;
    const uint32_t n = a.n;
    const uint32_t qv = n - a.bm->invalid;
    const uint32_t nsub = (n + kSubTile - 1) / kSubTile;
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
    uint64_t* s_q = s_qall + warp * kSubTile;
    const uint32_t lt = lanemask_lt();
    for (uint32_t sub = blockIdx.x * (kThreads / 32) + warp; sub < nsub; sub += gridDim.x * (kThreads / 32)) {
        const uint32_t sb = sub * kSubTile;
        // 1 + 2: striped over the sub-tile: element sb + 32 k + lane
        uint32_t nq = 0, emax = 0;
        uint64_t carry = (sb > 0 && sb - 1 < qv) ? a.sk[sb - 1] : kMaxKey;  // key before the element
#pragma unroll 2
        for (int k = 0; k < kSubTile / 32; ++k) {
            const uint32_t i = sb + (uint32_t)k * 32u + (uint32_t)lane;
            const bool valid = i < qv;
            const uint64_t q = valid ? a.sk[i] : kMaxKey;
            const uint32_t op = valid ? (a.sp[i] >> 30) : 0u;
            uint64_t prev = __shfl_up_sync(0xffffffffu, q, 1);
            if (lane == 0) prev = carry;
            carry = __shfl_sync(0xffffffffu, q, 31);
            const bool head = valid && (i == 0 || q != prev);
            const bool local = valid && (head || (k == 0 && lane == 0));
            const uint32_t e = (valid && (op == 1u || op == 2u)) ? 2u * i + 3u : (head ? 2u * i + 2u : 0u);
            emax = max(emax, e);
            const uint32_t b = __ballot_sync(0xffffffffu, local);
            if (local) s_q[nq + __popc(b & lt)] = q;
            nq += __popc(b);
        }
        emax = __reduce_max_sync(0xffffffffu, emax);
        if (lane == 0 && emax) atomicMax(&a.tile_max[sb / kApplyTile], emax);
        __syncwarp();
        // 3. descend the sub-tile's distinct keys, 32 per step
        for (uint32_t c = 0; c < nq; c += 32u) {
            const uint32_t j = c + (uint32_t)lane;
            const bool active = j < nq;
            const uint64_t q = active ? s_q[j] : kMaxKey;
            uint32_t lo = 0;
            int32_t r = -1;
            uint32_t dn = 0;
            uint64_t kr = 0;
            int top = (int)H;
            if (Ls <= H) {
                // Pinned levels Ls..H are in shared memory; level Ls holds every key of
                // the levels above it, so the entry the walk down those levels reaches
                // on level Ls -- its largest key <= q -- is found by one binary search.
                if (active) {
                    r = smem_rank(s_k + s_base[Ls], s_n[Ls], q);
                    lo = (r >= 0) ? s_d[s_base[Ls] + r] : 0u;
                }
                top = (int)Ls - 1;
            }
            for (int l = top; l >= (int)Lb; --l) {
                r = -1;
                dn = 0;
                warp_search<true>(a.lkeys + s_base[l], a.ldown + s_base[l], lo, s_n[l], q, active, r, dn, kr, a.err);
                if (active) lo = (r >= 0) ? dn : 0u;
            }
            r = -1;
            kr = 0;
            warp_search<false>(SK, nullptr, lo, size, q, active, r, dn, kr, a.err);
            if (active) {
                const bool exists = r >= 0 && kr == q;
                const uint8_t meta = exists ? SM[r] : (uint8_t)0;
                const bool live = exists && !(meta & kTomb);
                const uint32_t o = sb + j;
                a.loc[o] = (uint32_t)(r + 1);
                a.flags[o] = (uint8_t)((exists ? 1u : 0u) | (live ? 2u : 0u));
                a.val0[o] = live ? SV[r] : 0ull;
            }
        }
        __syncwarp();  // the list is reused by the next sub-tile
    }
}

}  // namespace

cudaError_t launch_descend(const DescendArgs& a, cudaStream_t s, int num_sms) {
    static bool attr_set = false;
    const int dyn = (int)((kSmemTopMax + kPad) * (sizeof(uint64_t) + sizeof(uint32_t)) + 8 * kSubTile * sizeof(uint64_t));
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_descend, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    if (a.n == 0) return cudaSuccess;
    const uint32_t blocks = ((a.n + kSubTile - 1) / kSubTile + 7) / 8, cap = (uint32_t)num_sms * 5u;
    k_descend<<<(int)(blocks < cap ? blocks : cap), kThreads, dyn, s>>>(a);
    return cudaGetLastError();
}

}  // namespace pi
