// K4 + K5: single ownership and query execution (Algorithms 3 and 4, Section 3.2.4).
//
// In the paper each execution thread owns the storage nodes between its first
// interception and the next thread's, handing queries over to its neighbour so that
// no node has two writers; within a thread the queries run in order. Here the whole
// sorted batch is one array and ownership is computed, not negotiated:
//  * a key run is a maximal stretch of equal keys in the sorted batch (its queries are
//    in arrival order, by the stable sort);
//  * every query reports the state of its key just before it: that is the effect of
//    the last insert/delete before it in its run, or, if there is none, the state the
//    descent found in the storage layer. An inclusive max-scan over
//        e_i = 2i+3 if query i writes, 2i+2 if it heads a run, 0 otherwise
//    gives, at i-1, either the index of that last write (odd) or the run head (even);
//  * the LAST query of each run is the run's only owner: it writes the run's final
//    state to the storage node (value, delete flag), or emits a new node when the key
//    is not in the storage layer and ends up present (Algorithm 4, insertNode).
//
// The max-scan is split across kernels so no tile of k_apply ever waits on another:
// the descent's first kernel already walks the sorted batch and leaves each 2048-query
// tile's exclusive max prefix of e (tile_pref); k_apply is then fully data-parallel. The descent stored one result per distinct key -- per local
// run head (a query whose key differs from the previous one, and the first query of
// every 256-query sub-tile) in sorted order -- so a query's storage-layer state is
// found at its run head's dense index.
// New nodes are staged per tile and packed in key order by k_new_scan + k_new_pack.

#include "common.cuh"

namespace pi {
namespace {

constexpr int kThreads = 256;
constexpr int kApThreads = 512;                  // k_apply: two CTAs per SM at 64 registers
constexpr int kItems = kApplyTile / kApThreads;  // 4 sorted queries per thread
constexpr uint32_t kSeqMask = (1u << 30) - 1u;

__device__ __forceinline__ void store_result(pi_result_t* res, uint32_t seq, uint64_t v, uint32_t st) {
    uint4 w;
    w.x = (uint32_t)v;
    w.y = (uint32_t)(v >> 32);
    w.z = st;
    w.w = 0u;
    *reinterpret_cast<uint4*>(res + seq) = w;
}

__global__ void __launch_bounds__(kApThreads, 2) k_apply(ApplyArgs a) {
    pdl_wait();
    pdl_trigger();
    __shared__ uint32_t s_tmp[33];
    __shared__ int32_t s_delta[kLevelSlots];
    __shared__ int32_t s_tomb;
    __shared__ uint32_t s_changes, s_dirty;
    __shared__ uint32_t s_chist[kLevelSlots];  // built-level membership changes by height

    const int tid = threadIdx.x;
    if (block_sees_error(&a.m->error)) return;
    const uint32_t n = a.n;
    const uint32_t qv = n - a.bm->invalid;
    const uint32_t cur = a.m->cur;
    const uint32_t Lb = a.m->Lb;  // lowest built index level: changes below it leave the index alone
    uint64_t* SV = a.st.vals[cur];
    uint8_t* SM = a.st.meta[cur];
    const uint32_t tile = blockIdx.x;
    if (tid < kLevelSlots) {
        s_delta[tid] = 0;
        s_chist[tid] = 0;
    }
    if (tid == 0) {
        s_tomb = 0;
        s_changes = 0;
        s_dirty = 0;
    }
    const uint32_t base = tile * kApplyTile + tid * kItems;

    uint64_t key[kItems];
    uint32_t pay[kItems];
    uint32_t e[kItems];
    uint32_t dres[kItems];
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        const uint32_t i = base + k;
        key[k] = i < qv ? a.sk[i] : kMaxKey;
        pay[k] = i < n ? a.sp[i] : 0u;
    }
    const uint64_t kprev = (base > 0 && base - 1 < qv) ? a.sk[base - 1] : kMaxKey;
    const uint64_t knext = (base + kItems < qv) ? a.sk[base + kItems] : kMaxKey;
    // the descent's prefixes for this tile (its markers' maximum before it, the dense
    // index of its first local run head), loaded with the batch (a block barrier below
    // would keep them from being hoisted)
    const uint32_t tpref = a.tile_pref[tile];
    const uint32_t dbase = a.sub_pref[tile * (kApplyTile / kSubTile)];
    uint32_t agg = 0;
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        const uint32_t i = base + k;
        const bool valid = i < qv;
        const uint64_t prev = k ? key[k - 1] : kprev;
        const bool head = valid && (i == 0 || key[k] != prev);
        const uint32_t op = pay[k] >> 30;
        const bool write = valid && (op == 1u || op == 2u);
        e[k] = write ? 2u * i + 3u : (head ? 2u * i + 2u : 0u);
        agg = max(agg, e[k]);
    }
    const uint32_t texcl = block_excl_max<kApThreads>(agg, s_tmp, nullptr);
    uint32_t M = max(tpref, texcl);
    // dense index of each query's local run head: the tile's first one plus the local
    // heads before it in the tile (a local head is a run head or a 256-query sub-tile's
    // first query, as the descent counted them)
    uint32_t lh = 0, nh = 0;
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        const uint32_t i = base + k;
        const uint64_t prev = k ? key[k - 1] : kprev;
        const bool local = i < qv && (i == 0 || key[k] != prev || (i % kSubTile) == 0);
        lh |= (local ? 1u : 0u) << k;
        nh += local ? 1u : 0u;
    }
    uint32_t hidx = dbase + block_excl_sum<kApThreads>(nh, s_tmp, nullptr);  // dense index of the next head
    uint32_t new_here = 0, new_mask = 0, chg_here = 0, chg_mask = 0;
    // Per query: its run head's result index, and the gathers of its prior state, all
    // issued before any store so that their latencies overlap: the run head's state, or,
    // when an earlier query of its run wrote (the marker names it), that query's payload.
    uint32_t fromw = 0, insw = 0, flx = 0;  // bit k: from an earlier write; that write inserts; flags
    uint64_t val[kItems];
    uint32_t pj[kItems];
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        const uint32_t mex = M;
        const uint32_t minc = max(M, e[k]);
        M = minc;
        e[k] = minc;  // keep the inclusive value for the owners and the new-node pass
        dres[k] = hidx + ((lh >> k) & 1u) - 1u;  // this query's run head's result
        hidx += (lh >> k) & 1u;
        const uint64_t prev = k ? key[k - 1] : kprev;
        const bool q = base + k < qv;
        const bool fw = q && (base + k != 0 && key[k] == prev) && (mex & 1u);
        fromw |= (fw ? 1u : 0u) << k;
        flx |= (q ? (uint32_t)a.flags[dres[k]] : 0u) << (2 * k);
        val[k] = q ? a.val0[dres[k]] : 0ull;
        pj[k] = fw ? a.sp[(mex - 3u) >> 1] : 0u;
    }
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        if (!((fromw >> k) & 1u)) {
            if (!((flx >> (2 * k + 1)) & 1u)) val[k] = 0ull;  // the run head's key is not live
            continue;
        }
        const bool ins = (pj[k] >> 30) == 1u;
        insw |= (ins ? 1u : 0u) << k;
        val[k] = ins ? a.uvals[pj[k] & kSeqMask] : 0ull;
    }
#pragma unroll
    for (int k = 0; k < kItems; ++k) {
        const uint32_t i = base + k;
        if (i >= n) continue;
        const uint32_t seq = pay[k] & kSeqMask;
        if (i >= qv) {
            store_result(a.results, seq, 0ull, PI_R_INVALID);
            continue;
        }
        const uint32_t dj = dres[k];
        const bool exists = (flx >> (2 * k)) & 1u, live0 = (flx >> (2 * k + 1)) & 1u;
        const bool pl = ((fromw >> k) & 1u) ? ((insw >> k) & 1u) != 0 : live0;
        store_result(a.results, seq, val[k], pl ? PI_R_PRESENT : PI_R_ABSENT);

        const uint64_t next = (k + 1 < kItems) ? key[k + 1] : knext;
        const bool last = next != key[k];
        const uint32_t minc = e[k];
        if (!last || !(minc & 1u)) continue;  // not the owner, or the run never writes
        const uint32_t jw = (minc - 3u) >> 1;
        const uint32_t pw = (jw == i) ? pay[k] : a.sp[jw];
        const bool fin_live = (pw >> 30) == 1u;
        if (exists) {
            const uint32_t r = a.loc[dj] - 1u;
            if (a.wcount) atomicAdd(&a.wcount[r], 1u);
            const uint8_t mt = SM[r];
            const uint32_t h = mt & kHeightMask;
            if (fin_live) {
                SV[r] = a.uvals[pw & kSeqMask];
                SM[r] = (uint8_t)h;
            } else {
                SM[r] = (uint8_t)(h | kTomb);
            }
            if (fin_live != live0) {
                atomicAdd(&s_tomb, fin_live ? -1 : 1);
                atomicAdd(&s_changes, 1u);
                atomicAdd(&s_delta[1], fin_live ? 1 : -1);
                for (uint32_t l = 2; l <= h; ++l) {
                    atomicAdd(&s_delta[l], fin_live ? 1 : -1);
                    // the rebuild's per-tile count of the node's 4096-node tile
                    atomicAdd(&a.lcnt[(size_t)(l - 2) * a.lstride + (r >> 12)], fin_live ? 1u : 0xFFFFFFFFu);
                }
                if (h >= Lb) {
                    s_dirty = 1;
                    chg_here++;
                    chg_mask |= 1u << k;
                }
            }
        } else if (fin_live) {
            new_here++;
            new_mask |= 1u << k;
        }
    }
    // New nodes: staged in this tile's slice of the staging arrays, in key order.
    uint32_t tile_new = 0, slot = 0;
    if (__syncthreads_or(new_here != 0)) slot = block_excl_sum<kApThreads>(new_here, s_tmp, &tile_new);
    if (new_mask) {
        const uint32_t so = tile * kApplyTile;
#pragma unroll
        for (int k = 0; k < kItems; ++k) {
            if (!(new_mask & (1u << k))) continue;
            const uint32_t i = base + k;
            const uint32_t jw = (e[k] - 3u) >> 1;
            const uint32_t pw = (jw == i) ? pay[k] : a.sp[jw];
            const uint32_t h = tower_height(key[k], a.hp);
            a.stage.keys[so + slot] = key[k];
            a.stage.vals[so + slot] = a.uvals[pw & kSeqMask];
            a.stage.loc[so + slot] = a.loc[dres[k]];
            a.stage.height[so + slot] = (uint8_t)h;
            ++slot;
            atomicAdd(&s_changes, 1u);
            atomicAdd(&s_delta[1], 1);
            for (uint32_t l = 2; l <= h; ++l) atomicAdd(&s_delta[l], 1);
            if (h >= 2) s_dirty = 1;
        }
    }
    // Built-level membership changes: staged the same way, for an incremental rebuild.
    uint32_t tile_chg = 0, cslot = 0;
    if (__syncthreads_or(chg_here != 0)) cslot = block_excl_sum<kApThreads>(chg_here, s_tmp, &tile_chg);
    if (chg_mask) {
        const uint32_t so = tile * kApplyTile;
#pragma unroll
        for (int k = 0; k < kItems; ++k) {
            if (!(chg_mask & (1u << k))) continue;
            const uint32_t r = a.loc[dres[k]] - 1u;
            const uint8_t mt = SM[r];  // as this kernel left it
            const uint32_t h = mt & kHeightMask;
            a.cstage.keys[so + cslot] = key[k];
            a.cstage.pos[so + cslot] = r;
            a.cstage.hl[so + cslot] = (uint8_t)(h | ((mt & kTomb) ? 0u : 0x80u));
            ++cslot;
            atomicAdd(&s_chist[h < (uint32_t)kLevelSlots ? h : kLevelSlots - 1], 1u);
        }
    }
    __syncthreads();
    if (tid == 0) {
        a.tile_new[tile] = tile_new;
        a.tile_chg[tile] = tile_chg;
    }
    if (tid < kLevelSlots && s_chist[tid]) atomicAdd(&a.bm->chg_hist[tid], s_chist[tid]);
    if (tid < kLevelSlots && s_delta[tid]) atomicAdd(&a.bm->delta[tid], s_delta[tid]);
    if (tid == 0) {
        if (s_tomb) atomicAdd(&a.bm->tomb_delta, s_tomb);
        if (s_changes) atomicAdd(&a.bm->changes, s_changes);
        if (s_dirty) atomicOr(&a.bm->index_dirty, 1u);
    }
}

// Exclusive sums of the per-tile new-node and level-change counts (one CTA); totals ->
// bm->new_count and bm->nchg.
__global__ void __launch_bounds__(1024) k_new_scan(ApplyArgs a) {
    pdl_wait();
    pdl_trigger();
    __shared__ uint32_t s_tmp[33];
    __shared__ uint32_t s_carry, s_ccarry;
    if (block_sees_error(&a.m->error)) return;
    const uint32_t ntiles = (a.n + kApplyTile - 1) / kApplyTile;
    if (threadIdx.x == 0) {
        s_carry = 0;
        s_ccarry = 0;
    }
    __syncthreads();
    for (uint32_t b0 = 0; b0 < ntiles; b0 += 1024) {
        const uint32_t i = b0 + threadIdx.x;
        const uint32_t v = i < ntiles ? a.tile_new[i] : 0u;
        const uint32_t c = i < ntiles ? a.tile_chg[i] : 0u;
        uint32_t tot, ctot;
        const uint32_t ex = block_excl_sum<1024>(v, s_tmp, &tot);
        const uint32_t cex = block_excl_sum<1024>(c, s_tmp, &ctot);
        if (i < ntiles) {
            a.tile_pref[i] = s_carry + ex;  // tile_pref is free again
            a.tile_chg_pref[i] = s_ccarry + cex;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            s_carry += tot;
            s_ccarry += ctot;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        a.bm->new_count = s_carry;
        a.bm->nchg = s_ccarry;
    }
}

// Packs each tile's staged new nodes and level changes to their places in key order.
__global__ void __launch_bounds__(kThreads) k_new_pack(ApplyArgs a) {
    pdl_wait();
    pdl_trigger();
    if (*(volatile const uint32_t*)&a.m->error) return;  // no barrier in this kernel
    const uint32_t tile = blockIdx.x;
    const uint32_t so = tile * kApplyTile;
    const uint32_t c = a.tile_new[tile];
    if (c) {
        const uint32_t dst = a.tile_pref[tile];
        for (uint32_t j = threadIdx.x; j < c; j += kThreads) {
            a.nn.keys[dst + j] = a.stage.keys[so + j];
            a.nn.vals[dst + j] = a.stage.vals[so + j];
            a.nn.loc[dst + j] = a.stage.loc[so + j];
            a.nn.height[dst + j] = a.stage.height[so + j];
        }
    }
    const uint32_t cc = a.tile_chg[tile];
    if (cc) {
        const uint32_t dst = a.tile_chg_pref[tile];
        for (uint32_t j = threadIdx.x; j < cc; j += kThreads) {
            a.chg.keys[dst + j] = a.cstage.keys[so + j];
            a.chg.pos[dst + j] = a.cstage.pos[so + j];
            a.chg.hl[dst + j] = a.cstage.hl[so + j];
        }
    }
}

// Debug check of single ownership (Section 3.2.4): after k_apply, every storage node
// has been written by at most one query. Counts are summed into DevMeta::owner_writes
// and cleared for the next batch.
__global__ void __launch_bounds__(kThreads) k_owner_check(ApplyArgs a) {
    pdl_wait();
    pdl_trigger();
    __shared__ uint32_t s_sum;
    if (threadIdx.x == 0) s_sum = 0;
    __syncthreads();
    const uint32_t size = a.m->size;
    uint32_t sum = 0;
    for (uint32_t i = blockIdx.x * kThreads + threadIdx.x; i < size; i += gridDim.x * kThreads) {
        const uint32_t c = a.wcount[i];
        if (c) {
            sum += c;
            if (c > 1u) atomicOr(a.err, kErrOwner);
            a.wcount[i] = 0u;
        }
    }
    sum = __reduce_add_sync(0xffffffffu, sum);
    if ((threadIdx.x & 31) == 0 && sum) atomicAdd(&s_sum, sum);
    __syncthreads();
    if (threadIdx.x == 0 && s_sum) atomicAdd(&a.m->owner_writes, s_sum);
}

}  // namespace

cudaError_t launch_apply(const ApplyArgs& a, uint32_t& epoch, cudaStream_t s, int num_sms) {
    (void)epoch;
    (void)num_sms;
    if (a.n == 0) return cudaSuccess;
    const uint32_t tiles = (a.n + kApplyTile - 1) / kApplyTile;
    launch_dep(k_apply, tiles, kApThreads, 0, s, a);  // tile prefixes come from the descent's scan
    ++g_launches;
    launch_dep(k_new_scan, 1, 1024, 0, s, a);
    ++g_launches;
    launch_dep(k_new_pack, tiles, kThreads, 0, s, a);
    ++g_launches;
    return cudaGetLastError();
}

cudaError_t launch_owner_check(const ApplyArgs& a, cudaStream_t s, int num_sms) {
    if (!a.wcount) return cudaSuccess;
    launch_dep(k_owner_check, (uint32_t)num_sms * 8u, kThreads, 0, s, a);
    ++g_launches;
    return cudaGetLastError();
}

}  // namespace pi
