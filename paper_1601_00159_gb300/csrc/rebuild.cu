// K6: storage-layer merge and index-layer rebuild (Sections 4.1 and 4.4.4), plus the
// bulk build of a new index (Section 3.1) and the test-support export.
//
// Storage layer: contiguous sorted arrays keys / vals / meta (meta = height | F_del),
// double buffered. A delete only sets F_del (Algorithm 4), so a deleted node keeps its
// place and a later insert of the same key revives it in place. The storage layer is
// re-laid-out (merge) only when new nodes must be placed, or when delete-flagged nodes
// exceed 1/8 of it; the merge drops every delete-flagged node.
//
// Rebuild: the paper's daemon scans the storage layer and puts the key of every
// valid node of height > 1 into the index-layer arrays. Here one pass over the storage
// layer does it for all levels at once: per tile of 4096 nodes, keys and meta arrive in
// shared memory by TMA bulk copy; the tile counts its live nodes of height >= l for
// every level l; one decoupled look-back per level (a warp, one lane per level) gives
// the tile's offset in each level; then level by level the tile compacts its nodes of
// height >= l (a prefix sum) and writes them with their down pointers.
//
// Level sizes are not counted by the rebuild: the apply kernel keeps them current as
// deltas, so the layout (level bases, sentinels, staging split) is known before the
// pass and the pass writes every entry exactly once.

#include <cstddef>

#include "common.cuh"

namespace pi {
namespace {

constexpr int kThreads = 256;
constexpr int kNodes = 4096;             // storage nodes per tile
constexpr int kPer = kNodes / kThreads;  // 16 per thread
constexpr uint32_t kCtrMerge = 9, kCtrCreate = 11;

__device__ __forceinline__ bool merge_needed(const DevMeta* m, const BatchMeta* bm) {
    const uint32_t size = m->size;
    const uint32_t tombs = (uint32_t)((int32_t)m->tombs + bm->tomb_delta);
    return bm->new_count > 0 || (tombs > 0 && (uint64_t)tombs * 8u > size);
}

// Entries of the sorted a[0, n) below x, by a whole warp (every lane calls it and gets
// the result): each round
// probes 32 evenly spaced entries of the remaining interval at once, so a search of n
// entries takes about log32(n) rounds of one load per lane instead of log2(n) dependent
// loads.
__device__ __forceinline__ uint32_t warp_lower_bound_u32(const uint32_t* a, uint32_t n, uint32_t x) {
    const uint32_t lane = threadIdx.x & 31u;
    uint32_t lo = 0, hi = n;  // the count lies in [lo, hi]
    while (hi - lo > 32u) {
        const uint32_t step = (hi - lo + 31u) / 32u;
        const uint32_t p = lo + lane * step;
        const bool lt = p < hi && a[p] < x;
        const uint32_t c = (uint32_t)__popc(__ballot_sync(0xffffffffu, lt));  // probes below x
        if (c == 0) return lo;
        const uint32_t nlo = lo + (c - 1u) * step + 1u;
        const uint32_t pc = lo + c * step;
        hi = (c < 32u && pc < hi) ? pc : hi;
        lo = nlo;
    }
    const uint32_t p = lo + lane;
    return lo + (uint32_t)__popc(__ballot_sync(0xffffffffu, p < hi && a[p] < x));
}

// ---------------------------------------------------------------------------------
// Merge: old live nodes + new nodes -> the other storage buffer, in key order.
// A new node with loc = x goes right before old node x (after old node x - 1) and is
// handled by the tile that holds position x; the tiles cover positions [0, size].
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
        uint64_t t = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint64_t y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < kThreads / 32) tmp[lane] = t - w;
        if (lane == kThreads / 32 - 1) tmp[32] = t;
    }
    __syncthreads();
    const uint64_t r = tmp[warp] + x - v;
    if (total) *total = tmp[32];
    __syncthreads();
    return r;
}

// Live old nodes of every 4096-node tile (the meta bytes, 16 per thread in one 16-byte
// load; the storage arrays are padded by a whole tile), then, by the last CTA to finish,
// the tiles' exclusive prefix. No CTA waits for another.
__global__ void __launch_bounds__(kThreads) k_merge_count(RebuildArgs a) {
    pdl_wait();
    pdl_trigger();
    constexpr uint32_t kScan = 8;  // tiles per thread in the final scan
    __shared__ uint32_t s_tmp[33], s_warp[kThreads / 32], s_last;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const DevMeta* m = a.m;
    if (block_sees_error(&m->error)) return;
    if (!merge_needed(m, a.bm)) return;
    const uint32_t size = m->size, ntiles = size / kNodes + 1;
    const uint8_t* M0 = a.st.meta[m->cur];
    uint32_t* live = a.mcnt;
    uint32_t* pref = a.mcnt + a.lstride;
    for (uint32_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const uint32_t ts = tile * kNodes;
        const uint32_t cnt = (size > ts) ? min((uint32_t)kNodes, size - ts) : 0u;
        const uint32_t b0 = (uint32_t)tid * kPer;
        const uint4 mw = *reinterpret_cast<const uint4*>(M0 + ts + b0);
        const uint32_t words[4] = {mw.x, mw.y, mw.z, mw.w};
        uint32_t lc = 0;
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            const uint32_t mt = (words[k >> 2] >> (8 * (k & 3))) & 0xFFu;
            lc += (b0 + k < cnt && !(mt & kTomb)) ? 1u : 0u;
        }
        lc = __reduce_add_sync(0xffffffffu, lc);
        if (lane == 0) s_warp[warp] = lc;
        __syncthreads();
        if (tid == 0) {
            uint32_t t = 0;
#pragma unroll
            for (int w = 0; w < kThreads / 32; ++w) t += s_warp[w];
            live[tile] = t;
        }
        __syncthreads();
    }
    if (tid == 0) {
        __threadfence();  // this CTA's counts, before its arrival is counted
        s_last = atomicAdd(&a.bm->tile_ctr[kCtrMerge], 1u) == gridDim.x - 1u;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();  // every CTA has arrived: all counts are visible
    uint32_t carry = 0;
    for (uint32_t g0 = 0; g0 < ntiles; g0 += kThreads * kScan) {
        const uint32_t t0 = g0 + (uint32_t)tid * kScan;
        uint32_t c[kScan], sum = 0;
#pragma unroll
        for (uint32_t k = 0; k < kScan; ++k) {
            c[k] = t0 + k < ntiles ? __ldcg(&live[t0 + k]) : 0u;
            sum += c[k];
        }
        uint32_t tot;
        uint32_t r = carry + block_excl_sum<kThreads>(sum, s_tmp, &tot);
#pragma unroll
        for (uint32_t k = 0; k < kScan; ++k) {
            if (t0 + k < ntiles) pref[t0 + k] = r;
            r += c[k];
        }
        carry += tot;
    }
}

// One 4096-node tile per step: a blocked pass (16 consecutive positions per thread)
// counts the live old nodes and the new nodes inserted at each position, and one block
// scan of both counts gives every position its output offset within the tile (the
// tile's own offset is the count kernel's prefix plus the new nodes of earlier tiles);
// a striped pass then copies the old live nodes with coalesced loads and stores, and
// the new nodes go to their slots.
__global__ void __launch_bounds__(kThreads) k_merge(RebuildArgs a) {
    pdl_wait();
    pdl_trigger();
    __shared__ uint16_t s_lp[kNodes + 1];  // live old nodes before each position of the tile
    __shared__ uint32_t s_nl[kNodes];      // new nodes at or before each position
    __shared__ uint64_t s_tmp[33];
    __shared__ uint32_t s_jb, s_je;
    const int tid = threadIdx.x;
    const DevMeta* m = a.m;
    if (block_sees_error(&m->error)) return;
    if (!merge_needed(m, a.bm)) return;
    const uint32_t size = m->size, src = m->cur, dst = src ^ 1u;
    const uint32_t newc = a.bm->new_count;
    const uint32_t ntiles = size / kNodes + 1;
    const uint64_t* K0 = a.st.keys[src];
    const uint64_t* V0 = a.st.vals[src];
    const uint8_t* M0 = a.st.meta[src];
    uint64_t* K1 = a.st.keys[dst];
    uint64_t* V1 = a.st.vals[dst];
    uint8_t* M1 = a.st.meta[dst];
    for (uint32_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const uint32_t ts = tile * kNodes;
        __syncthreads();  // the previous tile's readers of s_nl and s_lp are done
        if (tid < 64) {  // warp 0: the tile's first new node; warp 1: the next tile's
            const uint32_t r = warp_lower_bound_u32(a.nn.loc, newc, tid < 32 ? ts : ts + kNodes);
            if (tid == 0) s_jb = r;
            if (tid == 32) s_je = r;
        }
        for (int x = tid; x < kNodes; x += kThreads) s_nl[x] = 0u;
        __syncthreads();
        const uint32_t cnt = (size > ts) ? min((uint32_t)kNodes, size - ts) : 0u;
        const uint32_t jb = s_jb, je = s_je;
        // new nodes per insertion position (loc - ts is in [0, kNodes))
        for (uint32_t j = jb + tid; j < je; j += kThreads) {
            const uint32_t x = a.nn.loc[j] - ts;
            if (x < (uint32_t)kNodes) atomicAdd(&s_nl[x], 1u);
            else atomicOr(a.err, kErrBounds);
        }
        __syncthreads();
        // blocked pass: positions [16 tid, 16 tid + 16); the storage arrays are padded by
        // a whole tile, so the 16-byte meta load stays in bounds past the last node
        const uint32_t b0 = (uint32_t)tid * kPer;
        const uint4 mw = *reinterpret_cast<const uint4*>(M0 + ts + b0);
        const uint32_t words[4] = {mw.x, mw.y, mw.z, mw.w};
        uint32_t live_bits = 0, lc = 0, nc = 0;
        uint32_t nat[kPer];
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            const uint32_t mt = (words[k >> 2] >> (8 * (k & 3))) & 0xFFu;
            const bool lv = b0 + k < cnt && !(mt & kTomb);
            live_bits |= (lv ? 1u : 0u) << k;
            lc += lv ? 1u : 0u;
            nat[k] = s_nl[b0 + k];
            nc += nat[k];
        }
        uint64_t tot;
        const uint64_t ex = block_excl_sum64((uint64_t)lc | ((uint64_t)nc << 32), s_tmp, &tot);
        const uint32_t tile_live = (uint32_t)tot;
        {
            uint32_t rl = (uint32_t)ex, rn = (uint32_t)(ex >> 32);
#pragma unroll
            for (int k = 0; k < kPer; ++k) {
                s_lp[b0 + k] = (uint16_t)rl;
                rl += (live_bits >> k) & 1u;
                rn += nat[k];
                s_nl[b0 + k] = rn;
            }
            if (tid == kThreads - 1) s_lp[kNodes] = (uint16_t)rl;
        }
        if (tid == 0 && tile_live != a.mcnt[tile]) atomicOr(a.err, kErrBounds);  // the two counts agree
        __syncthreads();
        const uint32_t out_base = a.mcnt[a.lstride + tile] + jb;
        // striped pass: old live nodes, coalesced; four positions per round, their loads
        // issued together (the source buffer is read-only here)
        for (uint32_t x0 = (uint32_t)tid; x0 < cnt; x0 += 4u * kThreads) {
            uint32_t mt[4];
            uint64_t kv[4], vv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const uint32_t x = x0 + (uint32_t)u * kThreads;
                const bool in = x < cnt;
                mt[u] = in ? (uint32_t)__ldg(M0 + ts + x) : (uint32_t)kTomb;
                kv[u] = in ? __ldg(K0 + ts + x) : 0ull;
                vv[u] = in ? __ldg(V0 + ts + x) : 0ull;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (mt[u] & kTomb) continue;
                const uint32_t x = x0 + (uint32_t)u * kThreads;
                const uint32_t o = out_base + s_lp[x] + s_nl[x];
                if (o >= a.st_cap) {
                    atomicOr(a.err, kErrBounds);
                    continue;
                }
                K1[o] = kv[u];
                V1[o] = vv[u];
                M1[o] = (uint8_t)mt[u];
            }
        }
        // new nodes of this tile, before the old node at their position
        for (uint32_t j = jb + tid; j < je; j += kThreads) {
            const uint32_t x = a.nn.loc[j] - ts;
            if (x >= (uint32_t)kNodes) continue;  // recorded above
            const uint32_t o = out_base + s_lp[x] + (j - jb);
            if (o >= a.st_cap) {
                atomicOr(a.err, kErrBounds);
                continue;
            }
            K1[o] = a.nn.keys[j];
            V1[o] = a.nn.vals[j];
            M1[o] = a.nn.height[j];
        }
    }
}

// ---------------------------------------------------------------------------------
// Layout: apply the batch's deltas, switch storage buffers after a merge, decide the
// rebuild, and lay the index levels out top-first with their sentinels.
// Thread 0: sizes, re-layout switch, rebuild decision and level layout. Returns true
// when the rebuild runs (the sentinels are then written by the caller's lanes).
__device__ bool level_bases_body(RebuildArgs a) {
    DevMeta* m = a.m;
    BatchMeta* bm = a.bm;
    if (*(volatile uint32_t*)&m->error) return false;
    const bool merged = merge_needed(m, bm);
    uint32_t tombs = (uint32_t)((int32_t)m->tombs + bm->tomb_delta);
    uint32_t size = m->size;
    if (merged) {
        size = size - tombs + bm->new_count;
        tombs = 0;
        m->cur ^= 1u;
    }
    if (size > a.st_cap) {  // cannot happen when the host reserved capacity
        atomicOr(a.err, kErrBounds);
        return false;
    }
    m->size = size;
    m->tombs = tombs;
    bm->merged = merged ? 1u : 0u;
    const uint32_t cur = m->cur;
    a.st.keys[cur][size] = kMaxKey;
    a.st.vals[cur][size] = 0;
    a.st.meta[cur][size] = 0;
    for (int l = 1; l < kLevelSlots; ++l) m->cnt[l] = (uint32_t)((int32_t)m->cnt[l] + bm->delta[l]);
    m->updates += bm->changes;
    m->sort_fix_big = bm->fix_big;
    if (a.force_rebuild != 2u) m->batches += 1;

    bool rebuild = a.force_rebuild || merged;
    if (!rebuild && bm->index_dirty) {
        if (a.rebuild_policy == 0) rebuild = true;
        else rebuild = (uint64_t)m->updates * 100u >= (uint64_t)a.threshold_pct * (uint64_t)(size ? size : 1u);
    }
    bm->rebuild = rebuild ? 1u : 0u;
    if (!rebuild) {
        if (bm->index_dirty) m->levels_exact = 0;  // deferred: the levels now lag the storage layer
        return false;
    }
    m->updates = 0;
    m->rebuilds += 1;
    // the layout being replaced, for an incremental rebuild
    const uint32_t oH = m->H, oLb = m->Lb;
    bm->old_H = oH;
    bm->old_total = m->index_total;
    for (int l = 0; l < kLevelSlots; ++l) {
        bm->old_n[l] = m->n[l];
        bm->old_base[l] = m->base[l];
    }

    uint32_t H = 1;
    for (int l = 2; l < kLevelSlots; ++l)
        if (m->cnt[l] > 0) H = (uint32_t)l;
    // Lowest level that fits: drop bottom levels (the descent then scans longer storage
    // gaps) rather than overrun the capacity; the host grows it later.
    const uint32_t Lb0 = a.min_lb > 2u ? a.min_lb : 2u;
    uint64_t need = 0;
    for (uint32_t l = Lb0; l <= H; ++l) need += (uint64_t)m->cnt[l] + 1u;
    uint32_t Lb = Lb0;
    uint64_t fit = need;
    while (Lb <= H && fit > a.index_cap) {
        fit -= (uint64_t)m->cnt[Lb] + 1u;
        ++Lb;
    }
    m->index_need = (uint32_t)need;
    m->grow_request = (Lb > Lb0) ? 1u : 0u;
    for (int l = 0; l < kLevelSlots; ++l) {
        m->n[l] = 0;
        m->base[l] = 0;
    }
    uint32_t off = 0;
    for (int l = (int)H; l >= (int)Lb; --l) {
        m->base[l] = off;
        m->n[l] = m->cnt[l];
        off += m->cnt[l] + 1u;
    }
    m->H = H;
    m->Lb = Lb;
    m->index_total = off;
    uint32_t Ls = H + 1;
    for (int l = (int)H; l >= (int)Lb; --l) {
        if (m->base[l] + m->n[l] + 1u <= a.smem_top) Ls = (uint32_t)l;
        else break;
    }
    m->Ls = Ls;
    m->smem_entries = (Ls <= H) ? m->base[Ls] + m->n[Ls] + 1u : 0u;
    // Incremental when the storage layer kept its layout and the old levels are exact:
    // the new levels are the old ones plus the batch's membership changes, written to
    // the other buffer. The per-level change lists must fit their arrays.
    bool inc = !merged && a.force_rebuild == 0 && m->levels_exact && Lb == oLb && oLb <= oH && Lb <= H;
    if (inc) {
        const uint32_t Hm = H > oH ? H : oH;
        uint64_t lists = 0, ge = 0;
        for (int l = kLevelSlots - 1; l >= (int)Lb; --l) {
            ge += bm->chg_hist[l];
            if ((uint32_t)l <= Hm) lists += ge + 1u;
        }
        inc = lists <= a.lst_cap;
    }
    bm->inc = inc ? 1u : 0u;
    if (inc) {
        m->lcur ^= 1u;
        m->inc_rebuilds += 1;
    }
    m->levels_exact = 1;
    __threadfence_block();
    return true;
}

// The body reads and writes the device meta and batch counters word by word on one
// thread; it works on shared-memory copies loaded and stored by the whole warp, so its
// dependent accesses cost shared-memory latency rather than L2 latency.
__global__ void k_level_bases(RebuildArgs a) {
    pdl_wait();
    pdl_trigger();
    __shared__ DevMeta s_m;
    __shared__ BatchMeta s_bm;
    __shared__ int s_go;
    constexpr int kMW = sizeof(DevMeta) / 4, kBW = sizeof(BatchMeta) / 4;
    static_assert(sizeof(DevMeta) % 4 == 0 && sizeof(BatchMeta) % 4 == 0, "word copies");
    constexpr int kErrWord = offsetof(DevMeta, error) / 4;
    uint32_t* sm = reinterpret_cast<uint32_t*>(&s_m);
    uint32_t* sb = reinterpret_cast<uint32_t*>(&s_bm);
    const uint32_t* gm = reinterpret_cast<const uint32_t*>(a.m);
    const uint32_t* gb = reinterpret_cast<const uint32_t*>(a.bm);
    for (int w = threadIdx.x; w < kMW; w += blockDim.x) sm[w] = gm[w];
    for (int w = threadIdx.x; w < kBW; w += blockDim.x) sb[w] = gb[w];
    if (threadIdx.x == 0) s_go = 0;
    __syncthreads();
    if (threadIdx.x == 0) {
        RebuildArgs b = a;
        b.m = &s_m;
        b.bm = &s_bm;
        s_go = level_bases_body(b) ? 1 : 0;
    }
    __syncthreads();
    // write back everything but the error word (errors are raised on the global copy)
    uint32_t* gmw = reinterpret_cast<uint32_t*>(a.m);
    for (int w = threadIdx.x; w < kMW; w += blockDim.x)
        if (w != kErrWord) gmw[w] = sm[w];
    uint32_t* gbw = reinterpret_cast<uint32_t*>(a.bm);
    for (int w = threadIdx.x; w < kBW; w += blockDim.x) gbw[w] = sb[w];  // nothing else runs on it now
    if (!s_go) return;
    // sentinels of the built levels, one lane per level
    const DevMeta& m = s_m;
    const int l = (int)m.Lb + (int)threadIdx.x;
    if (l <= (int)m.H) {
        const uint32_t sidx = m.base[l] + m.n[l];
        (m.lcur ? a.lkeys1 : a.lkeys)[sidx] = kMaxKey;
        (m.lcur ? a.ldown1 : a.ldown)[sidx] = (l > (int)m.Lb) ? m.n[l - 1] : m.size;
    }
}

// ---------------------------------------------------------------------------------
// Index-layer rebuild over tiles of 4096 storage nodes.
//   lcnt[(l - 2) * stride + tile] = live nodes of height >= l in the tile, for every
//   level l >= 2. The apply kernel keeps these counts current (its owners add or
//   remove one node per liveness change), so they are recounted from meta only after
//   the storage layer was re-laid-out (merge), at create, or after a capacity change.
//   scan:  per level, the exclusive prefix of the counts over tiles (one CTA/level)
//          into loff[(l - Lb) * ntiles + tile];
//   write: per tile, keys and meta arrive in shared memory by TMA bulk copy. Warp w
//          owns nodes [512 w, 512 w + 512) of the tile: it counts its nodes per level
//          (one ballot per level per 32 nodes), the warps' counts are prefixed across
//          the tile (one barrier), then the warp sweeps its nodes again and every node
//          of height >= l writes its key and down pointer to level l at the position
//          given by the same ballots.
__global__ void __launch_bounds__(256) k_rebuild_count(RebuildArgs a) {
    pdl_wait();
    pdl_trigger();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const DevMeta* m = a.m;
    if (*(volatile const uint32_t*)&m->error) return;  // no barrier in this kernel
    if (!a.bm->rebuild || !(a.bm->merged || a.force_rebuild)) return;
    const uint32_t size = m->size, cur = m->cur;
    const uint32_t ntiles = (size + kNodes - 1) / kNodes;
    for (uint32_t tile = blockIdx.x * 8u + (uint32_t)warp; tile < ntiles; tile += gridDim.x * 8u) {
    const uint32_t ts = tile * kNodes;
    const uint32_t cnt = min((uint32_t)kNodes, size - ts);
    const uint8_t* SM = a.st.meta[cur] + ts;
    uint32_t c = 0;  // lane i: nodes of height >= 2 + i
    for (uint32_t it = 0; it < kNodes / 512; ++it) {
        const uint32_t off = it * 512u + (uint32_t)lane * 16u;
        const uint4 w = *reinterpret_cast<const uint4*>(SM + off);  // padded past the end
        const uint32_t words[4] = {w.x, w.y, w.z, w.w};
        uint32_t hs[16];
        uint32_t hm = 0;
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const uint32_t mt = (words[k >> 2] >> (8 * (k & 3))) & 0xFFu;
            hs[k] = (off + k < cnt && !(mt & kTomb)) ? (mt & kHeightMask) : 0u;
            hm = max(hm, hs[k]);
        }
        const uint32_t wm = __reduce_max_sync(0xffffffffu, hm);
        for (uint32_t l = 2; l <= wm; ++l) {
            uint32_t loc = 0;
#pragma unroll
            for (int k = 0; k < 16; ++k) loc += hs[k] >= l ? 1u : 0u;
            const uint32_t tot = __reduce_add_sync(0xffffffffu, loc);
            if ((uint32_t)lane == l - 2) c += tot;
        }
    }
    if (lane < 32 && lane + 2 < kLevelSlots) a.lcnt[(size_t)lane * a.lstride + tile] = c;
    }
}

// Per built level, exclusive scan of the tile counts over tiles. Grid: (chunks, levels);
// each CTA scans kScanChunk tiles (4 per thread) and gets the prefix of the chunks
// before it by a warp-wide decoupled look-back (the chain is a few chunks long). The
// level's last chunk checks the total against the level size.
constexpr uint32_t kScanChunk = 4096;

__global__ void __launch_bounds__(1024) k_rebuild_scan(RebuildArgs a, uint32_t epoch) {
    pdl_wait();
    pdl_trigger();
    __shared__ uint32_t s_tmp[33];
    __shared__ uint32_t s_prefix;
    __shared__ int s_ok;
    const DevMeta* m = a.m;
    if (block_sees_error(&m->error)) return;
    if (!a.bm->rebuild || a.bm->inc) return;  // an incremental rebuild needs no tile offsets
    const uint32_t H = m->H, Lb = m->Lb, size = m->size;
    const uint32_t l = Lb + blockIdx.y;
    if (H < Lb || size == 0 || l > H) return;
    const uint32_t ntiles = (size + kNodes - 1) / kNodes;
    const uint32_t nchunks = (ntiles + kScanChunk - 1) / kScanChunk;
    const uint32_t chunk = blockIdx.x;
    if (chunk >= nchunks) return;
    const uint32_t* c = a.lcnt + (size_t)(l - 2) * a.lstride;
    uint32_t* o = a.loff + (size_t)(l - Lb) * ntiles;
    const uint32_t t0 = chunk * kScanChunk + threadIdx.x * 4u;
    uint32_t v[4], sum = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        v[k] = (t0 + k < ntiles) ? c[t0 + k] : 0u;
        sum += v[k];
    }
    uint32_t tot;
    uint32_t run = block_excl_sum<1024>(sum, s_tmp, &tot);
    if (threadIdx.x < 32) {
        bool ok;
        // descriptors: one row of 64 chunks per level (level counts of 2^30 nodes fit)
        const uint32_t ex = lookback_warp<false>(a.desc + (size_t)blockIdx.y * 64, chunk, epoch, tot, a.err, &ok);
        if (threadIdx.x == 0) {
            s_prefix = ex;
            s_ok = ok ? 1 : 0;
        }
    }
    __syncthreads();
    if (!s_ok) return;
    run += s_prefix;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (t0 + k < ntiles) o[t0 + k] = run;
        run += v[k];
    }
    if (chunk == nchunks - 1 && threadIdx.x == 0 && s_prefix + tot != m->n[l])
        atomicOr(a.err, kErrBounds);  // counts disagree with the level size
}

// Byte-wise arithmetic on a meta word holding four nodes (height in bits 0-5, delete
// flag in bit 7). live_heights clears the bytes of delete-flagged nodes; members(h, l)
// leaves bit 7 set in exactly the bytes whose height is >= l: 0x80 + h - l is >= 0x80
// iff h >= l, and never borrows from the next byte because h - l >= -33.
__device__ __forceinline__ uint32_t live_heights(uint32_t metaw) {
    const uint32_t t = (metaw >> 7) & 0x01010101u;  // 1 in the low bit of flagged bytes
    return metaw & ~(t * 0xFFu);
}
__device__ __forceinline__ uint32_t members(uint32_t hw, uint32_t l) {
    return ((hw | 0x80808080u) - l * 0x01010101u) & 0x80808080u;
}

constexpr uint32_t kMetaBytes = kNodes + 16;
constexpr uint32_t kWarpNodes = kNodes / 8;  // 512 nodes per warp

// One tile of 4096 nodes per CTA: the tile's meta arrives in shared memory by TMA bulk
// copy; keys are read from global memory only for the nodes that enter the index layer
// (about a quarter of them at p = 1/4, so key sectors holding none are never read).
// Warp w owns nodes [512 w, 512 w + 512); lane t holds nodes 16t..16t+15 of them.
//  1. per lane, a byte-wise membership test of its nodes for every level gives the
//     warp's count per level (lane i accumulates level Lb + i); the warps' counts are
//     prefixed across the tile (one barrier);
//  2. the lanes' level-Lb members (node indices) are placed in a per-warp list in
//     node order by one warp prefix sum;
//  3. the whole warp emits level Lb from the list, 32 consecutive entries per step
//     (coalesced stores), and compacts the list in place to the members of level
//     Lb + 1, keeping each one's index in level Lb for its down pointer; the next
//     levels repeat step 3 on the shrinking list.
__global__ void __launch_bounds__(kThreads) k_rebuild_write(RebuildArgs a) {
    pdl_wait();
    pdl_trigger();
    extern __shared__ __align__(16) uint8_t s_dyn[];
    uint8_t* s_meta = s_dyn;                                              // kNodes + 16
    uint32_t* s_list = reinterpret_cast<uint32_t*>(s_dyn + kMetaBytes);   // 8 x 512
    __shared__ __align__(8) uint64_t s_bar;
    __shared__ uint32_t s_wcnt[8][32];
    __shared__ uint32_t s_base[kLevelSlots], s_n[kLevelSlots];
    __shared__ int s_ok;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const DevMeta* m = a.m;
    if (a.bm->inc || !a.bm->rebuild) return;  // the incremental path writes the levels instead
    if (block_sees_error(&m->error)) return;
    const uint32_t H = m->H, Lb = m->Lb, size = m->size, cur = m->cur;
    if (H < Lb || size == 0) return;
    uint64_t* LK = m->lcur ? a.lkeys1 : a.lkeys;  // the index layer's buffer in use
    uint32_t* LD = m->lcur ? a.ldown1 : a.ldown;
    const uint32_t ntiles = (size + kNodes - 1) / kNodes;
    if (tid < kLevelSlots) {
        s_base[tid] = m->base[tid];
        s_n[tid] = m->n[tid];
    }
    if (tid == 0) mbar_init(&s_bar, 1);
    // A persistent loop over the tiles: the barrier's phase flips with every tile's copy.
    uint32_t phase = 0;
    for (uint32_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, phase ^= 1u) {
    const uint32_t ts = tile * kNodes;
    const uint32_t cnt = min((uint32_t)kNodes, size - ts);
    __syncthreads();  // the previous tile is done with shared memory
    if (tid == 0) {
        s_ok = 1;
        const uint32_t bm_ = ((cnt + 15u) / 16u) * 16u;
        mbar_arrive_expect_tx(&s_bar, bm_);
        bulk_g2s(s_meta, a.st.meta[cur] + ts, bm_, &s_bar);
    }
    const uint64_t* TK = a.st.keys[cur] + ts;  // this tile's keys
    __syncthreads();
    if (!mbar_wait_bounded(&s_bar, phase, a.err)) s_ok = 0;
    const uint32_t w0 = (uint32_t)warp * kWarpNodes;
    const uint32_t nb = w0 + (uint32_t)lane * 16u;
    uint32_t hw[4];
    {
        const uint4 v = *reinterpret_cast<const uint4*>(s_meta + nb);
        const uint32_t raw[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            uint32_t h = live_heights(raw[k]);
            const uint32_t first = nb + 4u * k;  // nodes past the storage layer's end are absent
            if (first + 4u > cnt) {
                const uint32_t keep = first >= cnt ? 0u : (cnt - first);
                h &= keep ? (0xFFFFFFFFu >> (8u * (4u - keep))) : 0u;
            }
            hw[k] = h;
        }
    }
    // 1. the warp's count per level
    uint32_t mine = 0;  // this lane's member count at level Lb
    {
        uint32_t c = 0;
        for (uint32_t l = Lb; l <= H; ++l) {
            uint32_t nl = 0;
#pragma unroll
            for (int k = 0; k < 4; ++k) nl += __popc(members(hw[k], l));
            if (l == Lb) mine = nl;
            const uint32_t tot = __reduce_add_sync(0xffffffffu, nl);
            if ((uint32_t)lane == l - Lb) c = tot;
            if (tot == 0) break;
        }
        s_wcnt[warp][lane] = c;
    }
    __syncthreads();
    if (!s_ok) {
        if (tid == 0) mbar_wait_bounded(&s_bar, phase, a.err);  // let the copy land
        return;
    }
    uint32_t wbase = 0;  // first position of this warp in level Lb + lane
    if (Lb + (uint32_t)lane <= H) {
        wbase = a.loff[(size_t)lane * ntiles + tile];
        for (int w = 0; w < warp; ++w) wbase += s_wcnt[w][lane];
    }
    // 2. level-Lb members in node order
    uint32_t* list = s_list + warp * kWarpNodes;
    uint32_t incl = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    uint32_t nlist = __shfl_sync(0xffffffffu, incl, 31);
    {
        uint32_t w = incl - mine;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            uint32_t mk = members(hw[k], Lb);
            while (mk) {
                const uint32_t bit = __ffs(mk) - 1;
                list[w++] = nb + 4u * k + (bit >> 3);  // node within the tile
                mk &= mk - 1;
            }
        }
    }
    __syncwarp();
    // 3. emit level after level from the list, compacting it in place
    const uint32_t lt = lanemask_lt();
    uint32_t prev_base = 0;
    for (uint32_t l = Lb; l <= H && nlist > 0; ++l) {
        const uint32_t base = __shfl_sync(0xffffffffu, wbase, (int)(l - Lb));
        uint32_t nnext = 0;
        for (uint32_t j0 = 0; j0 < nlist; j0 += 32u) {
            const uint32_t j = j0 + (uint32_t)lane;
            const bool in = j < nlist;
            const uint32_t e = in ? list[j] : 0u;  // node | index in level l - 1 << 16
            const uint32_t node = e & 0xFFFFu;
            const uint32_t h = in ? (uint32_t)(s_meta[node] & kHeightMask) : 0u;
            const uint32_t up = __ballot_sync(0xffffffffu, in && h > l);
            __syncwarp();  // every lane has read its entry before the list is overwritten
            if (in) {
                const uint32_t p = base + j;
                if (p < s_n[l]) {
                    const uint32_t g = s_base[l] + p;
                    LK[g] = TK[node];
                    LD[g] = (l == Lb) ? ts + node : prev_base + (e >> 16);
                } else {
                    atomicOr(a.err, kErrBounds);
                }
                if (h > l) list[nnext + __popc(up & lt)] = node | (j << 16);
            }
            nnext += __popc(up);
            __syncwarp();
        }
        nlist = nnext;
        prev_base = base;
    }
    }  // tiles
}

// ---------------------------------------------------------------------------------
// Bulk build: keep the last query of every key run of the sorted input (the last
// occurrence of a key wins), with its value and tower height; count level sizes.
__global__ void __launch_bounds__(kThreads) k_create_storage(CreateArgs a, uint32_t epoch) {
    pdl_wait();
    pdl_trigger();
    __shared__ uint32_t s_tmp[33];
    __shared__ uint32_t s_hist[kLevelSlots];
    __shared__ uint32_t s_tile, s_prefix, s_kept;
    __shared__ int s_ok;
    const int tid = threadIdx.x;
    const uint32_t n = a.n;
    const uint32_t ntiles = (n + kNodes - 1) / kNodes;
    if (tid < kLevelSlots) s_hist[tid] = 0;
    if (tid == 0) {
        s_ok = 1;
        s_kept = 0;
    }
    for (;;) {
        __syncthreads();
        if (tid == 0) s_tile = atomicAdd(&a.bm->tile_ctr[kCtrCreate], 1u);
        __syncthreads();
        const uint32_t tile = s_tile;
        if (tile >= ntiles) break;
        const uint32_t b0 = tile * kNodes + tid * kPer;
        uint32_t keep_bits = 0, c = 0;
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            const uint32_t i = b0 + k;
            bool keep = false;
            if (i < n) {
                const uint64_t key = a.sk[i];
                keep = key != kMaxKey && (i + 1 == n || a.sk[i + 1] != key);
            }
            keep_bits |= (keep ? 1u : 0u) << k;
            c += keep ? 1u : 0u;
        }
        uint32_t tot;
        const uint32_t ex = block_excl_sum<kThreads>(c, s_tmp, &tot);
        if (tid < 32) {
            bool ok;
            const uint32_t ex = lookback_warp<false>(a.desc, tile, epoch, tot, a.err, &ok);
            if (tid == 0) {
                s_prefix = ex;
                if (!ok) s_ok = 0;
                s_kept += tot;
            }
        }
        __syncthreads();
        if (!s_ok) break;
        uint32_t o = s_prefix + ex;
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            if (!((keep_bits >> k) & 1u)) continue;
            const uint32_t i = b0 + k;
            const uint64_t key = a.sk[i];
            const uint32_t h = tower_height(key, a.hp);
            if (o >= a.st_cap) {
                atomicOr(a.err, kErrBounds);
                break;
            }
            a.st.keys[0][o] = key;
            a.st.vals[0][o] = a.uvals[a.sp[i] & ((1u << 30) - 1u)];
            a.st.meta[0][o] = (uint8_t)h;
            atomicAdd(&s_hist[h], 1u);
            ++o;
        }
    }
    __syncthreads();
    if (tid == 0 && s_kept) atomicAdd(&a.m->size, s_kept);
    // s_hist[h] = nodes of height exactly h; cnt[l] = nodes of height >= l
    if (tid >= 1 && tid < kLevelSlots) {
        uint32_t c = 0;
        for (int h = tid; h < kLevelSlots; ++h) c += s_hist[h];
        if (c) atomicAdd(&a.m->cnt[tid], c);
    }
}

// Live pairs of the storage layer, in key order.
__global__ void __launch_bounds__(kThreads) k_export_live(Storage st, const DevMeta* m, uint64_t* ko,
                                                          uint64_t* vo, uint64_t cap, uint32_t* count,
                                                          uint64_t* desc, uint32_t* tile_ctr, uint32_t epoch,
                                                          uint32_t* err) {
    pdl_wait();
    pdl_trigger();
    __shared__ uint32_t s_tmp[33];
    __shared__ uint32_t s_tile, s_prefix;
    __shared__ int s_ok;
    const int tid = threadIdx.x;
    const uint32_t size = m->size, cur = m->cur;
    const uint32_t ntiles = (size + kNodes - 1) / kNodes;
    if (tid == 0) s_ok = 1;
    for (;;) {
        __syncthreads();
        if (tid == 0) s_tile = atomicAdd(tile_ctr, 1u);
        __syncthreads();
        const uint32_t tile = s_tile;
        if (tile >= ntiles) break;
        const uint32_t b0 = tile * kNodes + tid * kPer;
        uint32_t bits = 0, c = 0;
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            const uint32_t i = b0 + k;
            const bool lv = i < size && !(st.meta[cur][i] & kTomb);
            bits |= (lv ? 1u : 0u) << k;
            c += lv ? 1u : 0u;
        }
        uint32_t tot;
        const uint32_t ex = block_excl_sum<kThreads>(c, s_tmp, &tot);
        if (tid < 32) {
            bool ok;
            const uint32_t ex = lookback_warp<false>(desc, tile, epoch, tot, err, &ok);
            if (tid == 0) {
                s_prefix = ex;
                if (!ok) s_ok = 0;
                if (tile == ntiles - 1) *count = ex + tot;
            }
        }
        __syncthreads();
        if (!s_ok) break;
        uint64_t o = (uint64_t)s_prefix + ex;
        for (int k = 0; k < kPer; ++k) {
            if (!((bits >> k) & 1u)) continue;
            if (o < cap) {
                ko[o] = st.keys[cur][b0 + k];
                vo[o] = st.vals[cur][b0 + k];
            }
            ++o;
        }
    }
}

// Failure-path self-test: tile 1 waits for tile 0, which never publishes, so the
// bounded look-back must give up, record kErrTimeout and return.
__global__ void k_wait_selftest(uint64_t* desc, uint32_t* err) {
    bool ok = true;
    lookback_warp<false>(desc, 1u, 1u, 0u, err, &ok);
}

}  // namespace

cudaError_t launch_merge(const RebuildArgs& a, uint32_t& epoch, cudaStream_t s, int num_sms) {
    (void)epoch;  // the merge has no look-back
    const uint32_t tiles = a.size_ub / kNodes + 1;
    const uint32_t ccap = (uint32_t)num_sms * 8u, cap = (uint32_t)num_sms * 5u;  // the CTAs resident at once
    launch_dep(k_merge_count, tiles < ccap ? tiles : ccap, kThreads, 0, s, a);
    ++g_launches;
    launch_dep(k_merge, tiles < cap ? tiles : cap, kThreads, 0, s, a);
    ++g_launches;
    return cudaGetLastError();
}

cudaError_t launch_level_bases(const RebuildArgs& a, cudaStream_t s) {
    launch_dep(k_level_bases, 1, 32, 0, s, a);
    ++g_launches;
    return cudaGetLastError();
}

cudaError_t launch_rebuild_prep(const RebuildArgs& a, uint32_t& epoch, cudaStream_t s, int num_sms) {
    const uint32_t tiles = (a.size_ub + kNodes - 1) / kNodes + 1;
    const uint32_t cb = (tiles + 7) / 8, ccap = (uint32_t)num_sms * 4u;
    launch_dep(k_rebuild_count, cb < ccap ? cb : ccap, 256, 0, s, a);  // exits at once unless recounting
    ++g_launches;
    const uint32_t chunks = (tiles + kScanChunk - 1) / kScanChunk;
    launch_dep(k_rebuild_scan, dim3(chunks, kLevelSlots - 2), 1024, 0, s, a, ++epoch);
    ++g_launches;
    return cudaGetLastError();
}

cudaError_t launch_rebuild_write(const RebuildArgs& a, cudaStream_t s, int num_sms) {
    static bool attr_set = false;
    const int dyn = (int)(kMetaBytes + 8 * kWarpNodes * 4);
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_rebuild_write, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    const uint32_t tiles = (a.size_ub + kNodes - 1) / kNodes + 1;
    const uint32_t cap = (uint32_t)num_sms * 8u;  // persistent: the CTAs resident at once
    launch_dep(k_rebuild_write, tiles < cap ? tiles : cap, kThreads, dyn, s, a);
    ++g_launches;
    return cudaGetLastError();
}

cudaError_t launch_rebuild(const RebuildArgs& a, uint32_t& epoch, cudaStream_t s, int num_sms) {
    cudaError_t e = launch_rebuild_prep(a, epoch, s, num_sms);
    return e != cudaSuccess ? e : launch_rebuild_write(a, s, num_sms);
}

cudaError_t launch_create_storage(const CreateArgs& a, uint32_t& epoch, cudaStream_t s, int num_sms) {
    if (a.n == 0) return cudaSuccess;
    const uint32_t tiles = (a.n + kNodes - 1) / kNodes;
    const uint32_t cap = (uint32_t)num_sms * 4u;
    launch_dep(k_create_storage, (int)(tiles < cap ? tiles : cap), kThreads, 0, s, a, ++epoch);
    ++g_launches;
    return cudaGetLastError();
}

cudaError_t launch_export_live(const Storage& st, const DevMeta* m, uint64_t* keys_out, uint64_t* vals_out,
                               uint64_t cap, uint32_t* count, uint64_t* desc, uint32_t* tile_ctr,
                               uint32_t& epoch, uint32_t* err, cudaStream_t s, int num_sms, uint32_t size_ub) {
    const uint32_t tiles = size_ub / kNodes + 1;
    const uint32_t c = (uint32_t)num_sms * 4u;
    launch_dep(k_export_live, (int)(tiles < c ? tiles : c), kThreads, 0, s, st, m, keys_out, vals_out, cap, count, desc,
                                                                   tile_ctr, ++epoch, err);
    ++g_launches;
    return cudaGetLastError();
}

cudaError_t launch_wait_selftest(uint64_t* desc, uint32_t* err, cudaStream_t s) {
    k_wait_selftest<<<1, 32, 0, s>>>(desc, err);
    ++g_launches;
    return cudaGetLastError();
}

}  // namespace pi
