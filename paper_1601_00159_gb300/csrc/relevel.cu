// Incremental index-layer rebuild. When a batch leaves the storage layer's layout alone
// (no new node, no re-layout), the new index levels are the old ones minus the keys that
// were deleted and plus the keys that were revived, among the nodes of height >= the
// lowest built level; every other key keeps its storage position. The rebuild then reads
// the old levels (the buffer not in use after the layout step flipped DevMeta::lcur) and
// writes the new ones, instead of scanning the storage layer and gathering member keys:
//   k_relevel_lists   one CTA per level l: the batch's changes of height >= l, in key
//                     order, with the running count (inserts - deletes) before each;
//   k_relevel_write   every old entry moves by the running count of its level's list
//                     before its key (or goes, if deleted); its down pointer into level
//                     l - 1 moves by that level's running count; every insert lands at
//                     (old entries below its key) + (running count before it).
// The result equals a rebuild from the storage layer (Section 4.1): each level holds the
// live keys of height >= l in key order, with the position of the same key one level
// down (or in the storage layer, at the lowest built level).

#include "common.cuh"

namespace pi {
namespace {

constexpr int kT = 256;
constexpr uint32_t kItems = 8;
constexpr uint32_t kTile = kT * kItems;  // old entries per tile
constexpr uint32_t kSlice = 512;         // list entries staged in shared memory per tile and level

__device__ __forceinline__ uint32_t ge_count(const BatchMeta* bm, uint32_t l) {
    uint32_t c = 0;
    for (uint32_t h = l; h < (uint32_t)kLevelSlots; ++h) c += bm->chg_hist[h];
    return c;
}

// Three independent lower bounds advanced in lockstep, so their dependent loads overlap
// (an insert needs its place in two old levels and in the change list below).
__device__ __forceinline__ void lb3(const uint64_t* K0, uint32_t n0, const uint64_t* K1, uint32_t n1,
                                    const uint64_t* K2, uint32_t n2, uint64_t x, uint32_t& r0, uint32_t& r1,
                                    uint32_t& r2) {
    uint32_t lo0 = 0, hi0 = n0, lo1 = 0, hi1 = n1, lo2 = 0, hi2 = n2;
    while (lo0 < hi0 || lo1 < hi1 || lo2 < hi2) {
        const uint32_t m0 = (lo0 + hi0) >> 1, m1 = (lo1 + hi1) >> 1, m2 = (lo2 + hi2) >> 1;
        const bool a0 = lo0 < hi0, a1 = lo1 < hi1, a2 = lo2 < hi2;
        const uint64_t v0 = a0 ? K0[m0] : 0ull, v1 = a1 ? K1[m1] : 0ull, v2 = a2 ? K2[m2] : 0ull;
        if (a0) { if (v0 < x) lo0 = m0 + 1; else hi0 = m0; }
        if (a1) { if (v1 < x) lo1 = m1 + 1; else hi1 = m1; }
        if (a2) { if (v2 < x) lo2 = m2 + 1; else hi2 = m2; }
    }
    r0 = lo0;
    r1 = lo1;
    r2 = lo2;
}

// First index of K[0, n) (sorted) whose key is >= x.
__device__ __forceinline__ uint32_t lb_keys(const uint64_t* K, uint32_t n, uint64_t x) {
    uint32_t lo = 0, hi = n;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (K[mid] < x) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

__global__ void __launch_bounds__(1024) k_relevel_lists(RebuildArgs a) {
    pdl_wait();
    pdl_trigger();
    __shared__ uint32_t s_tmp[33];
    __shared__ uint32_t s_off;
    const DevMeta* m = a.m;
    BatchMeta* bm = a.bm;
    if (block_sees_error(&m->error)) return;
    if (!bm->inc) return;
    const uint32_t Lb = m->Lb, Hm = m->H > bm->old_H ? m->H : bm->old_H;
    const uint32_t l = Lb + blockIdx.x;
    if (l > Hm) return;
    if (threadIdx.x == 0) {
        uint32_t off = 0;
        for (uint32_t k = Lb; k < l; ++k) off += ge_count(bm, k) + 1u;
        s_off = off;
        bm->lst_off[l] = off;
    }
    __syncthreads();
    const uint32_t off = s_off, nchg = bm->nchg;
    constexpr uint32_t kPer = 8;  // consecutive changes per thread
    uint32_t carry = 0, icarry = 0;
    for (uint32_t c0 = 0; c0 < nchg; c0 += 1024u * kPer) {
        const uint32_t i0 = c0 + threadIdx.x * kPer;
        uint32_t sm = 0, im = 0;
#pragma unroll
        for (uint32_t k = 0; k < kPer; ++k) {
            const uint32_t i = i0 + k;
            const uint8_t hl = i < nchg ? a.chg.hl[i] : (uint8_t)0;
            if (i < nchg && (uint32_t)(hl & kHeightMask) >= l) {
                sm |= 1u << k;
                if (hl & 0x80u) im |= 1u << k;
            }
        }
        uint32_t tot, itot;
        uint32_t j = carry + block_excl_sum<1024>((uint32_t)__popc(sm), s_tmp, &tot);
        uint32_t ib = icarry + block_excl_sum<1024>((uint32_t)__popc(im), s_tmp, &itot);
#pragma unroll
        for (uint32_t k = 0; k < kPer; ++k) {
            if (!((sm >> k) & 1u)) continue;
            const uint32_t i = i0 + k;
            const bool ins = (im >> k) & 1u;
            if (off + j < a.lst_cap) {
                a.lst_keys[off + j] = a.chg.keys[i];
                a.lst_pos[off + j] = a.chg.pos[i];
                a.lst_ins[off + j] = ins ? 1u : 0u;
                a.lst_pref[off + j] = (int32_t)(2u * ib) - (int32_t)j;  // inserts - deletes before it
            } else {
                atomicOr(a.err, kErrBounds);
            }
            ++j;
            ib += ins ? 1u : 0u;
        }
        carry += tot;
        icarry += itot;
    }
    if (threadIdx.x == 0) {
        bm->lst_n[l] = carry;
        if (off + carry < a.lst_cap) a.lst_pref[off + carry] = (int32_t)(2u * icarry) - (int32_t)carry;
        else atomicOr(a.err, kErrBounds);
        if (carry != ge_count(bm, l)) atomicOr(a.err, kErrBounds);
    }
}

// First index of K[0, n) (sorted) whose key is >= x, found by the whole CTA: each round
// probes kT evenly spaced entries and keeps the gap where the predicate flips, so a list
// of up to kT^k entries takes k rounds of one load per thread.
__device__ uint32_t coop_lower_bound(const uint64_t* K, uint32_t n, uint64_t x) {
    uint32_t lo = 0, hi = n;  // answer in [lo, hi]
    while (hi > lo) {
        const uint32_t len = hi - lo;
        const uint32_t step = (len + kT - 1) / kT;
        const uint32_t p = lo + (uint32_t)threadIdx.x * step;
        const bool below = p < hi && K[p] < x;
        const uint32_t c = (uint32_t)__syncthreads_count(below);  // probes below x: a prefix
        if (step == 1) return lo + c;
        // the answer lies in (lo + (c - 1) * step, lo + c * step]
        const uint32_t nlo = c ? lo + (c - 1) * step + 1 : lo;
        const uint32_t nhi = lo + c * step < hi ? lo + c * step : hi;
        lo = nlo;
        hi = nhi;
    }
    return lo;
}

// Stages the entries of one level's list whose keys lie in [kmin, kmax] (and the running
// count after them); returns false when there are more than kSlice.
__device__ bool stage_slice(const RebuildArgs& a, uint32_t off, uint32_t n, uint64_t kmin, uint64_t kmax,
                            uint64_t* sk, int32_t* sp, uint32_t* s_j0, uint32_t* s_len) {
    const uint32_t lo = coop_lower_bound(a.lst_keys + off, n, kmin);
    const uint32_t hi = kmax == kMaxKey ? n : coop_lower_bound(a.lst_keys + off, n, kmax + 1u);
    const uint32_t len = hi - lo;
    if (threadIdx.x == 0) {
        *s_j0 = lo;
        *s_len = len;
    }
    if (len > kSlice) return false;
    for (uint32_t x = threadIdx.x; x < len; x += kT) {
        sk[x] = a.lst_keys[off + lo + x];
        sp[x] = a.lst_pref[off + lo + x];
    }
    if (threadIdx.x == 0) sp[len] = a.lst_pref[off + lo + len];
    return true;
}

// Entries of the staged slice below x.
__device__ __forceinline__ uint32_t slice_rank(const uint64_t* sk, uint32_t len, uint64_t x) {
    uint32_t lo = 0, hi = len;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (sk[mid] < x) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

__global__ void __launch_bounds__(kT, 4) k_relevel_write(RebuildArgs a) {
    pdl_wait();
    pdl_trigger();
    __shared__ uint32_t s_apref[kLevelSlots + 1], s_bpref[kLevelSlots + 1];
    __shared__ uint32_t s_ta, s_tb;
    __shared__ uint64_t s_k0[kSlice], s_k1[kSlice];
    __shared__ int32_t s_p0[kSlice + 1], s_p1[kSlice + 1];
    __shared__ uint32_t s_j0, s_len0, s_j1, s_len1;
    const DevMeta* m = a.m;
    const BatchMeta* bm = a.bm;
    if (block_sees_error(&m->error)) return;
    if (!bm->inc) return;
    const uint32_t Lb = m->Lb, H = m->H, oH = bm->old_H, Hm = H > oH ? H : oH;
    const uint64_t* OK = m->lcur ? a.lkeys : a.lkeys1;  // the previous buffer
    const uint32_t* OD = m->lcur ? a.ldown : a.ldown1;
    uint64_t* NK = m->lcur ? a.lkeys1 : a.lkeys;
    uint32_t* ND = m->lcur ? a.ldown1 : a.ldown;
    const int tid = threadIdx.x;
    if (tid == 0) {
        uint32_t t = 0;
        for (uint32_t l = Lb; l <= Hm + 1u && l <= (uint32_t)kLevelSlots; ++l) {
            s_bpref[l] = t;
            if (l <= Hm) t += (bm->lst_n[l] + kT - 1u) / kT;
        }
        s_tb = t;
        t = 0;
        for (uint32_t l = Lb; l <= Hm + 1u && l <= (uint32_t)kLevelSlots; ++l) {
            s_apref[l] = t;
            if (l <= oH) t += (bm->old_n[l] + kTile - 1u) / kTile;
        }
        s_ta = t;
    }
    __syncthreads();
    const uint32_t TA = s_ta, TB = s_tb;
    // The inserts come first: their searches are long chains of dependent loads, which
    // then overlap with the streaming of the old entries on the other CTAs.
    for (uint32_t t = blockIdx.x; t < TA + TB; t += gridDim.x) {
        if (t < TB) {
            uint32_t l = Lb;
            while (l < Hm && s_bpref[l + 1] <= t) ++l;
            const uint32_t c = (t - s_bpref[l]) * kT + (uint32_t)tid;
            const uint32_t off0 = bm->lst_off[l];
            if (c < bm->lst_n[l] && a.lst_ins[off0 + c]) {
                const uint64_t key = a.lst_keys[off0 + c];
                // its place among the old entries of level l, and (above the lowest level)
                // its place in level l - 1: old entries below it plus that list's running count
                const uint32_t off1 = l > Lb ? bm->lst_off[l - 1] : 0u;
                uint32_t lbo, j1, lbo1;
                lb3(OK + bm->old_base[l], l <= oH ? bm->old_n[l] : 0u, a.lst_keys + off1, l > Lb ? bm->lst_n[l - 1] : 0u,
                    OK + (l > Lb ? bm->old_base[l - 1] : 0u), (l > Lb && l - 1u <= oH) ? bm->old_n[l - 1] : 0u, key,
                    lbo, j1, lbo1);
                const uint32_t out = lbo + (uint32_t)a.lst_pref[off0 + c];
                const uint32_t nd = l == Lb ? a.lst_pos[off0 + c] : lbo1 + (uint32_t)a.lst_pref[off1 + j1];
                if (l <= H && out < m->n[l]) {
                    NK[m->base[l] + out] = key;
                    ND[m->base[l] + out] = nd;
                } else {
                    atomicOr(a.err, kErrBounds);
                }
            }
            continue;
        }
        // a tile of old entries of level l (warp-contiguous: entry i0 + k * kT + tid)
        const uint32_t ta = t - TB;
        uint32_t l = Lb;
        while (l < oH && s_apref[l + 1] <= ta) ++l;
        const uint32_t i0 = (ta - s_apref[l]) * kTile;
        const uint32_t on = bm->old_n[l];
        const uint32_t i1 = i0 + kTile < on ? i0 + kTile : on;
        const uint32_t ob = bm->old_base[l];
        const uint64_t kmin = OK[ob + i0], kmax = OK[ob + i1 - 1u];
        const uint32_t off0 = bm->lst_off[l], n0 = bm->lst_n[l];
        const bool st0 = stage_slice(a, off0, n0, kmin, kmax, s_k0, s_p0, &s_j0, &s_len0);
        bool st1 = true;
        uint32_t off1 = 0, n1 = 0;
        if (l > Lb) {
            off1 = bm->lst_off[l - 1];
            n1 = bm->lst_n[l - 1];
            st1 = stage_slice(a, off1, n1, kmin, kmax, s_k1, s_p1, &s_j1, &s_len1);
        }
        __syncthreads();
        const uint32_t nb = m->base[l], nl = m->n[l];
        uint64_t tk[kItems];
        uint32_t td[kItems];
#pragma unroll
        for (uint32_t k = 0; k < kItems; ++k) {  // every load of the tile in flight at once
            const uint32_t i = i0 + k * kT + (uint32_t)tid;
            tk[k] = i < i1 ? OK[ob + i] : 0ull;
            td[k] = i < i1 ? OD[ob + i] : 0u;
        }
#pragma unroll
        for (uint32_t k = 0; k < kItems; ++k) {
            const uint32_t i = i0 + k * kT + (uint32_t)tid;
            if (i >= i1) break;
            const uint64_t key = tk[k];
            uint32_t nd = td[k];
            bool hit;
            int32_t shift;
            if (st0) {
                const uint32_t x = slice_rank(s_k0, s_len0, key);
                hit = x < s_len0 && s_k0[x] == key;
                shift = s_p0[x];
            } else {
                const uint32_t j = lb_keys(a.lst_keys + off0, n0, key);
                hit = j < n0 && a.lst_keys[off0 + j] == key;
                shift = a.lst_pref[off0 + j];
            }
            if (hit) continue;  // the key was deleted (an existing entry is never an insert)
            const uint32_t out = i + (uint32_t)shift;
            if (l > Lb) {
                const int32_t s1 = st1 ? s_p1[slice_rank(s_k1, s_len1, key)]
                                       : a.lst_pref[off1 + lb_keys(a.lst_keys + off1, n1, key)];
                nd += (uint32_t)s1;
            }
            if (l <= H && out < nl) {
                NK[nb + out] = key;
                ND[nb + out] = nd;
            } else {
                atomicOr(a.err, kErrBounds);
            }
        }
        __syncthreads();
    }
}

}  // namespace

cudaError_t launch_relevel(const RebuildArgs& a, cudaStream_t s, int num_sms) {
    launch_dep(k_relevel_lists, kLevelSlots, 1024, 0, s, a);
    ++g_launches;
    launch_dep(k_relevel_write, (uint32_t)num_sms * 4u, kT, 0, s, a);  // the CTAs resident at once
    ++g_launches;
    return cudaGetLastError();
}

}  // namespace pi
