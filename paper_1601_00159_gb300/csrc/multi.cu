// Batching form: many independent indices, each with its own query batch, in one
// persistent launch (Algorithm 1 applied to every index of a set at once).
//
// Small indices and small batches leave the level-synchronous whole-GPU pipeline of a
// single index (tens of launches, each spread over all SMs) launch-bound. Here a CTA
// runs the whole pipeline of one index's batch by itself, and the CTAs of a persistent
// launch take batches from a device-side work queue, largest first:
//   sort        stable LSD radix sort of (key, arrival) over the varying key bytes,
//               chunks of kT x kMI queries ranked by warp ballots (kBits-bit digits);
//   distinct    the run heads of the sorted batch, compacted;
//   descent     each thread walks kMK distinct keys down the index together (one
//               independent gather per key per step); the top levels are staged in
//               shared memory and resolved by a binary search of the lowest staged one;
//   locate      the storage node with the largest key <= q;
//   apply       one chunked pass with running carries: a max-scan of write markers
//               gives every query the state of its key just before it (arrival order),
//               the last query of each key run owns the node and writes the final state;
//               keys that are new become a sorted list of new nodes;
//   merge       live old nodes and new nodes into the other storage buffer, by the
//               insertion points the descent found;
//   rebuild     the lowest built level from the storage layer, each higher level from
//               the one below it (heights recomputed from the seeded key hash).
// All state lives in the indices' own device arrays and DevMeta blocks, so the single-
// index entry points (export, info, the plain batch path) see the same index after it.
// The queue is filled before the launch, so taking an item is one atomicAdd and no CTA
// ever waits on another.

#include "common.cuh"

namespace pi {
namespace {

constexpr uint32_t kMSeqMask = (1u << 30) - 1u;
constexpr int kMI = 8;             // queries or nodes per thread in a chunked pass
constexpr int kMK = 8;             // distinct keys per thread walked down together
constexpr uint32_t kMTop = 2048;   // index entries staged in shared memory
constexpr uint32_t kMSeg = 256;    // colliding segments one CTA orders after the prefix passes

__device__ __forceinline__ void mstore_result(pi_result_t* res, uint32_t seq, uint64_t v, uint32_t st) {
    uint4 w;
    w.x = (uint32_t)v;
    w.y = (uint32_t)(v >> 32);
    w.z = st;
    w.w = 0u;
    *reinterpret_cast<uint4*>(res + seq) = w;
}

struct MShared {
    uint32_t tmp[33];
    uint64_t tmp64[33];
    uint32_t bmax[8], bnmin[8];
    uint32_t invalid;
    uint32_t item;
    uint32_t D, newc, dirty, changes, j1;
    uint32_t nseg, overflow;
    uint32_t seg[kMSeg];  // starts of segments the prefix fix-up orders
    int32_t tomb_delta;
    int32_t delta[kLevelSlots];
    SortPlan plan;
    DevMeta m;
};

struct MScratchPtrs {
    uint64_t *ka, *kb;
    uint32_t *pa, *pb;
    uint64_t* dq;   // distinct keys
    uint32_t* dr;   // storage position + 1 of the largest key <= q
    uint8_t* df;    // bit 0: exists, bit 1: live
    uint64_t* dv;   // value when live
    uint64_t *nk, *nv;
    uint8_t* nh;
    uint32_t* ni;   // insertion point (old node the new node precedes)
};

__device__ __forceinline__ uint64_t al256(uint64_t b) { return (b + 255u) & ~255ull; }

__device__ MScratchPtrs carve(uint8_t* base, uint32_t q) {
    MScratchPtrs p;
    uint64_t off = 0;
    const uint64_t c = (uint64_t)q + kPad;
    auto take = [&](uint64_t bytes) {
        uint8_t* r = base + off;
        off += al256(bytes);
        return r;
    };
    p.ka = reinterpret_cast<uint64_t*>(take(c * 8));
    p.kb = reinterpret_cast<uint64_t*>(take(c * 8));
    p.pa = reinterpret_cast<uint32_t*>(take(c * 4));
    p.pb = reinterpret_cast<uint32_t*>(take(c * 4));
    p.dq = reinterpret_cast<uint64_t*>(take(c * 8));
    p.dr = reinterpret_cast<uint32_t*>(take(c * 4));
    p.df = take(c);
    p.dv = reinterpret_cast<uint64_t*>(take(c * 8));
    p.nk = reinterpret_cast<uint64_t*>(take(c * 8));
    p.nv = reinterpret_cast<uint64_t*>(take(c * 8));
    p.nh = take(c);
    p.ni = reinterpret_cast<uint32_t*>(take(c * 4));
    return p;
}

// In-place exclusive scan of cnt[0, kR) by kT threads.
template <int kT, int kR>
__device__ __forceinline__ void small_excl_scan(uint32_t* cnt, uint32_t* tmp) {
    constexpr int per = (kR + kT - 1) / kT;
    uint32_t v[per];
    uint32_t sum = 0;
#pragma unroll
    for (int k = 0; k < per; ++k) {
        const int d = threadIdx.x * per + k;
        v[k] = d < kR ? cnt[d] : 0u;
        sum += v[k];
    }
    uint32_t run = block_excl_sum<kT>(sum, tmp, nullptr);
#pragma unroll
    for (int k = 0; k < per; ++k) {
        const int d = threadIdx.x * per + k;
        if (d < kR) cnt[d] = run;
        run += v[k];
    }
    __syncthreads();
}

// TMA bulk prefetch of [p, p + bytes) into L2 (p 16-byte aligned, bytes a multiple of 16).
__device__ __forceinline__ void l2_prefetch(const void* p, uint32_t bytes) {
    if (bytes) asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// Block-wide exclusive sum of 64-bit values over kT threads; total in *total.
template <int kT>
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
        const uint64_t w = lane < kT / 32 ? tmp[lane] : 0ull;
        uint64_t t = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint64_t y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < kT / 32) tmp[lane] = t - w;
        if (lane == kT / 32 - 1) tmp[32] = t;
    }
    __syncthreads();
    const uint64_t r = tmp[warp] + x - v;
    if (total) *total = tmp[32];
    __syncthreads();
    return r;
}

// Entries of the sorted a[0, n) below x, by a whole warp: each round probes 32 evenly
// spaced entries of the remaining interval, about log32(n) rounds of one load per lane.
__device__ __forceinline__ uint32_t warp_count_below(const uint32_t* a, uint32_t n, uint32_t x) {
    const uint32_t lane = threadIdx.x & 31u;
    uint32_t lo = 0, hi = n;  // the count lies in [lo, hi]
    while (hi - lo > 32u) {
        const uint32_t step = (hi - lo + 31u) / 32u;
        const uint32_t p = lo + lane * step;
        const uint32_t c = (uint32_t)__popc(__ballot_sync(0xffffffffu, p < hi && a[p] < x));
        if (c == 0) return lo;
        const uint32_t pc = lo + c * step;
        hi = (c < 32u && pc < hi) ? pc : hi;
        lo = lo + (c - 1u) * step + 1u;
    }
    const uint32_t p = lo + lane;
    return lo + (uint32_t)__popc(__ballot_sync(0xffffffffu, p < hi && a[p] < x));
}

// Largest index i in [lo - 1, ...) with K[i] <= q for up to kMK keys at once; K holds a
// sentinel 2^64-1 at or before index lim and is readable 3 entries past it. A key with
// K[lo] <= q unknown (lo = 0) may get -1. Each round loads four entries per active key,
// so the keys' loads are independent and in flight together.
__device__ __forceinline__ void multi_scan(const uint64_t* K, const uint64_t (&q)[kMK], uint32_t (&pos)[kMK],
                                           int32_t (&r)[kMK], uint32_t act, uint32_t lim, uint32_t* err) {
    uint32_t todo = act;
    while (todo) {
#pragma unroll
        for (int k = 0; k < kMK; ++k) {
            if (!((todo >> k) & 1u)) continue;
            const uint32_t i = pos[k];
            if (i > lim) {
                atomicOr(err, kErrBounds);
                r[k] = -1;
                todo &= ~(1u << k);
                continue;
            }
            const uint64_t k0 = K[i], k1 = K[i + 1], k2 = K[i + 2], k3 = K[i + 3];
            // leading entries <= q (entries past the sentinel belong to other arrays)
            const uint32_t c0 = k0 <= q[k], c1 = c0 & (k1 <= q[k]), c2 = c1 & (k2 <= q[k]), c3 = c2 & (k3 <= q[k]);
            const uint32_t c = c0 + c1 + c2 + c3;
            if (c < 4u) {
                r[k] = (int32_t)(i + c) - 1;
                todo &= ~(1u << k);
            } else {
                pos[k] = i + 4u;
            }
        }
    }
}

// One stable LSD pass over [lo, hi) of (src_k, src_p) by the kBits-bit digit at `shift`,
// into the same range of (dst_k, dst_p): a histogram, its exclusive scan, then chunks of
// kT x kMI elements ranked by warp ballots (elements in index order within a chunk).
template <int kT, int kBits>
__device__ void m_lsd_pass(const uint64_t* src_k, const uint32_t* src_p, uint64_t* dst_k, uint32_t* dst_p,
                           uint32_t lo, uint32_t hi, uint32_t shift, uint8_t* dsm, uint32_t* tmp, uint32_t* err) {
    constexpr int kW = kT / 32;
    constexpr int kR = 1 << kBits;
    constexpr uint32_t kC = (uint32_t)kT * kMI;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint32_t* whist = reinterpret_cast<uint32_t*>(dsm);  // [kW][kR]
    uint32_t* sbase = whist + kW * kR;                   // [kR]
    uint32_t* stot = sbase + kR;                         // [kR]
    for (int d = tid; d < kW * kR; d += kT) whist[d] = 0;
    for (int d = tid; d < kR; d += kT) sbase[d] = 0;
    __syncthreads();
    for (uint32_t i = lo + tid; i < hi; i += kT) atomicAdd(&sbase[(uint32_t)(src_k[i] >> shift) & (kR - 1)], 1u);
    __syncthreads();
    small_excl_scan<kT, kR>(sbase, tmp);
    for (uint32_t c0 = lo; c0 < hi; c0 += kC) {
        uint64_t key[kMI];
        uint32_t pay[kMI], dig[kMI], rank[kMI];
#pragma unroll
        for (int k = 0; k < kMI; ++k) {
            const uint32_t i = c0 + (uint32_t)warp * 32u * kMI + (uint32_t)k * 32u + (uint32_t)lane;
            const bool v = i < hi;
            key[k] = v ? src_k[i] : 0ull;
            pay[k] = v ? src_p[i] : 0u;
            dig[k] = v ? (uint32_t)(key[k] >> shift) & (kR - 1) : (uint32_t)kR;
        }
        warp_digit_ranks<kMI, kBits>(dig, rank, whist + warp * kR);
        __syncthreads();
        for (int d = tid; d < kR; d += kT) {
            uint32_t total = 0;
#pragma unroll 4
            for (int w = 0; w < kW; ++w) {
                const uint32_t cc = whist[w * kR + d];
                whist[w * kR + d] = total;
                total += cc;
            }
            stot[d] = total;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kMI; ++k) {
            const uint32_t d = dig[k];
            if (d < (uint32_t)kR) {
                const uint32_t pos = lo + sbase[d] + whist[warp * kR + d] + rank[k];
                if (pos < hi) {
                    dst_k[pos] = key[k];
                    dst_p[pos] = pay[k];
                } else {
                    atomicOr(err, kErrBounds);
                }
            }
        }
        __syncthreads();
        for (int d = tid; d < kR; d += kT) {
            sbase[d] += stot[d];
#pragma unroll 4
            for (int w = 0; w < kW; ++w) whist[w * kR + d] = 0;
        }
        __syncthreads();
    }
}

template <int kT, int kBits>
__device__ void m_item(const MultiArgs& a, const MItem& it, const MScratchPtrs& s, uint8_t* dsm, MShared& sh) {
    constexpr uint32_t kC = (uint32_t)kT * kMI;
    const int tid = threadIdx.x, lane = tid & 31;
    const MIndex& X = a.idx[it.index];
    const uint32_t n = it.n;
    uint32_t* err = &X.m->error;

    if (tid == 0) {
        sh.m = *X.m;
        sh.invalid = 0;
        sh.newc = 0;
        sh.dirty = 0;
        sh.changes = 0;
        sh.tomb_delta = 0;
    }
    if (tid < 8) {
        sh.bmax[tid] = 0;
        sh.bnmin[tid] = 0;
    }
    if (tid < kLevelSlots) sh.delta[tid] = 0;
    __syncthreads();
    if (sh.m.error || n == 0) return;
    const uint32_t cur = sh.m.cur;
    uint64_t* SK = X.st.keys[cur];
    uint64_t* SV = X.st.vals[cur];
    uint8_t* SM = X.st.meta[cur];
    uint64_t* LK = sh.m.lcur ? X.lkeys1 : X.lkeys;  // the index layer's buffer in use
    uint32_t* LD = sh.m.lcur ? X.ldown1 : X.ldown;

    // ---- pack + sort. Four passes on the most significant varying bytes, then the
    // segments of equal leading bytes that hold different keys are ordered by the rest
    // (as in the single-index sort). With more such segments than the list holds, the
    // batch is packed again and sorted with every pass.
    uint64_t* K = s.ka;
    uint32_t* P = s.pa;
    for (uint32_t budget = 4; budget <= 8; budget += 4) {
        if (tid < 8) {
            sh.bmax[tid] = 0;
            sh.bnmin[tid] = 0;
        }
        if (tid == 0) {
            sh.invalid = 0;
            sh.nseg = 0;
            sh.overflow = 0;
        }
        __syncthreads();
        {
            uint32_t mx[8], mn[8], inv = 0;
#pragma unroll
            for (int d = 0; d < 8; ++d) mx[d] = mn[d] = 0;
            for (uint32_t i = tid; i < n; i += kT) {
                const uint32_t op = it.ops[i];
                const uint64_t k = it.keys[i];
                const bool valid = op <= 2u && k != kMaxKey;
                s.ka[i] = valid ? k : kMaxKey;
                s.pa[i] = ((op & 3u) << 30) | i;
                inv += valid ? 0u : 1u;
                if (valid) {
#pragma unroll
                    for (int d = 0; d < 8; ++d) {
                        const uint32_t b = (uint32_t)(k >> (8 * d)) & 255u;
                        mx[d] = max(mx[d], b);
                        mn[d] = max(mn[d], 255u - b);
                    }
                }
            }
#pragma unroll
            for (int d = 0; d < 8; ++d) {
                mx[d] = __reduce_max_sync(0xffffffffu, mx[d]);
                mn[d] = __reduce_max_sync(0xffffffffu, mn[d]);
            }
            inv = __reduce_add_sync(0xffffffffu, inv);
            if (lane == 0) {
                if (inv) atomicAdd(&sh.invalid, inv);
#pragma unroll
                for (int d = 0; d < 8; ++d) {
                    atomicMax(&sh.bmax[d], mx[d]);
                    atomicMax(&sh.bnmin[d], mn[d]);
                }
            }
            __syncthreads();
            if (tid == 0) plan_digits(sh.bmax, sh.bnmin, sh.invalid, n, budget, sh.plan);
            __syncthreads();
        }
        K = s.ka;
        P = s.pa;
        uint64_t* K2 = s.kb;
        uint32_t* P2 = s.pb;
        for (uint32_t j = 0; j < sh.plan.npass; ++j)
            for (int sub = 0; sub < 8 / kBits; ++sub) {
                m_lsd_pass<kT, kBits>(K, P, K2, P2, 0u, n, 8u * sh.plan.digit[j] + (uint32_t)(sub * kBits), dsm,
                                      sh.tmp, err);
                uint64_t* tk = K; K = K2; K2 = tk;
                uint32_t* tp = P; P = P2; P2 = tp;
            }
        if (!sh.plan.fix) break;
        // segments of equal leading bytes that hold two keys: their starts, found from
        // every key change inside one (galloping back, then bisecting)
        const uint64_t pm = sh.plan.pmask;
        for (uint32_t i = 1 + tid; i < n; i += kT) {
            const uint64_t k0 = K[i - 1], k1 = K[i];
            if (k0 == k1 || ((k0 ^ k1) & pm) != 0) continue;
            const uint64_t mk = k1 & pm;
            uint32_t in = i - 1;
            uint64_t d = 1;
            while (d <= in && (K[in - d] & pm) == mk) {
                in -= (uint32_t)d;
                d <<= 1;
            }
            uint32_t lo = d <= in ? in - (uint32_t)d + 1 : 0u, hi = in;
            while (lo < hi) {
                const uint32_t mid = lo + (hi - lo) / 2;
                if ((K[mid] & pm) == mk) hi = mid;
                else lo = mid + 1;
            }
            const uint32_t slot = atomicAdd(&sh.nseg, 1u);
            if (slot < kMSeg) sh.seg[slot] = lo;
            else sh.overflow = 1;
        }
        __syncthreads();
        if (sh.overflow) continue;  // pack again and sort with every pass
        if (tid == 0) {  // ascending and unique (several key changes share a segment)
            uint32_t m = sh.nseg, u = 0;
            for (uint32_t a = 1; a < m; ++a) {
                const uint32_t v = sh.seg[a];
                uint32_t b = a;
                while (b > 0 && sh.seg[b - 1] > v) {
                    sh.seg[b] = sh.seg[b - 1];
                    --b;
                }
                sh.seg[b] = v;
            }
            for (uint32_t a = 0; a < m; ++a)
                if (a == 0 || sh.seg[a] != sh.seg[u - 1]) sh.seg[u++] = sh.seg[a];
            sh.nseg = u;
        }
        __syncthreads();
        const uint32_t nseg = sh.nseg;
        for (uint32_t x = 0; x < nseg; ++x) {
            const uint32_t s0 = sh.seg[x];
            if (tid == 0) {  // the segment's end: gallop forward, then bisect
                const uint64_t mk = K[s0] & pm;
                uint32_t in = s0;
                uint64_t d = 1;
                while (d < n - in && (K[in + d] & pm) == mk) {
                    in += (uint32_t)d;
                    d <<= 1;
                }
                uint32_t lo = in + 1, hi = (d < n - in) ? in + (uint32_t)d : n;
                while (lo < hi) {
                    const uint32_t mid = lo + (hi - lo) / 2;
                    if ((K[mid] & pm) == mk) lo = mid + 1;
                    else hi = mid;
                }
                sh.j1 = lo;
            }
            __syncthreads();
            const uint32_t e = sh.j1;
            // stable passes over the other bytes, ping-ponging through the other buffer
            uint64_t* A = K;
            uint32_t* AP = P;
            uint64_t* B = K2;
            uint32_t* BP = P2;
            for (uint32_t r = 0; r < sh.plan.nr; ++r)
                for (int sub = 0; sub < 8 / kBits; ++sub) {
                    m_lsd_pass<kT, kBits>(A, AP, B, BP, s0, e, 8u * sh.plan.rdig[r] + (uint32_t)(sub * kBits), dsm,
                                          sh.tmp, err);
                    uint64_t* tk = A; A = B; B = tk;
                    uint32_t* tp = AP; AP = BP; BP = tp;
                }
            if (A != K)
                for (uint32_t i = s0 + tid; i < e; i += kT) {
                    K[i] = A[i];
                    P[i] = AP[i];
                }
            __syncthreads();
        }
        break;
    }
    const uint32_t qv = n - sh.invalid;

    // ---- distinct keys of the valid prefix [0, qv)
    {
        uint32_t carry = 0;
        for (uint32_t c0 = 0; c0 < qv; c0 += kC) {
            const uint32_t j0 = c0 + (uint32_t)tid * kMI;
            uint64_t prev = (j0 > 0 && j0 - 1 < qv) ? K[j0 - 1] : 0ull;
            uint32_t hm = 0;
#pragma unroll
            for (int k = 0; k < kMI; ++k) {
                const uint32_t j = j0 + k;
                const uint64_t kk = j < qv ? K[j] : 0ull;
                if (j < qv && (j == 0 || kk != prev)) hm |= 1u << k;
                prev = kk;
            }
            uint32_t tot;
            uint32_t o = carry + block_excl_sum<kT>((uint32_t)__popc(hm), sh.tmp, &tot);
#pragma unroll
            for (int k = 0; k < kMI; ++k)
                if ((hm >> k) & 1u) s.dq[o++] = K[j0 + k];
            carry += tot;
        }
        if (tid == 0) sh.D = carry;
        __syncthreads();
    }
    const uint32_t D = sh.D;

    // ---- descent + locate for every distinct key
    {
        const DevMeta& m = sh.m;
        const uint32_t H = m.H, Lb = m.Lb, size = m.size;
        const bool built = Lb <= H && H >= 2;
        uint32_t Lp = H + 1;  // lowest level staged in shared memory (> H: none)
        if (built)
            for (int l = (int)H; l >= (int)Lb; --l) {
                if (m.base[l] + m.n[l] + 1u <= kMTop) Lp = (uint32_t)l;
                else break;
            }
        uint64_t* tk = reinterpret_cast<uint64_t*>(dsm);
        uint32_t* td = reinterpret_cast<uint32_t*>(dsm + kMTop * sizeof(uint64_t));
        const uint32_t nst = (built && Lp <= H) ? m.base[Lp] + m.n[Lp] + 1u : 0u;
        for (uint32_t i = tid; i < nst; i += kT) {
            tk[i] = LK[i];
            td[i] = LD[i];
        }
        __syncthreads();
        for (uint32_t d0 = 0; d0 < D; d0 += (uint32_t)kT * kMK) {
            uint64_t q[kMK];
            uint32_t pos[kMK];
            int32_t r[kMK];
            uint32_t act = 0;
#pragma unroll
            for (int k = 0; k < kMK; ++k) {
                const uint32_t d = d0 + (uint32_t)k * kT + (uint32_t)tid;
                q[k] = d < D ? s.dq[d] : kMaxKey;
                pos[k] = 0;
                r[k] = -1;
                if (d < D) act |= 1u << k;
            }
            int l = built ? (int)H : 0;
            if (built && Lp <= H) {
                // the staged level Lp holds every key of the levels above it
                const uint32_t b = m.base[Lp], cnt = m.n[Lp];
#pragma unroll
                for (int k = 0; k < kMK; ++k) {
                    uint32_t lo = 0, hi = cnt;  // first index with key > q
                    while (lo < hi) {
                        const uint32_t mid = (lo + hi) >> 1;
                        if (tk[b + mid] <= q[k]) lo = mid + 1;
                        else hi = mid;
                    }
                    pos[k] = lo ? td[b + lo - 1] : 0u;
                }
                l = (int)Lp - 1;
            }
            if (built)
                for (; l >= (int)Lb; --l) {
                    const uint32_t b = m.base[l];
                    multi_scan(LK + b, q, pos, r, act, m.n[l], err);
#pragma unroll
                    for (int k = 0; k < kMK; ++k) pos[k] = r[k] >= 0 ? LD[b + (uint32_t)r[k]] : 0u;
                }
            if (built) {
                multi_scan(SK, q, pos, r, act, size, err);
            } else {
#pragma unroll
                for (int k = 0; k < kMK; ++k) {  // no index level: binary search of the storage layer
                    uint32_t lo = 0, hi = size;
                    while (lo < hi) {
                        const uint32_t mid = (lo + hi) >> 1;
                        if (SK[mid] <= q[k]) lo = mid + 1;
                        else hi = mid;
                    }
                    r[k] = (int32_t)lo - 1;
                }
            }
#pragma unroll
            for (int k = 0; k < kMK; ++k) {
                if (!((act >> k) & 1u)) continue;
                const uint32_t d = d0 + (uint32_t)k * kT + (uint32_t)tid;
                const bool exists = r[k] >= 0 && SK[r[k]] == q[k];
                const bool live = exists && !(SM[r[k]] & kTomb);
                s.dr[d] = (uint32_t)(r[k] + 1);
                s.df[d] = (uint8_t)((exists ? 1u : 0u) | (live ? 2u : 0u));
                s.dv[d] = live ? SV[r[k]] : 0ull;
            }
        }
        __syncthreads();
    }

    // ---- results, ownership and apply: one pass over [0, qv) with running carries
    {
        uint32_t cmax = 0, cheads = 0, cnew = 0;
        for (uint32_t c0 = 0; c0 < qv; c0 += kC) {
            const uint32_t j0 = c0 + (uint32_t)tid * kMI;
            uint64_t key[kMI];
            uint32_t pay[kMI];
#pragma unroll
            for (int k = 0; k < kMI; ++k) {
                const uint32_t j = j0 + k;
                key[k] = j < qv ? K[j] : kMaxKey;
                pay[k] = j < qv ? P[j] : 0u;
            }
            const uint64_t kprev = (j0 > 0 && j0 - 1 < qv) ? K[j0 - 1] : kMaxKey;
            const uint64_t knext = (j0 + kMI < qv) ? K[j0 + kMI] : kMaxKey;
            uint32_t agg = 0, hm = 0, om = 0;
#pragma unroll
            for (int k = 0; k < kMI; ++k) {
                const uint32_t j = j0 + k;
                const bool valid = j < qv;
                const uint64_t prev = k ? key[k - 1] : kprev;
                const uint64_t next = k + 1 < kMI ? key[k + 1] : knext;
                const bool head = valid && (j == 0 || key[k] != prev);
                const bool last = valid && (j + 1 == qv || key[k] != next);
                const uint32_t op = pay[k] >> 30;
                const uint32_t e = (valid && (op == 1u || op == 2u)) ? 2u * j + 3u : (head ? 2u * j + 2u : 0u);
                agg = max(agg, e);
                hm |= (head ? 1u : 0u) << k;
                om |= (last ? 1u : 0u) << k;
            }
            uint32_t tmax;
            uint32_t M = max(cmax, block_excl_max<kT>(agg, sh.tmp, &tmax));
            uint32_t htot;
            uint32_t hidx = cheads + block_excl_sum<kT>((uint32_t)__popc(hm), sh.tmp, &htot);
            // First walk: every query's result; the owners' final states.
            uint32_t nm = 0, wm = 0, lm = 0;  // new node; run wrote; final live
            uint64_t fval[kMI];
            uint32_t djs[kMI];
#pragma unroll
            for (int k = 0; k < kMI; ++k) {
                const uint32_t j = j0 + k;
                fval[k] = 0;
                djs[k] = 0;
                if (j >= qv) continue;
                const bool head = (hm >> k) & 1u;
                hidx += head ? 1u : 0u;
                const uint32_t dj = hidx - 1u;
                djs[k] = dj;
                const uint32_t op = pay[k] >> 30;
                const uint32_t e = (op == 1u || op == 2u) ? 2u * j + 3u : (head ? 2u * j + 2u : 0u);
                const uint32_t mex = M;
                M = max(M, e);
                const uint8_t fl = s.df[dj];
                bool pl;
                uint64_t pv;
                bool wrote = false;
                if (!head && (mex & 1u)) {  // the last write before j lies in j's key run
                    const uint32_t pw = P[(mex - 3u) >> 1];
                    pl = (pw >> 30) == 1u;
                    pv = pl ? it.vals[pw & kMSeqMask] : 0ull;
                    wrote = true;
                } else {
                    pl = (fl & 2u) != 0;
                    pv = s.dv[dj];
                }
                mstore_result(it.results, pay[k] & kMSeqMask, pl ? pv : 0ull, pl ? PI_R_PRESENT : PI_R_ABSENT);
                if (!((om >> k) & 1u)) continue;
                bool flive = pl;
                uint64_t fv = pv;
                if (op == 1u) {
                    flive = true;
                    fv = it.vals[pay[k] & kMSeqMask];
                    wrote = true;
                } else if (op == 2u) {
                    flive = false;
                    fv = 0;
                    wrote = true;
                }
                fval[k] = fv;
                if (wrote) wm |= 1u << k;
                if (flive) lm |= 1u << k;
                if (wrote && !(fl & 1u) && flive) nm |= 1u << k;
            }
            uint32_t ntot;
            uint32_t slot = cnew + block_excl_sum<kT>((uint32_t)__popc(nm), sh.tmp, &ntot);
            // Second walk: the owners whose run wrote update their node or add a new one.
            int32_t tomb_d = 0;
            uint32_t chg = 0, dirty = 0;
#pragma unroll
            for (int k = 0; k < kMI; ++k) {
                if (!((wm >> k) & 1u)) continue;
                const uint32_t dj = djs[k];
                const uint8_t fl = s.df[dj];
                const bool flive = (lm >> k) & 1u;
                const bool live0 = (fl & 2u) != 0;
                if (fl & 1u) {
                    const uint32_t r = s.dr[dj] - 1u;
                    const uint8_t meta = SM[r];
                    const uint32_t h = meta & 0x3Fu;
                    if (flive) SV[r] = fval[k];
                    SM[r] = (uint8_t)(h | (flive ? 0u : kTomb));
                    if (flive != live0) {
                        tomb_d += flive ? -1 : 1;
                        ++chg;
                        if (h >= 2u) dirty = 1;
                        for (uint32_t l = 1; l <= h && l < (uint32_t)kLevelSlots; ++l)
                            atomicAdd(&sh.delta[l], flive ? 1 : -1);
                    }
                } else if (flive) {
                    const uint32_t h = tower_height(key[k], X.hp);
                    s.nk[slot] = key[k];
                    s.nv[slot] = fval[k];
                    s.nh[slot] = (uint8_t)h;
                    s.ni[slot] = s.dr[dj];
                    ++slot;
                    ++chg;
                    dirty = 1;
                    for (uint32_t l = 1; l <= h && l < (uint32_t)kLevelSlots; ++l) atomicAdd(&sh.delta[l], 1);
                }
            }
            if (tomb_d) atomicAdd(&sh.tomb_delta, tomb_d);
            if (chg) atomicAdd(&sh.changes, chg);
            if (dirty) sh.dirty = 1;
            cmax = max(cmax, tmax);
            cheads += htot;
            cnew += ntot;
        }
        // invalid queries
        for (uint32_t j = qv + tid; j < n; j += kT) mstore_result(it.results, P[j] & kMSeqMask, 0ull, PI_R_INVALID);
        if (tid == 0) sh.newc = cnew;
        __syncthreads();
        if (tid == 0) {
            DevMeta& m = sh.m;
            m.tombs = (uint32_t)((int32_t)m.tombs + sh.tomb_delta);
            for (int l = 1; l < kLevelSlots; ++l) m.cnt[l] = (uint32_t)((int32_t)m.cnt[l] + sh.delta[l]);
            m.updates += sh.changes;
            m.batches += 1;
        }
        __syncthreads();
    }

    // ---- the new level layout (before the merge, which may write the lowest level)
    const uint32_t M = sh.newc;
    const bool merged = M > 0 || (sh.m.tombs > 0 && (uint64_t)sh.m.tombs * 8u > sh.m.size);
    const bool relevel = merged || sh.dirty;
    if (relevel) {
        if (tid == 0) {
            DevMeta& m = sh.m;
            uint32_t H = 1;
            for (int l = 2; l < kLevelSlots; ++l)
                if (m.cnt[l] > 0) H = (uint32_t)l;
            const uint32_t Lb0 = X.min_lb > 2u ? X.min_lb : 2u;
            uint64_t need = 0;
            for (uint32_t l = Lb0; l <= H; ++l) need += (uint64_t)m.cnt[l] + 1u;
            uint32_t Lb = Lb0;
            uint64_t fit = need;
            while (Lb <= H && fit > X.idx_cap) {
                fit -= (uint64_t)m.cnt[Lb] + 1u;
                ++Lb;
            }
            m.index_need = (uint32_t)need;
            m.grow_request = (Lb > Lb0) ? 1u : 0u;
            for (int l = 0; l < kLevelSlots; ++l) {
                m.n[l] = 0;
                m.base[l] = 0;
            }
            uint32_t off = 0;
            for (int l = (int)H; l >= (int)Lb; --l) {
                m.base[l] = off;
                m.n[l] = m.cnt[l];
                off += m.cnt[l] + 1u;
            }
            m.H = H;
            m.Lb = Lb;
            m.index_total = off;
            uint32_t Ls = H + 1;
            for (int l = (int)H; l >= (int)Lb; --l) {
                if (m.base[l] + m.n[l] + 1u <= X.smem_top) Ls = (uint32_t)l;
                else break;
            }
            m.Ls = Ls;
            m.smem_entries = (Ls <= H) ? m.base[Ls] + m.n[Ls] + 1u : 0u;
            m.updates = 0;
            m.rebuilds += 1;
            m.levels_exact = 1;  // rebuilt in place from the storage layer
        }
        __syncthreads();
    }
    // A merge rewrites the storage layer in key order, so it also writes the lowest built
    // level: each member's key and new storage position, at its rank among the members.
    const bool fused = merged && sh.m.Lb <= sh.m.H;

    // ---- merge: live old nodes and the new nodes into the other storage buffer
    if (merged) {
        const uint32_t size = sh.m.size;
        const uint32_t dst = cur ^ 1u;
        uint64_t* DK = X.st.keys[dst];
        uint64_t* DV = X.st.vals[dst];
        uint8_t* DM = X.st.meta[dst];
        const uint32_t Lb = sh.m.Lb, lbase = sh.m.base[Lb];
        uint32_t* nmp = s.dr;  // members among the first j new nodes (the descent's output is dead)
        if (fused) {
            uint32_t run = 0;
            for (uint32_t g0 = 0; g0 < M; g0 += kC) {
                const uint32_t i0 = g0 + (uint32_t)tid * kMI;
                uint32_t mm = 0;
#pragma unroll
                for (int k = 0; k < kMI; ++k)
                    if (i0 + k < M && s.nh[i0 + k] >= Lb) mm |= 1u << k;
                uint32_t tot;
                uint32_t r = run + block_excl_sum<kT>((uint32_t)__popc(mm), sh.tmp, &tot);
#pragma unroll
                for (int k = 0; k < kMI; ++k) {
                    if (i0 + k < M) nmp[i0 + k] = r;
                    r += (mm >> k) & 1u;
                }
                run += tot;
            }
            if (tid == 0) nmp[M] = run;
            __syncthreads();
        }
        uint32_t* lp = reinterpret_cast<uint32_t*>(dsm);  // live old nodes before each chunk position
        uint32_t* nl = lp + kC;                             // new nodes at or before each chunk position
        uint32_t* ob = nl + kC;                             // old members of level Lb before each position
        uint32_t carry = 0, cmem = 0, j0 = 0;
        for (uint32_t c0 = 0; c0 < size; c0 += kC) {
            const uint32_t lim = c0 + kC < size ? c0 + kC : size;
            if (tid == 0 && lim < size) {  // the next chunk's nodes into L2 while this one is copied
                const uint32_t nx = lim, nn = (size - nx < kC ? size - nx : kC);
                // nx is a multiple of the chunk, so every start is 16-byte aligned; sizes
                // round up to 16 bytes (the storage arrays are padded past their end)
                l2_prefetch(SK + nx, (nn * 8u + 15u) & ~15u);
                l2_prefetch(SV + nx, (nn * 8u + 15u) & ~15u);
                l2_prefetch(SM + nx, (nn + 15u) & ~15u);
            }
            if (tid < 32) {  // new nodes placed before an old node of this chunk: [j0, j1)
                const uint32_t r = j0 + warp_count_below(s.ni + j0, M - j0, lim);
                if (tid == 0) sh.j1 = r;
            }
            for (uint32_t x = tid; x < kC; x += kT) nl[x] = 0u;
            __syncthreads();
            const uint32_t j1 = sh.j1;
            for (uint32_t j = j0 + tid; j < j1; j += kT) atomicAdd(&nl[s.ni[j] - c0], 1u);
            __syncthreads();
            // blocked: positions [kMI tid, kMI tid + kMI) of the chunk
            const uint32_t b0 = (uint32_t)tid * kMI, i0 = c0 + b0;
            uint32_t lmask = 0, omask = 0, nsum = 0;
            uint32_t nat[kMI];
            uint32_t hb[kMI];
            if (i0 + kMI <= size) {
                const uint2 w8 = *reinterpret_cast<const uint2*>(SM + i0);  // i0 is a multiple of 8
#pragma unroll
                for (int k = 0; k < kMI; ++k) hb[k] = ((k < 4 ? w8.x : w8.y) >> (8 * (k & 3))) & 0xFFu;
            } else {
#pragma unroll
                for (int k = 0; k < kMI; ++k) hb[k] = i0 + k < size ? (uint32_t)SM[i0 + k] : (uint32_t)kTomb;
            }
#pragma unroll
            for (int k = 0; k < kMI; ++k) {
                if (!(hb[k] & kTomb)) {
                    lmask |= 1u << k;
                    if (fused && (hb[k] & 0x3Fu) >= Lb) omask |= 1u << k;
                }
                nat[k] = nl[b0 + k];
                nsum += nat[k];
            }
            // one scan of three counts: live (bits 0-15), old members (16-31), new (32-63)
            uint64_t tot;
            const uint64_t ex = block_excl_sum64<kT>(
                (uint64_t)__popc(lmask) | ((uint64_t)__popc(omask) << 16) | ((uint64_t)nsum << 32), sh.tmp64, &tot);
            {
                uint32_t rl = carry + (uint32_t)(ex & 0xFFFFu), ro = cmem + (uint32_t)((ex >> 16) & 0xFFFFu);
                uint32_t rn = j0 + (uint32_t)(ex >> 32);
#pragma unroll
                for (int k = 0; k < kMI; ++k) {
                    lp[b0 + k] = rl;
                    ob[b0 + k] = ro;
                    rl += (lmask >> k) & 1u;
                    ro += (omask >> k) & 1u;
                    rn += nat[k];
                    nl[b0 + k] = rn;
                }
            }
            __syncthreads();
            // striped: the chunk's live old nodes, coalesced, four positions per round
            const uint32_t cnt = lim - c0;
            for (uint32_t x0 = tid; x0 < cnt; x0 += 4u * kT) {
                uint32_t mt[4];
                uint64_t kv[4], vv[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const uint32_t x = x0 + (uint32_t)u * kT;
                    const bool in = x < cnt;
                    mt[u] = in ? (uint32_t)SM[c0 + x] : (uint32_t)kTomb;
                    kv[u] = in ? SK[c0 + x] : 0ull;
                    vv[u] = in ? SV[c0 + x] : 0ull;
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    if (mt[u] & kTomb) continue;
                    const uint32_t x = x0 + (uint32_t)u * kT;
                    const uint32_t o = lp[x] + nl[x];
                    DK[o] = kv[u];
                    DV[o] = vv[u];
                    DM[o] = (uint8_t)(mt[u] & 0x3Fu);
                    if (fused && (mt[u] & 0x3Fu) >= Lb) {
                        const uint32_t r = ob[x] + nmp[nl[x]];
                        if (r < sh.m.n[Lb]) {
                            LK[lbase + r] = kv[u];
                            LD[lbase + r] = o;
                        }
                    }
                }
            }
            for (uint32_t j = j0 + tid; j < j1; j += kT) {
                const uint32_t x = s.ni[j] - c0;
                const uint32_t o = j + lp[x];
                DK[o] = s.nk[j];
                DV[o] = s.nv[j];
                DM[o] = s.nh[j];
                if (fused && s.nh[j] >= Lb) {
                    const uint32_t r = ob[x] + nmp[j];
                    if (r < sh.m.n[Lb]) {
                        LK[lbase + r] = s.nk[j];
                        LD[lbase + r] = o;
                    }
                }
            }
            carry += (uint32_t)(tot & 0xFFFFu);
            cmem += (uint32_t)((tot >> 16) & 0xFFFFu);
            j0 = j1;
            __syncthreads();
        }
        for (uint32_t j = j0 + tid; j < M; j += kT) {  // after the last old node
            const uint32_t o = j + carry;
            DK[o] = s.nk[j];
            DV[o] = s.nv[j];
            DM[o] = s.nh[j];
            if (fused && s.nh[j] >= Lb) {
                const uint32_t r = cmem + nmp[j];
                if (r < sh.m.n[Lb]) {
                    LK[lbase + r] = s.nk[j];
                    LD[lbase + r] = o;
                }
            }
        }
        const uint32_t nsize = carry + M;
        if (tid == 0) {
            if (nsize > X.st_cap) atomicOr(err, kErrBounds);
            if (fused && cmem + nmp[M] != sh.m.n[Lb]) atomicOr(err, kErrBounds);
            DK[nsize] = kMaxKey;
            DV[nsize] = 0;
            DM[nsize] = 0;
            sh.m.size = nsize;
            sh.m.tombs = 0;
            sh.m.cur = dst;
        }
        __syncthreads();
    }

    // ---- rebuild the index layer when the membership of any level changed
    if (relevel) {
        __syncthreads();
        const DevMeta& m = sh.m;
        const uint32_t H = m.H, Lb = m.Lb, size = m.size;
        const uint32_t ncur = m.cur;
        const uint64_t* RK = X.st.keys[ncur];
        const uint8_t* RM = X.st.meta[ncur];
        if (Lb <= H) {
            // level Lb from the storage layer: live nodes of height >= Lb (a merge wrote it)
            uint32_t carry = 0;
            if (!fused) {
            for (uint32_t c0 = 0; c0 < size; c0 += kC) {
                const uint32_t i0 = c0 + (uint32_t)tid * kMI;
                uint32_t mm = 0;
#pragma unroll
                for (int k = 0; k < kMI; ++k) {
                    const uint32_t i = i0 + k;
                    if (i < size) {
                        const uint8_t mt = RM[i];
                        if (!(mt & kTomb) && (mt & 0x3Fu) >= Lb) mm |= 1u << k;
                    }
                }
                uint32_t tot;
                uint32_t o = carry + block_excl_sum<kT>((uint32_t)__popc(mm), sh.tmp, &tot);
#pragma unroll
                for (int k = 0; k < kMI; ++k) {
                    if (!((mm >> k) & 1u)) continue;
                    if (o < m.n[Lb]) {
                        LK[m.base[Lb] + o] = RK[i0 + k];
                        LD[m.base[Lb] + o] = i0 + k;
                    }
                    ++o;
                }
                carry += tot;
            }
            if (tid == 0 && carry != m.n[Lb]) atomicOr(err, kErrBounds);
            }
            __syncthreads();
            // level l + 1 from level l: its members of height >= l + 1
            for (uint32_t l = Lb; l < H; ++l) {
                const uint32_t bl = m.base[l], nl = m.n[l], bu = m.base[l + 1], nu = m.n[l + 1];
                carry = 0;
                for (uint32_t c0 = 0; c0 < nl; c0 += kC) {
                    const uint32_t i0 = c0 + (uint32_t)tid * kMI;
                    uint32_t mm = 0;
                    uint64_t kk[kMI];
#pragma unroll
                    for (int k = 0; k < kMI; ++k) {
                        const uint32_t i = i0 + k;
                        kk[k] = i < nl ? LK[bl + i] : 0ull;
                        if (i < nl && tower_height(kk[k], X.hp) >= l + 1u) mm |= 1u << k;
                    }
                    uint32_t tot;
                    uint32_t o = carry + block_excl_sum<kT>((uint32_t)__popc(mm), sh.tmp, &tot);
#pragma unroll
                    for (int k = 0; k < kMI; ++k) {
                        if (!((mm >> k) & 1u)) continue;
                        if (o < nu) {
                            LK[bu + o] = kk[k];
                            LD[bu + o] = i0 + k;
                        }
                        ++o;
                    }
                    carry += tot;
                }
                if (tid == 0 && carry != nu) atomicOr(err, kErrBounds);
                __syncthreads();
            }
            for (uint32_t l = Lb + tid; l <= H; l += kT) {  // sentinels
                const uint32_t sidx = m.base[l] + m.n[l];
                LK[sidx] = kMaxKey;
                LD[sidx] = (l > Lb) ? m.n[l - 1] : size;
            }
        }
        __syncthreads();
    }

    // ---- publish the index's new state
    if (tid == 0) {
        DevMeta* gm = X.m;
        const DevMeta& m = sh.m;
        gm->cur = m.cur;
        gm->size = m.size;
        gm->tombs = m.tombs;
        gm->H = m.H;
        gm->Lb = m.Lb;
        gm->Ls = m.Ls;
        gm->smem_entries = m.smem_entries;
        gm->index_total = m.index_total;
        gm->index_need = m.index_need;
        gm->grow_request = m.grow_request;
        gm->updates = m.updates;
        gm->rebuilds = m.rebuilds;
        gm->levels_exact = m.levels_exact;
        gm->batches = m.batches;
        for (int l = 0; l < kLevelSlots; ++l) {
            gm->cnt[l] = m.cnt[l];
            gm->n[l] = m.n[l];
            gm->base[l] = m.base[l];
        }
        if (a.mirror) a.mirror[it.index] = *gm;  // the host reads the set's sizes from one copy
    }
    __syncthreads();
}

template <int kW, int kBits>
__global__ void __launch_bounds__(kW * 32) k_multi(MultiArgs a) {
    constexpr int kT = kW * 32;
    extern __shared__ __align__(16) uint8_t dsm[];
    __shared__ MShared sh;
    const MScratchPtrs s = carve(a.scratch + (uint64_t)blockIdx.x * a.stride, a.qcap);
    const uint32_t nitems = *a.nitems;
    for (;;) {
        if (threadIdx.x == 0) sh.item = atomicAdd(a.head, 1u);
        __syncthreads();
        const uint32_t item = sh.item;
        __syncthreads();
        if (item >= nitems) break;
        const MItem it = a.items[item];
        if (it.n <= a.qcap) m_item<kT, kBits>(a, it, s, dsm, sh);
        else if (threadIdx.x == 0) atomicOr(&a.idx[it.index].m->error, kErrBounds);
        __syncthreads();
    }
}

template <int kW, int kBits>
constexpr int multi_smem() {
    constexpr int kT = kW * 32;
    constexpr int sort = (kW * (1 << kBits) + 2 * (1 << kBits)) * 4;
    constexpr int top = (int)kMTop * 12;
    constexpr int merge = kT * kMI * 12;  // live, new-node and member prefixes per chunk position
    return sort > top ? (sort > merge ? sort : merge) : (top > merge ? top : merge);
}

// Sets the kernel's dynamic shared-memory limit (once; before any capture) and returns
// its resident CTAs per SM.
template <int kW, int kBits>
cudaError_t occupancy_t(int* blocks) {
    constexpr int dyn = multi_smem<kW, kBits>();
    cudaError_t e = cudaFuncSetAttribute(k_multi<kW, kBits>, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k_multi<kW, kBits>, kW * 32, dyn);
}

template <int kW, int kBits>
cudaError_t launch_multi_t(const MultiArgs& a, uint32_t grid, cudaStream_t s) {
    k_multi<kW, kBits><<<grid, kW * 32, multi_smem<kW, kBits>(), s>>>(a);
    ++g_launches;
    return cudaGetLastError();
}

}  // namespace

uint64_t multi_scratch_bytes(uint32_t qcap) {
    const uint64_t c = (uint64_t)qcap + kPad;
    auto al = [](uint64_t b) { return (b + 255u) & ~255ull; };
    return 2 * al(c * 8) + 2 * al(c * 4) + al(c * 8) + al(c * 4) + al(c) + al(c * 8) + 2 * al(c * 8) + al(c) +
           al(c * 4);
}

// multi_occupancy must have run for the variant first (it sets the shared-memory limit).
cudaError_t launch_multi(const MultiArgs& a, int warps, int radix_bits, uint32_t grid, cudaStream_t s) {
    if (grid == 0) return cudaSuccess;
    if (radix_bits == 8) {
        if (warps == 8) return launch_multi_t<8, 8>(a, grid, s);
        if (warps == 16) return launch_multi_t<16, 8>(a, grid, s);
        if (warps == 32) return launch_multi_t<32, 8>(a, grid, s);
    } else if (radix_bits == 4) {
        if (warps == 8) return launch_multi_t<8, 4>(a, grid, s);
        if (warps == 16) return launch_multi_t<16, 4>(a, grid, s);
        if (warps == 32) return launch_multi_t<32, 4>(a, grid, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t multi_occupancy(int warps, int radix_bits, int* blocks) {
    if (radix_bits == 8) {
        if (warps == 8) return occupancy_t<8, 8>(blocks);
        if (warps == 16) return occupancy_t<16, 8>(blocks);
        if (warps == 32) return occupancy_t<32, 8>(blocks);
    } else if (radix_bits == 4) {
        if (warps == 8) return occupancy_t<8, 4>(blocks);
        if (warps == 16) return occupancy_t<16, 4>(blocks);
        if (warps == 32) return occupancy_t<32, 4>(blocks);
    }
    return cudaErrorInvalidValue;
}

}  // namespace pi
