// alf_sweep.cuh -- the round loop of the sweep for one grid, run by one warp
// (the field-resident schedule and the near-source hierarchy share it).
#pragma once

#include "alf_internal.h"

namespace alf {

// order-preserving keys of non-negative times, and their warp minimum
ALF_D unsigned order_key(float v) { return __float_as_uint(v); }  // v >= 0
ALF_D unsigned long long order_key(double v) { return (unsigned long long)__double_as_longlong(v); }
ALF_D float from_key(unsigned k, float) { return __uint_as_float(k); }
ALF_D double from_key(unsigned long long k, double) { return __longlong_as_double((long long)k); }
ALF_D unsigned warp_min(unsigned v) { return __reduce_min_sync(0xffffffffu, v); }
ALF_D unsigned long long warp_min(unsigned long long v)
{
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
        v = w < v ? w : v;
    }
    return v;
}


// Which of the 12 diamond slots of node (i, j) lie inside the nx x ny grid: eight edge tests, combined per slot
// (slot order as kSlotDi / kSlotDj), instead of four bounds tests per slot.
struct SlotInGrid {
    bool v[12];
};
ALF_D SlotInGrid slots_in_grid(int i, int j, int nx, int ny)
{
    const bool l1 = i >= 1, l2 = i >= 2, r1 = i + 1 < nx, r2 = i + 2 < nx;
    const bool d1 = j >= 1, d2 = j >= 2, u1 = j + 1 < ny, u2 = j + 2 < ny;
    return SlotInGrid{{l1, r1, d1, u1, l1 && d1, r1 && d1, l1 && u1, r1 && u1, l2, r2, d2, u2}};
}

// One grid swept by one warp: a field, or one level of the near-source hierarchy.
template <typename T>
struct WarpGrid {
    T* tf;                      // times of the grid (frozen nodes carry the sign bit)
    int nx, ny;
    const uint32_t* map;        // region id of every node
    const RegionP<T>* reg;      // region constants of the sample
    T scale;                    // spacing of this grid / spacing of the regions' grid
    unsigned* list0;            // dirty lists and evaluation list, nx * ny entries each
    unsigned* list1;
    unsigned* el;
    T* ov;                      // time before / after each evaluation of a round
    T* nv;
    uint8_t* rec;               // records (may be null)
    unsigned* bm;               // dirty bitmap, (nx * ny + 31) / 32 words (shared memory)
    T band;                     // evaluation band beyond the front time
    unsigned max_rounds;
};

// clears the bitmap and makes the non-frozen nodes of the square of half-width r around (ci, cj) the first dirty
// set; returns its size
template <typename T>
ALF_D unsigned warp_seed_square(const WarpGrid<T>& g, int ci, int cj, int r)
{
    constexpr unsigned FULL = 0xffffffffu;
    const unsigned lane = threadIdx.x & 31u;
    const unsigned below = (1u << lane) - 1u;
    const unsigned words = (unsigned)((g.nx * g.ny + 31) / 32);
    for (unsigned w = lane; w < words; w += 32u) g.bm[w] = 0u;
    __syncwarp();
    unsigned nact = 0u;
    const int w = 2 * r + 1;
    for (int base = 0; base < w * w; base += 32) {
        const int k = base + (int)lane;
        bool take = false;
        unsigned n = 0u;
        if (k < w * w) {
            const int i = ci + k % w - r, j = cj + k / w - r;
            if (i >= 0 && j >= 0 && i < g.nx && j < g.ny) {
                n = (unsigned)(j * g.nx + i);
                take = !neg_bit(g.tf[n]);
            }
        }
        const unsigned bal = __ballot_sync(FULL, take);
        if (take) {
            g.list0[nact + __popc(bal & below)] = n;
            atomicOr(g.bm + (n >> 5), 1u << (n & 31u));
        }
        nact += __popc(bal);
    }
    __syncwarp();
    return nact;
}

// rounds of one grid to its fixed point; returns the evaluations, writes the rounds taken, false when the
// round cap was reached
template <typename T, bool VT = false>
ALF_D bool warp_sweep(const WarpGrid<T>& g, unsigned nact, unsigned long long& evals, unsigned& rounds,
                      unsigned long long& scanned)
{
    constexpr unsigned FULL = 0xffffffffu;
    const unsigned lane = threadIdx.x & 31u;
    const unsigned below = (1u << lane) - 1u;
    const T inf = alf_inf<T>();
    const int nx = g.nx, ny = g.ny;
    T* const tf = g.tf;
    unsigned par = 0u;
    rounds = 0u;
    evals = 0ull;
    scanned = 0ull;
    while (nact != 0u) {
        if (++rounds > g.max_rounds) return false;
        scanned += nact;
        const unsigned* LA = par ? g.list1 : g.list0;
        unsigned* LB = par ? g.list0 : g.list1;
        // front time of the dirty set and the band limit
        auto m = order_key(inf);
        for (unsigned k = lane; k < nact; k += 32u) {
            const auto v = order_key(tf[LA[k]]);
            m = v < m ? v : m;
        }
        const T lim = from_key(warp_min(m), T(0)) + g.band;
        // split: in-band (or still unknown) nodes are evaluated, the rest wait
        unsigned ne = 0u, nc = 0u;
        for (unsigned base = 0; base < nact; base += 32u) {
            const unsigned k = base + lane;
            const bool in = k < nact;
            bool ev = false;
            unsigned n = 0u;
            if (in) {
                n = LA[k];
                const T t = tf[n];
                ev = t <= lim || !(t < inf);
            }
            const unsigned be = __ballot_sync(FULL, in && ev), bc = __ballot_sync(FULL, in && !ev);
            if (in && ev) {
                g.el[ne + __popc(be & below)] = n;
                atomicAnd(g.bm + (n >> 5), ~(1u << (n & 31u)));
            } else if (in) {
                LB[nc + __popc(bc & below)] = n;
            }
            ne += __popc(be);
            nc += __popc(bc);
        }
        __syncwarp();
        // evaluate F at the in-band nodes (times updated in place)
        for (unsigned e = lane; e < ne; e += 32u) {
            const unsigned n = g.el[e];
            const int i = (int)(n % (unsigned)nx), j = (int)(n / (unsigned)nx);
            const SlotInGrid in = slots_in_grid(i, j, nx, ny);
            T nb[12];
#pragma unroll
            for (int q = 0; q < 12; ++q) nb[q] = in.v[q] ? tf[(int)n + sdj(q) * nx + sdi(q)] : inf;
            const T old = tf[n];
            RegionP<T> R = g.reg[__ldg(g.map + n)];
            if (g.scale != T(1)) {
                R.h *= g.scale;
#pragma unroll
                for (int c = 0; c < 4; ++c) R.fb[c] *= g.scale;
            }
            int rc;
            const T v = local_F<T, VT>(nb, (int)n, nx, R, rc);
            if (g.rec) g.rec[n] = (uint8_t)rc;
            if (!same_bits(v, old)) tf[n] = v;
            g.ov[e] = old;
            g.nv[e] = v;
        }
        evals += ne;
        __syncwarp();
        // marking: changed nodes wake their later known neighbours; in-band nodes seed
        // their unknown neighbours; an out-of-band node with unknown neighbours waits.  A lane's
        // push decisions come first (plain loads), then its dirty-bit test-and-sets (issued
        // independently of one another), then its slots (a warp prefix sum of the counts).
        for (unsigned base = 0; base < ne; base += 32u) {
            const unsigned e = base + lane;
            unsigned pm = 0u;  // bit q < 12: neighbour q; bit 12: the node itself (seeds later)
            unsigned n = 0u;
            int i = 0, j = 0;
            if (e < ne) {
                const T o = g.ov[e];
                const T v = g.nv[e];
                const bool changed = !same_bits(o, v);
                const bool inband = v <= lim;
                n = g.el[e];
                i = (int)(n % (unsigned)nx);
                j = (int)(n / (unsigned)nx);
                if (changed || inband) {
                    const T lo = v < o ? v : o;
                    bool seeds_later = false;
                    const SlotInGrid in = slots_in_grid(i, j, nx, ny);
#pragma unroll
                    for (int q = 0; q < 12; ++q) {
                        if (in.v[q]) {
                            const T tm = tf[(int)n + sdj(q) * nx + sdi(q)];
                            if (!neg_bit(tm)) {
                                bool push = false;
                                if (tm < inf) push = changed && lo <= tm;
                                else if (inband) push = true;
                                else seeds_later = true;
                                pm |= push ? 1u << q : 0u;
                            }
                        }
                    }
                    if (seeds_later && v < inf) pm |= 1u << 12;
                }
                unsigned dup = 0u;
#pragma unroll
                for (int q = 0; q < 13; ++q)
                    if ((pm >> q) & 1u) {
                        const unsigned mnode = q < 12 ? (unsigned)((j + sdj(q)) * nx + (i + sdi(q))) : n;
                        const unsigned bit = 1u << (mnode & 31u);
                        dup |= (atomicOr(g.bm + (mnode >> 5), bit) & bit) ? 1u << q : 0u;
                    }
                pm &= ~dup;
            }
            const unsigned cnt = (unsigned)__popc(pm);
            unsigned incl = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned y = __shfl_up_sync(FULL, incl, o);
                if ((int)lane >= o) incl += y;
            }
            unsigned slot = nc + incl - cnt;
#pragma unroll
            for (int q = 0; q < 13; ++q)
                if ((pm >> q) & 1u)
                    LB[slot++] = q < 12 ? (unsigned)((j + sdj(q)) * nx + (i + sdi(q))) : n;
            nc += __shfl_sync(FULL, incl, 31);
        }
        __syncwarp();
        nact = nc;
        par ^= 1u;
    }
    return true;
}


// ---------------------------------------------------------------------------
// The same rounds run by a whole CTA of NT threads on one grid (for few, large
// fields), or by a cluster of CS such CTAs on CS SMs: barriers between the
// steps, list slots reserved per warp with counters in shared memory (those of
// the cluster's rank 0 when CS > 1, reached through distributed shared memory).
// The dirty bitmap is in shared memory (rank 0's) or in global memory.
// ---------------------------------------------------------------------------
struct CtaSweepShared {
    unsigned cnt[3];       // near evaluation / carried (then marked) / far evaluation list sizes of the round
    unsigned long long kmin[32];
};

// rank of this CTA in its cluster (0 without clusters)
template <int CS>
ALF_D unsigned cluster_rank()
{
    if constexpr (CS == 1) {
        return 0u;
    } else {
        unsigned r;
        asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
        return r;
    }
}

// barrier of the CTA, or of the whole cluster with release / acquire ordering of
// the global and shared memory operations before and after it
template <int CS>
ALF_D void sweep_sync()
{
    if constexpr (CS == 1)
        __syncthreads();
    else
        asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// generic address of the same shared-memory object in the cluster's CTA `rank`
template <typename P>
ALF_D P* map_rank(P* ptr, unsigned rank)
{
    unsigned long long d;
    asm volatile("mapa.u64 %0, %1, %2;" : "=l"(d) : "l"((unsigned long long)ptr), "r"(rank));
    return (P*)d;
}

template <typename T>
ALF_D unsigned reserve(unsigned* counter, bool take, unsigned below)
{
    // warp-aggregated slot reservation: returns this lane's slot (valid when take)
    const unsigned bal = __ballot_sync(0xffffffffu, take);
    const unsigned lane = threadIdx.x & 31u;
    unsigned base = 0u;
    if (bal != 0u) {
        const int leader = __ffs(bal) - 1;
        if ((int)lane == leader) base = atomicAdd(counter, (unsigned)__popc(bal));
        base = __shfl_sync(0xffffffffu, base, leader);
    }
    return base + __popc(bal & below);
}

// clears the bitmap and seeds the square of half-width r around (ci, cj); returns the dirty-set size.
// S: the shared counters (rank 0's with clusters).
template <typename T, int NT, int CS = 1>
ALF_D unsigned cta_seed_square(const WarpGrid<T>& g, int ci, int cj, int r, CtaSweepShared& S)
{
    constexpr unsigned STRIDE = (unsigned)(NT * CS);
    const unsigned tid = cluster_rank<CS>() * NT + threadIdx.x;
    const unsigned below = (1u << (threadIdx.x & 31u)) - 1u;
    const unsigned words = (unsigned)((g.nx * g.ny + 31) / 32);
    for (unsigned w = tid; w < words; w += STRIDE) g.bm[w] = 0u;
    if (tid == 0) {
        S.cnt[1] = 0u;
        S.kmin[0] = ~0ull;
    }
    sweep_sync<CS>();
    const int w = 2 * r + 1;
    for (int base = 0; base < w * w; base += (int)STRIDE) {
        const int k = base + (int)tid;
        bool take = false;
        unsigned n = 0u;
        if (k < w * w) {
            const int i = ci + k % w - r, j = cj + k / w - r;
            if (i >= 0 && j >= 0 && i < g.nx && j < g.ny) {
                n = (unsigned)(j * g.nx + i);
                take = !neg_bit(g.tf[n]);
            }
        }
        const unsigned slot = reserve<T>(&S.cnt[1], take, below);
        if (take) {
            g.list0[slot] = n;
            atomicOr(g.bm + (n >> 5), 1u << (n & 31u));
        }
    }
    sweep_sync<CS>();
    const unsigned nact = S.cnt[1];
    sweep_sync<CS>();
    return nact;
}

template <typename T, int NT, bool VT = false, int CS = 1>
ALF_D bool cta_sweep(const WarpGrid<T>& g, unsigned nact, unsigned long long& evals, unsigned& rounds,
                     CtaSweepShared& S, unsigned long long& scanned)
{
    constexpr int NW = NT / 32;
    constexpr unsigned STRIDE = (unsigned)(NT * CS);
    const unsigned tid = cluster_rank<CS>() * NT + threadIdx.x;
    const unsigned lane = threadIdx.x & 31u, wid = threadIdx.x >> 5;
    const unsigned below = (1u << lane) - 1u;
    const T inf = alf_inf<T>();
    const int nx = g.nx, ny = g.ny;
    T* const tf = g.tf;
    unsigned par = 0u;
    rounds = 0u;
    evals = 0ull;
    scanned = 0ull;
    while (nact != 0u) {
        if (++rounds > g.max_rounds) return false;
        scanned += nact;
        const unsigned* LA = par ? g.list1 : g.list0;
        unsigned* LB = par ? g.list0 : g.list1;
        // front time of the dirty set
        auto m = order_key(inf);
        for (unsigned k = tid; k < nact; k += STRIDE) {
            const auto v = order_key(tf[LA[k]]);
            m = v < m ? v : m;
        }
        m = warp_min(m);
        if constexpr (CS == 1) {
            if (lane == 0) S.kmin[wid] = (unsigned long long)m;
        } else {
            // one minimum per round in rank 0, double-buffered: this round's slot was reset in the last one
            if (lane == 0) atomicMin(&S.kmin[par], (unsigned long long)m);
            if (tid == 0) S.kmin[par ^ 1u] = ~0ull;
        }
        if (tid == 0) {
            S.cnt[0] = 0u;
            S.cnt[1] = 0u;
            S.cnt[2] = 0u;
        }
        sweep_sync<CS>();
        auto mm = order_key(inf);
        if constexpr (CS == 1) {
#pragma unroll
            for (int w = 0; w < NW; ++w) {
                const auto v = (decltype(mm))S.kmin[w];
                mm = v < mm ? v : mm;
            }
        } else {
            mm = (decltype(mm))S.kmin[par];
        }
        const T front = from_key(mm, T(0));
        const T lim = front + g.band, near = front + T(0.75) * g.band;
        // split: the entries in the band (or without a value) are evaluated, those in its nearer three
        // quarters at the front of the evaluation list and the rest from its back, so that the first passes of
        // the round take the earliest nodes and later ones see their new values (on the weld batch: 2.23
        // evaluations per node at band 2 against 2.29 unordered at the best band, 1.5); the rest stay
        const unsigned last = (unsigned)(nx * ny) - 1u;
        for (unsigned base = 0; base < nact; base += STRIDE) {
            const unsigned k = base + tid;
            const bool in = k < nact;
            bool ev = false, nr = false;
            unsigned n = 0u;
            if (in) {
                n = LA[k];
                const T t = tf[n];
                ev = t <= lim || !(t < inf);
                nr = t <= near;
            }
            const unsigned sn = reserve<T>(&S.cnt[0], in && ev && nr, below);
            const unsigned sf = reserve<T>(&S.cnt[2], in && ev && !nr, below);
            const unsigned sc = reserve<T>(&S.cnt[1], in && !ev, below);
            if (in && ev) {
                g.el[nr ? sn : last - sf] = n;
                atomicAnd(g.bm + (n >> 5), ~(1u << (n & 31u)));
            } else if (in) {
                LB[sc] = n;
            }
        }
        sweep_sync<CS>();
        // entry e of the round: el[e] below nnear, el[last - (e - nnear)] after (the two parts never meet: the
        // dirty set holds each node once); its values before and after at the same index
        const unsigned nnear = S.cnt[0], ne = S.cnt[0] + S.cnt[2];
        // evaluate
        for (unsigned e0 = tid; e0 < ne; e0 += STRIDE) {
            const unsigned e = e0 < nnear ? e0 : last - (e0 - nnear);
            const unsigned n = g.el[e];
            const int i = (int)(n % (unsigned)nx), j = (int)(n / (unsigned)nx);
            const SlotInGrid in = slots_in_grid(i, j, nx, ny);
            T nb[12];
#pragma unroll
            for (int q = 0; q < 12; ++q) nb[q] = in.v[q] ? tf[(int)n + sdj(q) * nx + sdi(q)] : inf;
            const T old = tf[n];
            RegionP<T> R = g.reg[__ldg(g.map + n)];
            if (g.scale != T(1)) {
                R.h *= g.scale;
#pragma unroll
                for (int c = 0; c < 4; ++c) R.fb[c] *= g.scale;
            }
            int rc;
            const T v = local_F<T, VT>(nb, (int)n, nx, R, rc);
            if (g.rec) g.rec[n] = (uint8_t)rc;
            if (!same_bits(v, old)) tf[n] = v;
            g.ov[e] = old;
            g.nv[e] = v;
        }
        evals += ne;
        sweep_sync<CS>();
        // marking: a thread's push decisions first (plain loads), then its dirty-bit test-and-sets (issued
        // independently of one another), then one slot reservation per warp (prefix sum of the counts)
        for (unsigned base = 0; base < ne; base += STRIDE) {
            const unsigned e0 = base + tid;
            const unsigned e = e0 < nnear ? e0 : last - (e0 - nnear);
            unsigned pm = 0u;  // bit q < 12: neighbour q; bit 12: the node itself (seeds later)
            int i = 0, j = 0;
            unsigned n = 0u;
            if (e0 < ne) {
                const T o = g.ov[e];
                const T v = g.nv[e];
                const bool changed = !same_bits(o, v);
                const bool inband = v <= lim;
                n = g.el[e];
                i = (int)(n % (unsigned)nx);
                j = (int)(n / (unsigned)nx);
                if (changed || inband) {
                    const T lo = v < o ? v : o;
                    bool seeds_later = false;
                    const SlotInGrid in = slots_in_grid(i, j, nx, ny);
#pragma unroll
                    for (int q = 0; q < 12; ++q) {
                        if (in.v[q]) {
                            const T tm = tf[(int)n + sdj(q) * nx + sdi(q)];
                            if (!neg_bit(tm)) {
                                bool push = false;
                                if (tm < inf) push = changed && lo <= tm;
                                else if (inband) push = true;
                                else seeds_later = true;
                                pm |= push ? 1u << q : 0u;
                            }
                        }
                    }
                    if (seeds_later && v < inf) pm |= 1u << 12;
                }
                unsigned dup = 0u;
#pragma unroll
                for (int q = 0; q < 13; ++q)
                    if ((pm >> q) & 1u) {
                        const unsigned mnode = q < 12 ? (unsigned)((j + sdj(q)) * nx + (i + sdi(q))) : n;
                        const unsigned bit = 1u << (mnode & 31u);
                        dup |= (atomicOr(g.bm + (mnode >> 5), bit) & bit) ? 1u << q : 0u;
                    }
                pm &= ~dup;
            }
            // warp-inclusive prefix sum of the push counts, one reservation for the warp
            const unsigned cnt = (unsigned)__popc(pm);
            unsigned incl = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
                if ((int)lane >= o) incl += y;
            }
            const unsigned total = __shfl_sync(0xffffffffu, incl, 31);
            unsigned wbase = 0u;
            if (lane == 31u && total != 0u) wbase = atomicAdd(&S.cnt[1], total);
            wbase = __shfl_sync(0xffffffffu, wbase, 31);
            unsigned slot = wbase + incl - cnt;
#pragma unroll
            for (int q = 0; q < 13; ++q)
                if ((pm >> q) & 1u)
                    LB[slot++] = q < 12 ? (unsigned)((j + sdj(q)) * nx + (i + sdi(q))) : n;
        }
        sweep_sync<CS>();
        nact = S.cnt[1];
        sweep_sync<CS>();
        par ^= 1u;
    }
    return true;
}

}  // namespace alf
