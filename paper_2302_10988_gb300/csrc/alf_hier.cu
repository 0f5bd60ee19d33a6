// alf_hier.cu -- the near-source grid hierarchy of Sec. 4.4 on the GPU.
//
// Around each source, levels of relative density d_l cover the squares of
// Chebyshev half-width R_l original cells (clipped to the grid).  Fine nodes
// take the region of the nearest original node (unique for odd d).  On the
// finest level the nodes inside the source's own cell get the straight-ray
// time from the source.  Each level is swept with the local operator F at
// spacing h / d_l to its fixed point (the same warp routine as the field
// sweep); the heap FMM would stop that level as soon as it accepts a node on
// the boundary of its square, and since a heap accepts nodes in key order
// (tau, index) its known set at that moment is exactly the nodes whose key
// does not exceed the smallest key on the boundary.  The known nodes that
// coincide with nodes of the next (coarser) level are frozen there with their
// times; the last level hands them to the original grid, where they become
// the frozen nodes of the field (sign bit set, bit in the field's frozen box).
//
// One warp builds and sweeps all levels of one field; fields come from a
// counter.  Level grids live in a per-warp global scratch, the dirty bitmap
// in shared memory.
#include "alf_internal.h"
#include "alf_sweep.cuh"

namespace alf {

namespace {

// floor(a / d + 1/2) for integers, d > 0 odd: the nearest original node of fine offset a
ALF_D int nearest(int a, int d)
{
    const int num = 2 * a + d, den = 2 * d;
    return num >= 0 ? num / den : -((-num + den - 1) / den);
}

template <typename T>
struct HierScratch {
    T* tcur;
    T* tprev;
    uint32_t* map;
    unsigned* kprev;  // known bitmap of the previous level
    unsigned* list0;
    unsigned* list1;
    unsigned* el;
    T* ov;
    T* nv;
};

template <typename T>
ALF_D HierScratch<T> carve(void* base, size_t L)
{
    // T arrays first (aligned to their size), then the 32-bit arrays and the map
    char* p = (char*)base;
    HierScratch<T> s;
    s.tcur = (T*)p;
    p += L * sizeof(T);
    s.tprev = (T*)p;
    p += L * sizeof(T);
    s.ov = (T*)p;
    p += L * sizeof(T);
    s.nv = (T*)p;
    p += L * sizeof(T);
    s.list0 = (unsigned*)p;
    p += L * 4;
    s.list1 = (unsigned*)p;
    p += L * 4;
    s.el = (unsigned*)p;
    p += L * 4;
    s.kprev = (unsigned*)p;
    p += ((L + 31) / 32) * 4;
    s.map = (uint32_t*)p;
    return s;
}

}  // namespace

size_t hier_scratch_bytes(int precision, size_t L)
{
    const size_t tb = precision == ALF_FP64 ? 8 : 4;
    const size_t bytes = 4 * L * tb + 3 * L * 4 + ((L + 31) / 32) * 4 + L * 4;
    return (bytes + 255) / 256 * 256;
}

template <typename T, bool VT>
__global__ void __launch_bounds__(128) hier_kernel(HierLaunch a)
{
    extern __shared__ unsigned s_hbm[];
    constexpr unsigned FULL = 0xffffffffu;
    const unsigned lane = threadIdx.x & 31u;
    const unsigned wib = threadIdx.x >> 5;
    const unsigned gw = blockIdx.x * (blockDim.x >> 5) + wib;
    if (gw >= (unsigned)a.nwarps) return;
    const size_t L = a.level_cap;
    const HierScratch<T> S = carve<T>((char*)a.scratch + (size_t)gw * a.scratch_stride, L);
    unsigned* bm = s_hbm + (size_t)wib * ((L + 31) / 32);
    const T inf = alf_inf<T>();
    const RegionP<T>* regions = (const RegionP<T>*)a.regions;
    T* tcur = S.tcur;
    T* tprev = S.tprev;
    for (;;) {
        unsigned f = 0u, err = 0u;
        if (lane == 0) {
            f = atomicAdd(a.head, 1u);
            err = *reinterpret_cast<volatile unsigned*>(&a.q->error);
        }
        f = __shfl_sync(FULL, f, 0);
        err = __shfl_sync(FULL, err, 0);
        if (f >= (unsigned)a.nfields || err != 0u) return;
        const FieldDesc fd = a.fields[f];
        const int nx = fd.nx, ny = fd.ny, si = fd.si, sj = fd.sj;
        const uint32_t* omap = a.region_map + fd.map_off;
        const int rsrc = omap[(long long)sj * nx + si];
        const MatD msrc = a.mats[a.region_mat[rsrc]];
        const double th_src = a.theta[(size_t)fd.sample * a.nregions + rsrc];
        const double hb = a.h[fd.sample];
        int pa0 = 0, pb0 = 0, pw = 0, ph = 0, pd = 0;
        for (int l = 0; l <= a.nlev; ++l) {
            const int d = l < a.nlev ? a.dens[l] : 1;
            const int R = l < a.nlev ? a.rad[l] : a.box;
            // level grid: fine offsets [a0, a1] x [b0, b1], clipped to the grid
            const int a0 = max(-R * d, -si * d), a1 = min(R * d, (nx - 1 - si) * d);
            const int b0 = max(-R * d, -sj * d), b1 = min(R * d, (ny - 1 - sj) * d);
            const int w = a1 - a0 + 1, hgt = b1 - b0 + 1, N = w * hgt;
            if (l == a.nlev) {
                // hand the known nodes of the last level to the original grid
                T* tf = (T*)a.times + fd.node_off;
                unsigned* fbits = a.frozen_bits + (size_t)f * frozen_words(a.box);
                for (int n = (int)lane; n < N; n += 32) {
                    const int da = a0 + n % w, db = b0 + n / w;
                    const int qa = da * pd - pa0, qb = db * pd - pb0;
                    if (qa < 0 || qa >= pw || qb < 0 || qb >= ph) continue;
                    const int qn = qb * pw + qa;
                    if (!((S.kprev[qn >> 5] >> (qn & 31)) & 1u)) continue;
                    tf[(long long)(sj + db) * nx + (si + da)] = -abs_(tprev[qn]);
                    const int bw = 2 * a.box + 1, bit = (db + a.box) * bw + (da + a.box);
                    atomicOr(fbits + (bit >> 5), 1u << (bit & 31));
                }
                break;
            }
            // level setup: regions of the nearest original nodes, frozen nodes
            for (int n = (int)lane; n < N; n += 32) {
                const int da = a0 + n % w, db = b0 + n / w;
                S.map[n] = omap[(long long)(sj + nearest(db, d)) * nx + (si + nearest(da, d))];
                T t = inf;
                if (l == 0) {
                    if (2 * abs(da) < d && 2 * abs(db) < d) {
                        double v = 0.0;
                        if (da != 0 || db != 0) {
                            const double dist = sqrt((double)da * da + (double)db * db) * hb / d;
                            v = dist / group_speed64(msrc, a.group_model, atan2((double)db, (double)da) - th_src);
                        }
                        t = -T(v);
                    }
                } else {
                    const int qa = da * (pd / d) - pa0, qb = db * (pd / d) - pb0;
                    if (qa >= 0 && qa < pw && qb >= 0 && qb < ph) {
                        const int qn = qb * pw + qa;
                        if ((S.kprev[qn >> 5] >> (qn & 31)) & 1u) t = -abs_(tprev[qn]);
                    }
                }
                tcur[n] = t;
            }
            __syncwarp();
            WarpGrid<T> g;
            g.tf = tcur;
            g.nx = w;
            g.ny = hgt;
            g.map = S.map;
            g.reg = regions + (size_t)fd.sample * a.nregions;
            g.scale = T(1) / T(d);
            g.list0 = S.list0;
            g.list1 = S.list1;
            g.el = S.el;
            g.ov = S.ov;
            g.nv = S.nv;
            g.rec = nullptr;
            g.bm = bm;
            g.band = a.band_cells > 0.0 ? T(a.band_cells * fd.cell_time / d) : inf;
            g.max_rounds = a.max_rounds_per_node * (unsigned)(w + hgt);
            // first dirty set: the non-frozen nodes around the frozen ones (level 0: the source
            // cell; later levels: the previous level's square)
            const int reach = (l == 0 ? d / 2 : a.rad[l - 1] * d) + 2;
            const unsigned nact = warp_seed_square(g, -a0, -b0, reach);
            unsigned long long evals = 0ull, scanned = 0ull;
            unsigned rounds = 0u;
            if (!warp_sweep<T, VT>(g, nact, evals, rounds, scanned)) {
                if (lane == 0) atomicCAS(&a.q->error, 0u, (unsigned)ALF_ERR_NOT_CONVERGED);
                return;
            }
            // the level stops at the first boundary node in key order: its key bounds the known set
            const int lim = R * d;
            T tbest = inf;
            int ibest = 0x7fffffff;
            for (int n = (int)lane; n < N; n += 32) {
                const int da = a0 + n % w, db = b0 + n / w;
                if (abs(da) < lim && abs(db) < lim) continue;
                const T t = tcur[n];
                if (neg_bit(t) || !(t < inf)) continue;
                if (t < tbest || (t == tbest && n < ibest)) {
                    tbest = t;
                    ibest = n;
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const T ot = __shfl_xor_sync(FULL, tbest, o);
                const int oi = __shfl_xor_sync(FULL, ibest, o);
                if (ot < tbest || (ot == tbest && oi < ibest)) {
                    tbest = ot;
                    ibest = oi;
                }
            }
            // known = frozen, or reached with key <= the boundary key (all reached when no boundary node)
            const unsigned words = (unsigned)((N + 31) / 32);
            for (unsigned wd = 0; wd < words; ++wd) {
                const int n = (int)(wd * 32u + lane);
                bool kn = false;
                if (n < N) {
                    const T t = tcur[n];
                    kn = neg_bit(t) || (t < inf && (t < tbest || (t == tbest && n <= ibest)));
                }
                const unsigned bal = __ballot_sync(FULL, kn);
                if (lane == 0) S.kprev[wd] = bal;
            }
            __syncwarp();
            T* t_ = tprev;
            tprev = tcur;
            tcur = t_;
            pa0 = a0;
            pb0 = b0;
            pw = w;
            ph = hgt;
            pd = d;
        }
        __syncwarp();
    }
}

template <typename T, bool VT>
static cudaError_t hier_t(const HierLaunch& a, cudaStream_t st)
{
    const int wpb = 4;
    const size_t smem = (size_t)wpb * ((a.level_cap + 31) / 32) * sizeof(unsigned);
    if (smem > 48 * 1024) {
        const cudaError_t e =
            cudaFuncSetAttribute(hier_kernel<T, VT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    const int grid = (a.nwarps + wpb - 1) / wpb;
    hier_kernel<T, VT><<<grid, wpb * 32, smem, st>>>(a);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_init_hierarchy(int precision, const HierLaunch& a, cudaStream_t st)
{
    if (a.vtable) return precision == ALF_FP64 ? hier_t<double, true>(a, st) : hier_t<float, true>(a, st);
    return precision == ALF_FP64 ? hier_t<double, false>(a, st) : hier_t<float, false>(a, st);
}

}  // namespace alf
