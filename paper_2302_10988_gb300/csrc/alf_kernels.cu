// alf_kernels.cu -- sm_103a kernels of the forward travel-time solve.
//
//  prep_regions   per (sample, region): c/rho constants, orientation, straight-ray
//                 step times of the fallback (FP64 group->phase inversion)
//  fill_inf       every node of every field := +inf
//  init_radius    frozen straight-ray times around each source (Sec. 4.4)
//  fim_*          bulk-synchronous dirty-set sweep of the local operator F to its
//                 fixed point, all fields of the batch in every round
//  fim_warp       the same sweep with one warp per field, the whole solve in one launch
//  finalize       clears the frozen marks and gathers receiver times
//  check64        FP64 evaluation of F at every node of a solved field
#include <algorithm>
#include <atomic>
#include <cstdio>

#include "alf_internal.h"
#include "alf_sweep.cuh"
#include "alf_check.cuh"

namespace alf {

static std::atomic<unsigned long long> g_launches{0};
void note_launches(unsigned n) { g_launches += n; }
unsigned long long launches_so_far() { return g_launches.load(); }

// ---------------------------------------------------------------------------
// small device helpers
// ---------------------------------------------------------------------------

ALF_D unsigned ld_volatile(const unsigned* p) { return *reinterpret_cast<const volatile unsigned*>(p); }

ALF_D void set_error(QueueState* q, unsigned code) { atomicCAS(&q->error, 0u, code); }


// ---------------------------------------------------------------------------
// prep_regions
// ---------------------------------------------------------------------------
template <typename T>
__global__ void prep_regions_kernel(const MatD* mats, const uint32_t* region_mat, const double* theta, const double* h,
                                    int nsamples, int nregions, int group_model, RegionP<T>* out, const T* vtab)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nsamples * nregions) return;
    const int b = k / nregions, r = k % nregions;
    const MatD m = mats[region_mat[r]];
    const double th = theta[(size_t)b * nregions + r];
    const double hb = h[b];
    RegionP<T> R;
    R.a22 = T(m.a22);
    R.a33 = T(m.a33);
    R.a44 = T(m.a44);
    R.a2344 = T(m.a23 + m.a44);
    double s, c;
    sincos(th, &s, &c);
    R.cth = T(c);
    R.sth = T(s);
    const double kPi = 3.141592653589793;
    const double dirs[4] = {0.0, 0.5 * kPi, 0.25 * kPi, 0.75 * kPi};
    const double lens[4] = {1.0, 1.0, sqrt(2.0), sqrt(2.0)};
    for (int cls = 0; cls < 4; ++cls) {
        R.fb[cls] = T(lens[cls] * hb / group_speed64(m, group_model, dirs[cls] - th));
        const double e = 1e-6;
        R.dfb[cls] = T((lens[cls] * hb / group_speed64(m, group_model, dirs[cls] - th - e) -
                        lens[cls] * hb / group_speed64(m, group_model, dirs[cls] - th + e)) / (2.0 * e));
    }
    R.h = T(hb);
    R.sig = m.sv ? T(-1) : T(1);
    R.iso = m.iso;
    R.pad = 0;
    R.vtab = vtab ? vtab + (size_t)region_mat[r] * ALF_VTAB_N : nullptr;
    out[k] = R;
}

cudaError_t launch_prep_regions(int precision, const MatD* mats, const uint32_t* region_mat, const double* theta,
                                const double* h, int nsamples, int nregions, int group_model, void* regions_out,
                                cudaStream_t st, const void* vtab)
{
    const int n = nsamples * nregions;
    const int bs = 128, gs = (n + bs - 1) / bs;
    if (precision == ALF_FP64)
        prep_regions_kernel<double><<<gs, bs, 0, st>>>(mats, region_mat, theta, h, nsamples, nregions, group_model,
                                                       (RegionP<double>*)regions_out, (const double*)vtab);
    else
        prep_regions_kernel<float><<<gs, bs, 0, st>>>(mats, region_mat, theta, h, nsamples, nregions, group_model,
                                                      (RegionP<float>*)regions_out, (const float*)vtab);
    note_launches(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// fill_inf: 16-byte vector stores, scalar tail
// ---------------------------------------------------------------------------
template <typename T>
__global__ void fill_inf_kernel(T* p, size_t n)
{
    constexpr int V = 16 / sizeof(T);
    const size_t nvec = n / V;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    const T inf = alf_inf<T>();
    uint4 v;
    T* vt = reinterpret_cast<T*>(&v);
#pragma unroll
    for (int k = 0; k < V; ++k) vt[k] = inf;
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < nvec; k += stride)
        reinterpret_cast<uint4*>(p)[k] = v;
    if (blockIdx.x == 0 && threadIdx.x < n - nvec * V) p[nvec * V + threadIdx.x] = inf;
}

int device_sm_count()
{
    static std::atomic<int> cache[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return 1;
    if (dev < 64) {
        const int c = cache[dev].load();
        if (c > 0) return c;
    }
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) return 1;
    if (dev < 64) cache[dev].store(n);
    return n;
}

cudaError_t launch_fill_inf(int precision, void* times, size_t n, cudaStream_t st)
{
    const size_t nvec = n / (precision == ALF_FP64 ? 2 : 4);
    int grid = (int)((nvec + 255) / 256);
    const int cap = device_sm_count() * 16;  // a grid-stride loop over resident blocks
    if (grid > cap) grid = cap;
    if (grid < 1) grid = 1;
    if (precision == ALF_FP64) fill_inf_kernel<double><<<grid, 256, 0, st>>>((double*)times, n);
    else fill_inf_kernel<float><<<grid, 256, 0, st>>>((float*)times, n);
    note_launches(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// env_table: for the shear modes, the group slowness of every material along the angles 0, 1/8, ..., 180
// degrees from its axis, as the support function of its slowness curve, max over phase angles theta of
// cos(theta - psi) / v(theta) (Sec. 7 with Sec. 3.2: the mode's eigenvalue gives v).  One thread per entry:
// 4096 phase angles scanned over (psi - 90, psi + 90] degrees, then a golden-section search in the two scan
// steps around the best.  In FP64, at plan creation.
// ---------------------------------------------------------------------------
__global__ void env_table_kernel(const MatD* mats, int nmat, double* tab)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nmat * ALF_ENV_N) return;
    MatD m = mats[t / ALF_ENV_N];
    m.env = nullptr;
    if (m.iso) {  // the mode is isotropic in this material: the circle 1 / v
        tab[t] = 1.0 / sqrt(m.a22);
        return;
    }
    const double kPi = 3.141592653589793;
    const double psi = (t % ALF_ENV_N) * (kPi / (ALF_ENV_N - 1));
    auto g = [&](double th) {
        double sn, cs;
        sincos(th, &sn, &cs);
        return cos(th - psi) * rsqrt(qp_lambda64(m, cs, sn));
    };
    constexpr int NS = 4096;
    const double step = kPi / NS;
    double best = -1.0, bt = psi;
    for (int j = 1; j <= NS; ++j) {
        const double th = psi - 0.5 * kPi + j * step, v = g(th);
        if (v > best) {
            best = v;
            bt = th;
        }
    }
    double lo = bt - step, hi = bt + step;
    const double r = 0.6180339887498949;
    double x1 = hi - r * (hi - lo), x2 = lo + r * (hi - lo), g1 = g(x1), g2 = g(x2);
    for (int it = 0; it < 90; ++it) {
        if (g1 < g2) {
            lo = x1;
            x1 = x2;
            g1 = g2;
            x2 = lo + r * (hi - lo);
            g2 = g(x2);
        } else {
            hi = x2;
            x2 = x1;
            g2 = g1;
            x1 = hi - r * (hi - lo);
            g1 = g(x1);
        }
    }
    tab[t] = fmax(best, fmax(g1, g2));
}

cudaError_t launch_env_table(const MatD* mats, int nmat, double* tab, cudaStream_t st)
{
    const int n = nmat * ALF_ENV_N;
    env_table_kernel<<<(n + 127) / 128, 128, 0, st>>>(mats, nmat, tab);
    note_launches(1);
    return cudaGetLastError();
}

__global__ void set_status_kernel(QueueState* q, unsigned code) { set_error(q, code); }

cudaError_t launch_set_status(QueueState* q, unsigned code, cudaStream_t st)
{
    set_status_kernel<<<1, 1, 0, st>>>(q, code);
    note_launches(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// init_radius: one block per field; frozen nodes store -tau (sign bit = frozen)
// ---------------------------------------------------------------------------
template <typename T>
__global__ void init_radius_kernel(T* times, const FieldDesc* fields, const uint32_t* region_map,
                                   const uint32_t* region_mat, const MatD* mats, const double* theta, const double* h,
                                   int nregions, int r0, int group_model, unsigned* frozen_bits, int box)
{
    const FieldDesc fd = fields[blockIdx.x];
    const int si = fd.si, sj = fd.sj;
    const int rsrc = region_map[fd.map_off + (long long)sj * fd.nx + si];
    const MatD m = mats[region_mat[rsrc]];
    const double th = theta[(size_t)fd.sample * nregions + rsrc];
    const double hb = h[fd.sample];
    const int w = 2 * r0 + 1;
    for (int k = threadIdx.x; k < w * w; k += blockDim.x) {
        const int di = k % w - r0, dj = k / w - r0;
        const int i = si + di, j = sj + dj;
        if (i < 0 || j < 0 || i >= fd.nx || j >= fd.ny) continue;
        double t = 0.0;
        if (di != 0 || dj != 0) {
            const double dist = sqrt((double)(di * di + dj * dj)) * hb;
            t = dist / group_speed64(m, group_model, atan2((double)dj, (double)di) - th);
        }
        times[fd.node_off + (long long)j * fd.nx + i] = -T(t);
        const int bw = 2 * box + 1, bit = (dj + box) * bw + (di + box);
        atomicOr(frozen_bits + (size_t)blockIdx.x * frozen_words(box) + (bit >> 5), 1u << (bit & 31));
    }
}

cudaError_t launch_init_radius(int precision, void* times, const FieldDesc* fields, int nfields,
                               const uint32_t* region_map, const uint32_t* region_mat, const MatD* mats,
                               const double* theta, const double* h, int nregions, int r0, int group_model,
                               unsigned* frozen_bits, int box, cudaStream_t st)
{
    if (precision == ALF_FP64)
        init_radius_kernel<double><<<nfields, 128, 0, st>>>((double*)times, fields, region_map, region_mat, mats,
                                                            theta, h, nregions, r0, group_model, frozen_bits, box);
    else
        init_radius_kernel<float><<<nfields, 128, 0, st>>>((float*)times, fields, region_map, region_mat, mats, theta,
                                                           h, nregions, r0, group_model, frozen_bits, box);
    note_launches(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// fim: bulk-synchronous dirty-set sweep over all fields at once
// ---------------------------------------------------------------------------
// Every field keeps its dirty set -- nodes that may not be at the fixed point
// of F -- as a list (segment of the packed lists at the field's node offset)
// and a bitmap, so that a node is listed at most once.  A round is four
// launches over all fields:
//   prep   one warp per field: T = the smallest time in the dirty set; the
//          nodes that are unknown (+inf) or not later than T + band move to
//          the field's evaluation list (bitmap bit cleared); later nodes stay
//          dirty for the next round (they wait for the front, so that they
//          are not re-evaluated for every transient change upwind -- the band
//          keeps the sweep close to the heap's order with a whole band of the
//          front in flight);
//   scan   exclusive scan of the evaluation-list sizes (one flat index space);
//   eval   one thread per listed node of every field: F, time written in
//          place, old and new time kept for the marking step;
//   mark   for every changed node n, every known non-frozen diamond
//          neighbour m whose time can depend on n -- m not earlier than n's
//          old or new time (F at m only reads the neighbours that precede m in
//          key order) -- is marked dirty for the next round; unknown
//          neighbours are marked (for their first evaluation) only by a node
//          whose time is inside the band, and a node outside the band with
//          unknown neighbours marks itself, to seed them once the front
//          arrives.  This keeps the dirty sets a thin shell around the front.
// The marking runs after all writes of the round, so it compares against
// written times.  A field is at the fixed point of F when its dirty set is
// empty.  Frozen nodes carry the sign bit and are never listed.
// first dirty set of every field: the non-frozen nodes around the frozen box
template <typename T>
__global__ void fim_init_kernel(FimLaunch a)
{
    const unsigned lane = threadIdx.x & 31u;
    const size_t nw = (size_t)gridDim.x * blockDim.x / 32;
    for (size_t f = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) / 32; f < (size_t)a.nfields; f += nw) {
        const FieldDesc fd = a.fields[f];
        const int nx = fd.nx, ny = fd.ny;
        const T* tf = (const T*)a.times + fd.node_off;
        unsigned* bm = a.bitmap + a.bm_off[f];
        unsigned* list = a.list[0] + fd.node_off;
        const unsigned words = (unsigned)((nx * ny + 31) / 32);
        for (unsigned w = lane; w < words; w += 32u) bm[w] = 0u;
        __syncwarp();
        const int r = a.box + 2, w = 2 * r + 1;
        unsigned cnt = 0;
        for (int base = 0; base < w * w; base += 32) {
            const int k = base + (int)lane;
            bool take = false;
            unsigned n = 0;
            if (k < w * w) {
                const int i = fd.si + k % w - r, j = fd.sj + k / w - r;
                if (i >= 0 && j >= 0 && i < nx && j < ny) {
                    n = (unsigned)(j * nx + i);
                    take = !neg_bit(__ldcg(tf + n));
                }
            }
            const unsigned bal = __ballot_sync(0xffffffffu, take);
            if (take) {
                list[cnt + __popc(bal & ((1u << lane) - 1u))] = n;
                atomicOr(bm + (n >> 5), 1u << (n & 31u));
            }
            cnt += __popc(bal);
        }
        if (lane == 0) {
            a.cnt[f] = cnt;
            a.cnt[a.nfields + f] = 0u;
            a.rounds[f] = 0u;
        }
    }
}

template <typename T>
__global__ void fim_prep_kernel(FimLaunch a, int parity)
{
    const unsigned lane = threadIdx.x & 31u;
    const size_t nw = (size_t)gridDim.x * blockDim.x / 32;
    unsigned* cur_cnt = a.cnt + (size_t)parity * a.nfields;
    unsigned* nxt_cnt = a.cnt + (size_t)(parity ^ 1) * a.nfields;
    unsigned long long pending = 0;
    for (size_t f = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) / 32; f < (size_t)a.nfields; f += nw) {
        const unsigned nact = cur_cnt[f];
        const FieldDesc fd = a.fields[f];
        if (nact == 0u || a.rounds[f] >= a.max_rounds_per_node * (unsigned)(fd.nx + fd.ny)) {
            if (lane == 0) {
                if (nact != 0u) set_error(a.q, ALF_ERR_NOT_CONVERGED);  // livelock guard: the field is abandoned
                a.ecnt[f] = 0u;
                nxt_cnt[f] = 0u;
            }
            continue;
        }
        const T* tf = (const T*)a.times + fd.node_off;
        const unsigned* listA = a.list[parity] + fd.node_off;
        unsigned* listB = a.list[parity ^ 1] + fd.node_off;
        unsigned* el = a.elist + fd.node_off;
        unsigned* bm = a.bitmap + a.bm_off[f];
        auto m = order_key(alf_inf<T>());
        for (unsigned k = lane; k < nact; k += 32u) {
            const auto v = order_key(__ldcg(tf + listA[k]));
            m = v < m ? v : m;
        }
        const T band = a.band_cells > 0.0 ? T(a.band_cells * fd.cell_time) : alf_inf<T>();
        const T lim = from_key(warp_min(m), T(0)) + band;
        unsigned ne = 0, nc = 0;
        for (unsigned base = 0; base < nact; base += 32u) {
            const unsigned k = base + lane;
            bool in = k < nact, ev = false;
            unsigned n = 0;
            if (in) {
                n = listA[k];
                const T t = __ldcg(tf + n);
                ev = t <= lim || !(t < alf_inf<T>());
            }
            const unsigned be = __ballot_sync(0xffffffffu, in && ev), bc = __ballot_sync(0xffffffffu, in && !ev);
            const unsigned below = (1u << lane) - 1u;
            if (in && ev) {
                el[ne + __popc(be & below)] = n;
                atomicAnd(bm + (n >> 5), ~(1u << (n & 31u)));
            } else if (in) {
                listB[nc + __popc(bc & below)] = n;
            }
            ne += __popc(be);
            nc += __popc(bc);
        }
        if (lane == 0) {
            a.ecnt[f] = ne;
            nxt_cnt[f] = nc;
            a.rounds[f] += 1u;
            ((T*)a.flim)[f] = lim;
        }
        pending += nact;
    }
    (void)pending;
}

// exclusive scan of the per-field evaluation counts (one block)
__global__ void fim_scan_kernel(FimLaunch a)
{
    __shared__ unsigned s[1024];
    const int n = a.nfields;
    const int per = (n + 1023) / 1024;
    const int b0 = threadIdx.x * per, b1 = min(n, b0 + per);
    unsigned sum = 0;
    for (int f = b0; f < b1; ++f) sum += a.ecnt[f];
    s[threadIdx.x] = sum;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        const unsigned v = threadIdx.x >= (unsigned)o ? s[threadIdx.x - o] : 0u;
        __syncthreads();
        s[threadIdx.x] += v;
        __syncthreads();
    }
    unsigned run = s[threadIdx.x] - sum;
    for (int f = b0; f < b1; ++f) {
        a.eoff[f] = run;
        run += a.ecnt[f];
    }
    if (threadIdx.x == 1023) {
        a.eoff[n] = s[1023];
        if (s[1023]) atomicAdd(&a.q->visits, (unsigned long long)s[1023]);
    }
}

ALF_D int field_of(const unsigned* eoff, int nfields, unsigned e)
{
    int lo = 0, hi = nfields;  // largest f with eoff[f] <= e
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(eoff + mid) <= e) lo = mid; else hi = mid;
    }
    return lo;
}

template <typename T, int NT, bool VT>
__global__ void __launch_bounds__(NT) fim_eval_kernel(FimLaunch a)
{
    const unsigned E = a.eoff[a.nfields];
    T* times = (T*)a.times;
    T* oldv = (T*)a.oldv;
    T* newv = (T*)a.newv;
    const RegionP<T>* regions = (const RegionP<T>*)a.regions;
    const unsigned stride = gridDim.x * blockDim.x;
    for (unsigned e = blockIdx.x * blockDim.x + threadIdx.x; e < E; e += stride) {
        const int f = field_of(a.eoff, a.nfields, e);
        const FieldDesc fd = a.fields[f];
        const int nx = fd.nx, ny = fd.ny;
        T* tf = times + fd.node_off;
        const unsigned n = a.elist[fd.node_off + (e - a.eoff[f])];
        const int i = (int)(n % (unsigned)nx), j = (int)(n / (unsigned)nx);
        T nb[12];
#pragma unroll
        for (int q = 0; q < 12; ++q) {
            const int ii = i + sdi(q), jj = j + sdj(q);
            nb[q] = (ii >= 0 && jj >= 0 && ii < nx && jj < ny) ? __ldcg(tf + jj * nx + ii) : alf_inf<T>();
        }
        const T old = __ldcg(tf + n);
        const RegionP<T> R = regions[(size_t)fd.sample * a.nregions + __ldg(a.region_map + fd.map_off + n)];
        int rec;
        const T v = local_F<T, VT>(nb, (int)n, nx, R, rec);
        if (a.records) a.records[fd.node_off + n] = (uint8_t)rec;
        if (!same_bits(v, old)) __stcg(tf + n, v);
        oldv[e] = old;
        newv[e] = v;
        a.efield[e] = (unsigned)f;
    }
}

template <typename T>
__global__ void fim_mark_kernel(FimLaunch a, int parity)
{
    const unsigned E = a.eoff[a.nfields];
    const T* times = (const T*)a.times;
    const T* oldv = (const T*)a.oldv;
    const T* newv = (const T*)a.newv;
    const T* flim = (const T*)a.flim;
    unsigned* nxt_cnt = a.cnt + (size_t)(parity ^ 1) * a.nfields;
    const unsigned stride = gridDim.x * blockDim.x;
    for (unsigned e = blockIdx.x * blockDim.x + threadIdx.x; e < E; e += stride) {
        const T o = oldv[e], v = newv[e];
        const unsigned f = a.efield[e];
        const bool changed = !same_bits(o, v);
        const bool inband = v <= flim[f];
        if (!changed && !inband) continue;
        const FieldDesc fd = a.fields[f];
        const int nx = fd.nx, ny = fd.ny;
        const T* tf = times + fd.node_off;
        const unsigned n = a.elist[fd.node_off + (e - a.eoff[f])];
        const int i = (int)(n % (unsigned)nx), j = (int)(n / (unsigned)nx);
        const T lo = v < o ? v : o;
        unsigned* bm = a.bitmap + a.bm_off[f];
        unsigned* listB = a.list[parity ^ 1] + fd.node_off;
        auto push = [&](unsigned m) {
            const unsigned bit = 1u << (m & 31u);
            if (!(atomicOr(bm + (m >> 5), bit) & bit)) listB[atomicAdd(nxt_cnt + f, 1u)] = m;
        };
        bool seeds_later = false;
#pragma unroll
        for (int q = 0; q < 12; ++q) {
            const int ii = i + sdi(q), jj = j + sdj(q);
            if (ii < 0 || jj < 0 || ii >= nx || jj >= ny) continue;
            const unsigned m = (unsigned)(jj * nx + ii);
            const T tm = __ldcg(tf + m);
            if (neg_bit(tm)) continue;  // frozen
            if (tm < alf_inf<T>()) {
                if (changed && lo <= tm) push(m);
            } else if (inband) {
                push(m);             // first evaluation of an unknown neighbour
            } else {
                seeds_later = true;  // it is seeded when this node is in the band
            }
        }
        if (seeds_later && v < alf_inf<T>()) push(n);
    }
}

// work left after the last round: sum of the next-list sizes
__global__ void fim_pending_kernel(FimLaunch a, int parity, unsigned long long* out)
{
    const unsigned* c = a.cnt + (size_t)parity * a.nfields;
    unsigned long long s = 0;
    for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < a.nfields; f += gridDim.x * blockDim.x) s += c[f];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0 && s) atomicAdd(out, s);
}

// ---------------------------------------------------------------------------
// Field-resident sweep: one warp owns one field from its first dirty set to
// its fixed point.  Each round is the same sequence as the bulk-synchronous
// steps above -- front time T over the dirty set, the nodes within the band
// split off and evaluated, then the marking rule -- with warp barriers between
// the steps instead of kernel boundaries, and the field's dirty bitmap in
// shared memory.  Warps take fields from a queue ordered by decreasing size.
// All reads and writes of a field's times come from the one warp that owns it,
// so plain (L1-cached) loads see every update after the warp barrier.  The
// same routine sweeps the finer grids of the near-source hierarchy (spacing
// h / d, `scale` = 1 / d).
// ---------------------------------------------------------------------------
// FP32: registers capped so that four 4-warp CTAs fit an SM (what the shared bitmaps of 320 x 320 fields allow)
template <typename T, int NW, bool VT>
__global__ void __launch_bounds__(NW * 32, sizeof(T) == 4 ? 4 : 1)
    fim_warp_kernel(FimLaunch a, const unsigned* order, unsigned words_per_warp)
{
    extern __shared__ unsigned s_bm[];
    constexpr unsigned FULL = 0xffffffffu;
    const unsigned lane = threadIdx.x & 31u;
    const T inf = alf_inf<T>();
    for (;;) {
        unsigned fi = 0u, err = 0u;
        if (lane == 0) {
            fi = atomicAdd(&a.q->head, 1u);
            err = ld_volatile(&a.q->error);
        }
        fi = __shfl_sync(FULL, fi, 0);
        err = __shfl_sync(FULL, err, 0);
        if (fi >= (unsigned)a.nfields || err != 0u) return;
        const unsigned f = __ldg(order + fi);
        const FieldDesc fd = a.fields[f];
        WarpGrid<T> g;
        g.tf = (T*)a.times + fd.node_off;
        g.nx = fd.nx;
        g.ny = fd.ny;
        g.map = a.region_map + fd.map_off;
        g.reg = (const RegionP<T>*)a.regions + (size_t)fd.sample * a.nregions;
        g.scale = T(1);
        g.list0 = a.list[0] + fd.node_off;
        g.list1 = a.list[1] + fd.node_off;
        g.el = a.elist + fd.node_off;
        g.ov = (T*)a.oldv + fd.node_off;
        g.nv = (T*)a.newv + fd.node_off;
        g.rec = a.records ? a.records + fd.node_off : nullptr;
        g.bm = s_bm + (size_t)(threadIdx.x >> 5) * words_per_warp;
        g.band = a.band_cells > 0.0 ? T(a.band_cells * fd.cell_time) : inf;
        g.max_rounds = a.max_rounds_per_node * (unsigned)(fd.nx + fd.ny);
        // first dirty set: the non-frozen nodes of the square around the frozen box
        const unsigned nact = warp_seed_square(g, fd.si, fd.sj, a.box + 2);
        unsigned long long evals = 0ull, scanned = 0ull;
        unsigned rounds = 0u;
        const bool ok = warp_sweep<T, VT>(g, nact, evals, rounds, scanned);
        if (lane == 0) {
            if (!ok) set_error(a.q, ALF_ERR_NOT_CONVERGED);
            a.rounds[f] = rounds;
            atomicAdd(&a.q->visits, evals);
            atomicAdd(&a.q->dirty, scanned);
            atomicMax(&a.q->rounds, (unsigned long long)rounds);
        }
        __syncwarp();
    }
}

// Field-resident sweep by a whole CTA (few large fields), or by a cluster of CS CTAs on CS SMs (fewer fields
// than SMs): the same rounds, barriers between the steps.  The dirty bitmap is in shared memory (rank 0's)
// when the field's fits, else in the field's global bitmap.  Rank 0 takes the fields from the queue.
// CHK: once a field is solved, the same CTA runs the FP64 check of every node of it (the field is then still
// in L1/L2, and its FP64 work overlaps the ALU-bound sweep of the fields on the other CTAs of the SM).
template <typename T, int NT, bool VT, int CS, bool CHK = false>
__global__ void __launch_bounds__(NT, sizeof(T) == 4 ? 512 / NT : 1)
    fim_cta_kernel(FimLaunch a, const unsigned* order, unsigned smem_words)
{
    extern __shared__ unsigned s_cbm[];
    __shared__ CtaSweepShared sh;
    __shared__ unsigned s_f[2];  // field index, error code
    const T inf = alf_inf<T>();
    const unsigned rank = cluster_rank<CS>();
    CtaSweepShared& S = CS == 1 ? sh : *map_rank(&sh, 0u);
    const volatile unsigned* const f0 = CS == 1 ? s_f : map_rank(s_f, 0u);
    unsigned* const bm0 = CS == 1 ? s_cbm : map_rank(s_cbm, 0u);
    for (;;) {
        if (rank == 0 && threadIdx.x == 0) {
            s_f[0] = atomicAdd(&a.q->head, 1u);
            s_f[1] = ld_volatile(&a.q->error);
        }
        sweep_sync<CS>();
        const unsigned fi = f0[0], err = f0[1];
        sweep_sync<CS>();
        if (fi >= (unsigned)a.nfields || err != 0u) return;
        const unsigned f = __ldg(order + fi);
        const FieldDesc fd = a.fields[f];
        WarpGrid<T> g;
        g.tf = (T*)a.times + fd.node_off;
        g.nx = fd.nx;
        g.ny = fd.ny;
        g.map = a.region_map + fd.map_off;
        g.reg = (const RegionP<T>*)a.regions + (size_t)fd.sample * a.nregions;
        g.scale = T(1);
        g.list0 = a.list[0] + fd.node_off;
        g.list1 = a.list[1] + fd.node_off;
        g.el = a.elist + fd.node_off;
        g.ov = (T*)a.oldv + fd.node_off;
        g.nv = (T*)a.newv + fd.node_off;
        g.rec = a.records ? a.records + fd.node_off : nullptr;
        const unsigned words = (unsigned)((fd.nx * fd.ny + 31) / 32);
        g.bm = words <= smem_words ? bm0 : a.bitmap + a.bm_off[f];
        g.band = a.band_cells > 0.0 ? T(a.band_cells * fd.cell_time) : inf;
        g.max_rounds = a.max_rounds_per_node * (unsigned)(fd.nx + fd.ny);
        const unsigned nact = cta_seed_square<T, NT, CS>(g, fd.si, fd.sj, a.box + 2, S);
        unsigned long long evals = 0ull, scanned = 0ull;
        unsigned rounds = 0u;
        const bool ok = cta_sweep<T, NT, VT, CS>(g, nact, evals, rounds, S, scanned);
        if (rank == 0 && threadIdx.x == 0) {
            if (!ok) set_error(a.q, ALF_ERR_NOT_CONVERGED);
            a.rounds[f] = rounds;
            atomicAdd(&a.q->visits, evals);
            atomicAdd(&a.q->dirty, scanned);
            atomicMax(&a.q->rounds, (unsigned long long)rounds);
        }
        sweep_sync<CS>();
        if constexpr (CHK) {
            // the FP64 check of the field (as check64_kernel): largest relative residual, records that differ
            const unsigned* fb = a.frozen_bits + (size_t)f * frozen_words(a.box);
            const RegionP<double>* r64 = (const RegionP<double>*)a.regions64 + (size_t)fd.sample * a.nregions;
            float mx = 0.f;
            int flips = 0;
            for (int me = (int)(rank * NT + threadIdx.x); me < fd.nx * fd.ny; me += NT * CS) {
                double F;
                int rec;
                T tme;
                if (!check_node<T, VT>(g.tf, fb, a.box, fd, me, r64, g.map, F, rec, tme)) continue;
                const float res = fabsf((float)(F - (double)tme)) / (float)tme;
                if (tme > T(0)) mx = fmaxf(mx, res);
                if (g.rec && g.rec[me] != (uint8_t)rec) flips++;
            }
            for (int o = 16; o > 0; o >>= 1) {
                mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
                flips += __shfl_xor_sync(0xffffffffu, flips, o);
            }
            if ((threadIdx.x & 31u) == 0u) {
                // max of non-negative doubles through their bit patterns
                if (mx > 0.f)
                    atomicMax((unsigned long long*)(a.max_rel + f), (unsigned long long)__double_as_longlong((double)mx));
                if (flips) atomicAdd(a.n_flips + f, flips);
            }
        }
    }
}

// CTA sizes of the CTA-per-field sweep: 64, 128, 256 or 512 threads (2 to 16 warps on one field).  Fewer
// warps per field put more fields on an SM at once; more warps finish a large field sooner (512: a whole
// SM's FP32 register file for one field, for batches with no more fields than SMs).  Clusters of 2, 4 or 8
// 512-thread CTAs spread one field over as many SMs.
template <typename T, int NT, bool VT, int CS, bool CHK = false>
static cudaError_t fim_cta_smem(unsigned smem_words, size_t* smem)
{
    *smem = (size_t)smem_words * sizeof(unsigned);
    if (*smem <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(fim_cta_kernel<T, NT, VT, CS, CHK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)*smem);
}

// launch configuration of a cluster launch: nt threads per CTA, clusters of cs CTAs along x
static cudaLaunchConfig_t cta_config(int grid, int nt, int cs, size_t smem, cudaStream_t st, cudaLaunchAttribute* attr)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)nt);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

template <typename T, int NT, bool VT, int CS, bool CHK = false>
static cudaError_t fim_cta_t(const FimLaunch& a, const unsigned* order, unsigned smem_words, int grid,
                             cudaStream_t st)
{
    size_t smem = 0;
    cudaError_t e = fim_cta_smem<T, NT, VT, CS, CHK>(smem_words, &smem);
    if (e != cudaSuccess) return e;
    if constexpr (CS == 1) {
        fim_cta_kernel<T, NT, VT, 1, CHK><<<grid, NT, smem, st>>>(a, order, smem_words);
        e = cudaGetLastError();
    } else {
        cudaLaunchAttribute attr[1];
        const cudaLaunchConfig_t cfg = cta_config(grid, NT, CS, smem, st, attr);
        e = cudaLaunchKernelEx(&cfg, fim_cta_kernel<T, NT, VT, CS>, a, order, smem_words);
    }
    note_launches(1);
    return e;
}

template <typename T, bool VT>
static cudaError_t fim_cta_nt(const FimLaunch& a, const unsigned* order, unsigned smem_words, int grid, int nt,
                              int cs, cudaStream_t st)
{
    if (cs == 1) {
        switch (nt) {
        case 64: return fim_cta_t<T, 64, VT, 1>(a, order, smem_words, grid, st);
        case 128: return fim_cta_t<T, 128, VT, 1>(a, order, smem_words, grid, st);
        case 256: return fim_cta_t<T, 256, VT, 1>(a, order, smem_words, grid, st);
        case 512: return fim_cta_t<T, 512, VT, 1>(a, order, smem_words, grid, st);
        default: return cudaErrorInvalidValue;
        }
    }
    if (nt != 512) return cudaErrorInvalidValue;
    switch (cs) {
    case 2: return fim_cta_t<T, 512, VT, 2>(a, order, smem_words, grid, st);
    case 4: return fim_cta_t<T, 512, VT, 4>(a, order, smem_words, grid, st);
    case 8: return fim_cta_t<T, 512, VT, 8>(a, order, smem_words, grid, st);
    default: return cudaErrorInvalidValue;
    }
}

bool fim_cta_can_check(int precision, int vtable, int cluster)
{
    return precision == ALF_FP32 && !vtable && cluster == 1;
}

cudaError_t launch_fim_cta(int precision, const FimLaunch& a, const unsigned* order, unsigned smem_words, int grid,
                           int threads, int cluster, cudaStream_t st, bool check)
{
    if (check) {
        // the sweep with each field's FP64 check (FP32 fields, run-time Christoffel solve, one CTA per field)
        if (!fim_cta_can_check(precision, a.vtable, cluster)) return cudaErrorInvalidValue;
        switch (threads) {
        case 64: return fim_cta_t<float, 64, false, 1, true>(a, order, smem_words, grid, st);
        case 128: return fim_cta_t<float, 128, false, 1, true>(a, order, smem_words, grid, st);
        case 256: return fim_cta_t<float, 256, false, 1, true>(a, order, smem_words, grid, st);
        case 512: return fim_cta_t<float, 512, false, 1, true>(a, order, smem_words, grid, st);
        default: return cudaErrorInvalidValue;
        }
    }
    if (a.vtable)
        return precision == ALF_FP64 ? fim_cta_nt<double, true>(a, order, smem_words, grid, threads, cluster, st)
                                     : fim_cta_nt<float, true>(a, order, smem_words, grid, threads, cluster, st);
    return precision == ALF_FP64 ? fim_cta_nt<double, false>(a, order, smem_words, grid, threads, cluster, st)
                                 : fim_cta_nt<float, false>(a, order, smem_words, grid, threads, cluster, st);
}

// grid of the CTA-per-field sweep in CTAs: as many CTAs (clusters) as are resident at once; 0: does not fit
template <typename T, int NT, bool VT, int CS>
static int fim_cta_occ(unsigned smem_words, int nsm)
{
    size_t smem = 0;
    if (fim_cta_smem<T, NT, VT, CS>(smem_words, &smem) != cudaSuccess) return 0;
    int n = 0;
    if constexpr (CS == 1) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fim_cta_kernel<T, NT, VT, 1>, NT, smem) != cudaSuccess)
            return 0;
        return n * nsm;
    } else {
        cudaLaunchAttribute attr[1];
        const cudaLaunchConfig_t cfg = cta_config(CS * nsm, NT, CS, smem, nullptr, attr);
        if (cudaOccupancyMaxActiveClusters(&n, fim_cta_kernel<T, NT, VT, CS>, &cfg) != cudaSuccess) return 0;
        return n * CS;
    }
}

template <typename T, bool VT>
static int fim_cta_occ_nt(unsigned smem_words, int nt, int cs, int nsm)
{
    if (cs == 1) {
        switch (nt) {
        case 64: return fim_cta_occ<T, 64, VT, 1>(smem_words, nsm);
        case 128: return fim_cta_occ<T, 128, VT, 1>(smem_words, nsm);
        case 256: return fim_cta_occ<T, 256, VT, 1>(smem_words, nsm);
        case 512: return fim_cta_occ<T, 512, VT, 1>(smem_words, nsm);
        default: return 0;
        }
    }
    if (nt != 512) return 0;
    switch (cs) {
    case 2: return fim_cta_occ<T, 512, VT, 2>(smem_words, nsm);
    case 4: return fim_cta_occ<T, 512, VT, 4>(smem_words, nsm);
    case 8: return fim_cta_occ<T, 512, VT, 8>(smem_words, nsm);
    default: return 0;
    }
}

int fim_cta_grid(int precision, unsigned smem_words, bool vt, int threads, int cluster, int nsm)
{
    if (vt)
        return precision == ALF_FP64 ? fim_cta_occ_nt<double, true>(smem_words, threads, cluster, nsm)
                                     : fim_cta_occ_nt<float, true>(smem_words, threads, cluster, nsm);
    return precision == ALF_FP64 ? fim_cta_occ_nt<double, false>(smem_words, threads, cluster, nsm)
                                 : fim_cta_occ_nt<float, false>(smem_words, threads, cluster, nsm);
}

// dynamic shared memory of the field-resident sweep: one dirty bitmap per warp
template <typename T, bool VT>
static cudaError_t fim_warp_smem(unsigned words_per_warp, size_t* smem)
{
    *smem = (size_t)ALF_SWEEP_WARPS * words_per_warp * sizeof(unsigned);
    if (*smem <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(fim_warp_kernel<T, ALF_SWEEP_WARPS, VT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)*smem);
}

template <typename T, bool VT>
static cudaError_t fim_warp_t(const FimLaunch& a, const unsigned* order, unsigned words_per_warp, int grid,
                              cudaStream_t st)
{
    size_t smem = 0;
    cudaError_t e = fim_warp_smem<T, VT>(words_per_warp, &smem);
    if (e != cudaSuccess) return e;
    fim_warp_kernel<T, ALF_SWEEP_WARPS, VT><<<grid, ALF_SWEEP_WARPS * 32, smem, st>>>(a, order, words_per_warp);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_fim_warp(int precision, const FimLaunch& a, const unsigned* order, unsigned words_per_warp,
                            int grid, cudaStream_t st)
{
    if (a.vtable)
        return precision == ALF_FP64 ? fim_warp_t<double, true>(a, order, words_per_warp, grid, st)
                                     : fim_warp_t<float, true>(a, order, words_per_warp, grid, st);
    return precision == ALF_FP64 ? fim_warp_t<double, false>(a, order, words_per_warp, grid, st)
                                 : fim_warp_t<float, false>(a, order, words_per_warp, grid, st);
}

template <typename T, bool VT>
static int fim_warp_occ(unsigned words_per_warp)
{
    size_t smem = 0;
    if (fim_warp_smem<T, VT>(words_per_warp, &smem) != cudaSuccess) return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fim_warp_kernel<T, ALF_SWEEP_WARPS, VT>, ALF_SWEEP_WARPS * 32,
                                                      smem) != cudaSuccess)
        return 0;
    return n;
}

int fim_warp_ctas_per_sm(int precision, unsigned words_per_warp, bool vt)
{
    if (vt)
        return precision == ALF_FP64 ? fim_warp_occ<double, true>(words_per_warp) : fim_warp_occ<float, true>(words_per_warp);
    return precision == ALF_FP64 ? fim_warp_occ<double, false>(words_per_warp) : fim_warp_occ<float, false>(words_per_warp);
}

template <typename T>
static cudaError_t fim_round_t(const FimLaunch& a, int parity, int grid_fields, int grid_eval, int eval_block,
                               cudaEvent_t ev0, cudaEvent_t ev1, cudaStream_t st)
{
    fim_prep_kernel<T><<<grid_fields, 256, 0, st>>>(a, parity);
    fim_scan_kernel<<<1, 1024, 0, st>>>(a);
    if (ev0) cudaEventRecord(ev0, st);
    if (a.vtable) {
        if (eval_block == 256) fim_eval_kernel<T, 256, true><<<grid_eval / 2, 256, 0, st>>>(a);
        else fim_eval_kernel<T, 128, true><<<grid_eval, 128, 0, st>>>(a);
    } else {
        if (eval_block == 256) fim_eval_kernel<T, 256, false><<<grid_eval / 2, 256, 0, st>>>(a);
        else fim_eval_kernel<T, 128, false><<<grid_eval, 128, 0, st>>>(a);
    }
    if (ev1) cudaEventRecord(ev1, st);
    fim_mark_kernel<T><<<grid_eval, 256, 0, st>>>(a, parity);
    note_launches(4);
    return cudaGetLastError();
}

cudaError_t launch_fim_init(int precision, const FimLaunch& a, int grid_fields, cudaStream_t st)
{
    if (precision == ALF_FP64) fim_init_kernel<double><<<grid_fields, 256, 0, st>>>(a);
    else fim_init_kernel<float><<<grid_fields, 256, 0, st>>>(a);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_fim_round(int precision, const FimLaunch& a, int parity, int grid_fields, int grid_eval,
                             cudaStream_t st, int eval_block, cudaEvent_t ev0, cudaEvent_t ev1)
{
    return precision == ALF_FP64 ? fim_round_t<double>(a, parity, grid_fields, grid_eval, eval_block, ev0, ev1, st)
                                 : fim_round_t<float>(a, parity, grid_fields, grid_eval, eval_block, ev0, ev1, st);
}

cudaError_t launch_fim_pending(const FimLaunch& a, int parity, unsigned long long* out, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    fim_pending_kernel<<<64, 256, 0, st>>>(a, parity, out);
    note_launches(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// finalize: frozen marks cleared (box around each source), receiver times
// ---------------------------------------------------------------------------
template <typename T>
__global__ void finalize_kernel(T* times, const FieldDesc* fields, int box, const int32_t* rec_ij, int nsrc, int nrec,
                                T* rec_times, uint8_t* records)
{
    const int f = blockIdx.x;
    const FieldDesc fd = fields[f];
    const int w = 2 * box + 1;
    T* tf = times + fd.node_off;
    for (int k = threadIdx.x; k < w * w; k += blockDim.x) {
        const int i = fd.si + k % w - box, j = fd.sj + k / w - box;
        if (i < 0 || j < 0 || i >= fd.nx || j >= fd.ny) continue;
        T* p = tf + (long long)j * fd.nx + i;
        if (records && neg_bit(*p)) records[fd.node_off + (long long)j * fd.nx + i] = 254;
        *p = abs_(*p);
    }
    __syncthreads();
    if (rec_times) {
        const int b = fd.sample;
        for (int r = threadIdx.x; r < nrec; r += blockDim.x) {
            const int ri = rec_ij[((size_t)b * nrec + r) * 2], rj = rec_ij[((size_t)b * nrec + r) * 2 + 1];
            rec_times[(size_t)f * nrec + r] = abs_(tf[(long long)rj * fd.nx + ri]);
        }
    }
}

cudaError_t launch_finalize(int precision, void* times, const FieldDesc* fields, int nfields, int box,
                            const int32_t* rec_ij, int nsrc, int nrec, void* rec_times, uint8_t* records, cudaStream_t st)
{
    if (precision == ALF_FP64)
        finalize_kernel<double><<<nfields, 256, 0, st>>>((double*)times, fields, box, rec_ij, nsrc, nrec,
                                                         (double*)rec_times, records);
    else
        finalize_kernel<float><<<nfields, 256, 0, st>>>((float*)times, fields, box, rec_ij, nsrc, nrec,
                                                        (float*)rec_times, records);
    note_launches(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// check64: F in double precision at every node of a solved field (alf_check.cuh).  Frozen
// nodes come from the per-field bitmap of the initialisation box.
// ---------------------------------------------------------------------------
// FP32 fields: registers are capped at 80 (a bound of three CTAs of 256 threads) while the kernel runs two
// CTAs per SM.  The two take 40,960 of the SM's 65,536 registers and leave room for two CTAs of the adjoint
// sweep (24,576), so that the check and the adjoint, on separate streams after the solve, share the SMs (a
// step of the weld batch 495.6 -> 491.6 ms; the check alone 110 -> 115 ms, with a little spilling).
template <typename T, bool VT>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 1)
    check64_kernel(const T* times, const FieldDesc* fields, int nfields, const uint32_t* region_map,
                   const RegionP<double>* regions, int nregions, const uint8_t* records, const unsigned* frozen_bits,
                   int box, double* max_rel, int32_t* n_flips, double* F_out, uint8_t* rec_out)
{
    // persistent: the CTAs stride over (field, chunk) work items, so that a small grid leaves room on
    // the SMs for kernels of other streams while this one keeps the FP64 pipe busy
    constexpr int CH = 32;  // chunks per field
    __shared__ float s_max[256];
    __shared__ int s_flip[256];
    for (long long w = blockIdx.x; w < (long long)nfields * CH; w += gridDim.x) {
    const int f = (int)(w / CH), chunk = (int)(w % CH);
    const FieldDesc fd = fields[f];
    const unsigned* fb = frozen_bits + (size_t)f * frozen_words(box);
    const int n = fd.nx * fd.ny;
    float mx = 0.f;
    int flips = 0;
    const T* tf = times + fd.node_off;
    for (int me = chunk * blockDim.x + threadIdx.x; me < n; me += CH * blockDim.x) {
        double F;
        int rec;
        T tme;
        const bool checked = check_node<T, VT>(tf, fb, box, fd, me, regions + (size_t)fd.sample * nregions,
                                               region_map + fd.map_off, F, rec, tme);
        if (!checked) {
            if (F_out) F_out[fd.node_off + me] = F;
            if (rec_out) rec_out[fd.node_off + me] = (uint8_t)rec;
            continue;
        }
        // relative residual: the difference in FP64, its ratio in FP32
        const float res = fabsf((float)(F - (double)tme)) / (float)tme;
        if (tme > T(0)) mx = fmaxf(mx, res);
        if (records && records[fd.node_off + me] != (uint8_t)rec) flips++;
        if (F_out) F_out[fd.node_off + me] = F;
        if (rec_out) rec_out[fd.node_off + me] = (uint8_t)rec;
    }
    s_max[threadIdx.x] = mx;
    s_flip[threadIdx.x] = flips;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            s_max[threadIdx.x] = fmaxf(s_max[threadIdx.x], s_max[threadIdx.x + o]);
            s_flip[threadIdx.x] += s_flip[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        // max of non-negative doubles through their bit patterns
        if (s_max[0] > 0.f)
            atomicMax((unsigned long long*)(max_rel + f), (unsigned long long)__double_as_longlong((double)s_max[0]));
        if (s_flip[0]) atomicAdd(n_flips + f, s_flip[0]);
    }
    __syncthreads();
    }
}

cudaError_t launch_check64(int precision, const void* times, const FieldDesc* fields, int nfields,
                           const uint32_t* region_map, const void* regions64, int nregions, const uint8_t* records,
                           const unsigned* frozen_bits, int box, double* max_rel, int32_t* n_flips, int grid_ctas,
                           cudaStream_t st, int vtable, double* F_out, uint8_t* rec_out)
{
    cudaError_t e = cudaMemsetAsync(max_rel, 0, sizeof(double) * nfields, st);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(n_flips, 0, sizeof(int32_t) * nfields, st);
    if (e != cudaSuccess) return e;
    const int grid = std::max(1, grid_ctas);
    const RegionP<double>* R64 = (const RegionP<double>*)regions64;
    if (precision == ALF_FP64) {
        if (vtable)
            check64_kernel<double, true><<<grid, 256, 0, st>>>((const double*)times, fields, nfields, region_map, R64,
                                                               nregions, records, frozen_bits, box, max_rel, n_flips, F_out,
                                                               rec_out);
        else
            check64_kernel<double, false><<<grid, 256, 0, st>>>((const double*)times, fields, nfields, region_map, R64,
                                                                nregions, records, frozen_bits, box, max_rel, n_flips, F_out,
                                                               rec_out);
    } else {
        if (vtable)
            check64_kernel<float, true><<<grid, 256, 0, st>>>((const float*)times, fields, nfields, region_map, R64,
                                                              nregions, records, frozen_bits, box, max_rel, n_flips, F_out,
                                                               rec_out);
        else
            check64_kernel<float, false><<<grid, 256, 0, st>>>((const float*)times, fields, nfields, region_map, R64,
                                                               nregions, records, frozen_bits, box, max_rel, n_flips, F_out,
                                                               rec_out);
    }
    note_launches(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// eval_velocity
// ---------------------------------------------------------------------------
__global__ void eval_velocity_kernel(const MatD* mat, int kind, int group_model, int precision, const double* angles,
                                     double* out, int n)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const MatD m = *mat;
    const double a = angles[k];
    if (kind == 0) {
        double s, c;
        sincos(a, &s, &c);
        if (precision == ALF_FP64) {
            out[k] = sqrt(qp_lambda64(m, c, s));
        } else {
            RegionP<float> R;
            R.a22 = float(m.a22);
            R.a33 = float(m.a33);
            R.a44 = float(m.a44);
            R.a2344 = float(m.a23 + m.a44);
            R.cth = 1.0f;
            R.sth = 0.0f;
            R.sig = m.sv ? -1.0f : 1.0f;
            R.iso = m.iso;
            R.vtab = nullptr;  // the run-time Christoffel solve
            // a unit wavefront direction u whose normal (-u_y, u_x) is at angle a
            out[k] = (double)sqrtf(phase_L<float>(R, float(s), -float(c)));
        }
    } else {
        if (precision == ALF_FP64 || group_model == 1) out[k] = group_speed64(m, group_model, a);
        else
            out[k] = (double)group_paper32(m, float(m.a22), float(m.a33), float(m.a44), float(m.a23 + m.a44), (float)a);
    }
}

cudaError_t launch_eval_velocity(const MatD* mat, int kind, int group_model, int precision, const double* angles,
                                 double* out, int n, cudaStream_t st)
{
    eval_velocity_kernel<<<(n + 127) / 128, 128, 0, st>>>(mat, kind, group_model, precision, angles, out, n);
    return cudaGetLastError();
}

}  // namespace alf
