// alf_kernels.cu -- sm_103a kernels of the forward travel-time solve.
//
//  prep_regions   per (sample, region): c/rho constants, orientation, straight-ray
//                 step times of the fallback (FP64 group->phase inversion)
//  fill_inf       every node of every field := +inf
//  init_radius    frozen straight-ray times around each source (Sec. 4.4)
//  fim            persistent warp-per-field dirty-set sweep of the local operator F
//                 to its fixed point (fields taken from a global counter)
//  finalize       clears the frozen marks and gathers receiver times
//  check64        FP64 evaluation of F at every node of a solved field
#include <cstdio>

#include "alf_internal.h"

namespace alf {

// ---------------------------------------------------------------------------
// small device helpers
// ---------------------------------------------------------------------------
ALF_D unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

ALF_D unsigned ld_volatile(const unsigned* p) { return *reinterpret_cast<const volatile unsigned*>(p); }

ALF_D void set_error(QueueState* q, unsigned code) { atomicCAS(&q->error, 0u, code); }

template <typename T>
ALF_D T load_cg(const T* p)
{
    return __ldcg(p);
}

// ---------------------------------------------------------------------------
// prep_regions
// ---------------------------------------------------------------------------
template <typename T>
__global__ void prep_regions_kernel(const MatD* mats, const uint16_t* region_mat, const double* theta, const double* h,
                                    int nsamples, int nregions, int group_model, RegionP<T>* out)
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
    for (int cls = 0; cls < 4; ++cls) R.fb[cls] = T(lens[cls] * hb / group_speed64(m, group_model, dirs[cls] - th));
    R.h = T(hb);
    R.iso = m.iso;
    R.pad = 0;
    out[k] = R;
}

cudaError_t launch_prep_regions(int precision, const MatD* mats, const uint16_t* region_mat, const double* theta,
                                const double* h, int nsamples, int nregions, int group_model, void* regions_out,
                                cudaStream_t st)
{
    const int n = nsamples * nregions;
    const int bs = 128, gs = (n + bs - 1) / bs;
    if (precision == ALF_FP64)
        prep_regions_kernel<double><<<gs, bs, 0, st>>>(mats, region_mat, theta, h, nsamples, nregions, group_model,
                                                       (RegionP<double>*)regions_out);
    else
        prep_regions_kernel<float><<<gs, bs, 0, st>>>(mats, region_mat, theta, h, nsamples, nregions, group_model,
                                                      (RegionP<float>*)regions_out);
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

cudaError_t launch_fill_inf(int precision, void* times, size_t n, cudaStream_t st)
{
    const size_t nvec = n / (precision == ALF_FP64 ? 2 : 4);
    int grid = (int)((nvec + 255) / 256);
    if (grid > 152 * 16) grid = 152 * 16;
    if (grid < 1) grid = 1;
    if (precision == ALF_FP64) fill_inf_kernel<double><<<grid, 256, 0, st>>>((double*)times, n);
    else fill_inf_kernel<float><<<grid, 256, 0, st>>>((float*)times, n);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// init_radius: one block per field; frozen nodes store -tau (sign bit = frozen)
// ---------------------------------------------------------------------------
template <typename T>
__global__ void init_radius_kernel(T* times, const FieldDesc* fields, const uint16_t* region_map,
                                   const uint16_t* region_mat, const MatD* mats, const double* theta, const double* h,
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
                               const uint16_t* region_map, const uint16_t* region_mat, const MatD* mats,
                               const double* theta, const double* h, int nregions, int r0, int group_model,
                               unsigned* frozen_bits, int box, cudaStream_t st)
{
    if (precision == ALF_FP64)
        init_radius_kernel<double><<<nfields, 128, 0, st>>>((double*)times, fields, region_map, region_mat, mats,
                                                            theta, h, nregions, r0, group_model, frozen_bits, box);
    else
        init_radius_kernel<float><<<nfields, 128, 0, st>>>((float*)times, fields, region_map, region_mat, mats, theta,
                                                           h, nregions, r0, group_model, frozen_bits, box);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// fim: persistent warp-per-field dirty-set sweep
// ---------------------------------------------------------------------------
// Each warp takes whole fields from a global counter (largest fields first).
// For one field it keeps the dirty set -- nodes that may not be at the fixed
// point of F -- as a list in its own workspace, with a bitmap so that a node
// is listed at most once.  A round
//   1. takes T = the smallest time in the dirty set (warp min-reduction);
//   2. evaluates F at every dirty node that is still unknown (+inf) or not
//      later than T + band; later nodes wait for the front, so that they are
//      not re-evaluated for every transient change of their upwind neighbours
//      (the band keeps the sweep close to the heap's order while a whole band
//      of the front is in flight);
//   3. writes the changed times, and marks dirty every non-frozen diamond
//      neighbour m of a changed node n whose time can depend on n: m unknown,
//      or m not earlier than n's old or new time (F at m only reads the
//      neighbours that precede m in key order).
// The nodes due in a round are first compacted into an evaluation list, which
// is worked in chunks of 32 x kPerLane entries: a chunk is evaluated from the
// times as they stand (Jacobi within the chunk), then written, then its dirty
// marks are set, with __syncwarp between the three steps, so the marking rule
// always compares against written times.  The field is at the
// fixed point of F when the dirty set is empty.  Frozen nodes carry the sign
// bit and are never listed.
ALF_D unsigned ws_push(unsigned* bitmap, unsigned* list, unsigned* cnt, unsigned node)
{
    const unsigned bit = 1u << (node & 31u);
    if (!(atomicOr(bitmap + (node >> 5), bit) & bit)) {
        list[atomicAdd(cnt, 1u)] = node;
        return 1u;
    }
    return 0u;
}

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

constexpr int kPerLane = 2;

template <typename T, int WARPS>
__global__ void __launch_bounds__(32 * WARPS) fim_kernel(FimLaunch a)
{
    __shared__ unsigned s_cnt[WARPS], s_ecnt[WARPS];
    const unsigned lane = threadIdx.x & 31u, wib = threadIdx.x >> 5;
    const size_t gw = (size_t)blockIdx.x * WARPS + wib;
    unsigned* const ws = a.ws + gw * a.ws_stride;
    unsigned* const elist = ws + 2 * (size_t)a.list_cap;
    unsigned* const bitmap = ws + 3 * (size_t)a.list_cap;
    unsigned* const cnt = s_cnt + wib;
    unsigned* const ecnt = s_ecnt + wib;
    T* times = (T*)a.times;
    const RegionP<T>* regions = (const RegionP<T>*)a.regions;

    for (;;) {
        unsigned fo = 0;
        if (lane == 0) fo = atomicAdd(&a.q->head, 1u);
        fo = __shfl_sync(0xffffffffu, fo, 0);
        if (fo >= (unsigned)a.nfields || ld_volatile(&a.q->error) != 0u) return;
        const unsigned f = a.order[fo];
        const FieldDesc fd = a.fields[f];
        const int nx = fd.nx, ny = fd.ny;
        const unsigned N = (unsigned)(nx * ny);
        T* tf = times + fd.node_off;
        const RegionP<T>* reg = regions + (size_t)fd.sample * a.nregions;
        const uint16_t* map = a.region_map + fd.map_off;
        const T band = a.band_cells > 0.0 ? T(a.band_cells * fd.cell_time) : alf_inf<T>();
        unsigned* listA = ws;
        unsigned* listB = ws + a.list_cap;

        for (unsigned w = lane; w < (N + 31u) / 32u; w += 32u) bitmap[w] = 0u;
        if (lane == 0) *cnt = 0u;
        __syncwarp();
        {   // first dirty set: the non-frozen nodes around the frozen box
            const int r = a.box + 2, w = 2 * r + 1;
            for (int k = (int)lane; k < w * w; k += 32) {
                const int i = fd.si + k % w - r, j = fd.sj + k / w - r;
                if (i < 0 || j < 0 || i >= nx || j >= ny) continue;
                const unsigned n = (unsigned)(j * nx + i);
                if (!neg_bit(__ldcg(tf + n))) ws_push(bitmap, listA, cnt, n);
            }
        }
        __syncwarp();
        unsigned nact = *cnt;
        unsigned rounds = 0;
        unsigned long long evals = 0;
        const unsigned max_rounds = a.max_rounds_per_node * (unsigned)(nx + ny);
        while (nact > 0) {
            if (++rounds > max_rounds) {
                if (lane == 0) set_error(a.q, ALF_ERR_NOT_CONVERGED);
                break;
            }
            // 1. front time
            auto m = order_key(alf_inf<T>());
            for (unsigned k = lane; k < nact; k += 32u) {
                const auto v = order_key(__ldcg(tf + listA[k]));
                m = v < m ? v : m;
            }
            const T lim = from_key(warp_min(m), T(0)) + band;
            __syncwarp();
            if (lane == 0) {
                *cnt = 0u;
                *ecnt = 0u;
            }
            __syncwarp();
            // 2a. nodes due for evaluation leave the set and go to the evaluation list;
            //     nodes far ahead of the front stay dirty (their bit stays set)
            for (unsigned k = lane; k < nact; k += 32u) {
                const unsigned n = listA[k];
                const T t = __ldcg(tf + n);
                if (t <= lim || !(t < alf_inf<T>())) {
                    atomicAnd(bitmap + (n >> 5), ~(1u << (n & 31u)));
                    elist[atomicAdd(ecnt, 1u)] = n;
                } else {
                    listB[atomicAdd(cnt, 1u)] = n;
                }
            }
            __syncwarp();
            const unsigned ne = *ecnt;
            for (unsigned base = 0; base < ne; base += 32u * kPerLane) {
                unsigned node[kPerLane];
                T oldv[kPerLane], newv[kPerLane];
                bool ev[kPerLane];
                // 2b. evaluate a chunk with the times as they stand
#pragma unroll
                for (int r = 0; r < kPerLane; ++r) {
                    const unsigned k = base + (unsigned)r * 32u + lane;
                    ev[r] = k < ne;
                    node[r] = ev[r] ? elist[k] : 0u;
                }
#pragma unroll
                for (int r = 0; r < kPerLane; ++r) {
                    oldv[r] = newv[r] = alf_inf<T>();
                    if (!ev[r]) continue;
                    const unsigned n = node[r];
                    oldv[r] = __ldcg(tf + n);
                    const int i = (int)(n % (unsigned)nx), j = (int)(n / (unsigned)nx);
                    T nb[12];
#pragma unroll
                    for (int q = 0; q < 12; ++q) {
                        const int ii = i + kSlotDi[q], jj = j + kSlotDj[q];
                        nb[q] = (ii >= 0 && jj >= 0 && ii < nx && jj < ny) ? __ldcg(tf + jj * nx + ii) : alf_inf<T>();
                    }
                    const RegionP<T> R = reg[__ldg(map + n)];
                    int rec;
                    newv[r] = local_F<T>(nb, (int)n, nx, R, rec);
                    if (a.records) a.records[fd.node_off + n] = (uint8_t)rec;
                    ++evals;
                }
                __syncwarp();
                // 2c. write the changed times
#pragma unroll
                for (int r = 0; r < kPerLane; ++r)
                    if (ev[r] && !same_bits(newv[r], oldv[r])) __stcg(tf + node[r], newv[r]);
                __syncwarp();
                // 3. mark the neighbours that can depend on a changed node
#pragma unroll
                for (int r = 0; r < kPerLane; ++r) {
                    if (!ev[r] || same_bits(newv[r], oldv[r])) continue;
                    const unsigned n = node[r];
                    const int i = (int)(n % (unsigned)nx), j = (int)(n / (unsigned)nx);
                    const T lo = newv[r] < oldv[r] ? newv[r] : oldv[r];
#pragma unroll
                    for (int q = 0; q < 12; ++q) {
                        const int ii = i + kSlotDi[q], jj = j + kSlotDj[q];
                        if (ii < 0 || jj < 0 || ii >= nx || jj >= ny) continue;
                        const unsigned mm = (unsigned)(jj * nx + ii);
                        const T tm = __ldcg(tf + mm);
                        if (neg_bit(tm)) continue;  // frozen
                        if (!(tm < alf_inf<T>()) || lo <= tm) ws_push(bitmap, listB, cnt, mm);
                    }
                }
                __syncwarp();
            }
            nact = *cnt;
            unsigned* t = listA;
            listA = listB;
            listB = t;
            __syncwarp();
        }
        for (int o = 16; o > 0; o >>= 1) evals += __shfl_xor_sync(0xffffffffu, evals, o);
        if (lane == 0) {
            atomicAdd(&a.q->visits, evals);
            atomicAdd(&a.q->rounds, (unsigned long long)rounds);
        }
        __syncwarp();
    }
}

template <typename T, int WARPS>
static cudaError_t fim_t(int grid, const FimLaunch& a, cudaStream_t st)
{
    fim_kernel<T, WARPS><<<grid, 32 * WARPS, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_fim(int precision, int threads, int grid, const FimLaunch& a, cudaStream_t st)
{
    if (precision == ALF_FP64) {
        if (threads == 128) return fim_t<double, 4>(grid, a, st);
        if (threads == 512) return fim_t<double, 16>(grid, a, st);
        return fim_t<double, 8>(grid, a, st);
    }
    if (threads == 128) return fim_t<float, 4>(grid, a, st);
    if (threads == 512) return fim_t<float, 16>(grid, a, st);
    return fim_t<float, 8>(grid, a, st);
}

template <typename T, int WARPS>
static int occ_fim()
{
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fim_kernel<T, WARPS>, 32 * WARPS, 0);
    return n;
}

int fim_max_ctas_per_sm(int precision, int threads)
{
    if (precision == ALF_FP64)
        return threads == 128 ? occ_fim<double, 4>() : threads == 512 ? occ_fim<double, 16>() : occ_fim<double, 8>();
    return threads == 128 ? occ_fim<float, 4>() : threads == 512 ? occ_fim<float, 16>() : occ_fim<float, 8>();
}

// ---------------------------------------------------------------------------
// finalize: frozen marks cleared (box around each source), receiver times
// ---------------------------------------------------------------------------
template <typename T>
__global__ void finalize_kernel(T* times, const FieldDesc* fields, int box, const int32_t* rec_ij, int nsrc, int nrec,
                                T* rec_times)
{
    const int f = blockIdx.x;
    const FieldDesc fd = fields[f];
    const int w = 2 * box + 1;
    T* tf = times + fd.node_off;
    for (int k = threadIdx.x; k < w * w; k += blockDim.x) {
        const int i = fd.si + k % w - box, j = fd.sj + k / w - box;
        if (i < 0 || j < 0 || i >= fd.nx || j >= fd.ny) continue;
        T* p = tf + (long long)j * fd.nx + i;
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
                            const int32_t* rec_ij, int nsrc, int nrec, void* rec_times, cudaStream_t st)
{
    if (precision == ALF_FP64)
        finalize_kernel<double><<<nfields, 256, 0, st>>>((double*)times, fields, box, rec_ij, nsrc, nrec,
                                                         (double*)rec_times);
    else
        finalize_kernel<float><<<nfields, 256, 0, st>>>((float*)times, fields, box, rec_ij, nsrc, nrec,
                                                        (float*)rec_times);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// check64: F in double precision at every node of a solved field.  Frozen
// nodes come from the per-field bitmap of the initialisation box.
// ---------------------------------------------------------------------------
ALF_D bool box_frozen(const unsigned* bits, int box, const FieldDesc& fd, int i, int j)
{
    const int di = i - fd.si, dj = j - fd.sj;
    if (di < -box || di > box || dj < -box || dj > box) return false;
    const int bit = (dj + box) * (2 * box + 1) + (di + box);
    return (bits[bit >> 5] >> (bit & 31)) & 1u;
}

template <typename T>
__global__ void check64_kernel(const T* times, const FieldDesc* fields, const uint16_t* region_map,
                               const RegionP<double>* regions, int nregions, const uint8_t* records,
                               const unsigned* frozen_bits, int box, double* max_rel, int32_t* n_flips)
{
    const int f = blockIdx.y;
    const FieldDesc fd = fields[f];
    const unsigned* fb = frozen_bits + (size_t)f * frozen_words(box);
    const int n = fd.nx * fd.ny;
    __shared__ double s_max[256];
    __shared__ int s_flip[256];
    double mx = 0.0;
    int flips = 0;
    const T* tf = times + fd.node_off;
    for (int me = blockIdx.x * blockDim.x + threadIdx.x; me < n; me += gridDim.x * blockDim.x) {
        const int i = me % fd.nx, j = me / fd.nx;
        if (box_frozen(fb, box, fd, i, j)) continue;
        double nb[12];
        for (int k = 0; k < 12; ++k) {
            const int ii = i + kSlotDi[k], jj = j + kSlotDj[k];
            if (ii < 0 || jj < 0 || ii >= fd.nx || jj >= fd.ny) {
                nb[k] = alf_inf<double>();
            } else {
                const double v = fabs((double)tf[(long long)jj * fd.nx + ii]);
                nb[k] = box_frozen(fb, box, fd, ii, jj) ? -v : v;
            }
        }
        const RegionP<double> R = regions[(size_t)fd.sample * nregions + region_map[fd.map_off + me]];
        int rec;
        const double F = local_F<double>(nb, me, fd.nx, R, rec);
        const double t = fabs((double)tf[me]);
        if (t > 0.0 && t < alf_inf<double>()) mx = fmax(mx, fabs(F - t) / t);
        if (records && records[fd.node_off + me] != (uint8_t)rec) flips++;
    }
    s_max[threadIdx.x] = mx;
    s_flip[threadIdx.x] = flips;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            s_max[threadIdx.x] = fmax(s_max[threadIdx.x], s_max[threadIdx.x + o]);
            s_flip[threadIdx.x] += s_flip[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        // max of non-negative doubles through their bit patterns
        atomicMax((unsigned long long*)(max_rel + f), (unsigned long long)__double_as_longlong(s_max[0]));
        atomicAdd(n_flips + f, s_flip[0]);
    }
}

cudaError_t launch_check64(int precision, const void* times, const FieldDesc* fields, int nfields,
                           const uint16_t* region_map, const void* regions64, int nregions, const uint8_t* records,
                           const unsigned* frozen_bits, int box, double* max_rel, int32_t* n_flips, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(max_rel, 0, sizeof(double) * nfields, st);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(n_flips, 0, sizeof(int32_t) * nfields, st);
    if (e != cudaSuccess) return e;
    dim3 grid(32, nfields);
    if (precision == ALF_FP64)
        check64_kernel<double><<<grid, 256, 0, st>>>((const double*)times, fields, region_map,
                                                     (const RegionP<double>*)regions64, nregions, records,
                                                     frozen_bits, box, max_rel, n_flips);
    else
        check64_kernel<float><<<grid, 256, 0, st>>>((const float*)times, fields, region_map,
                                                    (const RegionP<double>*)regions64, nregions, records,
                                                    frozen_bits, box, max_rel, n_flips);
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
            R.iso = m.iso;
            // a unit wavefront direction u whose normal (-u_y, u_x) is at angle a
            out[k] = (double)sqrtf(phase_L<float>(R, float(s), -float(c)));
        }
    } else {
        if (precision == ALF_FP64 || group_model == 1) out[k] = group_speed64(m, group_model, a);
        else
            out[k] = (double)group_paper32(m, float(m.a22), float(m.a33), float(m.a44), float(m.a23 + m.a44), a);
    }
}

cudaError_t launch_eval_velocity(const MatD* mat, int kind, int group_model, int precision, const double* angles,
                                 double* out, int n, cudaStream_t st)
{
    eval_velocity_kernel<<<(n + 127) / 128, 128, 0, st>>>(mat, kind, group_model, precision, angles, out, n);
    return cudaGetLastError();
}

}  // namespace alf
