// alf_adjoint.cu -- reverse-mode gradient of receiver times with respect to
// region orientations (the gradient a Monte Carlo or variational inversion
// needs, Sec. 1 of the paper), by the discrete adjoint of the solve.
//
// At the fixed point every non-frozen node's time is one local formula -- the
// stencil its record names (Secs. 4.2-4.3) or the straight-ray fallback --
// applied to at most three earlier nodes and to the orientation at the node;
// a frozen node's time is the straight-ray time from the source (Sec. 4.4).
// The adjoint therefore runs on a DAG whose edges point from every node to
// the nodes it used:
//   weights   per node, the partial derivatives of its formula (analytic for
//             stencils; FP64 central differences of the group speed for the
//             fallback and the frozen nodes) and the in-degree of every
//             node (how many later nodes use it);
//   seed      lambda = dL/dT at the receivers;
//   rounds    Kahn's order: a node whose users have all been processed is
//             final; it adds lambda * weight to the nodes it used and releases
//             them (in-degree to zero -> next frontier).  Either all fields
//             advance in lockstep rounds (a few launches per round), or one
//             warp owns each field and runs all its rounds in one launch;
//   reduce    dL/dtheta_region = sum over the region's nodes of
//             lambda * d(time)/d(theta) (frozen nodes: the source's region).
// Every node is processed exactly once, so the sweep is exact and its work is
// linear in the number of nodes.
#include <algorithm>

#include "alf_internal.h"

namespace alf {

template <typename T>
struct AdjW {
    T w[3];   // d tau_D / d tau of the supporting nodes (stencil A, B, C; fallback: w[0] = 1)
    T wt;     // d tau_D / d theta
};

// analytic partial derivatives of the stencil time (see stencil_time)
template <typename T>
ALF_D void stencil_partials(int xA, int yA, int xB, int yB, int xC, int yC, T tA, T tB, T tC, const RegionP<T>& R,
                            T w[3], T& wt)
{
    const T den = tC - tA;
    const T a = (tB - tA) / den;
    const T Ex = T(xA) + a * T(xC - xA), Ey = T(yA) + a * T(yC - yA);
    const T ux = T(xB) - Ex, uy = T(yB) - Ey;
    const T cr = T(yB) * Ex - T(xB) * Ey;
    const T acr = abs_(cr), sgn = cr >= T(0) ? T(1) : T(-1);
    T L, dLux, dLuy, dLth;
    if (R.iso) {
        L = R.a22 * (ux * ux + uy * uy);
        dLux = T(2) * R.a22 * ux;
        dLuy = T(2) * R.a22 * uy;
        dLth = T(0);
    } else {
        const T C = R.sth * ux - R.cth * uy, S = R.cth * ux + R.sth * uy;
        const T al = C * C * R.a22 + S * S * R.a44, ga = C * C * R.a44 + S * S * R.a33, be = C * S * R.a2344;
        const T dm = al - ga;
        const T Rr = sqrt_(dm * dm + T(4) * be * be);
        L = T(0.5) * ((al + ga) + Rr);
        T dC = T(2) * C * (R.a22 + R.a44), dS = T(2) * S * (R.a44 + R.a33);
        if (Rr > T(0)) {
            dC += (dm * T(2) * C * (R.a22 - R.a44) + T(4) * be * S * R.a2344) / Rr;
            dS += (dm * T(2) * S * (R.a44 - R.a33) + T(4) * be * C * R.a2344) / Rr;
        }
        dC *= T(0.5);
        dS *= T(0.5);
        dLux = dC * R.sth + dS * R.cth;
        dLuy = -dC * R.cth + dS * R.sth;
        dLth = dC * S - dS * C;
    }
    const T rs = T(1) / sqrt_(L);
    const T r3 = rs * rs * rs;
    const T dcr = T(yB) * T(xC - xA) - T(xB) * T(yC - yA);
    const T dL = dLux * T(-(xC - xA)) + dLuy * T(-(yC - yA));
    const T dPhi_da = R.h * (sgn * dcr * rs - T(0.5) * acr * r3 * dL);
    const T inv = T(1) / den;
    w[0] = dPhi_da * (tB - tC) * inv * inv;
    w[1] = T(1) + dPhi_da * inv;
    w[2] = -dPhi_da * (tB - tA) * inv * inv;
    wt = -T(0.5) * R.h * acr * r3 * dLth;
}

ALF_D bool frozen_at(const unsigned* bits, int box, const FieldDesc& fd, int i, int j)
{
    const int di = i - fd.si, dj = j - fd.sj;
    if (di < -box || di > box || dj < -box || dj > box) return false;
    const int bit = (dj + box) * (2 * box + 1) + (di + box);
    return (bits[bit >> 5] >> (bit & 31)) & 1u;
}

// the nodes of the record's formula, in the order of the weights
ALF_D int support_slots(int rec, int s[3])
{
    if (rec < 32) {
        const int p = rec >> 1;
        s[0] = kPairA[p];
        s[1] = (rec & 1) ? kPairQ[p] : kPairP[p];
        s[2] = (rec & 1) ? kPairP[p] : kPairQ[p];
        return 3;
    }
    if (rec < 44) {
        s[0] = rec - 32;
        return 1;
    }
    return 0;
}

template <typename T>
__global__ void adj_weights_kernel(AdjLaunch a)
{
    const size_t total = a.total_nodes;
    const T* times = (const T*)a.times;
    AdjW<T>* W = (AdjW<T>*)a.weights;
    const RegionP<T>* regions = (const RegionP<T>*)a.regions;
    for (size_t g = (size_t)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += (size_t)gridDim.x * blockDim.x) {
        // field of node g: binary search over the node offsets
        int lo = 0, hi = a.nfields;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if ((size_t)a.fields[mid].node_off <= g) lo = mid; else hi = mid;
        }
        const FieldDesc fd = a.fields[lo];
        const unsigned n = (unsigned)(g - (size_t)fd.node_off);
        const int nx = fd.nx, ny = fd.ny;
        const int i = (int)(n % (unsigned)nx), j = (int)(n / (unsigned)nx);
        const unsigned* fb = a.frozen_bits + (size_t)lo * frozen_words(a.box);
        AdjW<T> w{};
        if (frozen_at(fb, a.box, fd, i, j)) {
            // straight-ray time from the source: derivative by the source orientation
            if (i != fd.si || j != fd.sj) {
                const int rs = a.region_map[fd.map_off + (long long)fd.sj * nx + fd.si];
                const MatD m = a.mats[a.region_mat[rs]];
                const double th = a.theta[(size_t)fd.sample * a.nregions + rs];
                const double di = i - fd.si, dj = j - fd.sj;
                const double dist = sqrt(di * di + dj * dj) * a.h[fd.sample];
                const double dir = atan2(dj, di);
                const double e = 1e-6;
                w.wt = T((dist / group_speed64(m, a.group_model, dir - th - e) -
                          dist / group_speed64(m, a.group_model, dir - th + e)) / (2.0 * e));
            }
            W[g] = w;
            continue;
        }
        const int rec = a.records[g];
        int s[3];
        int ns = support_slots(rec, s);
        for (int k = 0; k < ns; ++k) {  // a record from another solve could point outside the grid
            const int ii = i + kSlotDi[s[k]], jj = j + kSlotDj[s[k]];
            if (ii < 0 || jj < 0 || ii >= nx || jj >= ny) ns = 0;
        }
        if (ns == 3) {
            const T* tf = times + fd.node_off;
            T t3[3];
            for (int k = 0; k < 3; ++k) t3[k] = abs_(tf[(j + kSlotDj[s[k]]) * nx + i + kSlotDi[s[k]]]);
            const RegionP<T> R = regions[(size_t)fd.sample * a.nregions + a.region_map[fd.map_off + n]];
            stencil_partials<T>(kSlotDi[s[0]], kSlotDj[s[0]], kSlotDi[s[1]], kSlotDj[s[1]], kSlotDi[s[2]],
                                kSlotDj[s[2]], t3[0], t3[1], t3[2], R, w.w, w.wt);
        } else if (ns == 1) {
            const RegionP<T> R = regions[(size_t)fd.sample * a.nregions + a.region_map[fd.map_off + n]];
            w.w[0] = T(1);
            const int cls = kSlotClass[s[0]];
            w.wt = (s[0] >= 8 ? T(2) : T(1)) * R.dfb[cls];
        }
        for (int k = 0; k < ns; ++k)
            atomicAdd(a.indeg + fd.node_off + (j + kSlotDj[s[k]]) * nx + i + kSlotDi[s[k]], 1u);
        W[g] = w;
    }
}

template <typename T>
__global__ void adj_seed_kernel(AdjLaunch a, const T* dL_drec)
{
    const int total = a.nfields * a.nrec;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < total; k += gridDim.x * blockDim.x) {
        const int f = k / a.nrec, r = k % a.nrec;
        const FieldDesc fd = a.fields[f];
        const int ri = a.rec_ij[((size_t)fd.sample * a.nrec + r) * 2];
        const int rj = a.rec_ij[((size_t)fd.sample * a.nrec + r) * 2 + 1];
        atomicAdd((T*)a.lambda + fd.node_off + (long long)rj * fd.nx + ri, dL_drec[k]);
    }
}

// first frontier of every field: the nodes no later node uses (one warp per field)
__global__ void adj_frontier_kernel(AdjLaunch a)
{
    const unsigned lane = threadIdx.x & 31u;
    const size_t nw = (size_t)gridDim.x * blockDim.x / 32;
    for (size_t f = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) / 32; f < (size_t)a.nfields; f += nw) {
        const FieldDesc fd = a.fields[f];
        const unsigned N = (unsigned)(fd.nx * fd.ny);
        const unsigned* deg = a.indeg + fd.node_off;
        unsigned* list = a.list[0] + fd.node_off;
        unsigned cnt = 0;
        for (unsigned base = 0; base < N; base += 32u) {
            const unsigned n = base + lane;
            const bool take = n < N && deg[n] == 0u;
            const unsigned bal = __ballot_sync(0xffffffffu, take);
            if (take) list[cnt + __popc(bal & ((1u << lane) - 1u))] = n;
            cnt += __popc(bal);
        }
        if (lane == 0) {
            a.cnt[f] = cnt;
            a.cnt[a.nfields + f] = 0u;
        }
    }
}

__global__ void adj_scan_kernel(AdjLaunch a, int parity)
{
    __shared__ unsigned s[1024];
    const unsigned* c = a.cnt + (size_t)parity * a.nfields;
    const int n = a.nfields;
    const int per = (n + 1023) / 1024;
    const int b0 = threadIdx.x * per, b1 = min(n, b0 + per);
    unsigned sum = 0;
    for (int f = b0; f < b1; ++f) sum += c[f];
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
        run += c[f];
    }
    if (threadIdx.x == 1023) a.eoff[n] = s[1023];
}

template <typename T>
__global__ void adj_process_kernel(AdjLaunch a, int parity)
{
    const unsigned E = a.eoff[a.nfields];
    T* lam = (T*)a.lambda;
    const AdjW<T>* W = (const AdjW<T>*)a.weights;
    T* gnode = (T*)a.gnode;
    unsigned* nxt = a.cnt + (size_t)(parity ^ 1) * a.nfields;
    for (unsigned e = blockIdx.x * blockDim.x + threadIdx.x; e < E; e += gridDim.x * blockDim.x) {
        int lo = 0, hi = a.nfields;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (__ldg(a.eoff + mid) <= e) lo = mid; else hi = mid;
        }
        const FieldDesc fd = a.fields[lo];
        const unsigned n = a.list[parity][fd.node_off + (e - a.eoff[lo])];
        const size_t g = (size_t)fd.node_off + n;
        const T l = lam[g];
        const AdjW<T> w = W[g];
        gnode[g] = l * w.wt;
        const unsigned* fbits = a.frozen_bits + (size_t)lo * frozen_words(a.box);
        const int nx = fd.nx;
        const int i = (int)(n % (unsigned)nx), j = (int)(n / (unsigned)nx);
        if (frozen_at(fbits, a.box, fd, i, j)) continue;
        int s[3];
        int ns = support_slots(a.records[g], s);
        for (int k = 0; k < ns; ++k) {
            const int ii = i + kSlotDi[s[k]], jj = j + kSlotDj[s[k]];
            if (ii < 0 || jj < 0 || ii >= nx || jj >= fd.ny) ns = 0;
        }
        unsigned* list = a.list[parity ^ 1] + fd.node_off;
        for (int k = 0; k < ns; ++k) {
            const unsigned m = (unsigned)((j + kSlotDj[s[k]]) * nx + i + kSlotDi[s[k]]);
            atomicAdd(lam + fd.node_off + m, l * w.w[k]);
            __threadfence();
            if (atomicSub(a.indeg + fd.node_off + m, 1u) == 1u) list[atomicAdd(nxt + lo, 1u)] = m;
        }
    }
}

// first frontier of every field, one thread per node (field-resident schedule)
__global__ void adj_frontier_flat_kernel(AdjLaunch a)
{
    for (size_t g = (size_t)blockIdx.x * blockDim.x + threadIdx.x; g < a.total_nodes;
         g += (size_t)gridDim.x * blockDim.x) {
        if (a.indeg[g] != 0u) continue;
        int lo = 0, hi = a.nfields;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if ((size_t)a.fields[mid].node_off <= g) lo = mid; else hi = mid;
        }
        const size_t off = (size_t)a.fields[lo].node_off;
        a.list[0][off + atomicAdd(a.cnt + lo, 1u)] = (unsigned)(g - off);
    }
}

// Kahn rounds of one field by one warp, fields taken from a queue (largest first).  Only the owning
// warp touches a field's lambda and in-degrees, and the warp barrier at the end of a round orders a
// round's contributions before the next round reads them (through L2: __ldcg).
template <typename T>
__global__ void __launch_bounds__(256) adj_warp_kernel(AdjLaunch a)
{
    constexpr unsigned FULL = 0xffffffffu;
    const unsigned lane = threadIdx.x & 31u;
    const unsigned below = (1u << lane) - 1u;
    T* const lam = (T*)a.lambda;
    const AdjW<T>* W = (const AdjW<T>*)a.weights;
    T* const gnode = (T*)a.gnode;
    for (;;) {
        unsigned fi = 0u;
        if (lane == 0) fi = atomicAdd(a.head, 1u);
        fi = __shfl_sync(FULL, fi, 0);
        if (fi >= (unsigned)a.nfields) return;
        const unsigned f = __ldg(a.order + fi);
        const FieldDesc fd = a.fields[f];
        const int nx = fd.nx, ny = fd.ny;
        const size_t off = (size_t)fd.node_off;
        const unsigned* fbits = a.frozen_bits + (size_t)f * frozen_words(a.box);
        unsigned* const list0 = a.list[0] + off;
        unsigned* const list1 = a.list[1] + off;
        unsigned nact = a.cnt[f], par = 0u;
        while (nact != 0u) {
            const unsigned* LA = par ? list1 : list0;
            unsigned* LB = par ? list0 : list1;
            unsigned nc = 0u;
            for (unsigned base = 0; base < nact; base += 32u) {
                const unsigned e = base + lane;
                unsigned m[3] = {0u, 0u, 0u};
                bool fresh[3] = {false, false, false};
                if (e < nact) {
                    const unsigned n = LA[e];
                    const size_t g = off + n;
                    const T l = __ldcg(lam + g);
                    const AdjW<T> w = W[g];
                    gnode[g] = l * w.wt;
                    const int i = (int)(n % (unsigned)nx), j = (int)(n / (unsigned)nx);
                    if (!frozen_at(fbits, a.box, fd, i, j)) {
                        int s[3];
                        int ns = support_slots(a.records[g], s);
                        for (int k = 0; k < ns; ++k) {
                            const int ii = i + kSlotDi[s[k]], jj = j + kSlotDj[s[k]];
                            if (ii < 0 || jj < 0 || ii >= nx || jj >= ny) ns = 0;
                        }
#pragma unroll
                        for (int k = 0; k < 3; ++k)
                            if (k < ns) {
                                m[k] = (unsigned)((j + kSlotDj[s[k]]) * nx + i + kSlotDi[s[k]]);
                                atomicAdd(lam + off + m[k], l * w.w[k]);
                            }
#pragma unroll
                        for (int k = 0; k < 3; ++k)
                            if (k < ns) fresh[k] = atomicSub(a.indeg + off + m[k], 1u) == 1u;
                    }
                }
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const unsigned b = __ballot_sync(FULL, fresh[k]);
                    if (fresh[k]) LB[nc + __popc(b & below)] = m[k];
                    nc += __popc(b);
                }
            }
            __syncwarp();
            nact = nc;
            par ^= 1u;
        }
    }
}

// dL/dtheta: per field, the node contributions summed by region (frozen nodes: the source's region)
template <typename T>
__global__ void adj_reduce_kernel(AdjLaunch a, double* grad)
{
    extern __shared__ double acc[];
    const int f = blockIdx.x;
    const FieldDesc fd = a.fields[f];
    const bool use_smem = a.nregions <= 4096;
    if (use_smem)
        for (int r = threadIdx.x; r < a.nregions; r += blockDim.x) acc[r] = 0.0;
    __syncthreads();
    const T* gnode = (const T*)a.gnode + fd.node_off;
    const unsigned* fbits = a.frozen_bits + (size_t)f * frozen_words(a.box);
    const int rs = a.region_map[fd.map_off + (long long)fd.sj * fd.nx + fd.si];
    double* gb = grad + (size_t)fd.sample * a.nregions;
    const int N = fd.nx * fd.ny;
    for (int n = threadIdx.x; n < N; n += blockDim.x) {
        const T v = gnode[n];
        if (v == T(0)) continue;
        const int i = n % fd.nx, j = n / fd.nx;
        const int r = frozen_at(fbits, a.box, fd, i, j) ? rs : a.region_map[fd.map_off + n];
        if (use_smem) atomicAdd(acc + r, (double)v);
        else atomicAdd(gb + r, (double)v);
    }
    __syncthreads();
    if (use_smem)
        for (int r = threadIdx.x; r < a.nregions; r += blockDim.x)
            if (acc[r] != 0.0) atomicAdd(gb + r, acc[r]);
}

__global__ void adj_pending_kernel(AdjLaunch a, int parity, unsigned long long* out)
{
    const unsigned* c = a.cnt + (size_t)parity * a.nfields;
    unsigned long long s = 0;
    for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < a.nfields; f += gridDim.x * blockDim.x) s += c[f];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0 && s) atomicAdd(out, s);
}

template <typename T>
static cudaError_t adjoint_t(const AdjLaunch& a, const void* dL_drec, double* grad, unsigned long long* d_pending,
                             unsigned long long* h_pending, int grid, cudaStream_t st)
{
    cudaError_t e;
    if ((e = cudaMemsetAsync(a.lambda, 0, a.total_nodes * sizeof(T), st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(a.indeg, 0, a.total_nodes * sizeof(unsigned), st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(a.gnode, 0, a.total_nodes * sizeof(T), st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(grad, 0, (size_t)a.nsamples * a.nregions * sizeof(double), st)) != cudaSuccess) return e;
    adj_weights_kernel<T><<<grid, 256, 0, st>>>(a);
    adj_seed_kernel<T><<<64, 256, 0, st>>>(a, (const T*)dL_drec);
    if (a.warp_grid > 0) {
        // field-resident schedule: flat frontier, then every field's rounds in one launch
        if ((e = cudaMemsetAsync(a.cnt, 0, (size_t)a.nfields * sizeof(unsigned), st)) != cudaSuccess) return e;
        if ((e = cudaMemsetAsync(a.head, 0, sizeof(unsigned), st)) != cudaSuccess) return e;
        adj_frontier_flat_kernel<<<grid, 256, 0, st>>>(a);
        adj_warp_kernel<T><<<a.warp_grid, 256, 0, st>>>(a);
        const size_t smem = a.nregions <= 4096 ? (size_t)a.nregions * sizeof(double) : 0;
        adj_reduce_kernel<T><<<a.nfields, 256, smem, st>>>(a, grad);
        note_launches(5);
        return cudaGetLastError();
    }
    adj_frontier_kernel<<<std::max(1, std::min((a.nfields + 7) / 8, grid)), 256, 0, st>>>(a);
    note_launches(3);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    int parity = 0;
    for (long long r = 0; r < (long long)a.max_rounds;) {
        for (int k = 0; k < 32; ++k, ++r) {
            adj_scan_kernel<<<1, 1024, 0, st>>>(a, parity);
            if ((e = cudaMemsetAsync(a.cnt + (size_t)(parity ^ 1) * a.nfields, 0, a.nfields * sizeof(unsigned), st)) !=
                cudaSuccess)
                return e;
            adj_process_kernel<T><<<grid, 256, 0, st>>>(a, parity);
            note_launches(2);
            parity ^= 1;
        }
        if ((e = cudaMemsetAsync(d_pending, 0, sizeof(unsigned long long), st)) != cudaSuccess) return e;
        adj_pending_kernel<<<64, 256, 0, st>>>(a, parity, d_pending);
        note_launches(1);
        if ((e = cudaMemcpyAsync(h_pending, d_pending, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st)) !=
            cudaSuccess)
            return e;
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
        if (*h_pending == 0ull) break;
    }
    const size_t smem = a.nregions <= 4096 ? (size_t)a.nregions * sizeof(double) : 0;
    adj_reduce_kernel<T><<<a.nfields, 256, smem, st>>>(a, grad);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_adjoint(int precision, const AdjLaunch& a, const void* dL_drec, double* grad,
                           unsigned long long* d_pending, unsigned long long* h_pending, int grid, cudaStream_t st)
{
    return precision == ALF_FP64 ? adjoint_t<double>(a, dL_drec, grad, d_pending, h_pending, grid, st)
                                 : adjoint_t<float>(a, dL_drec, grad, d_pending, h_pending, grid, st);
}

}  // namespace alf
