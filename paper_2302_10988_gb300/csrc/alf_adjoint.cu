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
//   (everything the sweep touches per node -- weights, lambda, its
//   contribution lambda * dtau/dtheta, in-degree, its stencil record and
//   whether it is frozen -- sits in one 32-byte record (64 bytes in FP64):
//   the release that makes a node ready brings that sector into L2, where
//   the node's processing then finds all of it; a user's contribution and
//   its release of a support node are one vector atomic on the adjacent
//   (lambda, in-degree) pair in FP32);
//   seed      lambda = dL/dT at the receivers;
//   rounds    Kahn's order: a node whose users have all been processed is
//             final; it adds lambda * weight to the nodes it used and releases
//             them (in-degree to zero -> next frontier).  Either all fields
//             advance in lockstep rounds (a few launches per round), or one
//             warp owns each field and runs all its rounds in one launch;
//   reduce    dL/dtheta_region = sum over the region's nodes of
//             lambda * d(time)/d(theta) (frozen nodes: the source's region);
//             the field-resident sweep sums them per warp in shared memory
//             as it goes (regions <= 512), else a per-field block reduces.
// Every node is processed exactly once, so the sweep is exact and its work is
// linear in the number of nodes.
#include <algorithm>

#include "alf_internal.h"

namespace alf {

template <typename T>
struct alignas(8 * sizeof(T)) AdjNode {
    T w[3];           // d tau_D / d tau of the supporting nodes (stencil A, B, C; fallback: w[0] = 1)
    T wt;             // d tau_D / d theta
    T lam;            // dL / d tau_D
    T indeg;          // later nodes that use this one, not yet processed (a small integer, exact in T)
    T gn;             // lam * wt (the node's contribution to its region's gradient)
    T code;           // what the sweep needs of the node's formula, packed (adj_code): one sector a node visit
};

// The sweep's view of a node's formula, packed into 24 bits (exact in FP32): its support nodes as diamond
// slots (bits 0-11, four bits each, in the order of the weights), how many it releases (bits 12-13: 3 for a
// stencil, 1 for the fallback, 0 for a frozen node or a formula with a support point outside the grid),
// whether it is frozen (bit 14) and the region its contribution goes to (bits 15-23, when the regions are
// few enough for the sweep to sum them in shared memory: the node's own, a frozen node's source's).
#define ADJ_SMEM_REGIONS 512
ALF_HD unsigned adj_code(const int s[3], int ns, bool frozen, int region)
{
    return (unsigned)s[0] | ((unsigned)s[1] << 4) | ((unsigned)s[2] << 8) | ((unsigned)ns << 12) |
           (frozen ? 1u << 14 : 0u) | ((unsigned)(region & (ADJ_SMEM_REGIONS - 1)) << 15);
}
static_assert(sizeof(AdjNode<float>) == 32 && sizeof(AdjNode<double>) == 64, "one or two DRAM sectors per node");

// A processed user hands its contribution to a support node and releases it: lam += c, indeg -= 1; returns
// true when that was the last user (the support node is final).  FP32: one 8-byte vector atomic on the
// adjacent (lam, indeg) pair, so the contribution and the release land together; FP64: two atomics.
ALF_D bool release(AdjNode<float>* node, float c)
{
    const float2 old = atomicAdd(reinterpret_cast<float2*>(&node->lam), make_float2(c, -1.0f));
    return old.y == 1.0f;
}
ALF_D bool release(AdjNode<double>* node, double c)
{
    atomicAdd(&node->lam, c);
    return atomicAdd(&node->indeg, -1.0) == 1.0;
}

size_t adj_node_bytes(int precision) { return precision == ALF_FP64 ? sizeof(AdjNode<double>) : sizeof(AdjNode<float>); }

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
        L = T(0.5) * ((al + ga) + R.sig * Rr);
        T dC = T(2) * C * (R.a22 + R.a44), dS = T(2) * S * (R.a44 + R.a33);
        if (Rr > T(0)) {
            dC += R.sig * (dm * T(2) * C * (R.a22 - R.a44) + T(4) * be * S * R.a2344) / Rr;
            dS += R.sig * (dm * T(2) * S * (R.a44 - R.a33) + T(4) * be * C * R.a2344) / Rr;
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

// first device failure of the plan (later ones keep it)
ALF_D void adj_set_error(QueueState* q, unsigned code) { atomicCAS(&q->error, 0u, code); }

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
    s[0] = s[1] = s[2] = 0;
    if (rec < 32) {
        const int p = rec >> 1;
        s[0] = pair_a(p);
        s[1] = (rec & 1) ? pair_q(p) : pair_p(p);
        s[2] = (rec & 1) ? pair_p(p) : pair_q(p);
        return 3;
    }
    if (rec < 44) {
        s[0] = rec - 32;
        return 1;
    }
    return 0;
}

// support nodes of node (i, j) of a field (ns = 0 when a record points outside the grid)
ALF_D int support_nodes(int rec, int i, int j, int nx, int ny, unsigned m[3])
{
    int s[3];
    int ns = support_slots(rec, s);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int ii = i + slot_di(s[k]), jj = j + slot_dj(s[k]);
        if (k < ns && (ii < 0 || jj < 0 || ii >= nx || jj >= ny)) ns = 0;
        m[k] = (unsigned)(jj * nx + ii);
    }
    return ns;
}

// weights of every node and the in-degrees (the node records are zeroed before)
template <typename T>
__global__ void adj_weights_kernel(AdjLaunch a)
{
    const T* times = (const T*)a.times;
    AdjNode<T>* A = (AdjNode<T>*)a.nodes;
    const RegionP<T>* regions = (const RegionP<T>*)a.regions;
    // blockIdx.y strides over the fields, blockIdx.x and the threads over a field's nodes
    for (int f = blockIdx.y; f < a.nfields; f += gridDim.y) {
        const FieldDesc fd = a.fields[f];
        const unsigned N = (unsigned)(fd.nx * fd.ny);
        const int nx = fd.nx, ny = fd.ny;
        const unsigned* fb = a.frozen_bits + (size_t)f * frozen_words(a.box);
        AdjNode<T>* An = A + fd.node_off;
        for (unsigned n = blockIdx.x * blockDim.x + threadIdx.x; n < N; n += gridDim.x * blockDim.x) {
            const int i = (int)(n % (unsigned)nx), j = (int)(n / (unsigned)nx);
            T w0 = T(0), w1 = T(0), w2 = T(0), wt = T(0);
            const bool fz = frozen_at(fb, a.box, fd, i, j);
            if (fz) {
                // straight-ray time from the source: derivative by the source orientation
                if (i != fd.si || j != fd.sj) {
                    const int rs = a.region_map[fd.map_off + (long long)fd.sj * nx + fd.si];
                    const MatD m = a.mats[a.region_mat[rs]];
                    const double th = a.theta[(size_t)fd.sample * a.nregions + rs];
                    const double di = i - fd.si, dj = j - fd.sj;
                    const double dist = sqrt(di * di + dj * dj) * a.h[fd.sample];
                    const double dir = atan2(dj, di);
                    const double e = 1e-6;
                    wt = T((dist / group_speed64(m, a.group_model, dir - th - e) -
                            dist / group_speed64(m, a.group_model, dir - th + e)) / (2.0 * e));
                }
            } else {
                const int rec = a.records[fd.node_off + n];
                unsigned ms[3];
                const int ns = support_nodes(rec, i, j, nx, ny, ms);
                if (ns == 3) {
                    int s[3];
                    support_slots(rec, s);
                    const T* tf = times + fd.node_off;
                    const T tA = abs_(tf[ms[0]]), tB = abs_(tf[ms[1]]), tC = abs_(tf[ms[2]]);
                    const RegionP<T> R = regions[(size_t)fd.sample * a.nregions + a.region_map[fd.map_off + n]];
                    T w[3];
                    stencil_partials<T>(slot_di(s[0]), slot_dj(s[0]), slot_di(s[1]), slot_dj(s[1]), slot_di(s[2]),
                                        slot_dj(s[2]), tA, tB, tC, R, w, wt);
                    w0 = w[0];
                    w1 = w[1];
                    w2 = w[2];
                } else if (ns == 1) {
                    const RegionP<T> R = regions[(size_t)fd.sample * a.nregions + a.region_map[fd.map_off + n]];
                    const int q = rec - 32, cls = slot_cls(q);
                    const T d = cls == 0 ? R.dfb[0] : cls == 1 ? R.dfb[1] : cls == 2 ? R.dfb[2] : R.dfb[3];
                    w0 = T(1);
                    wt = (q >= 8 ? T(2) : T(1)) * d;
                }
#pragma unroll
                for (int k = 0; k < 3; ++k)
                    if (k < ns) atomicAdd(&An[ms[k]].indeg, T(1));
            }
            int s[3] = {0, 0, 0}, ns = 0, region = 0;
            if (fz) {
                region = a.region_map[fd.map_off + (long long)fd.sj * nx + fd.si];
            } else {
                const int rec = a.records[fd.node_off + n];
                unsigned ms[3];
                ns = support_nodes(rec, i, j, nx, ny, ms);
                support_slots(rec, s);
                region = a.region_map[fd.map_off + n];
            }
            AdjNode<T>& r = An[n];
            r.w[0] = w0;
            r.w[1] = w1;
            r.w[2] = w2;
            r.wt = wt;
            r.code = T(adj_code(s, ns, fz, a.nregions <= ADJ_SMEM_REGIONS ? region : 0));
        }
    }
}

template <typename T>
__global__ void adj_seed_kernel(AdjLaunch a, const T* dL_drec)
{
    AdjNode<T>* A = (AdjNode<T>*)a.nodes;
    const int total = a.nfields * a.nrec;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < total; k += gridDim.x * blockDim.x) {
        const int f = k / a.nrec, r = k % a.nrec;
        const FieldDesc fd = a.fields[f];
        const int ri = a.rec_ij[((size_t)fd.sample * a.nrec + r) * 2];
        const int rj = a.rec_ij[((size_t)fd.sample * a.nrec + r) * 2 + 1];
        atomicAdd(&A[fd.node_off + (long long)rj * fd.nx + ri].lam, dL_drec[k]);
    }
}

// first frontier of every field: the nodes no later node uses (one warp per field)
template <typename T>
__global__ void adj_frontier_kernel(AdjLaunch a)
{
    const unsigned lane = threadIdx.x & 31u;
    const AdjNode<T>* A = (const AdjNode<T>*)a.nodes;
    const size_t nw = (size_t)gridDim.x * blockDim.x / 32;
    for (size_t f = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) / 32; f < (size_t)a.nfields; f += nw) {
        const FieldDesc fd = a.fields[f];
        const unsigned N = (unsigned)(fd.nx * fd.ny);
        const AdjNode<T>* An = A + fd.node_off;
        unsigned* list = a.list[0] + fd.node_off;
        unsigned cnt = 0;
        for (unsigned base = 0; base < N; base += 32u) {
            const unsigned n = base + lane;
            const bool take = n < N && An[n].indeg == T(0);
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

// first frontier, one thread per node (field-resident schedule)
template <typename T>
__global__ void adj_frontier_flat_kernel(AdjLaunch a)
{
    const AdjNode<T>* A = (const AdjNode<T>*)a.nodes;
    for (int f = blockIdx.y; f < a.nfields; f += gridDim.y) {
        const FieldDesc fd = a.fields[f];
        const unsigned N = (unsigned)(fd.nx * fd.ny);
        const AdjNode<T>* An = A + fd.node_off;
        for (unsigned n = blockIdx.x * blockDim.x + threadIdx.x; n < N; n += gridDim.x * blockDim.x)
            if (An[n].indeg == T(0)) a.list[0][fd.node_off + atomicAdd(a.cnt + f, 1u)] = n;
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

// one Kahn round of every field (lockstep schedule): thread per frontier entry
template <typename T>
__global__ void adj_process_kernel(AdjLaunch a, int parity)
{
    const unsigned E = a.eoff[a.nfields];
    AdjNode<T>* A = (AdjNode<T>*)a.nodes;
    unsigned* nxt = a.cnt + (size_t)(parity ^ 1) * a.nfields;
    for (unsigned e = blockIdx.x * blockDim.x + threadIdx.x; e < E; e += gridDim.x * blockDim.x) {
        int lo = 0, hi = a.nfields;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (__ldg(a.eoff + mid) <= e) lo = mid; else hi = mid;
        }
        const FieldDesc fd = a.fields[lo];
        const unsigned n = a.list[parity][fd.node_off + (e - a.eoff[lo])];
        AdjNode<T>* An = A + fd.node_off;
        const T l = __ldcg(&An[n].lam);
        const T w0 = An[n].w[0], w1 = An[n].w[1], w2 = An[n].w[2];
        An[n].gn = l * An[n].wt;
        const unsigned* fbits = a.frozen_bits + (size_t)lo * frozen_words(a.box);
        const int nx = fd.nx;
        const int i = (int)(n % (unsigned)nx), j = (int)(n / (unsigned)nx);
        if (frozen_at(fbits, a.box, fd, i, j)) continue;
        unsigned ms[3];
        const int ns = support_nodes(a.records[fd.node_off + n], i, j, nx, fd.ny, ms);
        unsigned* list = a.list[parity ^ 1] + fd.node_off;
#pragma unroll
        for (int k = 0; k < 3; ++k)
            if (k < ns && release(&An[ms[k]], l * (k == 0 ? w0 : k == 1 ? w1 : w2)))
                list[atomicAdd(nxt + lo, 1u)] = ms[k];
    }
}

// Kahn rounds of one field by one warp, fields taken from a queue (largest first).  Only the owning
// warp touches a field's node records, and the warp barrier at the end of a round orders a round's
// contributions before the next round reads them (through L2: __ldcg).  With few regions the
// warp sums the region gradients in shared memory as it goes.  The sweep is a chain of rounds as long as
// the DAG is deep (thousands on a field of 10^5 nodes), so the latency of a round is the cost: the
// frontier lists stay in shared memory up to ADJ_CAP entries (beyond that, in the field's global lists),
// and a node's whole state is one sector already in L2.
#define ADJ_U 4      // frontier entries per lane per pass of the field-resident adjoint
#define ADJ_CAP 256  // frontier entries a warp keeps in shared memory per list

// FP32 fields: registers are capped at 48 (a bound of five CTAs of 256 threads; the kernel runs two per
// SM), so that two CTAs fit beside the two of the FP64 check, which runs on another stream after the solve.
template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 5 : 1)
    adj_warp_kernel(AdjLaunch a, double* grad, int smem_regions)
{
    extern __shared__ double s_acc[];
    constexpr unsigned FULL = 0xffffffffu;
    const unsigned lane = threadIdx.x & 31u;
    const unsigned below = (1u << lane) - 1u;
    double* acc = s_acc + (size_t)(threadIdx.x >> 5) * (smem_regions ? a.nregions : 0);
    unsigned* const s_lists = (unsigned*)(s_acc + (size_t)(blockDim.x >> 5) * (smem_regions ? a.nregions : 0)) +
                              (size_t)(threadIdx.x >> 5) * 2 * ADJ_CAP;
    AdjNode<T>* const A = (AdjNode<T>*)a.nodes;
    if (smem_regions)
        for (int r = (int)lane; r < a.nregions; r += 32) acc[r] = 0.0;
    __syncwarp();
    for (;;) {
        unsigned fi = 0u;
        if (lane == 0) fi = atomicAdd(a.head, 1u);
        fi = __shfl_sync(FULL, fi, 0);
        if (fi >= (unsigned)a.nfields) return;
        const unsigned f = __ldg(a.order + fi);
        const FieldDesc fd = a.fields[f];
        const int nx = fd.nx, ny = fd.ny;
        AdjNode<T>* const An = A + fd.node_off;
        unsigned* const list0 = a.list[0] + fd.node_off;
        unsigned* const list1 = a.list[1] + fd.node_off;
        unsigned nact = a.cnt[f], par = 0u;
        unsigned processed = 0u;  // Kahn's order reaches every node of a DAG exactly once
        bool first = true;        // the first frontier is all in the global list 0
        while (nact != 0u) {
            processed += nact;
            // entry e of a list: shared memory below ADJ_CAP (after the first round), else the global list
            const unsigned* LA = par ? list1 : list0;
            unsigned* LB = par ? list0 : list1;
            const unsigned* SA = s_lists + (par ? ADJ_CAP : 0u);
            unsigned* SB = s_lists + (par ? 0u : ADJ_CAP);
            unsigned nc = 0u;
            // up to ADJ_U entries per lane at once: their loads, then their releases, are independent, so a
            // round costs about one chain of memory round trips instead of one per 32 entries
            for (unsigned base = 0; base < nact; base += 32u * ADJ_U) {
                unsigned nn[ADJ_U], ms[ADJ_U][3];
                bool fresh[ADJ_U][3];
                T l[ADJ_U], w[ADJ_U][3], g[ADJ_U];
                int rec[ADJ_U];
#pragma unroll
                for (int u = 0; u < ADJ_U; ++u) {
                    const unsigned e = base + 32u * u + lane;
                    nn[u] = e < nact ? ((first || e >= ADJ_CAP) ? LA[e] : SA[e]) : ~0u;
                }
#pragma unroll
                for (int u = 0; u < ADJ_U; ++u) {
                    l[u] = w[u][0] = w[u][1] = w[u][2] = g[u] = T(0);
                    rec[u] = 255;
                    if (nn[u] != ~0u) {
                        const AdjNode<T>& r = An[nn[u]];
                        l[u] = __ldcg(&r.lam);
                        w[u][0] = r.w[0];
                        w[u][1] = r.w[1];
                        w[u][2] = r.w[2];
                        g[u] = l[u] * r.wt;
                        rec[u] = (int)r.code;
                    }
                }
#pragma unroll
                for (int u = 0; u < ADJ_U; ++u) {
                    fresh[u][0] = fresh[u][1] = fresh[u][2] = false;
                    ms[u][0] = ms[u][1] = ms[u][2] = 0u;
                    if (nn[u] == ~0u) continue;
                    const unsigned n = nn[u], code = (unsigned)rec[u];
                    if (smem_regions) {
                        if (g[u] != T(0)) atomicAdd(acc + ((code >> 15) & (ADJ_SMEM_REGIONS - 1)), (double)g[u]);
                    } else {
                        An[n].gn = g[u];
                    }
                    // the support nodes from their slots (checked against the grid when the code was made)
                    const int ns = (int)((code >> 12) & 3u);
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        const int q = (int)((code >> (4 * k)) & 15u);
                        ms[u][k] = (unsigned)((int)n + slot_dj(q) * nx + slot_di(q));
                        if (k < ns) fresh[u][k] = release(&An[ms[u][k]], l[u] * w[u][k]);
                    }
                }
#pragma unroll
                for (int u = 0; u < ADJ_U; ++u)
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        const unsigned b = __ballot_sync(FULL, fresh[u][k]);
                        if (fresh[u][k]) {
                            const unsigned idx = nc + __popc(b & below);
                            if (idx < ADJ_CAP) SB[idx] = ms[u][k];
                            else LB[idx] = ms[u][k];
                        }
                        nc += __popc(b);
                    }
            }
            __syncwarp();
            nact = nc;
            par ^= 1u;
            first = false;
        }
        // a node left unreleased sits on a cycle: the records do not describe one causal solve
        if (lane == 0 && processed != (unsigned)(nx * ny)) adj_set_error(a.q, ALF_ERR_INCONSISTENT_RECORDS);
        if (smem_regions) {
            // flush this field's region sums
            double* gb = grad + (size_t)fd.sample * a.nregions;
            for (int r = (int)lane; r < a.nregions; r += 32) {
                if (acc[r] != 0.0) atomicAdd(gb + r, acc[r]);
                acc[r] = 0.0;
            }
            __syncwarp();
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
    const AdjNode<T>* An = (const AdjNode<T>*)a.nodes + fd.node_off;
    const unsigned* fbits = a.frozen_bits + (size_t)f * frozen_words(a.box);
    const int rs = a.region_map[fd.map_off + (long long)fd.sj * fd.nx + fd.si];
    double* gb = grad + (size_t)fd.sample * a.nregions;
    const int N = fd.nx * fd.ny;
    for (int n = threadIdx.x; n < N; n += blockDim.x) {
        // every node is released once its users are processed; one that was not sits on a cycle
        if (An[n].indeg != T(0)) adj_set_error(a.q, ALF_ERR_INCONSISTENT_RECORDS);
        const T v = An[n].gn;
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
    if ((e = cudaMemsetAsync(a.nodes, 0, a.total_nodes * sizeof(AdjNode<T>), st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(grad, 0, (size_t)a.nsamples * a.nregions * sizeof(double), st)) != cudaSuccess) return e;
    const dim3 fgrid(8, (unsigned)std::min(a.nfields, 65535));
    adj_weights_kernel<T><<<fgrid, 256, 0, st>>>(a);
    adj_seed_kernel<T><<<64, 256, 0, st>>>(a, (const T*)dL_drec);
    note_launches(2);
    if (a.warp_grid > 0) {
        // field-resident schedule: flat frontier, then every field's rounds in one launch
        if ((e = cudaMemsetAsync(a.cnt, 0, (size_t)a.nfields * sizeof(unsigned), st)) != cudaSuccess) return e;
        if ((e = cudaMemsetAsync(a.head, 0, sizeof(unsigned), st)) != cudaSuccess) return e;
        adj_frontier_flat_kernel<T><<<fgrid, 256, 0, st>>>(a);
        const int smem_regions = a.nregions <= ADJ_SMEM_REGIONS ? 1 : 0;
        const size_t smem = (smem_regions ? (size_t)8 * a.nregions * sizeof(double) : 0) +
                            (size_t)8 * 2 * ADJ_CAP * sizeof(unsigned);
        adj_warp_kernel<T><<<a.warp_grid, 256, smem, st>>>(a, grad, smem_regions);
        note_launches(2);
        if (!smem_regions) {
            const size_t rs = a.nregions <= 4096 ? (size_t)a.nregions * sizeof(double) : 0;
            adj_reduce_kernel<T><<<a.nfields, 256, rs, st>>>(a, grad);
            note_launches(1);
        }
        return cudaGetLastError();
    }
    adj_frontier_kernel<T><<<std::max(1, std::min((a.nfields + 7) / 8, grid)), 256, 0, st>>>(a);
    note_launches(1);
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
    // the round cap ended the loop with nodes left in the frontiers
    if (*h_pending != 0ull && (e = launch_set_status(a.q, ALF_ERR_INCONSISTENT_RECORDS, st)) != cudaSuccess) return e;
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
