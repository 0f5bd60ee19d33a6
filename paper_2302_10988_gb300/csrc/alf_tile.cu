// alf_tile.cu -- the active-tile schedule of the sweep (sweep = 4).  Each field's grid is cut into 8 x 8
// tiles.  A warp loads a tile with a halo of two nodes into shared memory and iterates the local operator F
// (Secs. 4.2-4.3) on it until no node of the tile changes (a warp vote); a tile whose border nodes changed
// activates the neighbouring tiles whose stencils read them.  Rounds of active tiles run until none is left.
// F has a unique fixed point (the causal key order of Sec. 2), so the fields and records are those of the
// other schedules, bit for bit.  The schedule has no front band: every node of an active tile is evaluated.
#include "alf_internal.h"
#include "alf_sweep.cuh"

namespace alf {

#define TILE_N 8             // tile side in nodes (64 nodes: two per lane of a warp)
#define TILE_S (TILE_N + 4)  // side of the tile with its two-node halo
#define TILE_WARPS 8         // warps of a field's CTA; each works on one tile at a time
#define TILE_ITERS 64        // iterations per visit; a tile still changing after them is queued again

ALF_D void tile_set_error(QueueState* q, unsigned code) { atomicCAS(&q->error, 0u, code); }

// The tile nodes (bit 8 * lj + li) that a neighbouring tile's stencils read, by direction of that tile:
// 0 left, 1 right, 2 down, 3 up, 4 down-left, 5 down-right, 6 up-left, 7 up-right.  The stencil reaches two
// nodes along the axes and one along the diagonals, so the sides give two rows or columns, the corners one node.
ALF_D unsigned long long tile_border(int d)
{
    switch (d) {
    case 0: return 0x0303030303030303ull;
    case 1: return 0xC0C0C0C0C0C0C0C0ull;
    case 2: return 0x000000000000FFFFull;
    case 3: return 0xFFFF000000000000ull;
    case 4: return 0x0000000000000001ull;
    case 5: return 0x0000000000000080ull;
    case 6: return 0x0100000000000000ull;
    default: return 0x8000000000000000ull;
    }
}

// the nodes of the tile in the stencil of the tile node (li, lj)
ALF_D unsigned long long tile_stencil_mask(int li, int lj)
{
    unsigned long long m = 0ull;
#pragma unroll
    for (int q = 0; q < 12; ++q) {
        const int x = li + sdi(q), y = lj + sdj(q);
        if (x >= 0 && x < TILE_N && y >= 0 && y < TILE_N) m |= 1ull << (y * TILE_N + x);
    }
    return m;
}

// F at the tile node at buffer index s (grid node n): the twelve stencil times from the buffer, where a node
// outside the grid holds infinity
template <typename T, bool VT>
ALF_D T tile_eval(const T* buf, int s, int n, int nx, const uint32_t* map, const RegionP<T>* reg, int& rc)
{
    T nb[12];
#pragma unroll
    for (int q = 0; q < 12; ++q) nb[q] = buf[s + sdj(q) * TILE_S + sdi(q)];
    const RegionP<T> R = reg[__ldg(map + n)];
    return local_F<T, VT>(nb, n, nx, R, rc);
}

// adds tile u to the next round's list unless it is already there
ALF_D void tile_activate(unsigned* bm, unsigned* next_list, unsigned* next_count, unsigned u)
{
    const unsigned bit = 1u << (u & 31u);
    if (!(atomicOr(bm + (u >> 5), bit) & bit)) next_list[atomicAdd(next_count, 1u)] = u;
}

// One CTA per field, fields taken from the queue in the order `order`.  The field's tile bitmap (a tile in
// the next round's list) is in shared memory when it fits in smem_words words, else in the field's global
// bitmap; the round's lists are the field's segments of the dirty lists.
template <typename T, bool VT>
__global__ void __launch_bounds__(TILE_WARPS * 32, sizeof(T) == 4 ? 2 : 1)
    fim_tile_kernel(FimLaunch a, const unsigned* order, unsigned smem_words)
{
    extern __shared__ unsigned s_tbm[];
    __shared__ T s_buf[TILE_WARPS][TILE_S * TILE_S];
    __shared__ unsigned s_f[2];  // field index, error code
    __shared__ unsigned s_next;  // tiles in the next round's list
    const T inf = alf_inf<T>();
    const unsigned lane = threadIdx.x & 31u, wid = threadIdx.x >> 5;
    T* const buf = s_buf[wid];
    // the lane's two tile nodes: (li, lj0) and (li, lj0 + 4), bits lane and lane + 32 of a tile mask
    const int li = (int)(lane & 7u), lj0 = (int)(lane >> 3), lj1 = lj0 + 4;
    const unsigned long long nbm0 = tile_stencil_mask(li, lj0), nbm1 = tile_stencil_mask(li, lj1);
    const int s0 = (lj0 + 2) * TILE_S + li + 2, s1 = (lj1 + 2) * TILE_S + li + 2;
    for (;;) {
        if (threadIdx.x == 0) {
            s_f[0] = atomicAdd(&a.q->head, 1u);
            s_f[1] = *reinterpret_cast<const volatile unsigned*>(&a.q->error);
        }
        __syncthreads();
        const unsigned fi = s_f[0], err = s_f[1];
        __syncthreads();
        if (fi >= (unsigned)a.nfields || err != 0u) return;
        const unsigned f = __ldg(order + fi);
        const FieldDesc fd = a.fields[f];
        T* const tf = (T*)a.times + fd.node_off;
        const int nx = fd.nx, ny = fd.ny;
        const uint32_t* const map = a.region_map + fd.map_off;
        const RegionP<T>* const reg = (const RegionP<T>*)a.regions + (size_t)fd.sample * a.nregions;
        uint8_t* const rec = a.records ? a.records + fd.node_off : nullptr;
        const int ntx = (nx + TILE_N - 1) / TILE_N, nty = (ny + TILE_N - 1) / TILE_N;
        const unsigned words = ((unsigned)(ntx * nty) + 31u) / 32u;
        unsigned* const bm = words <= smem_words ? s_tbm : a.bitmap + a.bm_off[f];
        unsigned* const L0 = a.list[0] + fd.node_off;
        unsigned* const L1 = a.list[1] + fd.node_off;
        const unsigned max_rounds = a.max_rounds_per_node * (unsigned)(nx + ny);
        // the first round's tiles: those that meet the square of half-width box + 2 around the source (the
        // frozen box and the nodes next to it)
        const int r = a.box + 2;
        const int tx0 = max(fd.si - r, 0) / TILE_N, tx1 = min(fd.si + r, nx - 1) / TILE_N;
        const int ty0 = max(fd.sj - r, 0) / TILE_N, ty1 = min(fd.sj + r, ny - 1) / TILE_N;
        const unsigned sw = (unsigned)(tx1 - tx0 + 1);
        unsigned nact = sw * (unsigned)(ty1 - ty0 + 1);
        for (unsigned k = threadIdx.x; k < words; k += blockDim.x) bm[k] = 0u;
        for (unsigned k = threadIdx.x; k < nact; k += blockDim.x)
            L0[k] = (unsigned)(ty0 + (int)(k / sw)) * (unsigned)ntx + (unsigned)tx0 + k % sw;
        __syncthreads();
        unsigned par = 0u, rounds = 0u;
        unsigned evals = 0u, visits = 0u;  // this warp's, on this field
        bool ok = true;
        while (nact != 0u) {
            if (++rounds > max_rounds) {
                ok = false;
                break;
            }
            const unsigned* LA = par ? L1 : L0;
            unsigned* LB = par ? L0 : L1;
            // the round's tiles leave the bitmap before any is worked on, so that a tile activated again
            // during the round enters the next round's list once
            for (unsigned k = threadIdx.x; k < nact; k += blockDim.x) {
                const unsigned t = LA[k];
                atomicAnd(bm + (t >> 5), ~(1u << (t & 31u)));
            }
            if (threadIdx.x == 0) s_next = 0u;
            __syncthreads();
            for (unsigned k = wid; k < nact; k += TILE_WARPS) {
                const unsigned t = LA[k];
                const int tx = (int)(t % (unsigned)ntx), ty = (int)(t / (unsigned)ntx);
                const int i0 = tx * TILE_N, j0 = ty * TILE_N;
                for (int s = (int)lane; s < TILE_S * TILE_S; s += 32) {
                    const int gi = i0 - 2 + s % TILE_S, gj = j0 - 2 + s / TILE_S;
                    buf[s] = (gi >= 0 && gi < nx && gj >= 0 && gj < ny) ? tf[gj * nx + gi] : inf;
                }
                __syncwarp();
                const int gi = i0 + li, gj0 = j0 + lj0, gj1 = j0 + lj1;
                const int n0 = gj0 * nx + gi, n1 = gj1 * nx + gi;
                // nodes that are evaluated: inside the grid and not frozen (frozen times carry the sign bit)
                const bool e0 = gi < nx && gj0 < ny && !neg_bit(buf[s0]);
                const bool e1 = gi < nx && gj1 < ny && !neg_bit(buf[s1]);
                int rc0 = -1, rc1 = -1;  // record of the node's last evaluation in this visit (-1: none)
                // changed: the tile's nodes that changed in the last iteration; any: in the whole visit
                unsigned long long changed = 0ull, any = 0ull;
                int it = 0;
                do {
                    // an iteration reads the values of the last one (Jacobi within the tile): the first
                    // evaluates every node, later ones the nodes with a changed node in their stencil
                    const bool d0 = e0 && (it == 0 || (changed & nbm0) != 0ull);
                    const bool d1 = e1 && (it == 0 || (changed & nbm1) != 0ull);
                    const T o0 = buf[s0], o1 = buf[s1];
                    T v0 = o0, v1 = o1;
                    int r0 = 0, r1 = 0;
                    // one evaluation site for both nodes (F is large)
#pragma unroll 1
                    for (int h = 0; h < 2; ++h) {
                        if (!(h ? d1 : d0)) continue;
                        int rh;
                        const T v = tile_eval<T, VT>(buf, h ? s1 : s0, h ? n1 : n0, nx, map, reg, rh);
                        if (h) {
                            v1 = v;
                            r1 = rh;
                        } else {
                            v0 = v;
                            r0 = rh;
                        }
                    }
                    __syncwarp();
                    const bool c0 = d0 && !same_bits(v0, o0), c1 = d1 && !same_bits(v1, o1);
                    if (c0) buf[s0] = v0;
                    if (c1) buf[s1] = v1;
                    if (d0) rc0 = r0;
                    if (d1) rc1 = r1;
                    changed = (unsigned long long)__ballot_sync(0xffffffffu, c0) |
                              ((unsigned long long)__ballot_sync(0xffffffffu, c1) << 32);
                    any |= changed;
                    evals += (unsigned)__popc(__ballot_sync(0xffffffffu, d0)) +
                             (unsigned)__popc(__ballot_sync(0xffffffffu, d1));
                    __syncwarp();
                } while (changed != 0ull && ++it < TILE_ITERS);
                ++visits;
                // the visit's changes to the field, then the tiles that read them (and the tile itself if it
                // is still changing)
                if ((any >> lane) & 1ull) tf[n0] = buf[s0];
                if ((any >> (lane + 32u)) & 1ull) tf[n1] = buf[s1];
                if (rec && rc0 >= 0) rec[n0] = (uint8_t)rc0;
                if (rec && rc1 >= 0) rec[n1] = (uint8_t)rc1;
                if (lane < 8u && (any & tile_border((int)lane)) != 0ull) {
                    const int ux = tx + (lane == 0u || lane == 4u || lane == 6u ? -1 : lane == 2u || lane == 3u ? 0 : 1);
                    const int uy = ty + (lane < 2u ? 0 : lane == 2u || lane == 4u || lane == 5u ? -1 : 1);
                    if (ux >= 0 && ux < ntx && uy >= 0 && uy < nty) tile_activate(bm, LB, &s_next, (unsigned)(uy * ntx + ux));
                }
                if (lane == 8u && changed != 0ull) tile_activate(bm, LB, &s_next, t);
                __syncwarp();
            }
            __syncthreads();
            nact = s_next;
            __syncthreads();
            par ^= 1u;
        }
        // counts: evaluations, and the nodes of the visited tiles as the entries scanned
        if (lane == 0u) {
            atomicAdd(&a.q->visits, (unsigned long long)evals);
            atomicAdd(&a.q->dirty, (unsigned long long)visits * (TILE_N * TILE_N));
        }
        if (threadIdx.x == 0) {
            if (!ok) tile_set_error(a.q, ALF_ERR_NOT_CONVERGED);
            a.rounds[f] = rounds;
            atomicMax(&a.q->rounds, (unsigned long long)rounds);
        }
        __syncthreads();
    }
}

template <typename T, bool VT>
static cudaError_t fim_tile_smem(unsigned smem_words, size_t* smem)
{
    *smem = (size_t)smem_words * sizeof(unsigned);
    if (*smem + sizeof(T) * TILE_WARPS * TILE_S * TILE_S <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(fim_tile_kernel<T, VT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)*smem);
}

template <typename T, bool VT>
static cudaError_t fim_tile_t(const FimLaunch& a, const unsigned* order, unsigned smem_words, int grid,
                              cudaStream_t st)
{
    size_t smem = 0;
    const cudaError_t e = fim_tile_smem<T, VT>(smem_words, &smem);
    if (e != cudaSuccess) return e;
    fim_tile_kernel<T, VT><<<grid, TILE_WARPS * 32, smem, st>>>(a, order, smem_words);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_fim_tile(int precision, const FimLaunch& a, const unsigned* order, unsigned smem_words, int grid,
                            cudaStream_t st)
{
    if (a.vtable)
        return precision == ALF_FP64 ? fim_tile_t<double, true>(a, order, smem_words, grid, st)
                                     : fim_tile_t<float, true>(a, order, smem_words, grid, st);
    return precision == ALF_FP64 ? fim_tile_t<double, false>(a, order, smem_words, grid, st)
                                 : fim_tile_t<float, false>(a, order, smem_words, grid, st);
}

template <typename T, bool VT>
static int fim_tile_occ(unsigned smem_words, int nsm)
{
    size_t smem = 0;
    if (fim_tile_smem<T, VT>(smem_words, &smem) != cudaSuccess) return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fim_tile_kernel<T, VT>, TILE_WARPS * 32, smem) != cudaSuccess)
        return 0;
    return n * nsm;
}

int fim_tile_grid(int precision, unsigned smem_words, bool vt, int nsm)
{
    if (vt) return precision == ALF_FP64 ? fim_tile_occ<double, true>(smem_words, nsm)
                                         : fim_tile_occ<float, true>(smem_words, nsm);
    return precision == ALF_FP64 ? fim_tile_occ<double, false>(smem_words, nsm)
                                 : fim_tile_occ<float, false>(smem_words, nsm);
}

unsigned fim_tile_words(int nx, int ny)
{
    const unsigned tiles = (unsigned)(((nx + TILE_N - 1) / TILE_N) * ((ny + TILE_N - 1) / TILE_N));
    return (tiles + 31u) / 32u;
}

}  // namespace alf
