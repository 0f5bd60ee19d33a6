// alf_ray.cu -- Fermat plane-walk ray tracer (Sec. 5.1), one thread per
// (sample, source, receiver) ray.
//
// The ray starts at the receiver and walks toward the source through the
// source's travel-time field (reciprocity: the time from C to the source is
// the field value at C).  Each step:
//   * plane family (x = c, y = c, x - y = c, x + y = c) most perpendicular to
//     the last segment (the first step uses the direction to the target);
//   * the next plane of that family plane_step cells ahead of the current
//     point B along the family's normal, rounded to pass through grid nodes,
//     never beyond the target;
//   * cost(C) = |BC| / V_group(direction BC; node nearest the midpoint) + tau(C)
//     at the grid nodes C of that plane within +-halfwidth nodes of where the
//     current direction meets it;
//   * a parabola through every local minimum and its two neighbours, the
//     lowest vertex is the next point;
// and stops within stop_radius cells of the target, which is appended.
// The time along the finished polyline is integrated through the
// nearest-node cells (each segment split at x = k + 1/2, y = k + 1/2).
#include <type_traits>

#include "alf_internal.h"

namespace alf {

// Group speed along the angle phi from the material axis, in the ray's precision: the FP32 path stays on the
// FP32 pipe (the FP64 pipe runs at a small fraction of its rate) except where the inversion is ill-conditioned
// near the axes, the EXACT model's Newton solve and the shear modes' FP64 table.
ALF_D double group_speed_T(const MatD& m, const RegionP<double>& R, int model, double phi)
{
    (void)R;
    return group_speed64(m, model, phi);
}

ALF_D float group_speed_T(const MatD& m, const RegionP<float>& R, int model, float phi)
{
    if (m.env && !m.iso) return (float)env_speed64(m.env, (double)phi);
    if (model == 1) return (float)group_exact64(m, (double)phi);
    return group_paper32(m, R.a22, R.a33, R.a44, R.a2344, phi);
}

template <typename T>
struct RayCtx {
    int nx, ny;
    long long map_off;
    const uint32_t* map;
    const uint32_t* region_mat;
    const MatD* mats;
    const RegionP<T>* regions;  // of this sample
    const double* theta;        // of this sample
    int model;
    double h;
};

template <typename T>
ALF_D int node_at(const RayCtx<T>& c, T x, T y)
{
    int i = (int)floor(x + T(0.5)), j = (int)floor(y + T(0.5));
    i = min(max(i, 0), c.nx - 1);
    j = min(max(j, 0), c.ny - 1);
    return j * c.nx + i;
}

// straight-ray time of length len (cells) along (sx, sy) through node n.  FP64: the direction angle relative
// to the orientation as atan2 - theta; FP32: (sx, sy) rotated by the region's (cos, sin) of theta first, then
// one atan2, and the time in FP32.
ALF_D double piece_time(const RayCtx<double>& c, int n, double len, double sx, double sy)
{
    const int r = c.map[c.map_off + n];
    const MatD& m = c.mats[c.region_mat[r]];  // by reference: no local copy for the FP64 fallbacks
    const double V = group_speed_T(m, c.regions[r], c.model, atan2(sy, sx) - c.theta[r]);
    return len * c.h / V;
}

ALF_D float piece_time(const RayCtx<float>& c, int n, float len, float sx, float sy)
{
    const int r = c.map[c.map_off + n];
    const MatD& m = c.mats[c.region_mat[r]];
    const RegionP<float>& R = c.regions[r];
    const float phi = atan2f(sy * R.cth - sx * R.sth, sx * R.cth + sy * R.sth);
    const float V = group_speed_T(m, R, c.model, phi);
    return len * R.h / V;
}

// plane families: x = c, y = c, x - y = c, x + y = c; normal (fam_nx, fam_ny) and node step along the plane
ALF_D int fam_nx(int k) { return k == 1 ? 0 : 1; }
ALF_D int fam_ny(int k) { return k == 0 ? 0 : k == 1 ? 1 : k == 2 ? -1 : 1; }
ALF_D int fam_tx(int k) { return k == 0 ? 0 : 1; }
ALF_D int fam_ty(int k) { return k == 0 ? 1 : k == 1 ? 0 : k == 2 ? 1 : -1; }

template <typename T>
__global__ void ray_kernel(RayLaunch a)
{
    const long long ray = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nrays = (long long)a.nfields * a.nrec;
    if (ray >= nrays) return;
    const int f = (int)(ray / a.nrec), r = (int)(ray % a.nrec);
    const FieldDesc fd = a.fields[f];
    const int b = fd.sample;
    RayCtx<T> c;
    c.nx = fd.nx;
    c.ny = fd.ny;
    c.map_off = fd.map_off;
    c.map = a.region_map;
    c.region_mat = a.region_mat;
    c.mats = a.mats;
    c.regions = (const RegionP<T>*)a.regions + (size_t)b * a.nregions;
    c.theta = a.theta + (size_t)b * a.nregions;
    c.model = a.group_model;
    c.h = (double)((const RegionP<T>*)a.regions)[(size_t)b * a.nregions].h;
    const T* tau = (const T*)a.times + fd.node_off;
    T* pts = (T*)a.pts + (size_t)ray * a.max_pts * 2;

    const T xt = T(fd.si), yt = T(fd.sj);
    const T x0r = T(a.rec_ij[((size_t)b * a.nrec + r) * 2]), y0r = T(a.rec_ij[((size_t)b * a.nrec + r) * 2 + 1]);
    // one plane walk from the receiver to the source; famsel -1: the set most perpendicular to the ray at
    // every step, 0..3: one fixed set (Sec. 5.1).  Returns the point count.
    const T stop_r = T(a.stop_radius);
    auto walk = [&](int famsel, int& status) -> int {
    T bx = x0r, by = y0r;
    T dx = xt - bx, dy = yt - by;
    int np = 0;
    pts[0] = bx;
    pts[1] = by;
    np = 1;
    status = 1;
    while (np < a.max_pts) {
        const T rx = xt - bx, ry = yt - by;
        if (sqrt_(rx * rx + ry * ry) < stop_r) {
            pts[2 * np] = xt;
            pts[2 * np + 1] = yt;
            np++;
            status = 0;
            break;
        }
        const T dl = sqrt_(dx * dx + dy * dy);
        int fam = famsel;
        if (famsel < 0) {
            fam = 0;
            T bestc = T(-1);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const T nl = sqrt_(T(fam_nx(k) * fam_nx(k) + fam_ny(k) * fam_ny(k)));
                const T cs = abs_(dx * T(fam_nx(k)) + dy * T(fam_ny(k))) / (dl * nl);
                if (cs > bestc + T(1e-12)) {
                    bestc = cs;
                    fam = k;
                }
            }
        }
        const T nxf = T(fam_nx(fam)), nyf = T(fam_ny(fam));
        const T qB = nxf * bx + nyf * by, qT = nxf * xt + nyf * yt;
        const T dn = dx * nxf + dy * nyf;
        // a fixed set crosses its planes towards the target, each plane once
        const T sg = famsel >= 0 ? (qT - qB >= T(0) ? T(1) : T(-1)) : (dn >= T(0) ? T(1) : T(-1));
        const T scale = sqrt_(nxf * nxf + nyf * nyf);
        T qn = floor(qB + sg * T(a.plane_step) * scale + T(0.5));
        if (sg * (qn - qT) > T(0)) qn = floor(qT + T(0.5));
        if (sg * (qn - qB) < T(0.5)) {
            pts[2 * np] = xt;
            pts[2 * np + 1] = yt;
            np++;
            status = 0;
            break;
        }
        const T tt = (qn - qB) / dn;
        const T px = bx + tt * dx, py = by + tt * dy;
        T bxn, byn;
        if (fam == 0) {
            bxn = qn;
            byn = T(0);
        } else if (fam == 1) {
            bxn = T(0);
            byn = qn;
        } else if (fam == 2) {
            bxn = T(0);
            byn = -qn;
        } else {
            bxn = T(0);
            byn = qn;
        }
        const T stx = T(fam_tx(fam)), sty = T(fam_ty(fam));
        const T pc = fam == 0 ? py : px;
        int p0 = (int)floor(pc + T(0.5));
        {
            // the window is centred on the part of the plane inside the grid (a set of planes nearly
            // parallel to the ray meets the ray's line far off the grid)
            const int qi = (int)qn;
            int lo, hi;
            if (fam == 0) {
                lo = 0;
                hi = fd.ny - 1;
            } else if (fam == 1) {
                lo = 0;
                hi = fd.nx - 1;
            } else if (fam == 2) {
                lo = max(qi, 0);
                hi = min(fd.nx - 1, fd.ny - 1 + qi);
            } else {
                lo = max(qi - (fd.ny - 1), 0);
                hi = min(fd.nx - 1, qi);
            }
            if (lo <= hi) p0 = min(max(p0, lo), hi);
        }
        // candidates streamed in order of p: every local minimum (with its neighbours when they are
        // consecutive candidates) is refined by a parabola as soon as its right neighbour is known
        T best = alf_inf<T>();
        T bpos = T(0);
        T c1 = alf_inf<T>(), c2 = alf_inf<T>();
        int p1 = 0, p2 = 0, nv = 0;
        auto consider = [&](T cl, bool cl_ok, T ck, int pk, T cr, bool cr_ok) {
            if (!cl_ok) cl = alf_inf<T>();
            if (!cr_ok) cr = alf_inf<T>();
            if (!(ck < cl && ck <= cr)) return;
            T val = ck, off = T(0);
            if (cl_ok && cr_ok) {
                const T den = cl - T(2) * ck + cr;
                if (den > T(0)) {
                    off = (cl - cr) / (T(2) * den);
                    val = ck - (cl - cr) * (cl - cr) / (T(8) * den);
                }
            }
            if (val < best) {
                best = val;
                bpos = T(pk) + off;
            }
        };
        for (int p = p0 - a.halfwidth; p <= p0 + a.halfwidth; ++p) {
            const T cx = bxn + T(p) * stx, cy = byn + T(p) * sty;
            const int ci = (int)cx, cj = (int)cy;
            if (cx < T(0) || cy < T(0) || ci >= fd.nx || cj >= fd.ny) continue;
            const T tc = tau[(long long)cj * fd.nx + ci];
            if (!(tc < alf_inf<T>())) continue;
            const T sx = cx - bx, sy = cy - by;
            const T len = sqrt_(sx * sx + sy * sy);
            T seg = T(0);
            if (len > T(0)) {
                const int mn = node_at(c, T(0.5) * (bx + cx), T(0.5) * (by + cy));
                seg = piece_time(c, mn, len, sx, sy);
            }
            const T cost = seg + tc;
            if (nv >= 1) consider(c1, nv >= 2 && p1 == p2 - 1, c2, p2, cost, p == p2 + 1);
            c1 = c2;
            p1 = p2;
            c2 = cost;
            p2 = p;
            nv++;
        }
        if (nv == 0) break;
        consider(c1, nv >= 2 && p1 == p2 - 1, c2, p2, alf_inf<T>(), false);
        const T nxp = bxn + bpos * stx, nyp = byn + bpos * sty;
        dx = nxp - bx;
        dy = nyp - by;
        bx = nxp;
        by = nyp;
        pts[2 * np] = bx;
        pts[2 * np + 1] = by;
        np++;
    }
        return np;
    };
    // time along the polyline through the nearest-node cells
    auto path_time = [&](int np) -> T {
        T total = T(0);
        for (int s = 0; s + 1 < np; ++s) {
            const T x0 = pts[2 * s], y0 = pts[2 * s + 1], x1 = pts[2 * s + 2], y1 = pts[2 * s + 3];
            const T ddx = x1 - x0, ddy = y1 - y0;
            const T len = sqrt_(ddx * ddx + ddy * ddy);
            if (len == T(0)) continue;
            // crossings of x = k + 1/2 and y = k + 1/2 strictly inside the segment, merged in order
            const bool xinc = ddx > T(0), yinc = ddy > T(0);
            T kx = xinc ? floor(x0 - T(0.5)) + T(1.5) : ceil(x0 - T(0.5)) - T(0.5);
            T ky = yinc ? floor(y0 - T(0.5)) + T(1.5) : ceil(y0 - T(0.5)) - T(0.5);
            T tprev = T(0);
            for (int guard = 0; guard < 1 << 20; ++guard) {
                T tx = T(2), ty = T(2);
                if (ddx != T(0) && (xinc ? kx < x1 : kx > x1)) tx = (kx - x0) / ddx;
                if (ddy != T(0) && (yinc ? ky < y1 : ky > y1)) ty = (ky - y0) / ddy;
                T tn = fmin(tx, ty);
                const bool last = !(tn < T(1));
                if (last) tn = T(1);
                if (tn > tprev) {
                    const T tm = T(0.5) * (tprev + tn);
                    const int n = node_at(c, x0 + tm * ddx, y0 + tm * ddy);
                    total += piece_time(c, n, (tn - tprev) * len, ddx, ddy);
                    tprev = tn;
                }
                if (last) break;
                if (tx <= ty) kx += xinc ? T(1) : T(-1);
                if (ty <= tx) ky += yinc ? T(1) : T(-1);
            }
        }
        return total;
    };
    int status = 1, np = 0;
    T total = T(0);
    if (a.family == 4) {
        // the fastest of the four fixed sets (ties to the lower set), traced again to leave its points
        T best = alf_inf<T>();
        int bestf = -1;
        for (int fam = 0; fam < 4; ++fam) {
            int st = 1;
            const int n = walk(fam, st);
            if (st != 0) continue;
            const T tt = path_time(n);
            if (tt < best) {
                best = tt;
                bestf = fam;
            }
        }
        if (bestf < 0) {
            np = walk(0, status);
            if (a.ray_time) total = path_time(np);
        } else {
            np = walk(bestf, status);
            total = best;
        }
    } else {
        np = walk(a.family, status);
        if (a.ray_time) total = path_time(np);
    }
    a.npts[ray] = np;
    if (a.ray_status) a.ray_status[ray] = status;
    if (status != 0) atomicCAS(a.error, 0u, (unsigned)ALF_ERR_RAY_INCOMPLETE);
    if (a.ray_time) ((T*)a.ray_time)[ray] = total;
}

// ---------------------------------------------------------------------------
// Gradient of the ray times along their fixed paths with respect to the region
// orientations: a piece of length len (cells) in region r along direction dir
// takes len h / V(dir - theta_r), so d/dtheta_r = len h V'(dir - theta_r) / V^2,
// with V' by an FP64 central difference of the group speed.  Each ray adds
// dL/dT_ray times that to the gradient of its sample; consecutive pieces in one
// region are summed before the atomic add.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void ray_grad_kernel(RayLaunch a, const T* dL_dray, double* grad)
{
    const long long ray = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nrays = (long long)a.nfields * a.nrec;
    if (ray >= nrays) return;
    const double wray = (double)dL_dray[ray];
    const int np = a.npts[ray];
    if (wray == 0.0 || np < 2) return;
    const int f = (int)(ray / a.nrec);
    const FieldDesc fd = a.fields[f];
    const int b = fd.sample;
    const double h = a.h_of_sample[b];
    const double* theta = a.theta + (size_t)b * a.nregions;
    const uint32_t* map = a.region_map + fd.map_off;
    double* gb = grad + (size_t)b * a.nregions;
    const T* pts = (const T*)a.pts + (size_t)ray * a.max_pts * 2;
    int cur = -1;
    double acc = 0.0;
    for (int s = 0; s + 1 < np; ++s) {
        const double x0 = pts[2 * s], y0 = pts[2 * s + 1], x1 = pts[2 * s + 2], y1 = pts[2 * s + 3];
        const double ddx = x1 - x0, ddy = y1 - y0;
        const double len = sqrt(ddx * ddx + ddy * ddy);
        if (len == 0.0) continue;
        const double dir = atan2(ddy, ddx);
        const bool xinc = ddx > 0.0, yinc = ddy > 0.0;
        double kx = xinc ? floor(x0 - 0.5) + 1.5 : ceil(x0 - 0.5) - 0.5;
        double ky = yinc ? floor(y0 - 0.5) + 1.5 : ceil(y0 - 0.5) - 0.5;
        double tprev = 0.0;
        for (int guard = 0; guard < 1 << 20; ++guard) {
            double tx = 2.0, ty = 2.0;
            if (ddx != 0.0 && (xinc ? kx < x1 : kx > x1)) tx = (kx - x0) / ddx;
            if (ddy != 0.0 && (yinc ? ky < y1 : ky > y1)) ty = (ky - y0) / ddy;
            double tn = fmin(tx, ty);
            const bool last = !(tn < 1.0);
            if (last) tn = 1.0;
            if (tn > tprev) {
                const double tm = 0.5 * (tprev + tn);
                int i = (int)floor(x0 + tm * ddx + 0.5), j = (int)floor(y0 + tm * ddy + 0.5);
                i = min(max(i, 0), fd.nx - 1);
                j = min(max(j, 0), fd.ny - 1);
                const int r = map[(long long)j * fd.nx + i];
                const MatD& m = a.mats[a.region_mat[r]];
                if (!m.iso) {
                    const double phi = dir - theta[r], e = 1e-6;
                    const double V = group_speed64(m, a.group_model, phi);
                    const double dV = (group_speed64(m, a.group_model, phi + e) -
                                       group_speed64(m, a.group_model, phi - e)) / (2.0 * e);
                    if (r != cur) {
                        if (cur >= 0 && acc != 0.0) atomicAdd(gb + cur, wray * acc);
                        cur = r;
                        acc = 0.0;
                    }
                    acc += (tn - tprev) * len * h * dV / (V * V);
                }
                tprev = tn;
            }
            if (last) break;
            if (tx <= ty) kx += xinc ? 1.0 : -1.0;
            if (ty <= tx) ky += yinc ? 1.0 : -1.0;
        }
    }
    if (cur >= 0 && acc != 0.0) atomicAdd(gb + cur, wray * acc);
}

cudaError_t launch_ray_gradient(int precision, const RayLaunch& a, const void* dL_dray, double* grad, int nsamples,
                                cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(grad, 0, (size_t)nsamples * a.nregions * sizeof(double), st);
    if (e != cudaSuccess) return e;
    const long long nrays = (long long)a.nfields * a.nrec;
    if (nrays == 0) return cudaSuccess;
    const int bs = 128;
    const long long gs = (nrays + bs - 1) / bs;
    if (precision == ALF_FP64) ray_grad_kernel<double><<<(unsigned)gs, bs, 0, st>>>(a, (const double*)dL_dray, grad);
    else ray_grad_kernel<float><<<(unsigned)gs, bs, 0, st>>>(a, (const float*)dL_dray, grad);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_rays(int precision, const RayLaunch& a, cudaStream_t st)
{
    const long long nrays = (long long)a.nfields * a.nrec;
    if (nrays == 0) return cudaSuccess;
    const int bs = 64;
    const long long gs = (nrays + bs - 1) / bs;
    if (precision == ALF_FP64) ray_kernel<double><<<(unsigned)gs, bs, 0, st>>>(a);
    else ray_kernel<float><<<(unsigned)gs, bs, 0, st>>>(a);
    note_launches(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Packing of the traced rays (alf_pack_rays): offsets[r] = the points of the rays before r (an exclusive
// prefix sum of the point counts, in blocks of ALF_PACK_BLOCK rays: every block's sum, one block's scan of
// those sums, every block's own scan), then one warp per ray copies its points behind those of the rays
// before it.  A ray's slots past its count are not read, so the copy moves only the path's points.
// ---------------------------------------------------------------------------
#define ALF_PACK_BLOCK 1024

ALF_D long long ray_count(const int32_t* npts, long long r, int max_pts)
{
    const int n = npts[r];
    return n < 0 ? 0 : (n > max_pts ? max_pts : n);
}

// inclusive scan of v over the block (blockDim.x = ALF_PACK_BLOCK); returns this thread's inclusive sum
ALF_D long long block_inclusive_scan(long long v, long long* s_warp)
{
    const unsigned lane = threadIdx.x & 31u, wid = threadIdx.x >> 5;
    for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, v, o);
        if ((int)lane >= o) v += y;
    }
    if (lane == 31u) s_warp[wid] = v;
    __syncthreads();
    if (wid == 0) {
        long long w = lane < (blockDim.x >> 5) ? s_warp[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const long long y = __shfl_up_sync(0xffffffffu, w, o);
            if ((int)lane >= o) w += y;
        }
        s_warp[lane] = w;
    }
    __syncthreads();
    if (wid > 0) v += s_warp[wid - 1];
    return v;
}

__global__ void __launch_bounds__(ALF_PACK_BLOCK) ray_block_sums_kernel(const int32_t* npts, long long nrays,
                                                                         int max_pts, long long* block_sums)
{
    __shared__ long long s_warp[32];
    const long long r = (long long)blockIdx.x * ALF_PACK_BLOCK + threadIdx.x;
    const long long v = block_inclusive_scan(r < nrays ? ray_count(npts, r, max_pts) : 0, s_warp);
    if (threadIdx.x == ALF_PACK_BLOCK - 1) block_sums[blockIdx.x] = v;
}

// exclusive scan of the block sums in place, by one block; block_sums[nblocks] = the total
__global__ void __launch_bounds__(ALF_PACK_BLOCK) ray_scan_sums_kernel(long long* block_sums, long long nblocks)
{
    __shared__ long long s_warp[32];
    __shared__ long long s_carry;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (long long base = 0; base < nblocks; base += ALF_PACK_BLOCK) {
        const long long k = base + threadIdx.x;
        const long long v = k < nblocks ? block_sums[k] : 0;
        const long long incl = block_inclusive_scan(v, s_warp);
        const long long carry = s_carry;
        if (k < nblocks) block_sums[k] = carry + incl - v;
        __syncthreads();
        if (threadIdx.x == ALF_PACK_BLOCK - 1) s_carry = carry + incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) block_sums[nblocks] = s_carry;
}

__global__ void __launch_bounds__(ALF_PACK_BLOCK) ray_offsets_kernel(const int32_t* npts, long long nrays, int max_pts,
                                                                      const long long* block_off, long long* offsets)
{
    __shared__ long long s_warp[32];
    const long long r = (long long)blockIdx.x * ALF_PACK_BLOCK + threadIdx.x;
    const long long v = r < nrays ? ray_count(npts, r, max_pts) : 0;
    const long long incl = block_inclusive_scan(v, s_warp);
    if (r < nrays) offsets[r] = block_off[blockIdx.x] + incl - v;
    if (r == nrays - 1) offsets[nrays] = block_off[blockIdx.x] + incl;
}

template <typename T>
__global__ void ray_pack_kernel(const T* pts, const int32_t* npts, long long nrays, int max_pts,
                                const long long* offsets, T* packed)
{
    using T2 = typename std::conditional<sizeof(T) == 4, float2, double2>::type;
    const long long warps = (long long)gridDim.x * blockDim.x / 32;
    const unsigned lane = threadIdx.x & 31u;
    for (long long r = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / 32; r < nrays; r += warps) {
        const long long n = ray_count(npts, r, max_pts), off = offsets[r];
        const T2* src = (const T2*)pts + r * max_pts;
        T2* dst = (T2*)packed + off;
        for (long long k = lane; k < n; k += 32) dst[k] = src[k];
    }
}

cudaError_t launch_pack_rays(int precision, const void* pts, const int32_t* npts, long long nrays, int max_pts,
                             long long* block_sums, void* packed, long long* offsets, int grid, cudaStream_t st)
{
    if (nrays <= 0) return cudaMemsetAsync(offsets, 0, sizeof(long long), st);
    const long long nb = (nrays + ALF_PACK_BLOCK - 1) / ALF_PACK_BLOCK;
    ray_block_sums_kernel<<<(unsigned)nb, ALF_PACK_BLOCK, 0, st>>>(npts, nrays, max_pts, block_sums);
    ray_scan_sums_kernel<<<1, ALF_PACK_BLOCK, 0, st>>>(block_sums, nb);
    ray_offsets_kernel<<<(unsigned)nb, ALF_PACK_BLOCK, 0, st>>>(npts, nrays, max_pts, block_sums, offsets);
    if (precision == ALF_FP64)
        ray_pack_kernel<double><<<grid, 256, 0, st>>>((const double*)pts, npts, nrays, max_pts, offsets, (double*)packed);
    else
        ray_pack_kernel<float><<<grid, 256, 0, st>>>((const float*)pts, npts, nrays, max_pts, offsets, (float*)packed);
    note_launches(4);
    return cudaGetLastError();
}

}  // namespace alf
