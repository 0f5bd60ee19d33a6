// alf_check.cuh -- the FP64 convergence check of one node of a solved field (the precision policy's
// final check): the update U(S_D) of Secs. 4.2-4.3 in double precision with S_D the node's frozen neighbours
// and the neighbours whose key (tau, index) precedes its own.  Used by the check kernel and by the solve
// kernel that checks each field as soon as it is solved.
#pragma once

#include "alf_internal.h"
#include "alf_sweep.cuh"

namespace alf {

ALF_D bool box_frozen(const unsigned* bits, int box, const FieldDesc& fd, int i, int j)
{
    const int di = i - fd.si, dj = j - fd.sj;
    if (di < -box || di > box || dj < -box || dj > box) return false;
    const int bit = (dj + box) * (2 * box + 1) + (di + box);
    return (bits[bit >> 5] >> (bit & 31)) & 1u;
}

// At a fixed point, F at D reads exactly the neighbours that precede D in key
// order, so the check evaluates in FP64 the update U of that known set.  The
// FP64 pipe is the bottleneck, so only what needs it runs there: feasibility
// and the square metrics tau_C - tau_B are exact on the stored times (a
// difference of two FP32 times within a factor two of each other is exact in
// FP32; a node with any other feasible square takes the all-FP64 path), the
// best square is found by exact comparisons, and only its stencil time (the
// next best's when it is not usable) is evaluated in FP64.  Triangle metrics
// and the fallback, which need FP64 arithmetic, are evaluated only when no
// square is usable.  All decisions are the ones an all-FP64 evaluation makes.
template <typename T, bool VT>
ALF_D double check_pair_time(int bp, const T (&t)[12], const RegionP<double>& R, int& rec)
{
    // the pair's geometry as FP64 constants chosen by predicated moves (no integer-to-FP64 conversion, which
    // runs on the slow FP64 pipe); dxC, dyC: C - A
    double xA = 0.0, yA = 0.0, xB = 0.0, yB = 0.0, dxC = 0.0, dyC = 0.0;
    int r = 255;
    T tA = T(0), tB = T(0), tC = T(0);
#pragma unroll
    for (int p = 0; p < 16; ++p)
        if (p == bp) {
            const bool m1 = t[pp(p)] <= t[pq(p)];
            xA = double(sdi(pa(p)));
            yA = double(sdj(pa(p)));
            xB = m1 ? double(sdi(pp(p))) : double(sdi(pq(p)));
            yB = m1 ? double(sdj(pp(p))) : double(sdj(pq(p)));
            dxC = m1 ? double(sdi(pq(p)) - sdi(pa(p))) : double(sdi(pp(p)) - sdi(pa(p)));
            dyC = m1 ? double(sdj(pq(p)) - sdj(pa(p))) : double(sdj(pp(p)) - sdj(pa(p)));
            tA = t[pa(p)];
            tB = m1 ? t[pp(p)] : t[pq(p)];
            tC = m1 ? t[pq(p)] : t[pp(p)];
            r = 2 * p + (m1 ? 0 : 1);
        }
    // the stencil time with its geometry scaled by den = tau_C - tau_A (> 0 for a feasible pair): the
    // cross product scales by den and the phase term by den^2, so tau_D needs no division, and one
    // reciprocal square root instead of a square root and two divisions.  The differences of FP32
    // times are exact in FP64.
    const double num = (double)tB - (double)tA, den = (double)tC - (double)tA;
    const double Ex = xA * den + num * dxC, Ey = yA * den + num * dyC;
    const double ux = xB * den - Ex, uy = yB * den - Ey;
    const double cross = fabs(yB * Ex - xB * Ey);
    const double v = (double)tB + R.h * cross * rsqrt(phase_L<double, VT>(R, ux, uy));
    rec = r;
    return v > (double)tC ? v : alf_inf<double>();
}

// The check of node `me` of field fd (times tf, frozen bitmap fb, region constants `regions` and region map
// `map` of the field's sample).  Returns false, with F = its time and rec = 254 (frozen) or 255 (no value),
// for a node the check skips; else true with F = U(S_D) in FP64 and rec its record; tme is the stored time.
template <typename T, bool VT>
ALF_D bool check_node(const T* tf, const unsigned* fb, int box, const FieldDesc& fd, int me,
                      const RegionP<double>* regions, const uint32_t* map, double& F, int& rec, T& tme)
{
    const double inf64 = alf_inf<double>();
    const int i = me % fd.nx, j = me / fd.nx;
    tme = abs_(tf[me]);
    // frozen nodes and nodes without a value keep their time (records 254 / 255)
    const bool fz = box_frozen(fb, box, fd, i, j);
    if (fz || !(tme < alf_inf<T>())) {
        F = (double)tme;
        rec = fz ? 254 : 255;
        return false;
    }
    T t[12];
    unsigned known = 0u;
    const SlotInGrid in = slots_in_grid(i, j, fd.nx, fd.ny);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        const int ii = i + sdi(k), jj = j + sdj(k);
        t[k] = alf_inf<T>();
        if (!in.v[k]) continue;
        const T v = abs_(tf[me + sdj(k) * fd.nx + sdi(k)]);
        t[k] = v;
        const bool before = sord(k) < 12 ? v <= tme : v < tme;
        if (box_frozen(fb, box, fd, ii, jj) || before) known |= 1u << k;
    }
    const RegionP<double> R = regions[map[me]];
    // feasible pairs (exact comparisons) and the square metrics
    unsigned feas = 0u;
    bool exact = true;
    T msq[8];
#pragma unroll
    for (int p = 0; p < 16; ++p) {
        const T tA = t[pa(p)], tP = t[pp(p)], tQ = t[pq(p)];
        const bool ok = ((known >> pa(p)) & (known >> pp(p)) & (known >> pq(p)) & 1u) && tA < tP && tA < tQ;
        if (ok) feas |= 1u << p;
        if (p < 8) {
            const T lo = tP <= tQ ? tP : tQ, hi = tP <= tQ ? tQ : tP;
            msq[p] = hi - lo;
            if (ok && !(hi <= T(2) * lo)) exact = false;
        }
    }
    F = inf64;
    rec = 255;
    // squares: best metric first, the next best when a pair is not usable
    unsigned cand = feas & 0xFFu;
#pragma unroll 1
    for (int tries = 0; tries < 8 && cand; ++tries) {
        int bp = -1;
        if (exact) {
            T bm = alf_inf<T>();
#pragma unroll
            for (int p = 0; p < 8; ++p)
                if (((cand >> p) & 1u) && (bp < 0 || msq[p] < bm)) {
                    bm = msq[p];
                    bp = p;
                }
        } else {
            double bm = inf64;
#pragma unroll
            for (int p = 0; p < 8; ++p) {
                const double mp = fabs((double)t[pq(p)] - (double)t[pp(p)]);
                if (((cand >> p) & 1u) && (bp < 0 || mp < bm)) {
                    bm = mp;
                    bp = p;
                }
            }
        }
        cand &= ~(1u << bp);
        int r;
        const double v = check_pair_time<T, VT>(bp, t, R, r);
        if (v < inf64) {
            F = v;
            rec = r;
            break;
        }
    }
    // triangles (FP64 metrics), only when no square is usable
    cand = rec == 255 ? (feas & 0xFF00u) : 0u;
#pragma unroll 1
    for (int tries = 0; tries < 8 && cand; ++tries) {
        int bp = -1;
        double bm = inf64;
#pragma unroll
        for (int p = 8; p < 16; ++p) {
            const double mp = fabs((double)t[pq(p)] - ((1.4142135623730951 - 1.0) * (double)t[pa(p)] +
                                                       (2.0 - 1.4142135623730951) * (double)t[pp(p)]));
            if (((cand >> p) & 1u) && (bp < 0 || mp < bm)) {
                bm = mp;
                bp = p;
            }
        }
        cand &= ~(1u << bp);
        int r;
        const double v = check_pair_time<T, VT>(bp, t, R, r);
        if (v < inf64) {
            F = v;
            rec = r;
            break;
        }
    }
    if (rec == 255) {
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            if (!((known >> k) & 1u)) continue;
            const double g = (double)t[k] + ((k >= 8) ? 2.0 * R.fb[scls(k)] : R.fb[scls(k)]);
            if (g < F) {
                F = g;
                rec = 32 + k;
            }
        }
    }
    return true;
}

}  // namespace alf
