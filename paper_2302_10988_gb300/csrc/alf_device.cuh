// alf_device.cuh -- device building blocks of the ALI-FMM library (sm_103a).
//
//  * qP phase speed of the YZ-plane Christoffel matrix, written trig-free for
//    an unnormalised wavefront normal (Sec. 3.2);
//  * straight-ray (group) speed: the paper's group->phase inversion (Sec. 3.2)
//    in a division-free form, and the exact ray velocity by an FP64 Newton
//    solve;
//  * the stencil pairs of Sec. 4.1 over the 12-point diamond and the local
//    operator F of one node (Secs. 4.2-4.3 with the heap FMM's recompute rule
//    of Sec. 2 written as a causal fixed point).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace alf {

#define ALF_HD __host__ __device__ __forceinline__
#define ALF_D __device__ __forceinline__

// ---------------------------------------------------------------------------
// Per-(sample, region) constants of the local update.  a.. are stiffness / rho
// (m^2/s^2) of the YZ plane; (cth, sth) the orientation; fb[c] the straight-ray
// time over one diamond step of direction class c (x axis, y axis, diagonal
// (1,1), diagonal (1,-1); lengths 1, 1, sqrt2, sqrt2 cells) and its
// derivative by the orientation; h the spacing.
// ---------------------------------------------------------------------------
template <typename T>
struct RegionP {
    T a22, a33, a44, a2344;
    T cth, sth;
    T fb[4];
    T dfb[4];  // d fb / d theta (used by the adjoint)
    T h;
    T sig;     // root of the in-plane Christoffel block: +1 the larger (qP; SH by its constants), -1 the smaller (qSV)
    int iso;
    int pad;
    const T* vtab;  // velocity-table mode: phase speed of the region's material at 0..180 degrees, else null
};

// Per material, FP64, c / rho, for the plan's wave mode (Sec. 3.2; Sec. 7 for the shear modes):
//  qP   the YZ-plane constants, larger root;
//  qSV  the same constants, smaller root (sv = 1); an isotropic material keeps its shear lambda in a22;
//  SH   lambda = a66 cos^2 + a55 sin^2, written as the larger root of a block whose roots are a66 cos^2 +
//       a55 sin^2 and 0: a22 = a66, a33 = a55, a44 = 0, a23 = sqrt(a66 a55).
// env: for the shear modes, ALF_ENV_N envelope slownesses of the material (group speeds), else null.
struct MatD {
    double a22, a23, a33, a44;
    int iso;
    int sv;
    const double* env;
};
#define ALF_ENV_N 1441  // envelope slowness at 0, 1/8, ..., 180 degrees from the material axis

// ---------------------------------------------------------------------------
// Diamond slots: (-1,0) (1,0) (0,-1) (0,1) (-1,-1) (1,-1) (-1,1) (1,1)
//                (-2,0) (2,0) (0,-2) (0,2)
// ---------------------------------------------------------------------------
__constant__ static const int8_t kSlotDi[12] = {-1, 1, 0, 0, -1, 1, -1, 1, -2, 2, 0, 0};
__constant__ static const int8_t kSlotDj[12] = {0, 0, -1, 1, -1, -1, 1, 1, 0, 0, -2, 2};
// direction class of the step slot -> D, and whether it is two cells long
__constant__ static const int8_t kSlotClass[12] = {0, 0, 1, 1, 2, 3, 3, 2, 0, 0, 1, 1};

// Stencil pairs (Sec. 4.1 tables; pair p+1 of the paper).  A is the earliest
// point; P is member 1's B and Q member 1's C.  For the triangles (pairs 9-16)
// P is the axis point one cell from D and Q the diagonal point.  Pair 4 and
// pair 8 are taken with B and C of their two members swapped relative to each
// other, as the pairing rule states (their printed rows 4-1 and 8-2 are
// garbled).
__constant__ static const int8_t kPairA[16] = {4, 6, 7, 5, 8, 11, 10, 9, 11, 10, 10, 11, 8, 9, 9, 8};
__constant__ static const int8_t kPairP[16] = {2, 3, 1, 1, 4, 7, 5, 7, 3, 2, 2, 3, 0, 1, 1, 0};
__constant__ static const int8_t kPairQ[16] = {0, 0, 3, 2, 6, 6, 4, 5, 7, 5, 4, 6, 6, 7, 5, 4};

// pairs whose three slots include slot k (bit p)
ALF_HD unsigned pairs_of_slot(int k)
{
    // bit p set when slot k is one of kPairA[p], kPairP[p], kPairQ[p]
    constexpr unsigned t[12] = {
        0x9003u, 0x600Cu, 0x0609u, 0x0906u, 0x8451u, 0x42C8u, 0x1832u, 0x21A4u, 0x9010u, 0x6080u, 0x0640u, 0x0920u,
    };
    return t[k];
}

// words of the per-field bitmap of frozen nodes in the (2 box + 1)^2 box around the source
ALF_HD int frozen_words(int box) { return ((2 * box + 1) * (2 * box + 1) + 31) / 32; }

template <typename T>
ALF_D T alf_inf();
template <>
ALF_D float alf_inf<float>() { return __int_as_float(0x7f800000); }
template <>
ALF_D double alf_inf<double>() { return __longlong_as_double(0x7ff0000000000000LL); }

ALF_D bool neg_bit(float v) { return (__float_as_uint(v) >> 31) != 0u; }
ALF_D bool neg_bit(double v) { return (static_cast<unsigned long long>(__double_as_longlong(v)) >> 63) != 0ull; }
ALF_D bool same_bits(float a, float b) { return __float_as_uint(a) == __float_as_uint(b); }
ALF_D bool same_bits(double a, double b) { return __double_as_longlong(a) == __double_as_longlong(b); }
ALF_D float abs_(float v) { return fabsf(v); }
ALF_D double abs_(double v) { return fabs(v); }
// FP32: the hardware square-root approximation (relative error ~2^-23), well inside the FP32 path's budget
ALF_D float sqrt_(float v)
{
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
}
ALF_D double sqrt_(double v) { return sqrt(v); }

// ---------------------------------------------------------------------------
// Sec. 3.2 + 4.2: travel time from one stencil.  Offsets of A, B, C relative to
// D, their times, and the region constants.  The wavefront EB (E on AC with
// tau_E = tau_B), the distance |FD| and the phase speed along the normal of EB
// are evaluated without trigonometry: with u = B - E and the normal
// n = (-u_y, u_x), the relative phase angle has cos = n.axis/|u| and
// sin = axis x n/|u|, so |u|^2 * lambda/rho = ((a~ + g~) + sqrt((a~ - g~)^2 + 4 b~^2))/2
// with a~, g~, b~ built from the unnormalised components, and
// tau_D = tau_B + h |(D - E) x u| / sqrt(|u|^2 lambda/rho).
// ---------------------------------------------------------------------------
// |u|^2 * (qP lambda / rho) for the wavefront direction u (normal (-u_y, u_x)).
ALF_D float atan2_(float y, float x) { return atan2f(y, x); }
ALF_D double atan2_(double y, double x) { return atan2(y, x); }

template <typename T, bool VT = false>
ALF_D T phase_L(const RegionP<T>& R, T ux, T uy)
{
    if (R.iso) return R.a22 * (ux * ux + uy * uy);
    const T C = R.sth * ux - R.cth * uy;
    const T S = R.cth * ux + R.sth * uy;
    if constexpr (VT) {
        // velocity-table mode (Sec. 3, Sec. 4.2): the phase speed at the normal's angle from the material
        // axis, linearly interpolated between the table's integer degrees (180-degree symmetric)
        T deg = atan2_(S, C) * T(57.295779513082320876);
        if (deg < T(0)) deg += T(180);
        if (deg >= T(180)) deg -= T(180);
        int k = (int)floor(deg);
        k = k < 0 ? 0 : (k > 179 ? 179 : k);
        const T f = deg - T(k);
        const T v = (T(1) - f) * R.vtab[k] + f * R.vtab[k + 1];
        return (ux * ux + uy * uy) * v * v;
    }
    const T CC = C * C, SS = S * S;
    const T al = CC * R.a22 + SS * R.a44;
    const T ga = CC * R.a44 + SS * R.a33;
    const T be = C * S * R.a2344;
    const T dm = al - ga;
    return T(0.5) * ((al + ga) + R.sig * sqrt_(dm * dm + T(4) * be * be));
}

ALF_D float div_(float a, float b) { return __fdividef(a, b); }
ALF_D double div_(double a, double b) { return a / b; }
ALF_D float rsqrt_(float v) { return rsqrtf(v); }
ALF_D double rsqrt_(double v) { return 1.0 / sqrt(v); }

template <typename T, bool VT = false>
ALF_D T stencil_time(int xA, int yA, int xB, int yB, int xC, int yC, T tA, T tB, T tC, const RegionP<T>& R)
{
    const T a = div_(tB - tA, tC - tA);
    const T Ex = T(xA) + a * T(xC - xA);
    const T Ey = T(yA) + a * T(yC - yA);
    const T ux = T(xB) - Ex, uy = T(yB) - Ey;
    const T cross = abs_(T(yB) * Ex - T(xB) * Ey);
    return tB + R.h * cross * rsqrt_(phase_L<T, VT>(R, ux, uy));
}

// ---------------------------------------------------------------------------
// Static (compile-time) views of the slot and pair tables, so that the local
// operator below runs with every array in registers and the same instruction
// stream in every lane of a warp.
// ---------------------------------------------------------------------------
ALF_HD constexpr int sdi(int k) { return k == 0 ? -1 : k == 1 ? 1 : k == 4 ? -1 : k == 5 ? 1 : k == 6 ? -1 : k == 7 ? 1 : k == 8 ? -2 : k == 9 ? 2 : 0; }
ALF_HD constexpr int sdj(int k) { return k == 2 ? -1 : k == 3 ? 1 : k == 4 ? -1 : k == 5 ? -1 : k == 6 ? 1 : k == 7 ? 1 : k == 10 ? -2 : k == 11 ? 2 : 0; }
// position in row-major order inside the 5 x 5 box around D (D itself is 12)
ALF_HD constexpr int sord(int k) { return (sdj(k) + 2) * 5 + (sdi(k) + 2); }
ALF_HD constexpr int scls(int k) { return (k <= 1 || k == 8 || k == 9) ? 0 : (k <= 3 || k >= 10) ? 1 : (k == 4 || k == 7) ? 2 : 3; }
ALF_HD constexpr int pa(int p) { constexpr int t[16] = {4, 6, 7, 5, 8, 11, 10, 9, 11, 10, 10, 11, 8, 9, 9, 8}; return t[p]; }
ALF_HD constexpr int pp(int p) { constexpr int t[16] = {2, 3, 1, 1, 4, 7, 5, 7, 3, 2, 2, 3, 0, 1, 1, 0}; return t[p]; }
ALF_HD constexpr int pq(int p) { constexpr int t[16] = {0, 0, 3, 2, 6, 6, 4, 5, 7, 5, 4, 6, 6, 7, 5, 4}; return t[p]; }

// Sec. 4.2, the travel time at D from the stencil pair p, in gradient form.  The plane through (A, tA),
// (P, tP), (Q, tQ) has the time gradient g with g.(P - A) = tP - tA and g.(Q - A) = tQ - tA.  Its iso-line at
// the middle time tB = min(tP, tQ) is the paper's wavefront EB (E on AC at time tB, C the later of P, Q), with
// normal g; D lies |tau_lin(D) - tB| / |g| from it, tau_lin(D) = tA - g.A the plane's time at D.  So
//   tau_D = tB + h |tau_lin(D) - tB| / (|g| v(g / |g|)) = tB + h |tau_lin(D) - tB| / sqrt(|g|^2 lambda(g) / rho),
// the same time as the paper's construction, with no division.  The inverse of (P - A, Q - A) is a constant of
// the stencil: its determinant is +-1 or +-2, so g = (c1 dP + c2 dQ, c3 dP + c4 dQ) with every c in
// {0, +-1/2, +-1}, and A's offsets are in {-2, ..., 2}.  The pair's geometry travels as one word of six
// three-bit codes (2 c + 2 and offset + 2), so that the pair can be chosen at run time; every product with
// these constants is exact, so the time does not depend on how the constants arrive.
ALF_HD constexpr unsigned pair_geom(int p)
{
    const int xa = sdi(pa(p)), ya = sdj(pa(p));
    const int e1x = sdi(pp(p)) - xa, e1y = sdj(pp(p)) - ya;
    const int e2x = sdi(pq(p)) - xa, e2y = sdj(pq(p)) - ya;
    const int det = e1x * e2y - e1y * e2x;
    const int c[6] = {2 * e2y / det + 2, -2 * e1y / det + 2, -2 * e2x / det + 2, 2 * e1x / det + 2, xa + 2, ya + 2};
    unsigned w = 0u;
    for (int k = 0; k < 6; ++k) w |= (unsigned)c[k] << (3 * k);
    return w;
}

// code k of a geometry word as (code - 2) * scale, scale 1/2 or 1.  FP32: the code is placed in the low bits of
// 1.5 * 2^23 (whose ulp is 1), so the float equals 12582912 + code exactly and one FMA gives the value, exactly,
// with no integer-to-float conversion.
template <typename T>
ALF_D T geom_code(unsigned w, int k, T scale)
{
    return T((int)((w >> (3 * k)) & 7u) - 2) * scale;
}
template <>
ALF_D float geom_code<float>(unsigned w, int k, float scale)
{
    const float b = __uint_as_float(((w >> (3 * k)) & 7u) | 0x4B400000u);
    return fmaf(b, scale, -12582914.0f * scale);
}

template <typename T, bool VT = false>
ALF_D T pair_time_geom(unsigned geom, T tA, T tP, T tQ, const RegionP<T>& R)
{
    const T dP = tP - tA, dQ = tQ - tA;
    const T gx = geom_code<T>(geom, 0, T(0.5)) * dP + geom_code<T>(geom, 1, T(0.5)) * dQ;
    const T gy = geom_code<T>(geom, 2, T(0.5)) * dP + geom_code<T>(geom, 3, T(0.5)) * dQ;
    const T tB = tP < tQ ? tP : tQ;
    const T lin = tA - (geom_code<T>(geom, 4, T(1)) * gx + geom_code<T>(geom, 5, T(1)) * gy);
    // phase_L takes the wavefront direction u, whose normal (-u_y, u_x) is g
    return tB + R.h * abs_(lin - tB) * rsqrt_(phase_L<T, VT>(R, gy, -gx));
}

// Run-time lookups of the slot and pair tables (index known only at run time, e.g. from a
// record): fields packed into 64-bit immediates and extracted with shifts, so that lanes with
// different indices neither touch memory nor serialise on the constant cache.
ALF_HD constexpr unsigned long long pack_bits(int which, int bits)
{
    unsigned long long v = 0ull;
    const int n = which < 3 ? 12 : 16;
    for (int k = 0; k < n; ++k) {
        const int x = which == 0 ? sdi(k) + 2 : which == 1 ? sdj(k) + 2 : which == 2 ? scls(k)
                    : which == 3 ? pa(k) : which == 4 ? pp(k) : pq(k);
        v |= (unsigned long long)x << (bits * k);
    }
    return v;
}
ALF_HD int slot_di(int k)
{
    constexpr unsigned long long t = pack_bits(0, 3);
    return (int)((t >> (3 * k)) & 7ull) - 2;
}
ALF_HD int slot_dj(int k)
{
    constexpr unsigned long long t = pack_bits(1, 3);
    return (int)((t >> (3 * k)) & 7ull) - 2;
}
ALF_HD int slot_cls(int k)
{
    constexpr unsigned long long t = pack_bits(2, 2);
    return (int)((t >> (2 * k)) & 3ull);
}
ALF_HD int pair_a(int p)
{
    constexpr unsigned long long t = pack_bits(3, 4);
    return (int)((t >> (4 * p)) & 15ull);
}
ALF_HD int pair_p(int p)
{
    constexpr unsigned long long t = pack_bits(4, 4);
    return (int)((t >> (4 * p)) & 15ull);
}
ALF_HD int pair_q(int p)
{
    constexpr unsigned long long t = pack_bits(5, 4);
    return (int)((t >> (4 * p)) & 15ull);
}

// One comparison of the rank counts of the local operator: when a precedes b (a <= b with le, else a < b),
// add d to w (both counters in one word), or add dm to wm and take dk from wk -- predicated adds, with no
// select.
ALF_D void rank_count(unsigned& w, float a, float b, bool le, unsigned d)
{
    if (le) asm("{\n\t.reg .pred p;\n\tsetp.le.f32 p, %1, %2;\n\t@p add.u32 %0, %0, %3;\n\t}" : "+r"(w) : "f"(a), "f"(b), "r"(d));
    else asm("{\n\t.reg .pred p;\n\tsetp.lt.f32 p, %1, %2;\n\t@p add.u32 %0, %0, %3;\n\t}" : "+r"(w) : "f"(a), "f"(b), "r"(d));
}
ALF_D void rank_count(unsigned& wm, unsigned& wk, float a, float b, bool le, unsigned dm, unsigned dk)
{
    if (le)
        asm("{\n\t.reg .pred p;\n\tsetp.le.f32 p, %2, %3;\n\t@p add.u32 %0, %0, %4;\n\t@p sub.u32 %1, %1, %5;\n\t}"
            : "+r"(wm), "+r"(wk) : "f"(a), "f"(b), "r"(dm), "r"(dk));
    else
        asm("{\n\t.reg .pred p;\n\tsetp.lt.f32 p, %2, %3;\n\t@p add.u32 %0, %0, %4;\n\t@p sub.u32 %1, %1, %5;\n\t}"
            : "+r"(wm), "+r"(wk) : "f"(a), "f"(b), "r"(dm), "r"(dk));
}
ALF_D void rank_count(unsigned& w, double a, double b, bool le, unsigned d)
{
    if (le) asm("{\n\t.reg .pred p;\n\tsetp.le.f64 p, %1, %2;\n\t@p add.u32 %0, %0, %3;\n\t}" : "+r"(w) : "d"(a), "d"(b), "r"(d));
    else asm("{\n\t.reg .pred p;\n\tsetp.lt.f64 p, %1, %2;\n\t@p add.u32 %0, %0, %3;\n\t}" : "+r"(w) : "d"(a), "d"(b), "r"(d));
}
ALF_D void rank_count(unsigned& wm, unsigned& wk, double a, double b, bool le, unsigned dm, unsigned dk)
{
    if (le)
        asm("{\n\t.reg .pred p;\n\tsetp.le.f64 p, %2, %3;\n\t@p add.u32 %0, %0, %4;\n\t@p sub.u32 %1, %1, %5;\n\t}"
            : "+r"(wm), "+r"(wk) : "d"(a), "d"(b), "r"(dm), "r"(dk));
    else
        asm("{\n\t.reg .pred p;\n\tsetp.lt.f64 p, %2, %3;\n\t@p add.u32 %0, %0, %4;\n\t@p sub.u32 %1, %1, %5;\n\t}"
            : "+r"(wm), "+r"(wk) : "d"(a), "d"(b), "r"(dm), "r"(dk));
}

// ---------------------------------------------------------------------------
// The local operator F at node D (linear index `me`; the tie order of equal
// times is the linear index, which for diamond neighbours is the static order
// sord()).  nb[k] are the raw stored times of the diamond slots: frozen nodes
// carry the sign bit, unknown or outside nodes are +inf.
//
// Semantics (the heap FMM's recompute-on-accept rule written as a causal
// fixed point): the non-frozen finite neighbours join the known set one at a
// time in key order (tau, index); after each the update U is recomputed, and
// F is the value current when D's own key (U, me) precedes the next
// neighbour's key.  U(S) (Secs. 4.2-4.3): the usable square pair of smallest
// |tau_C - tau_B| (ties to the lower stencil row), else the usable triangle
// pair of smallest |tau_diag - ((sqrt2 - 1) tau_A + (2 - sqrt2) tau_axis)|,
// else the straight-ray fallback min_N tau_N + step_N / V_group.  A pair is
// usable when A, P, Q are known, tau_A < min(tau_P, tau_Q), and its time is
// later than its later support point.
//
// Implementation: the 16 pair metrics and times do not depend on the known
// set, so they are computed once.  A pair becomes available at the step of its
// latest member (rp = the largest rank of A, P, Q) and the fallback of slot q
// at the step of q.  Within a class the choice is a minimum over a growing
// set, so U changes only at steps where an item of the class in force (or of
// a preferred class) becomes available.  With c(u) = the number of candidates
// whose key precedes (u, me), the stop rule "(u_k, me) precedes the key of
// rank k + 1" reads c(u_k) <= k + 1, and while U stays at u the first step
// that satisfies it is c(u) - 1.  So the walk visits only the steps where U
// can change and stops as soon as c(u) - 1 comes before the next of them.
// ---------------------------------------------------------------------------
// VT: the velocity-table mode (the table lookup is compiled only into the kernels that use it)
template <typename T, bool VT = false>
ALF_D T local_F(const T* nb, int me, int nx, const RegionP<T>& R, int& rec)
{
    (void)me;
    (void)nx;
    const T inf = alf_inf<T>();
    T t[12];
    unsigned fz = 0u, cd = 0u;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        t[k] = abs_(nb[k]);
        if (neg_bit(nb[k])) fz |= 1u << k;
        else if (nb[k] < inf) cd |= 1u << k;
    }
    // rank of each candidate in key order (tau, then linear index = static slot order):
    // the number of candidates with a smaller key.  Non-candidates compare as +inf and
    // are then given rank -1 (frozen: known from the start) or 64 (unknown: never known).
    // (The pair loop runs over the full 12 x 12 square so that it unrolls completely and
    // the arrays stay in registers.)
    // The 12 counts are bytes of three words, biased by 64 so that no byte ever borrows or carries: byte k
    // starts at 64 + (11 - k) (as if every later slot preceded it) and each of the 66 comparisons, when k
    // precedes m, adds one to byte m and takes one from byte k -- one predicated add per word it touches.
    T kt[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) kt[k] = ((cd >> k) & 1u) ? t[k] : inf;
    unsigned W[3];
#pragma unroll
    for (int w = 0; w < 3; ++w) {
        W[w] = 0u;
#pragma unroll
        for (int b = 0; b < 4; ++b) W[w] |= (unsigned)(64 + 11 - (4 * w + b)) << (8 * b);
    }
#pragma unroll
    for (int k = 0; k < 12; ++k)
#pragma unroll
        for (int m = 0; m < 12; ++m) {
            if (m <= k) continue;
            // key(k) < key(m); on equal times the static order decides
            const unsigned im = 1u << (8 * (m & 3)), ik = 1u << (8 * (k & 3));
            if ((m >> 2) == (k >> 2)) rank_count(W[m >> 2], kt[k], kt[m], sord(k) < sord(m), im - ik);
            else rank_count(W[m >> 2], W[k >> 2], kt[k], kt[m], sord(k) < sord(m), im, ik);
        }
    int rk[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        const int c = (int)((W[k >> 2] >> (8 * (k & 3))) & 0xFFu) - 64;
        rk[k] = ((cd >> k) & 1u) ? c : (((fz >> k) & 1u) ? -1 : 64);
    }
    const int nc = __popc(cd);
    // pairs: metric (+inf when not feasible) and availability step; ev_*: bit (step + 1) of a feasible pair.
    // A feasible pair is usable when its time is later than C; that time is evaluated only when the walk
    // chooses the pair (a pair found not usable is set aside and the choice made again), so that one or two
    // stencil times are evaluated per node instead of one per feasible pair.
    T pm[16];
    int rp[16];
    unsigned ev_sq = 0u, ev_tr = 0u;
#pragma unroll
    for (int p = 0; p < 16; ++p) {
        constexpr T k1 = T(1.4142135623730951) - T(1.0);
        constexpr T k2 = T(2.0) - T(1.4142135623730951);
        const int A = pa(p), P = pp(p), Q = pq(p);
        const T tA = t[A], tP = t[P], tQ = t[Q];
        rp[p] = max(rk[A], max(rk[P], rk[Q]));
        pm[p] = inf;
        if (rp[p] < 64 && tA < tP && tA < tQ) {
            const bool m1 = tP <= tQ;
            const T tB = m1 ? tP : tQ, tC = m1 ? tQ : tP;
            pm[p] = (p < 8) ? (tC - tB) : abs_(tQ - (k1 * tA + k2 * tP));
            if (p < 8) ev_sq |= 1u << (rp[p] + 1);
            else ev_tr |= 1u << (rp[p] + 1);
        }
    }
    // straight-ray fallback values of the slots
    T g[12];
#pragma unroll
    for (int q = 0; q < 12; ++q) g[q] = t[q] + ((q >= 8) ? T(2) * R.fb[scls(q)] : R.fb[scls(q)]);
    const unsigned ev_all = ((1u << nc) - 1u) << 1;  // every candidate's step
    // walk over the steps at which U can change; the known set at step k is the frozen slots
    // and the candidates of rank <= k
    T u = inf;
    int urec = 255;
    int k = -1;
    {
        // Before the first pair is available U is a fallback value, never below gmin (the least fallback
        // value over every slot that is or becomes known), and c() grows with its argument: when
        // c(gmin) - 1 reaches the first pair's step, no step before it can stop, so the walk starts there.
        const unsigned ev_pair = ev_sq | ev_tr;
        if (ev_pair > 1u) {  // the first pair is not available from the start
            T gmin = inf;
#pragma unroll
            for (int q = 0; q < 12; ++q)
                if (rk[q] < 64 && g[q] < gmin) gmin = g[q];
            int cmin = 0;
#pragma unroll
            for (int q = 0; q < 12; ++q)
                cmin += (((cd >> q) & 1u) && (sord(q) < 12 ? t[q] <= gmin : t[q] < gmin)) ? 1 : 0;
            const int first = __ffs((int)ev_pair) - 2;
            if (cmin - 1 >= first) k = first;
        }
    }
    unsigned unusable = 0u;  // feasible pairs whose time is not later than C
    int last_p = -1;         // the last pair evaluated and its time
    T last_v = inf;
#pragma unroll 1
    for (int guard = 0; guard < 32; ++guard) {
        // the available, possibly usable pair of least metric: squares, else triangles (ties to the lower row)
        T bm = inf, sA = inf, sP = inf, sQ = inf;
        int bp = -1;
        unsigned geom = 0u;
#pragma unroll
        for (int p = 0; p < 8; ++p)
            if (rp[p] <= k && !((unusable >> p) & 1u) && pm[p] < bm) {
                bm = pm[p];
                bp = p;
                sA = t[pa(p)];
                sP = t[pp(p)];
                sQ = t[pq(p)];
                geom = pair_geom(p);
            }
        if (bp < 0) {
#pragma unroll
            for (int p = 8; p < 16; ++p)
                if (rp[p] <= k && !((unusable >> p) & 1u) && pm[p] < bm) {
                    bm = pm[p];
                    bp = p;
                    sA = t[pa(p)];
                    sP = t[pp(p)];
                    sQ = t[pq(p)];
                    geom = pair_geom(p);
                }
        }
        T bv = inf;
        int br = 255, cls = 2;
        if (bp >= 0) {
            const T v = bp == last_p ? last_v : pair_time_geom<T, VT>(geom, sA, sP, sQ, R);
            if (!(v > (sP <= sQ ? sQ : sP))) {
                unusable |= 1u << bp;
                continue;
            }
            last_p = bp;
            last_v = v;
            bv = v;
            br = 2 * bp + (sP <= sQ ? 0 : 1);
            cls = bp < 8 ? 0 : 1;
        } else {
#pragma unroll
            for (int q = 0; q < 12; ++q)
                if (rk[q] <= k && g[q] < bv) {
                    bv = g[q];
                    br = 32 + q;
                }
        }
        u = bv;
        urec = br;
        // c(u): candidates whose key (tau, linear index) precedes (u, me)
        int cnt = 0;
#pragma unroll
        for (int q = 0; q < 12; ++q) cnt += (((cd >> q) & 1u) && (sord(q) < 12 ? t[q] <= u : t[q] < u)) ? 1 : 0;
        if (cnt <= k + 1) break;
        const unsigned later = (cls == 0 ? ev_sq : cls == 1 ? (ev_sq | ev_tr) : ev_all) >> (k + 2);
        if (later == 0u) break;
        const int e = k + __ffs((int)later);  // next step at which U can change
        if (cnt - 1 < e) break;
        k = e;
    }
    rec = urec;
    return u;
}

// ---------------------------------------------------------------------------
// Velocity model in FP64 (used for per-region tables, initial times, checks).
// ---------------------------------------------------------------------------
__device__ inline double qp_lambda64(const MatD& m, double c, double s)  // c, s: unit direction cosines
{
    if (m.iso) return m.a22;
    const double al = c * c * m.a22 + s * s * m.a44;
    const double ga = c * c * m.a44 + s * s * m.a33;
    const double be = c * s * (m.a23 + m.a44);
    const double dm = al - ga;
    const double r = sqrt(dm * dm + 4.0 * be * be);
    return 0.5 * ((al + ga) + (m.sv ? -r : r));
}

// Shear modes: the group speed from the material's table of envelope slownesses (linear in slowness between
// the entries at multiples of 1/8 degree; 180-degree symmetric).
__device__ inline double env_speed64(const double* tab, double phi)
{
    double deg = phi * (180.0 / 3.141592653589793);
    deg -= 180.0 * floor(deg / 180.0);
    const double u = deg * ((ALF_ENV_N - 1) / 180.0);
    int k = (int)floor(u);
    k = k < 0 ? 0 : (k > ALF_ENV_N - 2 ? ALF_ENV_N - 2 : k);
    const double f = u - k;
    return 1.0 / ((1.0 - f) * tab[k] + f * tab[k + 1]);
}

// The paper's inversion (Sec. 3.2): find the phase angle theta whose qP
// polarisation is along the group angle phi.  Eliminating lambda between its
// two eigen-equations gives delta cos2t + eta sin2t + kappa = 0 with
// eta = -2 (c23 + c44) cos2phi / sin2phi; multiplied by sin2phi this is
// A cos X + B sin X = Cc (X = 2 theta), solved as X = atan2(B, A) +- acos(Cc/R).
// Of the two roots the qP one is where (cos phi, sin phi) has the larger
// Rayleigh quotient of M(theta).  Within 0.01 degree of a multiple of 90 the
// angle is rounded onto it, as in the paper.  Returns V = v(theta)/cos(theta-phi).
__device__ inline double group_paper64(const MatD& m, double phi)
{
    if (m.iso) return sqrt(m.a22);
    const double kPi = 3.141592653589793;
    double deg = phi * (180.0 / kPi);
    deg -= 180.0 * floor(deg / 180.0);  // [0, 180)
    const double k90 = 90.0 * rint(deg / 90.0);
    if (fabs(deg - k90) < 0.01) deg = k90;
    if (deg >= 180.0) deg -= 180.0;
    if (deg == 0.0) return sqrt(m.a22);
    if (deg == 90.0) return sqrt(m.a33);
    const double ph = deg * (kPi / 180.0);
    double s2p, c2p;
    sincos(2.0 * ph, &s2p, &c2p);
    const double delta = m.a22 + m.a33 - 2.0 * m.a44;
    const double kappa = m.a22 - m.a33;
    const double A = delta * s2p, B = -2.0 * (m.a23 + m.a44) * c2p, Cc = -kappa * s2p;
    const double Rr = sqrt(A * A + B * B);
    double q = Cc / Rr;
    q = fmin(1.0, fmax(-1.0, q));
    const double X0 = atan2(B, A), dX = acos(q);
    double cph, sph;
    sincos(ph, &sph, &cph);
    double best_t = 0.0, best_r = -1.0;
    for (int r = 0; r < 2; ++r) {
        const double th = 0.5 * (r == 0 ? X0 + dX : X0 - dX);
        double c, s;
        sincos(th, &s, &c);
        const double al = c * c * m.a22 + s * s * m.a44;
        const double ga = c * c * m.a44 + s * s * m.a33;
        const double be = c * s * (m.a23 + m.a44);
        const double rq = al * cph * cph + 2.0 * be * cph * sph + ga * sph * sph;
        if (rq > best_r) {
            best_r = rq;
            best_t = th;
        }
    }
    double dev = best_t - ph;  // wrap into (-pi/2, pi/2]
    dev -= kPi * rint(dev / kPi);
    double c, s;
    sincos(best_t, &s, &c);
    return sqrt(qp_lambda64(m, c, s)) / cos(dev);
}

// qP phase speed and its first two derivatives with respect to the phase angle.
__device__ inline void qp_v_derivs(const MatD& m, double th, double& v, double& dv, double& d2v)
{
    double s, c;
    sincos(th, &s, &c);
    const double s2 = 2.0 * s * c, c2 = c * c - s * s;
    const double al = c * c * m.a22 + s * s * m.a44, ga = c * c * m.a44 + s * s * m.a33;
    const double be = 0.5 * s2 * (m.a23 + m.a44);
    const double dal = s2 * (m.a44 - m.a22), dga = s2 * (m.a33 - m.a44), dbe = c2 * (m.a23 + m.a44);
    const double ddal = 2.0 * c2 * (m.a44 - m.a22), ddga = 2.0 * c2 * (m.a33 - m.a44),
                 ddbe = -2.0 * s2 * (m.a23 + m.a44);
    const double dm = al - ga, ddm = dal - dga, dddm = ddal - ddga;
    const double R = sqrt(dm * dm + 4.0 * be * be);
    const double lam = 0.5 * (al + ga + R);
    double dR = 0.0, ddR = 0.0;
    if (R > 0.0) {
        dR = (dm * ddm + 4.0 * be * dbe) / R;
        ddR = (ddm * ddm + dm * dddm + 4.0 * dbe * dbe + 4.0 * be * ddbe - dR * dR) / R;
    }
    const double dlam = 0.5 * (dal + dga + dR), ddlam = 0.5 * (ddal + ddga + ddR);
    v = sqrt(lam);
    dv = dlam / (2.0 * v);
    d2v = (0.5 * ddlam - dv * dv) / v;
}

// Exact ray velocity: solve psi(theta) = theta + atan2(v', v) = phi by Newton
// steps (dpsi/dtheta = v (v + v'') / (v^2 + v'^2)) kept inside the bracket
// [phi - pi/2, phi + pi/2] by bisection; V = sqrt(v^2 + v'^2).
__device__ inline double group_exact64(const MatD& m, double phi)
{
    if (m.iso) return sqrt(m.a22);
    const double kPi = 3.141592653589793;
    double lo = phi - 0.5 * kPi + 1e-12, hi = phi + 0.5 * kPi - 1e-12;
    double th = phi, v, dv, d2v;
    for (int it = 0; it < 60; ++it) {
        qp_v_derivs(m, th, v, dv, d2v);
        const double f = th + atan2(dv, v) - phi;
        if (f > 0.0) hi = th; else lo = th;
        const double fp = v * (v + d2v) / (v * v + dv * dv);
        double nt = th - f / fp;
        if (!(nt > lo && nt < hi) || !(fp > 0.0)) nt = 0.5 * (lo + hi);
        if (fabs(nt - th) < 1e-15 * (1.0 + fabs(th))) {
            th = nt;
            break;
        }
        th = nt;
    }
    qp_v_derivs(m, th, v, dv, d2v);
    return sqrt(v * v + dv * dv);
}

__device__ inline double group_speed64(const MatD& m, int model, double phi)
{
    if (m.iso) return sqrt(m.a22);  // an isotropic mode travels at its phase speed in every direction
    if (m.env) return env_speed64(m.env, phi);
    return model == 1 ? group_exact64(m, phi) : group_paper64(m, phi);
}

// FP32 paper inversion for the ray tracer; falls back to FP64 where the
// root's acos argument is within 1e-2 of +-1 (ill-conditioned in FP32) and
// near the axes where the 0.01-degree rounding applies.
__device__ inline float group_paper32(const MatD& m, float a22, float a33, float a44, float a2344, float phi)
{
    if (m.iso) return sqrtf(a22);
    if (m.env) return (float)env_speed64(m.env, (double)phi);
    const float kPi = 3.14159265358979f;
    float deg = phi * (180.0f / kPi);
    deg -= 180.0f * floorf(deg / 180.0f);
    const float k90 = 90.0f * rintf(deg / 90.0f);
    // within 0.05 degrees of a symmetry axis the inversion loses FP32 precision; there the speed differs from
    // the axis's (where group and phase coincide) by V''(0) phi^2 / 2, below 2e-6 relative at 8.7e-4 rad,
    // inside the FP32 path's error (the FP64 model rounds to the axis within 0.01 degrees, Sec. 3.2)
    if (fabsf(deg - k90) < 0.05f) return sqrtf(k90 == 90.0f ? a33 : a22);
    const float ph = deg * (kPi / 180.0f);
    float s2p, c2p;
    sincosf(2.0f * ph, &s2p, &c2p);
    const float delta = a22 + a33 - 2.0f * a44, kappa = a22 - a33;
    const float A = delta * s2p, B = -2.0f * a2344 * c2p, Cc = -kappa * s2p;
    const float Rr = sqrtf(A * A + B * B);
    const float q = Cc / Rr;
    if (fabsf(q) > 0.99f) return float(group_paper64(m, (double)phi));
    const float X0 = atan2f(B, A), dX = acosf(q);
    float cph, sph;
    sincosf(ph, &sph, &cph);
    float best_t = 0.0f, best_r = -1.0f, best_l = 0.0f;
    for (int r = 0; r < 2; ++r) {
        const float th = 0.5f * (r == 0 ? X0 + dX : X0 - dX);
        float c, s;
        sincosf(th, &s, &c);
        const float al = c * c * a22 + s * s * a44, ga = c * c * a44 + s * s * a33, be = c * s * a2344;
        const float rq = al * cph * cph + 2.0f * be * cph * sph + ga * sph * sph;
        if (rq > best_r) {
            best_r = rq;
            best_t = th;
            const float dm = al - ga;
            best_l = 0.5f * ((al + ga) + sqrtf(dm * dm + 4.0f * be * be));
        }
    }
    float dev = best_t - ph;
    dev -= kPi * rintf(dev / kPi);
    return sqrtf(best_l) / cosf(dev);
}

}  // namespace alf
