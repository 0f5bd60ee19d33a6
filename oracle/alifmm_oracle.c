/*
 * Plain FP64 CPU oracle of the ALI-FMM travel-time method and its Fermat ray
 * tracer (Ludlam, Tant, Dolean, Curtis: "Travel times and ray paths for
 * acoustic and elastic waves in generally anisotropic media", arXiv 2302.10988).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the correctness reference for the
 * CUDA library; only the test-suite, the smoke check and the CPU-baseline leg
 * of the benchmark load it.  It shares no code, header, table or constant
 * with the CUDA sources: every formula below is written out again from the
 * paper, in the paper's order, slowly and in double precision.
 *
 * Units: SI throughout (stiffness in Pa, density in kg/m^3, lengths in m,
 * times in s).  Grid node (i, j) sits at (x, y) = (i*h, j*h); the linear index
 * of a node is j*nx + i.  Angles are radians, counter-clockwise from +x.
 *
 * Readings of the paper that this file takes where the paper is silent or
 * garbled are marked [R#]; the list of them, with reasons, is kept in the
 * design notes of the repository.
 *
 * Parity status of each part (what pins it) is stated next to the part.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

#define OM_INF INFINITY

/* In-plane elastic constants of one orthotropic material in the YZ plane
 * (Sec. 3.2): only c22, c23, c33, c44 and the density enter the qP speed. */
typedef struct {
    double c22, c23, c33, c44, rho;
    double c55, c66; /* the out-of-plane shear constants: only the SH mode reads them */
} om_mat;

/* A medium on a regular grid: per-node material index and orientation.
 * theta[node] is the CCW angle from +x to the material's phase-angle-zero
 * axis (the axis along which the qP phase speed is sqrt(c22/rho)). */
typedef struct {
    int nx, ny;
    double h;
    const int32_t* mat_id;
    const double* theta;
    const om_mat* mats;
    int nmats;
    int group_model; /* 0 = the paper's group->phase inversion, 1 = exact ray velocity */
    int vtable;      /* 1: stencil updates take the phase speed by linear interpolation in a table of phase
                        speeds at integer degrees (Sec. 3, Sec. 4.2); 0: from the Christoffel matrix */
    int wave_mode;   /* 0: qP; 1: qSV; 2: SH (Sec. 7: the other eigenvalues of Sec. 3.2) */
    const double* env; /* wave modes 1, 2: per material, ENV_N first-arrival slownesses (see below) */
} om_medium;

/* counters exposed for tests */
static int64_t g_root_swaps = 0;     /* [R1] times the printed root failed the qP check */
static int64_t g_disc_clamps = 0;    /* negative discriminant clamped to zero */

/* Operation count of the local update (stencil times, metrics, the choice, the ordering of the
 * neighbours, the fallback): every floating-point add, subtract, multiply, divide, square root,
 * absolute value, comparison and libm call the code below executes counts 1.  The fallback's group
 * speed along a diamond direction depends only on the material and orientation of D, not on the
 * field, so a fallback candidate counts as its add and its comparison (2); group speeds themselves
 * are not counted.  The count gives the algorithmic work per node evaluation of a solve. */
static int64_t g_ops = 0;

int64_t om_counter(int which) { return which == 0 ? g_root_swaps : which == 1 ? g_disc_clamps : g_ops; }
void om_reset_counters(void) { g_root_swaps = 0; g_disc_clamps = 0; g_ops = 0; }

/* ------------------------------------------------------------------------ */
/* Sec. 3.1-3.2: velocities                                                   */
/* ------------------------------------------------------------------------ */

/* The paper's isotropic short-cut (Sec. 3.2: no Christoffel solve is needed
 * for isotropic materials, which are defined by a single speed). */
static int mat_is_isotropic(const om_mat* m)
{
    return m->c22 == m->c33 && m->c23 == m->c22 - 2.0 * m->c44;
}

/* Sec. 3.2: Christoffel matrix of the YZ plane at phase angle theta; the qP
 * eigenvalue is the larger root ((alpha+gamma) + sqrt((alpha-gamma)^2 + 4 beta^2))/2. */
double om_qp_lambda(const om_mat* m, double theta)
{
    if (mat_is_isotropic(m)) return m->c22;
    double c = cos(theta), s = sin(theta);
    double alpha = c * c * m->c22 + s * s * m->c44;
    double beta = c * s * (m->c23 + m->c44);
    double gamma = c * c * m->c44 + s * s * m->c33;
    return 0.5 * ((alpha + gamma) + sqrt((alpha - gamma) * (alpha - gamma) + 4.0 * beta * beta));
}

/* Sec. 3.1: phase speed v = sqrt(lambda / rho) (the paper's sigma is the density). */
double om_phase_velocity(const om_mat* m, double theta)
{
    return sqrt(om_qp_lambda(m, theta) / m->rho);
}

/* Sec. 3.2 and Sec. 7: the eigenvalue of the Christoffel matrix of each wave mode at phase angle theta.
 * mode 0 (qP): the larger root of the in-plane 2x2 block; mode 1 (qSV): the smaller root,
 * ((alpha + gamma) - sqrt((alpha - gamma)^2 + 4 beta^2)) / 2; mode 2 (SH): the out-of-plane eigenvalue
 * cos^2(theta) c66 + sin^2(theta) c55 (eigenvector (1, 0, 0)). */
double om_mode_lambda(const om_mat* m, int mode, double theta)
{
    if (mode == 0) return om_qp_lambda(m, theta);
    /* the isotropic short-cut of Sec. 3.2 for the shear modes: the shear constant in every direction */
    if (mode == 1 && mat_is_isotropic(m)) return m->c44;
    if (mode == 2 && m->c55 == m->c66) return m->c66;
    double c = cos(theta), s = sin(theta);
    if (mode == 2) return c * c * m->c66 + s * s * m->c55;
    double alpha = c * c * m->c22 + s * s * m->c44;
    double beta = c * s * (m->c23 + m->c44);
    double gamma = c * c * m->c44 + s * s * m->c33;
    return 0.5 * ((alpha + gamma) - sqrt((alpha - gamma) * (alpha - gamma) + 4.0 * beta * beta));
}

double om_mode_velocity(const om_mat* m, int mode, double theta)
{
    return sqrt(om_mode_lambda(m, mode, theta) / m->rho);
}

/* First-arrival group slowness of a mode along the angle psi from the material axis: the support function
 * of the slowness curve, max over phase angles theta of cos(theta - psi) / v(theta) (the wavefront of a point
 * source in a homogeneous medium is the envelope of the plane waves n.x = v(n) t, so the first arrival at
 * distance d along psi is d times this maximum).  It is single valued where the qSV ray surface has cusps.
 * Evaluated by a scan of 3600 phase angles over (psi - 90, psi + 90] degrees and a golden-section search
 * around the best one. */
double om_envelope_slowness(const om_mat* m, int mode, double psi)
{
    /* an isotropic mode (qSV of an isotropic solid, SH with c55 = c66) has the circle 1 / v */
    if ((mode == 1 && mat_is_isotropic(m)) || (mode == 2 && m->c55 == m->c66))
        return 1.0 / om_mode_velocity(m, mode, 0.0);
    const int n = 3600;
    const double step = M_PI / n;
    double best = -1.0, bt = psi;
    for (int k = 1; k <= n; ++k) {
        double th = psi - M_PI / 2 + k * step;
        double g = cos(th - psi) / om_mode_velocity(m, mode, th);
        if (g > best) {
            best = g;
            bt = th;
        }
    }
    double a = bt - step, b = bt + step;
    const double r = 0.5 * (sqrt(5.0) - 1.0);
    for (int it = 0; it < 80; ++it) {
        double x1 = b - r * (b - a), x2 = a + r * (b - a);
        double g1 = cos(x1 - psi) / om_mode_velocity(m, mode, x1);
        double g2 = cos(x2 - psi) / om_mode_velocity(m, mode, x2);
        if (g1 < g2) a = x1; else b = x2;
    }
    double th = 0.5 * (a + b);
    double g = cos(th - psi) / om_mode_velocity(m, mode, th);
    return g > best ? g : best;
}

/* [R20] The group speeds of the shear modes (source initialisation, fallback, rays) come from a table of the
 * envelope slowness at ENV_N angles 0, 1/8, ..., 180 degrees from the material axis, interpolated linearly in
 * slowness (the paper tabulates velocity curves in the same way, Sec. 3). */
#define ENV_N 1441
void om_envelope_table(const om_mat* m, int mode, double* tab)
{
    for (int k = 0; k < ENV_N; ++k) tab[k] = om_envelope_slowness(m, mode, k * M_PI / (ENV_N - 1));
}

double om_envelope_speed(const double* tab, double psi)
{
    double deg = psi * 180.0 / M_PI;
    deg -= 180.0 * floor(deg / 180.0); /* [0, 180) */
    double u = deg * (ENV_N - 1) / 180.0;
    int k = (int)floor(u);
    if (k > ENV_N - 2) k = ENV_N - 2;
    double f = u - k;
    return 1.0 / ((1.0 - f) * tab[k] + f * tab[k + 1]);
}

/* Sec. 3.2, Eq. lambda_1: lambda from the phase angle theta and group angle phi. */
static double lambda_from_eq1(const om_mat* m, double theta, double phi)
{
    return 0.5 * (cos(2.0 * theta) * (m->c22 - m->c44) + sin(2.0 * theta) * (m->c23 + m->c44) * tan(phi)
                  + (m->c22 + m->c44));
}

/* Wrap an angle difference into (-pi/2, pi/2]: directions are 180-degree symmetric. */
static double wrap_half_pi(double d)
{
    d = fmod(d, M_PI);
    if (d <= -M_PI / 2) d += M_PI;
    if (d > M_PI / 2) d -= M_PI;
    return d;
}

/* Sec. 3.2: the paper's group -> phase inversion.  Given the group angle phi
 * (relative to the material axis) it finds the phase angle theta for which
 * (0, cos phi, sin phi) is an eigenvector of M(theta) with the qP eigenvalue,
 * via delta, eta, kappa and the tan-substitution quadratic, then uses
 * |V| = |v| / cos(theta - phi) (Eq. group_vel).  Angles within 0.01 degrees of
 * a multiple of 90 are rounded onto it (end of Sec. 3.2).
 * Returns theta on the branch nearest phi and the group speed V. */
void om_group_paper(const om_mat* m, double phi, double* theta_out, double* V_out)
{
    if (mat_is_isotropic(m)) {
        *theta_out = phi;
        *V_out = sqrt(m->c22 / m->rho);
        return;
    }
    double deg = phi * 180.0 / M_PI;
    double base = floor(deg / 180.0) * 180.0;
    double r = deg - base; /* r in [0, 180) by 180-degree symmetry */
    double k90 = round(r / 90.0) * 90.0;
    if (fabs(r - k90) < 0.01) r = k90;
    if (r >= 180.0) {
        r -= 180.0;
        base += 180.0;
    }
    double theta_deg, lam;
    if (r == 0.0) {
        theta_deg = 0.0;
        lam = m->c22;
    } else if (r == 90.0) {
        theta_deg = 90.0;
        lam = m->c33;
    } else {
        double ph = r * M_PI / 180.0;
        double delta = m->c22 + m->c33 - 2.0 * m->c44;
        double eta = (m->c23 + m->c44) * (tan(ph) - 1.0 / tan(ph));
        double kappa = m->c22 - m->c33;
        double disc = eta * eta + delta * delta - kappa * kappa;
        if (disc < 0.0) {
            g_disc_clamps++;
            disc = 0.0;
        }
        double sq = sqrt(disc);
        double y_minus = (-eta - sq) / (kappa - delta);
        double y_plus = (-eta + sq) / (kappa - delta);
        /* the printed rule: '-' root for 0 < phi < 90, '+' root for 90 < phi < 180 */
        double y = (r < 90.0) ? y_minus : y_plus;
        double y_other = (r < 90.0) ? y_plus : y_minus;
        theta_deg = fmod(atan(y) * 180.0 / M_PI + 180.0, 180.0);
        lam = lambda_from_eq1(m, theta_deg * M_PI / 180.0, ph);
        /* [R1] the chosen root must give the qP (largest) eigenvalue and lie
         * within 90 degrees of phi; otherwise take the other root. */
        double lq = om_qp_lambda(m, theta_deg * M_PI / 180.0);
        double dev = wrap_half_pi((theta_deg - r) * M_PI / 180.0);
        if (!(fabs(lam - lq) <= 1e-9 * lq) || fabs(dev) >= M_PI / 2) {
            g_root_swaps++;
            theta_deg = fmod(atan(y_other) * 180.0 / M_PI + 180.0, 180.0);
            lam = lambda_from_eq1(m, theta_deg * M_PI / 180.0, ph);
        }
    }
    double v = sqrt(lam / m->rho);
    double dev = wrap_half_pi((theta_deg - r) * M_PI / 180.0);
    *theta_out = (base + r) * M_PI / 180.0 + dev;
    *V_out = v / cos(dev);
}

/* qP phase speed and its derivative with respect to the phase angle. */
static void qp_v_dv(const om_mat* m, double th, double* v, double* dv)
{
    double c = cos(th), s = sin(th);
    double al = c * c * m->c22 + s * s * m->c44;
    double ga = c * c * m->c44 + s * s * m->c33;
    double be = c * s * (m->c23 + m->c44);
    double s2 = 2.0 * s * c, c2 = c * c - s * s;
    double dal = s2 * (m->c44 - m->c22);
    double dga = s2 * (m->c33 - m->c44);
    double dbe = c2 * (m->c23 + m->c44);
    double R = sqrt((al - ga) * (al - ga) + 4.0 * be * be);
    double lam = 0.5 * (al + ga + R);
    double dR = R > 0.0 ? ((al - ga) * (dal - dga) + 4.0 * be * dbe) / R : 0.0;
    *v = sqrt(lam / m->rho);
    *dv = 0.5 * (dal + dga + dR) / (2.0 * m->rho * (*v));
}

/* Exact ray (group) velocity, Sec. 3.1: the energy travels along
 * psi(theta) = theta + atan2(v'(theta), v(theta)) with speed sqrt(v^2 + v'^2).
 * Given the group angle phi, theta is found by bisection on psi(theta) = phi
 * (psi is monotone for the convex qP slowness curve). */
void om_group_exact(const om_mat* m, double phi, double* theta_out, double* V_out)
{
    if (mat_is_isotropic(m)) {
        *theta_out = phi;
        *V_out = sqrt(m->c22 / m->rho);
        return;
    }
    double lo = phi - M_PI / 2 + 1e-12, hi = phi + M_PI / 2 - 1e-12;
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        double v, dv;
        qp_v_dv(m, mid, &v, &dv);
        double f = mid + atan2(dv, v) - phi;
        if (f > 0.0) hi = mid; else lo = mid;
    }
    double th = 0.5 * (lo + hi), v, dv;
    qp_v_dv(m, th, &v, &dv);
    *theta_out = th;
    *V_out = sqrt(v * v + dv * dv);
}

/* Group speed for a direction at absolute angle dir in a material rotated by theta_mat. */
double om_group_speed(const om_mat* m, int model, double dir, double theta_mat)
{
    double th, V;
    if (model == 1) om_group_exact(m, dir - theta_mat, &th, &V);
    else om_group_paper(m, dir - theta_mat, &th, &V);
    return V;
}

/* The medium's group speed of material `mat` along dir: the qP models above, or the shear modes' table. */
static double med_group_speed(const om_medium* M, int mat, double dir, double theta_mat)
{
    if (M->wave_mode != 0) {
        const om_mat* m = &M->mats[mat];
        /* an isotropic mode travels at its phase speed in every direction */
        if ((M->wave_mode == 1 && mat_is_isotropic(m)) || (M->wave_mode == 2 && m->c55 == m->c66))
            return om_mode_velocity(m, M->wave_mode, 0.0);
        return om_envelope_speed(M->env + (size_t)mat * ENV_N, dir - theta_mat);
    }
    return om_group_speed(&M->mats[mat], M->group_model, dir, theta_mat);
}

/* ------------------------------------------------------------------------ */
/* Sec. 4.1: the 32 stencils, written as printed (Tables square_sten and      */
/* triangle_sten), offsets (di, dj) of A, B, C relative to D = (i, j).         */
/* [R5a] row 4-1 and [R5b] row 8-2 are garbled in print; they are restored by  */
/* the stated pairing rule (same A and D, B and C swapped).                    */
/* ------------------------------------------------------------------------ */
static const int STENCIL[32][6] = {
    /* A(di,dj)  B(di,dj)  C(di,dj) */
    {-1, -1, 0, -1, -1, 0},  /* 1-1 */
    {-1, -1, -1, 0, 0, -1},  /* 1-2 */
    {-1, 1, 0, 1, -1, 0},    /* 2-1 */
    {-1, 1, -1, 0, 0, 1},    /* 2-2 */
    {1, 1, 1, 0, 0, 1},      /* 3-1 */
    {1, 1, 0, 1, 1, 0},      /* 3-2 */
    {1, -1, 1, 0, 0, -1},    /* 4-1 [R5a] */
    {1, -1, 0, -1, 1, 0},    /* 4-2 */
    {-2, 0, -1, -1, -1, 1},  /* 5-1 */
    {-2, 0, -1, 1, -1, -1},  /* 5-2 */
    {0, 2, 1, 1, -1, 1},     /* 6-1 */
    {0, 2, -1, 1, 1, 1},     /* 6-2 */
    {0, -2, 1, -1, -1, -1},  /* 7-1 */
    {0, -2, -1, -1, 1, -1},  /* 7-2 */
    {2, 0, 1, 1, 1, -1},     /* 8-1 */
    {2, 0, 1, -1, 1, 1},     /* 8-2 [R5b] */
    {0, 2, 0, 1, 1, 1},      /* 9-1 */
    {0, 2, 1, 1, 0, 1},      /* 9-2 */
    {0, -2, 0, -1, 1, -1},   /* 10-1 */
    {0, -2, 1, -1, 0, -1},   /* 10-2 */
    {0, -2, 0, -1, -1, -1},  /* 11-1 */
    {0, -2, -1, -1, 0, -1},  /* 11-2 */
    {0, 2, 0, 1, -1, 1},     /* 12-1 */
    {0, 2, -1, 1, 0, 1},     /* 12-2 */
    {-2, 0, -1, 0, -1, 1},   /* 13-1 */
    {-2, 0, -1, 1, -1, 0},   /* 13-2 */
    {2, 0, 1, 0, 1, 1},      /* 14-1 */
    {2, 0, 1, 1, 1, 0},      /* 14-2 */
    {2, 0, 1, 0, 1, -1},     /* 15-1 */
    {2, 0, 1, -1, 1, 0},     /* 15-2 */
    {-2, 0, -1, 0, -1, -1},  /* 16-1 */
    {-2, 0, -1, -1, -1, 0},  /* 16-2 */
};

/* the 12-point diamond around D, in the slot order used by stencil records */
static const int DIAMOND[12][2] = {
    {-1, 0}, {1, 0}, {0, -1}, {0, 1}, {-1, -1}, {1, -1}, {-1, 1}, {1, 1}, {-2, 0}, {2, 0}, {0, -2}, {0, 2},
};

const int* om_stencil_table(void) { return &STENCIL[0][0]; }
const int* om_diamond_table(void) { return &DIAMOND[0][0]; }

/* Sec. 4.1 Eq. wavefront_lin_int and Sec. 4.2: the travel time at D from the
 * stencil (A, B, C): E on AC with tau_E = tau_B, F the foot of D on line EB,
 * theta' = (theta_D - theta_n + 90) mod 180, tau_D = tau_B + |FD| / v(theta').
 * [R6] material and orientation are those of D.  Positions in grid units. */
static double stencil_time(const om_medium* M, int d, const double xa[3], const double ya[3], double tA, double tB,
                           double tC)
{
    double xA = xa[0], yA = ya[0], xB = xa[1], yB = ya[1], xC = xa[2], yC = ya[2];
    double xD = 0.0, yD = 0.0;
    /* a 3, E 8, |FD| 15, theta_n 3, theta' 4, v 26 (isotropic: 2), tau_D 3 */
    g_ops += mat_is_isotropic(&M->mats[M->mat_id[d]]) ? 38 : 62;
    double a = (tB - tA) / (tC - tA);
    double xE = (1.0 - a) * xA + a * xC;
    double yE = (1.0 - a) * yA + a * yC;
    double FD = fabs((yE - yB) * (xD - xE) + (xB - xE) * (yD - yE))
                / sqrt((xB - xE) * (xB - xE) + (yB - yE) * (yB - yE));
    double theta_n = atan2(yB - yE, xB - xE);
    double theta_p = fmod(M->theta[d] - theta_n + M_PI / 2, M_PI);
    if (theta_p < 0.0) theta_p += M_PI;
    double v;
    if (M->vtable) {
        /* [R19] the table holds the qP phase speed at every integer degree of 0..180 (180-degree symmetric)
           and is interpolated linearly in speed */
        double deg = theta_p * 180.0 / M_PI;
        int k = (int)floor(deg);
        if (k < 0) k = 0;
        if (k > 179) k = 179;
        double f = deg - k;
        const om_mat* m = &M->mats[M->mat_id[d]];
        double v0 = om_mode_velocity(m, M->wave_mode, k * M_PI / 180.0);
        double v1 = om_mode_velocity(m, M->wave_mode, (k + 1) * M_PI / 180.0);
        v = (1.0 - f) * v0 + f * v1;
    } else {
        v = om_mode_velocity(&M->mats[M->mat_id[d]], M->wave_mode, theta_p);
    }
    return tB + FD * M->h / v;
}

/* Value of one stencil row at node (i, j) given neighbour times; no checks. */
double om_stencil_value(const om_medium* M, const double* tau, int i, int j, int row)
{
    const int* s = STENCIL[row];
    double xa[3] = {s[0], s[2], s[4]}, ya[3] = {s[1], s[3], s[5]};
    int nx = M->nx;
    double tA = tau[(j + s[1]) * nx + i + s[0]];
    double tB = tau[(j + s[3]) * nx + i + s[2]];
    double tC = tau[(j + s[5]) * nx + i + s[4]];
    return stencil_time(M, j * nx + i, xa, ya, tA, tB, tC);
}

/* Sec. 4.3: stencil choice, and the update U(S) of node D from a known set S.
 * known[k] (k over the 12 diamond slots) says whether that neighbour is in S;
 * t[k] holds its time.  Returns the time and writes the record:
 *   0..31  stencil row (2*(pair-1) + member-1),
 *   32+k   the fallback through diamond slot k,
 *   -1     nothing known (time = +inf).
 * Rule:
 *  - a row is feasible when A, B, C are known and tau_A < tau_B <= tau_C;
 *  - [R17] it is used only when its result is later than all three of its
 *    points (tau_D > tau_C), the paper's "tau_D > tau_A" condition extended to
 *    B and C so that every update is causal;
 *  - squares (pairs 1-8) are preferred; among them the smallest |tau_C - tau_B|
 *    wins, ties to the lower row;
 *  - otherwise triangles (pairs 9-16) by the smallest
 *    |tau_diag - ((sqrt2-1) tau_A + (2-sqrt2) tau_axis)|, ties to the lower row;
 *  - [R8] with no usable row, the straight-ray time from the best known
 *    diamond neighbour N, tau_N + |ND| / V_group(N->D), material of D. */
static double update_from_set(const om_medium* M, int i, int j, const int known[12], const double t[12], int* rec)
{
    int nx = M->nx;
    int d = j * nx + i;
    double best_metric = OM_INF, best_val = OM_INF;
    int best_row = -1;
    for (int pass = 0; pass < 2 && best_row < 0; ++pass) {
        int r0 = pass == 0 ? 0 : 16, r1 = pass == 0 ? 16 : 32;
        for (int row = r0; row < r1; ++row) {
            const int* s = STENCIL[row];
            int slot[3];
            int ok = 1;
            for (int p = 0; p < 3; ++p) {
                slot[p] = -1;
                for (int k = 0; k < 12; ++k)
                    if (DIAMOND[k][0] == s[2 * p] && DIAMOND[k][1] == s[2 * p + 1]) slot[p] = k;
                if (slot[p] < 0 || !known[slot[p]]) ok = 0;
            }
            if (!ok) continue;
            double tA = t[slot[0]], tB = t[slot[1]], tC = t[slot[2]];
            g_ops += tA < tB ? 2 : 1;
            if (!(tA < tB && tB <= tC)) continue;
            double metric;
            if (pass == 0) {
                metric = fabs(tC - tB);
            } else {
                /* the diagonal point is the one with both offsets non-zero */
                int b_is_diag = (s[2] != 0 && s[3] != 0);
                double tdiag = b_is_diag ? tB : tC, taxis = b_is_diag ? tC : tB;
                metric = fabs(tdiag - ((sqrt(2.0) - 1.0) * tA + (2.0 - sqrt(2.0)) * taxis));
            }
            double xa[3] = {s[0], s[2], s[4]}, ya[3] = {s[1], s[3], s[5]};
            g_ops += pass == 0 ? 2 : 5;         /* the metric */
            double val = stencil_time(M, d, xa, ya, tA, tB, tC);
            g_ops += 2;                          /* [R17] and the choice */
            if (!(val > tC)) continue; /* [R17] */
            if (metric < best_metric) {
                best_metric = metric;
                best_val = val;
                best_row = row;
            }
        }
    }
    if (best_row >= 0) {
        *rec = best_row;
        return best_val;
    }
    /* [R8] fallback */
    double best = OM_INF;
    int bk = -1;
    for (int k = 0; k < 12; ++k) {
        if (!known[k]) continue;
        double di = -DIAMOND[k][0], dj = -DIAMOND[k][1]; /* direction N -> D */
        double len = sqrt(di * di + dj * dj);
        double V = med_group_speed(M, M->mat_id[d], atan2(dj, di), M->theta[d]);
        double val = t[k] + len * M->h / V;
        g_ops += 2;
        if (val < best) {
            best = val;
            bk = k;
        }
    }
    *rec = bk >= 0 ? 32 + bk : -1;
    return best;
}

static int in_grid(const om_medium* M, int i, int j) { return i >= 0 && j >= 0 && i < M->nx && j < M->ny; }

/* U(D) with S = the nodes flagged in `known_node`. */
static double update_node(const om_medium* M, const double* tau, const uint8_t* known_node, int i, int j, int* rec)
{
    int known[12];
    double t[12];
    for (int k = 0; k < 12; ++k) {
        int ii = i + DIAMOND[k][0], jj = j + DIAMOND[k][1];
        known[k] = 0;
        t[k] = OM_INF;
        if (in_grid(M, ii, jj) && known_node[jj * M->nx + ii]) {
            known[k] = 1;
            t[k] = tau[jj * M->nx + ii];
        }
    }
    return update_from_set(M, i, j, known, t, rec);
}

/* ------------------------------------------------------------------------ */
/* Sec. 2: the heap-ordered Fast Marching driver.                             */
/* [R10] accepting P recomputes every non-known D in P's diamond from all of  */
/* D's known neighbours and replaces tau_D by the new estimate (the update of */
/* a close point); the heap key is (tau, linear index) and a changed key is   */
/* pushed again (stale entries are skipped).  Frozen nodes are known from the */
/* start; the initial band is every non-frozen diamond neighbour of a frozen  */
/* node, computed from the frozen set.                                        */
/* ------------------------------------------------------------------------ */
typedef struct {
    double t;
    int idx;
} hent;

static int hless(hent a, hent b) { return a.t < b.t || (a.t == b.t && a.idx < b.idx); }

typedef struct {
    hent* a;
    int n, cap;
} heap_t;

static void hpush(heap_t* h, hent e)
{
    if (h->n == h->cap) {
        h->cap = h->cap ? 2 * h->cap : 1024;
        h->a = (hent*)realloc(h->a, sizeof(hent) * (size_t)h->cap);
    }
    int k = h->n++;
    h->a[k] = e;
    while (k > 0) {
        int p = (k - 1) / 2;
        if (!hless(h->a[k], h->a[p])) break;
        hent tmp = h->a[k];
        h->a[k] = h->a[p];
        h->a[p] = tmp;
        k = p;
    }
}

static hent hpop(heap_t* h)
{
    hent top = h->a[0];
    h->a[0] = h->a[--h->n];
    int k = 0;
    for (;;) {
        int l = 2 * k + 1, r = l + 1, m = k;
        if (l < h->n && hless(h->a[l], h->a[m])) m = l;
        if (r < h->n && hless(h->a[r], h->a[m])) m = r;
        if (m == k) break;
        hent tmp = h->a[k];
        h->a[k] = h->a[m];
        h->a[m] = tmp;
        k = m;
    }
    return top;
}

/* tau: in = times of frozen nodes, out = the field.  rec: per-node record
 * (-2 frozen).  order (optional): acceptance rank of every node (-1 frozen).
 * stats[0] = accepted nodes, stats[1] = nodes finalised by the fallback,
 * stats[2] = non-causal recomputes observed (must stay 0 under [R17]).
 * Returns 0, or 1 if some node was never reached. */
static int fmm_core(const om_medium* M, const uint8_t* frozen, double* tau, int16_t* rec, int32_t* order,
                    int64_t* stats, uint8_t* known_out, int stop_cheb, int si, int sj);

int om_fmm(const om_medium* M, const uint8_t* frozen, double* tau, int16_t* rec, int32_t* order, int64_t* stats)
{
    return fmm_core(M, frozen, tau, rec, order, stats, NULL, 0, 0, 0);
}

/* The driver proper.  With stop_cheb > 0 it stops right after accepting the
 * first node at Chebyshev distance >= stop_cheb from (si, sj) (Sec. 4.4 level
 * switch) and returns the known set in known_out. */
static int fmm_core(const om_medium* M, const uint8_t* frozen, double* tau, int16_t* rec, int32_t* order,
                    int64_t* stats, uint8_t* known_out, int stop_cheb, int si, int sj)
{
    int nx = M->nx, ny = M->ny, N = nx * ny;
    uint8_t* known = (uint8_t*)calloc((size_t)N, 1);
    heap_t H = {0, 0, 0};
    int64_t accepted = 0, noncausal = 0, fallback = 0;
    for (int n = 0; n < N; ++n) {
        if (frozen[n]) {
            known[n] = 1;
            rec[n] = -2;
            if (order) order[n] = -1;
        } else {
            tau[n] = OM_INF;
            rec[n] = -1;
            if (order) order[n] = -1;
        }
    }
    /* initial band */
    for (int n = 0; n < N; ++n) {
        if (frozen[n]) continue;
        int i = n % nx, j = n / nx, touches = 0;
        for (int k = 0; k < 12; ++k) {
            int ii = i + DIAMOND[k][0], jj = j + DIAMOND[k][1];
            if (in_grid(M, ii, jj) && frozen[jj * nx + ii]) touches = 1;
        }
        if (!touches) continue;
        int r;
        double u = update_node(M, tau, known, i, j, &r);
        if (u < tau[n]) {
            tau[n] = u;
            rec[n] = (int16_t)r;
            hent e = {u, n};
            hpush(&H, e);
        }
    }
    while (H.n > 0) {
        hent e = hpop(&H);
        int p = e.idx;
        if (known[p] || e.t != tau[p]) continue; /* stale entry */
        known[p] = 1;
        if (order) order[p] = (int32_t)accepted;
        accepted++;
        if (rec[p] >= 32) fallback++;
        int pi = p % nx, pj = p / nx;
        if (stop_cheb > 0 && (abs(pi - si) >= stop_cheb || abs(pj - sj) >= stop_cheb)) break;
        for (int k = 0; k < 12; ++k) {
            int i = pi + DIAMOND[k][0], j = pj + DIAMOND[k][1];
            if (!in_grid(M, i, j)) continue;
            int d = j * nx + i;
            if (known[d]) continue;
            int r;
            double u = update_node(M, tau, known, i, j, &r);
            rec[d] = (int16_t)r;
            if (u != tau[d]) {
                if (hless((hent){u, d}, (hent){tau[p], p})) noncausal++;
                tau[d] = u;
                hent f = {u, d};
                hpush(&H, f);
            }
        }
    }
    int unreached = 0;
    for (int n = 0; n < N; ++n)
        if (!known[n]) unreached = 1;
    if (known_out) memcpy(known_out, known, (size_t)N);
    free(H.a);
    free(known);
    if (stats) {
        stats[0] = accepted;
        stats[1] = fallback;
        stats[2] = noncausal;
    }
    return unreached;
}

/* ------------------------------------------------------------------------ */
/* The local characterisation of the heap result (the causal fixed point).   */
/* For non-frozen D: sort its non-frozen finite diamond neighbours by key     */
/* (tau, index) n_1 < n_2 < ...; S_k = frozen neighbours + {n_1..n_k};        */
/* u_k = U(S_k), with u_0 = +inf when D has no frozen neighbour;              */
/* F_D = u_K for the first K with (u_K, idx_D) < key(n_{K+1}) (no n_{K+1}:    */
/* K is the last).  Under [R17] every recompute is later than the node that   */
/* triggered it, so the heap accepts nodes in key order and its output        */
/* satisfies tau = F(tau); iterating F from +inf reaches the same field.      */
/* ------------------------------------------------------------------------ */
double om_F_node(const om_medium* M, const uint8_t* frozen, const double* tau, int i, int j, int* rec_out)
{
    int nx = M->nx;
    int d = j * nx + i;
    if (frozen[d]) {
        *rec_out = -2;
        return tau[d];
    }
    int known[12], cand[12], nc = 0, any_frozen = 0;
    double t[12];
    for (int k = 0; k < 12; ++k) {
        int ii = i + DIAMOND[k][0], jj = j + DIAMOND[k][1];
        known[k] = 0;
        t[k] = OM_INF;
        if (!in_grid(M, ii, jj)) continue;
        int n = jj * nx + ii;
        t[k] = tau[n];
        if (frozen[n]) {
            known[k] = 1;
            any_frozen = 1;
        } else if (tau[n] < OM_INF) {
            cand[nc++] = k;
        }
    }
    /* sort candidates by key (tau, linear index): insertion sort */
    for (int a = 1; a < nc; ++a) {
        int k = cand[a], b = a - 1;
        int nk = (j + DIAMOND[k][1]) * nx + i + DIAMOND[k][0];
        while (b >= 0) {
            int kb = cand[b];
            int nb = (j + DIAMOND[kb][1]) * nx + i + DIAMOND[kb][0];
            g_ops += t[kb] > t[k] ? 1 : 2;
            if (t[kb] > t[k] || (t[kb] == t[k] && nb > nk)) {
                cand[b + 1] = cand[b];
                --b;
            } else break;
        }
        cand[b + 1] = k;
    }
    double u = OM_INF;
    int urec = -1;
    if (any_frozen) u = update_from_set(M, i, j, known, t, &urec);
    for (int kk = 0;; ++kk) {
        if (kk == nc) break;
        int k = cand[kk];
        int nk = (j + DIAMOND[k][1]) * nx + i + DIAMOND[k][0];
        g_ops += u < t[k] ? 1 : 2;
        if (u < t[k] || (u == t[k] && d < nk)) break; /* D precedes the next neighbour */
        known[k] = 1;
        u = update_from_set(M, i, j, known, t, &urec);
    }
    *rec_out = urec;
    return u;
}

/* ------------------------------------------------------------------------ */
/* The update of a solved field with the known set fixed by the node's own   */
/* time: S_D = frozen neighbours + the non-frozen finite neighbours whose key */
/* (tau, index) precedes (tau_D, idx_D), and the check value U(S_D) (the     */
/* FP64 convergence check of a field solved in lower precision).  At the     */
/* causal fixed point the walk of om_F_node stops exactly at this set (every  */
/* neighbour it accepted precedes D, [R17], and the next one does not), so    */
/* U(S_D) = tau_D there, with the same record.  Frozen nodes and nodes        */
/* without a value return their time with record -2 / -1.                     */
/* Parity: pinned by that fixed-point identity on solved weld fields.         */
/* ------------------------------------------------------------------------ */
double om_F_check_node(const om_medium* M, const uint8_t* frozen, const double* tau, int i, int j, int* rec_out)
{
    int nx = M->nx;
    int d = j * nx + i;
    if (frozen[d]) {
        *rec_out = -2;
        return tau[d];
    }
    if (!(tau[d] < OM_INF)) {
        *rec_out = -1;
        return tau[d];
    }
    int known[12], nknown = 0;
    double t[12];
    for (int k = 0; k < 12; ++k) {
        int ii = i + DIAMOND[k][0], jj = j + DIAMOND[k][1];
        known[k] = 0;
        t[k] = OM_INF;
        if (!in_grid(M, ii, jj)) continue;
        int n = jj * nx + ii;
        t[k] = tau[n];
        if (frozen[n] || t[k] < tau[d] || (t[k] == tau[d] && n < d)) {
            known[k] = 1;
            ++nknown;
        }
    }
    int urec = -1;
    double u = nknown ? update_from_set(M, i, j, known, t, &urec) : OM_INF;
    *rec_out = urec;
    return u;
}

void om_F_check_all(const om_medium* M, const uint8_t* frozen, const double* tau_in, double* tau_out, int16_t* rec)
{
    for (int j = 0; j < M->ny; ++j)
        for (int i = 0; i < M->nx; ++i) {
            int r;
            tau_out[j * M->nx + i] = om_F_check_node(M, frozen, tau_in, i, j, &r);
            if (rec) rec[j * M->nx + i] = (int16_t)r;
        }
}

/* One simultaneous (Jacobi) application of F to every node. */
void om_F_all(const om_medium* M, const uint8_t* frozen, const double* tau_in, double* tau_out, int16_t* rec)
{
    for (int j = 0; j < M->ny; ++j)
        for (int i = 0; i < M->nx; ++i) {
            int r;
            tau_out[j * M->nx + i] = om_F_node(M, frozen, tau_in, i, j, &r);
            if (rec) rec[j * M->nx + i] = (int16_t)r;
        }
}

/* Iterate F from +inf (frozen nodes keep their times) until nothing changes.
 * Returns the number of sweeps, or -1 when max_iter is reached. */
int om_jacobi(const om_medium* M, const uint8_t* frozen, double* tau, int16_t* rec, int max_iter)
{
    int N = M->nx * M->ny;
    double* nxt = (double*)malloc(sizeof(double) * (size_t)N);
    for (int n = 0; n < N; ++n)
        if (!frozen[n]) tau[n] = OM_INF;
    int it;
    for (it = 1; it <= max_iter; ++it) {
        om_F_all(M, frozen, tau, nxt, rec);
        int changed = 0;
        for (int n = 0; n < N; ++n) {
            if (memcmp(&nxt[n], &tau[n], sizeof(double)) != 0) changed = 1;
            tau[n] = nxt[n];
        }
        if (!changed) break;
    }
    free(nxt);
    return it > max_iter ? -1 : it;
}

/* ------------------------------------------------------------------------ */
/* Source initialisation, simple mode: every node within Chebyshev distance  */
/* r0 of the source node is frozen with the straight-ray time                 */
/* |x - x_s| / V_group(direction; material and orientation of the source)     */
/* (Sec. 4.4: straight rays are exact while the medium around the source is   */
/* homogeneous).                                                              */
/* ------------------------------------------------------------------------ */
void om_init_radius(const om_medium* M, int si, int sj, int r0, uint8_t* frozen, double* tau)
{
    int nx = M->nx;
    int s = sj * nx + si;
    for (int n = 0; n < nx * M->ny; ++n) {
        frozen[n] = 0;
        tau[n] = OM_INF;
    }
    for (int dj = -r0; dj <= r0; ++dj)
        for (int di = -r0; di <= r0; ++di) {
            int i = si + di, j = sj + dj;
            if (!in_grid(M, i, j)) continue;
            int n = j * nx + i;
            frozen[n] = 1;
            if (di == 0 && dj == 0) {
                tau[n] = 0.0;
                continue;
            }
            double dist = sqrt((double)(di * di + dj * dj)) * M->h;
            tau[n] = dist / med_group_speed(M, M->mat_id[s], atan2((double)dj, (double)di), M->theta[s]);
        }
}

/* ------------------------------------------------------------------------ */
/* Sec. 5.1: ray tracing through a travel-time field by Fermat's principle.   */
/* The ray starts at `start` and walks to `target`, the source of the field   */
/* (reciprocity, Sec. 5.1).  Each step picks the plane family most            */
/* perpendicular to the last segment (first step: start -> target), places   */
/* the next plane of that family plane_step cells ahead (rounded so that it   */
/* passes through grid points) [R12], evaluates                               */
/*   cost(C) = |BC| / V_group(BC) + tau(C)                                    */
/* at the grid nodes C of the plane inside a window of +-halfwidth nodes      */
/* around the continuation of the last direction, fits a parabola through     */
/* every local minimum and its two neighbours and moves to the lowest         */
/* vertex.  It stops when closer than stop_radius cells to the target.        */
/* Segment material: the node nearest the segment midpoint.                   */
/* ------------------------------------------------------------------------ */
typedef struct {
    int plane_step;
    int halfwidth;
    double stop_radius;
    int max_pts;
    int family; /* -1: the family most perpendicular to the ray at every step; 0..3: one fixed family */
} om_ray_opts;

/* families: 0 vertical x=c, 1 horizontal y=c, 2 diagonal x-y=c, 3 diagonal x+y=c */
static const double FAM_N[4][2] = {{1, 0}, {0, 1}, {1, -1}, {1, 1}};
static const double FAM_T[4][2] = {{0, 1}, {1, 0}, {1, 1}, {1, -1}}; /* node step along the plane */

static double seg_time(const om_medium* M, double x0, double y0, double x1, double y1)
{
    double dx = x1 - x0, dy = y1 - y0;
    double len = sqrt(dx * dx + dy * dy);
    if (len == 0.0) return 0.0;
    int mi = (int)floor(0.5 * (x0 + x1) + 0.5), mj = (int)floor(0.5 * (y0 + y1) + 0.5);
    if (mi < 0) mi = 0;
    if (mj < 0) mj = 0;
    if (mi >= M->nx) mi = M->nx - 1;
    if (mj >= M->ny) mj = M->ny - 1;
    int n = mj * M->nx + mi;
    double V = med_group_speed(M, M->mat_id[n], atan2(dy, dx), M->theta[n]);
    return len * M->h / V;
}

/* returns 0 ok, 1 step cap reached; pts holds (x, y) pairs in grid units */
int om_trace_ray(const om_medium* M, const double* tau, double x0, double y0, double xt, double yt,
                 const om_ray_opts* o, double* pts, int* npts_out)
{
    int np = 0;
    int cap = o->max_pts;
    double bx = x0, by = y0, dx = xt - x0, dy = yt - y0;
    /* the candidates of one plane: at most 2 halfwidth + 1 nodes */
    double* cost = (double*)malloc(sizeof(double) * (size_t)(2 * o->halfwidth + 1));
    int* pidx = (int*)malloc(sizeof(int) * (size_t)(2 * o->halfwidth + 1));
    pts[2 * np] = bx;
    pts[2 * np + 1] = by;
    np++;
    int status = 1;
    while (np < cap) {
        double rx = xt - bx, ry = yt - by;
        if (sqrt(rx * rx + ry * ry) < o->stop_radius) {
            pts[2 * np] = xt;
            pts[2 * np + 1] = yt;
            np++;
            status = 0;
            break;
        }
        /* plane family most perpendicular to the current direction, or the fixed one (Sec. 5.1 uses
           each of the four sets on its own, and changes set along the ray) */
        double dl = sqrt(dx * dx + dy * dy);
        int fam = 0;
        if (o->family >= 0) {
            fam = o->family;
        } else {
            double bestc = -1.0;
            for (int f = 0; f < 4; ++f) {
                double nl = sqrt(FAM_N[f][0] * FAM_N[f][0] + FAM_N[f][1] * FAM_N[f][1]);
                double c = fabs(dx * FAM_N[f][0] + dy * FAM_N[f][1]) / (dl * nl);
                if (c > bestc + 1e-12) {
                    bestc = c;
                    fam = f;
                }
            }
        }
        double nxf = FAM_N[fam][0], nyf = FAM_N[fam][1];
        double qB = nxf * bx + nyf * by;
        double qT = nxf * xt + nyf * yt;
        /* a fixed family crosses its planes towards the target, each plane once */
        double sg = o->family >= 0 ? (qT - qB >= 0.0 ? 1.0 : -1.0) : ((dx * nxf + dy * nyf) >= 0.0 ? 1.0 : -1.0);
        double scale = sqrt(nxf * nxf + nyf * nyf); /* q units per cell of normal distance */
        double qn = floor(qB + sg * o->plane_step * scale + 0.5);
        /* [R12] never place the plane beyond the target */
        if (sg * (qn - qT) > 0.0) qn = floor(qT + 0.5);
        if (sg * (qn - qB) < 0.5) {
            /* the target lies between B and the next plane: finish */
            pts[2 * np] = xt;
            pts[2 * np + 1] = yt;
            np++;
            status = 0;
            break;
        }
        /* where the current direction meets the plane */
        double t = (qn - qB) / (dx * nxf + dy * nyf);
        double px = bx + t * dx, py = by + t * dy;
        /* node parameter p along the plane: node(p) = base + p * FAM_T */
        double bxn, byn; /* node at p = 0 on the plane */
        if (fam == 0) { bxn = qn; byn = 0; }
        else if (fam == 1) { bxn = 0; byn = qn; }
        else if (fam == 2) { bxn = 0; byn = -qn; }
        else { bxn = 0; byn = qn; }
        double tx = FAM_T[fam][0], ty = FAM_T[fam][1];
        double pc = (fam == 0) ? py : px; /* for families 1-3 the x coordinate is the parameter */
        int p0 = (int)floor(pc + 0.5);
        /* [R18] the window is centred on the part of the plane inside the grid: a set of planes nearly
           parallel to the ray meets the ray's line far off the grid */
        {
            int qi = (int)qn, lo, hi;
            if (fam == 0) { lo = 0; hi = M->ny - 1; }
            else if (fam == 1) { lo = 0; hi = M->nx - 1; }
            else if (fam == 2) { lo = qi > 0 ? qi : 0; hi = M->nx - 1 < M->ny - 1 + qi ? M->nx - 1 : M->ny - 1 + qi; }
            else { lo = qi - (M->ny - 1) > 0 ? qi - (M->ny - 1) : 0; hi = M->nx - 1 < qi ? M->nx - 1 : qi; }
            if (lo <= hi) {
                if (p0 < lo) p0 = lo;
                if (p0 > hi) p0 = hi;
            }
        }
        int plo = p0 - o->halfwidth, phi = p0 + o->halfwidth;
        /* clip to nodes inside the grid */
        int nc = 0;
        for (int p = plo; p <= phi; ++p) {
            double cx = bxn + p * tx, cy = byn + p * ty;
            int ci = (int)cx, cj = (int)cy;
            if (cx < 0 || cy < 0 || ci >= M->nx || cj >= M->ny) continue;
            double tc = tau[cj * M->nx + ci];
            if (!(tc < OM_INF)) continue;
            cost[nc] = seg_time(M, bx, by, cx, cy) + tc;
            pidx[nc] = p;
            nc++;
        }
        if (nc == 0) break; /* no candidate: incomplete */
        /* local minima, parabola through each and its neighbours */
        double best = OM_INF, bpos = 0.0;
        for (int k = 0; k < nc; ++k) {
            int contig_l = k > 0 && pidx[k - 1] == pidx[k] - 1;
            int contig_r = k + 1 < nc && pidx[k + 1] == pidx[k] + 1;
            double cl = contig_l ? cost[k - 1] : OM_INF;
            double cr = contig_r ? cost[k + 1] : OM_INF;
            if (!(cost[k] < cl && cost[k] <= cr)) continue;
            double val = cost[k], off = 0.0;
            if (contig_l && contig_r) {
                double den = cl - 2.0 * cost[k] + cr;
                if (den > 0.0) {
                    off = (cl - cr) / (2.0 * den);
                    val = cost[k] - (cl - cr) * (cl - cr) / (8.0 * den);
                }
            }
            if (val < best) {
                best = val;
                bpos = pidx[k] + off;
            }
        }
        double nxp = bxn + bpos * tx, nyp = byn + bpos * ty;
        dx = nxp - bx;
        dy = nyp - by;
        bx = nxp;
        by = nyp;
        pts[2 * np] = bx;
        pts[2 * np + 1] = by;
        np++;
    }
    free(cost);
    free(pidx);
    *npts_out = np;
    return status;
}

/* [R13] travel time along a polyline: every segment is split where it crosses
 * the borders x = k + 1/2, y = k + 1/2 of the nearest-node cells; each piece
 * takes the group speed of the node whose cell holds it, in the segment's
 * direction. */
double om_path_time(const om_medium* M, const double* pts, int npts)
{
    double total = 0.0;
    for (int s = 0; s + 1 < npts; ++s) {
        double x0 = pts[2 * s], y0 = pts[2 * s + 1], x1 = pts[2 * s + 2], y1 = pts[2 * s + 3];
        double dx = x1 - x0, dy = y1 - y0;
        double len = sqrt(dx * dx + dy * dy);
        if (len == 0.0) continue;
        double dir = atan2(dy, dx);
        /* crossing parameters */
        double ts[4096];
        int nt = 0;
        ts[nt++] = 0.0;
        if (dx != 0.0) {
            double a = fmin(x0, x1), b = fmax(x0, x1);
            for (double k = ceil(a - 0.5) + 0.5; k < b && nt < 4000; k += 1.0)
                if (k > a) ts[nt++] = (k - x0) / dx;
        }
        if (dy != 0.0) {
            double a = fmin(y0, y1), b = fmax(y0, y1);
            for (double k = ceil(a - 0.5) + 0.5; k < b && nt < 4090; k += 1.0)
                if (k > a) ts[nt++] = (k - y0) / dy;
        }
        ts[nt++] = 1.0;
        /* sort */
        for (int a = 1; a < nt; ++a) {
            double v = ts[a];
            int b = a - 1;
            while (b >= 0 && ts[b] > v) {
                ts[b + 1] = ts[b];
                --b;
            }
            ts[b + 1] = v;
        }
        for (int k = 0; k + 1 < nt; ++k) {
            double ta = ts[k], tb = ts[k + 1];
            if (tb <= ta) continue;
            double tm = 0.5 * (ta + tb);
            int mi = (int)floor(x0 + tm * dx + 0.5), mj = (int)floor(y0 + tm * dy + 0.5);
            if (mi < 0) mi = 0;
            if (mj < 0) mj = 0;
            if (mi >= M->nx) mi = M->nx - 1;
            if (mj >= M->ny) mj = M->ny - 1;
            int n = mj * M->nx + mi;
            double V = med_group_speed(M, M->mat_id[n], dir, M->theta[n]);
            total += (tb - ta) * len * M->h / V;
        }
    }
    return total;
}

/* ------------------------------------------------------------------------ */
/* Sec. 4.4: near-source grid hierarchy.  Levels of relative density d_l     */
/* (27, 9, 3 in the paper) cover the squares of Chebyshev half-width R_l     */
/* (1, 6, 13 original cells) around the source, clipped to the grid.  Fine   */
/* nodes take the material and orientation of the nearest original node      */
/* (unique for odd d).  On the finest level every node inside the source's  */
/* own cell (|dx|, |dy| < 1/2 original cell) gets the straight-ray time.     */
/* Each level runs the same FMM until [R11] a node on the boundary of its    */
/* square is accepted; the known nodes that coincide with nodes of the next  */
/* (coarser) level are carried over as frozen nodes there.  The last level   */
/* hands its known nodes to the original grid, where they are returned as    */
/* frozen nodes with their times.  Returns 0.                                 */
/* ------------------------------------------------------------------------ */
int om_init_hierarchy(const om_medium* M, int si, int sj, int nlev, const int* dens, const int* radius,
                      uint8_t* frozen_out, double* tau_out)
{
    int nx = M->nx, ny = M->ny;
    double th_src = M->theta[sj * nx + si];
    /* previous level's known set, on its own grid */
    uint8_t* pk = NULL;
    double* pt = NULL;
    int pa0 = 0, pb0 = 0, pw = 0, ph = 0, pdens = 0;
    for (int l = 0; l <= nlev; ++l) {
        int d = l < nlev ? dens[l] : 1;
        int R = l < nlev ? radius[l] : 0;
        /* level grid: fine offsets a in [a0, a1] (fine cells), clipped to the grid */
        int a0, a1, b0, b1;
        if (l < nlev) {
            a0 = -R * d; a1 = R * d; b0 = -R * d; b1 = R * d;
            if (a0 < -si * d) a0 = -si * d;
            if (a1 > (nx - 1 - si) * d) a1 = (nx - 1 - si) * d;
            if (b0 < -sj * d) b0 = -sj * d;
            if (b1 > (ny - 1 - sj) * d) b1 = (ny - 1 - sj) * d;
        } else {
            a0 = -si; a1 = nx - 1 - si; b0 = -sj; b1 = ny - 1 - sj;
        }
        int w = a1 - a0 + 1, hgt = b1 - b0 + 1, N = w * hgt;
        int32_t* mid = (int32_t*)malloc(sizeof(int32_t) * (size_t)N);
        double* th = (double*)malloc(sizeof(double) * (size_t)N);
        uint8_t* fr = (uint8_t*)calloc((size_t)N, 1);
        double* tau = (double*)malloc(sizeof(double) * (size_t)N);
        int16_t* rec = (int16_t*)malloc(sizeof(int16_t) * (size_t)N);
        uint8_t* kn = (uint8_t*)calloc((size_t)N, 1);
        for (int b = b0; b <= b1; ++b)
            for (int a = a0; a <= a1; ++a) {
                int n = (b - b0) * w + (a - a0);
                /* nearest original node (exact: 2a/d is never odd for odd d) */
                int oi = si + (int)floor((double)a / d + 0.5), oj = sj + (int)floor((double)b / d + 0.5);
                mid[n] = M->mat_id[oj * nx + oi];
                th[n] = M->theta[oj * nx + oi];
                tau[n] = OM_INF;
                if (l == 0) {
                    if (2 * abs(a) < d && 2 * abs(b) < d) {
                        fr[n] = 1;
                        double dist = sqrt((double)a * a + (double)b * b) * M->h / d;
                        tau[n] = (a == 0 && b == 0)
                                     ? 0.0
                                     : dist / med_group_speed(M, M->mat_id[sj * nx + si], atan2((double)b, (double)a),
                                                              th_src);
                    }
                } else {
                    /* coincides with a node of the previous level? */
                    int fa = a * (pdens / d), fb = b * (pdens / d);
                    int qa = fa - pa0, qb = fb - pb0;
                    if (qa >= 0 && qa < pw && qb >= 0 && qb < ph) {
                        int qn = qb * pw + qa;
                        if (pk[qn]) {
                            fr[n] = 1;
                            tau[n] = pt[qn];
                        }
                    }
                }
            }
        if (l == nlev) {
            for (int n = 0; n < N; ++n) {
                frozen_out[n] = fr[n];
                tau_out[n] = fr[n] ? tau[n] : OM_INF;
            }
            free(mid); free(th); free(fr); free(tau); free(rec); free(kn);
            break;
        }
        om_medium L = *M;
        L.nx = w;
        L.ny = hgt;
        L.h = M->h / d;
        L.mat_id = mid;
        L.theta = th;
        fmm_core(&L, fr, tau, rec, NULL, NULL, kn, R * d, -a0, -b0);
        /* when the square is clipped away on every side there is no boundary
           node; fmm_core then runs to completion and every node is known */
        free(pk);
        free(pt);
        pk = kn;
        pt = tau;
        pa0 = a0; pb0 = b0; pw = w; ph = hgt; pdens = d;
        free(mid); free(th); free(fr); free(rec);
    }
    free(pk);
    free(pt);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Discrete adjoint of the solve (reverse mode), for the misfit gradient.    */
/* Every non-frozen node's time is the chosen stencil (or fallback) applied  */
/* to at most three earlier nodes and to the orientation at the node; a      */
/* frozen node's time is the straight-ray time from the source, which        */
/* depends on the orientation at the source.  Walking the nodes in reverse   */
/* acceptance order, lambda_D = seed_D + sum over later users E of           */
/* lambda_E d tau_E / d tau_D, and dL/dtheta of a region sums                */
/* lambda_D d tau_D / d theta_D over its nodes (frozen nodes: the source's   */
/* region).  The local partial derivatives are central differences of the    */
/* local formulas above (steps 1e-4 of the stencil's time span, 1e-6 rad).   */
/* ------------------------------------------------------------------------ */
static double stencil_time_theta(const om_medium* M, int d, const double xa[3], const double ya[3], double tA,
                                 double tB, double tC, double theta)
{
    double* th = (double*)M->theta; /* the formula reads the orientation of D from the medium */
    double keep = th[d];
    th[d] = theta;
    double v = stencil_time(M, d, xa, ya, tA, tB, tC);
    th[d] = keep;
    return v;
}

/* seeds[node] = dL/dtau at that node; region[node] = region index of the node;
 * grad[nregions] += dL/dtheta.  order = acceptance ranks from om_fmm. */
void om_adjoint(const om_medium* M, const uint8_t* frozen, const double* tau, const int16_t* rec,
                const int32_t* order, const double* seeds, int si, int sj, const int32_t* region, int nregions,
                double* grad)
{
    int nx = M->nx, N = M->nx * M->ny;
    double* lam = (double*)malloc(sizeof(double) * (size_t)N);
    int* byrank = (int*)malloc(sizeof(int) * (size_t)N);
    int nacc = 0;
    for (int n = 0; n < N; ++n) {
        lam[n] = seeds[n];
        if (order[n] >= 0) nacc = order[n] + 1 > nacc ? order[n] + 1 : nacc;
    }
    for (int n = 0; n < N; ++n)
        if (order[n] >= 0) byrank[order[n]] = n;
    (void)nregions;
    for (int k = nacc - 1; k >= 0; --k) {
        int d = byrank[k];
        int i = d % nx, j = d / nx;
        int r = rec[d];
        const double th0 = M->theta[d];
        if (r >= 0 && r < 32) {
            const int* s = STENCIL[r];
            double xa[3] = {s[0], s[2], s[4]}, ya[3] = {s[1], s[3], s[5]};
            int nA = (j + s[1]) * nx + i + s[0], nB = (j + s[3]) * nx + i + s[2], nC = (j + s[5]) * nx + i + s[4];
            double tA = tau[nA], tB = tau[nB], tC = tau[nC];
            double e = 1e-4 * (tC - tA);
            double dA = (stencil_time(M, d, xa, ya, tA + e, tB, tC) - stencil_time(M, d, xa, ya, tA - e, tB, tC)) / (2 * e);
            double dB = (stencil_time(M, d, xa, ya, tA, tB + e, tC) - stencil_time(M, d, xa, ya, tA, tB - e, tC)) / (2 * e);
            double dC = (stencil_time(M, d, xa, ya, tA, tB, tC + e) - stencil_time(M, d, xa, ya, tA, tB, tC - e)) / (2 * e);
            double dT = (stencil_time_theta(M, d, xa, ya, tA, tB, tC, th0 + 1e-6)
                         - stencil_time_theta(M, d, xa, ya, tA, tB, tC, th0 - 1e-6)) / 2e-6;
            lam[nA] += lam[d] * dA;
            lam[nB] += lam[d] * dB;
            lam[nC] += lam[d] * dC;
            grad[region[d]] += lam[d] * dT;
        } else if (r >= 32) {
            int k2 = r - 32;
            int nN = (j + DIAMOND[k2][1]) * nx + i + DIAMOND[k2][0];
            double di = -DIAMOND[k2][0], dj = -DIAMOND[k2][1];
            double len = sqrt(di * di + dj * dj);
            double dir = atan2(dj, di);
            double Vp = med_group_speed(M, M->mat_id[d], dir, th0 + 1e-6);
            double Vm = med_group_speed(M, M->mat_id[d], dir, th0 - 1e-6);
            double dT = (len * M->h / Vp - len * M->h / Vm) / 2e-6;
            lam[nN] += lam[d];
            grad[region[d]] += lam[d] * dT;
        }
    }
    /* frozen nodes: straight-ray times from the source, orientation of the source */
    int s = sj * nx + si;
    for (int n = 0; n < N; ++n) {
        if (!frozen[n] || n == s || lam[n] == 0.0) continue;
        double di = n % nx - si, dj = n / nx - sj;
        double dist = sqrt(di * di + dj * dj) * M->h;
        double dir = atan2(dj, di);
        double th = M->theta[s];
        double dT = (dist / med_group_speed(M, M->mat_id[s], dir, th + 1e-6)
                     - dist / med_group_speed(M, M->mat_id[s], dir, th - 1e-6)) / 2e-6;
        grad[region[s]] += lam[n] * dT;
    }
    free(lam);
    free(byrank);
}
