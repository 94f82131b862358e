/*
 * impm_oracle.c -- plain FP64 CPU oracle of the IMPM elastomer substep.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * CPU-baseline leg of bench.py load this library.  The product path never
 * does, and this file shares no code with the CUDA path.
 *
 * Follows Sec. III-A of the paper: particle-to-grid (Eqs. 1-4), grid
 * boundary handling (Eq. 5), grid-to-particle (Eqs. 6-8), the relative-rest
 * check loop (Algorithm 1) and particle movement (Eq. 9).  Where the paper
 * is silent or garbled the readings are:
 *   weights      quadratic B-spline, 3x3x3 nodes, D^-1 = 4/dx^2 (Eqs. 1, 4, 7)
 *   Eq. 3        the affine term carries the particle mass: w m (v + C d)
 *   X_g          the position of the receiving node i
 *   S_p          Kirchhoff stress of compressible Neo-Hookean:
 *                tau = mu (F F^T - I) + lambda ln(J) I
 *   Eq. 7        C = (4/dx^2) sum_i w V_i (x_i - x_p)^T (grid velocity, outer product)
 *   gravity      added to nodes with M > 0 after Eq. 5
 *   walls        all velocity components zeroed on the 2-node ring at +-x, +-y, +z
 *   fixed base   nodes at physical z index <= 0 get V = 0; bottom-layer
 *                particles get v_z = 0 after G2P (Algorithm 1)
 *   object       rigid analytic SDF; stick/slip Coulomb projection at nodes
 *                with phi <= 0 (relative rest when |v_t| <= mu |v_n|)
 *   object particles (optional, the paper's own coupling, Sec. III-A and
 *                Sec. IV-B): the indenter as rigid particles at the pose of
 *                the substep, each with the prescribed velocity
 *                v_lin + omega z x (x - c), the affine field of that motion
 *                (C = omega [[0,-1,0],[1,0,0],[0,0,0]]) and no stress, added
 *                to the grid after the elastomer in every pass (Eqs. 1-3);
 *                the SDF contact projection is then off
 *   friction     Sec. VI names inaccurate relative sliding over long
 *                distances as a limitation; the optional kinetic
 *                coefficient mu_k <= mu sets the slip once |v_t| > mu |v_n|
 *                (|v_t| is reduced by mu_k |v_n|); mu_k <= 0 means mu_k = mu
 *   check        tangential (xy) velocity of the calibration particle x_e
 *                against the object velocity there; x_o = indenter tip
 *   state        x and F are updated once, on the accepted (or last) pass
 *
 * Serial, particle-index order; grid sums accumulate in that order.  IEEE
 * double, round to nearest, built with -ffp-contract=off.
 *
 * Pins (tests/test_oracle_pins.py): B-spline moments; Neo-Hookean stress
 * against finite differences of its energy, rotation covariance and Hooke's
 * law; P2G mass, momentum and APIC angular momentum; exact transfer of
 * affine velocity fields; Eq. 5 with gravity and the wall-ring and base
 * rules on a grid of known momenta; G2P of a uniform field with the
 * bottom-layer rule; free fall in closed form; energy balance of a free
 * elastic oscillation; uniaxial compression against linear elasticity; SDF
 * surface points, eikonal property and gradients; contact projection
 * invariants; surface readout closed forms; the displacement splat (rigid
 * translation, linear fields, untagged and unreached pixels); the sphere's
 * underside height map; keyframe interpolation; the
 * relative-rest loop (a pure press accepts every first pass; a sticking
 * slip needs repeated passes); the relative-rest check itself on
 * hand-worked slip and turn states (threshold x the object's tangential
 * speed, xy components only, the out-of-contact and no-tangential-motion
 * accepts); a sticking slip or turn drags the contact
 * patch the indenter's way by less than the indenter moved, and without
 * friction it stays in place; the static/kinetic projection on hand-worked
 * cases and a long slide whose drag falls with the kinetic coefficient;
 * object particles transfer the rigid motion to every node exactly (with
 * their total mass and momentum) and press the gel like the SDF contact.
 * Partly unpinned: the exact lag of the gel behind a sticking indenter over
 * long stick/slip trajectories has no closed form (checked against the
 * CUDA path).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_TAG_BOTTOM 0x80000000u
#define ORC_TAG_TOP 0x40000000u

enum { ORC_NONE = -1, ORC_SPHERE = 0, ORC_CYLINDER = 1, ORC_BOX = 2, ORC_PRISM = 3, ORC_PERLIN = 4 };
enum { ORC_BASE_FIXED = 0, ORC_BASE_SLIP = 1, ORC_BASE_FREE = 2 };
enum { ORC_OK = 0, ORC_ERR_DOMAIN = 1, ORC_ERR_NUMERIC = 2, ORC_ERR_ARG = 3 };

typedef struct {
    int cx, cy, cz;          /* gel cells */
    int nx, ny, nz;          /* node box */
    int ox, oy, oz;          /* box index of physical node 0 */
    int base_mode, walls, limit, ppc;
    int pad_;
    double dx, dt, rho, E, nu;
    double g[3];
    double threshold;
} orc_scene;

typedef struct {
    int kind;
    int pad_;
    double p[8];
    double mu;               /* (static) friction coefficient: stick when |v_t| <= mu |v_n| */
    double tip_offset;       /* SDF centre height above the tip */
    int perm[256];
    double mu_k;             /* kinetic coefficient of the slip; <= 0: mu */
    const double *obj_q;     /* n_obj object particles in the indenter frame (x, y, z about c) */
    long n_obj;              /* > 0: the object is these particles (no SDF contact) */
    double obj_m;            /* mass of one object particle */
} orc_indenter;

typedef struct {
    double tip[3];           /* x_o: lowest point of the object */
    double c[3];             /* SDF frame centre */
    double yaw, cs, sn;
    double vlin[3];          /* linear velocity over this substep */
    double omega;            /* yaw rate */
} orc_pose;

/* ------------------------------------------------------------------ basics */

/* Quadratic B-spline weights along one axis (reading of the kernel of Eq. 1). */
void orc_weights(double xp, double dx, int *base, double w[3])
{
    double u = xp / dx;
    int b = (int)floor(u - 0.5);
    double f = u - (double)b;
    w[0] = 0.5 * (1.5 - f) * (1.5 - f);
    w[1] = 0.75 - (f - 1.0) * (f - 1.0);
    w[2] = 0.5 * (f - 0.5) * (f - 0.5);
    *base = b;
}

void orc_lame(double E, double nu, double *mu, double *lam)
{
    *mu = E / (2.0 * (1.0 + nu));
    *lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
}

static double det3(const double F[9])
{
    return F[0] * (F[4] * F[8] - F[5] * F[7])
         - F[1] * (F[3] * F[8] - F[5] * F[6])
         + F[2] * (F[3] * F[7] - F[4] * F[6]);
}

/* S_p of Eq. 4: Kirchhoff stress of compressible Neo-Hookean. Row-major 3x3. */
int orc_kirchhoff(const double F[9], double mu, double lam, double tau[9])
{
    double J = det3(F);
    if (!(J > 0.0)) return ORC_ERR_NUMERIC;
    double lnJ = log(J);
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += F[r * 3 + k] * F[c * 3 + k];
            tau[r * 3 + c] = mu * (s - (r == c ? 1.0 : 0.0)) + (r == c ? lam * lnJ : 0.0);
        }
    return ORC_OK;
}

/* ------------------------------------------------------------------ pose */

/* Piecewise-linear indenter pose at substep k.  kf rows: substep, tip xyz, yaw. */
void orc_pose_eval(const double *kf, int nkf, int k, double dt, double tip_offset, orc_pose *o)
{
    int i = -1;
    for (int a = 0; a < nkf; ++a)
        if (kf[a * 5] <= (double)k) i = a;
    double tip[3], yaw, vl[3] = {0, 0, 0}, om = 0.0;
    if (i < 0 || i == nkf - 1) {
        int a = i < 0 ? 0 : i;
        tip[0] = kf[a * 5 + 1]; tip[1] = kf[a * 5 + 2]; tip[2] = kf[a * 5 + 3];
        yaw = kf[a * 5 + 4];
    } else {
        const double *p0 = kf + i * 5, *p1 = kf + (i + 1) * 5;
        double span = p1[0] - p0[0];
        double al = ((double)k - p0[0]) / span;
        for (int d = 0; d < 3; ++d) {
            tip[d] = p0[1 + d] + al * (p1[1 + d] - p0[1 + d]);
            vl[d] = (p1[1 + d] - p0[1 + d]) / (span * dt);
        }
        yaw = p0[4] + al * (p1[4] - p0[4]);
        om = (p1[4] - p0[4]) / (span * dt);
    }
    for (int d = 0; d < 3; ++d) { o->tip[d] = tip[d]; o->c[d] = tip[d]; o->vlin[d] = vl[d]; }
    o->c[2] = tip[2] + tip_offset;
    o->yaw = yaw; o->cs = cos(yaw); o->sn = sin(yaw); o->omega = om;
}

/* ------------------------------------------------------------------ SDFs */

static double sgn(double a) { return a < 0.0 ? -1.0 : 1.0; }

/* Rounded box in n dims (n = 2 or 3): half sizes h, edge radius re. */
static double round_box(int n, const double *q, const double *h, double re, double *g)
{
    double d[3], o[3], L2 = 0.0, dmax = -1e300;
    int kmax = 0;
    for (int a = 0; a < n; ++a) {
        d[a] = fabs(q[a]) - (h[a] - re);
        o[a] = d[a] > 0.0 ? d[a] : 0.0;
        L2 += o[a] * o[a];
        if (d[a] > dmax) { dmax = d[a]; kmax = a; }
    }
    double L = sqrt(L2);
    double phi = L + (dmax < 0.0 ? dmax : 0.0) - re;
    for (int a = 0; a < n; ++a) g[a] = 0.0;
    if (dmax > 0.0) {
        for (int a = 0; a < n; ++a) g[a] = sgn(q[a]) * o[a] / L;
    } else {
        g[kmax] = sgn(q[kmax]);
    }
    return phi;
}

/* Signed distance to an equilateral triangle (apex towards -z) of inradius r
 * in the (y, z) plane, exact, with gradient. */
static double tri_sdf(double y, double z, double r, double g[2])
{
    const double s3 = sqrt(3.0);
    double V[3][2] = {{0.0, -2.0 * r}, {s3 * r, r}, {-s3 * r, r}};
    double N[3][2] = {{0.0, 1.0}, {0.5 * s3, -0.5}, {-0.5 * s3, -0.5}};
    /* edge e joins V[(e+1)%3] and V[(e+2)%3]; its outward normal is N[e] */
    double smax = -1e300; int emax = 0;
    for (int e = 0; e < 3; ++e) {
        double s = N[e][0] * y + N[e][1] * z - r;
        if (s > smax) { smax = s; emax = e; }
    }
    if (smax <= 0.0) { g[0] = N[emax][0]; g[1] = N[emax][1]; return smax; }
    double best = 1e300, by = 0.0, bz = 0.0;
    for (int e = 0; e < 3; ++e) {
        const double *P0 = V[(e + 1) % 3], *P1 = V[(e + 2) % 3];
        double ey = P1[0] - P0[0], ez = P1[1] - P0[1];
        double t = ((y - P0[0]) * ey + (z - P0[1]) * ez) / (ey * ey + ez * ez);
        if (t < 0.0) t = 0.0;
        if (t > 1.0) t = 1.0;
        double cy = P0[0] + t * ey, cz = P0[1] + t * ez;
        double dd = sqrt((y - cy) * (y - cy) + (z - cz) * (z - cz));
        if (dd < best) { best = dd; by = y - cy; bz = z - cz; }
    }
    g[0] = by / best; g[1] = bz / best;
    return best;
}

/* Improved noise (Perlin 2002) on the plane z = 0, value and xy gradient. */
static double grad3(int h, double x, double y, double z)
{
    h &= 15;
    double u = h < 8 ? x : y;
    double v = h < 4 ? y : ((h == 12 || h == 14) ? x : z);
    return ((h & 1) ? -u : u) + ((h & 2) ? -v : v);
}

static double fade(double t) { return t * t * t * (t * (t * 6.0 - 15.0) + 10.0); }
static double dfade(double t) { return 30.0 * t * t * (t - 1.0) * (t - 1.0); }

static double noise2(const int *perm, double x, double y, double *gx, double *gy)
{
    double fx = floor(x), fy = floor(y);
    int X = ((int)fx) & 255, Y = ((int)fy) & 255;
    x -= fx; y -= fy;
#define P(i) perm[(i) & 255]
    int A = P(X) + Y, B = P(X + 1) + Y;
    int hAA = P(P(A)), hBA = P(P(B)), hAB = P(P(A + 1)), hBB = P(P(B + 1));
#undef P
    double g00 = grad3(hAA, x, y, 0.0), g10 = grad3(hBA, x - 1.0, y, 0.0);
    double g01 = grad3(hAB, x, y - 1.0, 0.0), g11 = grad3(hBB, x - 1.0, y - 1.0, 0.0);
    /* each corner gradient is linear: d/dx and d/dy of grad3 */
    double a00 = grad3(hAA, 1, 0, 0), b00 = grad3(hAA, 0, 1, 0);
    double a10 = grad3(hBA, 1, 0, 0), b10 = grad3(hBA, 0, 1, 0);
    double a01 = grad3(hAB, 1, 0, 0), b01 = grad3(hAB, 0, 1, 0);
    double a11 = grad3(hBB, 1, 0, 0), b11 = grad3(hBB, 0, 1, 0);
    double u = fade(x), v = fade(y), du = dfade(x), dv = dfade(y);
    double l0 = g00 + u * (g10 - g00), l1 = g01 + u * (g11 - g01);
    double n = l0 + v * (l1 - l0);
    double dl0x = a00 + u * (a10 - a00) + du * (g10 - g00);
    double dl1x = a01 + u * (a11 - a01) + du * (g11 - g01);
    double dl0y = b00 + u * (b10 - b00);
    double dl1y = b01 + u * (b11 - b01);
    *gx = dl0x + v * (dl1x - dl0x);
    *gy = dl0y + v * (dl1y - dl0y) + dv * (l1 - l0);
    return n;
}

/* SDF of the indenter in its local frame; g = local gradient. */
double orc_sdf_local(const orc_indenter *ind, const double q[3], double g[3])
{
    const double *p = ind->p;
    switch (ind->kind) {
    case ORC_SPHERE: {
        double d = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2]);
        if (d > 0.0) { g[0] = q[0] / d; g[1] = q[1] / d; g[2] = q[2] / d; }
        else { g[0] = 0.0; g[1] = 0.0; g[2] = -1.0; }
        return d - p[0];
    }
    case ORC_CYLINDER: {
        double rho = sqrt(q[0] * q[0] + q[1] * q[1]);
        double q2[2] = {rho, q[2]}, h2[2] = {p[0], 0.5 * p[1]}, g2[2];
        double phi = round_box(2, q2, h2, p[2], g2);
        double ex = 1.0, ey = 0.0;
        if (rho > 0.0) { ex = q[0] / rho; ey = q[1] / rho; }
        g[0] = g2[0] * ex; g[1] = g2[0] * ey; g[2] = g2[1];
        return phi;
    }
    case ORC_BOX:
        return round_box(3, q, p, p[3], g);
    case ORC_PRISM: {
        double re = p[2];
        double r = p[0] / (2.0 * sqrt(3.0)) - re;
        double g2[2];
        double d2 = tri_sdf(q[1], q[2], r, g2);
        double w0 = d2, w1 = fabs(q[0]) - (0.5 * p[1] - re);
        double o0 = w0 > 0.0 ? w0 : 0.0, o1 = w1 > 0.0 ? w1 : 0.0;
        double L = sqrt(o0 * o0 + o1 * o1);
        double m = w0 > w1 ? w0 : w1;
        double phi = (m < 0.0 ? m : 0.0) + L - re;
        double gw0, gw1;
        if (m > 0.0) { gw0 = o0 / L; gw1 = o1 / L; }
        else if (w0 > w1) { gw0 = 1.0; gw1 = 0.0; }
        else { gw0 = 0.0; gw1 = 1.0; }
        g[0] = gw1 * sgn(q[0]); g[1] = gw0 * g2[0]; g[2] = gw0 * g2[1];
        return phi;
    }
    case ORC_PERLIN: {
        double gb[3];
        double phi = round_box(3, q, p, p[3], gb);
        double amp = p[4], period = p[5], pers = p[6];
        int oct = (int)p[7];
        double f = 0.0, fx = 0.0, fy = 0.0, a = 1.0, s = 1.0 / period;
        for (int o = 0; o < oct; ++o) {
            double nx, ny;
            double nv = noise2(ind->perm, q[0] * s, q[1] * s, &nx, &ny);
            f += a * nv; fx += a * s * nx; fy += a * s * ny;
            a *= pers; s *= 2.0;
        }
        g[0] = gb[0] - amp * fx; g[1] = gb[1] - amp * fy; g[2] = gb[2];
        double gl = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
        g[0] /= gl; g[1] /= gl; g[2] /= gl;
        return phi - amp * f;
    }
    default:
        g[0] = 0.0; g[1] = 0.0; g[2] = 1.0;
        return 1e300;
    }
}

/* World-frame SDF and unit outward normal at xw for the given pose. */
double orc_sdf(const orc_indenter *ind, const orc_pose *ps, const double xw[3], double n[3])
{
    double d0 = xw[0] - ps->c[0], d1 = xw[1] - ps->c[1], d2 = xw[2] - ps->c[2];
    double q[3] = {ps->cs * d0 + ps->sn * d1, -ps->sn * d0 + ps->cs * d1, d2};
    double g[3];
    double phi = orc_sdf_local(ind, q, g);
    n[0] = ps->cs * g[0] - ps->sn * g[1];
    n[1] = ps->sn * g[0] + ps->cs * g[1];
    n[2] = g[2];
    return phi;
}

/* Rigid object velocity at xw: v_lin + omega z x (xw - c). */
static void object_velocity(const orc_pose *ps, const double xw[3], double vo[3])
{
    vo[0] = ps->vlin[0] - ps->omega * (xw[1] - ps->c[1]);
    vo[1] = ps->vlin[1] + ps->omega * (xw[0] - ps->c[0]);
    vo[2] = ps->vlin[2];
}

/* ------------------------------------------------------------------ P2G */

static long node_index(const orc_scene *s, int ax, int ay, int az)
{
    return ((long)az * s->ny + ay) * s->nx + ax;
}

/* Particle-to-grid, Eq. 1 (mass) and Eqs. 2-4 (momentum MG = MM + ME), of
 * particles p0..p1-1 added to M and MG laid out over the node sub-box whose
 * first node is lo[3] (box indices) and whose extent is dim[3]. */
static int p2g_range(const orc_scene *s, int p0, int p1, const double *x, const double *v,
                     const double *C, const double *F, const int lo[3], const int dim[3],
                     double *M, double *MG)
{
    double dx = s->dx, V0 = dx * dx * dx / s->ppc, mp = s->rho * V0, mu, lam;
    orc_lame(s->E, s->nu, &mu, &lam);
    double kME = -4.0 * s->dt / (dx * dx);
    for (int p = p0; p < p1; ++p) {
        int base[3];
        double w[3][3], tau[9];
        for (int a = 0; a < 3; ++a) orc_weights(x[p * 3 + a], dx, &base[a], w[a]);
        if (orc_kirchhoff(F + p * 9, mu, lam, tau) != ORC_OK) return ORC_ERR_NUMERIC;
        const double *vp = v + p * 3, *Cp = C + p * 9;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                for (int k = 0; k < 3; ++k) {
                    int ax = base[0] + i + s->ox, ay = base[1] + j + s->oy, az = base[2] + k + s->oz;
                    if (ax < 0 || ay < 0 || az < 0 || ax >= s->nx || ay >= s->ny || az >= s->nz)
                        return ORC_ERR_DOMAIN;
                    int lx = ax - lo[0], ly = ay - lo[1], lz = az - lo[2];
                    if (lx < 0 || ly < 0 || lz < 0 || lx >= dim[0] || ly >= dim[1] || lz >= dim[2])
                        return ORC_ERR_ARG;
                    long ni = ((long)lz * dim[1] + ly) * dim[0] + lx;
                    double wip = w[0][i] * w[1][j] * w[2][k];
                    double d[3] = {(base[0] + i) * dx - x[p * 3 + 0],
                                   (base[1] + j) * dx - x[p * 3 + 1],
                                   (base[2] + k) * dx - x[p * 3 + 2]};
                    M[ni] += wip * mp;                                   /* Eq. 1 */
                    for (int r = 0; r < 3; ++r) {
                        double Cd = Cp[r * 3 + 0] * d[0] + Cp[r * 3 + 1] * d[1] + Cp[r * 3 + 2] * d[2];
                        double Sd = tau[r * 3 + 0] * d[0] + tau[r * 3 + 1] * d[1] + tau[r * 3 + 2] * d[2];
                        double MM = wip * (mp * vp[r] + mp * Cd);        /* Eq. 3 */
                        double ME = kME * wip * V0 * Sd;                 /* Eq. 4 */
                        MG[ni * 3 + r] += MM + ME;                       /* Eq. 2 */
                    }
                }
    }
    return ORC_OK;
}

/* Particle-to-grid of the object particles (Eqs. 1-3, no stress term), added
 * to M and MG over the whole node box: each at the pose's world position
 * c + R(yaw) q with the rigid velocity and affine field of the pose. */
int orc_object_p2g(const orc_scene *s, const orc_indenter *ind, const orc_pose *ps, double *M, double *MG)
{
    double dx = s->dx, m = ind->obj_m;
    double Cq[9] = {0.0, -ps->omega, 0.0, ps->omega, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (long q = 0; q < ind->n_obj; ++q) {
        const double *ql = ind->obj_q + q * 3;
        double xw[3] = {ps->c[0] + ps->cs * ql[0] - ps->sn * ql[1], ps->c[1] + ps->sn * ql[0] + ps->cs * ql[1],
                        ps->c[2] + ql[2]};
        double vo[3], w[3][3];
        int base[3];
        object_velocity(ps, xw, vo);
        for (int a = 0; a < 3; ++a) orc_weights(xw[a], dx, &base[a], w[a]);
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                for (int k = 0; k < 3; ++k) {
                    int ax = base[0] + i + s->ox, ay = base[1] + j + s->oy, az = base[2] + k + s->oz;
                    if (ax < 0 || ay < 0 || az < 0 || ax >= s->nx || ay >= s->ny || az >= s->nz)
                        continue;                              /* outside the node box: no grid there */
                    long ni = node_index(s, ax, ay, az);
                    double wip = w[0][i] * w[1][j] * w[2][k];
                    double d[3] = {(base[0] + i) * dx - xw[0], (base[1] + j) * dx - xw[1], (base[2] + k) * dx - xw[2]};
                    M[ni] += wip * m;                                      /* Eq. 1 */
                    for (int r = 0; r < 3; ++r) {
                        double Cd = Cq[r * 3 + 0] * d[0] + Cq[r * 3 + 1] * d[1] + Cq[r * 3 + 2] * d[2];
                        MG[ni * 3 + r] += wip * m * (vo[r] + Cd);              /* Eqs. 2-3 */
                    }
                }
    }
    return ORC_OK;
}

/* Particle-to-grid of all particles in index order (the grid is cleared first). */
int orc_p2g(const orc_scene *s, int n, const double *x, const double *v,
            const double *C, const double *F, double *M, double *MG)
{
    long nn = (long)s->nx * s->ny * s->nz;
    memset(M, 0, sizeof(double) * nn);
    memset(MG, 0, sizeof(double) * 3 * nn);
    const int lo[3] = {0, 0, 0}, dim[3] = {s->nx, s->ny, s->nz};
    return p2g_range(s, 0, n, x, v, C, F, lo, dim, M, MG);
}

/* ------------------------------------------------------------------ grid */

/* Grid velocity (Eq. 5) + gravity, indenter contact, walls, fixed base, on
 * the node planes z0 <= az < z1; returns the number of contact nodes. */
static long grid_update_planes(const orc_scene *s, const orc_indenter *ind, const orc_pose *ps,
                               const double *M, const double *MG, double *V, int z0, int z1)
{
    long cnt = 0;
    for (int az = z0; az < z1; ++az)
        for (int ay = 0; ay < s->ny; ++ay)
            for (int ax = 0; ax < s->nx; ++ax) {
                long ni = node_index(s, ax, ay, az);
                double Vn[3] = {0.0, 0.0, 0.0};
                if (M[ni] > 0.0) {
                    for (int r = 0; r < 3; ++r) Vn[r] = MG[ni * 3 + r] / M[ni] + s->dt * s->g[r];
                    if (ind->kind != ORC_NONE && ind->n_obj <= 0) {
                        double xw[3] = {(ax - s->ox) * s->dx, (ay - s->oy) * s->dx, (az - s->oz) * s->dx};
                        double nrm[3], vo[3];
                        double phi = orc_sdf(ind, ps, xw, nrm);
                        if (phi <= 0.0) {
                            object_velocity(ps, xw, vo);
                            double vr[3] = {Vn[0] - vo[0], Vn[1] - vo[1], Vn[2] - vo[2]};
                            double vn = vr[0] * nrm[0] + vr[1] * nrm[1] + vr[2] * nrm[2];
                            if (vn < 0.0) {
                                double vt[3] = {vr[0] - vn * nrm[0], vr[1] - vn * nrm[1], vr[2] - vn * nrm[2]};
                                double vtl = sqrt(vt[0] * vt[0] + vt[1] * vt[1] + vt[2] * vt[2]);
                                double lim = ind->mu * (-vn);
                                double muk = ind->mu_k > 0.0 ? ind->mu_k : ind->mu;
                                if (vtl <= lim) {
                                    vr[0] = vr[1] = vr[2] = 0.0;        /* relative rest */
                                } else {
                                    double sc = 1.0 - muk * (-vn) / vtl;   /* Coulomb slip */
                                    vr[0] = vt[0] * sc; vr[1] = vt[1] * sc; vr[2] = vt[2] * sc;
                                }
                                for (int r = 0; r < 3; ++r) Vn[r] = vr[r] + vo[r];
                                ++cnt;
                            }
                        }
                    }
                }
                if (s->walls && (ax < 2 || ay < 2 || ax >= s->nx - 2 || ay >= s->ny - 2 || az >= s->nz - 2))
                    Vn[0] = Vn[1] = Vn[2] = 0.0;
                if (az - s->oz <= 0) {
                    if (s->base_mode == ORC_BASE_FIXED) Vn[0] = Vn[1] = Vn[2] = 0.0;
                    else if (s->base_mode == ORC_BASE_SLIP) Vn[2] = 0.0;
                }
                V[ni * 3 + 0] = Vn[0]; V[ni * 3 + 1] = Vn[1]; V[ni * 3 + 2] = Vn[2];
            }
    return cnt;
}

int orc_grid_update(const orc_scene *s, const orc_indenter *ind, const orc_pose *ps,
                    const double *M, const double *MG, double *V, long *n_contact)
{
    long cnt = grid_update_planes(s, ind, ps, M, MG, V, 0, s->nz);
    if (n_contact) *n_contact = cnt;
    return ORC_OK;
}

/* ------------------------------------------------------------------ G2P */

/* Grid-to-particle velocity (Eq. 6) and affine field (Eq. 7) at one point. */
static int g2p_point(const orc_scene *s, const double *V, const double xp[3], double v[3], double C[9])
{
    int base[3];
    double w[3][3], dx = s->dx, D = 4.0 / (dx * dx);
    for (int a = 0; a < 3; ++a) orc_weights(xp[a], dx, &base[a], w[a]);
    for (int r = 0; r < 3; ++r) v[r] = 0.0;
    for (int r = 0; r < 9; ++r) C[r] = 0.0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            for (int k = 0; k < 3; ++k) {
                int ax = base[0] + i + s->ox, ay = base[1] + j + s->oy, az = base[2] + k + s->oz;
                if (ax < 0 || ay < 0 || az < 0 || ax >= s->nx || ay >= s->ny || az >= s->nz)
                    return ORC_ERR_DOMAIN;
                long ni = node_index(s, ax, ay, az);
                double wgp = w[0][i] * w[1][j] * w[2][k];
                double d[3] = {(base[0] + i) * dx - xp[0], (base[1] + j) * dx - xp[1], (base[2] + k) * dx - xp[2]};
                for (int r = 0; r < 3; ++r) {
                    double Vr = V[ni * 3 + r];
                    v[r] += wgp * Vr;                                    /* Eq. 6 */
                    for (int c = 0; c < 3; ++c) C[r * 3 + c] += D * wgp * Vr * d[c];   /* Eq. 7 */
                }
            }
    return ORC_OK;
}

int orc_g2p(const orc_scene *s, int n, const double *x, const uint32_t *tag, const double *V,
            double *v, double *C)
{
    for (int p = 0; p < n; ++p) {
        int rc = g2p_point(s, V, x + p * 3, v + p * 3, C + p * 9);
        if (rc != ORC_OK) return rc;
        /* Algorithm 1: bottom elastomer particles get zero z velocity */
        if ((tag[p] & ORC_TAG_BOTTOM) && s->base_mode != ORC_BASE_FREE) v[p * 3 + 2] = 0.0;
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------ Algorithm 1 */

/* x_e: the elastomer particle closest to x_o (ties: lowest index). */
int orc_nearest(int n, const double *x, const double xo[3])
{
    int best = 0;
    double bd = 1e300;
    for (int p = 0; p < n; ++p) {
        double a = x[p * 3] - xo[0], b = x[p * 3 + 1] - xo[1], c = x[p * 3 + 2] - xo[2];
        double d = a * a + b * b + c * c;
        if (d < bd) { bd = d; best = p; }
    }
    return best;
}

/* Relative-rest check at the calibration particle (reading of Algorithm 1). */
int orc_relrest_accept(const orc_scene *s, const orc_indenter *ind, const orc_pose *ps,
                       const double xe[3], const double ve[3])
{
    if (ind->kind == ORC_NONE) return 1;
    double nrm[3], vo[3];
    if (orc_sdf(ind, ps, xe, nrm) > s->dx) return 1;
    object_velocity(ps, xe, vo);
    double vot = sqrt(vo[0] * vo[0] + vo[1] * vo[1]);
    if (vot < 1e-6) return 1;
    double a = ve[0] - vo[0], b = ve[1] - vo[1];
    return sqrt(a * a + b * b) <= s->threshold * vot;
}

typedef struct {
    double *M, *MG, *V;
} orc_work;

/* One IMPM time step (Algorithm 1): passes of P2G, boundary handling and G2P
 * until the relative-rest check accepts or LIMIT passes ran, then F and x
 * move once (Eqs. 8-9). */
int orc_substep(const orc_scene *s, const orc_indenter *ind, const double *kf, int nkf, int k,
                int n, double *x, double *v, double *C, double *F, const uint32_t *tag,
                double *M, double *MG, double *V, int *passes, int *e_out, long *n_contact)
{
    orc_pose ps;
    orc_pose_eval(kf, nkf, k, s->dt, ind->tip_offset, &ps);
    int e = orc_nearest(n, x, ps.tip);
    int j = 0, rc;
    for (;;) {
        rc = orc_p2g(s, n, x, v, C, F, M, MG);
        if (rc) return rc;
        if (ind->n_obj > 0) orc_object_p2g(s, ind, &ps, M, MG);
        rc = orc_grid_update(s, ind, &ps, M, MG, V, n_contact);
        if (rc) return rc;
        rc = orc_g2p(s, n, x, tag, V, v, C);
        if (rc) return rc;
        int ok = orc_relrest_accept(s, ind, &ps, x + e * 3, v + e * 3);
        ++j;
        if (ok || j >= s->limit) break;
    }
    for (int p = 0; p < n; ++p) {
        double *Fp = F + p * 9, Fn[9];
        const double *Cp = C + p * 9;
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) {
                double a = Fp[r * 3 + c];
                for (int q = 0; q < 3; ++q) a += s->dt * Cp[r * 3 + q] * Fp[q * 3 + c];
                Fn[r * 3 + c] = a;                                       /* Eq. 8 */
            }
        memcpy(Fp, Fn, sizeof Fn);
        for (int d = 0; d < 3; ++d) x[p * 3 + d] += s->dt * v[p * 3 + d];   /* Eq. 9 */
        double J = det3(Fp);
        if (!(J > 0.0) || !isfinite(J) || !isfinite(x[p * 3]) || !isfinite(x[p * 3 + 1]) || !isfinite(x[p * 3 + 2]))
            return ORC_ERR_NUMERIC;
    }
    if (passes) *passes = j;
    if (e_out) *e_out = e;
    return ORC_OK;
}

/* Run substeps k0 .. k0+nsub-1; logs passes and x_e per substep (may be NULL). */
int orc_run(const orc_scene *s, const orc_indenter *ind, const double *kf, int nkf, int k0, int nsub,
            int n, double *x, double *v, double *C, double *F, const uint32_t *tag,
            int *pass_log, int *e_log)
{
    long nn = (long)s->nx * s->ny * s->nz;
    double *M = (double *)malloc(sizeof(double) * nn);
    double *MG = (double *)malloc(sizeof(double) * 3 * nn);
    double *V = (double *)malloc(sizeof(double) * 3 * nn);
    if (!M || !MG || !V) { free(M); free(MG); free(V); return ORC_ERR_ARG; }
    int rc = ORC_OK;
    for (int t = 0; t < nsub; ++t) {
        int ps = 0, e = 0;
        rc = orc_substep(s, ind, kf, nkf, k0 + t, n, x, v, C, F, tag, M, MG, V, &ps, &e, NULL);
        if (rc) break;
        if (pass_log) pass_log[t] = ps;
        if (e_log) e_log[t] = e;
    }
    free(M); free(MG); free(V);
    return rc;
}

/* ------------------------------------------------------------------ all-cores variant */

/* Threads that orc_run_par uses by default (1 without OpenMP). */
int orc_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

typedef struct {
    int p0, p1;              /* particle chunk */
    int lo[3], dim[3];       /* node sub-box covered by the chunk's stencils */
    double *M, *MG;          /* private grid over that box */
    size_t cap;              /* nodes allocated */
    int rc;
} orc_chunk;

/* P2G of one chunk into its private grid: the sub-box is the bounding box of
 * the chunk's 3x3x3 stencils. */
static void chunk_p2g(const orc_scene *s, orc_chunk *c, const double *x, const double *v,
                      const double *C, const double *F)
{
    int mn[3] = {s->nx, s->ny, s->nz}, mx[3] = {-1, -1, -1};
    const int off[3] = {s->ox, s->oy, s->oz};
    for (int p = c->p0; p < c->p1; ++p)
        for (int a = 0; a < 3; ++a) {
            int b;
            double w[3];
            orc_weights(x[p * 3 + a], s->dx, &b, w);
            b += off[a];
            if (b < mn[a]) mn[a] = b;
            if (b + 2 > mx[a]) mx[a] = b + 2;
        }
    if (c->p1 <= c->p0) { c->rc = ORC_OK; c->dim[0] = c->dim[1] = c->dim[2] = 0; return; }
    size_t nodes = 1;
    for (int a = 0; a < 3; ++a) {
        c->lo[a] = mn[a];
        c->dim[a] = mx[a] - mn[a] + 1;
        nodes *= (size_t)c->dim[a];
    }
    if (nodes > c->cap) {
        free(c->M); free(c->MG);
        c->M = (double *)malloc(sizeof(double) * nodes);
        c->MG = (double *)malloc(sizeof(double) * 3 * nodes);
        c->cap = (c->M && c->MG) ? nodes : 0;
        if (!c->cap) { c->rc = ORC_ERR_ARG; return; }
    }
    memset(c->M, 0, sizeof(double) * nodes);
    memset(c->MG, 0, sizeof(double) * 3 * nodes);
    c->rc = p2g_range(s, c->p0, c->p1, x, v, C, F, c->lo, c->dim, c->M, c->MG);
}

/* The grid sums of Eqs. 1-2 from the chunks' private grids, added in chunk
 * order, on the node planes z0 <= az < z1. */
static void reduce_planes(const orc_scene *s, const orc_chunk *ch, int T, double *M, double *MG, int z0, int z1)
{
    for (int az = z0; az < z1; ++az)
        for (int ay = 0; ay < s->ny; ++ay)
            for (int ax = 0; ax < s->nx; ++ax) {
                double m = 0.0, g0 = 0.0, g1 = 0.0, g2 = 0.0;
                for (int t = 0; t < T; ++t) {
                    const orc_chunk *c = ch + t;
                    int lx = ax - c->lo[0], ly = ay - c->lo[1], lz = az - c->lo[2];
                    if (lx < 0 || ly < 0 || lz < 0 || lx >= c->dim[0] || ly >= c->dim[1] || lz >= c->dim[2])
                        continue;
                    long li = ((long)lz * c->dim[1] + ly) * c->dim[0] + lx;
                    m += c->M[li];
                    g0 += c->MG[li * 3]; g1 += c->MG[li * 3 + 1]; g2 += c->MG[li * 3 + 2];
                }
                long ni = node_index(s, ax, ay, az);
                M[ni] = m;
                MG[ni * 3] = g0; MG[ni * 3 + 1] = g1; MG[ni * 3 + 2] = g2;
            }
}

/* orc_run with its loops shared among nthreads threads (<= 0: orc_threads()):
 * particles in nthreads contiguous index chunks, each P2G'd into a private
 * grid that is summed in chunk order; node and particle loops split by range;
 * the nearest particle is the chunk minima compared in chunk order (ties go
 * to the lowest index, as in orc_nearest).  Same arithmetic per particle and
 * node as orc_run; only the order of the grid sums differs, so results agree
 * with orc_run to rounding.  Used for the all-cores CPU baseline and for
 * oracle runs too large for one core. */
int orc_run_par(const orc_scene *s, const orc_indenter *ind, const double *kf, int nkf, int k0, int nsub,
                int n, double *x, double *v, double *C, double *F, const uint32_t *tag,
                int *pass_log, int *e_log, int nthreads)
{
    int T = nthreads > 0 ? nthreads : orc_threads();
    if (T > n) T = n > 0 ? n : 1;
    long nn = (long)s->nx * s->ny * s->nz;
    double *M = (double *)malloc(sizeof(double) * nn);
    double *MG = (double *)malloc(sizeof(double) * 3 * nn);
    double *V = (double *)malloc(sizeof(double) * 3 * nn);
    orc_chunk *ch = (orc_chunk *)calloc((size_t)T, sizeof(orc_chunk));
    int *best = (int *)malloc(sizeof(int) * T), *rcs = (int *)malloc(sizeof(int) * T);
    double *bestd = (double *)malloc(sizeof(double) * T);
    int rc = ORC_OK;
    if (!M || !MG || !V || !ch || !best || !rcs || !bestd) rc = ORC_ERR_ARG;
    for (int t = 0; rc == ORC_OK && t < T; ++t) {
        ch[t].p0 = (int)((long)n * t / T);
        ch[t].p1 = (int)((long)n * (t + 1) / T);
    }
    for (int st = 0; rc == ORC_OK && st < nsub; ++st) {
        orc_pose ps;
        orc_pose_eval(kf, nkf, k0 + st, s->dt, ind->tip_offset, &ps);
        /* x_e: nearest particle to the tip */
#pragma omp parallel for schedule(static, 1) num_threads(T)
        for (int t = 0; t < T; ++t) {
            int b = ch[t].p0;
            double bd = 1e300;
            for (int p = ch[t].p0; p < ch[t].p1; ++p) {
                double a = x[p * 3] - ps.tip[0], bb = x[p * 3 + 1] - ps.tip[1], c = x[p * 3 + 2] - ps.tip[2];
                double d = a * a + bb * bb + c * c;
                if (d < bd) { bd = d; b = p; }
            }
            best[t] = b;
            bestd[t] = bd;
        }
        int e = best[0];
        double ed = bestd[0];
        for (int t = 1; t < T; ++t)
            if (bestd[t] < ed) { ed = bestd[t]; e = best[t]; }
        int j = 0;
        for (;;) {
#pragma omp parallel for schedule(static, 1) num_threads(T)
            for (int t = 0; t < T; ++t) chunk_p2g(s, ch + t, x, v, C, F);
            for (int t = 0; t < T; ++t)
                if (ch[t].rc != ORC_OK && rc == ORC_OK) rc = ch[t].rc;
            if (rc) break;
            if (ind->n_obj > 0) {
                /* the object particles are added after the elastomer's sums */
#pragma omp parallel for schedule(static, 1) num_threads(T)
                for (int t = 0; t < T; ++t) {
                    int z0 = (int)((long)s->nz * t / T), z1 = (int)((long)s->nz * (t + 1) / T);
                    reduce_planes(s, ch, T, M, MG, z0, z1);
                }
                orc_object_p2g(s, ind, &ps, M, MG);
#pragma omp parallel for schedule(static, 1) num_threads(T)
                for (int t = 0; t < T; ++t) {
                    int z0 = (int)((long)s->nz * t / T), z1 = (int)((long)s->nz * (t + 1) / T);
                    grid_update_planes(s, ind, &ps, M, MG, V, z0, z1);
                }
            } else {
#pragma omp parallel for schedule(static, 1) num_threads(T)
                for (int t = 0; t < T; ++t) {
                    int z0 = (int)((long)s->nz * t / T), z1 = (int)((long)s->nz * (t + 1) / T);
                    reduce_planes(s, ch, T, M, MG, z0, z1);
                    grid_update_planes(s, ind, &ps, M, MG, V, z0, z1);
                }
            }
#pragma omp parallel for schedule(static, 1) num_threads(T)
            for (int t = 0; t < T; ++t)
                rcs[t] = orc_g2p(s, ch[t].p1 - ch[t].p0, x + (long)ch[t].p0 * 3, tag + ch[t].p0, V,
                                 v + (long)ch[t].p0 * 3, C + (long)ch[t].p0 * 9);
            for (int t = 0; t < T; ++t)
                if (rcs[t] != ORC_OK && rc == ORC_OK) rc = rcs[t];
            if (rc) break;
            int ok = orc_relrest_accept(s, ind, &ps, x + e * 3, v + e * 3);
            ++j;
            if (ok || j >= s->limit) break;
        }
        if (rc) break;
#pragma omp parallel for schedule(static, 1) num_threads(T)
        for (int t = 0; t < T; ++t) {
            rcs[t] = ORC_OK;
            for (int p = ch[t].p0; p < ch[t].p1; ++p) {
                double *Fp = F + (long)p * 9, Fn[9];
                const double *Cp = C + (long)p * 9;
                for (int r = 0; r < 3; ++r)
                    for (int c = 0; c < 3; ++c) {
                        double a = Fp[r * 3 + c];
                        for (int q = 0; q < 3; ++q) a += s->dt * Cp[r * 3 + q] * Fp[q * 3 + c];
                        Fn[r * 3 + c] = a;                               /* Eq. 8 */
                    }
                memcpy(Fp, Fn, sizeof Fn);
                for (int d = 0; d < 3; ++d) x[(long)p * 3 + d] += s->dt * v[(long)p * 3 + d];   /* Eq. 9 */
                double J = det3(Fp);
                if (!(J > 0.0) || !isfinite(J) || !isfinite(x[(long)p * 3]) || !isfinite(x[(long)p * 3 + 1]) ||
                    !isfinite(x[(long)p * 3 + 2]))
                    rcs[t] = ORC_ERR_NUMERIC;
            }
        }
        for (int t = 0; t < T; ++t)
            if (rcs[t] != ORC_OK && rc == ORC_OK) rc = rcs[t];
        if (rc) break;
        if (pass_log) pass_log[st] = j;
        if (e_log) e_log[st] = e;
    }
    if (ch)
        for (int t = 0; t < T; ++t) { free(ch[t].M); free(ch[t].MG); }
    free(ch); free(best); free(bestd); free(rcs);
    free(M); free(MG); free(V);
    return rc;
}

/* ------------------------------------------------------------------ surface */

static double bspline2(double t)
{
    t = fabs(t);
    if (t < 0.5) return 0.75 - t * t;
    if (t < 1.5) return 0.5 * (1.5 - t) * (1.5 - t);
    return 0.0;
}

/* Height field of the top-layer particles on a W x H pixel grid at the given
 * pitch (pixel centres at (u+0.5)*pitch), 2-D quadratic B-spline splat;
 * empty pixels read h_empty; normals from central differences of h. */
void orc_surface(int n, const double *x, const uint32_t *tag, int W, int H, double pitch,
                 double h_empty, double *height, double *normal)
{
    double *num = (double *)calloc((size_t)W * H, sizeof(double));
    double *den = (double *)calloc((size_t)W * H, sizeof(double));
    for (int p = 0; p < n; ++p) {
        if (!(tag[p] & ORC_TAG_TOP)) continue;
        double px = x[p * 3] / pitch - 0.5, py = x[p * 3 + 1] / pitch - 0.5;
        int u0 = (int)floor(px) - 1, v0 = (int)floor(py) - 1;
        for (int b = v0; b <= v0 + 3; ++b)
            for (int a = u0; a <= u0 + 3; ++a) {
                if (a < 0 || b < 0 || a >= W || b >= H) continue;
                double w = bspline2(px - a) * bspline2(py - b);
                if (w == 0.0) continue;
                num[(long)b * W + a] += w * x[p * 3 + 2];
                den[(long)b * W + a] += w;
            }
    }
    for (long i = 0; i < (long)W * H; ++i) height[i] = den[i] > 0.0 ? num[i] / den[i] : h_empty;
    for (int b = 0; b < H; ++b)
        for (int a = 0; a < W; ++a) {
            int al = a > 0 ? a - 1 : a, ar = a < W - 1 ? a + 1 : a;
            int bl = b > 0 ? b - 1 : b, br = b < H - 1 ? b + 1 : b;
            double hx = (height[(long)b * W + ar] - height[(long)b * W + al]) / ((ar - al) * pitch);
            double hy = (height[(long)br * W + a] - height[(long)bl * W + a]) / ((br - bl) * pitch);
            double L = sqrt(hx * hx + hy * hy + 1.0);
            long i = (long)b * W + a;
            normal[i * 3 + 0] = -hx / L; normal[i * 3 + 1] = -hy / L; normal[i * 3 + 2] = 1.0 / L;
        }
    free(num); free(den);
}

/* ------------------------------------------------------------------ surrogate inputs/targets */

/* Displacement x - X of the top-layer particles, splatted with the 2-D
 * quadratic B-spline at the reference positions X; empty pixels read 0. */
void orc_surface_disp(int n, const double *x, const double *xref, const uint32_t *tag, int W, int H,
                      double pitch, double *u)
{
    double *acc = (double *)calloc((size_t)W * H * 4, sizeof(double));
    for (int p = 0; p < n; ++p) {
        if (!(tag[p] & ORC_TAG_TOP)) continue;
        double px = xref[p * 3] / pitch - 0.5, py = xref[p * 3 + 1] / pitch - 0.5;
        int u0 = (int)floor(px) - 1, v0 = (int)floor(py) - 1;
        for (int b = v0; b <= v0 + 3; ++b)
            for (int a = u0; a <= u0 + 3; ++a) {
                if (a < 0 || b < 0 || a >= W || b >= H) continue;
                double w = bspline2(px - a) * bspline2(py - b);
                if (w == 0.0) continue;
                double *c = acc + ((long)b * W + a) * 4;
                for (int d = 0; d < 3; ++d) c[d] += w * (x[p * 3 + d] - xref[p * 3 + d]);
                c[3] += w;
            }
    }
    for (long i = 0; i < (long)W * H; ++i)
        for (int d = 0; d < 3; ++d) u[i * 3 + d] = acc[i * 4 + 3] > 0.0 ? acc[i * 4 + d] / acc[i * 4 + 3] : 0.0;
    free(acc);
}

/* Height of the indenter's underside above the gel top H per pixel column:
 * scan up from H - clip in steps of `step` and bisect the first entry into
 * the shape (phi <= 0) to 1e-13 m; a column that starts inside reads -clip,
 * one that never enters the shape below H + clip reads +clip. */
void orc_indenter_height(const orc_indenter *ind, const orc_pose *ps, double Hgel, int W, int H, double pitch,
                         double clip, double step, double *h)
{
    for (int v = 0; v < H; ++v)
        for (int a = 0; a < W; ++a) {
            double xw[3] = {(a + 0.5) * pitch, (v + 0.5) * pitch, Hgel - clip}, nrm[3];
            double out = clip;
            double lo = xw[2];
            if (orc_sdf(ind, ps, xw, nrm) <= 0.0) {
                out = -clip;
            } else {
                for (double z = lo + step; z <= Hgel + clip + step; z += step) {
                    xw[2] = z;
                    if (orc_sdf(ind, ps, xw, nrm) <= 0.0) {
                        double hi = z;                 /* phi(lo) > 0 >= phi(hi) */
                        while (hi - lo > 1e-13) {
                            double mid = 0.5 * (lo + hi);
                            xw[2] = mid;
                            if (orc_sdf(ind, ps, xw, nrm) <= 0.0) hi = mid; else lo = mid;
                        }
                        out = 0.5 * (lo + hi) - Hgel;
                        break;
                    }
                    lo = z;
                }
            }
            if (out > clip) out = clip;
            if (out < -clip) out = -clip;
            h[(long)v * W + a] = out;
        }
}
