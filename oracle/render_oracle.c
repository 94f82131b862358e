/*
 * render_oracle.c -- plain FP64 CPU oracle of the sensor image: a path
 * tracer over the elastomer surface's height field, and the image metrics.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * CPU-baseline leg of bench.py load this library.  It shares no code with
 * the CUDA path.
 *
 * Follows Sec. III-B of the paper (reverse rays from the camera, diffuse
 * reflections at the rough membrane, attenuation per reflection, the sum of
 * what reaches the lights) and Sec. IV-B (maximum roughness, four LEDs,
 * 128 samples per pixel); the image metrics follow Sec. IV (MSE, PSNR,
 * SSIM).  Readings where the paper is silent:
 *   surface     z = h(x, y), bilinear over the readout grid (pixel (i, j) at
 *               ((j + 0.5) p, (i + 0.5) p)), clamped at the edges; normal
 *               from central differences of h over +-p/2; the gel is below
 *   membrane    Lambertian with a per-pixel albedo (the base texture);
 *               seen from the gel side (inner normal -n)
 *   camera      orthographic from below, one jittered primary hit per sample
 *   LEDs        one-sided rectangles c +- u +- v emitting radiance L on the
 *               side of u x v; a path that reaches one adds its throughput
 *               times L and ends
 *   bounces     cosine-weighted directions about the inner normal (in the
 *               continuous orthonormal basis of Duff et al., JCGT 2017); the ray
 *               ends at the floor plane z = z_floor (the camera window,
 *               absorbing) or when max_bounces reflections are used; it
 *               meets the surface again where z - h(x, y) first turns >= 0,
 *               found by steps of p/2 within the height range of h and 12
 *               bisections
 *   random      SplitMix64 (Steele, Lea and Flood, OOPSLA 2014) of the
 *               counter ((pixel * spp + s) * 32 + bounce) * 4 + dim, 24-bit
 *               uniforms (exact in single and double precision)
 *   SSIM        Wang et al. (2004): 11 x 11 Gaussian window, sigma 1.5,
 *               K1 = 0.01, K2 = 0.03, over windows inside the image, mean
 *               over the map and channels
 *
 * Pins (tests/test_render_pins.py): the one-bounce render of a flat
 * surface under one LED against the irradiance of Lambert's polygon
 * formula; zero albedo and dark LEDs give black; mirror symmetry; MSE,
 * PSNR and SSIM closed forms and a brute-force SSIM.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

#define RO_OK 0
#define RO_ERR_ARG 1
#define RO_MAX_LIGHTS 4
#define RO_PI 3.14159265358979323846

typedef struct {
    double c[RO_MAX_LIGHTS][3];     /* LED rectangle centres */
    double u[RO_MAX_LIGHTS][3];     /* half-edge vectors: the LED is c + a u + b v, |a|, |b| <= 1 */
    double v[RO_MAX_LIGHTS][3];
    double L[RO_MAX_LIGHTS][3];     /* RGB radiance, emitted on the side of u x v */
    int n_lights;
    int spp, max_bounces;
    int pad_;
    double z_floor;                 /* absorbing plane below the surface */
    uint64_t seed;
} ro_desc;

/* ------------------------------------------------------------------ random */

static uint64_t splitmix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

double ro_uniform(uint64_t seed, uint64_t counter)
{
    uint64_t z = splitmix64(seed + (counter + 1) * 0x9E3779B97F4A7C15ull);
    return (double)(z >> 40) * (1.0 / 16777216.0);
}

/* ------------------------------------------------------------------ surface */

typedef struct {
    const double *h, *albedo;
    int W, H;
    double p, hmin, hmax;
} ro_surf;

static double clampd(double a, double lo, double hi) { return a < lo ? lo : (a > hi ? hi : a); }

double ro_height(const ro_surf *s, double x, double y)
{
    double u = clampd(x / s->p - 0.5, 0.0, s->W - 1), v = clampd(y / s->p - 0.5, 0.0, s->H - 1);
    int j0 = (int)floor(u), i0 = (int)floor(v);
    if (j0 > s->W - 2) j0 = s->W - 2;
    if (i0 > s->H - 2) i0 = s->H - 2;
    double fu = u - j0, fv = v - i0;
    const double *r0 = s->h + (long)i0 * s->W, *r1 = r0 + s->W;
    return (1.0 - fv) * ((1.0 - fu) * r0[j0] + fu * r0[j0 + 1]) + fv * ((1.0 - fu) * r1[j0] + fu * r1[j0 + 1]);
}

static void surf_normal(const ro_surf *s, double x, double y, double n[3])
{
    double hp = 0.5 * s->p;
    double gx = (ro_height(s, x + hp, y) - ro_height(s, x - hp, y)) / s->p;
    double gy = (ro_height(s, x, y + hp) - ro_height(s, x, y - hp)) / s->p;
    double l = sqrt(gx * gx + gy * gy + 1.0);
    n[0] = -gx / l; n[1] = -gy / l; n[2] = 1.0 / l;
}

static const double *surf_albedo(const ro_surf *s, double x, double y)
{
    int j = (int)floor(x / s->p), i = (int)floor(y / s->p);
    if (j < 0) j = 0;
    if (j > s->W - 1) j = s->W - 1;
    if (i < 0) i = 0;
    if (i > s->H - 1) i = s->H - 1;
    return s->albedo + ((long)i * s->W + j) * 3;
}

/* ------------------------------------------------------------------ one path */

/* Cosine-weighted direction about the unit normal m (pdf cos / pi), in the
 * orthonormal basis (t, b, m) of Duff et al., "Building an Orthonormal
 * Basis, Revisited" (JCGT 2017), which is continuous in m away from
 * m_z = 0 (a nearly flat membrane gets nearly the same basis in any
 * precision). */
static void cosine_dir(const double m[3], double u0, double u1, double w[3])
{
    double sg = m[2] >= 0.0 ? 1.0 : -1.0;
    double a = -1.0 / (sg + m[2]), bb = m[0] * m[1] * a;
    double t[3] = {1.0 + sg * m[0] * m[0] * a, sg * bb, -sg * m[0]};
    double b[3] = {bb, sg + m[1] * m[1] * a, -m[1]};
    double r = sqrt(u0), ph = 2.0 * RO_PI * u1, c = r * cos(ph), sn = r * sin(ph), z = sqrt(1.0 - u0);
    for (int k = 0; k < 3; ++k) w[k] = c * t[k] + sn * b[k] + z * m[k];
}

/* Nearest LED hit along P + t w (emitting side only): its index, or -1. */
static int hit_light(const ro_desc *d, const double P[3], const double w[3], double *tbest)
{
    int best = -1;
    for (int k = 0; k < d->n_lights; ++k) {
        const double *c = d->c[k], *u = d->u[k], *v = d->v[k];
        double e[3] = {u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2], u[0] * v[1] - u[1] * v[0]};
        double we = w[0] * e[0] + w[1] * e[1] + w[2] * e[2];
        if (!(we < 0.0)) continue;                                   /* back side or parallel */
        double t = ((c[0] - P[0]) * e[0] + (c[1] - P[1]) * e[1] + (c[2] - P[2]) * e[2]) / we;
        if (!(t > 0.0) || !(t < *tbest)) continue;
        double q[3] = {P[0] + t * w[0] - c[0], P[1] + t * w[1] - c[1], P[2] + t * w[2] - c[2]};
        double a = (q[0] * u[0] + q[1] * u[1] + q[2] * u[2]) / (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
        double bb = (q[0] * v[0] + q[1] * v[1] + q[2] * v[2]) / (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        if (fabs(a) <= 1.0 && fabs(bb) <= 1.0) { *tbest = t; best = k; }
    }
    return best;
}

/* First return of P + t w to the surface for 0 < t < tmax (z - h >= 0), or
 * a negative value: steps of p/2 while the ray is within the height range
 * of h, then 12 bisections. */
static double hit_surface(const ro_surf *s, const double P[3], const double w[3], double tmax)
{
    double tend = tmax;
    if (w[2] < 0.0) tend = fmin(tend, (s->hmin - P[2]) / w[2]);
    else if (w[2] > 0.0) tend = fmin(tend, (s->hmax - P[2]) / w[2]);
    double dt = 0.5 * s->p, t0 = 0.0;
    for (int it = 0; it < 4096; ++it) {
        double t1 = t0 + dt;
        if (t1 > tend) return -1.0;
        double f = P[2] + t1 * w[2] - ro_height(s, P[0] + t1 * w[0], P[1] + t1 * w[1]);
        if (f >= 0.0) {
            double lo = t0, hi = t1;
            for (int k = 0; k < 12; ++k) {
                double tm = 0.5 * (lo + hi);
                double fm = P[2] + tm * w[2] - ro_height(s, P[0] + tm * w[0], P[1] + tm * w[1]);
                if (fm >= 0.0) hi = tm; else lo = tm;
            }
            return hi;
        }
        t0 = t1;
    }
    return -1.0;
}

/* Radiance (RGB) of sample s of pixel (i, j). */
static void trace(const ro_surf *sf, const ro_desc *d, int i, int j, int s, double out[3])
{
    uint64_t base = ((uint64_t)((long)i * sf->W + j) * (uint64_t)d->spp + (uint64_t)s) * 32u;
    double x = (j + ro_uniform(d->seed, base * 4 + 0)) * sf->p;
    double y = (i + ro_uniform(d->seed, base * 4 + 1)) * sf->p;
    double P[3] = {x, y, ro_height(sf, x, y)}, n[3], T[3];
    surf_normal(sf, x, y, n);
    const double *a = surf_albedo(sf, x, y);
    for (int k = 0; k < 3; ++k) { T[k] = a[k]; out[k] = 0.0; }
    for (int b = 0; b < d->max_bounces && b < 32; ++b) {
        uint64_t key = (base + (uint64_t)b) * 4;
        double m[3] = {-n[0], -n[1], -n[2]}, w[3];
        cosine_dir(m, ro_uniform(d->seed, key + 2), ro_uniform(d->seed, key + 3), w);
        double tb = 1e300;
        int lk = hit_light(d, P, w, &tb);
        if (w[2] < 0.0) {
            double tf = (d->z_floor - P[2]) / w[2];
            if (tf < tb) { tb = tf; lk = -1; }                    /* the floor is nearer: absorbed */
        }
        double ts = hit_surface(sf, P, w, tb);
        if (ts > 0.0) {                                            /* reflected again by the membrane */
            P[0] += ts * w[0]; P[1] += ts * w[1];
            P[2] = ro_height(sf, P[0], P[1]);
            surf_normal(sf, P[0], P[1], n);
            a = surf_albedo(sf, P[0], P[1]);
            for (int k = 0; k < 3; ++k) T[k] *= a[k];
            continue;
        }
        if (lk >= 0)
            for (int k = 0; k < 3; ++k) out[k] += T[k] * d->L[lk][k];
        break;
    }
}

/* The image: rgb[(i * W + j) * 3 + c], the mean of spp samples per pixel.
 * h: H x W heights; albedo: H x W x 3. */
int ro_render(const double *h, const double *albedo, int W, int H, double pitch, const ro_desc *d, double *rgb)
{
    if (W < 2 || H < 2 || !(pitch > 0.0) || d->spp < 1 || d->max_bounces < 1 || d->n_lights < 0 ||
        d->n_lights > RO_MAX_LIGHTS)
        return RO_ERR_ARG;
    ro_surf sf = {h, albedo, W, H, pitch, h[0], h[0]};
    for (long q = 0; q < (long)W * H; ++q) {
        if (h[q] < sf.hmin) sf.hmin = h[q];
        if (h[q] > sf.hmax) sf.hmax = h[q];
    }
    for (int i = 0; i < H; ++i)
        for (int j = 0; j < W; ++j) {
            double acc[3] = {0.0, 0.0, 0.0}, o[3];
            for (int s = 0; s < d->spp; ++s) {
                trace(&sf, d, i, j, s, o);
                for (int k = 0; k < 3; ++k) acc[k] += o[k];
            }
            for (int k = 0; k < 3; ++k) rgb[((long)i * W + j) * 3 + k] = acc[k] / d->spp;
        }
    return RO_OK;
}

/* ------------------------------------------------------------------ metrics */

/* Mean squared error over all H x W x C values, and PSNR = 10 log10(MAX^2 /
 * MSE) (infinite for equal images). */
void ro_mse_psnr(const double *a, const double *b, long n, double max_value, double *mse, double *psnr)
{
    double s = 0.0;
    for (long q = 0; q < n; ++q) s += (a[q] - b[q]) * (a[q] - b[q]);
    *mse = s / (double)n;
    *psnr = *mse > 0.0 ? 10.0 * log10(max_value * max_value / *mse) : INFINITY;
}

/* Mean SSIM (Wang et al. 2004) of H x W x C images: per channel and per
 * window position (window inside the image), the Gaussian-weighted means,
 * variances and covariance of an 11 x 11 window (sigma 1.5, weights summing
 * to 1) in the SSIM formula with c1 = (0.01 MAX)^2, c2 = (0.03 MAX)^2. */
int ro_ssim(const double *a, const double *b, int W, int H, int C, double max_value, double *ssim)
{
    if (W < 11 || H < 11 || C < 1) return RO_ERR_ARG;
    double g[11], gs = 0.0;
    for (int k = 0; k < 11; ++k) { g[k] = exp(-(k - 5) * (k - 5) / (2.0 * 1.5 * 1.5)); gs += g[k]; }
    for (int k = 0; k < 11; ++k) g[k] /= gs;
    double c1 = (0.01 * max_value) * (0.01 * max_value), c2 = (0.03 * max_value) * (0.03 * max_value);
    double total = 0.0;
    long count = 0;
    for (int c = 0; c < C; ++c)
        for (int i = 0; i + 11 <= H; ++i)
            for (int j = 0; j + 11 <= W; ++j) {
                double mx = 0.0, my = 0.0, sxx = 0.0, syy = 0.0, sxy = 0.0;
                for (int u = 0; u < 11; ++u)
                    for (int v = 0; v < 11; ++v) {
                        double w = g[u] * g[v];
                        double x = a[((long)(i + u) * W + j + v) * C + c], y = b[((long)(i + u) * W + j + v) * C + c];
                        mx += w * x; my += w * y;
                        sxx += w * x * x; syy += w * y * y; sxy += w * x * y;
                    }
                double vx = sxx - mx * mx, vy = syy - my * my, cxy = sxy - mx * my;
                total += ((2.0 * mx * my + c1) * (2.0 * cxy + c2)) / ((mx * mx + my * my + c1) * (vx + vy + c2));
                ++count;
            }
    *ssim = total / (double)count;
    return RO_OK;
}
