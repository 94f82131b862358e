// tsim_device.cuh -- device data layout and per-particle / per-node math of
// the IMPM substep (Sec. III-A, Eqs. 1-9, Algorithm 1), FP32 on sm_103a.
//
// Layout in HBM (one context, all instances concatenated):
//   cell blocks   4x4x4 cells; block b owns particle slots [b*CAP, b*CAP+cnt[b])
//   particle SoA  P[par][c*S + slot], c = 0..2 position, 3..11 F (row-major);
//                 a cell-block slot holds its position in cell units relative
//                 to the block's first node, q = x/dx + o - g (see box_cells),
//                 a spill slot the position in metres;
//                 T[par][slot] tag; two parities, the fused kernel reads one
//                 and writes the other when x and F move.
//   VC            v (3) and C (9) per slot, stored only when asked for
//   grid          acc[node] = (M, MG) accumulated by P2G; vel[node] = V
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace tsim {

constexpr int BLK = 4;               // cells per cell-block edge
constexpr int CAP = 640;             // particle slots per cell block (1.25x the 512 of 8 ppc; the rest spill)
constexpr int NT = 128;              // threads of the fused transfer kernel (2 per cell)
constexpr int GV = 6;                // G2P node window edge (BLK + 2)
constexpr int GA = 8;                // P2G node window edge (BLK + 4: +-1 cell of motion)
constexpr int GAZ = 68;              // z stride of the P2G window (64 + 4: conflict-free banks)
constexpr int GAN = GAZ * GA;        // floats per P2G window channel
constexpr int NCELL = BLK * BLK * BLK;
constexpr int SORTC = CAP + 2 * NCELL;   // u16 per block of a stored cell sort: order, counts, offsets
constexpr int MAX_KF = 64;
constexpr int SPILL_CTAS = 16;       // extra CTAs of every transfer launch that process the spill slots
constexpr int LOGN = 32768;           // per-substep log ring (passes, calibration particle) per instance

constexpr uint32_t TAG_BOTTOM = 0x80000000u;
constexpr uint32_t TAG_TOP = 0x40000000u;
constexpr uint32_t ID_MASK = 0x1FFFFFFFu;

enum : uint32_t { ST_NUMERIC = 1u, ST_DOMAIN = 2u, ST_CAPACITY = 4u, ST_TIMEOUT = 8u };
enum { K_NONE = -1, K_SPHERE = 0, K_CYLINDER = 1, K_BOX = 2, K_PRISM = 3, K_PERLIN = 4 };
enum { BASE_FIXED = 0, BASE_SLIP = 1, BASE_FREE = 2 };

struct Inst {                      // per-instance constants
    int nx, ny, nz, ox, oy, oz;
    int nbx, nby, nbz, nblocks;
    int block0;                    // first global cell block
    int n_particles;
    long long node0;               // first node in acc / vel
    long long id0;                 // first particle in the id-ordered staging arrays
    float dx, inv_dx, dt, H;
    float mp, V0, mu, lam, kME;    // kME = -4 dt V0 / dx^2 (Eq. 4)
    float g[3];
    int base_mode, walls, limit;
    float threshold;
    int ind_kind;
    float ip[8];
    float fric, fric_k, tip_offset;     // static (stick) and kinetic (slip) Coulomb coefficients
    int nkf;
    int spc;                       // spill slots of this instance (particles beyond a full cell block)
    long long sp0;                 // first spill slot
    // particle-represented indenter (the paper's coupling): nobj > 0 particles
    // objq[obj0 ..] in the indenter frame, each of mass objm; no SDF contact then
    long long obj0;
    int nobj, objcap;
    float objm;
};

struct Pose {
    float tip[3], c[3];
    float cs, sn, omega;
    float vlin[3];
    float tip_next[3];
};

struct InstState {                 // mutable per instance
    Pose pose;
    unsigned long long e_key;      // nearest particle to the next tip: (squared-distance bits << 32) | slot
    float xe[3];
    int e_id;
    int xs[3];                     // box index of the first node of x_e's 3x3x3 G2P stencil
    int phase;                     // 0 iterating, 1 accepted: the commit transfer moves x and F
    int pass;
    unsigned int status;
    int dirty;
    long long passes_total;
    long long substeps;
    int nsp[2];                    // particles in the spill slots, per parity
    int sp_max;                    // most particles held in the spill slots at one time
    int pad_;
    long long spilled;             // spill-slot particles summed over committed substeps
};

struct Global {
    long long k_next, k_cur, k_end;
    int par_next, par_cur;
};

struct Dev {                       // device pointers (passed by value to kernels)
    float *P[2];
    uint32_t *T[2];
    int *cnt[2];
    float *VC;
    long long S;                   // slots per parity and component
    float4 *acc, *vel;
    int *blk_inst;
    unsigned short *sortc;         // per cell block, the cell sort of its first repeat pass in a substep
    float4 *objq;                  // object particles of all instances (indenter frame, xyz)
    Inst *inst;
    InstState *ist;
    Global *G;
    const float *kf;               // MAX_KF rows of 5 per instance
    const int *perm;               // 256 per instance
    int2 *log;                     // LOGN per instance
    // id-ordered staging (for writes and reads of particle state)
    float *sx, *sv, *sC, *sF;
    uint32_t *stag;
    // packed grid-update launch: per 128-node chunk (instance, its first chunk);
    // every instance's node range is padded to a multiple of 512 nodes
    const int2 *gchunk;
    long long n_gchunk;
    int n_inst;
    int n_blocks;                  // cell blocks of all instances
};

// Slot of the t-th particle position of instance I in parity par: t < nblocks *
// CAP walks the cell blocks' slots, the rest the instance's spill slots; -1
// where that position holds no particle.
__device__ __forceinline__ long long inst_slot(const Dev &d, const Inst &I, int inst, int par, long long t)
{
    const long long nb = (long long)I.nblocks * CAP;
    if (t < nb) {
        const int b = I.block0 + (int)(t / CAP), r = (int)(t % CAP);
        return r < min(d.cnt[par][b], CAP) ? (long long)b * CAP + r : -1;
    }
    const long long sp = t - nb;
    return sp < min(d.ist[inst].nsp[par], I.spc) ? I.sp0 + sp : -1;
}

// ----------------------------------------------------------------- positions
//
// Inside the cell blocks a particle's position is stored in cell units
// relative to the block's first node: q = u - g with u = x/dx + o the
// position in node-box cells (o: box index of physical node 0) and g the box
// index of the block's first node (a multiple of 4).  Subtracting the integer
// g from u is exact, so floor(q - 0.5) is the particle's base node in the
// block exactly as floor(u - 0.5) is in the box, and a particle that moves
// to a neighbouring block shifts q by exactly 4.  Since q < 4.5, the FP32
// rounding of the per-substep move is 25 to 80 times below that of a position
// in metres on a 40-60 mm pad.

// Box index of the first node of local cell block lb.
__device__ __forceinline__ void block_first_node(const Inst &I, int lb, int g[3])
{
    g[0] = (lb % I.nbx) * BLK;
    g[1] = ((lb / I.nbx) % I.nby) * BLK;
    g[2] = (lb / (I.nbx * I.nby)) * BLK;
}

// u = x/dx + o: a position in metres as node-box cells.
__device__ __forceinline__ float box_cells(float x, float inv_dx, int o) { return x * inv_dx + (float)o; }

// Metres of a stored block-relative position q (first node g, box offset o).
__device__ __forceinline__ float block_to_metres(float q, int g, int o, float dx) { return (q + (float)(g - o)) * dx; }

// Metres of the particle at the t-th position of instance I (slot = its slot
// from inst_slot): cell-block positions are converted, spill slots hold metres.
__device__ __forceinline__ void slot_metres(const Dev &d, const Inst &I, int par, long long t, long long slot,
                                            float x[3])
{
    const float *P = d.P[par];
    if (t < (long long)I.nblocks * CAP) {
        int g[3];
        block_first_node(I, (int)(t / CAP), g);
        x[0] = block_to_metres(P[slot], g[0], I.ox, I.dx);
        x[1] = block_to_metres(P[d.S + slot], g[1], I.oy, I.dx);
        x[2] = block_to_metres(P[2 * d.S + slot], g[2], I.oz, I.dx);
    } else {
        x[0] = P[slot];
        x[1] = P[d.S + slot];
        x[2] = P[2 * d.S + slot];
    }
}

// ----------------------------------------------------------------- B-spline

// Quadratic B-spline weights on one axis of a position u in cell units: the
// base node, the fractional offset f = u - base in [0.5, 1.5) and the 3
// weights.
__device__ __forceinline__ void bspline_cells(float u, int &base, float &f, float w[3])
{
    base = (int)floorf(u - 0.5f);
    f = u - (float)base;
    float a = 1.5f - f, b = f - 1.0f, c = f - 0.5f;
    w[0] = 0.5f * a * a;
    w[1] = 0.75f - b * b;
    w[2] = 0.5f * c * c;
}

// The same for a position x in metres: base node (physical index).
__device__ __forceinline__ void bspline(float x, float inv_dx, int &base, float &f, float w[3])
{
    bspline_cells(x * inv_dx, base, f, w);
}

// Kirchhoff stress of compressible Neo-Hookean: mu (F F^T - I) + lam ln J I.
__device__ __forceinline__ float kirchhoff(const float F[9], float mu, float lam, float tau[9])
{
    float J = F[0] * (F[4] * F[8] - F[5] * F[7]) - F[1] * (F[3] * F[8] - F[5] * F[6]) +
              F[2] * (F[3] * F[7] - F[4] * F[6]);
    float lj = lam * logf(J);
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = r; c < 3; ++c) {
            float s = F[r * 3] * F[c * 3] + F[r * 3 + 1] * F[c * 3 + 1] + F[r * 3 + 2] * F[c * 3 + 2];
            float t = mu * (s - (r == c ? 1.f : 0.f)) + (r == c ? lj : 0.f);
            tau[r * 3 + c] = t;
            tau[c * 3 + r] = t;
        }
    return J;
}

// ----------------------------------------------------------------- pose

// Piecewise-linear pose at substep k from MAX_KF rows (substep, tip xyz, yaw);
// evaluated in FP64, stored in FP32.
__device__ inline void pose_tip(const float *kf, int nkf, long long k, double out[4],
                                double vel[4], double dt)
{
    int i = -1;
    for (int a = 0; a < nkf; ++a)
        if ((double)kf[a * 5] <= (double)k) i = a;
    if (nkf == 0) {
        for (int d = 0; d < 4; ++d) { out[d] = d == 2 ? 1e3 : 0.0; vel[d] = 0.0; }
        return;
    }
    if (i < 0 || i == nkf - 1) {
        int a = i < 0 ? 0 : i;
        for (int d = 0; d < 4; ++d) { out[d] = (double)kf[a * 5 + 1 + d]; vel[d] = 0.0; }
        return;
    }
    const float *p0 = kf + i * 5, *p1 = kf + (i + 1) * 5;
    double span = (double)p1[0] - (double)p0[0];
    double al = ((double)k - (double)p0[0]) / span;
    for (int d = 0; d < 4; ++d) {
        double a = p0[1 + d], b = p1[1 + d];
        out[d] = a + al * (b - a);
        vel[d] = (b - a) / (span * dt);
    }
}

__device__ inline void pose_eval(const Inst &I, const float *kf, long long k, Pose &P)
{
    double t[4], v[4], tn[4], vn[4];
    pose_tip(kf, I.nkf, k, t, v, (double)I.dt);
    pose_tip(kf, I.nkf, k + 1, tn, vn, (double)I.dt);
    for (int d = 0; d < 3; ++d) {
        P.tip[d] = (float)t[d];
        P.c[d] = (float)(d == 2 ? t[2] + (double)I.tip_offset : t[d]);
        P.vlin[d] = (float)v[d];
        P.tip_next[d] = (float)tn[d];
    }
    // the yaw is interpolated in FP64; its FP32 sine and cosine are exact to
    // ~1e-7 rad (sub-nanometre at the indenter's size) and far cheaper than FP64
    float sn, cs;
    sincosf((float)t[3], &sn, &cs);
    P.cs = cs;
    P.sn = sn;
    P.omega = (float)v[3];
}

// ----------------------------------------------------------------- indenter SDFs

__device__ __forceinline__ float sgnf(float a) { return a < 0.f ? -1.f : 1.f; }

// rounded box in n = 2 or 3 dims (half sizes h, edge radius re)
template <int N>
__device__ __forceinline__ float sd_round_box(const float *q, const float *h, float re, float *g)
{
    float d[N], o[N], L2 = 0.f, dmax = -3.0e38f;
    int kmax = 0;
#pragma unroll
    for (int a = 0; a < N; ++a) {
        d[a] = fabsf(q[a]) - (h[a] - re);
        o[a] = fmaxf(d[a], 0.f);
        L2 += o[a] * o[a];
        if (d[a] > dmax) { dmax = d[a]; kmax = a; }
    }
    float L = sqrtf(L2);
#pragma unroll
    for (int a = 0; a < N; ++a) g[a] = 0.f;
    if (dmax > 0.f) {
#pragma unroll
        for (int a = 0; a < N; ++a) g[a] = sgnf(q[a]) * o[a] / L;
    } else {
#pragma unroll
        for (int a = 0; a < N; ++a)
            if (a == kmax) g[a] = sgnf(q[a]);
    }
    return L + fminf(dmax, 0.f) - re;
}

// equilateral triangle of inradius r in (y, z), apex towards -z, exact SDF
__device__ __forceinline__ float sd_triangle(float y, float z, float r, float g[2])
{
    const float s3 = 1.7320508075688772f;
    const float Vy[3] = {0.f, s3 * r, -s3 * r}, Vz[3] = {-2.f * r, r, r};
    const float Ny[3] = {0.f, 0.5f * s3, -0.5f * s3}, Nz[3] = {1.f, -0.5f, -0.5f};
    float smax = -3.0e38f;
    int emax = 0;
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        float s = Ny[e] * y + Nz[e] * z - r;
        if (s > smax) { smax = s; emax = e; }
    }
    if (smax <= 0.f) {
        g[0] = Ny[emax];
        g[1] = Nz[emax];
        return smax;
    }
    float best = 3.0e38f, by = 0.f, bz = 0.f;
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        int i0 = (e + 1) % 3, i1 = (e + 2) % 3;
        float ey = Vy[i1] - Vy[i0], ez = Vz[i1] - Vz[i0];
        float t = ((y - Vy[i0]) * ey + (z - Vz[i0]) * ez) / (ey * ey + ez * ez);
        t = fminf(fmaxf(t, 0.f), 1.f);
        float dy = y - (Vy[i0] + t * ey), dz = z - (Vz[i0] + t * ez);
        float dd = sqrtf(dy * dy + dz * dz);
        if (dd < best) { best = dd; by = dy; bz = dz; }
    }
    g[0] = by / best;
    g[1] = bz / best;
    return best;
}

// Improved noise (K. Perlin, 2002) on the plane z = 0 with its xy gradient.
__device__ __forceinline__ float pgrad(int h, float x, float y)
{
    h &= 15;
    float u = h < 8 ? x : y;
    float v = h < 4 ? y : ((h == 12 || h == 14) ? x : 0.f);
    return ((h & 1) ? -u : u) + ((h & 2) ? -v : v);
}

__device__ inline float noise2(const int *perm, float x, float y, float &gx, float &gy)
{
    float fx = floorf(x), fy = floorf(y);
    int X = ((int)fx) & 255, Y = ((int)fy) & 255;
    x -= fx;
    y -= fy;
    auto P = [&](int i) { return perm[i & 255]; };
    int A = P(X) + Y, B = P(X + 1) + Y;
    int h00 = P(P(A)), h10 = P(P(B)), h01 = P(P(A + 1)), h11 = P(P(B + 1));
    float g00 = pgrad(h00, x, y), g10 = pgrad(h10, x - 1.f, y);
    float g01 = pgrad(h01, x, y - 1.f), g11 = pgrad(h11, x - 1.f, y - 1.f);
    float ax00 = pgrad(h00, 1.f, 0.f), ay00 = pgrad(h00, 0.f, 1.f);
    float ax10 = pgrad(h10, 1.f, 0.f), ay10 = pgrad(h10, 0.f, 1.f);
    float ax01 = pgrad(h01, 1.f, 0.f), ay01 = pgrad(h01, 0.f, 1.f);
    float ax11 = pgrad(h11, 1.f, 0.f), ay11 = pgrad(h11, 0.f, 1.f);
    float u = x * x * x * (x * (x * 6.f - 15.f) + 10.f);
    float v = y * y * y * (y * (y * 6.f - 15.f) + 10.f);
    float du = 30.f * x * x * (x - 1.f) * (x - 1.f);
    float dv = 30.f * y * y * (y - 1.f) * (y - 1.f);
    float l0 = g00 + u * (g10 - g00), l1 = g01 + u * (g11 - g01);
    float l0x = ax00 + u * (ax10 - ax00) + du * (g10 - g00);
    float l1x = ax01 + u * (ax11 - ax01) + du * (g11 - g01);
    float l0y = ay00 + u * (ay10 - ay00), l1y = ay01 + u * (ay11 - ay01);
    gx = l0x + v * (l1x - l0x);
    gy = l0y + v * (l1y - l0y) + dv * (l1 - l0);
    return l0 + v * (l1 - l0);
}

// SDF of the indenter in its local frame with its (unit) gradient.
__device__ inline float sdf_local(int kind, const float *p, const int *perm, const float q[3],
                                  float g[3])
{
    switch (kind) {
    case K_SPHERE: {
        float d = sqrtf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2]);
        if (d > 0.f) { g[0] = q[0] / d; g[1] = q[1] / d; g[2] = q[2] / d; }
        else { g[0] = 0.f; g[1] = 0.f; g[2] = -1.f; }
        return d - p[0];
    }
    case K_CYLINDER: {
        float rho = sqrtf(q[0] * q[0] + q[1] * q[1]);
        float q2[2] = {rho, q[2]}, h2[2] = {p[0], 0.5f * p[1]}, g2[2];
        float phi = sd_round_box<2>(q2, h2, p[2], g2);
        float ex = 1.f, ey = 0.f;
        if (rho > 0.f) { ex = q[0] / rho; ey = q[1] / rho; }
        g[0] = g2[0] * ex; g[1] = g2[0] * ey; g[2] = g2[1];
        return phi;
    }
    case K_BOX:
        return sd_round_box<3>(q, p, p[3], g);
    case K_PRISM: {
        float re = p[2];
        float r = p[0] * 0.28867513459481287f - re;     // side / (2 sqrt 3) - re
        float g2[2];
        float d2 = sd_triangle(q[1], q[2], r, g2);
        float w0 = d2, w1 = fabsf(q[0]) - (0.5f * p[1] - re);
        float o0 = fmaxf(w0, 0.f), o1 = fmaxf(w1, 0.f);
        float L = sqrtf(o0 * o0 + o1 * o1);
        float m = fmaxf(w0, w1);
        float gw0, gw1;
        if (m > 0.f) { gw0 = o0 / L; gw1 = o1 / L; }
        else if (w0 > w1) { gw0 = 1.f; gw1 = 0.f; }
        else { gw0 = 0.f; gw1 = 1.f; }
        g[0] = gw1 * sgnf(q[0]); g[1] = gw0 * g2[0]; g[2] = gw0 * g2[1];
        return fminf(m, 0.f) + L - re;
    }
    case K_PERLIN: {
        float gb[3];
        float phi = sd_round_box<3>(q, p, p[3], gb);
        float amp = p[4], pers = p[6];
        int oct = (int)p[7];
        float f = 0.f, fx = 0.f, fy = 0.f, a = 1.f, s = 1.f / p[5];
        for (int o = 0; o < oct; ++o) {
            float nx, ny;
            float nv = noise2(perm, q[0] * s, q[1] * s, nx, ny);
            f += a * nv; fx += a * s * nx; fy += a * s * ny;
            a *= pers; s *= 2.f;
        }
        g[0] = gb[0] - amp * fx; g[1] = gb[1] - amp * fy; g[2] = gb[2];
        float gl = rsqrtf(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
        g[0] *= gl; g[1] *= gl; g[2] *= gl;
        return phi - amp * f;
    }
    default:
        g[0] = 0.f; g[1] = 0.f; g[2] = 1.f;
        return 3.0e38f;
    }
}

// World-frame SDF value and unit outward normal at xw for pose P.
__device__ inline float sdf_world(const Inst &I, const int *perm, const Pose &P, const float xw[3],
                                  float n[3])
{
    float d0 = xw[0] - P.c[0], d1 = xw[1] - P.c[1];
    float q[3] = {P.cs * d0 + P.sn * d1, -P.sn * d0 + P.cs * d1, xw[2] - P.c[2]};
    float g[3];
    float phi = sdf_local(I.ind_kind, I.ip, perm, q, g);
    n[0] = P.cs * g[0] - P.sn * g[1];
    n[1] = P.sn * g[0] + P.cs * g[1];
    n[2] = g[2];
    return phi;
}

__device__ __forceinline__ void object_velocity(const Pose &P, const float xw[3], float vo[3])
{
    vo[0] = P.vlin[0] - P.omega * (xw[1] - P.c[1]);
    vo[1] = P.vlin[1] + P.omega * (xw[0] - P.c[0]);
    vo[2] = P.vlin[2];
}

}  // namespace tsim
