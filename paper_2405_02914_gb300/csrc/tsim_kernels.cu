// tsim_kernels.cu -- sm_103a kernels of the IMPM substep.
//
// One substep (Algorithm 1) for all instances in lockstep:
//   k_round_begin     pose of substep k (and the tip at k+1), reset pass state,
//                     x_e and its stencil, empty the commit's cell-block counters
//   k_grid            Eq. 5 + gravity + stick/slip SDF contact + walls + base,
//                     one sweep over the node box; clears the P2G accumulator.
//                     Its CTA 0 updates x_e's 27 stencil nodes itself and runs
//                     the relative-rest check at the calibration particle x_e
//   k_transfer<ITER>  fused G2P (Eqs. 6-7) -> P2G (Eqs. 1-4) of a repeated pass:
//                     x and F stay, v and C go straight back to the grid
//   k_transfer<COMMIT> fused G2P -> F, x move (Eqs. 8-9) -> re-bin into the
//                     cell block of the new position -> P2G of the moved state
//                     (the first pass of the next substep)
// The velocity and affine field live on the grid between substeps; only x,
// F and the tag persist per particle.
#include <cuda_runtime.h>

#include <algorithm>

#include "tsim_device.cuh"
#include "tsim_kernels.h"

namespace tsim {

__device__ __forceinline__ void atomic_or_status(InstState *S, unsigned int bits)
{
    atomicOr(&S->status, bits);
}

__device__ __forceinline__ long long node_of(const Inst &I, int ax, int ay, int az)
{
    return I.node0 + ((long long)az * I.ny + ay) * I.nx + ax;
}

// ---------------------------------------------------------------- round begin

// Thread inst of the grid, per instance: pose of substep k (and the tip at
// k+1), pass state reset, and x_e of Algorithm 1 -- the particle nearest to
// the tip x_o -- from the key that the previous commit (or prologue) left
// behind: (squared-distance bits << 32) | slot of that particle in the
// current state, with the first node of its G2P stencil.  All threads empty
// the cell-block counters that this substep's commit fills.  Nothing in
// this kernel writes the global substep counters.
__global__ void k_round_begin(Dev d)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    {
        int *dst = d.cnt[d.G->par_next ^ 1];
        for (int b = g; b < d.n_blocks; b += gridDim.x * blockDim.x) dst[b] = 0;
    }
    const int inst = g;
    if (inst >= d.n_inst) return;
    InstState *S = d.ist + inst;
    const Inst &I = d.inst[inst];
    const long long k = d.G->k_next;
    const int par = d.G->par_next;
    Pose P;
    pose_eval(I, d.kf + (long long)inst * MAX_KF * 5, k, P);
    S->pose = P;
    S->phase = 0;
    S->pass = 0;
    // the commit of this substep fills the other parity's spill slots afresh
    const int nsp = min(S->nsp[par], I.spc);
    S->spilled += nsp;
    if (nsp > S->sp_max) S->sp_max = nsp;
    S->nsp[par ^ 1] = 0;
    const unsigned long long key = S->e_key;
    S->e_key = ~0ull;                              // the commit of this substep fills it again
    if (key == ~0ull) {
        S->e_id = -1;
        S->xs[0] = S->xs[1] = S->xs[2] = -1;
    } else {
        const long long slot = (long long)(key & 0xffffffffull);
        // a cell-block slot of this instance holds block cells: position t = slot - block0 * CAP
        const long long t = slot < I.sp0 ? slot - (long long)I.block0 * CAP : (long long)I.nblocks * CAP;
        float xe[3];
        slot_metres(d, I, par, t, slot, xe);
        S->xe[0] = xe[0];
        S->xe[1] = xe[1];
        S->xe[2] = xe[2];
        S->e_id = (int)(d.T[par][slot] & ID_MASK);
        const int o[3] = {I.ox, I.oy, I.oz};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            int b;
            float f, w[3];
            bspline(xe[a], I.inv_dx, b, f, w);
            S->xs[a] = b + o[a];
        }
    }
}

__global__ void k_set_end(Dev d, long long n)
{
    d.G->k_end = d.G->k_next + n;
}

// ---------------------------------------------------------------- grid update

// Grid velocity of node (ax, ay, az) of instance inst (box indices) from its
// P2G sums a = (M, MG) with M > 0: Eq. 5 + gravity, SDF contact with Coulomb
// stick/slip, walls, base.
__device__ __forceinline__ void grid_velocity(const Dev &d, const Inst &I, const InstState *S, int inst, float4 a,
                                              int ax, int ay, int az, float V[3])
{
    V[0] = a.y / a.x + I.dt * I.g[0];
    V[1] = a.z / a.x + I.dt * I.g[1];
    V[2] = a.w / a.x + I.dt * I.g[2];
    if (I.ind_kind != K_NONE && I.nobj == 0) {         // object particles replace the SDF contact
        const Pose &P = S->pose;
        float xw[3] = {(ax - I.ox) * I.dx, (ay - I.oy) * I.dx, (az - I.oz) * I.dx};
        float n[3];
        float phi = sdf_world(I, d.perm + inst * 256, P, xw, n);
        if (phi <= 0.f) {
            float vo[3];
            object_velocity(P, xw, vo);
            float vr[3] = {V[0] - vo[0], V[1] - vo[1], V[2] - vo[2]};
            float vn = vr[0] * n[0] + vr[1] * n[1] + vr[2] * n[2];
            if (vn < 0.f) {
                float vt[3] = {vr[0] - vn * n[0], vr[1] - vn * n[1], vr[2] - vn * n[2]};
                float vtl = sqrtf(vt[0] * vt[0] + vt[1] * vt[1] + vt[2] * vt[2]);
                float lim = I.fric * (-vn);
                // rest, or Coulomb slip with the kinetic coefficient
                float sc = vtl <= lim ? 0.f : 1.f - I.fric_k * (-vn) / vtl;
#pragma unroll
                for (int r = 0; r < 3; ++r) V[r] = vt[r] * sc + vo[r];
            }
        }
    }
    if (I.walls && (ax < 2 || ay < 2 || ax >= I.nx - 2 || ay >= I.ny - 2 || az >= I.nz - 2))
        V[0] = V[1] = V[2] = 0.f;
    if (az - I.oz <= 0) {
        if (I.base_mode == BASE_FIXED) V[0] = V[1] = V[2] = 0.f;
        else if (I.base_mode == BASE_SLIP) V[2] = 0.f;
    }
}

// x_e's 3x3x3 stencil (first node xs, box indices) lies inside the node box.
__device__ __forceinline__ bool xe_stencil_inside(const Inst &I, const int xs[3])
{
    return xs[0] >= 0 && xs[1] >= 0 && xs[2] >= 0 && xs[0] + 2 < I.nx && xs[1] + 2 < I.ny && xs[2] + 2 < I.nz;
}

// Grid update of node t (x fastest) of instance inst by the node sweep; it
// clears the node's P2G accumulator.  A node without mass is left as it is
// (no G2P gives it weight).  The 27 nodes of x_e's stencil belong to the
// check CTA of the same launch, which needs their velocities.
__device__ __forceinline__ void grid_node(const Dev &d, int inst, long long t)
{
    const Inst &I = d.inst[inst];
    const long long nn = (long long)I.nx * I.ny * I.nz;
    if (t >= nn) return;
    const float4 a = d.acc[I.node0 + t];
    if (!(a.x > 0.f)) return;
    const InstState *S = d.ist + inst;
    // a node box has fewer than 2^31 nodes: 32-bit index arithmetic
    const unsigned int tu = (unsigned int)t, nx = (unsigned int)I.nx, ny = (unsigned int)I.ny;
    const unsigned int row = tu / nx;
    const int ax = (int)(tu - row * nx), ay = (int)(row % ny), az = (int)(row / ny);
    const int xs[3] = {S->xs[0], S->xs[1], S->xs[2]};
    if (xe_stencil_inside(I, xs) && (unsigned)(ax - xs[0]) < 3u && (unsigned)(ay - xs[1]) < 3u &&
        (unsigned)(az - xs[2]) < 3u)
        return;
    float V[3];
    grid_velocity(d, I, S, inst, a, ax, ay, az, V);
    d.vel[I.node0 + t] = make_float4(V[0], V[1], V[2], 0.f);
    d.acc[I.node0 + t] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// ---------------------------------------------------------------- relative-rest check

// The check CTA of a grid update launch, one warp per instance.  Its 27 lanes
// first do the grid update of x_e's stencil nodes (the node sweep leaves them
// out) and keep the velocities in registers; then each instance still
// iterating compares the tangential velocity at x_e (G2P of those nodes) with
// the object's (Algorithm 1) and either commits or asks for another pass; a
// pass count >= LIMIT always commits, so the device-driven loop of the graph
// ends after at most LIMIT passes.  On the first pass of a substep it also
// advances the global substep counters.  Thread 0 alone sets the loop
// condition, once per launch.  Nothing else in the launch reads what this
// CTA writes.
__device__ void check_cta(const Dev &d, cudaGraphConditionalHandle h, int use_cond)
{
    __shared__ int s_any;
    __shared__ int s_first;
    if (threadIdx.x == 0) {
        s_any = 0;
        s_first = d.ist[0].pass == 0 && d.ist[0].phase == 0;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int si = lane / 9, sj = (lane / 3) % 3, sk = lane % 3;
    for (int inst = threadIdx.x >> 5; inst < d.n_inst; inst += blockDim.x >> 5) {
        InstState *S = d.ist + inst;
        const Inst &I = d.inst[inst];
        const int xs[3] = {S->xs[0], S->xs[1], S->xs[2]};
        const bool inside = xe_stencil_inside(I, xs);
        float V[3] = {0.f, 0.f, 0.f};
        if (inside && lane < 27) {
            const int ax = xs[0] + si, ay = xs[1] + sj, az = xs[2] + sk;
            const long long node = I.node0 + ((long long)az * I.ny + ay) * I.nx + ax;
            const float4 a = d.acc[node];
            if (a.x > 0.f) {
                grid_velocity(d, I, S, inst, a, ax, ay, az, V);
                d.vel[node] = make_float4(V[0], V[1], V[2], 0.f);
                d.acc[node] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
        if (S->phase != 0) continue;        // committing or done: the commit transfer follows the loop
        bool accept = true;
        const Pose &P = S->pose;
        if (I.ind_kind != K_NONE && S->e_id >= 0) {
            const float xe[3] = {S->xe[0], S->xe[1], S->xe[2]};
            float n[3];
            const float phi = sdf_world(I, d.perm + inst * 256, P, xe, n);
            if (phi <= I.dx) {
                float vo[3];
                object_velocity(P, xe, vo);
                const float vot = sqrtf(vo[0] * vo[0] + vo[1] * vo[1]);
                if (vot >= 1e-6f) {
                    // G2P (Eq. 6) of the tangential velocity at x_e
                    float ve0 = 0.f, ve1 = 0.f;
                    if (inside && lane < 27) {
                        int base[3];
                        float f[3], w[3][3];
#pragma unroll
                        for (int a = 0; a < 3; ++a) bspline(xe[a], I.inv_dx, base[a], f[a], w[a]);
                        const float wt = w[0][si] * w[1][sj] * w[2][sk];
                        ve0 = wt * V[0];
                        ve1 = wt * V[1];
                    }
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        ve0 += __shfl_xor_sync(0xffffffffu, ve0, o);
                        ve1 += __shfl_xor_sync(0xffffffffu, ve1, o);
                    }
                    const float a = ve0 - vo[0], b = ve1 - vo[1];
                    accept = sqrtf(a * a + b * b) <= I.threshold * vot;
                }
            }
        }
        __syncwarp();
        if (lane == 0) {
            const int pass = S->pass + 1;
            S->pass = pass;
            S->passes_total += 1;
            if (accept || pass >= I.limit) {
                S->phase = 1;
                const long long s = S->substeps;
                d.log[(long long)inst * LOGN + (s % LOGN)] = make_int2(pass, S->e_id);
                S->substeps = s + 1;
            } else {
                atomicOr(&s_any, 1);
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (s_first) {
            const long long k = d.G->k_next;
            const int par = d.G->par_next;
            d.G->k_cur = k;
            d.G->par_cur = par;
            d.G->k_next = k + 1;
            d.G->par_next = par ^ 1;
        }
        if (use_cond) cudaGraphSetConditional(h, s_any ? 1u : 0u);
    }
}

// The grid update with the relative-rest check: CTA 0 of the launch is the
// check CTA, the others sweep the nodes.  One launch row per instance
// (blockIdx.y), sized by the largest instance.
__global__ void __launch_bounds__(512) k_grid(Dev d, cudaGraphConditionalHandle h, int use_cond)
{
    if (blockIdx.x == 0) {
        if (blockIdx.y == 0) check_cta(d, h, use_cond);
        return;
    }
    grid_node(d, blockIdx.y, (long long)(blockIdx.x - 1) * blockDim.x + threadIdx.x);
}

// The same as one 1-D launch over all instances' node ranges packed back to
// back (no empty CTAs for the smaller instances of an uneven batch); a CTA of
// up to 512 threads never straddles two instances.
__global__ void __launch_bounds__(512) k_grid_flat(Dev d, cudaGraphConditionalHandle h, int use_cond)
{
    if (blockIdx.x == 0) {
        check_cta(d, h, use_cond);
        return;
    }
    const long long g = (long long)(blockIdx.x - 1) * blockDim.x + threadIdx.x;
    const int2 e = d.gchunk[g >> 7];
    grid_node(d, e.x, g - ((long long)e.y << 7));
}

// ---------------------------------------------------------------- fused transfer

enum { MODE_PROLOGUE = 0, MODE_ITER = 1, MODE_COMMIT = 2 };

// Shared memory of one cell block (dynamic, 44 KB: five CTAs per SM).
struct TransferSmem {
    // staged x (0..2), F (3..11) and tag bits (12) of the block's particles (TMA);
    // phase 1 overwrites a particle's entries with its P2G coefficients:
    // Q (0..8), m v (9..11), fractional offset f of the new position (12..14;
    // -1 in row 12: the particle left its cell).  Row 13 holds the sort keys
    // (cell | rank in the cell << 6, -1: invalid) until phase 1 starts; after
    // phase 2 has read the rows they hold the per-warp node slabs
    float P[15][CAP];
    float4 V[GV * GV * GV];        // grid velocities of the G2P window
    unsigned short idx[CAP];       // particle order sorted by cell
    int ccount[NCELL], coff[NCELL];
    unsigned long long bar;        // mbarrier of the bulk copies
    unsigned long long key[NT / 32];
    float tip[3];
    Inst inst;                     // the instance constants, copied once per CTA
};

// Per-warp node slab of the P2G combine: warp w holds the 4x4 cells of z layer
// w, whose 3x3x3 stencils cover 6 x 6 x 3 nodes, one float4 (M, MG) per node;
// the two threads of a cell add their channel pairs to the two halves of a
// node's float4, and with rows of 6 nodes the 16 cells of a warp fill each
// bank group exactly twice (two wavefronts, the minimum for 256 bytes).
constexpr int SLX = 6, SLY = 6, SLZ = 3;
constexpr int SLAB = SLX * SLY * SLZ;  // float4 nodes per warp slab
static_assert((NT / 32) * SLAB * 4 <= 15 * CAP, "the slabs fit in the staging rows");
static_assert(NT == 2 * NCELL && NCELL / (NT / 32) == 16, "two threads per cell, one z layer of cells per warp");

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// packed FP32 pairs (one Blackwell instruction per pair)
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 fadd2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 fmul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 dup2(float a) { return make_float2(a, a); }

// G2P of one particle from the block's velocity window (Eqs. 6-7), factorised
// over the tensor-product weights: per (i, j) row the k-sums, per i the
// j-sums, then the i-sum; d = x_i - x_p in cells.  Window nodes hold
// (V_x, V_y, V_z, V_z), so one packed FMA takes both the weight and the
// weight-times-offset sum of V_z.  Returns v and D = sum w V d^T.
__device__ __forceinline__ void g2p_window(const float4 *__restrict__ Vw, int cx, int cy, int cz,
                                           const float w[3][3], const float f[3], float v[3], float D[9])
{
    float2 wx[3], wy[3], wz[3], ex[3], ey[3], ez[3], wez[3];
    float exs[3], eys[3], wxs[3];
#pragma unroll
    for (int o = 0; o < 3; ++o) {
        exs[o] = w[0][o] * ((float)o - f[0]);
        eys[o] = w[1][o] * ((float)o - f[1]);
        wxs[o] = w[0][o];
        wx[o] = dup2(w[0][o]); ex[o] = dup2(exs[o]);
        wy[o] = dup2(w[1][o]); ey[o] = dup2(eys[o]);
        wz[o] = dup2(w[2][o]); ez[o] = dup2(w[2][o] * ((float)o - f[2]));
        wez[o] = make_float2(w[2][o], w[2][o] * ((float)o - f[2]));
    }
    const float2 z2 = make_float2(0.f, 0.f);
    // v = (vxy, vzD.x), D_zz = vzD.y
    float2 vxy = z2, vzD = z2, Dxxy = z2, Dyxy = z2, Dzxy = z2;
    float Dxz = 0.f, Dyz = 0.f;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        float2 Uxy = z2, Uyxy = z2, Uzxy = z2, UzUzz = z2;
        float Uyz = 0.f;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            float2 Txy = z2, Tzxy = z2, Tzwe = z2;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const float4 V = Vw[((cz + k) * GV + (cy + j)) * GV + (cx + i)];
                const float2 Vxy = make_float2(V.x, V.y), Vzz = make_float2(V.z, V.w);
                Txy = ffma2(wz[k], Vxy, Txy);
                Tzxy = ffma2(ez[k], Vxy, Tzxy);
                Tzwe = ffma2(wez[k], Vzz, Tzwe);          // (sum wz V_z, sum ez V_z)
            }
            Uxy = ffma2(wy[j], Txy, Uxy);
            Uyxy = ffma2(ey[j], Txy, Uyxy);
            Uzxy = ffma2(wy[j], Tzxy, Uzxy);
            UzUzz = ffma2(wy[j], Tzwe, UzUzz);           // (sum wy wz V_z, sum wy ez V_z)
            Uyz = fmaf(eys[j], Tzwe.x, Uyz);             // sum ey wz V_z
        }
        vxy = ffma2(wx[i], Uxy, vxy);
        Dxxy = ffma2(ex[i], Uxy, Dxxy);
        Dyxy = ffma2(wx[i], Uyxy, Dyxy);
        Dzxy = ffma2(wx[i], Uzxy, Dzxy);
        vzD = ffma2(wx[i], UzUzz, vzD);                  // (v_z, D_zz)
        Dxz = fmaf(exs[i], UzUzz.x, Dxz);
        Dyz = fmaf(wxs[i], Uyz, Dyz);
    }
    v[0] = vxy.x; v[1] = vxy.y; v[2] = vzD.x;
    // D[r][c] = sum w V_r d_c
    D[0] = Dxxy.x; D[3] = Dxxy.y; D[6] = Dxz;
    D[1] = Dyxy.x; D[4] = Dyxy.y; D[7] = Dyz;
    D[2] = Dzxy.x; D[5] = Dzxy.y; D[8] = vzD.y;
}


__device__ __forceinline__ void mbar_init(unsigned long long *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// 1-D bulk copy global -> shared (TMA); both addresses 16-byte aligned, size a multiple of 16.
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, unsigned long long *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: gives up after ~1e6 polls (each poll may suspend briefly).
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long *bar, uint32_t parity)
{
    for (int it = 0; it < (1 << 20); ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// P2G of one particle straight into the grid with global vector atomics
// (Eqs. 1-4); used for the few particles whose stencil left their cell.
__device__ __noinline__ void p2g_global(float4 *acc, const Inst &I, int bx, int by, int bz, const float w[3][3],
                                        const float f[3], const float Q[9], const float mv[3], float mp)
{
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            for (int k = 0; k < 3; ++k) {
                const float wt = w[0][i] * w[1][j] * w[2][k];
                const float d0 = (float)i - f[0], d1 = (float)j - f[1], d2 = (float)k - f[2];
                atomicAdd(&acc[node_of(I, bx + i, by + j, bz + k)],
                          make_float4(wt * mp, wt * (mv[0] + Q[0] * d0 + Q[1] * d1 + Q[2] * d2),
                                      wt * (mv[1] + Q[3] * d0 + Q[4] * d1 + Q[5] * d2),
                                      wt * (mv[2] + Q[6] * d0 + Q[7] * d1 + Q[8] * d2)));
            }
}

// Claim a destination slot for a particle moving into cell block key: the
// block's next slot, or, when the block is full, the next spill slot of the
// instance (-1 when those are full too).
__device__ __forceinline__ long long claim_spill(const Dev &d, const Inst &I, int inst, int dpar)
{
    const int sp = atomicAdd(&d.ist[inst].nsp[dpar], 1);
    return sp < I.spc ? I.sp0 + sp : -1;
}

// One particle held in a spill slot, through the same pass as the particles
// of the cell blocks (Eqs. 1-9): G2P from the grid, the move on a commit
// pass, stress, P2G with global atomics, re-binning, candidate key.
template <int MODE>
__device__ void spill_particle(const Dev &d, const Inst &I, InstState *S, int inst, int par, long long slot)
{
    const long long SS = d.S;
    const float *src = d.P[par];
    float x[3], F[9], v[3], C[9];
#pragma unroll
    for (int c = 0; c < 3; ++c) x[c] = src[c * SS + slot];
#pragma unroll
    for (int c = 0; c < 9; ++c) F[c] = src[(3 + c) * SS + slot];
    const uint32_t tag = d.T[par][slot];
    // spill slots hold metres; the stencil is found in node-box cells (box_cells)
    const int oo[3] = {I.ox, I.oy, I.oz};
    int base[3];
    float f[3], w[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a) bspline_cells(box_cells(x[a], I.inv_dx, oo[a]), base[a], f[a], w[a]);
    const int ax0 = base[0], ay0 = base[1], az0 = base[2];
    if (ax0 < 0 || ay0 < 0 || az0 < 0 || ax0 + 2 >= I.nx || ay0 + 2 >= I.ny || az0 + 2 >= I.nz) {
        atomicOr(&S->status, ST_DOMAIN);
        return;
    }
    if (MODE == MODE_PROLOGUE) {
#pragma unroll
        for (int c = 0; c < 3; ++c) v[c] = d.VC[c * SS + slot];
#pragma unroll
        for (int c = 0; c < 9; ++c) C[c] = d.VC[(3 + c) * SS + slot];
    } else {
        // v = sum w V (Eq. 6), C = 4/dx^2 sum w V (x_i - x_p)^T (Eq. 7), d in cells
#pragma unroll
        for (int c = 0; c < 3; ++c) v[c] = 0.f;
#pragma unroll
        for (int c = 0; c < 9; ++c) C[c] = 0.f;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                for (int k = 0; k < 3; ++k) {
                    const float4 V = d.vel[node_of(I, ax0 + i, ay0 + j, az0 + k)];
                    const float wt = w[0][i] * w[1][j] * w[2][k];
                    const float dd[3] = {(float)i - f[0], (float)j - f[1], (float)k - f[2]};
                    const float Vr[3] = {V.x, V.y, V.z};
#pragma unroll
                    for (int r = 0; r < 3; ++r) {
                        v[r] += wt * Vr[r];
#pragma unroll
                        for (int c = 0; c < 3; ++c) C[r * 3 + c] += wt * Vr[r] * dd[c];
                    }
                }
#pragma unroll
        for (int c = 0; c < 9; ++c) C[c] *= 4.f * I.inv_dx;
        if ((tag & TAG_BOTTOM) && I.base_mode != BASE_FREE) v[2] = 0.f;   // Algorithm 1
    }
    if (MODE == MODE_COMMIT) {
        float Fn[9];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c)
                Fn[r * 3 + c] = F[r * 3 + c] + I.dt * (C[r * 3] * F[c] + C[r * 3 + 1] * F[3 + c] + C[r * 3 + 2] * F[6 + c]);
#pragma unroll
        for (int c = 0; c < 9; ++c) F[c] = Fn[c];
#pragma unroll
        for (int c = 0; c < 3; ++c) x[c] += I.dt * v[c];
    }
    float tau[9];
    const float J = kirchhoff(F, I.mu, I.lam, tau);
    if (!(J > 0.f) || !isfinite(J) || !isfinite(x[0]) || !isfinite(x[1]) || !isfinite(x[2])) {
        atomicOr(&S->status, ST_NUMERIC);
        return;
    }
    int nb[3];
    float nf[3], nw[3][3], u[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        u[a] = box_cells(x[a], I.inv_dx, oo[a]);
        bspline_cells(u[a], nb[a], nf[a], nw[a]);
    }
    if (nb[0] < 0 || nb[1] < 0 || nb[2] < 0 || nb[0] + 2 >= I.nx || nb[1] + 2 >= I.ny || nb[2] + 2 >= I.nz) {
        atomicOr(&S->status, ST_DOMAIN);
        return;
    }
    float Q[9];
#pragma unroll
    for (int c = 0; c < 9; ++c) Q[c] = (I.mp * C[c] + I.kME * tau[c]) * I.dx;
    const float mv[3] = {I.mp * v[0], I.mp * v[1], I.mp * v[2]};
    p2g_global(d.acc, I, nb[0], nb[1], nb[2], nw, nf, Q, mv, I.mp);
    long long cand = slot;
    if (MODE == MODE_COMMIT) {
        const int key = I.block0 + ((nb[2] / BLK) * I.nby + (nb[1] / BLK)) * I.nbx + (nb[0] / BLK);
        const int rr = atomicAdd(&d.cnt[par ^ 1][key], 1);
        const long long ds = rr < CAP ? (long long)key * CAP + rr : claim_spill(d, I, inst, par ^ 1);
        if (ds < 0) {
            atomicOr(&S->status, ST_CAPACITY);
            return;
        }
        float *dst = d.P[par ^ 1];
        // a cell-block slot takes the position in that block's cells (exact: u minus
        // an integer), a spill slot in metres
#pragma unroll
        for (int c = 0; c < 3; ++c) dst[c * SS + ds] = rr < CAP ? u[c] - (float)((nb[c] / BLK) * BLK) : x[c];
#pragma unroll
        for (int c = 0; c < 9; ++c) dst[(3 + c) * SS + ds] = F[c];
        d.T[par ^ 1][ds] = tag;
        if (d.G->k_cur + 1 == d.G->k_end) {
#pragma unroll
            for (int c = 0; c < 3; ++c) d.VC[c * SS + ds] = v[c];
#pragma unroll
            for (int c = 0; c < 9; ++c) d.VC[(3 + c) * SS + ds] = C[c];
        }
        cand = ds;
    }
    if (MODE != MODE_ITER) {
        float tip[3];
        if (MODE == MODE_PROLOGUE) {
            double t4[4], v4[4];
            pose_tip(d.kf + (long long)inst * MAX_KF * 5, I.nkf, d.G->k_next, t4, v4, (double)I.dt);
            tip[0] = (float)t4[0]; tip[1] = (float)t4[1]; tip[2] = (float)t4[2];
        } else {
            tip[0] = S->pose.tip_next[0]; tip[1] = S->pose.tip_next[1]; tip[2] = S->pose.tip_next[2];
        }
        // candidate distances are compared in cells, as in the cell blocks
        const float e0 = (x[0] - tip[0]) * I.inv_dx, e1 = (x[1] - tip[1]) * I.inv_dx, e2 = (x[2] - tip[2]) * I.inv_dx;
        const float dd = e0 * e0 + e1 * e1 + e2 * e2;
        const unsigned long long kk = ((unsigned long long)__float_as_uint(dd) << 32) | (unsigned int)cand;
        if (kk < *((volatile unsigned long long *)&S->e_key)) atomicMin(&S->e_key, kk);
    }
}

// Companion of every transfer launch (SPILL_CTAS CTAs of NT threads): the
// spill slots of every instance taking part in the pass, grid-strided.
template <int MODE>
__global__ void __launch_bounds__(NT) k_spill(Dev d)
{
    const int c = blockIdx.x;
    for (int inst = 0; inst < d.n_inst; ++inst) {
        InstState *S = d.ist + inst;
        int par;
        if (MODE == MODE_PROLOGUE) {
            if (!S->dirty) continue;
            par = d.G->par_next;
        } else {
            const int ph = S->phase;
            if (MODE == MODE_ITER && ph != 0) continue;
            if (MODE == MODE_COMMIT && ph != 1) continue;
            par = d.G->par_cur;
        }
        const Inst &I = d.inst[inst];
        const int nsp = min(S->nsp[par], I.spc);
        for (int sp = c * NT + (int)threadIdx.x; sp < nsp; sp += SPILL_CTAS * NT)
            spill_particle<MODE>(d, I, S, inst, par, I.sp0 + sp);
    }
}

// One CTA per cell block of 4x4x4 cells:
//   0. bulk-copy the block's x, F and tags into shared memory (TMA);
//   1. particle-parallel: G2P from the shared velocity window (Eqs. 6-7), the
//      F and x move on a commit pass (Eqs. 8-9), Kirchhoff stress (Eq. 4),
//      re-binning and the write of the moved state; the particle's P2G
//      coefficients replace its staged data, and a counting sort groups the
//      particles by cell (the particles of a cell share one 27-node stencil);
//   2. cell-parallel: the two threads of a cell accumulate its 27-node
//      stencil (Eqs. 1-4) in registers over all its particles, one thread
//      the channels (M, MG_x), the other (MG_y, MG_z); each warp (one z layer
//      of cells) then adds its stencils into its own node slab in 27
//      warp-synchronous offset rounds;
//   3. the slabs are summed per node and go to the grid with one vector
//      atomic per touched node.
template <int MODE>
__global__ void __launch_bounds__(NT, 5) k_transfer(Dev d, int block_offset)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    TransferSmem &sm = *reinterpret_cast<TransferSmem *>(smem_raw);

    const int b = block_offset + blockIdx.x;
    const int inst = d.blk_inst[b];
    InstState *S = d.ist + inst;
    int par;
    if (MODE == MODE_PROLOGUE) {
        if (!S->dirty) return;
        par = d.G->par_next;
    } else {
        const int ph = S->phase;
        if (MODE == MODE_ITER && ph != 0) return;
        if (MODE == MODE_COMMIT && ph != 1) return;
        par = d.G->par_cur;
    }
    const bool moves = MODE == MODE_COMMIT;
    const bool cands = MODE != MODE_ITER;
    const int count = min(d.cnt[par][b], CAP);          // an overflowed block was latched as an error
    if (count == 0) return;                             // no particles: no P2G, no moves, no candidate
    // x has not moved since the first repeat pass of this substep, which
    // stored its cell sort: the later repeat passes load it instead of sorting
    const bool reuse = MODE == MODE_ITER && S->pass >= 2;
    unsigned short *sortc = d.sortc + (long long)b * SORTC;

    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const long long SS = d.S;
    const long long slot0 = (long long)b * CAP;
    static_assert(sizeof(Inst) % 4 == 0 && sizeof(Inst) / 4 <= NT, "Inst is copied one word per thread");
    if (tid < (int)(sizeof(Inst) / 4))
        reinterpret_cast<int *>(&sm.inst)[tid] = reinterpret_cast<const int *>(d.inst + inst)[tid];

    // 0. bulk copies of the particle arrays (16-byte multiples; the slack is inside the block's slots)
    if (tid == 0) {
        mbar_init(&sm.bar, 1);
        if (count > 0) {
            const uint32_t bytes = (uint32_t)(((count + 3) & ~3) * 4);
            mbar_expect_tx(&sm.bar, 13u * bytes + (reuse ? (uint32_t)(SORTC * 2) : 0u));
            const float *src = d.P[par];
            for (int c = 0; c < 12; ++c) bulk_load(sm.P[c], src + c * SS + slot0, bytes, &sm.bar);
            bulk_load(sm.P[12], d.T[par] + slot0, bytes, &sm.bar);
            if (reuse) {
                bulk_load(sm.idx, sortc, CAP * 2, &sm.bar);
                bulk_load(sm.P[14], sortc + CAP, 2 * NCELL * 2, &sm.bar);   // row 14 is free until phase 1
            }
        }
        if (MODE == MODE_PROLOGUE) {
            double t4[4], v4[4];
            const Inst &Ig = d.inst[inst];
            pose_tip(d.kf + (long long)inst * MAX_KF * 5, Ig.nkf, d.G->k_next, t4, v4, (double)Ig.dt);
            sm.tip[0] = (float)t4[0]; sm.tip[1] = (float)t4[1]; sm.tip[2] = (float)t4[2];
        } else {
            sm.tip[0] = S->pose.tip_next[0]; sm.tip[1] = S->pose.tip_next[1]; sm.tip[2] = S->pose.tip_next[2];
        }
    }
    if (tid < NCELL) sm.ccount[tid] = 0;
    __syncthreads();
    const Inst &I = sm.inst;
    const int lb = b - I.block0;
    const int gx0 = (lb % I.nbx) * BLK, gy0 = ((lb / I.nbx) % I.nby) * BLK, gz0 = (lb / (I.nbx * I.nby)) * BLK;
    const float inv_dx = I.inv_dx, dt = I.dt;
    if (MODE != MODE_PROLOGUE) {
        for (int t = tid; t < GV * GV * GV; t += NT) {
            const int lx = t % GV, ly = (t / GV) % GV, lz = t / (GV * GV);
            const int ax = gx0 + lx, ay = gy0 + ly, az = gz0 + lz;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (ax < I.nx && ay < I.ny && az < I.nz) v = d.vel[node_of(I, ax, ay, az)];
            v.w = v.z;                                   // (V_x, V_y, V_z, V_z): see g2p_window
            sm.V[t] = v;
        }
    }
    const bool got = count == 0 || mbar_wait_bounded(&sm.bar, 0);
    if (!__syncthreads_and(got)) {
        // the run is reported as failed; before the CTA releases its shared
        // memory, wait (again bounded) for the copies still in flight
        if (tid == 0) {
            atomic_or_status(S, ST_TIMEOUT);
            mbar_wait_bounded(&sm.bar, 0);
        }
        return;
    }

    // 0b. counting sort of the staged particles by the cell of their staged
    //     position; phase 1 then runs in cell order, so that the lanes of a
    //     cell read the same window nodes in the G2P
    unsigned int err = 0;
    if (reuse) {
        const unsigned short *st = reinterpret_cast<const unsigned short *>(sm.P[14]);
        if (tid < NCELL) {
            sm.ccount[tid] = st[tid];
            sm.coff[tid] = st[NCELL + tid];
        }
        __syncthreads();
    } else {
        for (int r = tid; r < count; r += NT) {
            // staged positions are block-relative cells: the base node is the cell in the block
            int lx, ly, lz;
            float ff, ww[3];
            bspline_cells(sm.P[0][r], lx, ff, ww);
            bspline_cells(sm.P[1][r], ly, ff, ww);
            bspline_cells(sm.P[2][r], lz, ff, ww);
            int e = -1;
            if (lx < 0 || ly < 0 || lz < 0 || lx >= BLK || ly >= BLK || lz >= BLK) {
                err |= ST_DOMAIN;
            } else {
                const int c = (lz * BLK + ly) * BLK + lx;
                e = c | atomicAdd(&sm.ccount[c], 1) << 6;
            }
            reinterpret_cast<int *>(sm.P[13])[r] = e;
        }
        __syncthreads();
        if (tid < 32) {                                  // exclusive scan of the 64 cell counts
            const int a0 = sm.ccount[2 * tid], a1 = sm.ccount[2 * tid + 1];
            int incl = a0 + a1;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, o);
                if (tid >= o) incl += y;
            }
            const int excl = incl - a0 - a1;
            sm.coff[2 * tid] = excl;
            sm.coff[2 * tid + 1] = excl + a0;
        }
        __syncthreads();
        for (int r = tid; r < count; r += NT) {
            const int e = reinterpret_cast<const int *>(sm.P[13])[r];
            if (e >= 0) sm.idx[sm.coff[e & 63] + (e >> 6)] = (unsigned short)r;
        }
        __syncthreads();
        if (MODE == MODE_ITER) {
            // the first repeat pass of the substep keeps the sort for the others
            const int ns = sm.coff[NCELL - 1] + sm.ccount[NCELL - 1];
            for (int i = tid; i < ns; i += NT) sortc[i] = sm.idx[i];
            if (tid < NCELL) {
                sortc[CAP + tid] = (unsigned short)sm.ccount[tid];
                sortc[CAP + NCELL + tid] = (unsigned short)sm.coff[tid];
            }
        }
    }
    // (a stored sort holds indices below the count of the pass that made it)
    const int nsorted = min(sm.coff[NCELL - 1] + sm.ccount[NCELL - 1], count);

    // 1. particle-parallel pass (in cell order)
    // the next tip in this block's cells (candidate distances are compared in cells)
    const float tip0 = box_cells(sm.tip[0], inv_dx, I.ox) - (float)gx0;
    const float tip1 = box_cells(sm.tip[1], inv_dx, I.oy) - (float)gy0;
    const float tip2 = box_cells(sm.tip[2], inv_dx, I.oz) - (float)gz0;
    const float dtdx = dt * inv_dx;                 // the move in cells per unit velocity
    float *dst = d.P[par ^ 1];
    uint32_t *dstT = d.T[par ^ 1];
    int *cntDst = d.cnt[par ^ 1];
    const bool store_vc = moves && (d.G->k_cur + 1 == d.G->k_end);
    unsigned long long best = ~0ull;
    for (int s0 = 0; s0 < count; s0 += NT) {
        bool valid = s0 + tid < nsorted;
        const int r = valid ? sm.idx[s0 + tid] : 0;
        float x[3], F[9], v[3] = {0.f, 0.f, 0.f}, C[9];
        uint32_t tag = 0;
        int cl = 255;
        float f[3];                 // fractional offset of the staged position (reused when x stays)
        int bx = 0, by = 0, bz = 0;
        if (valid) {
            float w[3][3];
            bspline_cells(sm.P[0][r], bx, f[0], w[0]);
            bspline_cells(sm.P[1][r], by, f[1], w[1]);
            bspline_cells(sm.P[2][r], bz, f[2], w[2]);
            const int lx = bx, ly = by, lz = bz;
            if (lx < 0 || ly < 0 || lz < 0 || lx >= BLK || ly >= BLK || lz >= BLK) {
                err |= ST_DOMAIN;
                valid = false;
            } else {
                cl = (lz * BLK + ly) * BLK + lx;
                if (MODE == MODE_PROLOGUE) {
                    const long long slot = slot0 + r;
#pragma unroll
                    for (int c = 0; c < 3; ++c) v[c] = d.VC[c * SS + slot];
#pragma unroll
                    for (int c = 0; c < 9; ++c) C[c] = d.VC[(3 + c) * SS + slot];
                } else {
                    // G2P: v = sum w V (Eq. 6), C = 4/dx^2 sum w V (x_i - x_p)^T (Eq. 7)
                    g2p_window(sm.V, lx, ly, lz, w, f, v, C);
                    const float s4 = 4.f * inv_dx;   // (4/dx^2) * dx: d above is in cells
#pragma unroll
                    for (int c = 0; c < 9; ++c) C[c] *= s4;
                }
            }
        }
        // x, F and the tag are read from shared memory only now, so that they
        // are not held in registers across the G2P
        asm volatile("" ::: "memory");
        if (valid) {
#pragma unroll
            for (int c = 0; c < 3; ++c) x[c] = sm.P[c][r];
#pragma unroll
            for (int c = 0; c < 9; ++c) F[c] = sm.P[3 + c][r];
            tag = __float_as_uint(sm.P[12][r]);
            if (MODE != MODE_PROLOGUE && (tag & TAG_BOTTOM) && I.base_mode != BASE_FREE) v[2] = 0.f;   // Algorithm 1
        }
        if (valid && moves) {
            // F <- (I + dt C) F (Eq. 8); x <- x + dt v (Eq. 9)
            float Fn[9];
#pragma unroll
            for (int rr = 0; rr < 3; ++rr)
#pragma unroll
                for (int cc = 0; cc < 3; ++cc)
                    Fn[rr * 3 + cc] = F[rr * 3 + cc] + dt * (C[rr * 3] * F[cc] + C[rr * 3 + 1] * F[3 + cc] +
                                                             C[rr * 3 + 2] * F[6 + cc]);
#pragma unroll
            for (int c = 0; c < 9; ++c) F[c] = Fn[c];
#pragma unroll
            for (int c = 0; c < 3; ++c) x[c] += dtdx * v[c];
        }
        int nb[3] = {0, 0, 0};
        long long cand_slot = moves ? -1 : slot0 + r;   // commit: set where the particle is written
        if (valid) {
            // stress (S_p of Eq. 4) and the P2G coefficients of the state that enters P2G
            float tau[9];
            const float J = kirchhoff(F, I.mu, I.lam, tau);
            if (!(J > 0.f) || !isfinite(J) || !isfinite(x[0]) || !isfinite(x[1]) || !isfinite(x[2])) {
                err |= ST_NUMERIC;
                valid = false;
            } else {
                // the position that enters P2G: moved on a commit pass, else the staged one
                float nf[3];
                if (moves) {
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        float wt[3];
                        bspline_cells(x[a], nb[a], nf[a], wt);
                    }
                } else {
                    nb[0] = bx; nb[1] = by; nb[2] = bz;
                    nf[0] = f[0]; nf[1] = f[1]; nf[2] = f[2];
                }
                nb[0] += gx0; nb[1] += gy0; nb[2] += gz0;             // box index of the new base node
                const int wx = nb[0] - (gx0 - 1), wy = nb[1] - (gy0 - 1), wz = nb[2] - (gz0 - 1);
                if (nb[0] < 0 || nb[1] < 0 || nb[2] < 0 || nb[0] + 2 >= I.nx || nb[1] + 2 >= I.ny ||
                    nb[2] + 2 >= I.nz || wx < 0 || wy < 0 || wz < 0 || wx + 2 >= GA || wy + 2 >= GA ||
                    wz + 2 >= GA) {
                    err |= ST_DOMAIN;
                    valid = false;
                } else {
                    // P2G: M += w m (Eq. 1); MG += w (m v + m C d) - 4 dt/dx^2 V0 w tau d (Eqs. 2-4);
                    // Q carries one cell of d so that d can be counted in cells
                    float Q[9];
#pragma unroll
                    for (int c = 0; c < 9; ++c) Q[c] = (I.mp * C[c] + I.kME * tau[c]) * I.dx;
                    const float mv[3] = {I.mp * v[0], I.mp * v[1], I.mp * v[2]};
                    const bool stays = wx == (cl & 3) + 1 && wy == ((cl >> 2) & 3) + 1 && wz == (cl >> 4) + 1;
                    if (stays) {
#pragma unroll
                        for (int c = 0; c < 9; ++c) sm.P[c][r] = Q[c];
#pragma unroll
                        for (int c = 0; c < 3; ++c) sm.P[9 + c][r] = mv[c];
#pragma unroll
                        for (int c = 0; c < 3; ++c) sm.P[12 + c][r] = nf[c];
                    } else {
                        float nw[3][3];
#pragma unroll
                        for (int a = 0; a < 3; ++a) {
                            const float u = 1.5f - nf[a], bq = nf[a] - 1.f, cq = nf[a] - 0.5f;
                            nw[a][0] = 0.5f * u * u; nw[a][1] = 0.75f - bq * bq; nw[a][2] = 0.5f * cq * cq;
                        }
                        p2g_global(d.acc, I, nb[0], nb[1], nb[2], nw, nf, Q, mv, I.mp);
                        cl = 255;
                    }
                }
            }
        }
        if (!valid) cl = 255;
        // particles that left their cell (or failed) are taken out of the cell-parallel P2G
        if (s0 + tid < nsorted && cl == 255) sm.P[12][r] = -1.f;
        if (moves) {
            // re-bin into the cell block of the new position: warp-aggregated slot claims
            unsigned int key = 0xffffffffu;
            if (valid) key = (unsigned int)(I.block0 + ((nb[2] / BLK) * I.nby + (nb[1] / BLK)) * I.nbx + (nb[0] / BLK));
            const unsigned int peers = __match_any_sync(0xffffffffu, key);
            const int leader = __ffs(peers) - 1;
            const int rank = __popc(peers & ((1u << lane) - 1u));
            int basepos = 0;
            if (lane == leader && key != 0xffffffffu) basepos = atomicAdd(&cntDst[key], __popc(peers));
            basepos = __shfl_sync(0xffffffffu, basepos, leader);
            if (valid) {
                const int rr = basepos + rank;
                // a full block sends the particle to its instance's spill slots
                const long long ds = rr < CAP ? (long long)key * CAP + rr : claim_spill(d, I, inst, par ^ 1);
                if (ds < 0) {
                    err |= ST_CAPACITY;
                } else {
                    cand_slot = ds;
                    // into the destination block's cells, or metres in a spill slot.  The
                    // shift by -4 or 0 is exact; a shift by +4 of a q just below 0.5 can round
                    // up to 4.5, so the result is kept below 4.5 (one ulp at most)
                    const int g0[3] = {gx0, gy0, gz0}, oo[3] = {I.ox, I.oy, I.oz};
                    const float q_hi = __int_as_float(0x408fffff);       // the float below 4.5
#pragma unroll
                    for (int c = 0; c < 3; ++c)
                        dst[c * SS + ds] = rr < CAP ? fminf(x[c] - (float)((nb[c] / BLK) * BLK - g0[c]), q_hi)
                                                    : block_to_metres(x[c], g0[c], oo[c], I.dx);
#pragma unroll
                    for (int c = 0; c < 9; ++c) dst[(3 + c) * SS + ds] = F[c];
                    dstT[ds] = tag;
                    if (store_vc) {
#pragma unroll
                        for (int c = 0; c < 3; ++c) d.VC[c * SS + ds] = v[c];
#pragma unroll
                        for (int c = 0; c < 9; ++c) d.VC[(3 + c) * SS + ds] = C[c];
                    }
                }
            }
        }
        if (cands && valid && cand_slot >= 0) {
            const float e0 = x[0] - tip0, e1 = x[1] - tip1, e2 = x[2] - tip2;
            const float dd = e0 * e0 + e1 * e1 + e2 * e2;
            const unsigned long long kk = ((unsigned long long)__float_as_uint(dd) << 32) | (unsigned int)cand_slot;
            if (kk < best) best = kk;
        }
    }
    if (err) atomic_or_status(S, err);
    __syncthreads();

    // 2. cell-parallel P2G: the two threads of a cell (adjacent lanes) each
    //    take two of the four channels over all the cell's particles; a
    //    channel's value at node (i, j, k) is w (a + q . d) with (a, q) = (1, 0)
    //    for M and (m v_r, row r of Q) for MG_r, d = (i - f0, j - f1, k - f2)
    {
        const int cl = tid >> 1, h = tid & 1;
        const int clx = cl & 3, cly = (cl >> 2) & 3;
        const int ncl = sm.ccount[cl], off = sm.coff[cl];
        const float2 z2 = make_float2(0.f, 0.f);
        float2 acc[27];
#pragma unroll
        for (int o = 0; o < 27; ++o) acc[o] = z2;
        const float *rowA1 = sm.P[9 + 2 * h], *rowQ1 = sm.P[6 * h];
        for (int it = 0; it < ncl; ++it) {
            const int r = sm.idx[off + it];
            const float f0 = sm.P[12][r];
            if (f0 < 0.f) continue;                         // left its cell: P2G done with global atomics
            const float f1 = sm.P[13][r], f2 = sm.P[14][r];
            const float a1 = rowA1[r], q10 = rowQ1[r], q11 = rowQ1[CAP + r], q12 = rowQ1[2 * CAP + r];
            float a0 = 1.f, q00 = 0.f, q01 = 0.f, q02 = 0.f;
            if (h) { a0 = sm.P[10][r]; q00 = sm.P[3][r]; q01 = sm.P[4][r]; q02 = sm.P[5][r]; }
            float wx[3], wy[3], wz[3];
            {
                float a = 1.5f - f0, bb = f0 - 1.f, cc = f0 - 0.5f;
                wx[0] = 0.5f * a * a; wx[1] = 0.75f - bb * bb; wx[2] = 0.5f * cc * cc;
                a = 1.5f - f1; bb = f1 - 1.f; cc = f1 - 0.5f;
                wy[0] = 0.5f * a * a; wy[1] = 0.75f - bb * bb; wy[2] = 0.5f * cc * cc;
                a = 1.5f - f2; bb = f2 - 1.f; cc = f2 - 0.5f;
                wz[0] = 0.5f * a * a; wz[1] = 0.75f - bb * bb; wz[2] = 0.5f * cc * cc;
            }
            // value = w_i w_j w_k (A(i) + Y(j)) + w_i w_j (w_k Z(k)): the x and y
            // parts ride on the (i, j) product, the z part is folded into H(k)
            float2 A2[3], Y2[3], H2[3], wz2[3];
#pragma unroll
            for (int o = 0; o < 3; ++o) {
                const float d0 = (float)o - f0, d1 = (float)o - f1, d2 = (float)o - f2;
                A2[o] = make_float2(fmaf(q00, d0, a0), fmaf(q10, d0, a1));
                Y2[o] = make_float2(q01 * d1, q11 * d1);
                H2[o] = make_float2(wz[o] * (q02 * d2), wz[o] * (q12 * d2));
                wz2[o] = dup2(wz[o]);
            }
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    const float2 wij = dup2(wx[i] * wy[j]);
                    const float2 G = fmul2(wij, fadd2(A2[i], Y2[j]));
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        const int o = (i * 3 + j) * 3 + k;
                        acc[o] = ffma2(G, wz2[k], acc[o]);
                        acc[o] = ffma2(wij, H2[k], acc[o]);
                    }
                }
        }
        // every warp has read its particles' rows: the rows now hold the slabs
        __syncthreads();
        float4 *slab = reinterpret_cast<float4 *>(&sm.P[0][0]) + (tid >> 5) * SLAB;
        for (int t = lane; t < SLAB; t += 32) slab[t] = make_float4(0.f, 0.f, 0.f, 0.f);
        __syncwarp();
        float2 *half2 = reinterpret_cast<float2 *>(slab) + h;
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j)
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    // within a round the 16 cells of the warp write 16 different nodes
                    const int o = (i * 3 + j) * 3 + k;
                    const int n = (k * SLY + cly + j) * SLX + clx + i;
                    half2[2 * n] = fadd2(half2[2 * n], acc[o]);
                    __syncwarp();
                }
    }
    __syncthreads();
    // 3. slabs -> grid: node plane z of the block window gets the slabs of the
    //    (up to three) cell layers below it; one vector atomic per touched node
    //    (M was accumulated per unit mass)
    {
        const float4 *slabs = reinterpret_cast<const float4 *>(&sm.P[0][0]);
        const float mp = I.mp;
        for (int t = tid; t < (BLK + 2) * (BLK + 2) * (BLK + 2); t += NT) {
            const int X = t % (BLK + 2), Y = (t / (BLK + 2)) % (BLK + 2), Z = t / ((BLK + 2) * (BLK + 2));
            float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
            const int w0 = Z >= 2 ? Z - 2 : 0, w1 = Z < BLK ? Z : BLK - 1;
            for (int w = w0; w <= w1; ++w) {
                const float4 q = slabs[w * SLAB + ((Z - w) * SLY + Y) * SLX + X];
                a.x += q.x; a.y += q.y; a.z += q.z; a.w += q.w;
            }
            if (a.x != 0.f) {
                const int ax = gx0 + X, ay = gy0 + Y, az = gz0 + Z;
                if (ax < I.nx && ay < I.ny && az < I.nz)
                    atomicAdd(&d.acc[node_of(I, ax, ay, az)], make_float4(a.x * mp, a.y, a.z, a.w));
            }
        }
    }
    if (cands) {
        // nearest particle to the next tip: CTA minimum, then one atomic per CTA that improves it
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long ok = __shfl_down_sync(0xffffffffu, best, o);
            if (ok < best) best = ok;
        }
        if (lane == 0) sm.key[tid >> 5] = best;
        __syncthreads();
        if (tid == 0) {
            unsigned long long m = sm.key[0];
            for (int a = 1; a < NT / 32; ++a)
                if (sm.key[a] < m) m = sm.key[a];
            if (m < *((volatile unsigned long long *)&S->e_key)) atomicMin(&S->e_key, m);
        }
    }
}

size_t transfer_smem_bytes() { return sizeof(TransferSmem); }
static_assert(offsetof(TransferSmem, idx) % 16 == 0 && (CAP * 2) % 16 == 0 && (2 * NCELL * 2) % 16 == 0 &&
                  (SORTC * 2) % 16 == 0,
              "bulk copies of the stored cell sort: 16-byte aligned, 16-byte multiples");

// ---------------------------------------------------------------- object particles

// P2G (Eqs. 1-3, no stress term) of the particle-represented indenter of
// instance inst0 + blockIdx.y, one thread per object particle: rigid, at the
// indenter pose of the state that enters this P2G (substep k for a repeat
// pass, k + 1 for a commit, the next substep for a prologue), each with the
// prescribed velocity v_lin + omega z x (x - c) and the affine field of that
// motion, C = omega [[0,-1,0],[1,0,0],[0,0,0]]; global vector atomics.
// Nodes outside the node box receive nothing.
template <int MODE>
__global__ void __launch_bounds__(256) k_object_p2g(Dev d, int inst0)
{
    const int inst = inst0 + blockIdx.y;
    const Inst &I = d.inst[inst];
    if ((long long)blockIdx.x * blockDim.x >= I.nobj) return;
    const InstState *S = d.ist + inst;
    if (MODE == MODE_PROLOGUE) {
        if (!S->dirty) return;
    } else {
        const int ph = S->phase;
        if (MODE == MODE_ITER && ph != 0) return;
        if (MODE == MODE_COMMIT && ph != 1) return;
    }
    __shared__ Pose sp;
    if (threadIdx.x == 0) {
        if (MODE == MODE_ITER) sp = S->pose;
        else pose_eval(I, d.kf + (long long)inst * MAX_KF * 5, MODE == MODE_COMMIT ? d.G->k_cur + 1 : d.G->k_next, sp);
    }
    __syncthreads();
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= I.nobj) return;
    const float4 ql = d.objq[I.obj0 + q];
    const float xw[3] = {sp.c[0] + sp.cs * ql.x - sp.sn * ql.y, sp.c[1] + sp.sn * ql.x + sp.cs * ql.y, sp.c[2] + ql.z};
    float vo[3];
    object_velocity(sp, xw, vo);
    int base[3];
    float f[3], w[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a) bspline(xw[a], I.inv_dx, base[a], f[a], w[a]);
    const float m = I.objm, om = sp.omega * I.dx;     // C d with d in cells: omega dx (-d_y, d_x, 0)
    for (int i = 0; i < 3; ++i) {
        const int ax = base[0] + i + I.ox;
        if (ax < 0 || ax >= I.nx) continue;
        for (int j = 0; j < 3; ++j) {
            const int ay = base[1] + j + I.oy;
            if (ay < 0 || ay >= I.ny) continue;
            const float dxc = (float)i - f[0], dyc = (float)j - f[1];
            const float u0 = vo[0] - om * dyc, u1 = vo[1] + om * dxc;
            for (int k = 0; k < 3; ++k) {
                const int az = base[2] + k + I.oz;
                if (az < 0 || az >= I.nz) continue;
                const float wm = w[0][i] * w[1][j] * w[2][k] * m;
                atomicAdd(&d.acc[node_of(I, ax, ay, az)], make_float4(wm, wm * u0, wm * u1, wm * vo[2]));
            }
        }
    }
}

// ---------------------------------------------------------------- staging <-> slots

__global__ void k_bin_staged(Dev d, int inst, int par)
{
    const Inst &I = d.inst[inst];
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= I.n_particles) return;
    const long long sid = I.id0 + t;
    float x[3] = {d.sx[sid * 3], d.sx[sid * 3 + 1], d.sx[sid * 3 + 2]};
    int ab[3];
    float u[3];
    const int nn[3] = {I.nx, I.ny, I.nz}, oo[3] = {I.ox, I.oy, I.oz};
    bool ok = isfinite(x[0]) && isfinite(x[1]) && isfinite(x[2]);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        float f, w[3];
        u[a] = box_cells(x[a], I.inv_dx, oo[a]);
        bspline_cells(u[a], ab[a], f, w);
        if (ab[a] < 0 || ab[a] + 2 >= nn[a]) ok = false;
    }
    const uint32_t tag = d.stag[sid];
    if ((tag & ID_MASK) >= (uint32_t)I.n_particles) ok = false;
    if (!ok) {
        atomic_or_status(d.ist + inst, ST_DOMAIN);
        return;
    }
    const int blk = I.block0 + ((ab[2] / BLK) * I.nby + ab[1] / BLK) * I.nbx + ab[0] / BLK;
    const int r = atomicAdd(&d.cnt[par][blk], 1);
    const long long slot = r < CAP ? (long long)blk * CAP + r : claim_spill(d, I, inst, par);
    if (slot < 0) {
        atomic_or_status(d.ist + inst, ST_CAPACITY);
        return;
    }
    const long long SS = d.S;
    float *P = d.P[par];
    // a cell-block slot holds the position in the block's cells, a spill slot metres
#pragma unroll
    for (int c = 0; c < 3; ++c) P[c * SS + slot] = r < CAP ? u[c] - (float)((ab[c] / BLK) * BLK) : x[c];
#pragma unroll
    for (int c = 0; c < 9; ++c) P[(3 + c) * SS + slot] = d.sF[sid * 9 + c];
    d.T[par][slot] = tag;
#pragma unroll
    for (int c = 0; c < 3; ++c) d.VC[c * SS + slot] = d.sv[sid * 3 + c];
#pragma unroll
    for (int c = 0; c < 9; ++c) d.VC[(3 + c) * SS + slot] = d.sC[sid * 9 + c];
}

__global__ void k_gather(Dev d, int inst, int par)
{
    const Inst &I = d.inst[inst];
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)I.nblocks * CAP + I.spc) return;
    const long long slot = inst_slot(d, I, inst, par, t);
    if (slot < 0) return;
    const long long SS = d.S;
    const uint32_t tag = d.T[par][slot];
    const uint32_t id = tag & ID_MASK;
    if (id >= (uint32_t)I.n_particles) {
        atomic_or_status(d.ist + inst, ST_DOMAIN);
        return;
    }
    const long long sid = I.id0 + id;
    const float *P = d.P[par];
    float x[3];
    slot_metres(d, I, par, t, slot, x);
#pragma unroll
    for (int c = 0; c < 3; ++c) d.sx[sid * 3 + c] = x[c];
#pragma unroll
    for (int c = 0; c < 9; ++c) d.sF[sid * 9 + c] = P[(3 + c) * SS + slot];
#pragma unroll
    for (int c = 0; c < 3; ++c) d.sv[sid * 3 + c] = d.VC[c * SS + slot];
#pragma unroll
    for (int c = 0; c < 9; ++c) d.sC[sid * 9 + c] = d.VC[(3 + c) * SS + slot];
    d.stag[sid] = tag;
}

__global__ void k_pick(Dev d, int inst, const int *ids, int m, float *out)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m) return;
    const Inst &I = d.inst[inst];
    const int id = ids[t];
    if (id < 0 || id >= I.n_particles) {
        out[t * 3] = out[t * 3 + 1] = out[t * 3 + 2] = __int_as_float(0x7fc00000);
        return;
    }
    const long long sid = I.id0 + id;
    out[t * 3] = d.sx[sid * 3];
    out[t * 3 + 1] = d.sx[sid * 3 + 1];
    out[t * 3 + 2] = d.sx[sid * 3 + 2];
}

// ---------------------------------------------------------------- surface readout

__device__ __forceinline__ float bspline_kernel(float t)
{
    t = fabsf(t);
    if (t < 0.5f) return 0.75f - t * t;
    if (t < 1.5f) { const float a = 1.5f - t; return 0.5f * a * a; }
    return 0.f;
}

__global__ void k_surface_splat(Dev d, int inst, int par, float *num, float *den, int W, int H,
                                float inv_pitch)
{
    const Inst &I = d.inst[inst];
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)I.nblocks * CAP + I.spc) return;
    const long long slot = inst_slot(d, I, inst, par, t);
    if (slot < 0) return;
    if (!(d.T[par][slot] & TAG_TOP)) return;
    float xm[3];
    slot_metres(d, I, par, t, slot, xm);
    const float x = xm[0], y = xm[1], z = xm[2];
    const float px = x * inv_pitch - 0.5f, py = y * inv_pitch - 0.5f;
    const int u0 = (int)floorf(px) - 1, v0 = (int)floorf(py) - 1;
    for (int bb = v0; bb <= v0 + 3; ++bb) {
        if (bb < 0 || bb >= H) continue;
        const float wy = bspline_kernel(py - (float)bb);
        if (wy == 0.f) continue;
        for (int a = u0; a <= u0 + 3; ++a) {
            if (a < 0 || a >= W) continue;
            const float w = bspline_kernel(px - (float)a) * wy;
            if (w == 0.f) continue;
            atomicAdd(num + (long long)bb * W + a, w * z);
            atomicAdd(den + (long long)bb * W + a, w);
        }
    }
}

__global__ void k_surface_height(const float *num, const float *den, float *h, int WH, float h_empty)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < WH) h[t] = den[t] > 0.f ? num[t] / den[t] : h_empty;
}

__global__ void k_surface_normal(const float *h, float *nrm, int W, int H, float pitch)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= W * H) return;
    const int a = t % W, b = t / W;
    const int al = a > 0 ? a - 1 : a, ar = a < W - 1 ? a + 1 : a;
    const int bl = b > 0 ? b - 1 : b, br = b < H - 1 ? b + 1 : b;
    const float hx = (h[b * W + ar] - h[b * W + al]) / ((float)(ar - al) * pitch);
    const float hy = (h[br * W + a] - h[bl * W + a]) / ((float)(br - bl) * pitch);
    const float L = rsqrtf(hx * hx + hy * hy + 1.f);
    nrm[t * 3] = -hx * L;
    nrm[t * 3 + 1] = -hy * L;
    nrm[t * 3 + 2] = L;
}

// Displacement u = x - X of the surface particles, splatted with the 2-D
// quadratic B-spline at their reference positions X (Lagrangian field).
__global__ void k_surface_disp(Dev d, int inst, int par, const float *__restrict__ xref, float *acc, int W,
                               int H, float inv_pitch)
{
    const Inst &I = d.inst[inst];
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)I.nblocks * CAP + I.spc) return;
    const long long slot = inst_slot(d, I, inst, par, t);
    if (slot < 0) return;
    const uint32_t tag = d.T[par][slot];
    if (!(tag & TAG_TOP)) return;
    const uint32_t id = tag & ID_MASK;
    if (id >= (uint32_t)I.n_particles) return;
    float xm[3];
    slot_metres(d, I, par, t, slot, xm);
    const float X = xref[(long long)id * 3], Y = xref[(long long)id * 3 + 1], Z = xref[(long long)id * 3 + 2];
    const float ux = xm[0] - X, uy = xm[1] - Y, uz = xm[2] - Z;
    const float px = X * inv_pitch - 0.5f, py = Y * inv_pitch - 0.5f;
    const int u0 = (int)floorf(px) - 1, v0 = (int)floorf(py) - 1;
    for (int bb = v0; bb <= v0 + 3; ++bb) {
        if (bb < 0 || bb >= H) continue;
        const float wy = bspline_kernel(py - (float)bb);
        if (wy == 0.f) continue;
        for (int a = u0; a <= u0 + 3; ++a) {
            if (a < 0 || a >= W) continue;
            const float w = bspline_kernel(px - (float)a) * wy;
            if (w == 0.f) continue;
            float *c = acc + ((long long)bb * W + a) * 4;
            atomicAdd(c, w * ux);
            atomicAdd(c + 1, w * uy);
            atomicAdd(c + 2, w * uz);
            atomicAdd(c + 3, w);
        }
    }
}

__global__ void k_surface_disp_finish(const float *acc, float *u, int WH)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= WH) return;
    const float w = acc[t * 4 + 3];
    const float iw = w > 0.f ? 1.f / w : 0.f;
    u[t * 3] = acc[t * 4] * iw;
    u[t * 3 + 1] = acc[t * 4 + 1] * iw;
    u[t * 3 + 2] = acc[t * 4 + 2] * iw;
}

// Height of the indenter's underside above the gel top at the current pose
// (the pose of the next substep), by sphere tracing the SDF straight up each
// pixel column from gel top - clip; columns that miss the shape read +clip,
// heights are clamped to [-clip, clip].
__global__ void k_indenter_height(Dev d, int inst, float *h, int W, int H, float pitch, float clip)
{
    __shared__ Pose P;
    const Inst &I = d.inst[inst];
    if (threadIdx.x == 0) pose_eval(I, d.kf + (long long)inst * MAX_KF * 5, d.G->k_next, P);
    __syncthreads();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= W * H) return;
    const float xw0 = ((t % W) + 0.5f) * pitch, xw1 = ((t / W) + 0.5f) * pitch;
    if (I.ind_kind == K_NONE) { h[t] = clip; return; }
    const int *perm = d.perm + inst * 256;
    float z = I.H - clip;
    float out = clip;
    for (int it = 0; it < 128; ++it) {
        const float xw[3] = {xw0, xw1, z};
        float n[3];
        const float phi = sdf_world(I, perm, P, xw, n);
        if (phi < 1e-4f * I.dx) { out = z - I.H; break; }
        z += 0.8f * phi;
        if (z > I.H + clip) break;
    }
    h[t] = fminf(fmaxf(out, -clip), clip);
}

// ---------------------------------------------------------------- launchers

static inline unsigned int cdiv(long long a, long long b) { return (unsigned int)((a + b - 1) / b); }

void launch_round_begin(const Dev &d, cudaStream_t s)
{
    k_round_begin<<<round_begin_ctas(d), 256, 0, s>>>(d);
}

// threads for one per instance and about eight counters to clear each
unsigned int round_begin_ctas(const Dev &d)
{
    return (unsigned int)std::max(cdiv(d.n_inst, 256), std::min(cdiv(d.n_blocks, 256 * 8), 1024u));
}
void launch_set_end(const Dev &d, long long n, cudaStream_t s) { k_set_end<<<1, 1, 0, s>>>(d, n); }

void grid_launch_shape(const Dev &d, long long max_nodes, int threads, int flat, dim3 &grid, dim3 &block)
{
    block = dim3(threads);           // CTA 0 is the check CTA
    if (flat) grid = dim3((unsigned int)(d.n_gchunk * 128 / threads) + 1);
    else grid = dim3((unsigned int)cdiv(max_nodes, threads) + 1, d.n_inst);
}

void launch_grid(const Dev &d, long long max_nodes, int threads, int flat, cudaStream_t s)
{
    dim3 g, b;
    grid_launch_shape(d, max_nodes, threads, flat, g, b);
    if (flat) k_grid_flat<<<g, b, 0, s>>>(d, 0, 0);
    else k_grid<<<g, b, 0, s>>>(d, 0, 0);
}

// the transfer kernels take the largest shared-memory carveout, so that five
// CTAs of 44 KB fit on an SM
template <int MODE>
static cudaError_t setup_transfer(int bytes)
{
    cudaError_t e = cudaFuncSetAttribute(k_transfer<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_transfer<MODE>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 cudaSharedmemCarveoutMaxShared);
    return e;
}

cudaError_t setup_kernels()
{
    const int bytes = (int)sizeof(TransferSmem);
    cudaError_t e = setup_transfer<MODE_PROLOGUE>(bytes);
    if (e == cudaSuccess) e = setup_transfer<MODE_ITER>(bytes);
    if (e == cudaSuccess) e = setup_transfer<MODE_COMMIT>(bytes);
    return e;
}

int block_slots() { return CAP; }

void launch_object_p2g(const Dev &d, int mode, int inst0, int rows, int max_obj, cudaStream_t s)
{
    if (max_obj <= 0 || rows <= 0) return;
    const dim3 g(cdiv(max_obj, 256), rows);
    if (mode == MODE_PROLOGUE) k_object_p2g<MODE_PROLOGUE><<<g, 256, 0, s>>>(d, inst0);
    else if (mode == MODE_ITER) k_object_p2g<MODE_ITER><<<g, 256, 0, s>>>(d, inst0);
    else k_object_p2g<MODE_COMMIT><<<g, 256, 0, s>>>(d, inst0);
}

void *fn_object_p2g(int mode)
{
    return mode == MODE_PROLOGUE ? (void *)k_object_p2g<MODE_PROLOGUE>
                                 : mode == MODE_ITER ? (void *)k_object_p2g<MODE_ITER> : (void *)k_object_p2g<MODE_COMMIT>;
}

void launch_transfer(const Dev &d, int mode, int block_offset, int nblocks, cudaStream_t s)
{
    if (nblocks <= 0) return;
    const size_t sh = sizeof(TransferSmem);
    if (mode == MODE_PROLOGUE) {
        k_transfer<MODE_PROLOGUE><<<nblocks, NT, sh, s>>>(d, block_offset);
        k_spill<MODE_PROLOGUE><<<SPILL_CTAS, NT, 0, s>>>(d);
    } else if (mode == MODE_ITER) {
        k_transfer<MODE_ITER><<<nblocks, NT, sh, s>>>(d, block_offset);
        k_spill<MODE_ITER><<<SPILL_CTAS, NT, 0, s>>>(d);
    } else {
        k_transfer<MODE_COMMIT><<<nblocks, NT, sh, s>>>(d, block_offset);
        k_spill<MODE_COMMIT><<<SPILL_CTAS, NT, 0, s>>>(d);
    }
}

void launch_bin_staged(const Dev &d, int inst, int n, int par, cudaStream_t s)
{
    k_bin_staged<<<cdiv(n, 256), 256, 0, s>>>(d, inst, par);
}

void launch_gather(const Dev &d, int inst, long long positions, int par, cudaStream_t s)
{
    k_gather<<<cdiv(positions, 256), 256, 0, s>>>(d, inst, par);
}

void launch_pick(const Dev &d, int inst, const int *ids, int m, float *out, cudaStream_t s)
{
    k_pick<<<cdiv(m, 128), 128, 0, s>>>(d, inst, ids, m, out);
}

void launch_surface(const Dev &d, int inst, long long positions, int par, float *num, float *den, float *h,
                    float *nrm, int W, int H, float pitch, float h_empty, cudaStream_t s)
{
    cudaMemsetAsync(num, 0, sizeof(float) * (size_t)W * H, s);
    cudaMemsetAsync(den, 0, sizeof(float) * (size_t)W * H, s);
    k_surface_splat<<<cdiv(positions, 256), 256, 0, s>>>(d, inst, par, num, den, W, H, 1.f / pitch);
    k_surface_height<<<cdiv((long long)W * H, 256), 256, 0, s>>>(num, den, h, W * H, h_empty);
    k_surface_normal<<<cdiv((long long)W * H, 256), 256, 0, s>>>(h, nrm, W, H, pitch);
}

void launch_surface_disp(const Dev &d, int inst, long long positions, int par, const float *xref, float *acc,
                         float *u, int W, int H, float pitch, cudaStream_t s)
{
    cudaMemsetAsync(acc, 0, sizeof(float) * 4 * (size_t)W * H, s);
    k_surface_disp<<<cdiv(positions, 256), 256, 0, s>>>(d, inst, par, xref, acc, W, H, 1.f / pitch);
    k_surface_disp_finish<<<cdiv((long long)W * H, 256), 256, 0, s>>>(acc, u, W * H);
}

void launch_indenter_height(const Dev &d, int inst, float *h, int W, int H, float pitch, float clip, cudaStream_t s)
{
    k_indenter_height<<<cdiv((long long)W * H, 128), 128, 0, s>>>(d, inst, h, W, H, pitch, clip);
}

// kernel handles for graph construction
void *fn_round_begin() { return (void *)k_round_begin; }
void *fn_grid(int flat) { return flat ? (void *)k_grid_flat : (void *)k_grid; }
void *fn_transfer(int mode)
{
    if (mode == MODE_PROLOGUE) return (void *)k_transfer<MODE_PROLOGUE>;
    if (mode == MODE_ITER) return (void *)k_transfer<MODE_ITER>;
    return (void *)k_transfer<MODE_COMMIT>;
}
void *fn_spill(int mode)
{
    if (mode == MODE_PROLOGUE) return (void *)k_spill<MODE_PROLOGUE>;
    if (mode == MODE_ITER) return (void *)k_spill<MODE_ITER>;
    return (void *)k_spill<MODE_COMMIT>;
}

}  // namespace tsim
