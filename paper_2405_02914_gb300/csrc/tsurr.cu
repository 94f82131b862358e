// tsurr.cu -- learned surface surrogate: 3x3 convolutions as implicit GEMMs
// on the BF16 tensor cores with FP32 accumulation.  The forward
// (k_conv_fwd_tc), the data gradient (k_conv_dgrad_tc) and the weight
// gradient (k_conv_wgrad_tc) run on tcgen05.mma with TMEM accumulators, fed
// by TMA tensor copies; weight gradients of output widths that are not a
// multiple of 16 (frames below 128 x 128) keep an mma.sync m16n8k16 kernel
// (k_conv_wgrad).  Fused bias / skip / ReLU epilogues, nearest upsampling
// folded into the operand addressing, masked loss with a residual indicator
// channel, Adam.  Architecture and loss: include/tsurr.h.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>   // CUtensorMap and the cuTensorMapEncodeTiled signature (entry point fetched at run time)

#include <cmath>
#include <cstdint>
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/tsim.h"
#include "../../include/tsurr.h"

void tsim_record_error(const std::string &msg);   // tsim_api.cu: the text tsim_last_error returns

namespace {

typedef __nv_bfloat16 bf16;

constexpr int BM = 64, BN = 64, BK = 16, GT = 128;   // CTA tile and threads (4 warps of 32x32)
constexpr int NL = 9;
constexpr int CIN_PAD = 16, COUT_PAD = 16;

__device__ __forceinline__ float bf2f(bf16 v) { return __bfloat162float(v); }
__device__ __forceinline__ bf16 f2bf(float v) { return __float2bfloat16_rn(v); }

__device__ __forceinline__ void mma16816(float c[4], const uint32_t a[4], const uint32_t b[2])
{
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                 "{%0,%1,%2,%3};"
                 : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// One BK = 16 step of the warp's 32x32 tile.  A is stored [m][k] and B [n][k]
// in shared memory with a row stride of S 32-bit words (two BF16 each).
template <int S>
__device__ __forceinline__ void mma_tile(const uint32_t *A32, const uint32_t *B32, float acc[2][4][4], int wm,
                                         int wn, int lane)
{
    const int gid = lane >> 2, tig = lane & 3;
    uint32_t a[2][4], b[4][2];
#pragma unroll
    for (int mi = 0; mi < 2; ++mi) {
        const int r = wm * 32 + mi * 16 + gid;
        a[mi][0] = A32[r * S + tig];
        a[mi][1] = A32[(r + 8) * S + tig];
        a[mi][2] = A32[r * S + 4 + tig];
        a[mi][3] = A32[(r + 8) * S + 4 + tig];
    }
#pragma unroll
    for (int ni = 0; ni < 4; ++ni) {
        const int n = wn * 32 + ni * 8 + gid;
        b[ni][0] = B32[n * S + tig];
        b[ni][1] = B32[n * S + 4 + tig];
    }
#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni) mma16816(acc[mi][ni], a[mi], b[ni]);
}

struct Conv {
    const bf16 *in;          // physical input [B][hin][win][cin]
    int B, hin, win, cin;
    int up, stride;          // logical input = nearest x2 of in when up; output = logical / stride
    int hl, wl, hout, wout, cout;
    const bf16 *w;           // [cout][3][3][cin]
    const bf16 *wT;          // [cin][3][3][cout]
    const float *bias;
    const bf16 *skip;        // added before the ReLU (same shape as the output) or null
    int relu;
    bf16 *out;               // [B][hout][wout][cout] BF16, or
    float *out32;            // FP32 output keeping the first out32_ch channels
    int out32_ch;
};

// ---------------------------------------------------------------- forward on tcgen05

// The forward convolutions run on the 5th-generation tensor cores as
// implicit GEMMs, D[pixels][cout] = A[pixels][9 cin] B[cout][9 cin]^T, with
// UMMA M = 128 pixels, N = cout, K = 16 per instruction and the accumulator in
// tensor memory (TMEM).  Both operands are fetched by TMA tensor copies that
// land directly in the swizzled K-major layout the UMMA descriptors name
// (rows of 32, 64 or 128 bytes, 8-row swizzle atoms): the A tile of one chunk
// of cw = min(cin, 64) channels of one tap is a 4-D box {cw channels, bw x bh
// pixels, 1 image} of the NHWC input at the tap's offset (zero fill outside
// the image = the convolution's zero padding; stride-2 layers sample every
// other pixel through the tensor map's element strides), the B tile a 2-D box
// {cw k, cout rows} of the weights.  An output tile is a
// bw x bh rectangle of one image (bw * bh <= 128 rows of M).  Layers that read
// a nearest x2 upsampling of their input are split into the four output
// phases (2i + a, 2j + b): for a phase, tap (ky, kx) reads low-resolution
// pixel (i + floor((a + ky - 1) / 2), j + floor((b + kx - 1) / 2)), so each
// phase is a stride-1 gather of the low-resolution input with the same nine
// taps and weights (the arithmetic is that of the upsampled convolution).
constexpr int TC_M = 128;          // rows of M per tile (UMMA M)
constexpr int TC_MAX_STAGES = 16;  // shared-memory stages of 64 K each (4 UMMAs of K = 16)
constexpr int TC_WAIT = 1 << 22;   // polls before a wait gives up
constexpr int TC_THREADS = 192;    // warp 0 issues TMA, warp 1 the UMMAs, warps 2-5 run the epilogue

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void bar_init_n(uint32_t bar, uint32_t n)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(n) : "memory");
}
__device__ __forceinline__ void bar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void bar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t parity)
{
    for (int it = 0; it < TC_WAIT; ++it) {
        uint32_t ok;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     " selp.u32 %0, 1, 0, p;\n}"
                     : "=r"(ok)
                     : "r"(bar), "r"(parity)
                     : "memory");
        if (ok) return true;
    }
    return false;
}

// TMA tensor loads into shared memory, completion counted on an mbarrier
__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap *map, int c0, int c1, int c2, int c3,
                                            uint32_t bar)
{
    asm volatile("cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, "
                 "%3, %4, %5}], [%6];" ::"r"(dst),
                 "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
                 : "memory");
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int c0, int c1, uint32_t bar)
{
    asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, "
                 "%3}], [%4];" ::"r"(dst),
                 "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(bar)
                 : "memory");
}

// Shared-memory matrix descriptor of a K-major operand whose rows are `row`
// bytes of K (32, 64 or 128) in the matching swizzled layout that TMA writes
// (8-row atoms of 8 x row bytes, 16-byte units XOR-permuted within a row by
// the row index): start address in 16-byte units, leading byte offset unused
// (1), stride byte offset = 8 rows, descriptor version 1 (bits 46-48 = 0b001),
// layout type at bits 61-63 (6: 32-byte, 4: 64-byte, 2: 128-byte swizzle).
// A K16 slice j of the row starts 32 j bytes into it.
__device__ __forceinline__ uint64_t umma_desc_sw(uint32_t addr, uint32_t row)
{
    const uint64_t layout = row == 128 ? 2 : (row == 64 ? 4 : 6);
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | (1ull << 16) | ((uint64_t)((8 * row) >> 4) << 32) | (1ull << 46) |
           (layout << 61);
}

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), BF16
// A and B (bits 7-9, 10-12 = 1), both K-major, N >> 3 at bits 17-22, M >> 4 at
// bits 24-28.
__device__ __forceinline__ uint32_t umma_idesc(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                 " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
                 ::"r"(d), "l"(a), "l"(b), "r"(idesc), "r"(acc)
                 : "memory");
}
__device__ __forceinline__ void umma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                 "[%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                   "=r"(r[15])
                 : "r"(taddr)
                 : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// A chunk is cw = min(cin, 64) channels of one tap (an A box of 128 rows x
// 2 cw bytes and a B box of cout rows x 2 cw bytes, each starting on a
// 1024-byte boundary, the swizzle atom); a stage holds 64 / cw chunks, so
// every stage carries K = 64; as many stages as fit in 220 KB.
constexpr uint32_t TC_SMEM_MAX = 220u * 1024u;
// layers with cout <= 64 keep their ring within 110 KB so that two CTAs (two
// pipelines and epilogues) share an SM
__host__ __device__ inline uint32_t tc_smem_budget(int cout) { return cout <= 64 ? 110u * 1024u : TC_SMEM_MAX; }
__host__ __device__ inline uint32_t tc_a_slot(int cw) { return (uint32_t)TC_M * 2u * (uint32_t)cw; }
__host__ __device__ inline uint32_t tc_b_slot(int cout, int cw)
{
    return ((uint32_t)cout * 2u * (uint32_t)cw + 1023u) & ~1023u;
}
__host__ __device__ inline uint32_t tc_stage_bytes(int cout, int cw)
{
    return (uint32_t)(64 / cw) * (tc_a_slot(cw) + tc_b_slot(cout, cw));
}
__host__ __device__ inline int tc_stages(int cout, int cw)
{
    const int s = (int)((tc_smem_budget(cout) - 2048u) / tc_stage_bytes(cout, cw));
    return s < 3 ? 3 : (s > TC_MAX_STAGES ? TC_MAX_STAGES : s);
}
// + 1024 alignment slack + full/empty barriers (16 x 16) + accumulator
// barriers and the TMEM address (64) + the packed tap tables (4 phases x 36
// taps x 4 bytes + ntap[4] = 592), rounded up
__host__ __device__ inline uint32_t tc_smem_bytes(int cout, int cw)
{
    return (uint32_t)tc_stages(cout, cw) * tc_stage_bytes(cout, cw) + 1024 + 16 * TC_MAX_STAGES + 64 + 640;
}
// TMEM columns for two accumulators of n columns (a power of two >= 32)
__host__ __device__ inline uint32_t tc_tmem_cols(int n)
{
    uint32_t c = 32;
    while (c < 2u * (uint32_t)n) c <<= 1;
    return c;
}

struct TcConv {
    int N, cin, K, cw, nkt;        // cout, input channels, 9 cin, channels per chunk, stages per tile
    int up, stride;                // nearest x2 input (4 output phases) or the input sampling stride
    int gw, gh;                    // tile grid: output size, or the low-resolution input size when up
    int bw, bh, ntx, nty, nph;     // tile rectangle, tiles per image row/column, phases (1 or 4)
    long long ntiles;
    int hout, wout;
    const float *bias;
    const bf16 *skip;              // added before the ReLU (same shape as the output) or null
    int relu;
    bf16 *out;                     // [B][hout][wout][N] BF16, or
    float *out32;                  // FP32 output keeping the first out32_ch channels
    int out32_ch;
};

// Persistent, warp-specialised: each CTA walks output tiles (tile =
// blockIdx.x, += gridDim.x).  The TMA thread fills a ring of stages, one
// expect_tx arrival per stage on full[s]; the UMMA thread waits on full[s],
// issues the stage's UMMAs into accumulator (tile & 1) and commits them to
// empty[s] (which the TMA thread waits on before refilling the stage) and, at
// the end of a tile, to accf[b].  The epilogue warps drain accumulator b with
// tcgen05.ld while the next tile accumulates into the other, then release it
// on acce[b].  Every wait is bounded; a wait that gives up sets *err.
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_conv_fwd_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, TcConv c, int *err)
{
    extern __shared__ unsigned char tc_raw[];
    const int N = c.N, cw = c.cw;
    const uint32_t row = 2u * (uint32_t)cw, stage_bytes = tc_stage_bytes(N, cw);
    const uint32_t a_slot = tc_a_slot(cw), b_slot = tc_b_slot(N, cw), b_base = (uint32_t)(64 / cw) * a_slot;
    const uint32_t a_box = (uint32_t)(c.bw * c.bh) * row, b_box = (uint32_t)N * row;
    const int NS = tc_stages(N, cw), kslices = cw / 16, cps = 64 / cw;
    const int nchunks = 9 * (c.cin / cw);
    // stages 1024-byte aligned; then full[16], empty[16], accf[2], acce[2], the TMEM address
    const uint32_t raw = (uint32_t)__cvta_generic_to_shared(tc_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    const uint32_t full = base + NS * stage_bytes, empty = full + 8 * TC_MAX_STAGES;
    const uint32_t accf = empty + 8 * TC_MAX_STAGES, acce = accf + 16, tslot = acce + 16;
    const uint32_t *tslot_p = reinterpret_cast<const uint32_t *>(tc_raw + (tslot - raw));
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const uint32_t ncols = tc_tmem_cols(N);

    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tslot), "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (t == 0) {
        for (int s = 0; s < NS; ++s) {
            bar_init_n(full + 8 * s, 1);
            bar_init_n(empty + 8 * s, 1);
        }
        for (int b = 0; b < 2; ++b) {
            bar_init_n(accf + 8 * b, 1);
            bar_init_n(acce + 8 * b, 128);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot_p;
    bool ok = true;

    if (warp == 0) {
        if (lane == 0) {
            uint32_t s = 0, lap = 0;                       // ring slot and completed laps of the ring
            for (long long tile = blockIdx.x; tile < c.ntiles && ok; tile += gridDim.x) {
                long long rest = tile;
                const int ph = (int)(rest % c.nph);
                rest /= c.nph;
                const int tx = (int)(rest % c.ntx);
                rest /= c.ntx;
                const int ty = (int)(rest % c.nty);
                const int b = (int)(rest / c.nty);
                const int X0 = tx * c.bw, Y0 = ty * c.bh, pa = ph >> 1, pb = ph & 1;
                int ky = 0, kx = 0, ci = 0, left = nchunks;   // next chunk: tap (ky, kx), channels ci ..
                for (int kt = 0; kt < c.nkt; ++kt) {
                    // the stage was last read by the UMMAs of the previous lap
                    if (lap > 0 && !bar_wait(empty + 8 * s, (lap - 1) & 1)) {
                        ok = false;
                        break;
                    }
                    const int nq = min(cps, left);            // chunks in this stage
                    left -= nq;
                    bar_expect_tx(full + 8 * s, (uint32_t)nq * (a_box + b_box));
                    const uint32_t sa = base + s * stage_bytes, sb = sa + b_base;
                    for (int q = 0; q < nq; ++q) {
                        int x, y;
                        if (c.up) {
                            x = X0 + ((pb + kx + 1) >> 1) - 1;
                            y = Y0 + ((pa + ky + 1) >> 1) - 1;
                        } else {
                            x = c.stride * X0 + kx - 1;
                            y = c.stride * Y0 + ky - 1;
                        }
                        tma_load_4d(sa + q * a_slot, &tmA, ci, x, y, b, full + 8 * s);
                        tma_load_2d(sb + q * b_slot, &tmB, (3 * ky + kx) * c.cin + ci, 0, full + 8 * s);
                        ci += cw;
                        if (ci == c.cin) {
                            ci = 0;
                            if (++kx == 3) {
                                kx = 0;
                                ++ky;
                            }
                        }
                    }
                    if (++s == (uint32_t)NS) {
                        s = 0;
                        ++lap;
                    }
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = umma_idesc(TC_M, N);
            uint32_t s = 0, lap = 0;
            int it = 0;
            for (long long tile = blockIdx.x; tile < c.ntiles && ok; tile += gridDim.x, ++it) {
                const int b = it & 1;
                // accumulator b was last drained by the epilogue of tile it - 2
                if (it >= 2 && !bar_wait(acce + 8 * b, ((it >> 1) - 1) & 1)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(b * N);
                int left = nchunks;
                for (int kt = 0; kt < c.nkt; ++kt) {
                    if (!bar_wait(full + 8 * s, lap & 1)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t sa = base + s * stage_bytes, sb = sa + b_base;
                    const int nq = min(cps, left);
                    left -= nq;
                    for (int q = 0; q < nq; ++q)
                        for (int j = 0; j < kslices; ++j)
                            umma_bf16(d, umma_desc_sw(sa + q * a_slot + 32 * j, row),
                                      umma_desc_sw(sb + q * b_slot + 32 * j, row), idesc, (kt | q | j) != 0);
                    umma_commit(empty + 8 * s);
                    if (++s == (uint32_t)NS) {
                        s = 0;
                        ++lap;
                    }
                }
                umma_commit(accf + 8 * b);      // tracks every UMMA of the tile
            }
        }
    } else {
        // epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 = tile rows 32 (w % 4) .. + 31
        const int e = warp & 3;
        int it = 0;
        for (long long tile = blockIdx.x; tile < c.ntiles && ok; tile += gridDim.x, ++it) {
            const int b = it & 1;
            long long rest = tile;
            const int ph = (int)(rest % c.nph);
            rest /= c.nph;
            const int tx = (int)(rest % c.ntx);
            rest /= c.ntx;
            const int ty = (int)(rest % c.nty);
            const int bimg = (int)(rest / c.nty);
            const int r = e * 32 + lane;
            const int gx = tx * c.bw + r % c.bw, gy = ty * c.bh + r / c.bw;
            const bool valid = r < c.bw * c.bh && gx < c.gw && gy < c.gh;
            const int oy = c.up ? 2 * gy + (ph >> 1) : gy, ox = c.up ? 2 * gx + (ph & 1) : gx;
            const long long pix = ((long long)bimg * c.hout + oy) * c.wout + ox;
            // the skip values of the first 16 channels are requested before the
            // wait for the accumulator, those of chunk c0 + 16 before chunk c0 is used
            const uint4 *sp = c.skip && valid ? reinterpret_cast<const uint4 *>(c.skip + pix * N) : nullptr;
            uint4 s_next[2] = {make_uint4(0u, 0u, 0u, 0u), make_uint4(0u, 0u, 0u, 0u)};
            if (sp) {
                s_next[0] = sp[0];
                s_next[1] = sp[1];
            }
            // warp-uniform decision: tcgen05.ld below must be executed by all 32 lanes
            if (!__all_sync(0xffffffffu, bar_wait(accf + 8 * b, (it >> 1) & 1))) {
                ok = false;
                break;
            }
            tc_fence_after();
            for (int c0 = 0; c0 < N; c0 += 16) {
                uint32_t rr[16];
                tmem_ld16(tmem + ((uint32_t)(e * 32) << 16) + (uint32_t)(b * N + c0), rr);
                const uint4 s_cur[2] = {s_next[0], s_next[1]};
                if (sp && c0 + 16 < N) {
                    s_next[0] = sp[(c0 + 16) / 8];
                    s_next[1] = sp[(c0 + 16) / 8 + 1];
                }
                if (!valid) continue;
                float v[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(rr[j]) + c.bias[c0 + j];
                if (sp) {
                    const bf16 *se = reinterpret_cast<const bf16 *>(s_cur);
#pragma unroll
                    for (int j = 0; j < 16; ++j) v[j] += bf2f(se[j]);
                }
                if (c.relu) {
#pragma unroll
                    for (int j = 0; j < 16; ++j) v[j] = fmaxf(v[j], 0.f);
                }
                if (c.out32) {
                    for (int j = 0; j < 16 && c0 + j < c.out32_ch; ++j) c.out32[pix * c.out32_ch + c0 + j] = v[j];
                } else {
                    uint4 o2[2];
                    bf16 *oe = reinterpret_cast<bf16 *>(o2);
#pragma unroll
                    for (int j = 0; j < 16; ++j) oe[j] = f2bf(v[j]);
                    uint4 *op = reinterpret_cast<uint4 *>(c.out + pix * N + c0);
                    op[0] = o2[0];
                    op[1] = o2[1];
                }
            }
            tc_fence_before();
            bar_arrive(acce + 8 * b);
        }
    }
    tc_fence_before();
    const bool all_ok = __syncthreads_and(ok);
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
    if (t == 0 && !all_ok) atomicOr(err, 1);
}

// ---------------------------------------------------------------- data gradient

constexpr int TC_MAX_TAPS = 36;

// The data gradient of a layer as a convolution-like contraction on the
// tensor cores: acc32[pixel][n] += sum over taps t and channels c of
// W^T[n][t][c] * dY[sample(pixel, t)][c].  Pixels are tiled by bw x bh
// rectangles of a gh x gw grid (per image); with nph = 4 the grid is split
// into output phases (a, b), and grid point (gy, gx) of phase (a, b) is
// pixel (pm gy + a, pm gx + b).  Tap t of phase ph reads dY at (s_in Y0 +
// tdy, s_in X0 + tdx) + s_in (row, column) of the tile (the tensor map
// samples every s_in-th pixel) and the weights of tap tw (3 ky + kx).
struct TcGrad {
    int N, cin, cw;                // output channels (UMMA N), input channels, channels per chunk
    int s_in, pm;                  // input sampling stride, output stride of the phase grid
    int gw, gh;                    // tile grid
    int bw, bh, ntx, nty, nph;     // tile rectangle, tiles per image row/column, phases (1 or 4)
    const uint32_t *taps;          // device: 4 x TC_MAX_TAPS packed taps (dy + 128) | (dx + 128) << 8 | w << 16,
                                   // then ntap[4]
    long long ntiles;
    int hout, wout;                // output tensor size
    float *acc32;                  // [B][hout][wout][N] FP32, accumulated into (+=)
};


// Persistent, warp-specialised: each CTA walks output tiles (tile =
// blockIdx.x, += gridDim.x).  The TMA thread fills a ring of stages, one
// expect_tx arrival per stage on full[s]; the UMMA thread waits on full[s],
// issues the stage's UMMAs into accumulator (tile & 1) and commits them to
// empty[s] (which the TMA thread waits on before refilling the stage) and, at
// the end of a tile, to accf[b].  The epilogue warps drain accumulator b with
// tcgen05.ld while the next tile accumulates into the other, then release it
// on acce[b].  Every wait is bounded; a wait that gives up sets *err.  The
// pipeline is that of k_conv_fwd_tc with the taps read from the tables and a
// per-phase tap count; the forward keeps its own kernel (computed taps), which
// measured about 6% faster than this one on the forward layers.
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_conv_dgrad_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, TcGrad c,
                    int *err)
{
    extern __shared__ unsigned char tc_raw[];
    const int N = c.N, cw = c.cw;
    const uint32_t row = 2u * (uint32_t)cw, stage_bytes = tc_stage_bytes(N, cw);
    const uint32_t a_slot = tc_a_slot(cw), b_slot = tc_b_slot(N, cw), b_base = (uint32_t)(64 / cw) * a_slot;
    const uint32_t a_box = (uint32_t)(c.bw * c.bh) * row, b_box = (uint32_t)N * row;
    const int NS = tc_stages(N, cw), kslices = cw / 16, cps = 64 / cw, per_tap = c.cin / cw;
    // stages 1024-byte aligned; then full[16], empty[16], accf[2], acce[2], the TMEM address
    const uint32_t raw = (uint32_t)__cvta_generic_to_shared(tc_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    const uint32_t full = base + NS * stage_bytes, empty = full + 8 * TC_MAX_STAGES;
    const uint32_t accf = empty + 8 * TC_MAX_STAGES, acce = accf + 16, tslot = acce + 16;
    const uint32_t *tslot_p = reinterpret_cast<const uint32_t *>(tc_raw + (tslot - raw));
    // tap tables in shared memory: (dy + 128) | (dx + 128) << 8 | w << 16 per tap, then ntap[4]
    uint32_t *taps_s = reinterpret_cast<uint32_t *>(tc_raw + (tslot + 64 - raw));
    int *ntap_s = reinterpret_cast<int *>(taps_s + 4 * TC_MAX_TAPS);
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const uint32_t ncols = tc_tmem_cols(N);

    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tslot), "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    for (int i = t; i < 4 * TC_MAX_TAPS + 4; i += TC_THREADS) taps_s[i] = c.taps[i];
    if (t == 0) {
        for (int s = 0; s < NS; ++s) {
            bar_init_n(full + 8 * s, 1);
            bar_init_n(empty + 8 * s, 1);
        }
        for (int b = 0; b < 2; ++b) {
            bar_init_n(accf + 8 * b, 1);
            bar_init_n(acce + 8 * b, 128);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot_p;
    bool ok = true;

    if (warp == 0) {
        if (lane == 0) {
            uint32_t s = 0, lap = 0;                       // ring slot and completed laps of the ring
            for (long long tile = blockIdx.x; tile < c.ntiles && ok; tile += gridDim.x) {
                long long rest = tile;
                const int ph = (int)(rest % c.nph);
                rest /= c.nph;
                const int tx = (int)(rest % c.ntx);
                rest /= c.ntx;
                const int ty = (int)(rest % c.nty);
                const int b = (int)(rest / c.nty);
                const int X0 = c.s_in * tx * c.bw, Y0 = c.s_in * ty * c.bh;
                const int nch = ntap_s[ph] * per_tap, nkt = (nch + cps - 1) / cps;
                const uint32_t *tp = taps_s + ph * TC_MAX_TAPS;
                int ti = 0, ci = 0, left = nch;                // next chunk: tap ti, channels ci ..
                for (int kt = 0; kt < nkt; ++kt) {
                    // the stage was last read by the UMMAs of the previous lap
                    if (lap > 0 && !bar_wait(empty + 8 * s, (lap - 1) & 1)) {
                        ok = false;
                        break;
                    }
                    const int nq = min(cps, left);            // chunks in this stage
                    left -= nq;
                    bar_expect_tx(full + 8 * s, (uint32_t)nq * (a_box + b_box));
                    const uint32_t sa = base + s * stage_bytes, sb = sa + b_base;
                    for (int q = 0; q < nq; ++q) {
                        const uint32_t e = tp[ti];
                        const int x = X0 + (int)((e >> 8) & 255u) - 128, y = Y0 + (int)(e & 255u) - 128;
                        tma_load_4d(sa + q * a_slot, &tmA, ci, x, y, b, full + 8 * s);
                        tma_load_2d(sb + q * b_slot, &tmB, (int)(e >> 16) * c.cin + ci, 0, full + 8 * s);
                        ci += cw;
                        if (ci == c.cin) {
                            ci = 0;
                            ++ti;
                        }
                    }
                    if (++s == (uint32_t)NS) {
                        s = 0;
                        ++lap;
                    }
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = umma_idesc(TC_M, N);
            uint32_t s = 0, lap = 0;
            int it = 0;
            for (long long tile = blockIdx.x; tile < c.ntiles && ok; tile += gridDim.x, ++it) {
                const int b = it & 1;
                const int nch = ntap_s[(int)(tile % c.nph)] * per_tap, nkt = (nch + cps - 1) / cps;
                // accumulator b was last drained by the epilogue of tile it - 2
                if (it >= 2 && !bar_wait(acce + 8 * b, ((it >> 1) - 1) & 1)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(b * N);
                int left = nch;
                for (int kt = 0; kt < nkt; ++kt) {
                    if (!bar_wait(full + 8 * s, lap & 1)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t sa = base + s * stage_bytes, sb = sa + b_base;
                    const int nq = min(cps, left);
                    left -= nq;
                    for (int q = 0; q < nq; ++q)
                        for (int j = 0; j < kslices; ++j)
                            umma_bf16(d, umma_desc_sw(sa + q * a_slot + 32 * j, row),
                                      umma_desc_sw(sb + q * b_slot + 32 * j, row), idesc, (kt | q | j) != 0);
                    umma_commit(empty + 8 * s);
                    if (++s == (uint32_t)NS) {
                        s = 0;
                        ++lap;
                    }
                }
                umma_commit(accf + 8 * b);      // tracks every UMMA of the tile
            }
        }
    } else {
        // epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 = tile rows 32 (w % 4) .. + 31
        const int e = warp & 3;
        int it = 0;
        for (long long tile = blockIdx.x; tile < c.ntiles && ok; tile += gridDim.x, ++it) {
            const int b = it & 1;
            long long rest = tile;
            const int ph = (int)(rest % c.nph);
            rest /= c.nph;
            const int tx = (int)(rest % c.ntx);
            rest /= c.ntx;
            const int ty = (int)(rest % c.nty);
            const int bimg = (int)(rest / c.nty);
            const int r = e * 32 + lane;
            const int gx = tx * c.bw + r % c.bw, gy = ty * c.bh + r / c.bw;
            const bool valid = r < c.bw * c.bh && gx < c.gw && gy < c.gh;
            const int oy = c.pm * gy + (ph >> 1), ox = c.pm * gx + (ph & 1);
            const long long pix = ((long long)bimg * c.hout + oy) * c.wout + ox;
            // warp-uniform decision: tcgen05.ld below must be executed by all 32 lanes
            if (!__all_sync(0xffffffffu, bar_wait(accf + 8 * b, (it >> 1) & 1))) {
                ok = false;
                break;
            }
            tc_fence_after();
            float4 *dp = reinterpret_cast<float4 *>(c.acc32 + pix * N);
            for (int c0 = 0; c0 < N; c0 += 16) {
                uint32_t rr[16];
                tmem_ld16(tmem + ((uint32_t)(e * 32) << 16) + (uint32_t)(b * N + c0), rr);
                if (!valid) continue;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    float4 a = dp[c0 / 4 + j];
                    a.x += __uint_as_float(rr[4 * j]);
                    a.y += __uint_as_float(rr[4 * j + 1]);
                    a.z += __uint_as_float(rr[4 * j + 2]);
                    a.w += __uint_as_float(rr[4 * j + 3]);
                    dp[c0 / 4 + j] = a;
                }
            }
            tc_fence_before();
            bar_arrive(acce + 8 * b);
        }
    }
    tc_fence_before();
    const bool all_ok = __syncthreads_and(ok);
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
    if (t == 0 && !all_ok) atomicOr(err, 1);
}

// ---------------------------------------------------------------- weight gradient on tcgen05

// dW[co][ky][kx][ci] = sum over output pixels p of dY[p][co] X(p, ky, kx)[ci],
// where X(p, ky, kx) is the layer's input at the tap's position, is a GEMM
// with the pixels as K: D[co][ci] = A[co][p] B[ci][p]^T for each tap.  Both
// operands are made K-major by writing them channel-major first:
//   dYT[co][b][y][x]           the output gradient, transposed;
//   G[kx][ci][b][r][x]         the input, transposed, with the tap's column
//                              offset (and the layer's column sampling:
//                              stride 2, or the nearest x2 upsampling)
//                              applied, one copy per kx;
// so that an output row segment of kw pixels is one TMA box of either operand
// ({kw pixels, 1 row, 1 image, channels}: kw * 2 bytes per channel row, the
// swizzle span) and the tap's row offset is the box's row coordinate:
// r = y + ky - 1 (stride 1), 2 y + ky - 1 (stride 2), (y + ky - 1) >> 1
// (upsampled input; rows outside the image read as zeros).  kw = 64, 32 or
// 16 (the output width must be a multiple of 16).

// G[k][c][b][r][xo] = src[b][r][xs(xo, k)][c] (zero where xs leaves the
// image), k < nk; mode 0: xs = xo + k - off, mode 1: xs = 2 xo + k - off,
// mode 2: u = xo + k - off inside [0, wout), xs = u >> 1.  A thread takes
// eight channels (16-byte loads) of eight consecutive xo and writes eight
// 16-byte runs, one per channel; the channel groups run fastest across
// threads so that the loads of a warp are contiguous.  b runs over the
// batch B, the layout keeps maxB images; ch is a multiple of 8.
__global__ void k_wg_gather(const bf16 *__restrict__ src, bf16 *__restrict__ dst, int B, int maxB, int rows,
                            int win, int wout, int ch, int nk, int off, int mode)
{
    const int ng = wout / 8, cq = ch / 8;
    const long long total = (long long)nk * B * rows * ng * cq;
    const long long cstride = (long long)maxB * rows * wout;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int c = 8 * (int)(i % cq);
        long long rest = i / cq;
        const int xg = (int)(rest % ng);
        rest /= ng;
        const int r = (int)(rest % rows);
        rest /= rows;
        const int b = (int)(rest % B);
        const int k = (int)(rest / B);
        uint4 ov[8];
        bf16 *oe = reinterpret_cast<bf16 *>(ov);      // oe[q * 8 + j]: channel c + q, pixel j
        const bf16 *srow = src + ((long long)b * rows + r) * win * ch + c;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int xo = xg * 8 + j;
            int xs;
            bool in;
            if (mode == 2) {
                const int u = xo + k - off;
                in = u >= 0 && u < wout;
                xs = u >> 1;
            } else {
                xs = (mode == 1 ? 2 * xo : xo) + k - off;
                in = xs >= 0 && xs < win;
            }
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (in) v = *reinterpret_cast<const uint4 *>(srow + (long long)xs * ch);
            const bf16 *ve = reinterpret_cast<const bf16 *>(&v);
#pragma unroll
            for (int q = 0; q < 8; ++q) oe[q * 8 + j] = ve[q];
        }
        bf16 *d0 = dst + ((((long long)k * ch + c) * maxB + b) * rows + r) * wout + xg * 8;
#pragma unroll
        for (int q = 0; q < 8; ++q) *reinterpret_cast<uint4 *>(d0 + q * cstride) = ov[q];
    }
}

struct TcWgrad {
    int N, ci, co, kw, nseg;       // UMMA N, input and output channels, pixels per chunk, chunks per output row
    int swap;                      // 0: M = co (A = dYT), N = ci (B = G); 1: M = ci (A = G), N = co (B = dYT)
    int hout, mode;                // output rows; row offset rule: 0 stride 1, 1 stride 2, 2 upsampled input
    int mdim, mblocks, arows;      // M-side channels, their 128-row blocks, rows of the A box (min(mdim, 128))
    long long nchunks;             // chunks of the batch (B * hout * nseg)
    int cpsplit, splits;           // chunks per split, splits
    long long nunits;              // 9 taps x mblocks x splits
    float *dw;                     // the layer's weight gradient [co][9][ci], accumulated into (FP32 atomics)
};

// Same pipeline as k_conv_fwd_tc (TMA thread, UMMA thread, four epilogue
// warps, double-buffered TMEM accumulator); a work unit is (tap, 128-row
// block of co, split of the pixel chunks), ordered so that the nine taps of
// a split run side by side and share its output-gradient boxes in L2.  The
// epilogue adds the unit's D to dW with FP32 atomics: D[co][ci] (vectors of
// four ci) or, with the operands swapped for thin layers (cout < cin, cout <
// 128, so that fewer of the 128 M rows are padding), D[ci][co] (one ci per
// lane, coalesced across the warp).
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_conv_wgrad_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, TcWgrad c,
                    int *err)
{
    extern __shared__ unsigned char tc_raw[];
    const int N = c.N, kw = c.kw;
    const uint32_t row = 2u * (uint32_t)kw, stage_bytes = tc_stage_bytes(N, kw);
    const uint32_t a_slot = tc_a_slot(kw), b_slot = tc_b_slot(N, kw), b_base = (uint32_t)(64 / kw) * a_slot;
    const uint32_t a_box = (uint32_t)c.arows * row, b_box = (uint32_t)N * row;
    const int NS = tc_stages(N, kw), kslices = kw / 16, cps = 64 / kw;
    const uint32_t raw = (uint32_t)__cvta_generic_to_shared(tc_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    const uint32_t full = base + NS * stage_bytes, empty = full + 8 * TC_MAX_STAGES;
    const uint32_t accf = empty + 8 * TC_MAX_STAGES, acce = accf + 16, tslot = acce + 16;
    const uint32_t *tslot_p = reinterpret_cast<const uint32_t *>(tc_raw + (tslot - raw));
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const uint32_t ncols = tc_tmem_cols(N);

    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tslot), "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (t == 0) {
        for (int s = 0; s < NS; ++s) {
            bar_init_n(full + 8 * s, 1);
            bar_init_n(empty + 8 * s, 1);
        }
        for (int b = 0; b < 2; ++b) {
            bar_init_n(accf + 8 * b, 1);
            bar_init_n(acce + 8 * b, 128);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot_p;
    bool ok = true;

    if (warp == 0) {
        if (lane == 0) {
            uint32_t s = 0, lap = 0;
            for (long long u = blockIdx.x; u < c.nunits && ok; u += gridDim.x) {
                const int tap = (int)(u % 9);
                const long long rest = u / 9;
                const int mb = (int)(rest % c.mblocks);
                const int sp = (int)(rest / c.mblocks);
                const int ky = tap / 3, kx = tap - 3 * ky;
                const long long c0 = (long long)sp * c.cpsplit;
                const int n = (int)min((long long)c.cpsplit, c.nchunks - c0);
                const int nkt = (n + cps - 1) / cps;
                // first chunk: output row segment seg of row y of image b
                int seg = (int)(c0 % c.nseg);
                const long long ry0 = c0 / c.nseg;
                int y = (int)(ry0 % c.hout), b = (int)(ry0 / c.hout);
                int left = n;
                for (int kt = 0; kt < nkt; ++kt) {
                    if (lap > 0 && !bar_wait(empty + 8 * s, (lap - 1) & 1)) {
                        ok = false;
                        break;
                    }
                    const int nq = min(cps, left);
                    left -= nq;
                    bar_expect_tx(full + 8 * s, (uint32_t)nq * (a_box + b_box));
                    const uint32_t sa = base + s * stage_bytes, sb = sa + b_base;
                    for (int q = 0; q < nq; ++q) {
                        const int yr = c.mode == 1 ? 2 * y + ky - 1 : (c.mode == 2 ? (y + ky - 1) >> 1 : y + ky - 1);
                        if (c.swap) {
                            tma_load_4d(sa + q * a_slot, &tmA, seg * kw, yr, b, kx * c.ci + mb * 128, full + 8 * s);
                            tma_load_4d(sb + q * b_slot, &tmB, seg * kw, y, b, 0, full + 8 * s);
                        } else {
                            tma_load_4d(sa + q * a_slot, &tmA, seg * kw, y, b, mb * 128, full + 8 * s);
                            tma_load_4d(sb + q * b_slot, &tmB, seg * kw, yr, b, kx * c.ci, full + 8 * s);
                        }
                        if (++seg == c.nseg) {
                            seg = 0;
                            if (++y == c.hout) {
                                y = 0;
                                ++b;
                            }
                        }
                    }
                    if (++s == (uint32_t)NS) {
                        s = 0;
                        ++lap;
                    }
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = umma_idesc(TC_M, N);
            uint32_t s = 0, lap = 0;
            int it = 0;
            for (long long u = blockIdx.x; u < c.nunits && ok; u += gridDim.x, ++it) {
                const int b = it & 1;
                const long long rest = u / 9;
                const int sp = (int)(rest / c.mblocks);
                const int n = (int)min((long long)c.cpsplit, c.nchunks - (long long)sp * c.cpsplit);
                const int nkt = (n + cps - 1) / cps;
                if (it >= 2 && !bar_wait(acce + 8 * b, ((it >> 1) - 1) & 1)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(b * N);
                int left = n;
                for (int kt = 0; kt < nkt; ++kt) {
                    if (!bar_wait(full + 8 * s, lap & 1)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t sa = base + s * stage_bytes, sb = sa + b_base;
                    const int nq = min(cps, left);
                    left -= nq;
                    for (int q = 0; q < nq; ++q)
                        for (int j = 0; j < kslices; ++j)
                            umma_bf16(d, umma_desc_sw(sa + q * a_slot + 32 * j, row),
                                      umma_desc_sw(sb + q * b_slot + 32 * j, row), idesc, (kt | q | j) != 0);
                    umma_commit(empty + 8 * s);
                    if (++s == (uint32_t)NS) {
                        s = 0;
                        ++lap;
                    }
                }
                umma_commit(accf + 8 * b);
            }
        }
    } else {
        // epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 = rows of the M side
        const int e = warp & 3;
        int it = 0;
        for (long long u = blockIdx.x; u < c.nunits && ok; u += gridDim.x, ++it) {
            const int b = it & 1;
            const int tap = (int)(u % 9);
            const int mb = (int)((u / 9) % c.mblocks);
            const int m = mb * 128 + e * 32 + lane;      // co, or ci when swapped
            const bool valid = m < c.mdim;
            if (!__all_sync(0xffffffffu, bar_wait(accf + 8 * b, (it >> 1) & 1))) {
                ok = false;
                break;
            }
            tc_fence_after();
            for (int c0 = 0; c0 < N; c0 += 16) {
                uint32_t rr[16];
                tmem_ld16(tmem + ((uint32_t)(e * 32) << 16) + (uint32_t)(b * N + c0), rr);
                if (!valid) continue;
                if (c.swap) {
                    // column n = co: dW[co][tap][m]
                    float *dp = c.dw + (long long)tap * c.ci + m;
#pragma unroll
                    for (int j = 0; j < 16; ++j) atomicAdd(dp + (long long)(c0 + j) * 9 * c.ci, __uint_as_float(rr[j]));
                } else {
                    float4 *dp = reinterpret_cast<float4 *>(c.dw + ((long long)m * 9 + tap) * c.ci + c0);
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        atomicAdd(dp + j, make_float4(__uint_as_float(rr[4 * j]), __uint_as_float(rr[4 * j + 1]),
                                                      __uint_as_float(rr[4 * j + 2]), __uint_as_float(rr[4 * j + 3])));
                }
            }
            tc_fence_before();
            bar_arrive(acce + 8 * b);
        }
    }
    tc_fence_before();
    const bool all_ok = __syncthreads_and(ok);
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
    if (t == 0 && !all_ok) atomicOr(err, 1);
}

// ---------------------------------------------------------------- weight gradient (narrow layers)

constexpr int WS = 9;   // row stride (32-bit words) of the transposed tiles: 18 BF16

// dW[co][ky][kx][ci] += sum over output pixels of dpre[p][co] * in_logical[p shifted][ci];
// split over pixel ranges (blockIdx.z), FP32 atomics into dW.  Used for the
// layers whose output width is not a multiple of 16 (small frames).
__global__ void __launch_bounds__(GT) k_conv_wgrad(Conv c, const bf16 *dpre, float *dW, int pix_per_split)
{
    __shared__ __align__(16) bf16 As[BM * 2 * WS];
    __shared__ __align__(16) bf16 Bs[BN * 2 * WS];
    const int M = c.cout, N = 9 * c.cin, P = c.B * c.hout * c.wout;
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
    const int p_begin = blockIdx.z * pix_per_split, p_end = min(P, p_begin + pix_per_split);
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5, wm = warp & 1, wn = warp >> 1;
    const int lp = t & 15, c8 = (t >> 4) * 8;        // pixel within the K tile, 8-wide channel group
    const int n = n0 + c8;
    const bool nv = n < N;
    int kk = 0, ci = 0, ky = 0, kx = 0;
    if (nv) { kk = n / c.cin; ci = n % c.cin; ky = kk / 3; kx = kk % 3; }
    const int co = m0 + c8;
    const bool cv = co < M;
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j][0] = acc[i][j][1] = acc[i][j][2] = acc[i][j][3] = 0.f;
    for (int p0 = p_begin; p0 < p_end; p0 += BK) {
        const int p = p0 + lp;
        uint4 va = make_uint4(0u, 0u, 0u, 0u), vb = make_uint4(0u, 0u, 0u, 0u);
        if (p < p_end) {
            if (cv) va = *reinterpret_cast<const uint4 *>(dpre + (size_t)p * c.cout + co);
            if (nv) {
                const int ox = p % c.wout, oy = (p / c.wout) % c.hout, bb = p / (c.wout * c.hout);
                int iy = oy * c.stride + ky - 1, ix = ox * c.stride + kx - 1;
                if (iy >= 0 && iy < c.hl && ix >= 0 && ix < c.wl) {
                    if (c.up) { iy >>= 1; ix >>= 1; }
                    vb = *reinterpret_cast<const uint4 *>(c.in + (((size_t)bb * c.hin + iy) * c.win + ix) * c.cin + ci);
                }
            }
        }
        const bf16 *ea = reinterpret_cast<const bf16 *>(&va), *eb = reinterpret_cast<const bf16 *>(&vb);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            As[(c8 + j) * 2 * WS + lp] = ea[j];
            Bs[(c8 + j) * 2 * WS + lp] = eb[j];
        }
        __syncthreads();
        mma_tile<WS>(reinterpret_cast<const uint32_t *>(As), reinterpret_cast<const uint32_t *>(Bs), acc, wm, wn,
                     lane);
        __syncthreads();
    }
    const int gid = lane >> 2, tig = lane & 3;
#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int row = m0 + wm * 32 + mi * 16 + gid + (e >= 2 ? 8 : 0);
                const int col = n0 + wn * 32 + ni * 8 + 2 * tig + (e & 1);
                if (row < M && col < N) atomicAdd(dW + (size_t)row * N + col, acc[mi][ni][e]);
            }
}

// ---------------------------------------------------------------- elementwise

__global__ void k_input(const float *x, bf16 *xin, long long npix)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= npix * CIN_PAD) return;
    const long long p = i / CIN_PAD;
    const int ch = (int)(i % CIN_PAD);
    xin[i] = f2bf(ch < TSURR_CIN ? x[p * TSURR_CIN + ch] : 0.f);
}

__global__ void k_mask_sum(const float *mask, long long npix, float *sum)
{
    float s = 0.f;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < npix; i += (long long)gridDim.x * blockDim.x)
        s += mask[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(sum, s);
}

// loss terms and the output-layer gradient (16 channels, 4 used)
__global__ void k_loss(const float *y, const float *tgt, const float *mask, const float *msum, long long npix,
                       bf16 *dpre, double *loss)
{
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    float l = 0.f;
    if (p < npix) {
        const float m = mask[p];
        const float inv = *msum > 0.f ? 1.f / *msum : 0.f;
        float r[3], e2 = 0.f;
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) { r[ch] = y[p * 4 + ch] - tgt[p * 3 + ch]; e2 += r[ch] * r[ch]; }
        const float ri = y[p * 4 + 3] - sqrtf(e2);
        l = m * (e2 + ri * ri) * inv;
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) dpre[p * COUT_PAD + ch] = f2bf(2.f * m * r[ch] * inv);
        dpre[p * COUT_PAD + 3] = f2bf(2.f * m * ri * inv);
#pragma unroll
        for (int ch = 4; ch < COUT_PAD; ++ch) dpre[p * COUT_PAD + ch] = f2bf(0.f);
    }
    for (int o = 16; o > 0; o >>= 1) l += __shfl_down_sync(0xffffffffu, l, o);
    if ((threadIdx.x & 31) == 0 && l != 0.f) atomicAdd(loss, (double)l);
}

// gradient at a layer output -> gradient before the ReLU (BF16 for the GEMMs),
// also added to the gradient of the skip source when the layer has one
// eight elements per thread (n8 = elements / 8; every layer's channel count is a multiple of 8)
__global__ void k_dpre(const float *d, const bf16 *a, bf16 *dpre, float *skip_grad, long long n8, int relu)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n8) return;
    const float4 d0 = reinterpret_cast<const float4 *>(d)[2 * i], d1 = reinterpret_cast<const float4 *>(d)[2 * i + 1];
    float g[8] = {d0.x, d0.y, d0.z, d0.w, d1.x, d1.y, d1.z, d1.w};
    const uint4 av = reinterpret_cast<const uint4 *>(a)[i];
    const bf16 *ae = reinterpret_cast<const bf16 *>(&av);
    uint4 ov;
    bf16 *oe = reinterpret_cast<bf16 *>(&ov);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        if (relu && !(bf2f(ae[j]) > 0.f)) g[j] = 0.f;
        oe[j] = f2bf(g[j]);
    }
    reinterpret_cast<uint4 *>(dpre)[i] = ov;
    if (skip_grad) {
        float4 *sp = reinterpret_cast<float4 *>(skip_grad) + 2 * i;
        float4 s0 = sp[0], s1 = sp[1];
        s0.x += g[0]; s0.y += g[1]; s0.z += g[2]; s0.w += g[3];
        s1.x += g[4]; s1.y += g[5]; s1.z += g[6]; s1.w += g[7];
        sp[0] = s0;
        sp[1] = s1;
    }
}

// db[c] += sum over pixels of dpre[p][c].  Each thread sums one group of
// eight channels (a 16-byte load) over a strided set of pixels: the grid
// stride is a multiple of 256 and ch / 8 divides 256, so a thread keeps its
// group.  The block adds its threads' partial sums in shared memory and
// issues one atomic per channel.
constexpr int BG_THREADS = 256;
__global__ void __launch_bounds__(BG_THREADS) k_bias_grad(const bf16 *dpre, long long npix, int ch, float *db)
{
    __shared__ float part[BG_THREADS * 8];
    const int groups = ch / 8;
    const long long nvec = npix * groups;
    float s[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll 4
    for (long long v = (long long)blockIdx.x * BG_THREADS + threadIdx.x; v < nvec; v += (long long)gridDim.x * BG_THREADS) {
        const uint4 u = reinterpret_cast<const uint4 *>(dpre)[v];
        const bf16 *e = reinterpret_cast<const bf16 *>(&u);
#pragma unroll
        for (int j = 0; j < 8; ++j) s[j] += bf2f(e[j]);
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) part[threadIdx.x * 8 + j] = s[j];
    __syncthreads();
    for (int c = threadIdx.x; c < ch; c += BG_THREADS) {
        float t = 0.f;
        for (int k = c / 8; k < BG_THREADS; k += groups) t += part[k * 8 + c % 8];
        atomicAdd(db + c, t);
    }
}

__global__ void k_adam(float *p, const float *g, float *m1, float *m2, long long n, float lr, float b1, float b2,
                       float eps, float c1, float c2)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float a = b1 * m1[i] + (1.f - b1) * gi;
    const float b = b2 * m2[i] + (1.f - b2) * gi * gi;
    m1[i] = a;
    m2[i] = b;
    p[i] -= lr * (a / c1) / (sqrtf(b / c2) + eps);
}

// FP32 master weights -> BF16 [cout][3][3][cin] and the transposed [cin][3][3][cout]
__global__ void k_weights(const float *w, bf16 *wb, bf16 *wt, int cout, int cin)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= cout * 9 * cin) return;
    const int ci = i % cin, kk = (i / cin) % 9, co = i / (9 * cin);
    const bf16 v = f2bf(w[i]);
    wb[i] = v;
    wt[((size_t)ci * 9 + kk) * cout + co] = v;
}

inline unsigned cdiv(long long a, long long b) { return (unsigned)((a + b - 1) / b); }

}  // namespace

// ---------------------------------------------------------------- host side

struct tsurr_net {
    int maxB = 0, H = 0, W = 0;
    cudaStream_t s = nullptr;
    int cin[NL], cout[NL], hin[NL], win[NL], stride[NL], up[NL], relu[NL], skip[NL], src[NL];
    long long woff[NL], boff[NL];
    long long nparam = 0;
    float *p = nullptr, *g = nullptr, *m1 = nullptr, *m2 = nullptr;
    bf16 *wb[NL] = {}, *wt[NL] = {};
    bf16 *wmem = nullptr;
    bf16 *act[NL + 1] = {};      // act[0] = padded input, act[i+1] = output of layer i (BF16)
    float *dact[NL + 1] = {};    // FP32 gradients of act[1..8]
    float *y = nullptr;          // FP32 network output [B][H][W][4]
    bf16 *dpre = nullptr;
    float *msum = nullptr;
    double *loss = nullptr;
    float *xbuf = nullptr, *tbuf = nullptr, *mbuf = nullptr;
    int *err = nullptr;          // set by a kernel whose bounded wait gave up
    int num_sms = 1;
    CUtensorMap tmA[NL], tmB[NL];   // TMA maps of each layer's input (at max_batch) and BF16 weights
    TcConv tc[NL];                  // tile geometry of each layer's forward
    CUtensorMap tmAd[NL], tmBd[NL]; // data gradient: maps of the layer's output gradient and transposed weights
    TcGrad tcd[NL];                 // data gradient of each layer (L >= 1)
    uint32_t *taps = nullptr;       // device copy of the data gradients' packed tap tables (NL tables)
    bool wg_tc[NL] = {};            // weight gradient on tcgen05 (output width a multiple of 16)
    CUtensorMap tmAw[NL], tmBw[NL]; // weight gradient: maps of dYT and G
    TcWgrad tcw[NL];
    bf16 *dyt = nullptr;            // output gradient, channel-major [co][maxB][hout][wout]
    bf16 *gx = nullptr;             // layer input, channel-major with column offsets [3][ci][maxB][rows][wout]
    std::vector<void *> allocs;
};

static int sfail(int code, const std::string &m)
{
    tsim_record_error(m);
    return code;
}

#define SCU(call)                                                                              \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return sfail(TSIM_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));   \
    } while (0)

static long long act_elems(const tsurr_net *n, int i, int B)
{
    // i = 0: padded input; i >= 1: output of layer i-1
    if (i == 0) return (long long)B * n->H * n->W * CIN_PAD;
    const int L = i - 1;
    const int hl = n->up[L] ? 2 * n->hin[L] : n->hin[L], wl = n->up[L] ? 2 * n->win[L] : n->win[L];
    return (long long)B * (hl / n->stride[L]) * (wl / n->stride[L]) * n->cout[L];
}

static Conv conv_of(const tsurr_net *n, int L, int B)
{
    Conv c;
    memset(&c, 0, sizeof(c));
    c.in = n->act[n->src[L]];
    c.B = B;
    c.hin = n->hin[L];
    c.win = n->win[L];
    c.cin = n->cin[L];
    c.up = n->up[L];
    c.stride = n->stride[L];
    c.hl = c.up ? 2 * c.hin : c.hin;
    c.wl = c.up ? 2 * c.win : c.win;
    c.hout = c.hl / c.stride;
    c.wout = c.wl / c.stride;
    c.cout = n->cout[L];
    c.w = n->wb[L];
    c.wT = n->wt[L];
    c.bias = n->p + n->boff[L];
    c.skip = n->skip[L] >= 0 ? n->act[n->skip[L]] : nullptr;
    c.relu = n->relu[L];
    c.out = n->act[L + 1];
    c.out32 = nullptr;
    return c;
}

// TMA maps and tile geometry of the nine forward convolutions (once per net)
using EncodeFn = PFN_cuTensorMapEncodeTiled_v12000;

// tile geometry of an op on a gh x gw grid
template <class C>
static void tc_tiles(C &c, int gh, int gw)
{
    c.gw = gw;
    c.gh = gh;
    c.bw = std::min(gw, TC_M);
    c.bh = std::max(1, std::min(gh, TC_M / c.bw));
    c.ntx = (gw + c.bw - 1) / c.bw;
    c.nty = (gh + c.bh - 1) / c.bh;
}

// packed tap tables of every op, host copy (uploaded once per net)
struct TapTable {
    uint32_t e[4 * TC_MAX_TAPS + 4];
};

static void tc_tap(TapTable &tt, int ph, int dy, int dx, int w)
{
    uint32_t &n = tt.e[4 * TC_MAX_TAPS + ph];
    tt.e[ph * TC_MAX_TAPS + n] = (uint32_t)(dy + 128) | ((uint32_t)(dx + 128) << 8) | ((uint32_t)w << 16);
    ++n;
}

// TMA maps of an op: input NHWC [maxB][h][w][cin] sampled every es-th pixel
// in boxes of cw channels x bw x bh samples, weights [N rows][9 cin]
template <class C>
static bool tc_maps(EncodeFn encode, const C &c, int es_, const void *in, int h, int w, int maxB, const void *wts,
                    CUtensorMap *ma, CUtensorMap *mb, std::string *why)
{
    const cuuint32_t es = (cuuint32_t)es_;
    const cuuint64_t gdim[4] = {(cuuint64_t)c.cin, (cuuint64_t)w, (cuuint64_t)h, (cuuint64_t)maxB};
    const cuuint64_t gstr[3] = {(cuuint64_t)c.cin * 2, (cuuint64_t)w * c.cin * 2, (cuuint64_t)h * w * c.cin * 2};
    const cuuint32_t box[4] = {(cuuint32_t)c.cw, (cuuint32_t)c.bw * es, (cuuint32_t)c.bh * es, 1};
    const cuuint32_t estr[4] = {1, es, es, 1};
    const CUtensorMapSwizzle swz = c.cw == 64 ? CU_TENSOR_MAP_SWIZZLE_128B
                                              : (c.cw == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B);
    CUresult r = encode(ma, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void *>(in), gdim, gstr, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, swz, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        *why = "input tensor map: error " + std::to_string((int)r);
        return false;
    }
    const cuuint64_t wdim[2] = {(cuuint64_t)9 * c.cin, (cuuint64_t)c.N};
    const cuuint64_t wstr[1] = {(cuuint64_t)9 * c.cin * 2};
    const cuuint32_t wbox[2] = {(cuuint32_t)c.cw, (cuuint32_t)c.N};
    const cuuint32_t westr[2] = {1, 1};
    r = encode(mb, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(wts), wdim, wstr, wbox, westr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, swz, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        *why = "weight tensor map: error " + std::to_string((int)r);
        return false;
    }
    return true;
}

// Tap tables, tile geometry and TMA maps of the nine forward convolutions and
// of the data gradients of layers 1..8 (once per net).
//  forward, stride s:  out[y][x] = sum_t W[t] in[s y + ky - 1][s x + kx - 1]
//  forward, up:        phase (a, b): low-res in[i + floor((a + ky - 1) / 2)][..]
//  gradient, stride 1: dX[y][x] = sum_t W^T[t] dY[y + 1 - ky][x + 1 - kx]
//  gradient, stride 2: phase (a, b) of dX: taps with (a + 1 - ky) even,
//                      dY[i + (a + 1 - ky) / 2][..]
//  gradient, up:       dX[i][j] = sum over the 2 x 2 upsampled children (a, b)
//                      and the nine taps of W^T dY[2 i + a + 1 - ky][..]
static bool setup_convs(tsurr_net *n, std::string *why)
{
    static EncodeFn encode = nullptr;
    if (!encode) {
        cudaDriverEntryPointQueryResult q;
        void *fn = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn) {
            *why = "cuTensorMapEncodeTiled is not available";
            return false;
        }
        encode = reinterpret_cast<EncodeFn>(fn);
    }
    std::vector<TapTable> tabs(NL);
    memset(tabs.data(), 0, tabs.size() * sizeof(TapTable));
    const size_t TT = sizeof(TapTable) / sizeof(uint32_t);
    for (int L = 0; L < NL; ++L) {
        const int hin = n->hin[L], win = n->win[L], cin = n->cin[L], cout = n->cout[L];
        const int up = n->up[L], st = n->stride[L];
        TapTable &tg = tabs[L];
        const int hout = (up ? 2 * hin : hin) / st, wout = (up ? 2 * win : win) / st;
        // forward: taps computed in the kernel from up / stride
        TcConv &c = n->tc[L];
        memset(&c, 0, sizeof(c));
        c.N = cout;
        c.cin = cin;
        c.K = 9 * cin;
        c.cw = std::min(cin, 64);
        c.nkt = (9 * (cin / c.cw) + (64 / c.cw) - 1) / (64 / c.cw);
        c.up = up;
        c.stride = st;
        c.hout = hout;
        c.wout = wout;
        c.nph = up ? 4 : 1;
        c.relu = n->relu[L];
        if (up) tc_tiles(c, hin, win);
        else tc_tiles(c, hout, wout);
        std::string w2;
        if (!tc_maps(encode, c, up ? 1 : st, n->act[n->src[L]], hin, win, n->maxB, n->wb[L], &n->tmA[L], &n->tmB[L],
                     &w2)) {
            *why = "layer " + std::to_string(L) + " forward " + w2;
            return false;
        }
        if (L == 0) continue;          // no gradient towards the network input
        // data gradient: input = the layer's output gradient (cout channels), N = cin
        TcGrad &d = n->tcd[L];
        memset(&d, 0, sizeof(d));
        d.N = cin;
        d.cin = cout;
        d.cw = std::min(cout, 64);
        d.hout = hin;
        d.wout = win;
        d.taps = n->taps + L * TT;
        if (up) {
            d.s_in = 2;
            d.pm = 1;
            d.nph = 1;
            tc_tiles(d, hin, win);
            for (int a = 0; a < 2; ++a)
                for (int b = 0; b < 2; ++b)
                    for (int t = 0; t < 9; ++t) tc_tap(tg, 0, a + 1 - t / 3, b + 1 - t % 3, t);
        } else if (st == 2) {
            d.s_in = 1;
            d.pm = 2;
            d.nph = 4;
            tc_tiles(d, hout, wout);
            for (int ph = 0; ph < 4; ++ph)
                for (int t = 0; t < 9; ++t) {
                    const int a = ph >> 1, b = ph & 1, ky = t / 3, kx = t % 3;
                    if (((a + 1 - ky) & 1) == 0 && ((b + 1 - kx) & 1) == 0)
                        tc_tap(tg, ph, (a + 1 - ky) / 2, (b + 1 - kx) / 2, t);
                }
        } else {
            d.s_in = 1;
            d.pm = 1;
            d.nph = 1;
            tc_tiles(d, hin, win);
            for (int t = 0; t < 9; ++t) tc_tap(tg, 0, 1 - t / 3, 1 - t % 3, t);
        }
        if (!tc_maps(encode, d, d.s_in, n->dpre, hout, wout, n->maxB, n->wt[L], &n->tmAd[L], &n->tmBd[L], &w2)) {
            *why = "layer " + std::to_string(L) + " gradient " + w2;
            return false;
        }
    }
    if (cudaMemcpy(n->taps, tabs.data(), tabs.size() * sizeof(TapTable), cudaMemcpyHostToDevice) != cudaSuccess) {
        *why = "upload of the tap tables failed";
        return false;
    }
    // weight gradients on tcgen05: maps of dYT {wout, hout, maxB, co} and
    // G {wout, rows, maxB, 3 ci}, boxes of one row segment of kw pixels
    for (int L = 0; L < NL; ++L) {
        if (!n->wg_tc[L]) continue;
        const int up = n->up[L], st = n->stride[L], ci = n->cin[L], co = n->cout[L];
        const int hout = (up ? 2 * n->hin[L] : n->hin[L]) / st, wout = (up ? 2 * n->win[L] : n->win[L]) / st;
        const int rows = n->hin[L];
        TcWgrad &w = n->tcw[L];
        memset(&w, 0, sizeof(w));
        w.swap = co < TC_M && ci > co;
        w.N = w.swap ? co : ci;
        w.ci = ci;
        w.co = co;
        w.mdim = w.swap ? ci : co;
        w.kw = wout % 64 == 0 ? 64 : (wout % 32 == 0 ? 32 : 16);
        w.nseg = wout / w.kw;
        w.hout = hout;
        w.mode = up ? 2 : (st == 2 ? 1 : 0);
        w.mblocks = (w.mdim + TC_M - 1) / TC_M;
        w.arows = std::min(w.mdim, TC_M);
        const CUtensorMapSwizzle swz = w.kw == 64 ? CU_TENSOR_MAP_SWIZZLE_128B
                                                  : (w.kw == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B);
        const cuuint32_t estr[4] = {1, 1, 1, 1};
        const cuuint64_t adim[4] = {(cuuint64_t)wout, (cuuint64_t)hout, (cuuint64_t)n->maxB, (cuuint64_t)co};
        const cuuint64_t astr[3] = {(cuuint64_t)wout * 2, (cuuint64_t)hout * wout * 2,
                                    (cuuint64_t)n->maxB * hout * wout * 2};
        // dYT with boxes of min(co, 128) rows (A) or co rows (B); G with boxes
        // of ci rows (B) or min(ci, 128) rows (A)
        const cuuint32_t ybox[4] = {(cuuint32_t)w.kw, 1, 1, (cuuint32_t)(w.swap ? co : w.arows)};
        CUresult r = encode(w.swap ? &n->tmBw[L] : &n->tmAw[L], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, (void *)n->dyt,
                            adim, astr, ybox, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, swz,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        const cuuint64_t bdim[4] = {(cuuint64_t)wout, (cuuint64_t)rows, (cuuint64_t)n->maxB, (cuuint64_t)3 * ci};
        const cuuint64_t bstr[3] = {(cuuint64_t)wout * 2, (cuuint64_t)rows * wout * 2,
                                    (cuuint64_t)n->maxB * rows * wout * 2};
        const cuuint32_t gbox[4] = {(cuuint32_t)w.kw, 1, 1, (cuuint32_t)(w.swap ? w.arows : ci)};
        if (r == CUDA_SUCCESS)
            r = encode(w.swap ? &n->tmAw[L] : &n->tmBw[L], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, (void *)n->gx, bdim,
                       bstr, gbox, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, swz, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                       CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) {
            *why = "layer " + std::to_string(L) + " weight-gradient tensor map: error " + std::to_string((int)r);
            return false;
        }
    }
    return true;
}

// weight gradient of layer L on tcgen05 for a batch of B: channel-major
// copies of the output gradient and of the input, then the contraction
static void launch_wgrad_tc(tsurr_net *n, int L, int B)
{
    TcWgrad w = n->tcw[L];
    const int up = n->up[L], st = n->stride[L], ci = n->cin[L], co = n->cout[L];
    const int wout = w.nseg * w.kw, rows = n->hin[L];
    const unsigned gmax = (unsigned)(8 * n->num_sms);
    const long long ty = (long long)B * w.hout * (wout / 8) * (co / 8);
    k_wg_gather<<<std::min(cdiv(ty, 256), gmax), 256, 0, n->s>>>(n->dpre, n->dyt, B, n->maxB, w.hout, wout, wout, co,
                                                                  1, 0, 0);
    const long long tg = 3LL * B * rows * (wout / 8) * (ci / 8);
    k_wg_gather<<<std::min(cdiv(tg, 256), gmax), 256, 0, n->s>>>(n->act[n->src[L]], n->gx, B, n->maxB, rows,
                                                                  n->win[L], wout, ci, 3, 1, up ? 2 : (st == 2 ? 1 : 0));
    const int cps = 64 / w.kw;
    const int per_sm = w.N <= 64 ? 2 : 1;                                       // see tc_smem_budget
    w.nchunks = (long long)B * w.hout * w.nseg;
    const long long want = std::max<long long>(1, (2LL * per_sm * n->num_sms + 9 * w.mblocks - 1) / (9 * w.mblocks));
    w.cpsplit = (int)std::max<long long>(8LL * cps, (w.nchunks + want - 1) / want);
    w.splits = (int)((w.nchunks + w.cpsplit - 1) / w.cpsplit);
    w.nunits = 9LL * w.mblocks * w.splits;
    w.dw = n->g + n->woff[L];
    const unsigned grid = (unsigned)std::min<long long>(w.nunits, (long long)per_sm * n->num_sms);
    k_conv_wgrad_tc<<<grid, TC_THREADS, tc_smem_bytes(w.N, w.kw), n->s>>>(n->tmAw[L], n->tmBw[L], w, n->err);
}

// persistent grid: every SM holds one CTA, two for N <= 64 (see tc_smem_budget)
static unsigned tc_grid(const tsurr_net *n, int N, long long ntiles)
{
    const int per_sm = N <= 64 ? 2 : 1;
    return (unsigned)std::min<long long>(ntiles, (long long)per_sm * n->num_sms);
}

extern "C" int tsurr_create(int max_batch, int height, int width, void *stream, tsurr_net **out)
{
    if (!out) return sfail(TSIM_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (max_batch < 1 || max_batch > 4096 || height < 8 || width < 8 || height % 8 || width % 8 || height > 512 ||
        width > 512)
        return sfail(TSIM_ERR_INVALID_ARG, "need 1 <= max_batch <= 4096 and 8 <= H, W <= 512, multiples of 8");
    tsurr_net *n = new tsurr_net();
    n->maxB = max_batch;
    n->H = height;
    n->W = width;
    n->s = (cudaStream_t)stream;
    const int H = height, W = width;
    // layer table (see tsurr.h)
    const int ci[NL] = {CIN_PAD, 32, 64, 128, 256, 256, 128, 64, 32};
    const int co[NL] = {32, 64, 128, 256, 256, 128, 64, 32, COUT_PAD};
    const int hi[NL] = {H, H, H / 2, H / 4, H / 8, H / 8, H / 4, H / 2, H};
    const int st[NL] = {1, 2, 2, 2, 1, 1, 1, 1, 1};
    const int upv[NL] = {0, 0, 0, 0, 0, 1, 1, 1, 0};
    const int sk[NL] = {-1, -1, -1, -1, -1, 3, 2, 1, -1};   // act index added before the ReLU
    for (int L = 0; L < NL; ++L) {
        n->cin[L] = ci[L];
        n->cout[L] = co[L];
        n->hin[L] = hi[L];
        n->win[L] = hi[L] * W / H;
        n->stride[L] = st[L];
        n->up[L] = upv[L];
        n->relu[L] = L < NL - 1;
        n->skip[L] = sk[L];
        n->src[L] = L;   // layer L reads act[L]
        n->woff[L] = n->nparam;
        n->nparam += (long long)co[L] * 9 * ci[L];
        n->boff[L] = n->nparam;
        n->nparam += co[L];
    }
    auto alloc = [&](void **p, size_t bytes) -> bool {
        if (cudaMalloc(p, bytes) != cudaSuccess) return false;
        n->allocs.push_back(*p);
        return true;
    };
    long long wtotal = 0;
    for (int L = 0; L < NL; ++L) wtotal += (long long)co[L] * 9 * ci[L];
    bool ok = alloc((void **)&n->p, n->nparam * 4) && alloc((void **)&n->g, n->nparam * 4) &&
              alloc((void **)&n->m1, n->nparam * 4) && alloc((void **)&n->m2, n->nparam * 4) &&
              alloc((void **)&n->wmem, wtotal * 2 * sizeof(bf16));
    long long wo = 0;
    for (int L = 0; L < NL && ok; ++L) {
        n->wb[L] = n->wmem + wo;
        n->wt[L] = n->wmem + wtotal + wo;
        wo += (long long)co[L] * 9 * ci[L];
    }
    long long maxl = 0;
    for (int i = 0; i <= NL && ok; ++i) {
        const long long e = act_elems(n, i, max_batch);
        ok = alloc((void **)&n->act[i], e * sizeof(bf16));
        if (ok && i >= 1) ok = alloc((void **)&n->dact[i], e * sizeof(float));
        if (i >= 1 && e > maxl) maxl = e;
    }
    const long long npix = (long long)max_batch * H * W;
    ok = ok && alloc((void **)&n->y, npix * 4 * sizeof(float)) && alloc((void **)&n->dpre, maxl * sizeof(bf16)) &&
         alloc((void **)&n->msum, 64) && alloc((void **)&n->loss, 64) &&
         alloc((void **)&n->xbuf, npix * TSURR_CIN * sizeof(float)) &&
         alloc((void **)&n->tbuf, npix * 3 * sizeof(float)) && alloc((void **)&n->mbuf, npix * sizeof(float)) &&
         alloc((void **)&n->err, 64) && alloc((void **)&n->taps, NL * sizeof(TapTable));
    // channel-major operands of the tcgen05 weight gradients (layers whose
    // output width is a multiple of 16)
    long long gmax = 0;
    for (int L = 0; L < NL; ++L) {
        const int wout = (upv[L] ? 2 * n->win[L] : n->win[L]) / st[L];
        n->wg_tc[L] = wout % 16 == 0;
        if (n->wg_tc[L]) gmax = std::max(gmax, 3LL * ci[L] * max_batch * hi[L] * wout);
    }
    ok = ok && alloc((void **)&n->dyt, maxl * sizeof(bf16)) &&
         alloc((void **)&n->gx, std::max<long long>(gmax, 8) * sizeof(bf16));
    if (!ok) {
        cudaGetLastError();
        for (void *p : n->allocs) cudaFree(p);
        delete n;
        return sfail(TSIM_ERR_OOM, "tsurr_create: device allocation failed");
    }
    cudaMemsetAsync(n->p, 0, n->nparam * 4, n->s);
    cudaMemsetAsync(n->g, 0, n->nparam * 4, n->s);
    cudaMemsetAsync(n->m1, 0, n->nparam * 4, n->s);
    cudaMemsetAsync(n->m2, 0, n->nparam * 4, n->s);
    cudaMemsetAsync(n->wmem, 0, wtotal * 2 * sizeof(bf16), n->s);
    cudaMemsetAsync(n->err, 0, 64, n->s);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n->num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n->num_sms < 1)
        n->num_sms = 1;
    if (cudaFuncSetAttribute(k_conv_fwd_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(TC_SMEM_MAX + 2048)) !=
            cudaSuccess ||
        cudaFuncSetAttribute(k_conv_dgrad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(TC_SMEM_MAX + 2048)) != cudaSuccess ||
        cudaFuncSetAttribute(k_conv_wgrad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(TC_SMEM_MAX + 2048)) != cudaSuccess ||
        cudaStreamSynchronize(n->s) != cudaSuccess) {
        for (void *p : n->allocs) cudaFree(p);
        delete n;
        return sfail(TSIM_ERR_CUDA, "tsurr_create: initialisation failed");
    }
    std::string why;
    if (!setup_convs(n, &why)) {
        for (void *p : n->allocs) cudaFree(p);
        delete n;
        return sfail(TSIM_ERR_CUDA, "tsurr_create: " + why);
    }
    *out = n;
    return TSIM_OK;
}

extern "C" void tsurr_destroy(tsurr_net *n)
{
    if (!n) return;
    cudaStreamSynchronize(n->s);
    for (void *p : n->allocs) cudaFree(p);
    delete n;
}

extern "C" int64_t tsurr_num_params(const tsurr_net *n) { return n ? n->nparam : 0; }

static int refresh_weights(tsurr_net *n)
{
    for (int L = 0; L < NL; ++L) {
        const int cnt = n->cout[L] * 9 * n->cin[L];
        k_weights<<<cdiv(cnt, 256), 256, 0, n->s>>>(n->p + n->woff[L], n->wb[L], n->wt[L], n->cout[L], n->cin[L]);
    }
    SCU(cudaGetLastError());
    return TSIM_OK;
}

extern "C" int tsurr_set_params(tsurr_net *n, const float *p, int64_t cnt, int on_device)
{
    if (!n || !p || cnt != n->nparam) return sfail(TSIM_ERR_INVALID_ARG, "tsurr_set_params: need all parameters");
    SCU(cudaMemcpyAsync(n->p, p, cnt * 4, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, n->s));
    SCU(cudaMemsetAsync(n->m1, 0, cnt * 4, n->s));
    SCU(cudaMemsetAsync(n->m2, 0, cnt * 4, n->s));
    int rc = refresh_weights(n);
    if (rc) return rc;
    SCU(cudaStreamSynchronize(n->s));
    return TSIM_OK;
}

extern "C" int tsurr_get_params(tsurr_net *n, float *p, int64_t cnt, int on_device)
{
    if (!n || !p || cnt != n->nparam) return sfail(TSIM_ERR_INVALID_ARG, "tsurr_get_params: need all parameters");
    SCU(cudaMemcpyAsync(p, n->p, cnt * 4, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, n->s));
    SCU(cudaStreamSynchronize(n->s));
    return TSIM_OK;
}

extern "C" int tsurr_get_grads(tsurr_net *n, float *g, int64_t cnt, int on_device)
{
    if (!n || !g || cnt != n->nparam) return sfail(TSIM_ERR_INVALID_ARG, "tsurr_get_grads: need all parameters");
    SCU(cudaMemcpyAsync(g, n->g, cnt * 4, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, n->s));
    SCU(cudaStreamSynchronize(n->s));
    return TSIM_OK;
}

static int run_forward(tsurr_net *n, const float *x, int B)
{
    const long long npix = (long long)B * n->H * n->W;
    k_input<<<cdiv(npix * CIN_PAD, 256), 256, 0, n->s>>>(x, n->act[0], npix);
    for (int L = 0; L < NL; ++L) {
        TcConv c = n->tc[L];
        c.ntiles = (long long)B * c.nty * c.ntx * c.nph;
        c.bias = n->p + n->boff[L];
        c.skip = n->skip[L] >= 0 ? n->act[n->skip[L]] : nullptr;
        c.out = n->act[L + 1];
        c.out32 = nullptr;
        if (L == NL - 1) {
            c.out = nullptr;
            c.out32 = n->y;
            c.out32_ch = TSURR_COUT;
        }
        k_conv_fwd_tc<<<tc_grid(n, c.N, c.ntiles), TC_THREADS, tc_smem_bytes(c.N, c.cw), n->s>>>(n->tmA[L], n->tmB[L],
                                                                                                  c, n->err);
    }
    SCU(cudaGetLastError());
    return TSIM_OK;
}

// latched device errors (a bounded wait that gave up); synchronises
static int check_err(tsurr_net *n)
{
    int e = 0;
    SCU(cudaMemcpyAsync(&e, n->err, sizeof(int), cudaMemcpyDeviceToHost, n->s));
    SCU(cudaStreamSynchronize(n->s));
    if (e) return sfail(TSIM_ERR_TIMEOUT, "tsurr: a tensor-core pipeline wait gave up");
    return TSIM_OK;
}

static const float *stage(tsurr_net *n, const float *src, float *buf, size_t bytes, int on_device, int *rc)
{
    *rc = TSIM_OK;
    if (on_device) return src;
    if (cudaMemcpyAsync(buf, src, bytes, cudaMemcpyHostToDevice, n->s) != cudaSuccess)
        *rc = sfail(TSIM_ERR_CUDA, "tsurr: host to device copy failed");
    return buf;
}

extern "C" int tsurr_forward(tsurr_net *n, const float *x, int B, float *y, int on_device)
{
    if (!n || !x || !y || B < 1 || B > n->maxB) return sfail(TSIM_ERR_INVALID_ARG, "tsurr_forward: bad arguments");
    const long long npix = (long long)B * n->H * n->W;
    int rc;
    const float *xd = stage(n, x, n->xbuf, npix * TSURR_CIN * 4, on_device, &rc);
    if (rc) return rc;
    rc = run_forward(n, xd, B);
    if (rc) return rc;
    SCU(cudaMemcpyAsync(y, n->y, npix * 4 * sizeof(float), on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                        n->s));
    return on_device ? TSIM_OK : check_err(n);
}

extern "C" int tsurr_sync(tsurr_net *n)
{
    if (!n) return sfail(TSIM_ERR_INVALID_ARG, "tsurr_sync: net is NULL");
    return check_err(n);
}

extern "C" int tsurr_backward(tsurr_net *n, const float *x, const float *target, const float *mask, int B,
                              double *loss, int on_device)
{
    if (!n || !x || !target || !mask || B < 1 || B > n->maxB)
        return sfail(TSIM_ERR_INVALID_ARG, "tsurr_backward: bad arguments");
    const long long npix = (long long)B * n->H * n->W;
    int rc;
    const float *xd = stage(n, x, n->xbuf, npix * TSURR_CIN * 4, on_device, &rc);
    if (rc) return rc;
    const float *td = stage(n, target, n->tbuf, npix * 3 * 4, on_device, &rc);
    if (rc) return rc;
    const float *md = stage(n, mask, n->mbuf, npix * 4, on_device, &rc);
    if (rc) return rc;
    rc = run_forward(n, xd, B);
    if (rc) return rc;
    SCU(cudaMemsetAsync(n->g, 0, n->nparam * 4, n->s));
    SCU(cudaMemsetAsync(n->msum, 0, 64, n->s));
    SCU(cudaMemsetAsync(n->loss, 0, 64, n->s));
    for (int i = 1; i <= NL; ++i) SCU(cudaMemsetAsync(n->dact[i], 0, act_elems(n, i, B) * sizeof(float), n->s));
    k_mask_sum<<<256, 256, 0, n->s>>>(md, npix, n->msum);
    // output layer: gradient of the loss w.r.t. its (pre-activation) output
    k_loss<<<cdiv(npix, 256), 256, 0, n->s>>>(n->y, td, md, n->msum, npix, n->dpre, n->loss);
    for (int L = NL - 1; L >= 0; --L) {
        Conv c = conv_of(n, L, B);
        const long long nout = (long long)B * c.hout * c.wout * c.cout;
        if (L < NL - 1) {
            float *skipg = n->skip[L] >= 0 ? n->dact[n->skip[L]] : nullptr;
            k_dpre<<<cdiv(nout / 8, 256), 256, 0, n->s>>>(n->dact[L + 1], n->act[L + 1], n->dpre, skipg, nout / 8, 1);
        }
        // weight and bias gradients
        const long long P = (long long)B * c.hout * c.wout;
        if (n->wg_tc[L]) {
            launch_wgrad_tc(n, L, B);
        } else {
            const int splits = (int)std::max<long long>(1, std::min<long long>(256, P / 2048));
            int pps = (int)((P + splits - 1) / splits);
            pps = (pps + BK - 1) / BK * BK;
            dim3 gw(cdiv(c.cout, BM), cdiv(9LL * c.cin, BN), cdiv(P, pps));
            k_conv_wgrad<<<gw, GT, 0, n->s>>>(c, n->dpre, n->g + n->woff[L], pps);
        }
        const long long nvec = P * (c.cout / 8);
        const unsigned bg = (unsigned)std::max<long long>(1, std::min<long long>(cdiv(nvec, 8LL * BG_THREADS),
                                                                                  4LL * n->num_sms));
        k_bias_grad<<<bg, BG_THREADS, 0, n->s>>>(n->dpre, P, c.cout, n->g + n->boff[L]);
        // data gradient towards the layer input (not needed for the network input), on the
        // tensor cores, accumulated into the FP32 gradient of that activation
        if (L > 0) {
            TcGrad d = n->tcd[L];
            d.ntiles = (long long)B * d.nty * d.ntx * d.nph;
            d.acc32 = n->dact[L];
            k_conv_dgrad_tc<<<tc_grid(n, d.N, d.ntiles), TC_THREADS, tc_smem_bytes(d.N, d.cw), n->s>>>(
                n->tmAd[L], n->tmBd[L], d, n->err);
        }
    }
    SCU(cudaGetLastError());
    double l = 0.0;
    SCU(cudaMemcpyAsync(&l, n->loss, sizeof(double), cudaMemcpyDeviceToHost, n->s));
    rc = check_err(n);
    if (rc) return rc;
    if (loss) *loss = l;
    return TSIM_OK;
}

extern "C" int tsurr_adam(tsurr_net *n, float lr, float b1, float b2, float eps, int t)
{
    if (!n || t < 1 || !(lr > 0.f) || !(b1 >= 0.f && b1 < 1.f) || !(b2 >= 0.f && b2 < 1.f) || !(eps > 0.f))
        return sfail(TSIM_ERR_INVALID_ARG, "tsurr_adam: bad arguments");
    const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
    k_adam<<<cdiv(n->nparam, 256), 256, 0, n->s>>>(n->p, n->g, n->m1, n->m2, n->nparam, lr, b1, b2, eps, c1, c2);
    return refresh_weights(n);
}

// ---------------------------------------------------------------- serving helpers

namespace {

// x[b, y, x, :] = [h, px, py, s_0 .. s_8] with px = (x + 0.5) / W * 2 - 1 and
// py = (y + 0.5) / H * 2 - 1: one thread per pixel, three 16-byte stores.
__global__ void k_features(const float *__restrict__ h, const float *__restrict__ sc, long long npix, int H, int W,
                           float *__restrict__ x)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= npix) return;
    const long long hw = (long long)H * W;
    const long long b = t / hw;
    const int rem = (int)(t - b * hw);
    const int yy = rem / W, xx = rem - yy * W;
    const float *s = sc + b * 9;
    float4 *o = reinterpret_cast<float4 *>(x + t * 12);
    o[0] = make_float4(h[t], ((float)xx + 0.5f) / (float)W * 2.f - 1.f, ((float)yy + 0.5f) / (float)H * 2.f - 1.f,
                       s[0]);
    o[1] = make_float4(s[1], s[2], s[3], s[4]);
    o[2] = make_float4(s[5], s[6], s[7], s[8]);
}

// One CTA per frame: sqrt(mean over the pixels of y[..., 3]^2) / press.
__global__ void __launch_bounds__(256) k_indicator(const float *__restrict__ y, const float *__restrict__ press,
                                                   int HW, float *__restrict__ out)
{
    __shared__ float part[8];
    const float *yb = y + (long long)blockIdx.x * HW * 4;
    float s = 0.f;
    for (int p = threadIdx.x; p < HW; p += blockDim.x) {
        const float e = yb[(long long)p * 4 + 3];
        s = fmaf(e, e, s);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float a = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) a += part[w];
        out[blockIdx.x] = sqrtf(a / (float)HW) / press[blockIdx.x];
    }
}

}  // namespace

extern "C" int tsurr_features(const float *height, const float *scalars, int batch, int height_px, int width_px,
                              float *x, void *stream)
{
    if (!height || !scalars || !x || batch < 1 || height_px < 1 || width_px < 1)
        return sfail(TSIM_ERR_INVALID_ARG, "tsurr_features: bad arguments");
    if ((uintptr_t)x % 16 != 0) return sfail(TSIM_ERR_INVALID_ARG, "tsurr_features: x must be 16-byte aligned");
    const long long npix = (long long)batch * height_px * width_px;
    k_features<<<(unsigned int)((npix + 255) / 256), 256, 0, (cudaStream_t)stream>>>(height, scalars, npix, height_px,
                                                                                    width_px, x);
    SCU(cudaGetLastError());
    return TSIM_OK;
}

extern "C" int tsurr_indicator(const float *y, const float *press, int batch, int height_px, int width_px,
                               float *out, void *stream)
{
    if (!y || !press || !out || batch < 1 || height_px < 1 || width_px < 1)
        return sfail(TSIM_ERR_INVALID_ARG, "tsurr_indicator: bad arguments");
    k_indicator<<<batch, 256, 0, (cudaStream_t)stream>>>(y, press, height_px * width_px, out);
    SCU(cudaGetLastError());
    return TSIM_OK;
}
