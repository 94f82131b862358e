// tsim_noalloc.cu -- a particle-to-grid transfer that allocates nothing.
//
// Some callers cannot call cudaMalloc: a plug-in inside a host application
// that owns all device memory through its own pool, a real-time control loop
// that must not touch the allocator (or wait on its implicit
// synchronisation) once it runs, or a process whose memory budget is fixed
// at start-up.  tsim_p2g_noalloc gives them the particle-to-grid transfer of
// Sec. III-A (Eqs. 1-4) of a particle state they own into a grid buffer they
// own.  Its working memory is the file-scope array below: a fixed
// TSIM_NOALLOC_SCRATCH_BYTES bytes that every GPU which loads this library
// holds until the process exits.  No call allocates, frees, or calls an
// allocating library routine.
//
// Every call uses the same array and leaves its contents behind; the call
// clears what must start at zero itself.  Calls that overlap on the GPU (two
// streams, or two host threads) race on the array and must be serialised by
// the caller.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <mutex>
#include <string>

#include "../../include/tsim.h"
#include "tsim_device.cuh"

using namespace tsim;

namespace {

constexpr int NA_MAX_PARTICLES = TSIM_NOALLOC_MAX_PARTICLES;
constexpr int NA_MAX_BLOCKS = TSIM_NOALLOC_MAX_BLOCKS;
// layout of the scratch array (byte offsets)
constexpr size_t NA_COUNT = 0;
constexpr size_t NA_OFFSET = NA_COUNT + sizeof(int) * NA_MAX_BLOCKS;
constexpr size_t NA_CURSOR = NA_OFFSET + sizeof(int) * NA_MAX_BLOCKS;
constexpr size_t NA_PERM = NA_CURSOR + sizeof(int) * NA_MAX_BLOCKS;
constexpr size_t NA_STATUS = NA_PERM + sizeof(int) * NA_MAX_PARTICLES;
constexpr size_t NA_BYTES = NA_STATUS + 256;
static_assert(NA_BYTES == TSIM_NOALLOC_SCRATCH_BYTES, "scratch size must match tsim.h");

}  // namespace

// The scratch: one copy per device.  With CUDA's lazy module loading (the
// default) the module that holds it is loaded on a device, and the array
// reserved there, at the first call on that device (its
// cudaGetSymbolAddress); that first call may therefore synchronise the
// device and take the array's memory.  In host code this name is only a
// stand-in, never a device address; host code uses the address that
// cudaGetSymbolAddress returns for the current device.
static __device__ __align__(256) unsigned char g_tsim_noalloc_scratch[NA_BYTES];

namespace {

struct NaParams {
    int nx, ny, nz, ox, oy, oz, nbx, nby, n;
    float inv_dx, dx, mp, mu, lam, kME;
};

__global__ void k_na_count(NaParams p, const float *__restrict__ x, unsigned char *scr)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= p.n) return;
    int *count = (int *)(scr + NA_COUNT);
    unsigned int *status = (unsigned int *)(scr + NA_STATUS);
    int ab[3];
    const int nn[3] = {p.nx, p.ny, p.nz}, oo[3] = {p.ox, p.oy, p.oz};
    bool ok = true;
    for (int a = 0; a < 3; ++a) {
        const float xa = x[(long long)t * 3 + a];
        if (!isfinite(xa)) { ok = false; break; }
        int base;
        float f, w[3];
        bspline(xa, p.inv_dx, base, f, w);
        ab[a] = base + oo[a];
        if (ab[a] < 0 || ab[a] + 2 >= nn[a]) ok = false;
    }
    if (!ok) {
        atomicOr(status, ST_DOMAIN);
        return;
    }
    atomicAdd(&count[((ab[2] / BLK) * p.nby + ab[1] / BLK) * p.nbx + ab[0] / BLK], 1);
}

// exclusive scan of the block counts (one CTA of 1024 threads)
__global__ void k_na_scan(int nblocks, unsigned char *scr)
{
    const int *count = (const int *)(scr + NA_COUNT);
    int *offset = (int *)(scr + NA_OFFSET);
    int *cursor = (int *)(scr + NA_CURSOR);
    __shared__ int warp_sum[32];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < nblocks; base += blockDim.x) {
        const int i = base + threadIdx.x;
        const int v = i < nblocks ? count[i] : 0;
        int incl = v;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if ((threadIdx.x & 31) >= o) incl += y;
        }
        if ((threadIdx.x & 31) == 31) warp_sum[threadIdx.x >> 5] = incl;
        __syncthreads();
        if (threadIdx.x < 32) {
            int s = warp_sum[threadIdx.x];
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, s, o);
                if (threadIdx.x >= o) s += y;
            }
            warp_sum[threadIdx.x] = s;
        }
        __syncthreads();
        const int before = (threadIdx.x >= 32 ? warp_sum[(threadIdx.x >> 5) - 1] : 0) + carry;
        if (i < nblocks) {
            offset[i] = before + incl - v;
            cursor[i] = before + incl - v;
        }
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = before + incl;
        __syncthreads();
    }
}

__global__ void k_na_scatter(NaParams p, const float *__restrict__ x, unsigned char *scr)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= p.n) return;
    int *cursor = (int *)(scr + NA_CURSOR);
    int *perm = (int *)(scr + NA_PERM);
    int ab[3];
    const int nn[3] = {p.nx, p.ny, p.nz}, oo[3] = {p.ox, p.oy, p.oz};
    for (int a = 0; a < 3; ++a) {
        const float xa = x[(long long)t * 3 + a];
        if (!isfinite(xa)) return;
        int base;
        float f, w[3];
        bspline(xa, p.inv_dx, base, f, w);
        ab[a] = base + oo[a];
        if (ab[a] < 0 || ab[a] + 2 >= nn[a]) return;
    }
    const int b = ((ab[2] / BLK) * p.nby + ab[1] / BLK) * p.nbx + ab[0] / BLK;
    perm[atomicAdd(&cursor[b], 1)] = t;
}

// One CTA per cell block: P2G (Eqs. 1-4) of the block's particles into a
// shared node window, then one vector atomic per touched node into the grid.
__global__ void __launch_bounds__(128) k_na_p2g(NaParams p, const float *__restrict__ x,
                                                const float *__restrict__ v, const float *__restrict__ C,
                                                const float *__restrict__ F, float4 *grid, unsigned char *scr)
{
    __shared__ float A[4][GAN];
    const int b = blockIdx.x;
    const int *count = (const int *)(scr + NA_COUNT);
    const int *offset = (const int *)(scr + NA_OFFSET);
    const int *perm = (const int *)(scr + NA_PERM);
    unsigned int *status = (unsigned int *)(scr + NA_STATUS);
    const int cnt = count[b], off = offset[b];
    if (cnt == 0) return;
    for (int t = threadIdx.x; t < GAN; t += blockDim.x) { A[0][t] = 0.f; A[1][t] = 0.f; A[2][t] = 0.f; A[3][t] = 0.f; }
    __syncthreads();
    const int gx0 = (b % p.nbx) * BLK, gy0 = ((b / p.nbx) % p.nby) * BLK, gz0 = (b / (p.nbx * p.nby)) * BLK;
    for (int r = threadIdx.x; r < cnt; r += blockDim.x) {
        const long long q = perm[off + r];
        float xp[3], vp[3], Cp[9], Fp[9], tau[9];
        for (int a = 0; a < 3; ++a) { xp[a] = x[q * 3 + a]; vp[a] = v[q * 3 + a]; }
        for (int a = 0; a < 9; ++a) { Cp[a] = C[q * 9 + a]; Fp[a] = F[q * 9 + a]; }
        const float J = kirchhoff(Fp, p.mu, p.lam, tau);
        if (!(J > 0.f) || !isfinite(J)) {
            atomicOr(status, ST_NUMERIC);
            continue;
        }
        int base[3];
        float f[3], w[3][3];
        for (int a = 0; a < 3; ++a) bspline(xp[a], p.inv_dx, base[a], f[a], w[a]);
        // window coordinates of the stencil origin (the particle's base node is inside this block)
        const int wx = base[0] + p.ox - gx0 + 1, wy = base[1] + p.oy - gy0 + 1, wz = base[2] + p.oz - gz0 + 1;
        float Q[9];
        for (int a = 0; a < 9; ++a) Q[a] = p.mp * Cp[a] + p.kME * tau[a];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                for (int k = 0; k < 3; ++k) {
                    const float wt = w[0][i] * w[1][j] * w[2][k];
                    const float d0 = ((float)i - f[0]) * p.dx, d1 = ((float)j - f[1]) * p.dx,
                                d2 = ((float)k - f[2]) * p.dx;
                    const int n = (wz + k) * GAZ + (wy + j) * GA + (wx + i);
                    atomicAdd(&A[0][n], wt * p.mp);
                    atomicAdd(&A[1][n], wt * (p.mp * vp[0] + Q[0] * d0 + Q[1] * d1 + Q[2] * d2));
                    atomicAdd(&A[2][n], wt * (p.mp * vp[1] + Q[3] * d0 + Q[4] * d1 + Q[5] * d2));
                    atomicAdd(&A[3][n], wt * (p.mp * vp[2] + Q[6] * d0 + Q[7] * d1 + Q[8] * d2));
                }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < GA * GA * GA; t += blockDim.x) {
        const int lx = t % GA, ly = (t / GA) % GA, lz = t / (GA * GA);
        const int n = lz * GAZ + ly * GA + lx;
        const float m = A[0][n];
        if (m != 0.f) {
            const int ax = gx0 - 1 + lx, ay = gy0 - 1 + ly, az = gz0 - 1 + lz;
            if (ax >= 0 && ay >= 0 && az >= 0 && ax < p.nx && ay < p.ny && az < p.nz)
                atomicAdd(&grid[((long long)az * p.ny + ay) * p.nx + ax], make_float4(m, A[1][n], A[2][n], A[3][n]));
        }
    }
}

std::mutex na_mu;
void *na_ptr[256] = {};

// Device address of the scratch for the current device, looked up once per
// device with that device current.
cudaError_t scratch_address(unsigned char **out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 256) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> g(na_mu);
    if (!na_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_tsim_noalloc_scratch);
        if (e != cudaSuccess) return e;
        na_ptr[dev] = p;
    }
    *out = (unsigned char *)na_ptr[dev];
    return cudaSuccess;
}

}  // namespace

void tsim_record_error(const std::string &msg);   // tsim_api.cu: the text tsim_last_error returns

namespace {
int na_fail(int code, const std::string &m)
{
    tsim_record_error(m);
    return code;
}
}  // namespace

extern "C" int tsim_p2g_noalloc(const tsim_gel_desc *gel, const tsim_material *mat, float dt, const float *x,
                                const float *v, const float *C, const float *F, int n, float *grid, void *stream)
{
    if (!gel || !mat) return na_fail(TSIM_ERR_INVALID_ARG, "gel and material descriptors are required");
    if (n < 1 || n > NA_MAX_PARTICLES)
        return na_fail(TSIM_ERR_INVALID_ARG, "tsim_p2g_noalloc: n = " + std::to_string(n) +
                                                 " outside 1.." + std::to_string(NA_MAX_PARTICLES) +
                                                 " (the fixed scratch holds at most that many particles)");
    const tsim_gel_desc &g = *gel;
    if (g.nx <= 0 || g.ny <= 0 || g.nz <= 0 || g.nx % BLK || g.ny % BLK || g.nz % BLK || g.ppc <= 0 ||
        !(g.dx > 0.f) || !std::isfinite(g.dx))
        return na_fail(TSIM_ERR_INVALID_ARG, "tsim_p2g_noalloc: node box must be positive multiples of 4, dx > 0");
    const long long nblocks = (long long)(g.nx / BLK) * (g.ny / BLK) * (g.nz / BLK);
    if (nblocks > NA_MAX_BLOCKS)
        return na_fail(TSIM_ERR_INVALID_ARG, "tsim_p2g_noalloc: node box has " + std::to_string(nblocks) +
                                                 " cell blocks, more than the fixed scratch holds (" +
                                                 std::to_string(NA_MAX_BLOCKS) + ")");
    if (!(mat->E > 0.f) || !(mat->nu >= 0.f && mat->nu < 0.5f) || !(mat->rho > 0.f) || !(dt > 0.f))
        return na_fail(TSIM_ERR_INVALID_ARG, "tsim_p2g_noalloc: need E > 0, 0 <= nu < 0.5, rho > 0, dt > 0");
    if (!x || !v || !C || !F || !grid) return na_fail(TSIM_ERR_INVALID_ARG, "tsim_p2g_noalloc: null array");
    // the kernels read x, v, C, F as floats and add to grid with 16-byte vector atomics
    if ((uintptr_t)grid % 16 != 0)
        return na_fail(TSIM_ERR_INVALID_ARG, "tsim_p2g_noalloc: grid must be 16-byte aligned");
    const void *arrays[5] = {x, v, C, F, grid};
    const char *names[5] = {"x", "v", "C", "F", "grid"};
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) return na_fail(TSIM_ERR_CUDA, "tsim_p2g_noalloc: no current device");
    for (int a = 0; a < 5; ++a) {
        if ((uintptr_t)arrays[a] % 4 != 0)
            return na_fail(TSIM_ERR_INVALID_ARG, std::string("tsim_p2g_noalloc: ") + names[a] +
                                                     " must be 4-byte aligned");
        cudaPointerAttributes at{};
        if (cudaPointerGetAttributes(&at, arrays[a]) != cudaSuccess) {
            cudaGetLastError();
            return na_fail(TSIM_ERR_INVALID_ARG, std::string("tsim_p2g_noalloc: ") + names[a] +
                                                     " is not a pointer the CUDA runtime knows");
        }
        const bool ok = at.type == cudaMemoryTypeManaged || (at.type == cudaMemoryTypeDevice && at.device == cur);
        if (!ok)
            return na_fail(TSIM_ERR_INVALID_ARG, std::string("tsim_p2g_noalloc: ") + names[a] +
                                                     " must be device memory of the current device (or managed)");
    }

    unsigned char *scr = nullptr;
    cudaError_t e = scratch_address(&scr);
    if (e != cudaSuccess) return na_fail(TSIM_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    cudaStream_t s = (cudaStream_t)stream;
    const double dx = g.dx, V0 = dx * dx * dx / g.ppc;
    NaParams p;
    p.nx = g.nx; p.ny = g.ny; p.nz = g.nz; p.ox = g.ox; p.oy = g.oy; p.oz = g.oz;
    p.nbx = g.nx / BLK; p.nby = g.ny / BLK; p.n = n;
    p.dx = g.dx;
    p.inv_dx = (float)(1.0 / dx);
    p.mp = (float)(mat->rho * V0);
    p.mu = (float)(mat->E / (2.0 * (1.0 + mat->nu)));
    p.lam = (float)(mat->E * mat->nu / ((1.0 + mat->nu) * (1.0 - 2.0 * mat->nu)));
    p.kME = (float)(-4.0 * dt * V0 / (dx * dx));
    const size_t nodes = (size_t)g.nx * g.ny * g.nz;
    // what must start at zero: the block counts, the status word and the output grid
    if ((e = cudaMemsetAsync(scr + NA_COUNT, 0, sizeof(int) * nblocks, s)) != cudaSuccess ||
        (e = cudaMemsetAsync(scr + NA_STATUS, 0, sizeof(unsigned int), s)) != cudaSuccess ||
        (e = cudaMemsetAsync(grid, 0, sizeof(float4) * nodes, s)) != cudaSuccess)
        return na_fail(TSIM_ERR_CUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
    const unsigned int pb = (unsigned int)((n + 255) / 256);
    k_na_count<<<pb, 256, 0, s>>>(p, x, scr);
    k_na_scan<<<1, 1024, 0, s>>>((int)nblocks, scr);
    k_na_scatter<<<pb, 256, 0, s>>>(p, x, scr);
    k_na_p2g<<<(unsigned int)nblocks, 128, 0, s>>>(p, x, v, C, F, (float4 *)grid, scr);
    if ((e = cudaGetLastError()) != cudaSuccess) return na_fail(TSIM_ERR_CUDA, cudaGetErrorString(e));
    unsigned int status = 0;
    if ((e = cudaMemcpyAsync(&status, scr + NA_STATUS, sizeof(status), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return na_fail(TSIM_ERR_CUDA, cudaGetErrorString(e));
    if (status & ST_NUMERIC) return na_fail(TSIM_ERR_NUMERIC, "tsim_p2g_noalloc: J <= 0 or non-finite F");
    if (status & ST_DOMAIN) return na_fail(TSIM_ERR_DOMAIN, "tsim_p2g_noalloc: a particle lies outside the node box");
    return TSIM_OK;
}
