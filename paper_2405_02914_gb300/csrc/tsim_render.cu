// tsim_render.cu -- sm_103a kernels of the sensor image: a path tracer over
// the elastomer surface's height field (Sec. III-B: reverse rays from the
// camera, diffuse reflections at the rough membrane, attenuation per
// reflection, what reaches the LEDs), and the image metrics MSE, PSNR and
// SSIM (Sec. IV).
//
// Model: the surface is z = h(x, y), bilinear over the readout grid (pixel
// (i, j) at ((j + 0.5) p, (i + 0.5) p)), clamped at the edges, its normal
// from central differences over +-p/2; the Lambertian membrane (albedo per
// pixel) is seen from the gel below by an orthographic camera, one jittered
// primary hit per sample.  Each reflection takes a cosine-weighted
// direction about the inner normal; a path ends on the nearest LED (a
// one-sided rectangle c +- u +- v emitting L on the side of u x v: it adds
// throughput x L), on the absorbing floor z = z_floor, or after
// max_bounces reflections; it meets the membrane again where z - h first
// turns >= 0 (steps of p/2 within the height range of h, 12 bisections).
// Random numbers: SplitMix64 (Steele, Lea and Flood, OOPSLA 2014) of the
// counter ((pixel * spp + s) * 32 + bounce) * 4 + dim, as 24-bit uniforms.
//
// One CTA of one warp per 32 samples of a pixel, summed with shuffles and
// float atomics into the pixel.  The path tracer is bound by ALU and L1 latency
// (the height field of a 128 x 128 readout is 64 KB, cache-resident).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <string>

#include "../../include/tsim.h"

namespace trender {


struct Desc {
    float c[TSIM_MAX_LEDS][3], u[TSIM_MAX_LEDS][3], v[TSIM_MAX_LEDS][3], L[TSIM_MAX_LEDS][3];
    float e[TSIM_MAX_LEDS][3];          // u x v
    float iu2[TSIM_MAX_LEDS], iv2[TSIM_MAX_LEDS];
    int n_lights, spp, max_bounces;
    float z_floor;
    unsigned long long seed;
};

__device__ float g_hrange[2];                       // min, max of the current height field
__device__ double g_sum[2];                         // metric accumulators

__device__ __forceinline__ float uniform24(unsigned long long seed, unsigned long long counter)
{
    unsigned long long z = seed + (counter + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z = z ^ (z >> 31);
    return (float)(z >> 40) * (1.0f / 16777216.0f);
}

struct Surf {
    const float *h, *alb;
    int W, H;
    float p, inv_p, hmin, hmax;
};

__device__ __forceinline__ float height(const Surf &s, float x, float y)
{
    const float u = fminf(fmaxf(x * s.inv_p - 0.5f, 0.f), (float)(s.W - 1));
    const float v = fminf(fmaxf(y * s.inv_p - 0.5f, 0.f), (float)(s.H - 1));
    const int j0 = min((int)floorf(u), s.W - 2), i0 = min((int)floorf(v), s.H - 2);
    const float fu = u - (float)j0, fv = v - (float)i0;
    const float *r0 = s.h + (long long)i0 * s.W, *r1 = r0 + s.W;
    const float a = (1.f - fu) * __ldg(r0 + j0) + fu * __ldg(r0 + j0 + 1);
    const float b = (1.f - fu) * __ldg(r1 + j0) + fu * __ldg(r1 + j0 + 1);
    return (1.f - fv) * a + fv * b;
}

__device__ __forceinline__ void normal_at(const Surf &s, float x, float y, float n[3])
{
    const float hp = 0.5f * s.p;
    const float gx = (height(s, x + hp, y) - height(s, x - hp, y)) * s.inv_p;
    const float gy = (height(s, x, y + hp) - height(s, x, y - hp)) * s.inv_p;
    const float il = rsqrtf(gx * gx + gy * gy + 1.f);
    n[0] = -gx * il; n[1] = -gy * il; n[2] = il;
}

__device__ __forceinline__ const float *albedo_at(const Surf &s, float x, float y)
{
    const int j = min(max((int)floorf(x * s.inv_p), 0), s.W - 1), i = min(max((int)floorf(y * s.inv_p), 0), s.H - 1);
    return s.alb + ((long long)i * s.W + j) * 3;
}

// cosine-weighted direction about the unit normal m, in the orthonormal
// basis of Duff et al. (JCGT 2017), continuous in m away from m_z = 0
__device__ __forceinline__ void cosine_dir(const float m[3], float u0, float u1, float w[3])
{
    const float sg = m[2] >= 0.f ? 1.f : -1.f;
    const float a = -1.f / (sg + m[2]), bb = m[0] * m[1] * a;
    const float t[3] = {1.f + sg * m[0] * m[0] * a, sg * bb, -sg * m[0]};
    const float b[3] = {bb, sg + m[1] * m[1] * a, -m[1]};
    float sn, cs;
    sincospif(2.f * u1, &sn, &cs);
    const float r = sqrtf(u0), z = sqrtf(1.f - u0);
    for (int k = 0; k < 3; ++k) w[k] = r * cs * t[k] + r * sn * b[k] + z * m[k];
}

// nearest LED along P + t w (emitting side only), or -1
__device__ __forceinline__ int hit_light(const Desc &d, const float P[3], const float w[3], float &tbest)
{
    int best = -1;
    for (int k = 0; k < d.n_lights; ++k) {
        const float we = w[0] * d.e[k][0] + w[1] * d.e[k][1] + w[2] * d.e[k][2];
        if (!(we < 0.f)) continue;
        const float t = ((d.c[k][0] - P[0]) * d.e[k][0] + (d.c[k][1] - P[1]) * d.e[k][1] +
                         (d.c[k][2] - P[2]) * d.e[k][2]) / we;
        if (!(t > 0.f) || !(t < tbest)) continue;
        const float q[3] = {P[0] + t * w[0] - d.c[k][0], P[1] + t * w[1] - d.c[k][1], P[2] + t * w[2] - d.c[k][2]};
        const float a = (q[0] * d.u[k][0] + q[1] * d.u[k][1] + q[2] * d.u[k][2]) * d.iu2[k];
        const float b = (q[0] * d.v[k][0] + q[1] * d.v[k][1] + q[2] * d.v[k][2]) * d.iv2[k];
        if (fabsf(a) <= 1.f && fabsf(b) <= 1.f) { tbest = t; best = k; }
    }
    return best;
}

// first return of P + t w to the membrane for 0 < t < tmax, or -1
__device__ __forceinline__ float hit_surface(const Surf &s, const float P[3], const float w[3], float tmax)
{
    float tend = tmax;
    if (w[2] < 0.f) tend = fminf(tend, (s.hmin - P[2]) / w[2]);
    else if (w[2] > 0.f) tend = fminf(tend, (s.hmax - P[2]) / w[2]);
    const float dt = 0.5f * s.p;
    float t0 = 0.f;
    for (int it = 0; it < 4096; ++it) {
        const float t1 = t0 + dt;
        if (t1 > tend) return -1.f;
        const float f = P[2] + t1 * w[2] - height(s, P[0] + t1 * w[0], P[1] + t1 * w[1]);
        if (f >= 0.f) {
            float lo = t0, hi = t1;
            for (int k = 0; k < 12; ++k) {
                const float tm = 0.5f * (lo + hi);
                const float fm = P[2] + tm * w[2] - height(s, P[0] + tm * w[0], P[1] + tm * w[1]);
                if (fm >= 0.f) hi = tm; else lo = tm;
            }
            return hi;
        }
        t0 = t1;
    }
    return -1.f;
}

__device__ __forceinline__ void trace(const Surf &sf, const Desc &d, int i, int j, int s, float out[3])
{
    const unsigned long long base =
        ((unsigned long long)((long long)i * sf.W + j) * (unsigned long long)d.spp + (unsigned long long)s) * 32ull;
    const float x = ((float)j + uniform24(d.seed, base * 4 + 0)) * sf.p;
    const float y = ((float)i + uniform24(d.seed, base * 4 + 1)) * sf.p;
    float P[3] = {x, y, height(sf, x, y)}, n[3], T[3];
    normal_at(sf, x, y, n);
    const float *a = albedo_at(sf, x, y);
    for (int k = 0; k < 3; ++k) { T[k] = __ldg(a + k); out[k] = 0.f; }
    for (int b = 0; b < d.max_bounces && b < 32; ++b) {
        const unsigned long long key = (base + (unsigned long long)b) * 4;
        const float m[3] = {-n[0], -n[1], -n[2]};
        float w[3];
        cosine_dir(m, uniform24(d.seed, key + 2), uniform24(d.seed, key + 3), w);
        float tb = 3.0e38f;
        int lk = hit_light(d, P, w, tb);
        if (w[2] < 0.f) {
            const float tf = (d.z_floor - P[2]) / w[2];
            if (tf < tb) { tb = tf; lk = -1; }
        }
        const float ts = hit_surface(sf, P, w, tb);
        if (ts > 0.f) {
            P[0] += ts * w[0]; P[1] += ts * w[1];
            P[2] = height(sf, P[0], P[1]);
            normal_at(sf, P[0], P[1], n);
            a = albedo_at(sf, P[0], P[1]);
            for (int k = 0; k < 3; ++k) T[k] *= __ldg(a + k);
            continue;
        }
        if (lk >= 0)
            for (int k = 0; k < 3; ++k) out[k] += T[k] * d.L[lk][k];
        break;
    }
}

// min and max of the height field (one CTA)
__global__ void __launch_bounds__(1024) k_hrange(const float *h, long long n)
{
    __shared__ float smin[32], smax[32];
    float lo = 3.0e38f, hi = -3.0e38f;
    for (long long q = threadIdx.x; q < n; q += blockDim.x) {
        const float v = h[q];
        lo = fminf(lo, v);
        hi = fmaxf(hi, v);
    }
    for (int o = 16; o > 0; o >>= 1) {
        lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if ((threadIdx.x & 31) == 0) { smin[threadIdx.x >> 5] = lo; smax[threadIdx.x >> 5] = hi; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < (int)(blockDim.x >> 5); ++k) { lo = fminf(lo, smin[k]); hi = fmaxf(hi, smax[k]); }
        g_hrange[0] = fminf(lo, smin[0]);
        g_hrange[1] = fmaxf(hi, smax[0]);
    }
}

// one CTA of one warp per 32 samples of a pixel (blockIdx.x: pixel,
// blockIdx.y: group of 32 samples): a lane traces one path, the warp sums
// them with shuffles and adds its share to the pixel (zeroed before).  A
// CTA holds its registers until its slowest path ends, so small CTAs keep
// the SMs busy when path lengths vary.
__global__ void __launch_bounds__(32) k_render(const float *h, const float *alb, int W, int H, float p, Desc d,
                                               float *rgb)
{
    const int pix = blockIdx.x, lane = threadIdx.x, s = blockIdx.y * 32 + lane;
    const int i = pix / W, j = pix - i * W;
    const Surf sf = {h, alb, W, H, p, 1.f / p, g_hrange[0], g_hrange[1]};
    float acc[3] = {0.f, 0.f, 0.f};
    if (s < d.spp) trace(sf, d, i, j, s, acc);
    for (int k = 0; k < 3; ++k)
        for (int off = 16; off > 0; off >>= 1) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], off);
    if (lane < 3)
        atomicAdd(rgb + (long long)pix * 3 + lane, (lane == 0 ? acc[0] : lane == 1 ? acc[1] : acc[2]) / (float)d.spp);
}

// ---------------------------------------------------------------- metrics

__global__ void k_metrics_zero() { g_sum[0] = 0.0; g_sum[1] = 0.0; }

__device__ __forceinline__ void block_add(double v, double *dst)
{
    __shared__ double red[32];
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        atomicAdd(dst, s);
    }
}

// sum of squared differences
__global__ void __launch_bounds__(256) k_sqdiff(const float *a, const float *b, long long n)
{
    double s = 0.0;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        const double d = (double)a[q] - (double)b[q];
        s += d * d;
    }
    block_add(s, &g_sum[0]);
}

// SSIM of each window inside the image, one thread per (window, channel):
// Gaussian 11 x 11 (sigma 1.5) weighted means, variances and covariance
__global__ void __launch_bounds__(256) k_ssim(const float *a, const float *b, int W, int H, int C, float c1, float c2)
{
    __shared__ float g[11];
    if (threadIdx.x < 11) {
        float s = 0.f;
        for (int k = 0; k < 11; ++k) s += expf(-(float)((k - 5) * (k - 5)) / 4.5f);
        g[threadIdx.x] = expf(-(float)((threadIdx.x - 5) * (threadIdx.x - 5)) / 4.5f) / s;
    }
    __syncthreads();
    const int ow = W - 10, oh = H - 10;
    const long long n = (long long)ow * oh * C;
    double local = 0.0;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(q % C), j = (int)((q / C) % ow), i = (int)(q / ((long long)C * ow));
        float mx = 0.f, my = 0.f, sxx = 0.f, syy = 0.f, sxy = 0.f;
        for (int u = 0; u < 11; ++u)
            for (int v = 0; v < 11; ++v) {
                const float w = g[u] * g[v];
                const long long o = ((long long)(i + u) * W + j + v) * C + c;
                const float x = a[o], y = b[o];
                mx += w * x; my += w * y;
                sxx += w * x * x; syy += w * y * y; sxy += w * x * y;
            }
        const float vx = sxx - mx * mx, vy = syy - my * my, cxy = sxy - mx * my;
        local += (double)(((2.f * mx * my + c1) * (2.f * cxy + c2)) / ((mx * mx + my * my + c1) * (vx + vy + c2)));
    }
    block_add(local, &g_sum[1]);
}

static int device_array(const void *p)
{
    cudaPointerAttributes at;
    if (!p || cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace trender

void tsim_record_error(const std::string &msg);

using namespace trender;

extern "C" int tsim_render(const float *height, const float *albedo, int W, int H, float pitch,
                           const tsim_render_desc *desc, float *rgb, void *stream)
{
    if (!desc || W < 2 || H < 2 || !(pitch > 0.f) || desc->spp < 1 || desc->max_bounces < 1 ||
        desc->max_bounces > 32 || desc->n_lights < 0 || desc->n_lights > TSIM_MAX_LEDS) {
        tsim_record_error("tsim_render: W, H >= 2, pitch > 0, spp >= 1, 1 <= max_bounces <= 32, 0..4 LEDs");
        return TSIM_ERR_INVALID_ARG;
    }
    if (!device_array(height) || !device_array(albedo) || !device_array(rgb) ||
        ((uintptr_t)height | (uintptr_t)albedo | (uintptr_t)rgb) % 4) {
        tsim_record_error("tsim_render: height, albedo and rgb must be 4-byte aligned device arrays");
        return TSIM_ERR_INVALID_ARG;
    }
    Desc d{};
    for (int k = 0; k < desc->n_lights; ++k) {
        const float *u = desc->u[k], *v = desc->v[k];
        for (int a = 0; a < 3; ++a) {
            d.c[k][a] = desc->c[k][a]; d.u[k][a] = u[a]; d.v[k][a] = v[a]; d.L[k][a] = desc->L[k][a];
        }
        d.e[k][0] = u[1] * v[2] - u[2] * v[1];
        d.e[k][1] = u[2] * v[0] - u[0] * v[2];
        d.e[k][2] = u[0] * v[1] - u[1] * v[0];
        const float uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2], vv = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
        if (!(uu > 0.f) || !(vv > 0.f)) {
            tsim_record_error("tsim_render: an LED has a zero edge");
            return TSIM_ERR_INVALID_ARG;
        }
        d.iu2[k] = 1.f / uu;
        d.iv2[k] = 1.f / vv;
    }
    d.n_lights = desc->n_lights;
    d.spp = desc->spp;
    d.max_bounces = desc->max_bounces;
    d.z_floor = desc->z_floor;
    d.seed = (unsigned long long)desc->seed;
    cudaStream_t s = (cudaStream_t)stream;
    k_hrange<<<1, 1024, 0, s>>>(height, (long long)W * H);
    cudaMemsetAsync(rgb, 0, sizeof(float) * 3 * (size_t)W * H, s);
    k_render<<<dim3((unsigned int)(W * H), (unsigned int)((desc->spp + 31) / 32)), 32, 0, s>>>(height, albedo, W, H,
                                                                                             pitch, d, rgb);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        tsim_record_error(std::string("tsim_render: ") + cudaGetErrorString(e));
        return TSIM_ERR_CUDA;
    }
    return TSIM_OK;
}

extern "C" int tsim_image_metrics(const float *a, const float *b, int W, int H, int C, float max_value, double *out,
                                  void *stream)
{
    if (!out || W < 11 || H < 11 || C < 1 || !(max_value > 0.f)) {
        tsim_record_error("tsim_image_metrics: images of at least 11 x 11, C >= 1, max_value > 0, out given");
        return TSIM_ERR_INVALID_ARG;
    }
    if (!device_array(a) || !device_array(b) || ((uintptr_t)a | (uintptr_t)b) % 4) {
        tsim_record_error("tsim_image_metrics: a and b must be 4-byte aligned device arrays");
        return TSIM_ERR_INVALID_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const long long n = (long long)W * H * C;
    const float c1 = (0.01f * max_value) * (0.01f * max_value), c2 = (0.03f * max_value) * (0.03f * max_value);
    k_metrics_zero<<<1, 1, 0, s>>>();
    k_sqdiff<<<(unsigned int)std::min<long long>((n + 255) / 256, 1216), 256, 0, s>>>(a, b, n);
    const long long nw = (long long)(W - 10) * (H - 10) * C;
    k_ssim<<<(unsigned int)std::min<long long>((nw + 255) / 256, 1216), 256, 0, s>>>(a, b, W, H, C, c1, c2);
    double sums[2];
    cudaError_t e = cudaMemcpyFromSymbolAsync(sums, g_sum, sizeof(sums), 0, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        tsim_record_error(std::string("tsim_image_metrics: ") + cudaGetErrorString(e));
        return TSIM_ERR_CUDA;
    }
    out[0] = sums[0] / (double)n;
    out[1] = out[0] > 0.0 ? 10.0 * log10((double)max_value * max_value / out[0]) : INFINITY;
    out[2] = sums[1] / (double)nw;
    return TSIM_OK;
}
