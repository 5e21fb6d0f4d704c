// mslice_recon.cu -- reconstruction helpers of libmslice: the coarse-to-fine
// parameter map E (coarse reconstruction voxels onto the multislice grid,
// Sec. 4.1-4.2), its adjoint E^T, and a fused ADAM step (Sec. 4.1).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "mslice.h"

namespace {

bool bad_coarse(const mslice_params* p, const mslice_coarse* c) {
    if (!p || !c) return true;
    if (c->cx < 1 || c->cz < 1 || c->cy < 1 || c->bx < 1 || c->bz < 1 || c->by < 1) return true;
    if (c->x0 < 0 || c->z0 < 0 || c->y0 < 0) return true;
    if ((long)c->x0 + (long)c->cx * c->bx > p->ns) return true;
    if ((long)c->z0 + (long)c->cz * c->bz > p->nz) return true;
    if ((long)c->y0 + (long)c->cy * c->by > p->ny) return true;
    return p->ny < 1 || p->nz < 1 || p->ns < 1;
}

// one block per fine row (x, z) of the coarse block at a time, threads along y
__global__ void k_coarse_to_fine(const float* __restrict__ theta, float2* __restrict__ vol, mslice_coarse c,
                                 int ny, int nz) {
    const int bzs = c.cz * c.bz, bys = c.cy * c.by;
    const long rows = (long)c.cx * c.bx * bzs;
    for (long r = blockIdx.x; r < rows; r += gridDim.x) {
        const int xx = (int)(r / bzs), zz = (int)(r % bzs);
        const float* th = theta + ((size_t)(xx / c.bx) * c.cz + zz / c.bz) * c.cy;
        float2* out = vol + ((size_t)(c.x0 + xx) * nz + (c.z0 + zz)) * ny + c.y0;
        for (int yy = threadIdx.x; yy < bys; yy += blockDim.x) {
            const float d = __ldg(th + yy / c.by);
            out[yy] = make_float2(c.base_delta + d, fmaf(c.beta_ratio, d, c.base_beta));
        }
    }
}

// one thread per coarse voxel, fixed summation order over its block
__global__ void k_fine_to_coarse(const float2* __restrict__ grad, float* __restrict__ g, mslice_coarse c,
                                 int ny, int nz) {
    const long n = (long)c.cx * c.cz * c.cy;
    const long stride = (long)gridDim.x * blockDim.x;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const long cc = i % c.cy, b = (i / c.cy) % c.cz, a = i / ((long)c.cy * c.cz);
        float s = 0.f;
        for (int ix = 0; ix < c.bx; ++ix)
            for (int iz = 0; iz < c.bz; ++iz) {
                const float2* row = grad + ((size_t)(c.x0 + a * c.bx + ix) * nz + (c.z0 + b * c.bz + iz)) * ny +
                                    (c.y0 + cc * c.by);
                for (int iy = 0; iy < c.by; ++iy) {
                    const float2 v = row[iy];
                    s += fmaf(c.beta_ratio, v.y, v.x);
                }
            }
        g[i] = s;
    }
}

__global__ void k_adam(float* __restrict__ th, float* __restrict__ m, float* __restrict__ v,
                       const float* __restrict__ g, size_t n, float lr, float b1, float b2, float eps, float c1,
                       float c2, float lo, float hi) {
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float gi = g[i];
        const float mi = fmaf(b1, m[i], (1.f - b1) * gi);
        const float vi = fmaf(b2, v[i], (1.f - b2) * gi * gi);
        m[i] = mi;
        v[i] = vi;
        float t = th[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        th[i] = fminf(fmaxf(t, lo), hi);
    }
}

struct SnapLevels {
    float v[8];
    int n;
};

// nearest level, the lower one on a tie (levels in any order)
__global__ void k_snap(float* __restrict__ th, size_t n, SnapLevels L) {
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float x = th[i];
        float best = L.v[0], bd = fabsf(x - L.v[0]);
        for (int k = 1; k < L.n; ++k) {
            const float d = fabsf(x - L.v[k]);
            if (d < bd || (d == bd && L.v[k] < best)) {
                bd = d;
                best = L.v[k];
            }
        }
        th[i] = best;
    }
}

// shrink-wrap support update (Sec. 4.2): separable Gaussian blur, maximum,
// threshold.  Products and sums are rounded one by one (no fused
// multiply-add) and taken in tap order, so the support decision is
// reproducible.
constexpr int kMaxTapRadius = 16;
struct Taps {
    float w[2 * kMaxTapRadius + 1];
    int r;
};

__global__ void k_blur_axis(const float* __restrict__ in, float* __restrict__ out, int cx, int cz, int cy, int axis,
                            Taps T) {
    const long n = (long)cx * cz * cy;
    const long stride = axis == 2 ? 1 : (axis == 1 ? cy : (long)cz * cy);
    const int len = axis == 2 ? cy : (axis == 1 ? cz : cx);
    const long gs = (long)gridDim.x * blockDim.x;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gs) {
        const int pos = (int)((i / stride) % len);
        float acc = 0.f;
        for (int t = -T.r; t <= T.r; ++t) {
            const int q = pos + t;
            if (q >= 0 && q < len) acc = __fadd_rn(acc, __fmul_rn(T.w[t + T.r], in[i + (long)t * stride]));
        }
        out[i] = acc;
    }
}

__global__ void __launch_bounds__(1024) k_max(const float* __restrict__ b, long n, float* __restrict__ mx) {
    __shared__ float red[32];
    float m = -INFINITY;
    for (long i = threadIdx.x; i < n; i += blockDim.x) m = fmaxf(m, b[i]);
    for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        m = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : -INFINITY;
        for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (threadIdx.x == 0) *mx = m;
    }
}

__global__ void k_support(float* __restrict__ th, const float* __restrict__ b, long n, const float* __restrict__ mx,
                          float threshold, int* __restrict__ kept) {
    const float thr = __fmul_rn(threshold, *mx);
    const long gs = (long)gridDim.x * blockDim.x;
    int mine = 0;
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gs) {
        if (b[i] >= thr) ++mine;
        else th[i] = 0.f;
    }
    if (kept) {
        for (int o = 16; o; o >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, o);
        if ((threadIdx.x & 31) == 0 && mine) atomicAdd(kept, mine);
    }
}

unsigned blocks_for(size_t n) {
    size_t b = (n + 255) / 256;
    return (unsigned)(b > 4096 ? 4096 : (b ? b : 1));
}

}  // namespace

extern "C" {

int mslice_coarse_to_fine(const mslice_params* p, const mslice_coarse* c, const float* theta, float* vol,
                          void* stream) {
    if (bad_coarse(p, c) || !theta || !vol) return MSLICE_EINVAL;
    const size_t rows = (size_t)c->cx * c->bx * c->cz * c->bz;
    const unsigned nb = (unsigned)(rows < 8192 ? rows : 8192);
    k_coarse_to_fine<<<nb, 256, 0, (cudaStream_t)stream>>>(theta, (float2*)vol, *c, p->ny, p->nz);
    return cudaGetLastError() == cudaSuccess ? MSLICE_OK : MSLICE_ELAUNCH;
}

int mslice_fine_to_coarse(const mslice_params* p, const mslice_coarse* c, const float* grad_vol, float* g_theta,
                          void* stream) {
    if (bad_coarse(p, c) || !grad_vol || !g_theta) return MSLICE_EINVAL;
    const size_t n = (size_t)c->cx * c->cz * c->cy;
    k_fine_to_coarse<<<blocks_for(n), 256, 0, (cudaStream_t)stream>>>((const float2*)grad_vol, g_theta, *c, p->ny,
                                                                      p->nz);
    return cudaGetLastError() == cudaSuccess ? MSLICE_OK : MSLICE_ELAUNCH;
}

int mslice_snap(float* theta, size_t n, const float* levels, int nlevels, void* stream) {
    if (!theta || !levels || nlevels < 1 || nlevels > 8) return MSLICE_EINVAL;
    if (n == 0) return MSLICE_OK;
    SnapLevels L{};
    for (int k = 0; k < nlevels; ++k) L.v[k] = levels[k];
    L.n = nlevels;
    k_snap<<<blocks_for(n), 256, 0, (cudaStream_t)stream>>>(theta, n, L);
    return cudaGetLastError() == cudaSuccess ? MSLICE_OK : MSLICE_ELAUNCH;
}

size_t mslice_shrinkwrap_workspace(size_t n) { return (2 * n + 64) * sizeof(float); }

int mslice_shrinkwrap(float* theta, int cx, int cz, int cy, float sigma, float threshold, int* kept, void* ws,
                      size_t ws_bytes, void* stream) {
    if (!theta || !ws || cx < 1 || cz < 1 || cy < 1 || !(sigma > 0.f) || !(threshold >= 0.f && threshold <= 1.f))
        return MSLICE_EINVAL;
    const size_t n = (size_t)cx * cz * cy;
    if (ws_bytes < mslice_shrinkwrap_workspace(n) || ((uintptr_t)ws & 15)) return MSLICE_EINVAL;
    const int r = (int)floor(3.0 * (double)sigma + 0.5);
    if (r > kMaxTapRadius) return MSLICE_EUNSUPPORTED;
    Taps T{};
    T.r = r;
    double w[2 * kMaxTapRadius + 1], total = 0.0;
    for (int t = -r; t <= r; ++t) {
        w[t + r] = exp(-(double)(t * t) / (2.0 * (double)sigma * (double)sigma));
        total += w[t + r];
    }
    for (int k = 0; k <= 2 * r; ++k) T.w[k] = (float)(w[k] / total);
    cudaStream_t st = (cudaStream_t)stream;
    float* a = (float*)ws;
    float* b = a + n;
    float* mx = b + n;
    if (kept && cudaMemsetAsync(kept, 0, sizeof(int), st) != cudaSuccess) return MSLICE_ELAUNCH;
    k_blur_axis<<<blocks_for(n), 256, 0, st>>>(theta, a, cx, cz, cy, 2, T);
    k_blur_axis<<<blocks_for(n), 256, 0, st>>>(a, b, cx, cz, cy, 1, T);
    k_blur_axis<<<blocks_for(n), 256, 0, st>>>(b, a, cx, cz, cy, 0, T);
    k_max<<<1, 1024, 0, st>>>(a, (long)n, mx);
    k_support<<<blocks_for(n), 256, 0, st>>>(theta, a, (long)n, mx, threshold, kept);
    return cudaGetLastError() == cudaSuccess ? MSLICE_OK : MSLICE_ELAUNCH;
}

int mslice_adam_step(float* theta, float* m, float* v, const float* grad, size_t n, float lr, float b1, float b2,
                     float eps, int t, float lo, float hi, void* stream) {
    if (!theta || !m || !v || !grad || t < 1 || !(b1 >= 0.f && b1 < 1.f) || !(b2 >= 0.f && b2 < 1.f) ||
        !(eps > 0.f) || !(lo <= hi))
        return MSLICE_EINVAL;
    if (n == 0) return MSLICE_OK;
    const float c1 = (float)(1.0 - pow((double)b1, (double)t));
    const float c2 = (float)(1.0 - pow((double)b2, (double)t));
    k_adam<<<blocks_for(n), 256, 0, (cudaStream_t)stream>>>(theta, m, v, grad, n, lr, b1, b2, eps, c1, c2, lo, hi);
    return cudaGetLastError() == cudaSuccess ? MSLICE_OK : MSLICE_ELAUNCH;
}

}  // extern "C"
