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
