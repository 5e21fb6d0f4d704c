// mslice_rotate.cu -- frame rotation of the index volume (Eq. 2-3): the
// lab-frame volume n(X, Y, Z) = R_pitch(alpha_i) R_yaw(psi) n(x, y, z) by
// trilinear resampling of the sample-frame volume, and its transpose.
//
// Axes (x, z, y): x along the beam (slice j, x = j Delta), z the surface normal
// (row l, z = l dz), y in plane (column m, y = m dy); both volumes use that
// lattice.  With M = R_pitch(alpha) R_yaw(psi),
//   R_pitch: x' = cos(a) x - sin(a) z,  z' = sin(a) x + cos(a) z
//   R_yaw:   x' = cos(p) x - sin(p) y,  y' = sin(p) x + cos(p) y
// the lab voxel at r samples the sample volume at s = c + M^T (r - c): the
// surface rises along +x by tan(alpha), so a straight beam along +x meets it
// from above at alpha, and a sample feature drifts toward +y by tan(psi).
// Indices are clamped to [0, n-1] per axis (the volume extends past its faces
// by its edge values: substrate below, vacuum above).
//
// Precision.  The fractional sample index f = b + A (j, l, m) is formed
// without FP32 cancellation: the row part b + A_j j + A_l l in FP64 once per
// row and lane, split into an integer and a float fraction; the column part
// A_m m as hi * m + lo * m with hi carrying 12 significant bits, so hi * m is
// exact in FP32 for m < 2^12, and its fraction is taken exactly.  The weights
// are then good to about 1e-7 absolute, at any volume size.
//
// The forward is bound by HBM: 8 B read (mostly from L2: neighbouring lab
// voxels share sample voxels) and 8 B written per voxel.  The transpose is a
// gather: every sample voxel sums, in a fixed order, the lab voxels whose
// stencils touch it, each stencil recomputed as the forward computes it, so
// its result is bitwise reproducible (no atomics).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "mslice.h"

namespace {

struct RotMap {
    double b[3];        // f_k = b_k + A[k][0] j + A[k][1] l + A[k][2] m
    double A[3][2];     // the row coefficients (j, l)
    float hi[3], lo[3]; // A[k][2] = hi + lo, hi with 12 significant bits
    int n[3];           // ns, nz, ny
    float Af[3][3];     // A in FP32 (lab-index steps of the fractional sample index)
    float C[3][3];      // A^-1 (sample-index steps of the lab index), for the gather's candidate box
    float inv_ay;       // 1 / A[2][2] (0 when |A[2][2]| <= 1e-3: every lab column is a candidate)
    int fmin[3], fmax[3];    // range of the fractional sample index over the lab volume (its corners)
    int y_identity;     // f_y = m exactly and f_x, f_z independent of m (no yaw): the y stencil is the identity
};

// fraction-split index of one axis: lower lattice index and upper weight,
// clamped to the volume
__device__ __forceinline__ void axis_stencil(int ri, float rf, float hi, float lo, int m, int n, int& i0, int& i1,
                                             float& w) {
    const float t = hi * (float)m;          // exact: 12-bit hi times m < 2^12
    const float ti = floorf(t);
    const float frac = rf + (t - ti) + lo * (float)m;
    const float fi = floorf(frac);
    const int i = ri + (int)ti + (int)fi;
    w = frac - fi;
    // past a face: the face value itself, with weight 0 on a neighbour (so
    // that the edge value passes through exactly)
    if (i < 0) {
        i0 = 0;
        w = 0.f;
    } else if (i >= n - 1) {
        i0 = n - 1;
        w = 0.f;
    } else {
        i0 = i;
    }
    i1 = i0 + 1 < n ? i0 + 1 : n - 1;
}

struct Stencil {
    size_t a00, a01, a10, a11;   // sample rows (x0,z0) (x0,z1) (x1,z0) (x1,z1)
    int y0, y1;
    float w000, w001, w100, w101, wy;
};

__device__ __forceinline__ Stencil stencil(const RotMap& R, const int (&ri)[3], const float (&rf)[3], int m) {
    int x0, x1, z0, z1;
    float wx, wz;
    Stencil S;
    axis_stencil(ri[0], rf[0], R.hi[0], R.lo[0], m, R.n[0], x0, x1, wx);
    axis_stencil(ri[1], rf[1], R.hi[1], R.lo[1], m, R.n[1], z0, z1, wz);
    axis_stencil(ri[2], rf[2], R.hi[2], R.lo[2], m, R.n[2], S.y0, S.y1, S.wy);
    const size_t plane = (size_t)R.n[1] * R.n[2];
    S.a00 = (size_t)x0 * plane + (size_t)z0 * R.n[2];
    S.a01 = (size_t)x0 * plane + (size_t)z1 * R.n[2];
    S.a10 = (size_t)x1 * plane + (size_t)z0 * R.n[2];
    S.a11 = (size_t)x1 * plane + (size_t)z1 * R.n[2];
    S.w000 = (1.f - wx) * (1.f - wz);
    S.w001 = (1.f - wx) * wz;
    S.w100 = wx * (1.f - wz);
    S.w101 = wx * wz;
    return S;
}

__device__ __forceinline__ float2 lerp_y(const float2* __restrict__ in, size_t a, const Stencil& S) {
    const float2 v0 = __ldg(in + a + S.y0), v1 = __ldg(in + a + S.y1);
    return make_float2(fmaf(S.wy, v1.x - v0.x, v0.x), fmaf(S.wy, v1.y - v0.y, v0.y));
}

__device__ __forceinline__ float2 gather(const float2* __restrict__ in, const Stencil& S) {
    const float2 p00 = lerp_y(in, S.a00, S), p01 = lerp_y(in, S.a01, S);
    const float2 p10 = lerp_y(in, S.a10, S), p11 = lerp_y(in, S.a11, S);
    return make_float2(S.w000 * p00.x + S.w001 * p01.x + S.w100 * p10.x + S.w101 * p11.x,
                       S.w000 * p00.y + S.w001 * p01.y + S.w100 * p10.y + S.w101 * p11.y);
}

// one warp per lab row (j, l), lanes along y, two voxels per lane and step
// (their loads in flight together).  Lanes 0..2 form the row's FP64 index
// terms, one axis each, and pass them to the warp.
__global__ void __launch_bounds__(256) k_rotate(const float2* __restrict__ in, float2* __restrict__ out,
                                                const RotMap R) {
    const int lane = threadIdx.x & 31;
    const unsigned rows = (unsigned)R.n[0] * (unsigned)R.n[1];
    const unsigned warps = gridDim.x * (blockDim.x >> 5);
    const int ny = R.n[2];
    for (unsigned row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); row < rows; row += warps) {
        const unsigned j = row / (unsigned)R.n[1], l = row - j * (unsigned)R.n[1];
        int ri_k = 0;
        float rf_k = 0.f;
        if (lane < 3) {
            const double b = lane == 0 ? R.b[0] : (lane == 1 ? R.b[1] : R.b[2]);
            const double aj = lane == 0 ? R.A[0][0] : (lane == 1 ? R.A[1][0] : R.A[2][0]);
            const double al = lane == 0 ? R.A[0][1] : (lane == 1 ? R.A[1][1] : R.A[2][1]);
            const double f = fma(al, (double)l, fma(aj, (double)j, b));
            const double fl = floor(f);
            ri_k = (int)fl;
            rf_k = (float)(f - fl);
        }
        int ri[3];
        float rf[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            ri[k] = __shfl_sync(0xffffffffu, ri_k, k);
            rf[k] = __shfl_sync(0xffffffffu, rf_k, k);
        }
        const size_t o = (size_t)row * ny;
        for (int m = lane; m < ny; m += 64) {
            const bool two = m + 32 < ny;
            const Stencil S0 = stencil(R, ri, rf, m);
            const Stencil S1 = stencil(R, ri, rf, two ? m + 32 : m);
            const float2 v0 = gather(in, S0);
            const float2 v1 = gather(in, S1);
            out[o + m] = v0;
            if (two) out[o + m + 32] = v1;
        }
    }
}

// The forward without yaw (RotMap::y_identity): the y stencil is the identity
// (lower index m, weight 0) and the x and z stencils do not depend on m, so
// every voxel of lab row (j, l) takes the same four sample rows with the same
// four weights.  One warp per lab row, the stencil formed once, four columns
// per lane in flight; the sum w000 p00 + w001 p01 + w100 p10 + w101 p11 is
// k_rotate's with p = v0 + 0 (v1 - v0) = v0, the same value for finite data.
__global__ void __launch_bounds__(256) k_rotate_xz(const float2* __restrict__ in, float2* __restrict__ out,
                                                   const RotMap R) {
    const int lane = threadIdx.x & 31;
    const unsigned rows = (unsigned)R.n[0] * (unsigned)R.n[1];
    const unsigned warps = gridDim.x * (blockDim.x >> 5);
    const int ny = R.n[2];
    for (unsigned row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); row < rows; row += warps) {
        const unsigned j = row / (unsigned)R.n[1], l = row - j * (unsigned)R.n[1];
        int ri_k = 0;
        float rf_k = 0.f;
        if (lane < 3) {
            const double b = lane == 0 ? R.b[0] : (lane == 1 ? R.b[1] : R.b[2]);
            const double aj = lane == 0 ? R.A[0][0] : (lane == 1 ? R.A[1][0] : R.A[2][0]);
            const double al = lane == 0 ? R.A[0][1] : (lane == 1 ? R.A[1][1] : R.A[2][1]);
            const double f = fma(al, (double)l, fma(aj, (double)j, b));
            const double fl = floor(f);
            ri_k = (int)fl;
            rf_k = (float)(f - fl);
        }
        int ri[3];
        float rf[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            ri[k] = __shfl_sync(0xffffffffu, ri_k, k);
            rf[k] = __shfl_sync(0xffffffffu, rf_k, k);
        }
        const Stencil S = stencil(R, ri, rf, 0);   // x and z parts: the same for every column
        const float2 *p00 = in + S.a00, *p01 = in + S.a01, *p10 = in + S.a10, *p11 = in + S.a11;
        float2* o = out + (size_t)row * ny;
        for (int m0 = 0; m0 < ny; m0 += 128) {
            float2 v[4][4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int m = m0 + 32 * c + lane;
                if (m < ny) {
                    v[c][0] = __ldg(p00 + m);
                    v[c][1] = __ldg(p01 + m);
                    v[c][2] = __ldg(p10 + m);
                    v[c][3] = __ldg(p11 + m);
                }
            }
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int m = m0 + 32 * c + lane;
                if (m < ny)
                    o[m] = make_float2(S.w000 * v[c][0].x + S.w001 * v[c][1].x + S.w100 * v[c][2].x + S.w101 * v[c][3].x,
                                       S.w000 * v[c][0].y + S.w001 * v[c][1].y + S.w100 * v[c][2].y + S.w101 * v[c][3].y);
            }
        }
    }
}

// weight of sample index s in the stencil of lab column m along one axis:
// axis_stencil's arithmetic with the indices kept as exact integers in FP32
// (|index| < 2^24), so that no conversion is needed (ri, m, n, s as floats)
__device__ __forceinline__ float axis_weight(float ri, float rf, float hi, float lo, float m, float n, float s) {
    const float t = hi * m;
    const float ti = floorf(t);
    const float frac = rf + (t - ti) + lo * m;
    const float fi = floorf(frac);
    const float i = ri + ti + fi;
    float w = frac - fi, i0 = i;
    if (i < 0.f) {
        i0 = 0.f;
        w = 0.f;
    } else if (i >= n - 1.f) {
        i0 = n - 1.f;
        w = 0.f;
    }
    const float i1 = i0 + 1.f < n ? i0 + 1.f : n - 1.f;
    return (i0 == s ? 1.f - w : 0.f) + (i1 == s ? w : 0.f);
}

// lab-offset range [lo, hi] of one lab axis i reaching the sample window
// D_k = [dlo_k, dhi_k] (infinite at the volume's faces) through C
__device__ __forceinline__ void lab_range(const float (&C)[3], const float (&dlo)[3], const float (&dhi)[3],
                                          float& lo, float& hi) {
    lo = 0.f;
    hi = 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if (C[k] == 0.f) continue;
        const float a = C[k] * dlo[k], b = C[k] * dhi[k];
        lo += fminf(a, b);
        hi += fmaxf(a, b);
    }
}

// Transpose R^T as a gather: one warp per sample row (x, z), lanes along y in
// chunks of 32.  The lab row (x, z) is the reference: its FP64 index terms
// are formed once, as the forward forms them, and a candidate lab row
// (x + dx, z + dz) takes them plus FP32 offsets.  For each candidate lab voxel
// the three axis stencils are computed as in the forward and the weight of
// this sample voxel is its product; the candidates are visited in a fixed
// order (dx, dz, then lab column), so the sum is bitwise reproducible.  A
// sample voxel on a y face takes every lab column past the face (up to the
// volume's y shift, ~90 columns at 0.5 deg yaw over 1024 slices): the whole
// warp walks such a window, and a fixed xor tree adds the lanes' partial sums
// (also reproducible), instead of one lane walking it while 31 wait.  The
// candidate box is the lab image of the sample window [s - 1, s + 1] per axis
// (at the volume's faces, where the forward clamps, out to the farthest index
// a lab voxel reaches), with a tolerance of 1e-3 index units; the window's
// offsets from the reference are integer differences plus the FP32 fraction,
// so the tolerance holds at any volume size.
__global__ void __launch_bounds__(256) k_rotate_gather(const float2* __restrict__ g_lab,
                                                       float2* __restrict__ g_sample, const RotMap R) {
    const int lane = threadIdx.x & 31;
    const unsigned rows = (unsigned)R.n[0] * (unsigned)R.n[1];
    const unsigned warps = gridDim.x * (blockDim.x >> 5);
    const int ns = R.n[0], nz = R.n[1], ny = R.n[2];
    for (unsigned row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); row < rows; row += warps) {
        const int sx = (int)(row / (unsigned)nz), sz = (int)(row - (unsigned)sx * (unsigned)nz);
        // reference lab row (sx, sz): integer and fraction of each axis's row term
        int ri_k = 0;
        float rf_k = 0.f;
        if (lane < 3) {
            const double b = lane == 0 ? R.b[0] : (lane == 1 ? R.b[1] : R.b[2]);
            const double aj = lane == 0 ? R.A[0][0] : (lane == 1 ? R.A[1][0] : R.A[2][0]);
            const double al = lane == 0 ? R.A[0][1] : (lane == 1 ? R.A[1][1] : R.A[2][1]);
            const double f = fma(al, (double)sz, fma(aj, (double)sx, b));
            const double fl = floor(f);
            ri_k = (int)fl;
            rf_k = (float)(f - fl);
        }
        int ri[3];
        float rf[3], rif[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            ri[k] = __shfl_sync(0xffffffffu, ri_k, k);
            rf[k] = __shfl_sync(0xffffffffu, rf_k, k);
            rif[k] = (float)ri[k];
        }
        const float sxf = (float)sx, szf = (float)sz, nsf = (float)ns, nzf = (float)nz, nyf = (float)ny;
        // sample window of the row, relative to the reference's row terms
        // (integer difference, then the fraction)
        const float dxlo = (float)((sx == 0 ? min(R.fmin[0], -1) : sx - 1) - ri[0]) - rf[0];
        const float dxhi = (float)((sx == ns - 1 ? max(R.fmax[0], ns) : sx + 1) - ri[0]) - rf[0];
        const float dzlo = (float)((sz == 0 ? min(R.fmin[1], -1) : sz - 1) - ri[1]) - rf[1];
        const float dzhi = (float)((sz == nz - 1 ? max(R.fmax[1], nz) : sz + 1) - ri[1]) - rf[1];
        const float tol = 1e-3f;
        for (int c0 = 0; c0 < ny; c0 += 32) {
            const int sy = c0 + lane;
            const bool active = sy < ny;
            const float syf = (float)sy;
            const int ylast = c0 + 31 < ny - 1 ? c0 + 31 : ny - 1;
            // the warp's candidate rows: the lab image of the chunk's window
            const float dlo[3] = {dxlo, dzlo, (float)((c0 == 0 ? min(R.fmin[2], -1) : c0 - 1) - ri[2]) - rf[2]};
            const float dhi[3] = {dxhi, dzhi, (float)((ylast == ny - 1 ? max(R.fmax[2], ny) : ylast + 1) - ri[2]) - rf[2]};
            float xlo, xhi, zlo, zhi;
            lab_range(R.C[0], dlo, dhi, xlo, xhi);
            lab_range(R.C[1], dlo, dhi, zlo, zhi);
            const int dx0 = (int)fmaxf(ceilf(xlo - tol), (float)-sx), dx1 = (int)fminf(floorf(xhi + tol), (float)(ns - 1 - sx));
            const int dz0 = (int)fmaxf(ceilf(zlo - tol), (float)-sz), dz1 = (int)fminf(floorf(zhi + tol), (float)(nz - 1 - sz));
            // this lane's window along y
            const float ylo = (float)((sy == 0 ? min(R.fmin[2], -1) : sy - 1) - ri[2]) - rf[2];
            const float yhi = (float)((sy == ny - 1 ? max(R.fmax[2], ny) : sy + 1) - ri[2]) - rf[2];
            // the candidate rows in order; for each, this lane's lab columns in
            // order.  A wide window (a sample voxel on a y face, which takes
            // every lab column past that face) is walked by the whole warp, and
            // a fixed xor tree sums the lanes' partial sums into the owner's.
            float2 acc = make_float2(0.f, 0.f);
            for (int dx = dx0; dx <= dx1; ++dx) {
                for (int dz = dz0; dz <= dz1; ++dz) {
                    float rfc[3];
#pragma unroll
                    for (int k = 0; k < 3; ++k) rfc[k] = rf[k] + R.Af[k][0] * (float)dx + R.Af[k][1] * (float)dz;
                    const float2* src = g_lab + ((size_t)(sx + dx) * nz + (size_t)(sz + dz)) * ny;
                    // lab columns whose y index can reach sy: A_y2 m in the window less the row offset
                    int m0 = 0, m1 = -1;
                    if (active) {
                        const float off = R.Af[2][0] * (float)dx + R.Af[2][1] * (float)dz;
                        m1 = ny - 1;
                        if (R.inv_ay != 0.f) {
                            float a = (ylo - off) * R.inv_ay, b = (yhi - off) * R.inv_ay;
                            if (a > b) { const float tmp = a; a = b; b = tmp; }
                            m0 = (int)fmaxf(ceilf(a - tol), 0.f);
                            m1 = (int)fminf(floorf(b + tol), (float)(ny - 1));
                        }
                    }
                    const bool wide = m1 - m0 >= 3;
                    if (!wide) {
                        float mf = (float)m0;
                        for (int m = m0; m <= m1; ++m, mf += 1.f) {
                            const float wy = axis_weight(rif[2], rfc[2], R.hi[2], R.lo[2], mf, nyf, syf);
                            const float wx = axis_weight(rif[0], rfc[0], R.hi[0], R.lo[0], mf, nsf, sxf);
                            const float wz = axis_weight(rif[1], rfc[1], R.hi[1], R.lo[1], mf, nzf, szf);
                            const float wt = (wx * wz) * wy;
                            if (wt != 0.f) {
                                const float2 g = __ldg(src + m);
                                acc.x = fmaf(wt, g.x, acc.x);
                                acc.y = fmaf(wt, g.y, acc.y);
                            }
                        }
                    }
                    unsigned wm = __ballot_sync(0xffffffffu, wide);
                    while (wm) {
                        const int L = __ffs(wm) - 1;
                        wm &= wm - 1;
                        const int w0 = __shfl_sync(0xffffffffu, m0, L), w1 = __shfl_sync(0xffffffffu, m1, L);
                        const float syL = __shfl_sync(0xffffffffu, syf, L);
                        float2 part = make_float2(0.f, 0.f);
                        for (int m = w0 + lane; m <= w1; m += 32) {
                            const float mf = (float)m;
                            const float wy = axis_weight(rif[2], rfc[2], R.hi[2], R.lo[2], mf, nyf, syL);
                            const float wx = axis_weight(rif[0], rfc[0], R.hi[0], R.lo[0], mf, nsf, sxf);
                            const float wz = axis_weight(rif[1], rfc[1], R.hi[1], R.lo[1], mf, nzf, szf);
                            const float wt = (wx * wz) * wy;
                            if (wt != 0.f) {
                                const float2 g = __ldg(src + m);
                                part.x = fmaf(wt, g.x, part.x);
                                part.y = fmaf(wt, g.y, part.y);
                            }
                        }
#pragma unroll
                        for (int o = 16; o > 0; o >>= 1) {
                            part.x += __shfl_xor_sync(0xffffffffu, part.x, o);
                            part.y += __shfl_xor_sync(0xffffffffu, part.y, o);
                        }
                        if (lane == L) {
                            acc.x += part.x;
                            acc.y += part.y;
                        }
                    }
                }
            }
            if (active) g_sample[(size_t)row * ny + sy] = acc;
        }
    }
}

// dst[c] (+)= sum over the CNT listed lab rows, in list order, of lw[k] times
// row k's column (lane + 32 c), onto 0 (first) or onto dst's own earlier sum:
// four column chunks at a time, every row's loads before the sums
template <int CNT>
__device__ __forceinline__ void sum_rows(const float2* __restrict__ g_lab, float2* __restrict__ dst,
                                         const unsigned (&lrow)[4], const float (&lw)[4], int ny, int nc, int lane,
                                         bool first) {
    for (int c0 = 0; c0 < nc; c0 += 4) {
        float2 g[CNT > 0 ? CNT : 1][4];
#pragma unroll
        for (int k = 0; k < CNT; ++k) {
            const float2* src = g_lab + (size_t)lrow[k] * ny + lane + 32 * c0;
#pragma unroll
            for (int c = 0; c < 4; ++c)
                g[k][c] = (c0 + c < nc && lane + 32 * (c0 + c) < ny) ? __ldg(src + 32 * c) : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            if (c0 + c >= nc || lane + 32 * (c0 + c) >= ny) continue;
            float2 a = first ? make_float2(0.f, 0.f) : dst[32 * (c0 + c)];
#pragma unroll
            for (int k = 0; k < CNT; ++k) {
                a.x = fmaf(lw[k], g[k][c].x, a.x);
                a.y = fmaf(lw[k], g[k][c].y, a.y);
            }
            dst[32 * (c0 + c)] = a;
        }
    }
}

// The transpose without yaw (RotMap::y_identity): the y stencil is the
// identity (weight 1 at m = sy, 0 at its neighbour), and the x and z stencils
// do not depend on m, so a candidate lab row (x + dx, z + dz) adds its column
// sy with one weight wx wz for the whole row.  One warp per sample row: the
// candidate rows are weighed once, and the contributing ones are summed over
// all the row's columns (lane c holds columns c, c + 32, ...).  The candidate
// rows, their weights and the order of the sum are those of k_rotate_gather,
// which gives bitwise the same sums (up to the sign of zero sums).
__global__ void __launch_bounds__(256, 3) k_rotate_gather_xz(const float2* __restrict__ g_lab,
                                                          float2* __restrict__ g_sample, const RotMap R) {
    const int lane = threadIdx.x & 31;
    const unsigned rows = (unsigned)R.n[0] * (unsigned)R.n[1];
    const unsigned warps = gridDim.x * (blockDim.x >> 5);
    const int ns = R.n[0], nz = R.n[1], ny = R.n[2];
    const int nc = (ny + 31) >> 5;   // <= 32 column chunks
    for (unsigned row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); row < rows; row += warps) {
        const int sx = (int)(row / (unsigned)nz), sz = (int)(row - (unsigned)sx * (unsigned)nz);
        int ri_k = 0;
        float rf_k = 0.f;
        if (lane < 2) {
            const double b = lane == 0 ? R.b[0] : R.b[1];
            const double aj = lane == 0 ? R.A[0][0] : R.A[1][0];
            const double al = lane == 0 ? R.A[0][1] : R.A[1][1];
            const double f = fma(al, (double)sz, fma(aj, (double)sx, b));
            const double fl = floor(f);
            ri_k = (int)fl;
            rf_k = (float)(f - fl);
        }
        int ri[2];
        float rf[2], rif[2];
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            ri[k] = __shfl_sync(0xffffffffu, ri_k, k);
            rf[k] = __shfl_sync(0xffffffffu, rf_k, k);
            rif[k] = (float)ri[k];
        }
        const float sxf = (float)sx, szf = (float)sz, nsf = (float)ns, nzf = (float)nz;
        const float dlo[3] = {(float)((sx == 0 ? min(R.fmin[0], -1) : sx - 1) - ri[0]) - rf[0],
                              (float)((sz == 0 ? min(R.fmin[1], -1) : sz - 1) - ri[1]) - rf[1], 0.f};
        const float dhi[3] = {(float)((sx == ns - 1 ? max(R.fmax[0], ns) : sx + 1) - ri[0]) - rf[0],
                              (float)((sz == nz - 1 ? max(R.fmax[1], nz) : sz + 1) - ri[1]) - rf[1], 0.f};
        const float tol = 1e-3f;
        float xlo, xhi, zlo, zhi;
        lab_range(R.C[0], dlo, dhi, xlo, xhi);
        lab_range(R.C[1], dlo, dhi, zlo, zhi);
        const int dx0 = (int)fmaxf(ceilf(xlo - tol), (float)-sx), dx1 = (int)fminf(floorf(xhi + tol), (float)(ns - 1 - sx));
        const int dz0 = (int)fmaxf(ceilf(zlo - tol), (float)-sz), dz1 = (int)fminf(floorf(zhi + tol), (float)(nz - 1 - sz));
        float2* dst = g_sample + (size_t)row * ny + lane;
        // the contributing rows (nonzero weight) in candidate order, four at
        // a time (2 to 4 in all away from the faces; a sample row on an x or z
        // face takes every lab row past that face), each batch summed onto
        // the previous batches' sums
        int dx = dz0 <= dz1 ? dx0 : dx1 + 1, dz = dz0;   // an empty z range: no candidates
        bool first = true;
        for (;;) {
            unsigned lrow[4] = {0u, 0u, 0u, 0u};
            float lw[4] = {0.f, 0.f, 0.f, 0.f};
            int cnt = 0;
            while (dx <= dx1 && cnt < 4) {
                const float rfx = rf[0] + R.Af[0][0] * (float)dx + R.Af[0][1] * (float)dz;
                const float rfz = rf[1] + R.Af[1][0] * (float)dx + R.Af[1][1] * (float)dz;
                const float wx = axis_weight(rif[0], rfx, R.hi[0], R.lo[0], 0.f, nsf, sxf);
                const float wz = axis_weight(rif[1], rfz, R.hi[1], R.lo[1], 0.f, nzf, szf);
                const float wt = wx * wz;
                if (wt != 0.f) {   // uniform over the warp
                    const unsigned r = (unsigned)(sx + dx) * (unsigned)nz + (unsigned)(sz + dz);
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        if (k == cnt) {
                            lrow[k] = r;
                            lw[k] = wt;
                        }
                    }
                    ++cnt;
                }
                if (++dz > dz1) { dz = dz0; ++dx; }
            }
            if (cnt == 0 && !first) break;
            switch (cnt) {   // uniform over the warp
                case 0: sum_rows<0>(g_lab, dst, lrow, lw, ny, nc, lane, first); break;
                case 1: sum_rows<1>(g_lab, dst, lrow, lw, ny, nc, lane, first); break;
                case 2: sum_rows<2>(g_lab, dst, lrow, lw, ny, nc, lane, first); break;
                case 3: sum_rows<3>(g_lab, dst, lrow, lw, ny, nc, lane, first); break;
                default: sum_rows<4>(g_lab, dst, lrow, lw, ny, nc, lane, first); break;
            }
            first = false;
            if (dx > dx1) break;
        }
    }
}

// 12-significant-bit head of a (the tail a - head is exact in double)
double head12(double a) {
    if (a == 0.0 || !isfinite(a)) return 0.0;
    int e;
    frexp(a, &e);
    return ldexp(nearbyint(ldexp(a, 12 - e)), e - 12);
}

int make_map(const mslice_params* p, double alpha, double psi, const double* c, RotMap* R) {
    if (!p || !c) return MSLICE_EINVAL;
    if (p->ns < 1 || p->nz < 1 || p->ny < 1 || p->ny > MSLICE_MAX_N || p->nz > MSLICE_MAX_N) return MSLICE_EINVAL;
    if (!(p->slice_nm > 0) || !(p->dz_nm > 0) || !(p->dy_nm > 0)) return MSLICE_EINVAL;
    if (!isfinite(alpha) || !isfinite(psi) || !isfinite(c[0]) || !isfinite(c[1]) || !isfinite(c[2]))
        return MSLICE_EINVAL;
    const double ca = cos(alpha), sa = sin(alpha), cp = cos(psi), sp = sin(psi);
    // M = R_pitch R_yaw on (x, z, y)
    const double P[3][3] = {{ca, -sa, 0.0}, {sa, ca, 0.0}, {0.0, 0.0, 1.0}};
    const double Y[3][3] = {{cp, 0.0, -sp}, {0.0, 1.0, 0.0}, {sp, 0.0, cp}};
    double M[3][3];
    for (int i = 0; i < 3; ++i)
        for (int k = 0; k < 3; ++k) M[i][k] = P[i][0] * Y[0][k] + P[i][1] * Y[1][k] + P[i][2] * Y[2][k];
    const double sp3[3] = {p->slice_nm, p->dz_nm, p->dy_nm};
    // f_k = (c_k + sum_i M[i][k] (r_i - c_i)) / sp_k,  r_i = idx_i sp_i
    for (int k = 0; k < 3; ++k) {
        double b = c[k];
        for (int i = 0; i < 3; ++i) b -= M[i][k] * c[i];
        R->b[k] = b / sp3[k];
        R->A[k][0] = M[0][k] * sp3[0] / sp3[k];
        R->A[k][1] = M[1][k] * sp3[1] / sp3[k];
        const double am = M[2][k] * sp3[2] / sp3[k];
        const double h = head12(am);
        R->hi[k] = (float)h;
        R->lo[k] = (float)(am - h);
    }
    R->n[0] = p->ns;
    R->n[1] = p->nz;
    R->n[2] = p->ny;
    R->inv_ay = fabs(M[2][2]) > 1e-3 ? (float)(1.0 / M[2][2]) : 0.f;   // A[2][2] = M[2][2]
    // A (f per lab index) and its inverse C = S^-1 M S (M orthogonal): lab
    // index per unit of f, S the spacings
    for (int k = 0; k < 3; ++k)
        for (int i = 0; i < 3; ++i) {
            R->Af[k][i] = (float)(M[i][k] * sp3[i] / sp3[k]);
            R->C[i][k] = (float)(M[i][k] * sp3[k] / sp3[i]);
        }
    // the kernel keeps rows and lattice indices in 32 bits: the map is affine,
    // so its extremes over the volume are at the corners
    if ((double)p->ns * p->nz >= 2147483648.0) return MSLICE_EUNSUPPORTED;
    for (int k = 0; k < 3; ++k) {
        double lo = 0.0, hi = 0.0;
        for (int cj = 0; cj < 2; ++cj)
            for (int cl = 0; cl < 2; ++cl)
                for (int cm = 0; cm < 2; ++cm) {
                    const double f = R->b[k] + R->A[k][0] * (cj ? p->ns - 1 : 0) + R->A[k][1] * (cl ? p->nz - 1 : 0) +
                                     ((double)R->hi[k] + R->lo[k]) * (cm ? p->ny - 1 : 0);
                    if (!(fabs(f) < 1073741824.0)) return MSLICE_EUNSUPPORTED;
                    if ((cj | cl | cm) == 0 || f < lo) lo = f;
                    if ((cj | cl | cm) == 0 || f > hi) hi = f;
                }
        // the gather's face windows reach the extreme index of the lab volume
        R->fmin[k] = (int)floor(lo) - 1;
        R->fmax[k] = (int)ceil(hi) + 1;
    }
    R->y_identity = R->hi[0] == 0.f && R->lo[0] == 0.f && R->hi[1] == 0.f && R->lo[1] == 0.f && R->A[2][0] == 0.0 &&
                    R->A[2][1] == 0.0 && R->b[2] == 0.0 && R->hi[2] == 1.f && R->lo[2] == 0.f &&
                    R->C[0][2] == 0.f && R->C[1][2] == 0.f;
    return MSLICE_OK;
}

int device_sms() {
    static int cache[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
    if (cache[dev] <= 0 && cudaDeviceGetAttribute(&cache[dev], cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 152;
    return cache[dev] > 0 ? cache[dev] : 152;
}

int launch(const mslice_params* p, double alpha, double psi, const double* c, const float* in, float* out,
           bool adjoint, void* stream) {
    RotMap R;
    int rc = make_map(p, alpha, psi, c, &R);
    if (rc) return rc;
    if (!in || !out || in == out || ((uintptr_t)in & 7) || ((uintptr_t)out & 7)) return MSLICE_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    const long long rows = (long long)p->ns * p->nz;
    const long long cap = (long long)device_sms() * 32;   // a few waves of 8-warp blocks per SM
    const unsigned blocks = (unsigned)(rows / 8 + 1 < cap ? rows / 8 + 1 : cap);
    if (adjoint) {
        if (R.y_identity)
            k_rotate_gather_xz<<<blocks, 256, 0, st>>>((const float2*)in, (float2*)out, R);
        else
            k_rotate_gather<<<blocks, 256, 0, st>>>((const float2*)in, (float2*)out, R);
    } else {
        if (R.y_identity)
            k_rotate_xz<<<blocks, 256, 0, st>>>((const float2*)in, (float2*)out, R);
        else
            k_rotate<<<blocks, 256, 0, st>>>((const float2*)in, (float2*)out, R);
    }
    return cudaGetLastError() == cudaSuccess ? MSLICE_OK : MSLICE_ELAUNCH;
}

}  // namespace

extern "C" {

int mslice_rotate(const mslice_params* p, double alpha_rad, double psi_rad, const double* center_nm,
                  const float* vol_sample, float* vol_lab, void* stream) {
    return launch(p, alpha_rad, psi_rad, center_nm, vol_sample, vol_lab, false, stream);
}

int mslice_rotate_adjoint(const mslice_params* p, double alpha_rad, double psi_rad, const double* center_nm,
                          const float* g_lab, float* g_sample, void* stream) {
    return launch(p, alpha_rad, psi_rad, center_nm, g_lab, g_sample, true, stream);
}

}  // extern "C"
