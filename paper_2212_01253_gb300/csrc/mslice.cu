// mslice.cu -- host side of libmslice: the C ABI of include/mslice.h, plan and
// workspace layout, launch sequencing of the persistent kernels, the FP64
// set-up and transmission kernels, and tracing.  The slice-step device code
// is in mslice_device.cuh; its size-specialised instances are compiled in
// separate translation units (mslice_inst.cu, one per row length).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "mslice.h"
#include "mslice_slice.cuh"
#include "mslice_kernels.h"

namespace {

// ---------------------------------------------------------------------------
// FP64 set-up of the constant arrays
// ---------------------------------------------------------------------------
struct SetupArgs {
    int ny, nz, nw;
    double slice_nm, wavelength_nm, dy_nm, dz_nm;
    double sin_alpha[MSLICE_MAX_ANGLES];
    double sin_psi[MSLICE_MAX_ANGLES];
    float2* tab;       // Wt_y | Wt_z | P_y/ny | P_z/nz
    float2* tab_half;  // the same with P over Delta/2, or null
    float2* probe_z;   // [nw][nz]
    float2* probe_y;   // [nw][ny] exp(-i k sin(psi_w) y_m)
    float2* py_out;    // optional, unnormalised
    float2* pz_out;
    float2* probe_z_out;
};

// stage-2 twiddle for table slot i of a length-n transform: exp(-2 pi i b r2 / n)
__device__ float2 twiddle_entry(int i, int n) {
    if (n <= 32) return make_float2(1.f, 0.f);
    const int r2 = i / 32, b = i % 32;
    double s, c;
    sincospi(2.0 * (double)(b * r2) / (double)n, &s, &c);
    return make_float2((float)c, (float)(-s));
}

// exp(-i Delta k_f^2 / 2k) with k_f = 2 pi f / (n d): phase = pi Delta lambda f^2 / (n d)^2
__device__ double2 propagator_entry(int m, int n, double d, double slice, double lam) {
    const int f = (m < (n + 1) / 2) ? m : m - n;
    const double nd = (double)n * d;
    const double x = slice * lam * (double)f * (double)f / (nd * nd);
    double s, c;
    sincospi(x, &s, &c);
    return make_double2(c, -s);
}

__global__ void k_setup(const SetupArgs S) {
    const int ny = S.ny, nz = S.nz;
    const int total = 2 * (ny + nz) + S.nw * (nz + ny);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        if (i < ny) {
            S.tab[i] = twiddle_entry(i, ny);
            if (S.tab_half) S.tab_half[i] = S.tab[i];
        } else if (i < ny + nz) {
            S.tab[i] = twiddle_entry(i - ny, nz);
            if (S.tab_half) S.tab_half[i] = S.tab[i];
        } else if (i < 2 * ny + nz) {
            const int m = i - ny - nz;
            const double2 p = propagator_entry(m, ny, S.dy_nm, S.slice_nm, S.wavelength_nm);
            S.tab[i] = make_float2((float)(p.x / ny), (float)(p.y / ny));
            if (S.py_out) S.py_out[m] = make_float2((float)p.x, (float)p.y);
            if (S.tab_half) {
                const double2 h = propagator_entry(m, ny, S.dy_nm, 0.5 * S.slice_nm, S.wavelength_nm);
                S.tab_half[i] = make_float2((float)(h.x / ny), (float)(h.y / ny));
            }
        } else if (i < 2 * (ny + nz)) {
            const int l = i - 2 * ny - nz;
            const double2 p = propagator_entry(l, nz, S.dz_nm, S.slice_nm, S.wavelength_nm);
            S.tab[i] = make_float2((float)(p.x / nz), (float)(p.y / nz));
            if (S.pz_out) S.pz_out[l] = make_float2((float)p.x, (float)p.y);
            if (S.tab_half) {
                const double2 h = propagator_entry(l, nz, S.dz_nm, 0.5 * S.slice_nm, S.wavelength_nm);
                S.tab_half[i] = make_float2((float)(h.x / nz), (float)(h.y / nz));
            }
        } else if (i >= 2 * (ny + nz) + S.nw * nz) {
            // exp(-i k sin(psi_w) y_m) = exp(-i pi (2 sin(psi_w) m dy / lambda))
            const int q = i - 2 * (ny + nz) - S.nw * nz;
            const int w = q / ny, m = q % ny;
            double s, c;
            sincospi(2.0 * S.sin_psi[w] * (double)m * S.dy_nm / S.wavelength_nm, &s, &c);
            S.probe_y[q] = make_float2((float)c, (float)(-s));
        } else {
            const int q = i - 2 * (ny + nz);
            const int w = q / nz, l = q % nz;
            // exp(-i k sin(alpha) z_l) = exp(-i pi (2 sin(alpha) l dz / lambda))
            double s, c;
            sincospi(2.0 * S.sin_alpha[w] * (double)l * S.dz_nm / S.wavelength_nm, &s, &c);
            const float2 v = make_float2((float)c, (float)(-s));
            S.probe_z[q] = v;
            if (S.probe_z_out) S.probe_z_out[q] = v;
        }
    }
}

// Angular-spectrum propagator over Delta on the 2-D frequency grid, in FP64:
// exp(i Delta (sqrt(k^2 - kp^2) - k)) = exp(-i Delta kp^2 / (sqrt(k^2 - kp^2) + k))
// (no cancellation), and exp(-Delta sqrt(kp^2 - k^2)) exp(-i Delta k) past
// kp = k (evanescent); stored / (ny nz) for the unnormalised transforms.
__global__ void k_setup_p2d(float2* __restrict__ p2d, int ny, int nz, double dy, double dz, double slice,
                            double lam) {
    const double k = 2.0 * M_PI / lam;
    const size_t n = (size_t)ny * nz;
    const double inv = 1.0 / ((double)ny * (double)nz);
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int l = (int)(i / ny), m = (int)(i % ny);
        const int fy = (m < (ny + 1) / 2) ? m : m - ny, fz = (l < (nz + 1) / 2) ? l : l - nz;
        const double ky = 2.0 * M_PI * fy / (ny * dy), kz = 2.0 * M_PI * fz / (nz * dz);
        const double kp2 = ky * ky + kz * kz;
        double s, c, amp = inv;
        if (kp2 < k * k) {
            sincos(-slice * kp2 / (sqrt(k * k - kp2) + k), &s, &c);
        } else {
            amp *= exp(-slice * sqrt(kp2 - k * k));
            sincos(-slice * k, &s, &c);
        }
        p2d[i] = make_float2((float)(amp * c), (float)(amp * s));
    }
}

// t = exp(-i k Delta (delta - i beta)) = exp(-k Delta beta) (cos(k Delta delta) - i sin(...)).
// The phase arguments k Delta delta and k Delta beta are products with the
// FP64 constant k Delta = kd_hi + kd_lo (two floats): fmaf(v, kd_hi, v * kd_lo)
// is within one float ulp of the FP64 product, without FP64 arithmetic per
// voxel.  Two voxels per thread and iteration (16-byte accesses).
// exact 1 - n^2 (Eq. 1): t = exp(-i kd (w - w^2/2)), w = delta - i beta, i.e. the
// linearised form evaluated at delta' = delta - (delta^2 - beta^2)/2 and
// beta' = beta (1 - delta)
__device__ __forceinline__ float2 exact_dbeta(float d, float b) {
    return make_float2(d - 0.5f * (d * d - b * b), b * (1.f - d));
}

// t of one voxel (minus_one = 0), or u = t - 1 (minus_one = 1) computed without
// cancellation.  With phi = kd delta, b = kd beta, A = exp(-b) and
// (sh, ch) = (sin, cos)(phi / 2): sin phi = 2 sh ch, cos phi - 1 = -2 sh^2, so
// Re u = (A - 1) - 2 A sh^2 with A - 1 = expm1(-b), Im u = -2 A sh ch.  The
// slice loops apply t as a + a u: for the weak scatterers here |u| ~ 1e-2, so
// FP32 holds u to ~1e-10 absolute where it holds t only to ~3e-8, an error
// that would otherwise repeat in every slice of a uniform material.
__device__ __forceinline__ float2 trans_value(float d, float b, float kd_hi, float kd_lo, int minus_one) {
    float sh, ch;
    sincosf(fmaf(d, 0.5f * kd_hi, d * (0.5f * kd_lo)), &sh, &ch);   // phi / 2 (exact halving)
    const float at = fmaf(b, kd_hi, b * kd_lo);
    const float em1 = expm1f(-at), a = 1.f + em1;
    const float two_sh = 2.f * sh;
    if (!minus_one) return make_float2(a * fmaf(-two_sh, sh, 1.f), -a * two_sh * ch);
    return make_float2(fmaf(-a * two_sh, sh, em1), -a * two_sh * ch);
}

__global__ void k_transmission(const float4* __restrict__ vol, float4* __restrict__ tv, size_t n2, float kd_hi,
                               float kd_lo, int exact, int minus_one) {
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += stride) {
        float4 v = __ldcs(vol + i);
        if (exact) {
            const float2 e0 = exact_dbeta(v.x, v.y), e1 = exact_dbeta(v.z, v.w);
            v = make_float4(e0.x, e0.y, e1.x, e1.y);
        }
        const float2 t0 = trans_value(v.x, v.y, kd_hi, kd_lo, minus_one);
        const float2 t1 = trans_value(v.z, v.w, kd_hi, kd_lo, minus_one);
        __stcg(tv + i, make_float4(t0.x, t0.y, t1.x, t1.y));
    }
}

// odd voxel count: the last voxel
__global__ void k_transmission_tail(const float2* __restrict__ vol, float2* __restrict__ tv, float kd_hi,
                                    float kd_lo, int exact, int minus_one) {
    const float2 v = exact ? exact_dbeta(vol[0].x, vol[0].y) : vol[0];
    tv[0] = trans_value(v.x, v.y, kd_hi, kd_lo, minus_one);
}

// g_psi = 2 dL/dI Psi: vector-Jacobian product of I = |Psi|^2
__global__ void k_intensity_vjp(const float2* __restrict__ psi, const float* __restrict__ dI,
                                float2* __restrict__ g, size_t n) {
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        g[i] = cscale(__ldg(psi + i), 2.f * __ldg(dI + i));
}

__global__ void k_debug_wait(unsigned* ctrl, unsigned withhold, long long timeout_ns) {
    __shared__ int s_ok;
    Grid grid{ctrl, gridDim.x, 0u, timeout_ns, &s_ok};
    if (!grid.sync(withhold)) return;
    grid.finish();
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
bool is_pow2(int n) { return n >= 1 && (n & (n - 1)) == 0; }
size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

int validate(const mslice_params* p) {
    if (!p) return MSLICE_EINVAL;
    if (!is_pow2(p->ny) || !is_pow2(p->nz) || p->ny > MSLICE_MAX_N || p->nz > MSLICE_MAX_N) return MSLICE_EINVAL;
    if (p->ns < 1 || p->nw < 1 || p->nw > MSLICE_MAX_ANGLES) return MSLICE_EINVAL;
    if (!(p->wavelength_nm > 0) || !(p->slice_nm > 0) || !(p->dy_nm > 0) || !(p->dz_nm > 0)) return MSLICE_EINVAL;
    for (int w = 0; w < p->nw; ++w)
        if (!(fabs(p->alpha_i_rad[w]) < 1.5707963)) return MSLICE_EINVAL;
    for (int w = 0; w < p->nw; ++w)
        if (!(fabs(p->psi_rad[w]) < 0.1)) return MSLICE_EINVAL;
    if (p->flags & ~(MSLICE_EXIT_WAVE | MSLICE_PER_STRUCTURE | MSLICE_EXACT_TRANSMISSION | MSLICE_STRANG |
                     MSLICE_ANGULAR))
        return MSLICE_EINVAL;
    if (p->grid_blocks < 0 || p->col_width < 0 || p->schedule < 0 || p->schedule > 2) return MSLICE_EINVAL;
    if (p->col_width > 0 && !col_cw_ok(p->col_width, p->nz > 32 ? p->nz / 32 : 1)) return MSLICE_EINVAL;
    return MSLICE_OK;
}

struct Layout {
    size_t ctrl, partials, tab, probe_z, probe_y, tvol, field, gfield, gpart, ckpt, seg;
    size_t tab_half, probe_half, zero_t;  // symmetric splitting only (0 otherwise)
    size_t p2d;                           // angular spectrum only (0 otherwise)
    size_t p2d_half;                      // angular spectrum with the symmetric splitting
    size_t loss_task, loss_wsum;          // one-pass loss partials (loss + gradient)
    size_t total;
    int K, nseg;
};

Layout make_layout(const mslice_params* p, int op) {
    Layout L{};
    const size_t npx = (size_t)p->ny * p->nz;
    const size_t fb = (size_t)p->nw * npx * sizeof(float2);
    L.K = p->checkpoint_every > 0 ? p->checkpoint_every : 32;
    if (L.K > p->ns) L.K = p->ns;
    L.nseg = (p->ns + L.K - 1) / L.K;
    size_t off = 0;
    L.ctrl = off; off = align256(off + kCtrlBytes);
    L.partials = off; off = align256(off + kPartialBytes);
    L.tab = off; off = align256(off + 2 * (size_t)(p->ny + p->nz) * sizeof(float2));
    L.probe_z = off; off = align256(off + (size_t)p->nw * p->nz * sizeof(float2));
    L.probe_y = off; off = align256(off + (size_t)p->nw * p->ny * sizeof(float2));
    const size_t nvol = (p->flags & MSLICE_PER_STRUCTURE) ? (size_t)p->nw : 1;
    L.tvol = off; off = align256(off + nvol * p->ns * npx * sizeof(float2));
    L.field = off; off = align256(off + fb);
    if (p->flags & MSLICE_ANGULAR) {
        L.p2d = off; off = align256(off + npx * sizeof(float2));
        if (p->flags & MSLICE_STRANG) {
            L.p2d_half = off; off = align256(off + npx * sizeof(float2));
        }
    }
    if (p->flags & MSLICE_STRANG) {
        L.tab_half = off; off = align256(off + 2 * (size_t)(p->ny + p->nz) * sizeof(float2));
        L.probe_half = off; off = align256(off + fb);
        L.zero_t = off; off = align256(off + npx * sizeof(float2));
    }
    if (op == MSLICE_OP_ADJOINT || op == MSLICE_OP_LOSS_GRAD) {
        L.gfield = off; off = align256(off + fb);
        // per-wavefield gradient partials, double-buffered by slice parity
        // (one-pass loop, and the split-phase schedule of the two-pass loop)
        L.gpart = off; off = align256(off + (p->nw > 1 && !(p->flags & MSLICE_PER_STRUCTURE) ? 2 * fb : 0));
        L.ckpt = off; off = align256(off + (size_t)L.nseg * fb);
        L.seg = off; off = align256(off + (size_t)L.K * fb);
        // one FP64 partial per task of the detector pass (<= nw max(ny, nz)
        // tasks on either axis) and per-wavefield sums
        const size_t nmax = (size_t)(p->ny > p->nz ? p->ny : p->nz);
        L.loss_task = off; off = align256(off + (size_t)p->nw * nmax * sizeof(double));
        L.loss_wsum = off; off = align256(off + (size_t)p->nw * sizeof(double));
    }
    L.total = off;
    return L;
}

size_t smem_bytes(int ny, int nz, int cw) {
    // tables, with room for the second propagator of the one-pass last slice
    const size_t tabs = 3 * (size_t)(ny + nz) * sizeof(float2);
    size_t row = 0, col = 0;
    if (ny > 32) row = (size_t)(MS_THREADS / (ny / 32)) * (ny + ny / 32) * sizeof(float2);
    if (nz > 32) {
        const int T = nz / 32, groups = MS_THREADS / (cw * T);
        col = (size_t)groups * cw * col_rs(nz, cw) * sizeof(float2);
    }
    return tabs + (row > col ? row : col);
}

// last failing CUDA runtime call, for mslice_last_cuda_error()
thread_local char g_err[160] = "";
bool note(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return false;
    snprintf(g_err, sizeof(g_err), "%s: %s (%d)", what, cudaGetErrorString(e), (int)e);
    return true;
}

struct DevInfo {
    bool init = false;
    int sms = 0;
    int occ = 0;
};
DevInfo g_dev[64];

// persistent kernels used by one call: the slice loops (size-specialised when
// an instance exists, generic otherwise) and the once-per-call kernels
using KernelSet = ms_kernel_set;

// the size-specialised instance when there is one (the angular spectrum: the
// two-pass kernels with the column pass on (k_y, k_z)), else the run-time-size
// kernels
KernelSet sweep_kernels(int ny, int nz, bool angular) {
    KernelSet ks = angular ? ms_generic_kernels_angular() : ms_generic_kernels_paraxial();
    ms_kernel_pair k{nullptr, nullptr};
    switch (ny) {
        case 64: k = angular ? ms_sweep_kernels_as_ny64(nz) : ms_sweep_kernels_ny64(nz); break;
        case 128: k = angular ? ms_sweep_kernels_as_ny128(nz) : ms_sweep_kernels_ny128(nz); break;
        case 256: k = angular ? ms_sweep_kernels_as_ny256(nz) : ms_sweep_kernels_ny256(nz); break;
        case 512: k = angular ? ms_sweep_kernels_as_ny512(nz) : ms_sweep_kernels_ny512(nz); break;
        case 1024: k = angular ? ms_sweep_kernels_as_ny1024(nz) : ms_sweep_kernels_ny1024(nz); break;
        default: break;
    }
    if (k.fwd && k.adj) {
        ks.fwd = k.fwd;
        ks.adj = k.adj;
    }
    return ks;
}

// raise the dynamic shared-memory limit of a kernel once per device
constexpr int kMaxConfigured = 128;
const void* g_configured[64][kMaxConfigured];
int g_nconfigured[64];

int configure(int dev, const void* k) {
    for (int i = 0; i < g_nconfigured[dev]; ++i)
        if (g_configured[dev][i] == k) return MSLICE_OK;
    int maxopt = 0;
    if (note(cudaDeviceGetAttribute(&maxopt, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev), "cudaDeviceGetAttribute"))
        return MSLICE_ELAUNCH;
    cudaFuncAttributes fa;
    if (note(cudaFuncGetAttributes(&fa, k), "cudaFuncGetAttributes")) return MSLICE_ELAUNCH;
    const int dyn = maxopt - (int)fa.sharedSizeBytes;
    if (note(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn), "cudaFuncSetAttribute"))
        return MSLICE_ELAUNCH;
    if (g_nconfigured[dev] < kMaxConfigured) g_configured[dev][g_nconfigured[dev]++] = k;
    return MSLICE_OK;
}

int device_info(size_t smem, const KernelSet& ks, DevInfo** out) {
    int dev = 0;
    if (note(cudaGetDevice(&dev), "cudaGetDevice") || dev < 0 || dev >= 64) return MSLICE_ELAUNCH;
    DevInfo& D = g_dev[dev];
    if (!D.init) {
        if (note(cudaDeviceGetAttribute(&D.sms, cudaDevAttrMultiProcessorCount, dev), "cudaDeviceGetAttribute"))
            return MSLICE_ELAUNCH;
        D.init = true;
    }
    const void* used[7] = {ks.fwd, ks.adj, ks.last_far, ks.last_loss, ks.last_exit, ks.adj_start_seed,
                           ks.adj_start};
    int occ = 1 << 30;
    for (const void* k : used) {
        if (!k) continue;
        int rc = configure(dev, k);
        if (rc) return rc;
        int o = 0;
        if (note(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k, MS_THREADS, smem),
                 "cudaOccupancyMaxActiveBlocksPerMultiprocessor"))
            return MSLICE_ELAUNCH;
        if (o < occ) occ = o;
    }
    D.occ = occ;
    *out = &D;
    return MSLICE_OK;
}

// column-group width of a call: the requested one if usable, else the default
int col_width(const mslice_params* p) {
    const int Tz = p->nz > 32 ? p->nz / 32 : 1;
    if (p->col_width > 0 && col_cw_ok(p->col_width, Tz)) return p->col_width;
    return col_cw(Tz);
}

int grid_size(const mslice_params* p, const DevInfo& D) {
    int maxg = D.sms * D.occ;
    if (maxg > kMaxGrid) maxg = kMaxGrid;
    if (maxg < 1) return 0;
    const int Ty = p->ny > 32 ? p->ny / 32 : 1, Tz = p->nz > 32 ? p->nz / 32 : 1;
    const long rows = (long)p->nz * p->nw;
    const long row_wtasks = (rows + (32 / Ty) - 1) / (32 / Ty);
    const int cw = col_width(p);
    const long col_tasks = (long)((p->ny + cw - 1) / cw) * p->nw;
    const long col_groups = MS_THREADS / (cw * Tz);
    long need = (row_wtasks + 3) / 4;
    const long need_c = (col_tasks + col_groups - 1) / col_groups;
    if (need_c > need) need = need_c;
    if (need < 1) need = 1;
    if (p->grid_blocks > 0) need = p->grid_blocks;
    return (int)(need < maxg ? need : maxg);
}

// ----- tracing: event pairs around launches while enabled
enum : int { KID_FWD = 0, KID_ADJ, KID_LAST, KID_ADJ_START, KID_TRANSMISSION, KID_SETUP, KID_COUNT };
const char* const kKernelNames[KID_COUNT] = {"k_fwd", "k_adj", "k_last", "k_adj_start", "k_transmission",
                                             "k_setup"};
struct ProfRec { int kid; cudaEvent_t a, b; double units; };
bool g_prof_on = false;
ProfRec* g_prof = nullptr;
int g_prof_n = 0, g_prof_cap = 0;

ProfRec* prof_begin(int kid, double units, cudaStream_t st) {
    if (!g_prof_on) return nullptr;
    if (g_prof_n == g_prof_cap) {
        const int cap = g_prof_cap ? 2 * g_prof_cap : 1024;
        ProfRec* n = (ProfRec*)realloc(g_prof, sizeof(ProfRec) * cap);
        if (!n) return nullptr;
        g_prof = n;
        g_prof_cap = cap;
    }
    ProfRec* r = &g_prof[g_prof_n];
    if (cudaEventCreate(&r->a) != cudaSuccess) return nullptr;
    if (cudaEventCreate(&r->b) != cudaSuccess) { cudaEventDestroy(r->a); return nullptr; }
    r->kid = kid;
    r->units = units;
    cudaEventRecord(r->a, st);
    ++g_prof_n;
    return r;
}
void prof_end(ProfRec* r, cudaStream_t st) {
    if (r) cudaEventRecord(r->b, st);
}

int launch_coop(const void* fn, int grid, size_t smem, const SweepArgs& a, cudaStream_t st, int kid,
                double units) {
    void* args[] = {(void*)&a};
    ProfRec* r = prof_begin(kid, units, st);
    // host-side range named after the kernel (slice range in the payload), for
    // profilers that attach an NVTX tool; a no-op otherwise
    nvtxEventAttributes_t ev{};
    ev.version = NVTX_VERSION;
    ev.size = NVTX_EVENT_ATTRIB_STRUCT_SIZE;
    ev.messageType = NVTX_MESSAGE_TYPE_ASCII;
    ev.message.ascii = kKernelNames[kid];
    ev.payloadType = NVTX_PAYLOAD_TYPE_INT32;
    ev.payload.iValue = a.j_begin;
    nvtxRangePushEx(&ev);
    cudaError_t e = cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(MS_THREADS), args, smem, st);
    nvtxRangePop();
    prof_end(r, st);
    return note(e, "cudaLaunchCooperativeKernel") ? MSLICE_ELAUNCH : MSLICE_OK;
}

// streaming multiprocessors of the current device (cached; 152 on GB300)
int device_sms() {
    static int cache[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
    if (cache[dev] <= 0 && cudaDeviceGetAttribute(&cache[dev], cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 152;
    return cache[dev] > 0 ? cache[dev] : 152;
}

int launch_transmission(const float2* vol, float2* tv, size_t nvox, double kd, int exact, int minus_one,
                        cudaStream_t st) {
    const float kd_hi = (float)kd;
    const float kd_lo = (float)(kd - (double)kd_hi);
    const size_t n2 = nvox / 2;
    if (n2) {
        size_t tb = (n2 + 255) / 256;
        const size_t cap = (size_t)device_sms() * 16;   // 16 resident 256-thread blocks per SM
        if (tb > cap) tb = cap;
        k_transmission<<<(unsigned)tb, 256, 0, st>>>((const float4*)vol, (float4*)tv, n2, kd_hi, kd_lo, exact, minus_one);
        if (note(cudaGetLastError(), "k_transmission launch")) return MSLICE_ELAUNCH;
    }
    if (nvox & 1) {
        k_transmission_tail<<<1, 1, 0, st>>>(vol + nvox - 1, tv + nvox - 1, kd_hi, kd_lo, exact, minus_one);
        if (note(cudaGetLastError(), "k_transmission_tail launch")) return MSLICE_ELAUNCH;
    }
    return MSLICE_OK;
}

// Buffers of each structure of a per-structure run (MSLICE_PER_STRUCTURE):
// contiguous [nw][...] arrays of the caller, or the separate buffers of the
// jobs of a batched call.
struct JobTable {
    const float2* vol[MSLICE_MAX_ANGLES];
    float2* grad[MSLICE_MAX_ANGLES];
    const float* meas[MSLICE_MAX_ANGLES];
    float* inten[MSLICE_MAX_ANGLES];
    double* loss[MSLICE_MAX_ANGLES];
};

// the table of contiguous [nw][ns][nz][ny] volumes / gradients and
// [nw][nz][ny] amplitudes / intensities (any of them may be null)
JobTable contiguous_table(const mslice_params* p, const float* vols, float* grads, const float* meas, float* inten) {
    JobTable jt{};
    const size_t npx = (size_t)p->ny * p->nz, nv = (size_t)p->ns * npx;
    for (int w = 0; w < p->nw; ++w) {
        jt.vol[w] = vols ? (const float2*)vols + w * nv : nullptr;
        jt.grad[w] = grads ? (float2*)grads + w * nv : nullptr;
        jt.meas[w] = meas ? meas + w * npx : nullptr;
        jt.inten[w] = inten ? inten + w * npx : nullptr;
    }
    return jt;
}

struct Plan {
    KernelSet ks;
    Layout L;
    char* ws;
    size_t smem;
    int grid;
    SweepArgs base;
    const float2* tab_half;  // P over Delta/2 (symmetric splitting), else null
    const float2* p2d_half;  // the angular spectrum's 2-D table over Delta/2, else null
};

// jt: per-structure buffers (per-structure runs: the transmission of each
// structure is computed from its own volume), else null
int prepare(const mslice_params* p, int op, const float* vol, const float* probe, void* ws, size_t ws_bytes,
            cudaStream_t st, Plan* P, float2* py_out = nullptr, float2* pz_out = nullptr,
            float2* probe_z_out = nullptr, const JobTable* jt = nullptr) {
    int rc = validate(p);
    if (rc) return rc;
    const bool per_w = (p->flags & MSLICE_PER_STRUCTURE) != 0;
    if (per_w && jt) {
        for (int w = 0; w < p->nw; ++w)
            if (!jt->vol[w] || ((uintptr_t)jt->vol[w] & 15)) return MSLICE_EINVAL;
        vol = (const float*)jt->vol[0];
    }
    if (!vol || !ws || ((uintptr_t)ws & 255) || ((uintptr_t)vol & 15) || ((uintptr_t)probe & 7)) return MSLICE_EINVAL;
    P->L = make_layout(p, op);
    if (ws_bytes < P->L.total) return MSLICE_EWORKSPACE;
    P->ws = (char*)ws;
    const int cw = col_width(p);
    P->smem = smem_bytes(p->ny, p->nz, cw);
    DevInfo* D = nullptr;
    P->ks = sweep_kernels(p->ny, p->nz, (p->flags & MSLICE_ANGULAR) != 0);
    if ((rc = device_info(P->smem, P->ks, &D))) return rc;
    P->grid = grid_size(p, *D);
    if (P->grid < 1) return MSLICE_EUNSUPPORTED;
    const Layout& L = P->L;
    char* w = P->ws;
    if (note(cudaMemsetAsync(w + L.ctrl, 0, kCtrlBytes, st), "cudaMemsetAsync")) return MSLICE_ELAUNCH;
    // FP64 tables
    SetupArgs S{};
    S.ny = p->ny; S.nz = p->nz; S.nw = p->nw;
    S.slice_nm = p->slice_nm; S.wavelength_nm = p->wavelength_nm; S.dy_nm = p->dy_nm; S.dz_nm = p->dz_nm;
    for (int i = 0; i < p->nw; ++i) {
        S.sin_alpha[i] = sin(p->alpha_i_rad[i]);
        S.sin_psi[i] = sin(p->psi_rad[i]);
    }
    S.tab = (float2*)(w + L.tab);
    const bool strang = (p->flags & MSLICE_STRANG) != 0;
    S.tab_half = strang ? (float2*)(w + L.tab_half) : nullptr;
    S.probe_z = (float2*)(w + L.probe_z);
    S.probe_y = (float2*)(w + L.probe_y);
    S.py_out = py_out; S.pz_out = pz_out; S.probe_z_out = probe_z_out;
    const int total = 2 * (p->ny + p->nz) + p->nw * (p->nz + p->ny);
    ProfRec* r = prof_begin(KID_SETUP, 0.0, st);
    k_setup<<<(total + 255) / 256, 256, 0, st>>>(S);
    prof_end(r, st);
    if (note(cudaGetLastError(), "k_setup launch")) return MSLICE_ELAUNCH;
    // transmission volume
    const double kd = 2.0 * M_PI / p->wavelength_nm * p->slice_nm;
    const size_t nvox = (size_t)p->ns * p->ny * p->nz * ((p->flags & MSLICE_PER_STRUCTURE) ? p->nw : 1);
    r = prof_begin(KID_TRANSMISSION, (double)nvox, st);
    const int exact = (p->flags & MSLICE_EXACT_TRANSMISSION) ? 1 : 0;
    // the workspace holds u = t - 1 (applied as a + a u by the slice loops)
    if (per_w && jt) {
        const size_t nv = (size_t)p->ns * p->ny * p->nz;
        for (int q = 0; q < p->nw && !rc; ++q)
            rc = launch_transmission(jt->vol[q], (float2*)(w + L.tvol) + q * nv, nv, kd, exact, 1, st);
    } else {
        rc = launch_transmission((const float2*)vol, (float2*)(w + L.tvol), nvox, kd, exact, 1, st);
    }
    prof_end(r, st);
    if (rc) return rc;
    SweepArgs& a = P->base;
    memset(&a, 0, sizeof(a));
    a.ny = p->ny; a.nz = p->nz; a.ns = p->ns; a.nw = p->nw;
    a.kd = (float)kd;
    a.ffy = (float)(1.0 / sqrt((double)p->ny));
    a.ffz = (float)(1.0 / sqrt((double)p->nz));
    a.tvol = (const float2*)(w + L.tvol);
    a.vol = (const float2*)vol;
    a.exact = exact;
    a.probe = (const float2*)probe;
    a.probe_z = (const float2*)(w + L.probe_z);
    bool tilt_y = false;
    for (int q = 0; q < p->nw; ++q) tilt_y = tilt_y || p->psi_rad[q] != 0.0;
    a.probe_y = tilt_y ? (const float2*)(w + L.probe_y) : nullptr;
    a.tab = (const float2*)(w + L.tab);
    a.field = (float2*)(w + L.field);
    if (op != MSLICE_OP_FORWARD) {
        a.gfield = (float2*)(w + L.gfield);
        a.gpart = (float2*)(w + L.gpart);
        a.ckpt = (float2*)(w + L.ckpt);
        a.seg = (float2*)(w + L.seg);
    }
    a.partials = (double*)(w + L.partials);
    if (op == MSLICE_OP_LOSS_GRAD) {
        a.loss_task = (double*)(w + L.loss_task);
        a.loss_wsum = (double*)(w + L.loss_wsum);
    }
    if (per_w && jt) {
        for (int q = 0; q < p->nw; ++q) {
            a.volw[q] = jt->vol[q];
            a.gradw[q] = jt->grad[q];
            a.measw[q] = jt->meas[q];
            a.intw[q] = jt->inten[q];
            a.lossw[q] = jt->loss[q];
        }
    }
    a.ctrl = (unsigned*)(w + L.ctrl);
    a.timeout_ns = kDefaultTimeoutNs;
    a.K = L.K;
    a.init_ckpt = -1;
    a.seg_from = 0x7fffffff;
    a.per_w = (p->flags & MSLICE_PER_STRUCTURE) ? 1 : 0;
    a.lcw = ilog2(cw);
    a.split = p->nw >= 2 && p->schedule == 2;
    P->p2d_half = nullptr;
    if (p->flags & MSLICE_ANGULAR) {
        const size_t n2 = (size_t)p->ny * p->nz;
        const unsigned blocks = (unsigned)((n2 + 255) / 256 < 4096 ? (n2 + 255) / 256 : 4096);
        k_setup_p2d<<<blocks, 256, 0, st>>>((float2*)(w + L.p2d), p->ny, p->nz, p->dy_nm, p->dz_nm, p->slice_nm,
                                            p->wavelength_nm);
        if (note(cudaGetLastError(), "k_setup_p2d launch")) return MSLICE_ELAUNCH;
        a.p2d = (const float2*)(w + L.p2d);
        if (strang) {
            k_setup_p2d<<<blocks, 256, 0, st>>>((float2*)(w + L.p2d_half), p->ny, p->nz, p->dy_nm, p->dz_nm,
                                                0.5 * p->slice_nm, p->wavelength_nm);
            if (note(cudaGetLastError(), "k_setup_p2d launch")) return MSLICE_ELAUNCH;
            P->p2d_half = (const float2*)(w + L.p2d_half);
        }
    }
    P->tab_half = nullptr;
    if (strang) {
        // symmetric splitting: phi_0' = F^-1 P(Delta/2) F phi_0 for every
        // wavefield, by the forward slice loop over one slice of vacuum
        // (u = t - 1 = 0, so a = phi exactly) with the half-step tables; the
        // slice loops then start from phi_0' as from a user probe
        if (note(cudaMemsetAsync(w + L.zero_t, 0, (size_t)p->ny * p->nz * sizeof(float2), st), "cudaMemsetAsync"))
            return MSLICE_ELAUNCH;
        P->tab_half = (const float2*)(w + L.tab_half);
        SweepArgs h = a;
        h.tvol = (const float2*)(w + L.zero_t);
        h.per_w = 0;
        h.tab = P->tab_half;
        h.field = (float2*)(w + L.probe_half);
        h.j_begin = 0; h.j_end = 1;
        h.prop_last = 1;
        h.flags = P->ks.one_pass ? F_PROP_FULL : 0;   // both axes' factors
        if (P->p2d_half) {
            // angular spectrum: the half step leaves (k_y, z) data in the field
            // buffer, which the first slice of the forward takes as the output
            // of a previous slice (its row pass transforms back to real space)
            h.p2d = P->p2d_half;
            h.field = (float2*)(w + L.field);
        }
        rc = launch_coop(P->ks.fwd, P->grid, P->smem, h, st, KID_FWD, (double)p->nw * p->ny * p->nz);
        if (rc) return rc;
        if (P->p2d_half) a.field_start = 1;
        else a.probe = (const float2*)(w + L.probe_half);
    }
    return MSLICE_OK;
}

// Gradient driver: forward over all slices keeping phi at every K-th slice
// (and a_j of the last segment), far field / loss, start of the adjoint, then
// segment by segment backward: recompute a_j of the segment from its
// checkpoint, run the adjoint slice loop over it.
int run_gradient(const mslice_params* p, Plan& P, bool loss, cudaStream_t st) {
    const Layout& L = P.L;
    const double u = (double)p->nw * p->ny * p->nz;  // units per slice
    const int last_seg0 = (L.nseg - 1) * L.K;
    int rc;
    SweepArgs a = P.base;
    a.flags = F_STORE_CKPT;
    a.seg_base = last_seg0;
    a.seg_from = last_seg0;
    a.j_begin = 0;
    if (loss) {
        if (p->ns > 1) {
            a.j_end = p->ns - 1;
            a.prop_last = 1;
            if ((rc = launch_coop(P.ks.fwd, P.grid, P.smem, a, st, KID_FWD, u * (p->ns - 1)))) return rc;
        }
        a.j_end = p->ns;
        if ((rc = launch_coop(P.ks.last_loss, P.grid, P.smem, a, st, KID_LAST, u))) return rc;
        // two-pass loop: F_y^H of the seed; the one-pass adjoint's first pass does it
        if (!P.ks.one_pass && (rc = launch_coop(P.ks.adj_start, P.grid, P.smem, a, st, KID_ADJ_START, 0.0)))
            return rc;
    } else {
        a.j_end = p->ns;
        a.prop_last = 0;
        if ((rc = launch_coop(P.ks.fwd, P.grid, P.smem, a, st, KID_FWD, u * (p->ns - 1)))) return rc;
        if ((rc = launch_coop(P.ks.adj_start_seed, P.grid, P.smem, a, st, KID_ADJ_START, 0.0)))
            return rc;
    }
    for (int s = L.nseg - 1; s >= 0; --s) {
        const int j0 = s * L.K, j1 = (j0 + L.K < p->ns) ? j0 + L.K : p->ns;
        if (s != L.nseg - 1) {
            SweepArgs f = P.base;
            f.j_begin = j0; f.j_end = j1;
            f.prop_last = 0;
            f.init_ckpt = s;
            f.field_start = 0;
            f.seg_base = j0; f.seg_from = j0;
            if ((rc = launch_coop(P.ks.fwd, P.grid, P.smem, f, st, KID_FWD, u * (j1 - j0 - 1)))) return rc;
        }
        SweepArgs b = P.base;
        b.j_begin = j0; b.j_end = j1;
        b.seg_base = j0;
        if (P.ks.one_pass) b.flags = F_FIRST_FAR;   // slice ns-1 starts with F^H
        if ((rc = launch_coop(P.ks.adj, P.grid, P.smem, b, st, KID_ADJ, u * (j1 - j0)))) return rc;
    }
    return MSLICE_OK;
}

// Forward launch sequence after prepare(): slice loop over [0, ns-1), then the
// last slice with the far field (or the exit wave)
int run_forward(const mslice_params* p, Plan& P, float* intensity, float* field_out, cudaStream_t st) {
    int rc;
    const double u = (double)p->nw * p->ny * p->nz;
    SweepArgs a = P.base;
    a.intensity = intensity;
    a.field_out = (float2*)field_out;
    a.j_begin = 0;
    if (p->ns > 1) {
        a.j_end = p->ns - 1;
        a.prop_last = 1;
        if ((rc = launch_coop(P.ks.fwd, P.grid, P.smem, a, st, KID_FWD, u * (p->ns - 1)))) return rc;
    }
    a.j_end = p->ns;
    if (p->flags & MSLICE_EXIT_WAVE) {
        // the last propagation is a half step (one-pass: only the factors after
        // the last transmission; slice ns-2's second factor is a full step)
        if (P.tab_half) {
            if (P.ks.one_pass) a.tab2 = P.tab_half;
            else if (P.p2d_half) a.p2d = P.p2d_half;   // angular spectrum: the last column pass
            else a.tab = P.tab_half;
        }
        return launch_coop(P.ks.last_exit, P.grid, P.smem, a, st, KID_LAST, u);
    }
    return launch_coop(P.ks.last_far, P.grid, P.smem, a, st, KID_LAST, u);
}

// ---------------------------------------------------------------------------
// batched runs of uneven structures (mslice_*_batched)
// ---------------------------------------------------------------------------
// sum of n doubles in index order (the batch's loss over its groups)
__global__ void k_sum_doubles(const double* __restrict__ x, int n, double* out) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += x[i];
    *out = s;
}

// Jobs of one grid shape, advanced as the wavefields of one per-structure run
// (at most MSLICE_MAX_ANGLES per group).
struct Group {
    int ny, nz, ns, n;
    int idx[MSLICE_MAX_ANGLES];   // job indices, in job order
    double cost;                  // modelled work in SM-seconds (lane assignment)
    size_t ws_off, ws_bytes;      // region of the batch workspace
    int lane;
    int blocks;                   // grid of the group's persistent kernels (0: the default grid)
};

constexpr int kMaxLanes = 16;
// throughput of the slice-loop kernels per SM (voxel-slice-steps of forward +
// adjoint per second) and the latency of one slice step (forward + adjoint:
// the grid barriers and the dependent loads), measured on 128..512-point
// grids; the plan uses them only to compare groups and lanes
constexpr double kUnitsPerSmSecond = 3.6e8;
constexpr double kSliceStepSeconds = 2.2e-5;

// parameters of a group's run: the common ones with the group's grid, angles
// and launch shape (blocks > 0: that many blocks)
mslice_params group_params(const mslice_params* common, const mslice_job* jobs, const Group& g, int blocks) {
    mslice_params q = *common;
    q.ny = g.ny; q.nz = g.nz; q.ns = g.ns; q.nw = g.n;
    for (int k = 0; k < g.n; ++k) {
        q.alpha_i_rad[k] = jobs[g.idx[k]].alpha_i_rad;
        q.psi_rad[k] = jobs[g.idx[k]].psi_rad;
    }
    q.flags |= MSLICE_PER_STRUCTURE;
    const int cw = jobs[g.idx[0]].col_width;
    if (cw > 0) q.col_width = cw;
    if (blocks > 0) q.grid_blocks = blocks;
    return q;
}

// blocks a group's slice loop keeps busy: one row task per warp, or one
// column task per column group, in every pass
long useful_blocks(const mslice_params& q) {
    const int Ty = q.ny > 32 ? q.ny / 32 : 1, Tz = q.nz > 32 ? q.nz / 32 : 1;
    const int cw = col_width(&q);
    const long row_tasks = (long)q.nz * q.nw, row_per_block = MS_THREADS / Ty;
    const long col_tasks = (long)((q.ny + cw - 1) / cw) * q.nw, col_per_block = MS_THREADS / (cw * Tz);
    const long r = (row_tasks + row_per_block - 1) / row_per_block, c = (col_tasks + col_per_block - 1) / col_per_block;
    return r > c ? r : c;
}

// Groups jobs by grid shape (in order of first appearance) and lays out the
// batch workspace: ngroups FP64 loss totals, then one workspace region per
// group.  The groups go longest first onto the least loaded lane; a group's
// size is its work in SM-seconds at the per-SM rate, but no less than its
// slices times the slice-step latency on an equal share of the SMs (slice loops
// of little work are bound by that latency, whatever their grid).  Returns 0
// or an error code.
int plan_batch(const mslice_params* common, const mslice_job* jobs, int njobs, int op, int lanes,
               std::vector<Group>& G, size_t* total, int sms) {
    if (!common || !jobs || njobs < 1 || lanes < 1 || lanes > kMaxLanes || sms < 1) return MSLICE_EINVAL;
    if (common->flags & MSLICE_ANGULAR) return MSLICE_EUNSUPPORTED;
    if (op == MSLICE_OP_LOSS_GRAD && (common->flags & MSLICE_EXIT_WAVE)) return MSLICE_EUNSUPPORTED;
    G.clear();
    for (int i = 0; i < njobs; ++i) {
        const mslice_job& jb = jobs[i];
        if (!is_pow2(jb.ny) || !is_pow2(jb.nz) || jb.ny > MSLICE_MAX_N || jb.nz > MSLICE_MAX_N || jb.ns < 1)
            return MSLICE_EINVAL;
        if (!jb.vol || ((uintptr_t)jb.vol & 15)) return MSLICE_EINVAL;
        if (op == MSLICE_OP_LOSS_GRAD && (!jb.meas_amp || !jb.grad_vol || !(jb.scale > 0.f))) return MSLICE_EINVAL;
        if (op == MSLICE_OP_FORWARD && !jb.intensity) return MSLICE_EINVAL;
        Group* g = nullptr;
        for (auto& h : G)
            if (h.ny == jb.ny && h.nz == jb.nz && h.ns == jb.ns && h.n < MSLICE_MAX_ANGLES) { g = &h; break; }
        if (!g) {
            G.push_back(Group{});
            g = &G.back();
            g->ny = jb.ny; g->nz = jb.nz; g->ns = jb.ns; g->n = 0;
        }
        g->idx[g->n++] = i;
    }
    const size_t ng = G.size();
    std::vector<long> useful(ng);
    std::vector<double> work(ng);
    std::vector<int> order(ng);
    for (size_t k = 0; k < ng; ++k) {
        Group& g = G[k];
        const mslice_params q = group_params(common, jobs, g, 0);
        if (validate(&q)) return MSLICE_EINVAL;
        useful[k] = useful_blocks(q);
        work[k] = (double)g.n * g.ny * g.nz * g.ns / kUnitsPerSmSecond;
        const double floor_sm = g.ns * kSliceStepSeconds * sms / lanes;
        g.cost = work[k] > floor_sm ? work[k] : floor_sm;
        g.blocks = 0;
        order[k] = (int)k;
    }
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return G[a].cost > G[b].cost; });
    std::vector<double> load(lanes, 0.0);
    for (int k : order) {
        int best = 0;
        for (int l = 1; l < lanes; ++l)
            if (load[l] < load[best]) best = l;
        G[k].lane = best;
        load[best] += G[k].cost;
    }
    if (lanes > 1) {
        // every group on the blocks its tasks fill, at most half the SMs: the
        // lanes' grids together may exceed the SMs (a cooperative grid starts
        // when all its blocks fit), which measured faster than splitting the
        // SMs between the lanes in proportion to their work, because runs of
        // different grid shapes side by side slow each other down (1.3-1.5x)
        // more than copies of one shape do (1.0-1.2x)
        for (size_t k = 0; k < ng; ++k) {
            const long cap = sms / 2 > 0 ? sms / 2 : 1;
            G[k].blocks = (int)(useful[k] < cap ? useful[k] : cap);
        }
    }
    size_t off = align256(ng * sizeof(double));
    for (Group& g : G) {
        const mslice_params q = group_params(common, jobs, g, g.blocks);
        if (validate(&q)) return MSLICE_EINVAL;
        g.ws_off = off;
        g.ws_bytes = make_layout(&q, op).total;
        off = align256(off + g.ws_bytes);
    }
    *total = off;
    return MSLICE_OK;
}

// library-owned streams and events of the lanes, per device (created on first use)
struct LaneSet {
    bool init = false;
    cudaStream_t s[kMaxLanes];
    cudaEvent_t fork, join[kMaxLanes];
};
LaneSet g_lane_sets[64];
std::mutex g_lane_mu;

int lane_set(LaneSet** out) {
    int dev = 0;
    if (note(cudaGetDevice(&dev), "cudaGetDevice") || dev < 0 || dev >= 64) return MSLICE_ELAUNCH;
    std::lock_guard<std::mutex> lock(g_lane_mu);
    LaneSet& L = g_lane_sets[dev];
    if (!L.init) {
        if (note(cudaEventCreateWithFlags(&L.fork, cudaEventDisableTiming), "cudaEventCreateWithFlags"))
            return MSLICE_ELAUNCH;
        for (int l = 0; l < kMaxLanes; ++l) {
            if (note(cudaStreamCreateWithFlags(&L.s[l], cudaStreamNonBlocking), "cudaStreamCreateWithFlags") ||
                note(cudaEventCreateWithFlags(&L.join[l], cudaEventDisableTiming), "cudaEventCreateWithFlags"))
                return MSLICE_ELAUNCH;
        }
        L.init = true;
    }
    *out = &L;
    return MSLICE_OK;
}

int run_batch(const mslice_params* common, const mslice_job* jobs, int njobs, int lanes, int op, double* loss_total,
              void* ws, size_t ws_bytes, cudaStream_t st) {
    if (!ws || ((uintptr_t)ws & 255)) return MSLICE_EINVAL;
    int dev = 0, sms = 0;
    if (note(cudaGetDevice(&dev), "cudaGetDevice") ||
        note(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "cudaDeviceGetAttribute"))
        return MSLICE_ELAUNCH;
    std::vector<Group> G;
    size_t total = 0;
    int rc = plan_batch(common, jobs, njobs, op, lanes, G, &total, sms);
    if (rc) return rc;
    if (ws_bytes < total) return MSLICE_EWORKSPACE;
    LaneSet* L = nullptr;
    if (lanes > 1) {
        if ((rc = lane_set(&L))) return rc;
        if (note(cudaEventRecord(L->fork, st), "cudaEventRecord")) return MSLICE_ELAUNCH;
        for (int l = 0; l < lanes; ++l)
            if (note(cudaStreamWaitEvent(L->s[l], L->fork, 0), "cudaStreamWaitEvent")) return MSLICE_ELAUNCH;
    }
    double* totals = (double*)ws;
    // every lane's groups in the order they were placed (longest first)
    std::vector<int> order(G.size());
    for (size_t k = 0; k < G.size(); ++k) order[k] = (int)k;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return G[a].cost > G[b].cost; });
    for (int k : order) {
        const Group& g = G[k];
        const cudaStream_t gs = lanes > 1 ? L->s[g.lane] : st;
        const mslice_params q = group_params(common, jobs, g, g.blocks);
        JobTable jt{};
        float scales[MSLICE_MAX_ANGLES];
        for (int w = 0; w < g.n; ++w) {
            const mslice_job& jb = jobs[g.idx[w]];
            jt.vol[w] = (const float2*)jb.vol;
            jt.grad[w] = (float2*)jb.grad_vol;
            jt.meas[w] = jb.meas_amp;
            jt.inten[w] = jb.intensity;
            jt.loss[w] = jb.loss_out;
            scales[w] = jb.scale;
        }
        Plan P;
        char* gws = (char*)ws + g.ws_off;
        rc = prepare(&q, op, nullptr, nullptr, gws, g.ws_bytes, gs, &P, nullptr, nullptr, nullptr, &jt);
        if (rc) return rc;
        if (op == MSLICE_OP_LOSS_GRAD) {
            P.base.scale = scales[0];
            for (int w = 0; w < g.n; ++w) P.base.scales[w] = scales[w];
            P.base.loss_out = totals + k;
            rc = run_gradient(&q, P, true, gs);
        } else {
            rc = run_forward(&q, P, nullptr, nullptr, gs);
        }
        if (rc) return rc;
    }
    if (lanes > 1) {
        for (int l = 0; l < lanes; ++l) {
            if (note(cudaEventRecord(L->join[l], L->s[l]), "cudaEventRecord") ||
                note(cudaStreamWaitEvent(st, L->join[l], 0), "cudaStreamWaitEvent"))
                return MSLICE_ELAUNCH;
        }
    }
    if (op == MSLICE_OP_LOSS_GRAD && loss_total) {
        k_sum_doubles<<<1, 1, 0, st>>>(totals, (int)G.size(), loss_total);
        if (note(cudaGetLastError(), "k_sum_doubles launch")) return MSLICE_ELAUNCH;
    }
    return MSLICE_OK;
}

// Allocation-free forward: the workspace is a fixed file-scope device array.
// Host code must not use g_static_ws directly (its host-side name is a stand-in,
// not a device address); its device address is taken once per device with
// cudaGetSymbolAddress, with that device current, and cached.  The cache is
// guarded by a mutex, so first calls from several host threads are safe.
constexpr size_t kStaticWsBytes = (size_t)32 << 20;
constexpr int kStaticMaxDevices = 64;
__device__ __align__(256) unsigned char g_static_ws[kStaticWsBytes];
void* g_static_ws_ptr[kStaticMaxDevices];
std::mutex g_static_mu;

// device address of g_static_ws on the current device (set-up on first use)
int static_workspace(void** out) {
    int dev = 0;
    if (note(cudaGetDevice(&dev), "cudaGetDevice")) return MSLICE_ELAUNCH;
    if (dev < 0 || dev >= kStaticMaxDevices) return MSLICE_EUNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_ws_ptr[dev]) {
        void* ptr = nullptr;
        if (note(cudaGetSymbolAddress(&ptr, g_static_ws), "cudaGetSymbolAddress")) return MSLICE_ELAUNCH;
        g_static_ws_ptr[dev] = ptr;
    }
    *out = g_static_ws_ptr[dev];
    return MSLICE_OK;
}

}  // namespace

extern "C" {

size_t mslice_workspace_size(const mslice_params* p, int op) {
    if (validate(p) != MSLICE_OK) return 0;
    if (op < MSLICE_OP_FORWARD || op > MSLICE_OP_LOSS_GRAD) return 0;
    return make_layout(p, op).total;
}

int mslice_forward(const mslice_params* p, const float* vol, const float* probe, float* intensity,
                   float* field_out, void* ws, size_t ws_bytes, void* stream) {
    cudaStream_t st = (cudaStream_t)stream;
    Plan P;
    if (!p) return MSLICE_EINVAL;
    if (!intensity && !field_out) return MSLICE_EINVAL;
    const JobTable jt = contiguous_table(p, vol, nullptr, nullptr, intensity);
    int rc = prepare(p, MSLICE_OP_FORWARD, vol, probe, ws, ws_bytes, st, &P, nullptr, nullptr, nullptr,
                     (p->flags & MSLICE_PER_STRUCTURE) ? &jt : nullptr);
    if (rc) return rc;
    return run_forward(p, P, intensity, field_out, st);
}


int mslice_forward_static(const mslice_params* p, const float* vol, const float* probe, float* intensity,
                          float* field_out, void* stream) {
    int rc = validate(p);
    if (rc) return rc;
    if (make_layout(p, MSLICE_OP_FORWARD).total > kStaticWsBytes) return MSLICE_EWORKSPACE;
    void* ws = nullptr;
    if ((rc = static_workspace(&ws))) return rc;
    return mslice_forward(p, vol, probe, intensity, field_out, ws, kStaticWsBytes, stream);
}

int mslice_forward_static_status(void* stream) {
    void* ws = nullptr;
    const int rc = static_workspace(&ws);
    if (rc) return rc;
    return mslice_status(ws, stream);
}

int mslice_adjoint(const mslice_params* p, const float* vol, const float* probe, const float* g_psi,
                   float* grad_vol, void* ws, size_t ws_bytes, void* stream) {
    cudaStream_t st = (cudaStream_t)stream;
    if (!g_psi || !grad_vol) return MSLICE_EINVAL;
    if (p && (p->flags & MSLICE_EXIT_WAVE)) return MSLICE_EUNSUPPORTED;
    if (!p) return MSLICE_EINVAL;
    Plan P;
    const JobTable jt = contiguous_table(p, vol, grad_vol, nullptr, nullptr);
    int rc = prepare(p, MSLICE_OP_ADJOINT, vol, probe, ws, ws_bytes, st, &P, nullptr, nullptr, nullptr,
                     (p->flags & MSLICE_PER_STRUCTURE) ? &jt : nullptr);
    if (rc) return rc;
    P.base.gpsi = (const float2*)g_psi;
    P.base.grad = (float2*)grad_vol;
    return run_gradient(p, P, false, st);
}

int mslice_loss_grad(const mslice_params* p, const float* vol, const float* probe, const float* meas_amp,
                     float scale, double* loss_out, float* grad_vol, float* intensity, void* ws,
                     size_t ws_bytes, void* stream) {
    cudaStream_t st = (cudaStream_t)stream;
    if (!meas_amp || !loss_out || !grad_vol || !(scale > 0.f)) return MSLICE_EINVAL;
    if (p && (p->flags & MSLICE_EXIT_WAVE)) return MSLICE_EUNSUPPORTED;
    if (!p) return MSLICE_EINVAL;
    Plan P;
    const JobTable jt = contiguous_table(p, vol, grad_vol, meas_amp, intensity);
    int rc = prepare(p, MSLICE_OP_LOSS_GRAD, vol, probe, ws, ws_bytes, st, &P, nullptr, nullptr, nullptr,
                     (p->flags & MSLICE_PER_STRUCTURE) ? &jt : nullptr);
    if (rc) return rc;
    P.base.meas = meas_amp;
    P.base.scale = scale;
    P.base.loss_out = loss_out;
    P.base.grad = (float2*)grad_vol;
    P.base.intensity = intensity;
    return run_gradient(p, P, true, st);
}

int mslice_loss_grad_multi(const mslice_params* p, const float* vols, const float* probe, const float* meas_amp,
                           const float* scales, double* loss_out, float* grad_vol, float* intensity, void* ws,
                           size_t ws_bytes, void* stream) {
    cudaStream_t st = (cudaStream_t)stream;
    if (!p || !meas_amp || !scales || !loss_out || !grad_vol) return MSLICE_EINVAL;
    if (p->flags & MSLICE_EXIT_WAVE) return MSLICE_EUNSUPPORTED;
    mslice_params q = *p;
    q.flags |= MSLICE_PER_STRUCTURE;
    if (q.nw < 1 || q.nw > MSLICE_MAX_ANGLES) return MSLICE_EINVAL;
    for (int w = 0; w < q.nw; ++w)
        if (!(scales[w] > 0.f)) return MSLICE_EINVAL;
    Plan P;
    const JobTable jt = contiguous_table(&q, vols, grad_vol, meas_amp, intensity);
    int rc = prepare(&q, MSLICE_OP_LOSS_GRAD, vols, probe, ws, ws_bytes, st, &P, nullptr, nullptr, nullptr, &jt);
    if (rc) return rc;
    P.base.meas = meas_amp;
    P.base.scale = scales[0];
    for (int w = 0; w < q.nw; ++w) P.base.scales[w] = scales[w];
    P.base.loss_out = loss_out;
    P.base.grad = (float2*)grad_vol;
    P.base.intensity = intensity;
    return run_gradient(&q, P, true, st);
}

size_t mslice_batched_workspace_size(const mslice_params* common, const mslice_job* jobs, int njobs, int op,
                                     int lanes) {
    if (op != MSLICE_OP_FORWARD && op != MSLICE_OP_LOSS_GRAD) return 0;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        sms = 152;
    std::vector<Group> G;
    size_t total = 0;
    if (plan_batch(common, jobs, njobs, op, lanes, G, &total, sms)) return 0;
    return total;
}

int mslice_batched_plan(const mslice_params* common, const mslice_job* jobs, int njobs, int op, int lanes,
                        int* group_of_job, int* lane_of_group, int* blocks_of_group, int* ngroups) {
    if (!ngroups) return MSLICE_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        sms = 152;
    std::vector<Group> G;
    size_t total = 0;
    const int rc = plan_batch(common, jobs, njobs, op, lanes, G, &total, sms);
    if (rc) return rc;
    *ngroups = (int)G.size();
    for (size_t k = 0; k < G.size(); ++k) {
        if (lane_of_group) lane_of_group[k] = G[k].lane;
        if (blocks_of_group) blocks_of_group[k] = G[k].blocks;
        if (group_of_job)
            for (int w = 0; w < G[k].n; ++w) group_of_job[G[k].idx[w]] = (int)k;
    }
    return MSLICE_OK;
}

int mslice_batched_status(const mslice_params* common, const mslice_job* jobs, int njobs, int op, int lanes,
                          const void* ws, void* stream) {
    if (!ws) return MSLICE_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return MSLICE_ELAUNCH;
    std::vector<Group> G;
    size_t total = 0;
    int rc = plan_batch(common, jobs, njobs, op, lanes, G, &total, sms);
    if (rc) return rc;
    for (const Group& g : G) {
        rc = mslice_status((const char*)ws + g.ws_off, stream);
        if (rc) return rc;
    }
    return MSLICE_OK;
}

int mslice_loss_grad_batched(const mslice_params* common, const mslice_job* jobs, int njobs, int lanes,
                             double* loss_total, void* ws, size_t ws_bytes, void* stream) {
    return run_batch(common, jobs, njobs, lanes, MSLICE_OP_LOSS_GRAD, loss_total, ws, ws_bytes, (cudaStream_t)stream);
}

int mslice_forward_batched(const mslice_params* common, const mslice_job* jobs, int njobs, int lanes, void* ws,
                           size_t ws_bytes, void* stream) {
    return run_batch(common, jobs, njobs, lanes, MSLICE_OP_FORWARD, nullptr, ws, ws_bytes, (cudaStream_t)stream);
}

int mslice_plan_tables(const mslice_params* p, float* py, float* pz, float* probe_z, void* ws, size_t ws_bytes,
                       void* stream) {
    int rc = validate(p);
    if (rc) return rc;
    if (!ws || ((uintptr_t)ws & 255)) return MSLICE_EINVAL;
    const Layout L = make_layout(p, MSLICE_OP_FORWARD);
    if (ws_bytes < L.total) return MSLICE_EWORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    char* w = (char*)ws;
    SetupArgs S{};
    S.ny = p->ny; S.nz = p->nz; S.nw = p->nw;
    S.slice_nm = p->slice_nm; S.wavelength_nm = p->wavelength_nm; S.dy_nm = p->dy_nm; S.dz_nm = p->dz_nm;
    for (int i = 0; i < p->nw; ++i) {
        S.sin_alpha[i] = sin(p->alpha_i_rad[i]);
        S.sin_psi[i] = sin(p->psi_rad[i]);
    }
    S.tab = (float2*)(w + L.tab);
    S.probe_z = (float2*)(w + L.probe_z);
    S.probe_y = (float2*)(w + L.probe_y);
    S.py_out = (float2*)py; S.pz_out = (float2*)pz; S.probe_z_out = (float2*)probe_z;
    const int total = 2 * (p->ny + p->nz) + p->nw * (p->nz + p->ny);
    k_setup<<<(total + 255) / 256, 256, 0, st>>>(S);
    return cudaGetLastError() == cudaSuccess ? MSLICE_OK : MSLICE_ELAUNCH;
}

int mslice_transmission(const mslice_params* p, const float* vol, float* t_out, void* stream) {
    int rc = validate(p);
    if (rc) return rc;
    if (!vol || !t_out || ((uintptr_t)vol & 15) || ((uintptr_t)t_out & 15)) return MSLICE_EINVAL;
    const double kd = 2.0 * M_PI / p->wavelength_nm * p->slice_nm;
    const size_t nvox = (size_t)p->ns * p->ny * p->nz;
    const size_t nv = nvox * ((p->flags & MSLICE_PER_STRUCTURE) ? p->nw : 1);
    return launch_transmission((const float2*)vol, (float2*)t_out, nv, kd,
                               (p->flags & MSLICE_EXACT_TRANSMISSION) ? 1 : 0, 0, (cudaStream_t)stream);
}

int mslice_intensity_vjp(const float* psi, const float* dI, float* g_psi, size_t n, void* stream) {
    if (!psi || !dI || !g_psi) return MSLICE_EINVAL;
    if (n == 0) return MSLICE_OK;
    int tb = (int)((n + 255) / 256);
    if (tb > 4096) tb = 4096;
    k_intensity_vjp<<<tb, 256, 0, (cudaStream_t)stream>>>((const float2*)psi, dI, (float2*)g_psi, n);
    return note(cudaGetLastError(), "k_intensity_vjp launch") ? MSLICE_ELAUNCH : MSLICE_OK;
}

int mslice_status(const void* ws, void* stream) {
    if (!ws) return MSLICE_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    unsigned status = 0;
    if (cudaMemcpyAsync(&status, ws, sizeof(unsigned), cudaMemcpyDeviceToHost, st) != cudaSuccess) return MSLICE_ELAUNCH;
    if (cudaStreamSynchronize(st) != cudaSuccess) return MSLICE_ELAUNCH;
    return (status & kStatusTimeout) ? MSLICE_ETIMEDOUT : MSLICE_OK;
}

int mslice_debug_wait(int nblocks, int withhold, long long timeout_ns, void* ws, size_t ws_bytes, void* stream) {
    if (!ws || ws_bytes < kCtrlBytes || nblocks < 1 || nblocks > 1024 || withhold < 0 || timeout_ns <= 0 ||
        timeout_ns > 10000000000LL)
        return MSLICE_EINVAL;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (nblocks > sms) return MSLICE_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemsetAsync(ws, 0, kCtrlBytes, st) != cudaSuccess) return MSLICE_ELAUNCH;
    unsigned* ctrl = (unsigned*)ws;
    unsigned wh = (unsigned)withhold;
    void* args[] = {(void*)&ctrl, (void*)&wh, (void*)&timeout_ns};
    cudaError_t e = cudaLaunchCooperativeKernel((const void*)k_debug_wait, dim3(nblocks), dim3(32), args, 0, st);
    return e == cudaSuccess ? MSLICE_OK : MSLICE_ELAUNCH;
}

int mslice_profile_enable(int on) {
    for (int i = 0; i < g_prof_n; ++i) {
        cudaEventDestroy(g_prof[i].a);
        cudaEventDestroy(g_prof[i].b);
    }
    g_prof_n = 0;
    g_prof_on = on != 0;
    return MSLICE_OK;
}

int mslice_profile_read(mslice_kernel_time* out, int max_entries) {
    if (!out || max_entries < 0) return MSLICE_EINVAL;
    mslice_kernel_time acc[KID_COUNT];
    memset(acc, 0, sizeof(acc));
    for (int i = 0; i < g_prof_n; ++i) {
        const ProfRec& r = g_prof[i];
        if (cudaEventSynchronize(r.b) != cudaSuccess) return MSLICE_ELAUNCH;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) return MSLICE_ELAUNCH;
        acc[r.kid].launches += 1;
        acc[r.kid].total_ms += ms;
        acc[r.kid].units += r.units;
    }
    int n = 0;
    for (int k = 0; k < KID_COUNT && n < max_entries; ++k) {
        if (!acc[k].launches) continue;
        out[n] = acc[k];
        strncpy(out[n].name, kKernelNames[k], sizeof(out[n].name) - 1);
        ++n;
    }
    return n;
}

const char* mslice_last_cuda_error(void) { return g_err; }

const char* mslice_strerror(int code) {
    switch (code) {
        case MSLICE_OK: return "ok";
        case MSLICE_EINVAL: return "invalid argument (size, pointer, alignment or parameter)";
        case MSLICE_EUNSUPPORTED: return "unsupported request";
        case MSLICE_ELAUNCH: return "CUDA launch or runtime call failed";
        case MSLICE_ETIMEDOUT: return "a bounded device-side wait ran out";
        case MSLICE_EWORKSPACE: return "workspace too small";
        default: return "unknown error";
    }
}

}  // extern "C"
