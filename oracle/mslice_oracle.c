/*
 * mslice_oracle.c -- plain, slow, FP64 CPU oracle for the reflection-geometry
 * multislice forward model and its gradient (arxiv 2212.01253).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or calls
 * this file: only the test-suite, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code, header, table or constant with the
 * CUDA library; it has its own parameter struct, its own FFT and its own
 * propagator.
 *
 * What it computes (all in double precision, complex128 interleaved re/im):
 *
 *   k       = 2*pi / lambda
 *   phi_0   = user probe, or the tilted plane wave
 *             exp(-i k (sin(alpha) z_l + sin(psi) y_m)), z_l = l dz, y_m = m dy
 *             (Sec. 2: grazing incidence alpha_i, the probe heading toward the
 *             substrate at z index 0; in-plane angle psi)
 *   for slice j = 1 .. Ns:                                   (Eq. 1)
 *       a_j   = exp(-i k Delta (delta_j - i beta_j)) * phi_{j-1}
 *               (transmission exp((k/2i) int (1-n^2) dZ) with n = 1-delta+i beta,
 *                linearised 1-n^2 ~ 2(delta - i beta), one voxel per slice;
 *                with `exact`, 1-n^2 = 2w - w^2, w = delta - i beta)
 *       phi_j = F^-1 [ exp(-i Delta (k_y^2 + k_z^2) / 2k) * F a_j ]
 *               (paraxial Fresnel propagator "C" of Fig. 1; the global phase
 *                exp(i k Delta) is dropped: it never changes |Psi|^2)
 *   Psi     = F_unitary a_Ns          (far field of the last exit wave, Fig. 1a;
 *                                      the final free propagation is a pure
 *                                      Fourier phase and is omitted)
 *   I       = |Psi|^2
 *   L       = sum (sqrt(s I) - m)^2   (Eq. 4 on amplitudes, without the 1/N)
 *
 * With `angular` the propagator is the angular spectrum of the Helmholtz
 * equation instead of its paraxial (Fresnel) form:
 *   exp(i Delta (sqrt(k^2 - k_y^2 - k_z^2) - k))
 *     = exp(-i Delta (k_y^2 + k_z^2) / (sqrt(k^2 - k_y^2 - k_z^2) + k)),
 * and for k_y^2 + k_z^2 > k^2 (evanescent) exp(-Delta sqrt(k_y^2 + k_z^2 - k^2))
 * times the carrier phase exp(-i Delta k).  The paraxial form is its
 * expansion to first order in (k_y^2 + k_z^2) / k^2.
 *
 * With `strang` the splitting is symmetric instead of transmission-first:
 * half a step of free propagation, then per slice the transmission and a full
 * step, the last step being a half step again:
 *   phi_0' = F^-1 [ exp(-i (Delta/2) (k_y^2 + k_z^2) / 2k) * F phi_0 ]
 *   the loop above from phi_0'; the exit wave phi_Ns = U(Delta/2) a_Ns.
 * The far field omits that final half step as it omits the full one (a
 * unit-modulus Fourier phase), so I, L and the adjoint are the loop above
 * started from phi_0'.  Over slices of uniform content this is second order
 * in Delta; the transmission-first form is first order.
 *
 *   k_y = 2*pi*fftfreq(Ny, dy), k_z = 2*pi*fftfreq(Nz, dz); forward DFT kernel
 *   e^{-i}; natural (unshifted) frequency order.
 *
 * The gradient is the exact adjoint of the steps above, evaluated from stored
 * a_j (no checkpointing here).  With g denoting dL/dRe + i dL/dIm:
 *   g_Psi      = 2 s (r - m) Psi / r,  r = sqrt(s I)   (0 where r == 0)
 *   g_{a_Ns}   = F_unitary^H g_Psi
 *   dL/ddelta_j = k Delta Im(a_j conj(g_{a_j})),  dL/dbeta_j = -k Delta Re(a_j conj(g_{a_j}))
 *   g_{phi_{j-1}} = conj(t_j) g_{a_j},   g_{a_{j-1}} = F^-1 conj(P) F g_{phi_{j-1}}
 *
 * DFTs: a naive O(N^2) sum for N <= 32 (or when forced), otherwise an
 * iterative radix-2 decimation-in-time FFT; both with twiddles from libm
 * cos/sin in double.  OpenMP over rows and columns.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

#define ORC_OK 0
#define ORC_EINVAL (-1)
#define ORC_ENOMEM (-2)

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

typedef struct {
    double wavelength_nm;     /* lambda */
    double slice_nm;          /* Delta, slice thickness along the beam */
    double dy_nm;             /* transverse pixel, in-plane */
    double dz_nm;             /* transverse pixel, surface normal */
    int32_t ny, nz, ns, nw;   /* grid, slices, number of wavefields (incidence angles) */
    const double *alpha_i_rad;/* [nw] incidence angles (probe tilted toward -z) */
    int32_t force_naive_dft;  /* 1: use the O(N^2) DFT at every size */
    int32_t exit_wave;        /* 1: forward returns phi_Ns (full last propagation) instead of Psi */
    int32_t exact;            /* 1: exact 1 - n^2 in the transmission instead of 2 (delta - i beta) */
    const double *psi_rad;    /* [nw] in-plane angle of each wavefield (NULL: 0): the default probe
                                 of wavefield w also carries exp(-i k sin(psi_w) y) */
    int32_t strang;           /* 1: symmetric splitting (half steps of propagation at both ends) */
    int32_t angular;          /* 1: angular-spectrum propagator instead of the paraxial one */
} orc_params;

static int is_pow2(int n) { return n >= 1 && (n & (n - 1)) == 0; }

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* w[k] = exp(-2 pi i k / n), k = 0..n-1 */
static cplx *make_roots(int n)
{
    cplx *w = (cplx *)malloc(sizeof(cplx) * (size_t)n);
    if (!w) return NULL;
    for (int k = 0; k < n; k++) {
        double a = 2.0 * M_PI * (double)k / (double)n;
        w[k] = cos(a) - I * sin(a);
    }
    return w;
}

/* In-place unnormalised 1-D DFT of n contiguous values.
 * sign < 0: X_k = sum_m x_m e^{-2 pi i m k / n};  sign > 0: e^{+...}. */
static void dft1(cplx *x, int n, int sign, const cplx *w, int naive, cplx *scratch)
{
    if (n == 1) return;
    if (naive) {
        for (int k = 0; k < n; k++) {
            cplx s = 0;
            for (int m = 0; m < n; m++) {
                int e = (int)(((int64_t)m * k) % n);
                s += x[m] * (sign < 0 ? w[e] : conj(w[e]));
            }
            scratch[k] = s;
        }
        memcpy(x, scratch, sizeof(cplx) * (size_t)n);
        return;
    }
    /* bit-reversal permutation */
    for (int i = 1, j = 0; i < n; i++) {
        int bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) { cplx t = x[i]; x[i] = x[j]; x[j] = t; }
    }
    /* butterflies: blocks of length len, twiddle e^{-+2 pi i k / len} */
    for (int len = 2; len <= n; len <<= 1) {
        int half = len >> 1, step = n / len;
        for (int i = 0; i < n; i += len) {
            for (int k = 0; k < half; k++) {
                cplx tw = sign < 0 ? w[k * step] : conj(w[k * step]);
                cplx u = x[i + k], v = x[i + k + half] * tw;
                x[i + k] = u + v;
                x[i + k + half] = u - v;
            }
        }
    }
}

typedef struct {
    int ny, nz, naive_y, naive_z;
    cplx *wy, *wz;
} plan2;

static int plan_init(plan2 *p, int ny, int nz, int force_naive)
{
    p->ny = ny; p->nz = nz;
    p->naive_y = force_naive || ny <= 32;
    p->naive_z = force_naive || nz <= 32;
    p->wy = make_roots(ny);
    p->wz = make_roots(nz);
    return (p->wy && p->wz) ? ORC_OK : ORC_ENOMEM;
}

static void plan_free(plan2 *p) { free(p->wy); free(p->wz); }

/* Unnormalised 2-D DFT of f[nz][ny] (y fastest): rows, then columns. */
static void dft2(const plan2 *p, cplx *f, int sign)
{
    const int ny = p->ny, nz = p->nz;
    int nmax = ny > nz ? ny : nz;
#pragma omp parallel
    {
        cplx *buf = (cplx *)malloc(sizeof(cplx) * (size_t)nmax);
        cplx *scr = (cplx *)malloc(sizeof(cplx) * (size_t)nmax);
#pragma omp for schedule(static)
        for (int l = 0; l < nz; l++)
            dft1(f + (size_t)l * ny, ny, sign, p->wy, p->naive_y, scr);
#pragma omp for schedule(static)
        for (int m = 0; m < ny; m++) {
            for (int l = 0; l < nz; l++) buf[l] = f[(size_t)l * ny + m];
            dft1(buf, nz, sign, p->wz, p->naive_z, scr);
            for (int l = 0; l < nz; l++) f[(size_t)l * ny + m] = buf[l];
        }
        free(buf);
        free(scr);
    }
}

/* numpy.fft.fftfreq(n, d) * 2 pi, entry m */
static double angular_freq(int m, int n, double d)
{
    int f = (m < (n + 1) / 2) ? m : m - n;
    return 2.0 * M_PI * (double)f / ((double)n * d);
}

/* Fresnel propagator of Eq. 1 on the full 2-D frequency grid over a distance
 * len (Delta, or Delta/2 for the half steps of the symmetric splitting):
 * P[l][m] = exp(-i len (k_y[m]^2 + k_z[l]^2) / (2k)); with q->angular the
 * angular-spectrum propagator written out in the header. */
static cplx *make_propagator(const orc_params *q, double len)
{
    const int ny = q->ny, nz = q->nz;
    const double k = 2.0 * M_PI / q->wavelength_nm;
    cplx *P = (cplx *)malloc(sizeof(cplx) * (size_t)ny * nz);
    if (!P) return NULL;
    for (int l = 0; l < nz; l++) {
        double kz = angular_freq(l, nz, q->dz_nm);
        for (int m = 0; m < ny; m++) {
            double ky = angular_freq(m, ny, q->dy_nm);
            const double kp2 = ky * ky + kz * kz;
            if (!q->angular)
                P[(size_t)l * ny + m] = cexp(-I * len * kp2 / (2.0 * k));
            else if (kp2 < k * k)
                P[(size_t)l * ny + m] = cexp(-I * len * kp2 / (sqrt(k * k - kp2) + k));
            else
                P[(size_t)l * ny + m] = exp(-len * sqrt(kp2 - k * k)) * cexp(-I * len * k);
        }
    }
    return P;
}

/* transmission of one voxel v = delta + i beta, w = delta - i beta:
 * exp((k/2i) Delta (1 - n^2)) with n = 1 - w; 1 - n^2 = 2 w - w^2 (Eq. 1), so
 * exp(-i k Delta (w - w^2/2)); linearised (exact == 0): exp(-i k Delta w) */
static cplx transmission(cplx v, double kd, int exact)
{
    const cplx w = conj(v);
    return cexp(-I * kd * (exact ? w - 0.5 * w * w : w));
}

static int check(const orc_params *q)
{
    if (!q || !is_pow2(q->ny) || !is_pow2(q->nz) || q->ns < 1 || q->nw < 1) return ORC_EINVAL;
    if (q->ny > 65536 || q->nz > 65536) return ORC_EINVAL;
    if (!(q->wavelength_nm > 0) || !(q->slice_nm > 0) || !(q->dy_nm > 0) || !(q->dz_nm > 0)) return ORC_EINVAL;
    return ORC_OK;
}

/* phi_0 for wavefield w */
static void initial_field(const orc_params *q, const cplx *probe, int w, cplx *phi)
{
    const size_t npx = (size_t)q->ny * q->nz;
    if (probe) {
        memcpy(phi, probe + (size_t)w * npx, sizeof(cplx) * npx);
        return;
    }
    const double k = 2.0 * M_PI / q->wavelength_nm;
    double alpha = q->alpha_i_rad ? q->alpha_i_rad[w] : 0.0;
    double psi = q->psi_rad ? q->psi_rad[w] : 0.0;
    for (int l = 0; l < q->nz; l++)
        for (int m = 0; m < q->ny; m++)
            phi[(size_t)l * q->ny + m] =
                cexp(-I * k * (sin(alpha) * ((double)l * q->dz_nm) + sin(psi) * ((double)m * q->dy_nm)));
}

/* phi <- F^-1 [ P F phi ]  (conj_p: use conj(P), the adjoint) */
static void propagate(const plan2 *p, const cplx *P, cplx *phi, int conj_p)
{
    const size_t npx = (size_t)p->ny * p->nz;
    const double inv_n = 1.0 / (double)npx;
    dft2(p, phi, -1);
#pragma omp parallel for schedule(static)
    for (size_t i = 0; i < npx; i++) phi[i] *= (conj_p ? conj(P[i]) : P[i]) * inv_n;
    dft2(p, phi, +1);
}

/* Runs the slice loop for wavefield w.  If a_store is non-NULL, stores a_j
 * for every slice ([ns][nz][ny]).  On return `out` holds Psi (far field,
 * unitary DFT of a_Ns) or, with exit_wave, phi_Ns. */
static void forward_one(const orc_params *q, const plan2 *p, const cplx *P, const cplx *Ph,
                        const cplx *vol, const cplx *probe, int w, cplx *phi, cplx *a_store, cplx *out)
{
    const size_t npx = (size_t)q->ny * q->nz;
    const double kd = (2.0 * M_PI / q->wavelength_nm) * q->slice_nm;
    initial_field(q, probe, w, phi);
    if (q->strang) propagate(p, Ph, phi, 0);
    for (int j = 0; j < q->ns; j++) {
        const cplx *v = vol + (size_t)j * npx;
#pragma omp parallel for schedule(static)
        for (size_t i = 0; i < npx; i++) phi[i] = transmission(v[i], kd, q->exact) * phi[i];
        if (a_store) memcpy(a_store + (size_t)j * npx, phi, sizeof(cplx) * npx);
        if (j < q->ns - 1) propagate(p, P, phi, 0);
    }
    if (q->exit_wave) {
        propagate(p, q->strang ? Ph : P, phi, 0);
        memcpy(out, phi, sizeof(cplx) * npx);
    } else {
        memcpy(out, phi, sizeof(cplx) * npx);
        dft2(p, out, -1);
        const double s = 1.0 / sqrt((double)npx);
        for (size_t i = 0; i < npx; i++) out[i] *= s;
    }
}

/* propagator tables for inspection: P_y[m] = exp(-i Delta k_y^2/2k), P_z likewise */
int orc_propagator_1d(const orc_params *q, double *py, double *pz)
{
    if (check(q)) return ORC_EINVAL;
    const double k = 2.0 * M_PI / q->wavelength_nm;
    cplx *Py = (cplx *)py, *Pz = (cplx *)pz;
    for (int m = 0; m < q->ny; m++) {
        double ky = angular_freq(m, q->ny, q->dy_nm);
        Py[m] = cexp(-I * q->slice_nm * ky * ky / (2.0 * k));
    }
    for (int l = 0; l < q->nz; l++) {
        double kz = angular_freq(l, q->nz, q->dz_nm);
        Pz[l] = cexp(-I * q->slice_nm * kz * kz / (2.0 * k));
    }
    return ORC_OK;
}

/* 1-D unnormalised DFT (sign -1 forward, +1 backward) for the FFT pins */
int orc_dft1d(int n, double *x, int sign, int naive)
{
    if (!is_pow2(n)) return ORC_EINVAL;
    cplx *w = make_roots(n), *scr = (cplx *)malloc(sizeof(cplx) * (size_t)n);
    if (!w || !scr) { free(w); free(scr); return ORC_ENOMEM; }
    dft1((cplx *)x, n, sign, w, naive, scr);
    free(w); free(scr);
    return ORC_OK;
}

/* 2-D unnormalised DFT of x[nz][ny] */
int orc_dft2d(int ny, int nz, double *x, int sign, int naive)
{
    if (!is_pow2(ny) || !is_pow2(nz)) return ORC_EINVAL;
    plan2 p;
    if (plan_init(&p, ny, nz, naive)) { plan_free(&p); return ORC_ENOMEM; }
    dft2(&p, (cplx *)x, sign);
    plan_free(&p);
    return ORC_OK;
}

/* Forward model.  vol [ns][nz][ny] complex (delta + i beta); probe NULL or
 * [nw][nz][ny]; intensity [nw][nz][ny] (may be NULL with exit_wave);
 * field_out NULL or [nw][nz][ny]: Psi, or phi_Ns when exit_wave. */
int orc_forward(const orc_params *q, const double *vol, const double *probe,
                double *intensity, double *field_out)
{
    if (check(q) || !vol) return ORC_EINVAL;
    const size_t npx = (size_t)q->ny * q->nz;
    plan2 p;
    cplx *P = make_propagator(q, q->slice_nm);
    cplx *Ph = q->strang ? make_propagator(q, 0.5 * q->slice_nm) : NULL;
    cplx *phi = (cplx *)malloc(sizeof(cplx) * npx), *out = (cplx *)malloc(sizeof(cplx) * npx);
    int rc = plan_init(&p, q->ny, q->nz, q->force_naive_dft);
    if (rc || !P || (q->strang && !Ph) || !phi || !out) { rc = ORC_ENOMEM; goto done; }
    for (int w = 0; w < q->nw; w++) {
        forward_one(q, &p, P, Ph, (const cplx *)vol, (const cplx *)probe, w, phi, NULL, out);
        if (field_out) memcpy((cplx *)field_out + (size_t)w * npx, out, sizeof(cplx) * npx);
        if (intensity)
            for (size_t i = 0; i < npx; i++) {
                double re = creal(out[i]), im = cimag(out[i]);
                intensity[(size_t)w * npx + i] = re * re + im * im;
            }
    }
done:
    plan_free(&p); free(P); free(Ph); free(phi); free(out);
    return rc;
}

/* Back-propagates g_Psi (per wavefield) into grad (accumulated over
 * wavefields).  a_store holds a_j of this wavefield. */
static void adjoint_one(const orc_params *q, const plan2 *p, const cplx *P, const cplx *vol,
                        const cplx *a_store, cplx *g, double *grad)
{
    const size_t npx = (size_t)q->ny * q->nz;
    const double kd = (2.0 * M_PI / q->wavelength_nm) * q->slice_nm;
    /* g_{a_Ns} = F_unitary^H g_Psi */
    dft2(p, g, +1);
    const double s = 1.0 / sqrt((double)npx);
    for (size_t i = 0; i < npx; i++) g[i] *= s;
    for (int j = q->ns - 1; j >= 0; j--) {
        const cplx *a = a_store + (size_t)j * npx;
        const cplx *v = vol + (size_t)j * npx;
        cplx *gr = (cplx *)grad + (size_t)j * npx;
#pragma omp parallel for schedule(static)
        for (size_t i = 0; i < npx; i++) {
            cplx ag = a[i] * conj(g[i]);
            /* dL/ddelta + i dL/dbeta = -i kd ag (d log t / dw = -i kd), times
             * (1 - w) for the exact form (d log t / dw = -i kd (1 - w)) */
            const cplx dw = q->exact ? 1.0 - conj(v[i]) : 1.0;
            gr[i] += -I * kd * dw * ag;
            g[i] = conj(transmission(v[i], kd, q->exact)) * g[i];
        }
        if (j > 0) propagate(p, P, g, 1);
    }
}

/* grad [ns][nz][ny] complex (dL/ddelta + i dL/dbeta) for a given detector
 * gradient g_psi [nw][nz][ny] (dL/dRe Psi + i dL/dIm Psi). */
int orc_adjoint(const orc_params *q, const double *vol, const double *probe,
                const double *g_psi, double *grad)
{
    if (check(q) || q->exit_wave || !vol || !g_psi || !grad) return ORC_EINVAL;
    const size_t npx = (size_t)q->ny * q->nz;
    plan2 p;
    cplx *P = make_propagator(q, q->slice_nm);
    cplx *Ph = q->strang ? make_propagator(q, 0.5 * q->slice_nm) : NULL;
    cplx *phi = (cplx *)malloc(sizeof(cplx) * npx), *out = (cplx *)malloc(sizeof(cplx) * npx);
    cplx *a = (cplx *)malloc(sizeof(cplx) * npx * (size_t)q->ns);
    int rc = plan_init(&p, q->ny, q->nz, q->force_naive_dft);
    if (rc || !P || (q->strang && !Ph) || !phi || !out || !a) { rc = ORC_ENOMEM; goto done; }
    memset(grad, 0, sizeof(cplx) * npx * (size_t)q->ns);
    for (int w = 0; w < q->nw; w++) {
        forward_one(q, &p, P, Ph, (const cplx *)vol, (const cplx *)probe, w, phi, a, out);
        memcpy(phi, (const cplx *)g_psi + (size_t)w * npx, sizeof(cplx) * npx);
        adjoint_one(q, &p, P, (const cplx *)vol, a, phi, grad);
    }
done:
    plan_free(&p); free(P); free(Ph); free(phi); free(out); free(a);
    return rc;
}

/* Loss L = sum_w sum_px (sqrt(s I) - m)^2 and its gradient on the volume.
 * meas_amp [nw][nz][ny] = sqrt(I_meas).  intensity optional output. */
int orc_loss_grad(const orc_params *q, const double *vol, const double *probe,
                  const double *meas_amp, double scale, double *loss, double *grad,
                  double *intensity)
{
    if (check(q) || q->exit_wave || !vol || !meas_amp || !loss || !grad || !(scale > 0)) return ORC_EINVAL;
    const size_t npx = (size_t)q->ny * q->nz;
    plan2 p;
    cplx *P = make_propagator(q, q->slice_nm);
    cplx *Ph = q->strang ? make_propagator(q, 0.5 * q->slice_nm) : NULL;
    cplx *phi = (cplx *)malloc(sizeof(cplx) * npx), *psi = (cplx *)malloc(sizeof(cplx) * npx);
    cplx *a = (cplx *)malloc(sizeof(cplx) * npx * (size_t)q->ns);
    int rc = plan_init(&p, q->ny, q->nz, q->force_naive_dft);
    if (rc || !P || (q->strang && !Ph) || !phi || !psi || !a) { rc = ORC_ENOMEM; goto done; }
    memset(grad, 0, sizeof(cplx) * npx * (size_t)q->ns);
    double L = 0.0;
    for (int w = 0; w < q->nw; w++) {
        forward_one(q, &p, P, Ph, (const cplx *)vol, (const cplx *)probe, w, phi, a, psi);
        const double *m = meas_amp + (size_t)w * npx;
        for (size_t i = 0; i < npx; i++) {
            double I2 = creal(psi[i]) * creal(psi[i]) + cimag(psi[i]) * cimag(psi[i]);
            if (intensity) intensity[(size_t)w * npx + i] = I2;
            double r = sqrt(scale * I2);
            L += (r - m[i]) * (r - m[i]);
            phi[i] = (r > 0.0) ? 2.0 * scale * (r - m[i]) / r * psi[i] : 0.0;
        }
        adjoint_one(q, &p, P, (const cplx *)vol, a, phi, grad);
    }
    *loss = L;
done:
    plan_free(&p); free(P); free(Ph); free(phi); free(psi); free(a);
    return rc;
}
