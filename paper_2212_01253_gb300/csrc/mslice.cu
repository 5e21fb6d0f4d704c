// mslice.cu -- GB300 (sm_103a) multislice forward model and adjoint for
// reflection-geometry Coherent Surface Scattering Imaging (arxiv 2212.01253).
//
// One slice (Eq. 1) is a pointwise transmission followed by a separable
// Fresnel propagation F^-1 P F with P(k_y, k_z) = P_y(k_y) P_z(k_z).  The 2-D
// FFT is split into a ROW pass (transmission, y-FFT, P_y, inverse y-FFT, all on
// one row held by a few threads) and a COLUMN pass (z-FFT, P_z, inverse z-FFT
// on a group of 16 columns).  Both passes of every slice run inside ONE
// persistent cooperative kernel per slice range: the wavefields (one per
// incidence angle, [nw][nz][ny] complex64, 2 MB each at 512^2) stay in L2
// between passes and a bounded grid barrier separates the passes.  The only
// HBM stream of the forward pass is the precomputed transmission volume.
//
// FFT of length N <= 1024 by T = N/32 threads (N > 32): each thread holds the
// 32 elements t + T*m, does a radix-32 DFT in registers (Stockham stage 1),
// exchanges once through padded shared memory, applies twiddles from a
// table and finishes with a radix-T DFT (stage 2).  The output lands in the
// same element pattern t + T*m, so the propagator multiply and the inverse
// FFT follow without another exchange.  N <= 32: one thread per transform.
//
// Precision: FFTs and products in FP32; the propagator tables, twiddles,
// default-probe phases and transmission phase arguments are formed in FP64.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include "mslice.h"

#define MS_THREADS 256
#define MS_WARPS (MS_THREADS / 32)

namespace {

constexpr unsigned kStatusTimeout = 1u;
constexpr size_t kCtrlBytes = 4096;
constexpr int kMaxGrid = 1024;
constexpr size_t kPartialBytes = kMaxGrid * sizeof(double);
constexpr long long kDefaultTimeoutNs = 2000000000LL;  // 2 s per grid wait

// ---------------------------------------------------------------------------
// complex helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// a * w
__device__ __forceinline__ float2 cmul(float2 a, float2 w) {
    return make_float2(fmaf(a.x, w.x, -a.y * w.y), fmaf(a.x, w.y, a.y * w.x));
}
// a * conj(w)
__device__ __forceinline__ float2 cmulc(float2 a, float2 w) {
    return make_float2(fmaf(a.x, w.x, a.y * w.y), fmaf(a.y, w.x, -a.x * w.y));
}

// cos(pi e / 16), e = 0..16 (correctly rounded from the double values)
__host__ __device__ constexpr float kcos32(int e) {
    return e == 0 ? 1.0f
         : e == 1 ? (float)0.9807852804032304
         : e == 2 ? (float)0.9238795325112867
         : e == 3 ? (float)0.8314696123025452
         : e == 4 ? (float)0.7071067811865476
         : e == 5 ? (float)0.5555702330196023
         : e == 6 ? (float)0.38268343236508984
         : e == 7 ? (float)0.19509032201612833
         : e == 8 ? 0.0f
         : -kcos32(16 - e);
}

template <int R> struct Log2 { static constexpr int value = 1 + Log2<R / 2>::value; };
template <> struct Log2<1> { static constexpr int value = 0; };

__host__ __device__ constexpr int brev(int r, int bits) {
    int o = 0;
    for (int i = 0; i < bits; ++i) o |= ((r >> i) & 1) << (bits - 1 - i);
    return o;
}

// a * exp(-+ 2 pi i e / 32), e in [0, 16); compile-time e after unrolling
template <bool INV>
__device__ __forceinline__ float2 tw32(float2 a, int e) {
    if (e == 0) return a;
    if (e == 8) return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
    const float c = kcos32(e);
    const float s = kcos32(e <= 8 ? 8 - e : e - 8);  // sin(pi e / 16)
    return INV ? make_float2(fmaf(a.x, c, -a.y * s), fmaf(a.y, c, a.x * s))
               : make_float2(fmaf(a.x, c, a.y * s), fmaf(a.y, c, -a.x * s));
}

// In-register DFT of the R values x[B + S*i], i = 0..R-1 (R <= 32), radix-2
// decimation in frequency, result in natural order.  Forward kernel
// exp(-2 pi i ...), inverse exp(+...), unnormalised.  Every register index is
// a compile-time constant (template recursion over the stages and over the
// bit-reversal), so the array never leaves the register file.
template <int R, int S, int HALF, bool INV>
struct DifStage {
    __device__ __forceinline__ static void run(float2 (&x)[32], const int B) {
#pragma unroll
        for (int blk = 0; blk < R; blk += 2 * HALF) {
#pragma unroll
            for (int k = 0; k < HALF; ++k) {
                const int i0 = B + S * (blk + k), i1 = i0 + S * HALF;
                const float2 a = x[i0], b = x[i1];
                x[i0] = cadd(a, b);
                x[i1] = tw32<INV>(csub(a, b), k * (32 / (2 * HALF)));
            }
        }
        DifStage<R, S, HALF / 2, INV>::run(x, B);
    }
};
template <int R, int S, bool INV>
struct DifStage<R, S, 0, INV> {
    __device__ __forceinline__ static void run(float2 (&)[32], const int) {}
};

template <int R, int S, int L, int I>
struct BitRev {
    __device__ __forceinline__ static void gather(const float2 (&x)[32], float2 (&tmp)[32], const int B) {
        constexpr int br = brev(I, L);
        tmp[I] = x[B + S * br];
        BitRev<R, S, L, I + 1>::gather(x, tmp, B);
    }
};
template <int R, int S, int L>
struct BitRev<R, S, L, R> {
    __device__ __forceinline__ static void gather(const float2 (&)[32], float2 (&)[32], const int) {}
};

template <int R, int S, bool INV>
__device__ __forceinline__ void dft_reg(float2 (&x)[32], const int B) {
    DifStage<R, S, R / 2, INV>::run(x, B);
    float2 tmp[32];
    BitRev<R, S, Log2<R>::value, 0>::gather(x, tmp, B);
#pragma unroll
    for (int r = 0; r < R; ++r) x[B + S * r] = tmp[r];
}

// Stockham stage 2 (radix TT = N/32, 32/TT butterflies per thread): twiddle
// Wt[r2*32 + b] = exp(-2 pi i b r2 / N), then DFT over r2 of x[q + (32/TT) r2].
template <int TT, bool INV>
__device__ __forceinline__ void stage2(float2 (&x)[32], const int t, const float2* __restrict__ Wt) {
    constexpr int Q = 32 / TT;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        const int b = t + TT * q;
#pragma unroll
        for (int r2 = 1; r2 < TT; ++r2) {
            const float2 w = Wt[r2 * 32 + b];
            x[q + Q * r2] = INV ? cmulc(x[q + Q * r2], w) : cmul(x[q + Q * r2], w);
        }
        dft_reg<TT, Q, INV>(x, q);
    }
}

// Length-n DFT of the distributed vector: thread t (of T = n/32) holds
// elements t + T*m in x[m]; on return it holds output bins t + T*m.
// reg: this transform's padded exchange region (index i -> i + i/32).
template <bool INV, class SyncF>
__device__ __forceinline__ void fft(float2 (&x)[32], const int n, const int T, const int t,
                                    float2* reg, const float2* __restrict__ Wt, SyncF sync) {
    if (n <= 32) {
        switch (n) {
            case 2: dft_reg<2, 1, INV>(x, 0); break;
            case 4: dft_reg<4, 1, INV>(x, 0); break;
            case 8: dft_reg<8, 1, INV>(x, 0); break;
            case 16: dft_reg<16, 1, INV>(x, 0); break;
            case 32: dft_reg<32, 1, INV>(x, 0); break;
            default: break;
        }
        return;
    }
    dft_reg<32, 1, INV>(x, 0);
    sync();
#pragma unroll
    for (int r = 0; r < 32; ++r) reg[33 * t + r] = x[r];
    sync();
#pragma unroll
    for (int m = 0; m < 32; ++m) {
        const int i = t + T * m;
        x[m] = reg[i + (i >> 5)];
    }
    switch (T) {
        case 2: stage2<2, INV>(x, t, Wt); break;
        case 4: stage2<4, INV>(x, t, Wt); break;
        case 8: stage2<8, INV>(x, t, Wt); break;
        case 16: stage2<16, INV>(x, t, Wt); break;
        case 32: stage2<32, INV>(x, t, Wt); break;
        default: break;
    }
}

// ---------------------------------------------------------------------------
// bounded grid barrier
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void red_release_add(unsigned* p, unsigned v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void named_bar(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// ctrl[0] = status bits, ctrl[1] = arrivals, ctrl[2] = exits
struct Grid {
    unsigned* ctrl;
    unsigned nblocks;
    unsigned epoch;  // barriers passed so far in this launch
    long long timeout_ns;
    int* s_ok;       // shared flag

    // Every block arrives, then waits until all nblocks (+ withhold) arrived or
    // the wait exceeded timeout_ns; returns false (uniformly per block) on
    // timeout or if another block already reported one.
    __device__ bool sync(unsigned withhold = 0) {
        __syncthreads();
        ++epoch;
        if (threadIdx.x == 0) {
            int ok = 1;
            const unsigned target = epoch * nblocks + withhold;
            __threadfence();
            red_release_add(&ctrl[1], 1u);
            unsigned long long t0 = globaltimer();
            unsigned spins = 0;
            while ((int)(ld_acquire(&ctrl[1]) - target) < 0) {
                if (++spins > 64) {
                    if (*(volatile unsigned*)&ctrl[0]) { ok = 0; break; }
                    if ((long long)(globaltimer() - t0) > timeout_ns) {
                        atomicOr(&ctrl[0], kStatusTimeout);
                        ok = 0;
                        break;
                    }
                    __nanosleep(32);
                }
            }
            __threadfence();
            *(volatile int*)s_ok = ok;
        }
        __syncthreads();
        return *(volatile int*)s_ok != 0;
    }
    // last block out resets the counters for the next launch on the stream
    __device__ void finish() {
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            const unsigned prev = atomicAdd(&ctrl[2], 1u);
            if (prev == nblocks - 1) {
                atomicExch(&ctrl[1], 0u);
                atomicExch(&ctrl[2], 0u);
                __threadfence();
            }
        }
    }
};

// ---------------------------------------------------------------------------
// sweep arguments
// ---------------------------------------------------------------------------
enum : int {
    F_STORE_CKPT = 1,   // forward: store phi_j at j % K == 0 into ckpt[j / K]
};

struct SweepArgs {
    int ny, nz, ns, nw;
    float kd;           // k * Delta
    float ffy, ffz;     // 1/sqrt(ny), 1/sqrt(nz)
    float scale;        // loss s
    const float2* tvol;     // [ns][nz][ny] transmission
    const float2* probe;    // [nw][nz][ny] or null
    const float2* probe_z;  // [nw][nz] default probe rows
    const float2* tab;      // Wt_y[ny] | Wt_z[nz] | P_y[ny]/ny | P_z[nz]/nz
    float2* field;          // [nw][nz][ny] forward state
    float2* gfield;         // [nw][nz][ny] adjoint state
    float2* gpart;          // [nw][nz][ny] per-wavefield gradient (nw > 1)
    float2* ckpt;           // [nseg][nw][nz][ny]
    float2* seg;            // [K][nw][nz][ny]  a_j of the current segment
    float2* grad;           // [ns][nz][ny]
    float* intensity;       // [nw][nz][ny] or null
    float2* field_out;      // [nw][nz][ny] or null
    const float* meas;      // [nw][nz][ny]
    const float2* gpsi;     // [nw][nz][ny]
    double* partials;       // [gridDim.x]
    double* loss_out;
    unsigned* ctrl;
    long long timeout_ns;
    int j_begin, j_end;
    int K;
    int flags;
    int init_ckpt;          // forward: first slice reads ckpt[init_ckpt] (-1: probe)
    int seg_base;           // slice of seg[0]
    int seg_from;           // forward: store a_j for j >= seg_from
    int prop_last;          // forward: the last slice of the range also propagates
};

struct Smem {
    float2* exch;    // exchange regions
    const float2* Wy;
    const float2* Wz;
    const float2* Py;
    const float2* Pz;
};

__host__ __device__ __forceinline__ int row_T(int n) { return n > 32 ? n / 32 : 1; }

// row-pass operations
enum : int {
    R_FWD = 0,       // a = t_j phi; [ckpt/seg stores]; [F^-1 P_y F]       -> field
    R_FAR = 1,       // a = t_j phi; [seg store]; F_y / sqrt(ny)           -> field
    R_ADJ = 2,       // grad_j from a_j, g; [g <- F^-1 conj(P_y) F conj(t_j) g] -> gfield
    R_ADJ_FAR = 3,   // g <- F_y^H g (unitary)                             -> gfield
};
// column-pass operations
enum : int {
    C_PROP = 0,      // F^-1 P_z F                                        field -> field
    C_ADJ = 1,       // F^-1 conj(P_z) F                                gfield -> gfield
    C_FAR = 2,       // Psi = F_z / sqrt(nz); I = |Psi|^2              field -> I, Psi
    C_FAR_LOSS = 3,  // C_FAR, loss partial, seed g, F_z^H g           field -> I, gfield
    C_EXIT = 4,      // C_PROP and write phi_Ns, |phi_Ns|^2            field -> field, outputs
    C_SEED = 5,      // F_z^H g_psi                                     gpsi -> gfield
};

// ----- row pass: one team of T = ny/32 threads (1 thread for ny <= 32) per row
template <int OP>
__device__ void row_pass(const SweepArgs& A, const Smem& S, const int j, const bool first, const bool propagate) {
    const int N = A.ny, T = row_T(N), P = N > 32 ? 32 : N;
    const int tpw = 32 / T;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int tm = lane / T, t = lane % T;
    float2* reg = S.exch + (size_t)(warp * tpw + tm) * (N + N / 32);
    const size_t npx = (size_t)A.ny * A.nz;
    const int ntasks = A.nz * A.nw;
    const int wtasks = (ntasks + tpw - 1) / tpw;
    auto sync = []() { __syncwarp(); };
    for (int wt = blockIdx.x * MS_WARPS + warp; wt < wtasks; wt += gridDim.x * MS_WARPS) {
        const int task = wt * tpw + tm;
        const bool active = task < ntasks;
        const int z = active ? task / A.nw : 0, w = active ? task % A.nw : 0;
        const size_t row = (size_t)w * npx + (size_t)z * N;
        float2 x[32];
#pragma unroll
        for (int m = 0; m < 32; ++m) x[m] = make_float2(0.f, 0.f);
        if constexpr (OP == R_FWD || OP == R_FAR) {
            if (active) {
                if (!first) {
#pragma unroll
                    for (int m = 0; m < 32; ++m) if (m < P) x[m] = __ldcg(A.field + row + t + T * m);
                } else if (A.init_ckpt >= 0) {
                    const float2* src = A.ckpt + (size_t)A.init_ckpt * A.nw * npx + row;
#pragma unroll
                    for (int m = 0; m < 32; ++m) if (m < P) x[m] = __ldcg(src + t + T * m);
                } else if (A.probe) {
#pragma unroll
                    for (int m = 0; m < 32; ++m) if (m < P) x[m] = __ldg(A.probe + row + t + T * m);
                } else {
                    const float2 v = A.probe_z[(size_t)w * A.nz + z];
#pragma unroll
                    for (int m = 0; m < 32; ++m) if (m < P) x[m] = v;
                }
                if ((A.flags & F_STORE_CKPT) && (j % A.K == 0)) {
                    float2* dst = A.ckpt + (size_t)(j / A.K) * A.nw * npx + row;
#pragma unroll
                    for (int m = 0; m < 32; ++m) if (m < P) __stcg(dst + t + T * m, x[m]);
                }
                const float2* tv = A.tvol + (size_t)j * npx + (size_t)z * N;
#pragma unroll
                for (int m = 0; m < 32; ++m) if (m < P) x[m] = cmul(x[m], __ldg(tv + t + T * m));
                if (j >= A.seg_from) {
                    float2* dst = A.seg + (size_t)(j - A.seg_base) * A.nw * npx + row;
#pragma unroll
                    for (int m = 0; m < 32; ++m) if (m < P) __stcg(dst + t + T * m, x[m]);
                }
            }
            if (OP == R_FWD && !propagate) continue;  // uniform
            fft<false>(x, N, T, t, reg, S.Wy, sync);
            if constexpr (OP == R_FAR) {
#pragma unroll
                for (int m = 0; m < 32; ++m) x[m] = cscale(x[m], A.ffy);
            } else {
#pragma unroll
                for (int m = 0; m < 32; ++m) if (m < P) x[m] = cmul(x[m], S.Py[t + T * m]);
                fft<true>(x, N, T, t, reg, S.Wy, sync);
            }
            if (active) {
#pragma unroll
                for (int m = 0; m < 32; ++m) if (m < P) __stcg(A.field + row + t + T * m, x[m]);
            }
        } else if constexpr (OP == R_ADJ) {
            if (active) {
#pragma unroll
                for (int m = 0; m < 32; ++m) if (m < P) x[m] = __ldcg(A.gfield + row + t + T * m);
                // x = g_{a_j}; gradient contribution -i kd a_j conj(g)
                const float2* a = A.seg + (size_t)(j - A.seg_base) * A.nw * npx + row;
                float2* gdst = (A.nw == 1) ? (A.grad + (size_t)j * npx + (size_t)z * N) : (A.gpart + row);
#pragma unroll
                for (int m = 0; m < 32; ++m) {
                    if (m < P) {
                        const float2 av = __ldcg(a + t + T * m), g = x[m];
                        const float re = fmaf(av.x, g.x, av.y * g.y);   // Re(a conj g)
                        const float im = fmaf(av.y, g.x, -av.x * g.y);  // Im(a conj g)
                        __stcg(gdst + t + T * m, make_float2(A.kd * im, -A.kd * re));
                    }
                }
                if (propagate) {
                    const float2* tv = A.tvol + (size_t)j * npx + (size_t)z * N;
#pragma unroll
                    for (int m = 0; m < 32; ++m) if (m < P) x[m] = cmulc(x[m], __ldg(tv + t + T * m));
                }
            }
            if (!propagate) continue;  // uniform
            fft<false>(x, N, T, t, reg, S.Wy, sync);
#pragma unroll
            for (int m = 0; m < 32; ++m) if (m < P) x[m] = cmulc(x[m], S.Py[t + T * m]);
            fft<true>(x, N, T, t, reg, S.Wy, sync);
            if (active) {
#pragma unroll
                for (int m = 0; m < 32; ++m) if (m < P) __stcg(A.gfield + row + t + T * m, x[m]);
            }
        } else {  // R_ADJ_FAR
            if (active) {
#pragma unroll
                for (int m = 0; m < 32; ++m) if (m < P) x[m] = __ldcg(A.gfield + row + t + T * m);
            }
            fft<true>(x, N, T, t, reg, S.Wy, sync);
            if (active) {
#pragma unroll
                for (int m = 0; m < 32; ++m) if (m < P) __stcg(A.gfield + row + t + T * m, cscale(x[m], A.ffy));
            }
        }
    }
}

// columns per column group: 16 (128-byte rows) while the group fits the CTA
__host__ __device__ __forceinline__ int col_cw(int T) { return T <= 16 ? 16 : 8; }
// exchange-region stride of one column: odd for 16-column groups, 2 mod 16
// for 8-column groups, so the lanes of a half-warp hit distinct banks
__host__ __device__ __forceinline__ int col_rs(int N, int cw) { return N + N / 32 + (cw == 16 ? 1 : 2); }

// ----- column pass: a group of cw*T threads per cw adjacent columns
template <int OP>
__device__ void col_pass(const SweepArgs& A, const Smem& S, double* s_red) {
    const int N = A.nz, T = row_T(N), P = N > 32 ? 32 : N;
    const int cw = col_cw(T);
    const int gthreads = cw * T;
    const int groups = MS_THREADS / gthreads;
    const int g = threadIdx.x / gthreads, gt = threadIdx.x % gthreads;
    const int c = gt % cw, t = gt / cw;
    float2* reg = S.exch + (size_t)(g * cw + c) * col_rs(N, cw);
    const size_t npx = (size_t)A.ny * A.nz;
    const int ncg = (A.ny + cw - 1) / cw;
    const int ntasks = ncg * A.nw;
    auto sync = [gthreads, g]() {
        if (gthreads <= 32) __syncwarp();
        else named_bar(1 + g, gthreads);
    };
    const float2* src = (OP == C_ADJ) ? A.gfield : (OP == C_SEED ? A.gpsi : A.field);
    double loss = 0.0;
    for (int task = blockIdx.x * groups + g; task < ntasks; task += gridDim.x * groups) {
        const int cg = task / A.nw, w = task % A.nw;
        const int col = cg * cw + c;
        const bool active = col < A.ny;
        const size_t base = (size_t)w * npx + col;
        float2 x[32];
#pragma unroll
        for (int m = 0; m < 32; ++m) {
            x[m] = make_float2(0.f, 0.f);
            if (active && m < P) x[m] = __ldcg(src + base + (size_t)(t + T * m) * A.ny);
        }
        if constexpr (OP != C_SEED) fft<false>(x, N, T, t, reg, S.Wz, sync);
        if constexpr (OP == C_FAR || OP == C_FAR_LOSS) {
#pragma unroll
            for (int m = 0; m < 32; ++m) {
                if (m < P) {
                    const float2 psi = cscale(x[m], A.ffz);
                    const float I = fmaf(psi.x, psi.x, psi.y * psi.y);
                    const size_t o = base + (size_t)(t + T * m) * A.ny;
                    if (active) {
                        if (A.intensity) __stcs(A.intensity + o, I);
                        if (A.field_out) __stcs(A.field_out + o, psi);
                    }
                    if constexpr (OP == C_FAR_LOSS) {
                        float2 gs = make_float2(0.f, 0.f);
                        if (active) {
                            const float r = sqrtf(A.scale * I);
                            const float d = r - __ldg(A.meas + o);
                            loss += (double)d * (double)d;
                            if (r > 0.f) gs = cscale(psi, 2.f * A.scale * d / r);
                        }
                        x[m] = gs;
                    }
                }
            }
            if constexpr (OP == C_FAR) continue;
        } else if constexpr (OP == C_ADJ) {
#pragma unroll
            for (int m = 0; m < 32; ++m) if (m < P) x[m] = cmulc(x[m], S.Pz[t + T * m]);
        } else if constexpr (OP == C_PROP || OP == C_EXIT) {
#pragma unroll
            for (int m = 0; m < 32; ++m) if (m < P) x[m] = cmul(x[m], S.Pz[t + T * m]);
        }
        fft<true>(x, N, T, t, reg, S.Wz, sync);
        if (!active) continue;
        if constexpr (OP == C_SEED || OP == C_FAR_LOSS) {
#pragma unroll
            for (int m = 0; m < 32; ++m)
                if (m < P) __stcg(A.gfield + base + (size_t)(t + T * m) * A.ny, cscale(x[m], A.ffz));
        } else {
            float2* dst = (OP == C_ADJ) ? A.gfield : A.field;
#pragma unroll
            for (int m = 0; m < 32; ++m) {
                if (m < P) {
                    const size_t o = base + (size_t)(t + T * m) * A.ny;
                    __stcg(dst + o, x[m]);
                    if constexpr (OP == C_EXIT) {
                        if (A.field_out) __stcs(A.field_out + o, x[m]);
                        if (A.intensity) __stcs(A.intensity + o, fmaf(x[m].x, x[m].x, x[m].y * x[m].y));
                    }
                }
            }
        }
    }
    if constexpr (OP == C_FAR_LOSS) {
        // block reduction of the FP64 loss partial, fixed order
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) loss += __shfl_xor_sync(0xffffffffu, loss, o);
        __syncthreads();
        if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = loss;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0.0;
            for (int i = 0; i < MS_WARPS; ++i) s += s_red[i];
            A.partials[blockIdx.x] = s;
        }
    }
}

// grad[j] = sum_w gpart[w]  (fixed order over w)
__device__ void reduce_gpart(const SweepArgs& A, int j) {
    const size_t npx = (size_t)A.ny * A.nz;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < npx; i += stride) {
        float2 s = __ldcg(A.gpart + i);
        for (int w = 1; w < A.nw; ++w) s = cadd(s, __ldcg(A.gpart + (size_t)w * npx + i));
        __stcs(A.grad + (size_t)j * npx + i, s);
    }
}

__device__ Smem load_tables(const SweepArgs& A, float2* base) {
    const int n = 2 * (A.ny + A.nz);
    for (int i = threadIdx.x; i < n; i += blockDim.x) base[i] = A.tab[i];
    __syncthreads();
    Smem S;
    S.Wy = base;
    S.Wz = base + A.ny;
    S.Py = base + A.ny + A.nz;
    S.Pz = base + 2 * A.ny + A.nz;
    S.exch = base + n;
    return S;
}

#define MS_KERNEL_PROLOGUE                                        \
    extern __shared__ float4 smem_raw[];                          \
    __shared__ int s_ok;                                          \
    __shared__ double s_red[MS_WARPS];                            \
    (void)s_red;                                                  \
    if (*(volatile unsigned*)&A.ctrl[0]) return;                  \
    const Smem S = load_tables(A, reinterpret_cast<float2*>(smem_raw)); \
    Grid grid{A.ctrl, gridDim.x, 0u, A.timeout_ns, &s_ok};

// Slice loop of the forward model, j in [j_begin, j_end): Eq. 1 per slice.
// The last slice of the range propagates only if A.prop_last.
__global__ void __launch_bounds__(MS_THREADS, 1) k_fwd(const SweepArgs A) {
    MS_KERNEL_PROLOGUE
    for (int j = A.j_begin; j < A.j_end; ++j) {
        const bool prop = (j < A.j_end - 1) || A.prop_last;
        row_pass<R_FWD>(A, S, j, j == A.j_begin, prop);
        if (prop) {
            if (!grid.sync()) return;
            col_pass<C_PROP>(A, S, s_red);
            if (j < A.j_end - 1 && !grid.sync()) return;
        }
    }
    grid.finish();
}

// Last slice (j = ns-1) with the far field, optionally the loss and its seed.
template <int COL>
__global__ void __launch_bounds__(MS_THREADS, 1) k_last(const SweepArgs A) {
    MS_KERNEL_PROLOGUE
    const int j = A.ns - 1;
    if constexpr (COL == C_EXIT) row_pass<R_FWD>(A, S, j, j == A.j_begin, true);
    else row_pass<R_FAR>(A, S, j, j == A.j_begin, true);
    if (!grid.sync()) return;
    col_pass<COL>(A, S, s_red);
    if constexpr (COL == C_FAR_LOSS) {
        if (!grid.sync()) return;
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            double sum = 0.0;
            for (unsigned b = 0; b < gridDim.x; ++b) sum += __ldcg(A.partials + b);
            *A.loss_out = sum;
        }
    }
    grid.finish();
}

// Start of the adjoint: [z-part of F_u^H on g_psi], then its y-part, so that
// gfield = g_{a_Ns} = F_u^H g_Psi.
template <bool SEED>
__global__ void __launch_bounds__(MS_THREADS, 1) k_adj_start(const SweepArgs A) {
    MS_KERNEL_PROLOGUE
    if constexpr (SEED) {
        col_pass<C_SEED>(A, S, s_red);
        if (!grid.sync()) return;
    }
    row_pass<R_ADJ_FAR>(A, S, A.ns - 1, false, true);
    grid.finish();
}

// Adjoint slice loop, j from j_end-1 down to j_begin (a_j in the segment buffer).
__global__ void __launch_bounds__(MS_THREADS, 1) k_adj(const SweepArgs A) {
    MS_KERNEL_PROLOGUE
    for (int j = A.j_end - 1; j >= A.j_begin; --j) {
        row_pass<R_ADJ>(A, S, j, false, j > 0);
        if (!grid.sync()) return;
        if (j > 0) col_pass<C_ADJ>(A, S, s_red);
        if (A.nw > 1) reduce_gpart(A, j);
        if (j > A.j_begin && !grid.sync()) return;
    }
    grid.finish();
}

// ---------------------------------------------------------------------------
// FP64 set-up of the constant arrays
// ---------------------------------------------------------------------------
struct SetupArgs {
    int ny, nz, nw;
    double slice_nm, wavelength_nm, dy_nm, dz_nm;
    double sin_alpha[MSLICE_MAX_ANGLES];
    float2* tab;       // Wt_y | Wt_z | P_y/ny | P_z/nz
    float2* probe_z;   // [nw][nz]
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
    const int total = 2 * (ny + nz) + S.nw * nz;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        if (i < ny) {
            S.tab[i] = twiddle_entry(i, ny);
        } else if (i < ny + nz) {
            S.tab[i] = twiddle_entry(i - ny, nz);
        } else if (i < 2 * ny + nz) {
            const int m = i - ny - nz;
            const double2 p = propagator_entry(m, ny, S.dy_nm, S.slice_nm, S.wavelength_nm);
            S.tab[i] = make_float2((float)(p.x / ny), (float)(p.y / ny));
            if (S.py_out) S.py_out[m] = make_float2((float)p.x, (float)p.y);
        } else if (i < 2 * (ny + nz)) {
            const int l = i - 2 * ny - nz;
            const double2 p = propagator_entry(l, nz, S.dz_nm, S.slice_nm, S.wavelength_nm);
            S.tab[i] = make_float2((float)(p.x / nz), (float)(p.y / nz));
            if (S.pz_out) S.pz_out[l] = make_float2((float)p.x, (float)p.y);
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

// t = exp(-i k Delta (delta - i beta)) = exp(-k Delta beta) (cos(k Delta delta) - i sin(...))
__global__ void k_transmission(const float2* __restrict__ vol, float2* __restrict__ tv, size_t n, double kd) {
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float2 v = __ldcs(vol + i);
        const float ph = (float)(kd * (double)v.x);
        const float mu = (float)(kd * (double)v.y);
        float s, c;
        sincosf(ph, &s, &c);
        const float a = expf(-mu);
        __stcg(tv + i, make_float2(a * c, -a * s));
    }
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
    if (p->psi_rad != 0.0) return MSLICE_EUNSUPPORTED;
    if (p->flags & ~MSLICE_EXIT_WAVE) return MSLICE_EINVAL;
    return MSLICE_OK;
}

struct Layout {
    size_t ctrl, partials, tab, probe_z, tvol, field, gfield, gpart, ckpt, seg, total;
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
    L.tvol = off; off = align256(off + (size_t)p->ns * npx * sizeof(float2));
    L.field = off; off = align256(off + fb);
    if (op == MSLICE_OP_ADJOINT || op == MSLICE_OP_LOSS_GRAD) {
        L.gfield = off; off = align256(off + fb);
        L.gpart = off; off = align256(off + (p->nw > 1 ? fb : 0));
        L.ckpt = off; off = align256(off + (size_t)L.nseg * fb);
        L.seg = off; off = align256(off + (size_t)L.K * fb);
    }
    L.total = off;
    return L;
}

size_t smem_bytes(int ny, int nz) {
    const size_t tabs = 2 * (size_t)(ny + nz) * sizeof(float2);
    size_t row = 0, col = 0;
    if (ny > 32) row = (size_t)(MS_THREADS / (ny / 32)) * (ny + ny / 32) * sizeof(float2);
    if (nz > 32) {
        const int T = nz / 32, cw = col_cw(T), groups = MS_THREADS / (cw * T);
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
    size_t occ_smem = (size_t)-1;
    bool attr = false;
};
DevInfo g_dev[64];

const void* const kCoopKernels[] = {
    (const void*)k_fwd, (const void*)k_adj, (const void*)k_last<C_FAR>, (const void*)k_last<C_FAR_LOSS>,
    (const void*)k_last<C_EXIT>, (const void*)k_adj_start<true>, (const void*)k_adj_start<false>,
};

int device_info(size_t smem, DevInfo** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return MSLICE_ELAUNCH;
    DevInfo& D = g_dev[dev];
    if (!D.init) {
        if (cudaDeviceGetAttribute(&D.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return MSLICE_ELAUNCH;
        D.init = true;
    }
    if (!D.attr) {
        int maxopt = 0;
        if (cudaDeviceGetAttribute(&maxopt, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
            return MSLICE_ELAUNCH;
        for (const void* k : kCoopKernels) {
            cudaFuncAttributes fa;
            if (note(cudaFuncGetAttributes(&fa, k), "cudaFuncGetAttributes")) return MSLICE_ELAUNCH;
            const int dyn = maxopt - (int)fa.sharedSizeBytes;
            if (note(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn),
                     "cudaFuncSetAttribute"))
                return MSLICE_ELAUNCH;
        }
        D.attr = true;
    }
    if (D.occ_smem != smem) {
        int occ = 1 << 30;
        for (const void* k : kCoopKernels) {
            int o = 0;
            if (note(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k, MS_THREADS, smem),
                     "cudaOccupancyMaxActiveBlocksPerMultiprocessor"))
                return MSLICE_ELAUNCH;
            if (o < occ) occ = o;
        }
        D.occ = occ;
        D.occ_smem = smem;
    }
    *out = &D;
    return MSLICE_OK;
}

int grid_size(const mslice_params* p, const DevInfo& D) {
    int maxg = D.sms * D.occ;
    if (maxg > kMaxGrid) maxg = kMaxGrid;
    if (maxg < 1) return 0;
    const int Ty = p->ny > 32 ? p->ny / 32 : 1, Tz = p->nz > 32 ? p->nz / 32 : 1;
    const long rows = (long)p->nz * p->nw;
    const long row_wtasks = (rows + (32 / Ty) - 1) / (32 / Ty);
    const int cw = col_cw(Tz);
    const long col_tasks = (long)((p->ny + cw - 1) / cw) * p->nw;
    const long col_groups = MS_THREADS / (cw * Tz);
    long need = (row_wtasks + 3) / 4;
    const long need_c = (col_tasks + col_groups - 1) / col_groups;
    if (need_c > need) need = need_c;
    if (need < 1) need = 1;
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
    cudaError_t e = cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(MS_THREADS), args, smem, st);
    prof_end(r, st);
    return note(e, "cudaLaunchCooperativeKernel") ? MSLICE_ELAUNCH : MSLICE_OK;
}

struct Plan {
    Layout L;
    char* ws;
    size_t smem;
    int grid;
    SweepArgs base;
};

int prepare(const mslice_params* p, int op, const float* vol, const float* probe, void* ws, size_t ws_bytes,
            cudaStream_t st, Plan* P, float2* py_out = nullptr, float2* pz_out = nullptr,
            float2* probe_z_out = nullptr) {
    int rc = validate(p);
    if (rc) return rc;
    if (!vol || !ws || ((uintptr_t)ws & 255) || ((uintptr_t)vol & 7) || ((uintptr_t)probe & 7)) return MSLICE_EINVAL;
    P->L = make_layout(p, op);
    if (ws_bytes < P->L.total) return MSLICE_EWORKSPACE;
    P->ws = (char*)ws;
    P->smem = smem_bytes(p->ny, p->nz);
    DevInfo* D = nullptr;
    if ((rc = device_info(P->smem, &D))) return rc;
    P->grid = grid_size(p, *D);
    if (P->grid < 1) return MSLICE_EUNSUPPORTED;
    const Layout& L = P->L;
    char* w = P->ws;
    if (note(cudaMemsetAsync(w + L.ctrl, 0, kCtrlBytes, st), "cudaMemsetAsync")) return MSLICE_ELAUNCH;
    // FP64 tables
    SetupArgs S{};
    S.ny = p->ny; S.nz = p->nz; S.nw = p->nw;
    S.slice_nm = p->slice_nm; S.wavelength_nm = p->wavelength_nm; S.dy_nm = p->dy_nm; S.dz_nm = p->dz_nm;
    for (int i = 0; i < p->nw; ++i) S.sin_alpha[i] = sin(p->alpha_i_rad[i]);
    S.tab = (float2*)(w + L.tab);
    S.probe_z = (float2*)(w + L.probe_z);
    S.py_out = py_out; S.pz_out = pz_out; S.probe_z_out = probe_z_out;
    const int total = 2 * (p->ny + p->nz) + p->nw * p->nz;
    ProfRec* r = prof_begin(KID_SETUP, 0.0, st);
    k_setup<<<(total + 255) / 256, 256, 0, st>>>(S);
    prof_end(r, st);
    if (note(cudaGetLastError(), "k_setup launch")) return MSLICE_ELAUNCH;
    // transmission volume
    const double kd = 2.0 * M_PI / p->wavelength_nm * p->slice_nm;
    const size_t nvox = (size_t)p->ns * p->ny * p->nz;
    int tb = (int)((nvox + 255) / 256);
    if (tb > 4 * 152 * 8) tb = 4 * 152 * 8;
    r = prof_begin(KID_TRANSMISSION, (double)nvox, st);
    k_transmission<<<tb, 256, 0, st>>>((const float2*)vol, (float2*)(w + L.tvol), nvox, kd);
    prof_end(r, st);
    if (note(cudaGetLastError(), "k_transmission launch")) return MSLICE_ELAUNCH;
    SweepArgs& a = P->base;
    memset(&a, 0, sizeof(a));
    a.ny = p->ny; a.nz = p->nz; a.ns = p->ns; a.nw = p->nw;
    a.kd = (float)kd;
    a.ffy = (float)(1.0 / sqrt((double)p->ny));
    a.ffz = (float)(1.0 / sqrt((double)p->nz));
    a.tvol = (const float2*)(w + L.tvol);
    a.probe = (const float2*)probe;
    a.probe_z = (const float2*)(w + L.probe_z);
    a.tab = (const float2*)(w + L.tab);
    a.field = (float2*)(w + L.field);
    if (op != MSLICE_OP_FORWARD) {
        a.gfield = (float2*)(w + L.gfield);
        a.gpart = (float2*)(w + L.gpart);
        a.ckpt = (float2*)(w + L.ckpt);
        a.seg = (float2*)(w + L.seg);
    }
    a.partials = (double*)(w + L.partials);
    a.ctrl = (unsigned*)(w + L.ctrl);
    a.timeout_ns = kDefaultTimeoutNs;
    a.K = L.K;
    a.init_ckpt = -1;
    a.seg_from = 0x7fffffff;
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
            if ((rc = launch_coop((const void*)k_fwd, P.grid, P.smem, a, st, KID_FWD, u * (p->ns - 1)))) return rc;
        }
        a.j_end = p->ns;
        if ((rc = launch_coop((const void*)k_last<C_FAR_LOSS>, P.grid, P.smem, a, st, KID_LAST, u))) return rc;
        if ((rc = launch_coop((const void*)k_adj_start<false>, P.grid, P.smem, a, st, KID_ADJ_START, 0.0)))
            return rc;
    } else {
        a.j_end = p->ns;
        a.prop_last = 0;
        if ((rc = launch_coop((const void*)k_fwd, P.grid, P.smem, a, st, KID_FWD, u * (p->ns - 1)))) return rc;
        if ((rc = launch_coop((const void*)k_adj_start<true>, P.grid, P.smem, a, st, KID_ADJ_START, 0.0)))
            return rc;
    }
    for (int s = L.nseg - 1; s >= 0; --s) {
        const int j0 = s * L.K, j1 = (j0 + L.K < p->ns) ? j0 + L.K : p->ns;
        if (s != L.nseg - 1) {
            SweepArgs f = P.base;
            f.j_begin = j0; f.j_end = j1;
            f.prop_last = 0;
            f.init_ckpt = s;
            f.seg_base = j0; f.seg_from = j0;
            if ((rc = launch_coop((const void*)k_fwd, P.grid, P.smem, f, st, KID_FWD, u * (j1 - j0 - 1)))) return rc;
        }
        SweepArgs b = P.base;
        b.j_begin = j0; b.j_end = j1;
        b.seg_base = j0;
        if ((rc = launch_coop((const void*)k_adj, P.grid, P.smem, b, st, KID_ADJ, u * (j1 - j0)))) return rc;
    }
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
    int rc = prepare(p, MSLICE_OP_FORWARD, vol, probe, ws, ws_bytes, st, &P);
    if (rc) return rc;
    if (!intensity && !field_out) return MSLICE_EINVAL;
    const double u = (double)p->nw * p->ny * p->nz;
    SweepArgs a = P.base;
    a.intensity = intensity;
    a.field_out = (float2*)field_out;
    a.j_begin = 0;
    if (p->ns > 1) {
        a.j_end = p->ns - 1;
        a.prop_last = 1;
        if ((rc = launch_coop((const void*)k_fwd, P.grid, P.smem, a, st, KID_FWD, u * (p->ns - 1)))) return rc;
    }
    a.j_end = p->ns;
    if (p->flags & MSLICE_EXIT_WAVE)
        return launch_coop((const void*)k_last<C_EXIT>, P.grid, P.smem, a, st, KID_LAST, u);
    return launch_coop((const void*)k_last<C_FAR>, P.grid, P.smem, a, st, KID_LAST, u);
}

int mslice_adjoint(const mslice_params* p, const float* vol, const float* probe, const float* g_psi,
                   float* grad_vol, void* ws, size_t ws_bytes, void* stream) {
    cudaStream_t st = (cudaStream_t)stream;
    if (!g_psi || !grad_vol) return MSLICE_EINVAL;
    if (p && (p->flags & MSLICE_EXIT_WAVE)) return MSLICE_EUNSUPPORTED;
    Plan P;
    int rc = prepare(p, MSLICE_OP_ADJOINT, vol, probe, ws, ws_bytes, st, &P);
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
    Plan P;
    int rc = prepare(p, MSLICE_OP_LOSS_GRAD, vol, probe, ws, ws_bytes, st, &P);
    if (rc) return rc;
    P.base.meas = meas_amp;
    P.base.scale = scale;
    P.base.loss_out = loss_out;
    P.base.grad = (float2*)grad_vol;
    P.base.intensity = intensity;
    return run_gradient(p, P, true, st);
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
    for (int i = 0; i < p->nw; ++i) S.sin_alpha[i] = sin(p->alpha_i_rad[i]);
    S.tab = (float2*)(w + L.tab);
    S.probe_z = (float2*)(w + L.probe_z);
    S.py_out = (float2*)py; S.pz_out = (float2*)pz; S.probe_z_out = (float2*)probe_z;
    const int total = 2 * (p->ny + p->nz) + p->nw * p->nz;
    k_setup<<<(total + 255) / 256, 256, 0, st>>>(S);
    return cudaGetLastError() == cudaSuccess ? MSLICE_OK : MSLICE_ELAUNCH;
}

int mslice_transmission(const mslice_params* p, const float* vol, float* t_out, void* stream) {
    int rc = validate(p);
    if (rc) return rc;
    if (!vol || !t_out) return MSLICE_EINVAL;
    const double kd = 2.0 * M_PI / p->wavelength_nm * p->slice_nm;
    const size_t nvox = (size_t)p->ns * p->ny * p->nz;
    int tb = (int)((nvox + 255) / 256);
    if (tb > 4 * 152 * 8) tb = 4 * 152 * 8;
    k_transmission<<<tb, 256, 0, (cudaStream_t)stream>>>((const float2*)vol, (float2*)t_out, nvox, kd);
    return cudaGetLastError() == cudaSuccess ? MSLICE_OK : MSLICE_ELAUNCH;
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
