// mslice_device.cuh -- device code of libmslice (sm_103a): FFT engine, bounded
// grid barrier and the row / column passes of the multislice slice step.
//
// One slice (Eq. 1) is a pointwise transmission followed by a separable
// Fresnel propagation F^-1 P F with P(k_y, k_z) = P_y(k_y) P_z(k_z).  The 2-D
// FFT is split into a ROW pass (transmission, y-FFT, P_y, inverse y-FFT on one
// row held by a few threads) and a COLUMN pass (z-FFT, P_z, inverse z-FFT on a
// group of 16 columns).  Both passes of every slice run inside ONE persistent
// cooperative kernel per slice range: the wavefields (one per incidence angle,
// [nw][nz][ny] complex64, 2 MB each at 512^2) stay in L2 between passes and a
// bounded grid barrier separates the passes.  The only HBM stream of the
// forward pass is the precomputed transmission volume, prefetched into L2 one
// slice ahead.
//
// FFT of length N <= 1024 by T = N/32 threads (N > 32): each thread holds the
// 32 elements t + T*m, does a radix-32 DFT in registers (Stockham stage 1),
// exchanges once through padded shared memory, applies twiddles from a table
// and finishes with a radix-T DFT (stage 2).  The output lands in the same
// element pattern t + T*m, so the propagator multiply and the inverse FFT
// follow without another exchange; the inverse reuses the forward code as
// conj(F(conj(.))).  N <= 32: one thread per transform.
//
// The hot kernels are templates on the compile-time row and column lengths
// (0 = read them at run time), so that their code has no size branches and
// fits the instruction cache.
//
// Every identifier lives in an anonymous namespace: each translation unit that
// includes this header owns the kernels it instantiates.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "mslice.h"

#ifndef MS_THREADS
#define MS_THREADS 256
#endif
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
// the same sums as one paired FP32 instruction (IEEE round-to-nearest per
// half: bitwise equal to cadd / csub)
__device__ __forceinline__ unsigned long long pk2(float2 a) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a.x), "f"(a.y));
    return r;
}
__device__ __forceinline__ float2 upk2(unsigned long long r) {
    float2 a;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a.x), "=f"(a.y) : "l"(r));
    return a;
}
__device__ __forceinline__ float2 cadd2(float2 a, float2 b) {
    unsigned long long r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(pk2(a)), "l"(pk2(b)));
    return upk2(r);
}
__device__ __forceinline__ float2 csub2(float2 a, float2 b) {
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(pk2(a)), "l"(pk2(b)));
    return upk2(r);
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// a * w
__device__ __forceinline__ float2 cmul(float2 a, float2 w) {
    return make_float2(fmaf(a.x, w.x, -a.y * w.y), fmaf(a.x, w.y, a.y * w.x));
}
// a * (1 + u) and a * conj(1 + u), u = t - 1 from the transmission volume
// (t is kept as t - 1: FP32 holds |u| ~ 1e-2 to ~1e-10 absolute, where it
// holds t = 1 + u only to ~3e-8, an error that would repeat in every slice of
// a uniform material)
__device__ __forceinline__ float2 cmul_t(float2 a, float2 u) {
    return make_float2(fmaf(a.x, u.x, fmaf(-a.y, u.y, a.x)), fmaf(a.x, u.y, fmaf(a.y, u.x, a.y)));
}
__device__ __forceinline__ float2 cmulc_t(float2 a, float2 u) {
    return make_float2(fmaf(a.x, u.x, fmaf(a.y, u.y, a.x)), fmaf(a.y, u.x, fmaf(-a.x, u.y, a.y)));
}
// a * conj(w)
__device__ __forceinline__ float2 cmulc(float2 a, float2 w) {
    return make_float2(fmaf(a.x, w.x, a.y * w.y), fmaf(a.y, w.x, -a.x * w.y));
}

// FP32 (cos, sin)(pi e / 16), e = 0..15, for the in-register radix stages,
// written by csrc/gen_unit_twiddles.py: within six ulps of the correctly
// rounded values, chosen so that c^2 + s^2 - 1 summed over the twiddles a
// whole length-64..1024 transform applies is about zero (|drift| <= 5.7e-9).
// Correctly rounded pairs all have c^2 + s^2 < 1, which makes every forward +
// inverse transform lose ~5e-8 of the energy, identically in every slice
// (1.4e-4 of the intensity after 1024 slices at 512^2).
__host__ __device__ __forceinline__ constexpr float kTwC(int e) {
    switch (e) {
        case 0: return 0x1.0000000000000p+0f;
        case 1: return 0x1.f6297c0000000p-1f;
        case 2: return 0x1.d906c00000000p-1f;
        case 3: return 0x1.a9b6640000000p-1f;
        case 4: return 0x1.6a09e60000000p-1f;
        case 5: return 0x1.1c73b20000000p-1f;
        case 6: return 0x1.87de200000000p-2f;
        case 7: return 0x1.8f8b900000000p-3f;
        case 8: return 0.0f;
        case 9: return -0x1.8f8b900000000p-3f;
        case 10: return -0x1.87de200000000p-2f;
        case 11: return -0x1.1c73b20000000p-1f;
        case 12: return -0x1.6a09e60000000p-1f;
        case 13: return -0x1.a9b6640000000p-1f;
        case 14: return -0x1.d906c00000000p-1f;
        default: return -0x1.f6297c0000000p-1f;
    }
}
__host__ __device__ __forceinline__ constexpr float kTwS(int e) {
    switch (e) {
        case 0: return 0.0f;
        case 1: return 0x1.8f8b900000000p-3f;
        case 2: return 0x1.87de200000000p-2f;
        case 3: return 0x1.1c73b20000000p-1f;
        case 4: return 0x1.6a09e60000000p-1f;
        case 5: return 0x1.a9b6640000000p-1f;
        case 6: return 0x1.d906c00000000p-1f;
        case 7: return 0x1.f6297c0000000p-1f;
        case 8: return 0x1.0000000000000p+0f;
        case 9: return 0x1.f6297c0000000p-1f;
        case 10: return 0x1.d906c00000000p-1f;
        case 11: return 0x1.a9b6640000000p-1f;
        case 12: return 0x1.6a09e60000000p-1f;
        case 13: return 0x1.1c73b20000000p-1f;
        case 14: return 0x1.87de200000000p-2f;
        default: return 0x1.8f8b900000000p-3f;
    }
}

// log2 of a power of two (loop, inlined)
__host__ __device__ __forceinline__ constexpr int ilog2(int n) {
    int l = 0;
    while (n > 1) { n >>= 1; ++l; }
    return l;
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
    const float c = kTwC(e), s = kTwS(e);
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
                x[i0] = cadd2(a, b);
                x[i1] = tw32<INV>(csub2(a, b), k * (32 / (2 * HALF)));
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

// x <- U x with U = F^-1 diag(Ptab) F (ADJ: U^H, conj(Ptab)); Ptab holds P/N.
// The inverse transform is conj(F(conj(.))), so both passes run the same
// forward FFT code (one copy in the binary, a rolled two-pass loop).
template <bool ADJ, class SyncF>
__device__ __forceinline__ void propagate(float2 (&x)[32], const int n, const int T, const int t, float2* reg,
                                          const float2* __restrict__ Wt, const float2* __restrict__ Ptab,
                                          SyncF sync) {
    const int P = n > 32 ? 32 : n;
#pragma unroll 1
    for (int pass = 0; pass < 2; ++pass) {
        fft<false>(x, n, T, t, reg, Wt, sync);
        if (pass == 0) {
#pragma unroll
            for (int m = 0; m < 32; ++m) {
                if (m < P) {
                    const float2 p = Ptab[t + T * m], X = x[m];
                    // forward: conj(X p);  adjoint: conj(X) p
                    x[m] = ADJ ? make_float2(fmaf(X.x, p.x, X.y * p.y), fmaf(X.x, p.y, -X.y * p.x))
                               : make_float2(fmaf(X.x, p.x, -X.y * p.y), -fmaf(X.x, p.y, X.y * p.x));
                }
            }
        }
    }
#pragma unroll
    for (int m = 0; m < 32; ++m) x[m].y = -x[m].y;
}

// x <- F^-1 diag(p) F x along a column (ADJ: conj(p)), p read from the 2-D
// angular-spectrum table: pcol[l * ny] for the column's bins l (the table
// holds P / (ny nz); both transforms are unnormalised).
template <bool ADJ, class SyncF>
__device__ __forceinline__ void propagate2d(float2 (&x)[32], const int n, const int T, const int t, float2* reg,
                                            const float2* __restrict__ Wt, const float2* __restrict__ pcol,
                                            const int ny, const bool active, SyncF sync) {
    const int P = n > 32 ? 32 : n;
    fft<false>(x, n, T, t, reg, Wt, sync);
#pragma unroll
    for (int m = 0; m < 32; ++m) {
        if (m < P && active) {
            const float2 p = __ldg(pcol + (size_t)(t + T * m) * ny);
            x[m] = ADJ ? cmulc(x[m], p) : cmul(x[m], p);
        }
    }
    fft<true>(x, n, T, t, reg, Wt, sync);
}

// L2 prefetch of this block's share of [base, base + bytes): one bulk request.
__device__ __forceinline__ void prefetch_l2(const void* base, size_t bytes) {
    if (threadIdx.x != 0 || (bytes & 15) || ((uintptr_t)base & 15)) return;
    const size_t share = ((bytes + gridDim.x - 1) / gridDim.x + 15) & ~(size_t)15;
    const size_t off = (size_t)blockIdx.x * share;
    if (off >= bytes) return;
    size_t n = bytes - off < share ? bytes - off : share;
    const char* p = (const char*)base + off;
    while (n) {
        const unsigned c = n > 65536 ? 65536u : (unsigned)n;
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(c) : "memory");
        p += c;
        n -= c;
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

// exchange synchronisation of one transform's threads: a warp (or part of
// one), or a named barrier over the warps of a column group
struct WarpSync {
    __device__ __forceinline__ void operator()() const { __syncwarp(); }
};
struct GroupSync {
    int id, nthreads;
    __device__ __forceinline__ void operator()() const {
        if (nthreads <= 32) __syncwarp();
        else named_bar(id, nthreads);
    }
};

// ctrl[0] = status bits, ctrl[1] = arrivals, ctrl[2] = exits, ctrl[3] = arrivals
// of the second wavefield group (split-phase schedule)
struct Grid {
    unsigned* ctrl;
    unsigned nblocks;
    unsigned epoch;  // barriers passed so far in this launch
    long long timeout_ns;
    int* s_ok;       // shared flag

    // Every block arrives, then waits until all nblocks (+ withhold) arrived or
    // the wait exceeded timeout_ns; returns false (uniformly per block) on
    // timeout or if another block already reported one.
    __device__ __forceinline__ bool sync(unsigned withhold = 0) {
        __syncthreads();
        ++epoch;
        if (threadIdx.x == 0) {
            int ok = 1;
            const unsigned target = epoch * nblocks + withhold;
            // The block's writes are ordered before this thread by the
            // __syncthreads above; the gpu-scope release publishes them and the
            // acquire loads below order the other blocks' writes before ours.
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
            *(volatile int*)s_ok = ok;
        }
        __syncthreads();
        return *(volatile int*)s_ok != 0;
    }
    // Split-phase barrier on arrival counter ctrl[slot] (slots 1 and 3): a block
    // arrives once its writes of a phase are done and waits for the phase only
    // when it needs the other blocks' results, doing other work in between.
    __device__ __forceinline__ void arrive(int slot) {
        __syncthreads();
        if (threadIdx.x == 0) red_release_add(&ctrl[slot], 1u);
    }
    // Wait until every block made `arrivals` arrivals on ctrl[slot]; false
    // (uniformly per block) on timeout or an error reported by another block.
    __device__ __forceinline__ bool wait(int slot, unsigned arrivals) {
        if (threadIdx.x == 0) {
            int ok = 1;
            const unsigned target = arrivals * nblocks;
            unsigned long long t0 = globaltimer();
            unsigned spins = 0;
            while ((int)(ld_acquire(&ctrl[slot]) - target) < 0) {
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
            *(volatile int*)s_ok = ok;
        }
        __syncthreads();
        return *(volatile int*)s_ok != 0;
    }
    // last block out resets the counters for the next launch on the stream
    __device__ __forceinline__ void finish() {
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            const unsigned prev = atomicAdd(&ctrl[2], 1u);
            if (prev == nblocks - 1) {
                atomicExch(&ctrl[1], 0u);
                atomicExch(&ctrl[3], 0u);
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
    const float2* vol;      // [ns][nz][ny] delta + i beta (read by the adjoint when exact)
    const float2* probe;    // [nw][nz][ny] or null
    const float2* probe_z;  // [nw][nz] default probe rows
    const float2* probe_y;  // [nw][ny] in-plane tilt of each default probe, or null (every psi = 0)
    const float2* tab;      // Wt_y[ny] | Wt_z[nz] | P_y[ny]/ny | P_z[nz]/nz
    float2* field;          // [nw][nz][ny] forward state
    float2* gfield;         // [nw][nz][ny] adjoint state
    float2* gpart;          // [nw][nz][ny] per-wavefield gradient (nw > 1); [2][..] by slice
                            // parity under the split-phase schedule
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
    int per_w;              // 1: wavefield w has its own volume (tvol, grad: [nw][ns][nz][ny])
    int lcw;                // log2 of the columns per column-pass group
    int split;              // 1: two wavefield groups with split-phase barriers
    int exact;              // 1: exact 1 - n^2 transmission (gradient factor 1 - conj(v))
    const float2* p2d;      // [nz][ny] angular-spectrum propagator / (ny nz) (AS kernels only)
    const float2* tab2;     // one-pass kernels: table whose P parts serve the last slice's
                            // post-transmission propagation (half steps), or null
    int field_start;        // two-pass kernels: the first slice of the launch reads `field` as the
                            // output of a previous slice ((k_y, z) data with the angular spectrum:
                            // the half-stepped probe of the symmetric splitting)
    double* loss_task;      // one-pass loss: FP64 partial of every task of the detector pass
    double* loss_wsum;      // one-pass loss: per-wavefield sums [nw]
    float scales[MSLICE_MAX_ANGLES];  // per-wavefield loss scale when per_w
    // one-pass kernels, per-structure runs (per_w): every structure's own
    // buffers, so that structures need not be contiguous
    const float2* volw[MSLICE_MAX_ANGLES];   // [ns][nz][ny] delta + i beta (exact adjoint factor)
    float2* gradw[MSLICE_MAX_ANGLES];        // [ns][nz][ny] gradient out
    const float* measw[MSLICE_MAX_ANGLES];   // [nz][ny] detector amplitudes
    float* intw[MSLICE_MAX_ANGLES];          // [nz][ny] intensity out (entries may be null)
    double* lossw[MSLICE_MAX_ANGLES];        // per-structure loss out (entries may be null)
};

// transmission row / gradient row of wavefield w at slice j, row z
__device__ __forceinline__ size_t vol_offset(const SweepArgs& A, int w, int j, int z, int N) {
    const size_t npx = (size_t)A.ny * A.nz;
    return (A.per_w ? (size_t)w * A.ns * npx : 0) + (size_t)j * npx + (size_t)z * N;
}

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
    R_EXIT = 4,      // AS: back from (k_y, z): phi_Ns, |phi_Ns|^2         field -> outputs
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

#ifndef MS_ADJ_CHUNK
#define MS_ADJ_CHUNK 32  // a_j values loaded ahead of their gradient stores (all of a thread's)
#endif

// ----- row pass: one team of T = ny/32 threads (1 thread for ny <= 32) per row
// AS (angular-spectrum propagator): the propagator is not separable, so it is
// applied in the column pass on (k_y, k_z) and the field stays in (k_y, z)
// between the passes.  The row pass of slice j > 0 first undoes the
// y-transform of slice j-1 (unnormalised inverse; the 1/(ny nz) is in the 2-D
// table), applies the transmission in real space and transforms along y
// again; the adjoint runs the same steps with conj(t_j).
template <int OP, int NC = 0, bool AS = false>
__device__ void row_pass(const SweepArgs& A, const Smem& S, const int j, const bool first, const bool prop,
                         const int w0 = 0, int wn = 0) {
    if (wn <= 0) wn = A.nw;
    const int N = NC ? NC : A.ny, T = row_T(N), P = N > 32 ? 32 : N;
    const int tpw = 32 / T;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int tm = lane / T, t = lane % T;
    float2* reg = S.exch + (size_t)(warp * tpw + tm) * (N + N / 32);
    const size_t npx = (size_t)A.ny * A.nz;
    const int ntasks = A.nz * wn;
    const int wtasks = (ntasks + tpw - 1) / tpw;
    const WarpSync sync;
    for (int wt = blockIdx.x * MS_WARPS + warp; wt < wtasks; wt += gridDim.x * MS_WARPS) {
        const int task = wt * tpw + tm;
        const bool active = task < ntasks;
        const int z = active ? task / wn : 0, w = w0 + (active ? task % wn : 0);
        const size_t row = (size_t)w * npx + (size_t)z * N;
        float2 x[32];
#pragma unroll
        for (int m = 0; m < 32; ++m) x[m] = make_float2(0.f, 0.f);
        // checkpoint store, transmission a = t_j phi, segment store (real space)
        auto transmit = [&]() {
            if ((A.flags & F_STORE_CKPT) && (j % A.K == 0)) {
                float2* dst = A.ckpt + (size_t)(j / A.K) * A.nw * npx + row;
#pragma unroll
                for (int m = 0; m < 32; ++m) if (m < P) __stcg(dst + t + T * m, x[m]);
            }
            const float2* tv = A.tvol + vol_offset(A, w, j, z, N);
#pragma unroll
            for (int m = 0; m < 32; ++m) if (m < P) x[m] = cmul_t(x[m], __ldg(tv + t + T * m));
            if (j >= A.seg_from) {
                float2* dst = A.seg + (size_t)(j - A.seg_base) * A.nw * npx + row;
#pragma unroll
                for (int m = 0; m < 32; ++m) if (m < P) __stcg(dst + t + T * m, x[m]);
            }
        };
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
                    if (A.probe_y) {
#pragma unroll
                        for (int m = 0; m < 32; ++m)
                            if (m < P) x[m] = cmul(v, __ldg(A.probe_y + (size_t)w * A.ny + t + T * m));
                    } else {
#pragma unroll
                        for (int m = 0; m < 32; ++m) if (m < P) x[m] = v;
                    }
                }
                if constexpr (!AS) transmit();
            }
            if constexpr (AS) {
                if (!first) fft<true>(x, N, T, t, reg, S.Wy, sync);   // uniform: back from (k_y, z)
                if (active) transmit();
            }
            if (OP == R_FWD && !prop) continue;  // uniform
            if constexpr (OP == R_FAR) {
                fft<false>(x, N, T, t, reg, S.Wy, sync);
#pragma unroll
                for (int m = 0; m < 32; ++m) x[m] = cscale(x[m], A.ffy);
            } else if constexpr (AS) {
                fft<false>(x, N, T, t, reg, S.Wy, sync);              // to (k_y, z)
            } else {
                propagate<false>(x, N, T, t, reg, S.Wy, S.Py, sync);
            }
            if (active) {
#pragma unroll
                for (int m = 0; m < 32; ++m) if (m < P) __stcg(A.field + row + t + T * m, x[m]);
            }
        } else if constexpr (OP == R_ADJ) {
            // gradient of slice j from a_j and g = g_{a_j}, then g <- conj(t_j) g
            auto grad_back = [&]() {
                // x = g_{a_j}; gradient contribution -i kd a_j conj(g).  The loads of
                // a chunk of a_j are all issued before the chunk's gradient stores (the
                // compiler may not move a load across a store it cannot prove disjoint).
                const float2* a = A.seg + (size_t)(j - A.seg_base) * A.nw * npx + row;
                float2* gdst = (A.nw == 1 || A.per_w) ? (A.grad + vol_offset(A, w, j, z, N))
                                                      : (A.gpart + (size_t)(A.split & j) * A.nw * npx + row);
                if (!A.exact) {
#pragma unroll
                    for (int c = 0; c < 32; c += MS_ADJ_CHUNK) {
                        float2 av[MS_ADJ_CHUNK];
#pragma unroll
                        for (int k = 0; k < MS_ADJ_CHUNK; ++k)
                            if (c + k < P) av[k] = __ldcg(a + t + T * (c + k));
#pragma unroll
                        for (int k = 0; k < MS_ADJ_CHUNK; ++k) {
                            if (c + k < P) {
                                const float2 g = x[c + k];
                                const float re = fmaf(av[k].x, g.x, av[k].y * g.y);   // Re(a conj g)
                                const float im = fmaf(av[k].y, g.x, -av[k].x * g.y);  // Im(a conj g)
                                __stcg(gdst + t + T * (c + k), make_float2(A.kd * im, -A.kd * re));
                            }
                        }
                    }
                } else {
                    // exact transmission: d log t / dw = -i kd (1 - w), w = conj(v)
                    const float2* vv = A.vol + vol_offset(A, w, j, z, N);
#pragma unroll
                    for (int c = 0; c < 32; c += 8) {
                        float2 av[8], vk[8];
#pragma unroll
                        for (int k = 0; k < 8; ++k) {
                            if (c + k < P) {
                                av[k] = __ldcg(a + t + T * (c + k));
                                vk[k] = __ldg(vv + t + T * (c + k));
                            }
                        }
#pragma unroll
                        for (int k = 0; k < 8; ++k) {
                            if (c + k < P) {
                                const float2 g = x[c + k];
                                const float re = fmaf(av[k].x, g.x, av[k].y * g.y);
                                const float im = fmaf(av[k].y, g.x, -av[k].x * g.y);
                                const float fr = 1.f - vk[k].x, fi = vk[k].y;       // 1 - conj(v)
                                const float cr = fmaf(fr, re, -fi * im), ci = fmaf(fr, im, fi * re);
                                __stcg(gdst + t + T * (c + k), make_float2(A.kd * ci, -A.kd * cr));
                            }
                        }
                    }
                }
                if (prop) {
                    const float2* tv = A.tvol + vol_offset(A, w, j, z, N);
#pragma unroll
                    for (int m = 0; m < 32; ++m) if (m < P) x[m] = cmulc_t(x[m], __ldg(tv + t + T * m));
                }
            };
            if (active) {
#pragma unroll
                for (int m = 0; m < 32; ++m) if (m < P) x[m] = __ldcg(A.gfield + row + t + T * m);
                if constexpr (!AS) grad_back();
            }
            if constexpr (AS) {
                fft<true>(x, N, T, t, reg, S.Wy, sync);               // uniform: back from (k_y, z)
                if (active) grad_back();
            }
            if (!prop) continue;  // uniform
            if constexpr (AS) {
                fft<false>(x, N, T, t, reg, S.Wy, sync);
            } else {
                propagate<true>(x, N, T, t, reg, S.Wy, S.Py, sync);
            }
            if (active) {
#pragma unroll
                for (int m = 0; m < 32; ++m) if (m < P) __stcg(A.gfield + row + t + T * m, x[m]);
            }
        } else if constexpr (OP == R_EXIT) {
            // the exit wave of the angular-spectrum loop: the last column pass
            // left (k_y, z) data scaled by 1/ny; the unnormalised inverse
            // y-transform returns phi_Ns
            if (active) {
#pragma unroll
                for (int m = 0; m < 32; ++m) if (m < P) x[m] = __ldcg(A.field + row + t + T * m);
            }
            fft<true>(x, N, T, t, reg, S.Wy, sync);
            if (active) {
#pragma unroll
                for (int m = 0; m < 32; ++m) {
                    if (m < P) {
                        if (A.field_out) __stcs(A.field_out + row + t + T * m, x[m]);
                        if (A.intensity) __stcs(A.intensity + row + t + T * m, fmaf(x[m].x, x[m].x, x[m].y * x[m].y));
                    }
                }
            }
        } else {  // R_ADJ_FAR
            if (active) {
#pragma unroll
                for (int m = 0; m < 32; ++m) if (m < P) x[m] = __ldcg(A.gfield + row + t + T * m);
            }
            // AS: only the scale; the next adjoint row pass's inverse y-transform
            // completes F_y^H
            if constexpr (!AS) fft<true>(x, N, T, t, reg, S.Wy, sync);
            if (active) {
#pragma unroll
                for (int m = 0; m < 32; ++m) if (m < P) __stcg(A.gfield + row + t + T * m, cscale(x[m], A.ffy));
            }
        }
    }
}

// default columns per column group: at least 4 (a full 32-byte sector per row
// and thread row) and enough that the group fills a warp (cw * T >= 32), so
// that the group's exchange barrier spans as few warps as possible
__host__ __device__ __forceinline__ int col_cw(int T) { return 32 / T > 4 ? 32 / T : 4; }
// a column-group width is usable if it is a power of two >= 4 (>= 32 / T for
// small T) whose group divides the block
__host__ __device__ __forceinline__ bool col_cw_ok(int cw, int T) {
    return cw >= 1 && cw <= 32 && (cw & (cw - 1)) == 0 && cw * T <= MS_THREADS && MS_THREADS % (cw * T) == 0 &&
           cw >= (32 / T > 4 ? 4 : 32 / T) && (T > 1 || cw == 32);
}
// exchange-region stride of one column, = 16/cw (mod 16) in 8-byte words, so
// that the cw columns x 16/cw thread rows of a half-warp hit 16 distinct banks
__host__ __device__ __forceinline__ int col_rs(int N, int cw) { return N + N / 32 + 16 / cw; }

// ----- column pass: a group of cw*T threads per cw adjacent columns
template <int OP, int NC = 0, bool AS = false, int NYC = 0>
__device__ void col_pass(const SweepArgs& A, const Smem& S, double* s_red, const int w0 = 0, int wn = 0) {
    if (wn <= 0) wn = A.nw;
    const int N = NC ? NC : A.nz, T = row_T(N), P = N > 32 ? 32 : N;
    const int NYr = NYC ? NYC : A.ny;   // row length: the column stride (compile-time when known)
    const int lcw = A.lcw, cw = 1 << lcw;
    const int lg = lcw + ilog2(T), gthreads = 1 << lg;
    const int groups = MS_THREADS >> lg;
    const int g = threadIdx.x >> lg, gt = threadIdx.x & (gthreads - 1);
    const int c = gt & (cw - 1), t = gt >> lcw;
    float2* reg = S.exch + (size_t)(g * cw + c) * col_rs(N, cw);
    const size_t npx = (size_t)A.ny * A.nz;
    const int ncg = (NYr + cw - 1) / cw;
    const int ntasks = ncg * wn;
    const GroupSync sync{1 + g, gthreads};
    const float2* src = (OP == C_ADJ) ? A.gfield : (OP == C_SEED ? A.gpsi : A.field);
    double loss = 0.0;
    for (int task = blockIdx.x * groups + g; task < ntasks; task += gridDim.x * groups) {
        const int cg = task / wn, w = w0 + task % wn;
        const int col = cg * cw + c;
        const bool active = col < NYr;
        const size_t base = (size_t)w * ((size_t)NYr * N) + col;
        float2 x[32];
#pragma unroll
        for (int m = 0; m < 32; ++m) {
            x[m] = make_float2(0.f, 0.f);
            if (active && m < P) x[m] = __ldcg(src + base + (size_t)(t + T * m) * NYr);
        }
        if constexpr (OP == C_PROP || OP == C_EXIT || OP == C_ADJ) {
            if constexpr (AS) propagate2d<OP == C_ADJ>(x, N, T, t, reg, S.Wz, A.p2d + col, NYr, active, sync);
            else propagate<OP == C_ADJ>(x, N, T, t, reg, S.Wz, S.Pz, sync);
        } else {
            if constexpr (OP != C_SEED) fft<false>(x, N, T, t, reg, S.Wz, sync);
            if constexpr (OP == C_FAR || OP == C_FAR_LOSS) {
#pragma unroll
                for (int m = 0; m < 32; ++m) {
                    if (m < P) {
                        const float2 psi = cscale(x[m], A.ffz);
                        const float I = fmaf(psi.x, psi.x, psi.y * psi.y);
                        const size_t o = base + (size_t)(t + T * m) * NYr;
                        if (active) {
                            if (A.intensity) __stcs(A.intensity + o, I);
                            if (A.field_out) __stcs(A.field_out + o, psi);
                        }
                        if constexpr (OP == C_FAR_LOSS) {
                            float2 gs = make_float2(0.f, 0.f);
                            if (active) {
                                const float sc = A.per_w ? A.scales[w] : A.scale;
                                const float r = sqrtf(sc * I);
                                const float d = r - __ldg(A.meas + o);
                                loss += (double)d * (double)d;
                                if (r > 0.f) gs = cscale(psi, 2.f * sc * d / r);
                            }
                            x[m] = gs;
                        }
                    }
                }
            }
            if constexpr (OP == C_FAR) continue;
            fft<true>(x, N, T, t, reg, S.Wz, sync);   // C_SEED, C_FAR_LOSS: F_z^H
        }
        if (!active) continue;
        if constexpr (OP == C_SEED || OP == C_FAR_LOSS) {
#pragma unroll
            for (int m = 0; m < 32; ++m)
                if (m < P) __stcg(A.gfield + base + (size_t)(t + T * m) * NYr, cscale(x[m], A.ffz));
        } else {
            float2* dst = (OP == C_ADJ) ? A.gfield : A.field;
#pragma unroll
            for (int m = 0; m < 32; ++m) {
                if (m < P) {
                    const size_t o = base + (size_t)(t + T * m) * NYr;
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

// grad[j] = sum_w gpart[w]  (fixed order over w).  Two grid points per thread
// step with 16-byte accesses when the sizes and the gradient pointer allow,
// the nw loads of a step issued before their sum.
__device__ void reduce_gpart(const SweepArgs& A, int j) {
    const size_t npx = (size_t)A.ny * A.nz;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    const size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const float2* gp = A.gpart + (size_t)(A.split & j) * A.nw * npx;
    float2* dst = A.grad + (size_t)j * npx;
    if ((npx & 1) == 0 && ((uintptr_t)dst & 15) == 0) {
        const size_t n4 = npx / 2;
        const float4* g4 = reinterpret_cast<const float4*>(gp);
        float4* d4 = reinterpret_cast<float4*>(dst);
        // two grid points per thread and step: all loads of both before either store
        for (size_t i = tid; i < n4; i += 2 * stride) {
            const size_t i2 = i + stride;
            const bool has2 = i2 < n4;
            float4 s1 = make_float4(0.f, 0.f, 0.f, 0.f), s2 = s1;
            for (int w0 = 0; w0 < A.nw; w0 += 4) {
                float4 v1[4], v2[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    if (w0 + k < A.nw) {
                        v1[k] = __ldcg(g4 + (size_t)(w0 + k) * n4 + i);
                        if (has2) v2[k] = __ldcg(g4 + (size_t)(w0 + k) * n4 + i2);
                    }
                }
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    if (w0 + k < A.nw) {
                        if (w0 + k == 0) {
                            s1 = v1[0];
                            s2 = v2[0];
                        } else {
                            s1.x += v1[k].x; s1.y += v1[k].y; s1.z += v1[k].z; s1.w += v1[k].w;
                            s2.x += v2[k].x; s2.y += v2[k].y; s2.z += v2[k].z; s2.w += v2[k].w;
                        }
                    }
                }
            }
            __stcs(d4 + i, s1);
            if (has2) __stcs(d4 + i2, s2);
        }
        return;
    }
    for (size_t i = tid; i < npx; i += stride) {
        float2 s = __ldcg(gp + i);
        for (int w = 1; w < A.nw; ++w) s = cadd(s, __ldcg(gp + (size_t)w * npx + i));
        __stcs(dst + i, s);
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
// The last slice of the range propagates only if A.prop_last.  NY, NZ: the
// compile-time row and column lengths (0: from A).
template <int NY, int NZ, bool AS = false>
__global__ void __launch_bounds__(MS_THREADS, 1) k_fwd_t(const SweepArgs A) {
    MS_KERNEL_PROLOGUE
    const size_t npx = (size_t)A.ny * A.nz;
    const size_t slice_bytes = npx * sizeof(float2);
    if (!A.split) {
        for (int j = A.j_begin; j < A.j_end; ++j) {
            const bool prop = (j < A.j_end - 1) || A.prop_last;
            row_pass<R_FWD, NY, AS>(A, S, j, j == A.j_begin && !A.field_start, prop);
            if (prop) {
                if (!grid.sync()) return;
                if (j + 1 < A.j_end) {
                    for (int w = 0; w < (A.per_w ? A.nw : 1); ++w)
                        prefetch_l2(A.tvol + (size_t)w * A.ns * npx * A.per_w + (size_t)(j + 1) * npx, slice_bytes);
                }
                col_pass<C_PROP, NZ, AS, NY>(A, S, s_red);
                if (j < A.j_end - 1 && !grid.sync()) return;
            }
        }
        grid.finish();
        return;
    }
    // Split-phase schedule: wavefields [0, h) and [h, nw) advance in the order
    // R0(j) R1(j) C0(j) C1(j) R0(j+1) ...; a block waits for the other blocks
    // only where it reads their results, one half-phase after it arrived, so the
    // barrier latency and the blocks' imbalance overlap with the other group.
    const int h = (A.nw + 1) / 2;
    const int gw0[2] = {0, h}, gwn[2] = {h, A.nw - h}, slot[2] = {1, 3};
    unsigned arr[2] = {0u, 0u};
    for (int j = A.j_begin; j < A.j_end; ++j) {
        const bool prop = (j < A.j_end - 1) || A.prop_last;
#pragma unroll
        for (int g = 0; g < 2; ++g) {
            if (j > A.j_begin && !grid.wait(slot[g], arr[g])) return;   // C_g(j-1) done
            row_pass<R_FWD, NY, AS>(A, S, j, j == A.j_begin && !A.field_start, prop, gw0[g], gwn[g]);
            if (prop) {
                grid.arrive(slot[g]);
                ++arr[g];
            }
        }
        if (!prop) break;
        if (j + 1 < A.j_end) {
            for (int w = 0; w < (A.per_w ? A.nw : 1); ++w)
                prefetch_l2(A.tvol + (size_t)w * A.ns * npx * A.per_w + (size_t)(j + 1) * npx, slice_bytes);
        }
#pragma unroll
        for (int g = 0; g < 2; ++g) {
            if (!grid.wait(slot[g], arr[g])) return;                       // R_g(j) done
            col_pass<C_PROP, NZ, AS, NY>(A, S, s_red, gw0[g], gwn[g]);
            if (j < A.j_end - 1) {
                grid.arrive(slot[g]);
                ++arr[g];
            }
        }
    }
    grid.finish();
}

// Last slice (j = ns-1) with the far field, optionally the loss and its seed.
template <int COL, bool AS = false>
__global__ void __launch_bounds__(MS_THREADS, 1) k_last(const SweepArgs A) {
    MS_KERNEL_PROLOGUE
    const int j = A.ns - 1;
    const bool first = j == A.j_begin && !A.field_start;
    if constexpr (COL == C_EXIT) row_pass<R_FWD, 0, AS>(A, S, j, first, true);
    else row_pass<R_FAR, 0, AS>(A, S, j, first, true);
    if (!grid.sync()) return;
    if constexpr (COL == C_EXIT && AS) {
        // angular spectrum: propagate on (k_y, k_z), then back to real space
        col_pass<C_PROP, 0, AS>(A, S, s_red);
        if (!grid.sync()) return;
        row_pass<R_EXIT, 0, AS>(A, S, j, false, true);
    } else {
        col_pass<COL, 0, AS>(A, S, s_red);
    }
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
template <bool SEED, bool AS = false>
__global__ void __launch_bounds__(MS_THREADS, 1) k_adj_start(const SweepArgs A) {
    MS_KERNEL_PROLOGUE
    if constexpr (SEED) {
        col_pass<C_SEED, 0, AS>(A, S, s_red);
        if (!grid.sync()) return;
    }
    row_pass<R_ADJ_FAR, 0, AS>(A, S, A.ns - 1, false, true);
    grid.finish();
}

// Adjoint slice loop, j from j_end-1 down to j_begin (a_j in the segment
// buffer).  The transmission and a_j of the next slice are prefetched into L2
// during the column pass.
template <int NY, int NZ, bool AS = false>
__global__ void __launch_bounds__(MS_THREADS, 1) k_adj_t(const SweepArgs A) {
    MS_KERNEL_PROLOGUE
    const size_t npx = (size_t)A.ny * A.nz;
    const bool reduce = A.nw > 1 && !A.per_w;
    if (!A.split) {
        for (int j = A.j_end - 1; j >= A.j_begin; --j) {
            row_pass<R_ADJ, NY, AS>(A, S, j, false, j > 0);
            if (!grid.sync()) return;
            if (j - 1 >= A.j_begin) {
                for (int w = 0; w < (A.per_w ? A.nw : 1); ++w)
                    prefetch_l2(A.tvol + (size_t)w * A.ns * npx * A.per_w + (size_t)(j - 1) * npx,
                                npx * sizeof(float2));
                prefetch_l2(A.seg + (size_t)(j - 1 - A.seg_base) * A.nw * npx, A.nw * npx * sizeof(float2));
            }
            if (j > 0) col_pass<C_ADJ, NZ, AS, NY>(A, S, s_red);
            if (reduce) reduce_gpart(A, j);
            if (j > A.j_begin && !grid.sync()) return;
        }
        grid.finish();
        return;
    }
    // Split-phase schedule as in k_fwd_t.  The gradient partials of slice j are
    // summed after R_1(j) is complete everywhere (which implies R_0(j): every
    // block arrives for R_1(j) after its own R_0(j)); they are double-buffered
    // by slice parity because R_0(j-1) may start before every block has read them.
    const int h = (A.nw + 1) / 2;
    const int gw0[2] = {0, h}, gwn[2] = {h, A.nw - h}, slot[2] = {1, 3};
    unsigned arr[2] = {0u, 0u};
    for (int j = A.j_end - 1; j >= A.j_begin; --j) {
#pragma unroll
        for (int g = 0; g < 2; ++g) {
            if (j < A.j_end - 1 && !grid.wait(slot[g], arr[g])) return;   // C_g(j+1) done
            row_pass<R_ADJ, NY, AS>(A, S, j, false, j > 0, gw0[g], gwn[g]);
            grid.arrive(slot[g]);
            ++arr[g];
        }
        if (j - 1 >= A.j_begin) {
            for (int w = 0; w < (A.per_w ? A.nw : 1); ++w)
                prefetch_l2(A.tvol + (size_t)w * A.ns * npx * A.per_w + (size_t)(j - 1) * npx, npx * sizeof(float2));
            prefetch_l2(A.seg + (size_t)(j - 1 - A.seg_base) * A.nw * npx, A.nw * npx * sizeof(float2));
        }
#pragma unroll
        for (int g = 0; g < 2; ++g) {
            if (!grid.wait(slot[g], arr[g])) return;                        // R_g(j) done
            if (j > 0) col_pass<C_ADJ, NZ, AS, NY>(A, S, s_red, gw0[g], gwn[g]);
            if (g == 1 && reduce) reduce_gpart(A, j);
            if (j > A.j_begin) {
                grid.arrive(slot[g]);
                ++arr[g];
            }
        }
    }
    grid.finish();
}

}  // namespace
