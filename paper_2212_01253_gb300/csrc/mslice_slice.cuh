// mslice_slice.cuh -- the slice loop with ONE pass per slice (paraxial
// propagator of Eq. 1), built on the FFT engine, the bounded grid barrier and
// the argument block of mslice_device.cuh.
//
// Eq. 1's propagator is separable, P(k_y, k_z) = P_y(k_y) P_z(k_z), so the
// propagation of a slice is U = U_y U_z = U_z U_y with U_y = F_y^-1 P_y F_y
// along the rows and U_z along the columns.  Slice j applies its two factors in
// the order (U_y, U_z) for even j and (U_z, U_y) for odd j.  The operator
// sequence of the whole loop,
//     t_0 U_y U_z | t_1 U_z U_y | t_2 U_y U_z | t_3 U_z U_y | ...
// then regroups into passes that each work along ONE axis:
//     [t_0 U_y] [U_z t_1 U_z] [U_y t_2 U_y] [U_z t_3 U_z] ...
// Pass j runs along the rows for even j and along the columns for odd j: it
// finishes slice j-1's propagation (the factor along its axis), applies the
// transmission t_j, and starts slice j's propagation (the same factor).  Between
// passes the stored field s_j = U_ax(j-1) a_{j-1} is "half propagated".  Per
// slice this is one grid barrier and one L2 round trip of the field instead of
// two; the FFT work is unchanged (four length-N transforms per grid point).
//
// The field phi_{j-1} that enters slice j (checkpoints) and a_j = t_j phi_{j-1}
// (segment buffer of the adjoint) both exist in registers inside pass j.  The
// adjoint runs the passes backward: g_{a_j} = U_ax^H g, the gradient of slice j,
// g <- conj(t_j) g, g <- U_ax^H g.  Its first pass starts with F_ax^H (the far
// field's transform along that axis) instead of U_ax^H.
//
// Rounding: U_y and U_z commute exactly but not in FP32; the order per slice is
// fixed by the parity of j, so every result is the same for any checkpoint
// interval, launch shape or slice range split.
#pragma once
#include "mslice_device.cuh"

#ifndef MS_MIN_BLOCKS
#define MS_MIN_BLOCKS 1
#endif

namespace {

enum : int {
    F_FIRST_FAR = 2,   // adjoint: the pass of slice ns-1 starts with F_ax^H (far field)
    F_PROP_FULL = 4,   // forward: after the range, apply the other axis's factor too
};

// pass operations
enum : int {
    P_FWD = 0,        // [U] ckpt, t, seg, [U]                           field -> field
    P_ADJ = 1,        // U^H (or F^H), gradient, conj(t), U^H             gfield -> gfield
    P_LAST_FAR = 2,   // [U] ckpt, t, seg, F / sqrt(N)                    field -> field
    P_LAST_EXIT = 3,  // [U] ckpt, t, seg, U (tab2)                       field -> field
    P_FAR = 4,        // F / sqrt(N): Psi, I = |Psi|^2                     field -> I, Psi
    P_FAR_LOSS = 5,   // P_FAR, loss partial, seed g, F^H g / sqrt(N)      field -> gfield
    P_EXIT = 6,       // U (tab2): phi_Ns, |phi_Ns|^2                      field -> outputs
    P_SEED = 7,       // F^H g_psi / sqrt(N)                                gpsi -> gfield
    P_PROP = 8,       // U                                                 field -> field
};

__host__ __device__ __forceinline__ int pass_axis(int j) { return j & 1; }
// threads of a column group of 2^lcw columns of T threads
__host__ __device__ __forceinline__ int gthreads_of(int lcw, int T) { return (1 << lcw) * T; }

// shared-memory tables of the one-pass kernels: Wt_y | Wt_z | P_y/ny | P_z/nz
// [| P2_y/ny | P2_z/nz from tab2]
struct Smem2 {
    float2* exch;
    const float2* W[2];    // twiddles by axis (0: y, 1: z)
    const float2* P[2];    // propagator / N by axis
    const float2* P2[2];   // second propagator (tab2, else P)
};

__device__ Smem2 load_tables2(const SweepArgs& A, float2* base) {
    const int n = 2 * (A.ny + A.nz);
    for (int i = threadIdx.x; i < n; i += blockDim.x) base[i] = A.tab[i];
    const int n2 = A.tab2 ? A.ny + A.nz : 0;
    for (int i = threadIdx.x; i < n2; i += blockDim.x) base[n + i] = A.tab2[A.ny + A.nz + i];
    __syncthreads();
    Smem2 S;
    S.W[0] = base;
    S.W[1] = base + A.ny;
    S.P[0] = base + A.ny + A.nz;
    S.P[1] = base + 2 * A.ny + A.nz;
    S.P2[0] = A.tab2 ? base + n : S.P[0];
    S.P2[1] = A.tab2 ? base + n + A.ny : S.P[1];
    S.exch = base + n + n2;
    return S;
}

// One pass along axis AX (0: rows, transforms along y; 1: columns, along z) at
// slice j.  NY, NZ: compile-time row and column lengths (0: from A).
//   rows:    a team of T = N/32 threads per row (several rows per warp), tasks
//            (z, w) with z major, so that the wavefields of a row share the
//            transmission row in L2;
//   columns: a group of cw columns x T threads, tasks (column group, w).
// Thread t of a team holds the elements t + T m (m < 32) of its row or column.
template <int AX, int OP, int NY, int NZ>
__device__ void pass(const SweepArgs& A, const Smem2& S, double* s_red, const int j, const bool first,
                     const bool prop) {
    constexpr int NC = AX == 0 ? NY : NZ;
    const int ny = NY ? NY : A.ny;
    const int N = NC ? NC : (AX == 0 ? A.ny : A.nz);
    const int T = row_T(N), P = N > 32 ? 32 : N;
    const size_t npx = (size_t)ny * (AX == 0 ? (NZ ? NZ : A.nz) : N);
    const int nw = A.nw;
    const float ff = AX == 0 ? A.ffy : A.ffz;
    const float2* W = S.W[AX];
    // team geometry and task range
    int t, ntasks, task0, tstep, tpt = 1;
    float2* reg;
    int lcw = 0, c = 0;
    GroupSync sync{0, 32};
    if constexpr (AX == 0) {
        const int tpw = 32 / T;
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        const int tm = lane / T;
        t = lane % T;
        reg = S.exch + (size_t)(warp * tpw + tm) * (N + N / 32);
        tpt = tpw;
        ntasks = A.nz * nw;
        task0 = (blockIdx.x * MS_WARPS + warp) * tpw + tm;
        tstep = gridDim.x * MS_WARPS * tpw;
        sync = GroupSync{0, T};   // T <= 32: __syncwarp
    } else {
        lcw = A.lcw;
        const int cw = 1 << lcw;
        const int lg = lcw + ilog2(T), gthreads = 1 << lg;
        const int groups = MS_THREADS >> lg;
        const int g = threadIdx.x >> lg, gt = threadIdx.x & (gthreads - 1);
        c = gt & (cw - 1);
        t = gt >> lcw;
        reg = S.exch + (size_t)(g * cw + c) * col_rs(N, cw);
        ntasks = ((ny + cw - 1) / cw) * nw;
        task0 = blockIdx.x * groups + g;
        tstep = gridDim.x * groups;
        sync = GroupSync{1 + g, gthreads};
    }
    // element m of the task sits at plane offset e0 + m * es
    const size_t es = AX == 0 ? (size_t)T : (size_t)T * ny;
    // rows: the teams of a warp iterate together, so that __syncwarp sees every
    // lane: team tm runs while the warp's first task (task - tm) is in range
    const int tlim = AX == 0 ? ntasks + task0 % tpt : ntasks;
    for (int task = task0; task < tlim; task += tstep) {
        bool active = task < ntasks;
        int w, e_row, col = 0;
        if constexpr (AX == 0) {
            const int tk = active ? task : 0;
            e_row = tk / nw;
            w = tk % nw;
        } else {
            const int cw = 1 << lcw;
            w = task % nw;
            col = (task / nw) * cw + c;
            active = col < ny;
            e_row = 0;
        }
        const size_t e0 = AX == 0 ? (size_t)e_row * ny + t : (size_t)t * ny + (active ? col : 0);
        const size_t fo = (size_t)w * npx + e0;                            // field-like [nw][nz][ny]
        const size_t vo = (A.per_w ? (size_t)w * A.ns * npx : 0) + (size_t)j * npx + e0;   // volume-like
        float2 x[32];
#pragma unroll
        for (int m = 0; m < 32; ++m) x[m] = make_float2(0.f, 0.f);

        if constexpr (OP == P_FWD || OP == P_LAST_FAR || OP == P_LAST_EXIT || OP == P_PROP) {
            if (active) {
                if (!first || OP == P_PROP) {
#pragma unroll
                    for (int m = 0; m < 32; ++m) if (m < P) x[m] = __ldcg(A.field + fo + m * es);
                } else if (A.init_ckpt >= 0) {
                    const float2* src = A.ckpt + (size_t)A.init_ckpt * nw * npx + fo;
#pragma unroll
                    for (int m = 0; m < 32; ++m) if (m < P) x[m] = __ldcg(src + m * es);
                } else if (A.probe) {
#pragma unroll
                    for (int m = 0; m < 32; ++m) if (m < P) x[m] = __ldg(A.probe + fo + m * es);
                } else if constexpr (AX == 0) {
                    const float2 v = A.probe_z[(size_t)w * A.nz + e_row];
#pragma unroll
                    for (int m = 0; m < 32; ++m)
                        if (m < P) x[m] = A.probe_y ? cmul(v, __ldg(A.probe_y + (size_t)w * ny + t + T * m)) : v;
                } else {
                    const float2 v = A.probe_y ? __ldg(A.probe_y + (size_t)w * ny + col) : make_float2(1.f, 0.f);
#pragma unroll
                    for (int m = 0; m < 32; ++m)
                        if (m < P) x[m] = cmul(__ldg(A.probe_z + (size_t)w * A.nz + t + T * m), v);
                }
            }
            if constexpr (OP == P_PROP) {
                propagate<false>(x, N, T, t, reg, W, S.P[AX], sync);
            } else {
                // the second factor of slice j-1's propagation (uniform condition)
                if (!first) propagate<false>(x, N, T, t, reg, W, S.P[AX], sync);
                if (active) {
                    if ((A.flags & F_STORE_CKPT) && (j % A.K == 0)) {
                        float2* dst = A.ckpt + (size_t)(j / A.K) * nw * npx + fo;
#pragma unroll
                        for (int m = 0; m < 32; ++m) if (m < P) __stcg(dst + m * es, x[m]);
                    }
                    const float2* tv = A.tvol + vo;
#pragma unroll
                    for (int m = 0; m < 32; ++m) if (m < P) x[m] = cmul_t(x[m], __ldg(tv + m * es));
                    if (j >= A.seg_from) {
                        float2* dst = A.seg + (size_t)(j - A.seg_base) * nw * npx + fo;
#pragma unroll
                        for (int m = 0; m < 32; ++m) if (m < P) __stcg(dst + m * es, x[m]);
                    }
                }
                if (OP == P_FWD && !prop) continue;   // uniform
                if constexpr (OP == P_LAST_FAR) {
                    fft<false>(x, N, T, t, reg, W, sync);
#pragma unroll
                    for (int m = 0; m < 32; ++m) x[m] = cscale(x[m], ff);
                } else if constexpr (OP == P_LAST_EXIT) {
                    propagate<false>(x, N, T, t, reg, W, S.P2[AX], sync);
                } else {
                    propagate<false>(x, N, T, t, reg, W, S.P[AX], sync);
                }
            }
            if (active) {
#pragma unroll
                for (int m = 0; m < 32; ++m) if (m < P) __stcg(A.field + fo + m * es, x[m]);
            }
        } else if constexpr (OP == P_ADJ) {
            if (active) {
#pragma unroll
                for (int m = 0; m < 32; ++m) if (m < P) x[m] = __ldcg(A.gfield + fo + m * es);
            }
            // U^H g_b t U^H as one rolled loop of four transforms; the pass of
            // slice ns-1 starts with F^H = conj F conj / sqrt(N) instead
            const bool far = (A.flags & F_FIRST_FAR) && j == A.ns - 1;   // uniform
            if (far) {
#pragma unroll
                for (int m = 0; m < 32; ++m) x[m].y = -x[m].y;
            }
#pragma unroll 1
            for (int s = far ? 1 : 0; s < 4; ++s) {
                fft<false>(x, N, T, t, reg, W, sync);
                if (!(s & 1)) {
                    const float2* Pt = S.P[AX];
#pragma unroll
                    for (int m = 0; m < 32; ++m) {
                        if (m < P) {
                            const float2 p = Pt[t + T * m], X = x[m];
                            x[m] = make_float2(fmaf(X.x, p.x, X.y * p.y), fmaf(X.x, p.y, -X.y * p.x));
                        }
                    }
                } else {
#pragma unroll
                    for (int m = 0; m < 32; ++m) x[m].y = -x[m].y;
                    if (s == 1) {
                        if (far) {
#pragma unroll
                            for (int m = 0; m < 32; ++m) x[m] = cscale(x[m], ff);
                        }
                        if (active) {
                            // x = g_{a_j}: gradient -i kd a_j conj(g) (linearised) or with the
                            // factor (1 - conj(v)) (exact); the loads of a chunk of a_j are
                            // issued before the chunk's stores, and marked evict-first (a_j is
                            // read once; the fields and gradient partials should stay in L2)
                            const float2* a = A.seg + (size_t)(j - A.seg_base) * nw * npx + fo;
                            float2* gdst = A.per_w ? (A.gradw[w] + (size_t)j * npx + e0)
                                           : (nw == 1 ? (A.grad + vo) : (A.gpart + (size_t)(j & 1) * nw * npx + fo));
                            if (!A.exact) {
#pragma unroll
                                for (int c0 = 0; c0 < 32; c0 += MS_ADJ_CHUNK) {
                                    float2 av[MS_ADJ_CHUNK];
#pragma unroll
                                    for (int k = 0; k < MS_ADJ_CHUNK; ++k)
                                        if (c0 + k < P) av[k] = __ldcs(a + (c0 + k) * es);
#pragma unroll
                                    for (int k = 0; k < MS_ADJ_CHUNK; ++k) {
                                        if (c0 + k < P) {
                                            const float2 g = x[c0 + k];
                                            const float re = fmaf(av[k].x, g.x, av[k].y * g.y);   // Re(a conj g)
                                            const float im = fmaf(av[k].y, g.x, -av[k].x * g.y);  // Im(a conj g)
                                            __stcg(gdst + (c0 + k) * es, make_float2(A.kd * im, -A.kd * re));
                                        }
                                    }
                                }
                            } else {
                                const float2* vv = A.per_w ? (A.volw[w] + (size_t)j * npx + e0) : (A.vol + vo);
#pragma unroll
                                for (int c0 = 0; c0 < 32; c0 += 8) {
                                    float2 av[8], vk[8];
#pragma unroll
                                    for (int k = 0; k < 8; ++k) {
                                        if (c0 + k < P) {
                                            av[k] = __ldcs(a + (c0 + k) * es);
                                            vk[k] = __ldg(vv + (c0 + k) * es);
                                        }
                                    }
#pragma unroll
                                    for (int k = 0; k < 8; ++k) {
                                        if (c0 + k < P) {
                                            const float2 g = x[c0 + k];
                                            const float re = fmaf(av[k].x, g.x, av[k].y * g.y);
                                            const float im = fmaf(av[k].y, g.x, -av[k].x * g.y);
                                            const float fr = 1.f - vk[k].x, fi = vk[k].y;       // 1 - conj(v)
                                            const float cr = fmaf(fr, re, -fi * im), ci = fmaf(fr, im, fi * re);
                                            __stcg(gdst + (c0 + k) * es, make_float2(A.kd * ci, -A.kd * cr));
                                        }
                                    }
                                }
                            }
                            if (prop) {
                                const float2* tv = A.tvol + vo;
#pragma unroll
                                for (int m = 0; m < 32; ++m) if (m < P) x[m] = cmulc_t(x[m], __ldg(tv + m * es));
                            }
                        }
                        if (!prop) break;   // uniform
                    }
                }
            }
            if (!prop) continue;   // uniform
            if (active) {
#pragma unroll
                for (int m = 0; m < 32; ++m) if (m < P) __stcg(A.gfield + fo + m * es, x[m]);
            }
        } else if constexpr (OP == P_SEED) {
            if (active) {
#pragma unroll
                for (int m = 0; m < 32; ++m) if (m < P) x[m] = __ldg(A.gpsi + fo + m * es);
            }
            fft<true>(x, N, T, t, reg, W, sync);
            if (active) {
#pragma unroll
                for (int m = 0; m < 32; ++m) if (m < P) __stcg(A.gfield + fo + m * es, cscale(x[m], ff));
            }
        } else {   // P_FAR, P_FAR_LOSS, P_EXIT
            if (active) {
#pragma unroll
                for (int m = 0; m < 32; ++m) if (m < P) x[m] = __ldcg(A.field + fo + m * es);
            }
            // intensity out: the structure's own buffer (per_w) or [nw][nz][ny]
            float* iout = A.per_w ? (A.intw[w] ? A.intw[w] + e0 : nullptr) : (A.intensity ? A.intensity + fo : nullptr);
            if constexpr (OP == P_EXIT) {
                propagate<false>(x, N, T, t, reg, W, S.P2[AX], sync);
                if (active) {
#pragma unroll
                    for (int m = 0; m < 32; ++m) {
                        if (m < P) {
                            if (A.field_out) __stcs(A.field_out + fo + m * es, x[m]);
                            if (iout) __stcs(iout + m * es, fmaf(x[m].x, x[m].x, x[m].y * x[m].y));
                        }
                    }
                }
                continue;
            } else {
                fft<false>(x, N, T, t, reg, W, sync);
                const float* mamp = A.per_w ? A.measw[w] + e0 : A.meas + fo;
                double tl = 0.0;   // this thread's share of the task's loss
#pragma unroll
                for (int m = 0; m < 32; ++m) {
                    if (m < P) {
                        const float2 psi = cscale(x[m], ff);
                        const float I = fmaf(psi.x, psi.x, psi.y * psi.y);
                        if (active) {
                            if (iout) __stcs(iout + m * es, I);
                            if (A.field_out) __stcs(A.field_out + fo + m * es, psi);
                        }
                        if constexpr (OP == P_FAR_LOSS) {
                            float2 gs = make_float2(0.f, 0.f);
                            if (active) {
                                const float sc = A.per_w ? A.scales[w] : A.scale;
                                const float r = sqrtf(sc * I);
                                const float d = r - __ldg(mamp + m * es);
                                tl += (double)d * (double)d;
                                if (r > 0.f) gs = cscale(psi, 2.f * sc * d / r);
                            }
                            x[m] = gs;
                        }
                    }
                }
                if constexpr (OP == P_FAR_LOSS) {
                    // the task's loss: summed over the team in a fixed order
                    // (xor butterfly in the warp, then the group's warps in
                    // order), one FP64 partial per task
                    const int span = AX == 0 ? T : gthreads_of(lcw, T);
                    for (int o = (span < 32 ? span : 32) >> 1; o > 0; o >>= 1) tl += __shfl_xor_sync(0xffffffffu, tl, o);
                    if (span > 32) {
                        const int g = threadIdx.x / span, gw = span >> 5;
                        sync();
                        if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = tl;
                        sync();
                        if ((threadIdx.x & (span - 1)) == 0) {
                            double sum = 0.0;
                            for (int i = 0; i < gw; ++i) sum += s_red[g * gw + i];
                            A.loss_task[task] = sum;
                        }
                    } else if (t == 0 && c == 0 && task < ntasks) {
                        A.loss_task[task] = tl;
                    }
                    fft<true>(x, N, T, t, reg, W, sync);
                    if (active) {
#pragma unroll
                        for (int m = 0; m < 32; ++m)
                            if (m < P) __stcg(A.gfield + fo + m * es, cscale(x[m], ff));
                    }
                }
            }
        }
    }
}

// pass along the axis of slice j (rows for even j, columns for odd j); AXO
// flips it (the far field's second transform)
template <int OP, int NY, int NZ>
__device__ __forceinline__ void pass_j(const SweepArgs& A, const Smem2& S, double* s_red, int j, bool first,
                                       bool prop, int axo = 0) {
    if (pass_axis(j) ^ axo) pass<1, OP, NY, NZ>(A, S, s_red, j, first, prop);
    else pass<0, OP, NY, NZ>(A, S, s_red, j, first, prop);
}

// grad[j] = sum_w gpart[j & 1][w] (fixed order over w), after pass j of the
// adjoint; the partials are double-buffered by slice parity because the
// blocks already run pass j-1 while others still sum slice j
__device__ void reduce_gpart_par(const SweepArgs& A, int j) {
    const size_t npx = (size_t)A.ny * A.nz;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    const size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const float2* gp = A.gpart + (size_t)(j & 1) * A.nw * npx;
    float2* dst = A.grad + (size_t)j * npx;
    if ((npx & 1) == 0 && ((uintptr_t)dst & 15) == 0) {
        const size_t n4 = npx / 2;
        const float4* g4 = reinterpret_cast<const float4*>(gp);
        float4* d4 = reinterpret_cast<float4*>(dst);
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

#define MS_KERNEL_PROLOGUE2                                       \
    extern __shared__ float4 smem_raw[];                          \
    __shared__ int s_ok;                                          \
    __shared__ double s_red[MS_WARPS];                            \
    (void)s_red;                                                  \
    if (*(volatile unsigned*)&A.ctrl[0]) return;                  \
    const Smem2 S = load_tables2(A, reinterpret_cast<float2*>(smem_raw)); \
    Grid grid{A.ctrl, gridDim.x, 0u, A.timeout_ns, &s_ok};

// L2 prefetch of slice j's transmission (every structure's when per_w)
__device__ __forceinline__ void prefetch_slice(const SweepArgs& A, const float2* base, int j) {
    const size_t npx = (size_t)A.ny * A.nz;
    for (int w = 0; w < (A.per_w ? A.nw : 1); ++w)
        prefetch_l2(base + (size_t)w * A.ns * npx * A.per_w + (size_t)j * npx, npx * sizeof(float2));
}

// Forward slice loop, slices [j_begin, j_end), one pass per slice.  The last
// slice of the range propagates (its own axis's factor) only if A.prop_last;
// with F_PROP_FULL the other axis's factor follows, so that the field is
// fully propagated.
template <int NY, int NZ>
__global__ void __launch_bounds__(MS_THREADS, MS_MIN_BLOCKS) k_slice_fwd(const SweepArgs A) {
    MS_KERNEL_PROLOGUE2
    for (int j = A.j_begin; j < A.j_end; ++j) {
        const bool last = j == A.j_end - 1;
        const bool prop = !last || A.prop_last;
        if (!last) prefetch_slice(A, A.tvol, j + 1);
        pass_j<P_FWD, NY, NZ>(A, S, s_red, j, j == A.j_begin, prop);
        if (!last || (A.flags & F_PROP_FULL)) {
            if (!grid.sync()) return;
        }
    }
    if (A.flags & F_PROP_FULL) pass_j<P_PROP, NY, NZ>(A, S, s_red, A.j_end - 1, false, true, 1);
    grid.finish();
}

// Adjoint slice loop, j from j_end-1 down to j_begin (a_j in the segment
// buffer).  With several wavefields on one volume, the per-wavefield gradient
// of slice j is summed after the barrier that follows its pass.
template <int NY, int NZ>
__global__ void __launch_bounds__(MS_THREADS, MS_MIN_BLOCKS) k_slice_adj(const SweepArgs A) {
    MS_KERNEL_PROLOGUE2
    const bool reduce = A.nw > 1 && !A.per_w;
    for (int j = A.j_end - 1; j >= A.j_begin; --j) {
        // the next slice's transmission into L2 (a_j is not prefetched: one
        // slice of it for every wavefield would evict the fields and partials)
        if (j - 1 >= A.j_begin) prefetch_slice(A, A.tvol, j - 1);
        pass_j<P_ADJ, NY, NZ>(A, S, s_red, j, false, j > 0);
        if (reduce || j > A.j_begin) {
            if (!grid.sync()) return;
        }
        if (reduce) reduce_gpart_par(A, j);
    }
    grid.finish();
}

// Last slice (j = ns-1): the pass along its axis (transmission, then the far
// field's transform along that axis, or the exit wave's propagation), then the
// other axis (far field, intensity, loss and seed with its transform back, or
// the exit wave).
template <int OP2>
__global__ void __launch_bounds__(MS_THREADS, 1) k_slice_last(const SweepArgs A) {
    MS_KERNEL_PROLOGUE2
    const int j = A.ns - 1;
    if constexpr (OP2 == P_EXIT) pass_j<P_LAST_EXIT, 0, 0>(A, S, s_red, j, j == A.j_begin, true);
    else pass_j<P_LAST_FAR, 0, 0>(A, S, s_red, j, j == A.j_begin, true);
    if (!grid.sync()) return;
    pass_j<OP2, 0, 0>(A, S, s_red, j, false, true, 1);
    if constexpr (OP2 == P_FAR_LOSS) {
        // per-wavefield loss: its tasks' partials in task order; then the
        // total over the wavefields in order (independent of the launch shape
        // apart from the column-group width, which sets the tasks)
        if (!grid.sync()) return;
        const int ax = pass_axis(j) ^ 1;
        const int ntasks = ax == 0 ? A.nz * A.nw : ((A.ny + (1 << A.lcw) - 1) >> A.lcw) * A.nw;
        const int nper = (ntasks + A.nw - 1) / A.nw;   // tasks of one wavefield
        for (int w = blockIdx.x; w < A.nw; w += gridDim.x) {   // uniform per block
            // thread i sums tasks i, i + blockDim, ... of wavefield w in order, then
            // a fixed tree over the threads (deterministic for the block size)
            double sum = 0.0;
            for (int i = threadIdx.x; i < nper; i += blockDim.x) {
                const int tk = w + i * A.nw;
                if (tk < ntasks) sum += __ldcg(A.loss_task + tk);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
            __syncthreads();
            if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = sum;
            __syncthreads();
            if (threadIdx.x == 0) {
                double tot = 0.0;
                for (int i = 0; i < MS_WARPS; ++i) tot += s_red[i];
                A.loss_wsum[w] = tot;
                if (A.per_w && A.lossw[w]) *A.lossw[w] = tot;
            }
        }
        if (!grid.sync()) return;
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            double sum = 0.0;
            for (int w = 0; w < A.nw; ++w) sum += __ldcg(A.loss_wsum + w);
            *A.loss_out = sum;
        }
    }
    grid.finish();
}

// Start of the adjoint for a given detector gradient: F^H along the axis other
// than that of slice ns-1 (the adjoint's first pass applies the rest).
template <int NY, int NZ>
__global__ void __launch_bounds__(MS_THREADS, 1) k_slice_seed(const SweepArgs A) {
    MS_KERNEL_PROLOGUE2
    pass_j<P_SEED, 0, 0>(A, S, s_red, A.ns - 1, false, true, 1);
    grid.finish();
}

}  // namespace
