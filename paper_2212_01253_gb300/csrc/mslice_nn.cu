// mslice_nn.cu -- kernels of the learned initialiser: a small network that
// maps a log-scaled detector image to a coarse delta volume, proposing the
// starting point of the gradient reconstruction (Sec. 4).  Dense layers run
// on the tensor cores (mma.sync m16n8k16: BF16 operands, FP32 accumulate);
// activations, biases, the loss and the optimiser state stay in FP32.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "mslice.h"

namespace {

constexpr int kTM = 64, kTN = 64, kTK = 32;  // block tile (rows of C, columns of C, k step)
constexpr int kPad = 8;                      // bf16 padding per smem row (16 bytes)

// two floats -> packed bf16x2 (lo in the low half), round to nearest even
__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
    uint32_t d;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
    return d;
}
__device__ __forceinline__ uint16_t to_bf16(float x) { return (uint16_t)(pack_bf16x2(x, 0.f) & 0xffffu); }

// How an operand tile (64 rows x 32 k) is read from global memory:
// K4: k is the unit-stride index (16-byte loads along k); R4: the row index is
// (16-byte loads along rows); SCALAR: anything else (one float per load).
enum : int { LD_SCALAR = 0, LD_K4 = 1, LD_R4 = 2 };

struct TileSrc {
    const float* p;
    long long srow, sk;
    int rows;      // valid rows (M or N)
    int mode;
};

__device__ __forceinline__ int tile_mode(const float* p, long long srow, long long sk) {
    const bool al = ((uintptr_t)p & 15) == 0;
    if (al && sk == 1 && (srow & 3) == 0) return LD_K4;
    if (al && srow == 1 && (sk & 3) == 0) return LD_R4;
    return LD_SCALAR;
}

// Each of the 128 threads holds 16 floats of the next tile.
struct TileRegs {
    float v[16];
};

__device__ __forceinline__ void tile_load(TileRegs& R, const TileSrc& S, int row0, int k0, int kend) {
    const int tid = threadIdx.x;
    if (S.mode == LD_K4) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int e = tid + 128 * q, r = e >> 3, c = (e & 7) * 4;
            const int row = row0 + r, k = k0 + c;
            if (row < S.rows && k + 3 < kend) {
                const float4 f = __ldg(reinterpret_cast<const float4*>(S.p + (long long)row * S.srow + k));
                R.v[4 * q] = f.x; R.v[4 * q + 1] = f.y; R.v[4 * q + 2] = f.z; R.v[4 * q + 3] = f.w;
            } else {
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    R.v[4 * q + i] = (row < S.rows && k + i < kend) ? __ldg(S.p + (long long)row * S.srow + k + i) : 0.f;
            }
        }
    } else if (S.mode == LD_R4) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int e = tid + 128 * q, c = e >> 4, r = (e & 15) * 4;
            const int row = row0 + r, k = k0 + c;
            if (row + 3 < S.rows && k < kend) {
                const float4 f = __ldg(reinterpret_cast<const float4*>(S.p + row + (long long)k * S.sk));
                R.v[4 * q] = f.x; R.v[4 * q + 1] = f.y; R.v[4 * q + 2] = f.z; R.v[4 * q + 3] = f.w;
            } else {
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    R.v[4 * q + i] = (row + i < S.rows && k < kend) ? __ldg(S.p + row + i + (long long)k * S.sk) : 0.f;
            }
        }
    } else {
        const bool kfast = S.sk == 1;
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const int e = tid + 128 * q;
            const int r = kfast ? e / kTK : e % kTM, c = kfast ? e % kTK : e / kTM;
            const int row = row0 + r, k = k0 + c;
            R.v[q] = (row < S.rows && k < kend) ? S.p[(long long)row * S.srow + (long long)k * S.sk] : 0.f;
        }
    }
}

__device__ __forceinline__ void tile_store(uint16_t (*sm)[kTK + kPad], const TileRegs& R, int mode, bool kfast) {
    const int tid = threadIdx.x;
    if (mode == LD_K4) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int e = tid + 128 * q, r = e >> 3, c = (e & 7) * 4;
            uint2 w;
            w.x = pack_bf16x2(R.v[4 * q], R.v[4 * q + 1]);
            w.y = pack_bf16x2(R.v[4 * q + 2], R.v[4 * q + 3]);
            *reinterpret_cast<uint2*>(&sm[r][c]) = w;
        }
    } else if (mode == LD_R4) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int e = tid + 128 * q, c = e >> 4, r = (e & 15) * 4;
#pragma unroll
            for (int i = 0; i < 4; ++i) sm[r + i][c] = to_bf16(R.v[4 * q + i]);
        }
    } else {
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const int e = tid + 128 * q;
            const int r = kfast ? e / kTK : e % kTM, c = kfast ? e % kTK : e / kTM;
            sm[r][c] = to_bf16(R.v[q]);
        }
    }
}

__device__ __forceinline__ void ldmatrix_x4(uint32_t (&d)[4], const void* smem_row) {
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(smem_row);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(d[0]), "=r"(d[1]), "=r"(d[2]), "=r"(d[3])
                 : "r"(a));
}

// C[m][n] = sum_k A(m, k) B(n, k) (+ bias[n]) (ReLU if relu), A(m,k) = A[m*sam + k*sak],
// B(n,k) = B[n*sbn + k*sbk]; operands rounded to BF16, FP32 accumulation
// (mma.sync m16n8k16).  The next k-tile is read into registers while the
// tensor cores work on the current one.  Split-K: blockIdx.z takes k in
// [z*kchunk, (z+1)*kchunk); with part != NULL the raw partial sums go to
// part[z][M][N] and k_splitk_reduce finishes them.
__global__ void __launch_bounds__(128) k_gemm(int M, int N, int K, const float* __restrict__ A, long long sam,
                                              long long sak, const float* __restrict__ Bm, long long sbn,
                                              long long sbk, float* __restrict__ C, long long ldc,
                                              const float* __restrict__ bias, int relu, float beta,
                                              float* __restrict__ part, int kchunk) {
    __shared__ __align__(16) uint16_t sA[kTM][kTK + kPad];
    __shared__ __align__(16) uint16_t sB[kTN][kTK + kPad];
    const int m0 = blockIdx.y * kTM, n0 = blockIdx.x * kTN;
    const int kbeg = blockIdx.z * kchunk;
    const int kend = min(K, kbeg + kchunk);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;  // 2x2 warps of 32x32
    const int g = lane >> 2, tq = lane & 3;
    const TileSrc SA{A, sam, sak, M, tile_mode(A, sam, sak)};
    const TileSrc SB{Bm, sbn, sbk, N, tile_mode(Bm, sbn, sbk)};
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.f;
    TileRegs ra, rb;
    tile_load(ra, SA, m0, kbeg, kend);
    tile_load(rb, SB, n0, kbeg, kend);
    tile_store(sA, ra, SA.mode, sak == 1);
    tile_store(sB, rb, SB.mode, sbk == 1);
    __syncthreads();
    // ldmatrix row addresses: A rows wm + 16 i + (lane % 16), k offset 8 (lane / 16);
    // B rows (n) wn + 8 (2 jj + lane / 16) + lane % 8, k offset 8 ((lane / 8) % 2)
    const int ar = lane & 15, ak = (lane >> 4) * 8;
    const int bn = ((lane >> 4) * 8) + (lane & 7), bk = ((lane >> 3) & 1) * 8;
    for (int k0 = kbeg; k0 < kend; k0 += kTK) {
        const bool more = k0 + kTK < kend;
        if (more) {
            tile_load(ra, SA, m0, k0 + kTK, kend);
            tile_load(rb, SB, n0, k0 + kTK, kend);
        }
#pragma unroll
        for (int kk = 0; kk < kTK; kk += 16) {
            uint32_t af[2][4], bf[4][2];
#pragma unroll
            for (int i = 0; i < 2; ++i) ldmatrix_x4(af[i], &sA[wm + 16 * i + ar][kk + ak]);
#pragma unroll
            for (int jj = 0; jj < 2; ++jj) {
                uint32_t t[4];
                ldmatrix_x4(t, &sB[wn + 16 * jj + bn][kk + bk]);
                bf[2 * jj][0] = t[0];
                bf[2 * jj][1] = t[1];
                bf[2 * jj + 1][0] = t[2];
                bf[2 * jj + 1][1] = t[3];
            }
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    asm volatile(
                        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
                        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
                        : "+f"(acc[i][j][0]), "+f"(acc[i][j][1]), "+f"(acc[i][j][2]), "+f"(acc[i][j][3])
                        : "r"(af[i][0]), "r"(af[i][1]), "r"(af[i][2]), "r"(af[i][3]), "r"(bf[j][0]),
                          "r"(bf[j][1]));
        }
        __syncthreads();
        if (more) {
            tile_store(sA, ra, SA.mode, sak == 1);
            tile_store(sB, rb, SB.mode, sbk == 1);
            __syncthreads();
        }
    }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int m = m0 + wm + 16 * i + g + (r >= 2 ? 8 : 0);
                const int n = n0 + wn + 8 * j + 2 * tq + (r & 1);
                if (m < M && n < N) {
                    float v = acc[i][j][r];
                    if (part) {
                        part[((size_t)blockIdx.z * M + m) * N + n] = v;
                        continue;
                    }
                    if (bias) v += bias[n];
                    if (relu) v = fmaxf(v, 0.f);
                    float* o = C + (long long)m * ldc + n;
                    *o = beta != 0.f ? fmaf(beta, *o, v) : v;
                }
            }
}

// sum of the split-K partials in split order, then bias, ReLU and beta
__global__ void k_splitk_reduce(const float* __restrict__ part, int splits, int M, int N, float* __restrict__ C,
                                long long ldc, const float* __restrict__ bias, int relu, float beta) {
    const size_t n_out = (size_t)M * N;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_out; i += (size_t)gridDim.x * blockDim.x) {
        const int m = (int)(i / N), n = (int)(i % N);
        float v = 0.f;
        for (int z = 0; z < splits; ++z) v += part[(size_t)z * n_out + i];
        if (bias) v += bias[n];
        if (relu) v = fmaxf(v, 0.f);
        float* o = C + (long long)m * ldc + n;
        *o = beta != 0.f ? fmaf(beta, *o, v) : v;
    }
}

// patch permutation: NHWC [B][H][W][C] <-> [B][H/p][W/p][p][p][C]
__global__ void k_space_to_depth(const float* __restrict__ in, float* __restrict__ out, int B, int H, int W, int C,
                                 int p, int inverse) {
    const size_t n = (size_t)B * H * W * C;
    const int hp = H / p, wp = W / p;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        size_t t = i;
        const int c = (int)(t % C); t /= C;
        const int dj = (int)(t % p); t /= p;
        const int di = (int)(t % p); t /= p;
        const int j = (int)(t % wp); t /= wp;
        const int ii = (int)(t % hp);
        const size_t b = t / hp;
        const size_t src = ((b * H + (size_t)ii * p + di) * W + (size_t)j * p + dj) * C + c;
        if (inverse)
            out[src] = in[i];
        else
            out[i] = in[src];
    }
}

// dz = dy * (y > 0) (ReLU backward, y the ReLU output)
__global__ void k_relu_back(const float* __restrict__ y, const float* __restrict__ dy, float* __restrict__ dz,
                            size_t n) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        dz[i] = y[i] > 0.f ? dy[i] : 0.f;
}

// y = hi * sigmoid(z); loss partial = sum (y - t)^2 / n_out per row; dz = dL/dz
__global__ void __launch_bounds__(1024) k_sigmoid_mse(const float* __restrict__ z, const float* __restrict__ t, float* __restrict__ y,
                              float* __restrict__ dz, double* __restrict__ row_loss, int rows, int cols, float hi) {
    const int r = blockIdx.x;
    if (r >= rows) return;
    double part = 0.0;
    const float inv = 1.f / (float)(rows * cols);
    for (int c = threadIdx.x; c < cols; c += blockDim.x) {
        const size_t i = (size_t)r * cols + c;
        const float s = 1.f / (1.f + expf(-z[i]));
        const float yi = hi * s;
        y[i] = yi;
        if (t) {
            const float d = yi - t[i];
            part += (double)d * (double)d;
            if (dz) dz[i] = 2.f * d * inv * hi * s * (1.f - s);
        }
    }
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
    __syncthreads();
    if (threadIdx.x == 0 && row_loss) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) s += red[w];
        row_loss[r] = s / (double)(rows * cols);
    }
}

// Network input from detector images [nimg][nz][ny] (natural FFT order):
// s = counts / sum(I) (s = 1 when counts == 0), amplitude a = sqrt(s I) (the
// input itself when counts < 0), plus 0.5 * noise when given (the standard
// deviation of a Poisson amplitude), and x = gain * log(1 + a^2), written
// centred (fftshift).  One block per image.
__global__ void __launch_bounds__(1024) k_detector_features(const float* __restrict__ I,
                                                            const float* __restrict__ noise, float* __restrict__ x,
                                                            int nz, int ny, float counts, float gain) {
    const size_t npx = (size_t)nz * ny;
    const float* Ii = I + blockIdx.x * npx;
    __shared__ double red[32];
    __shared__ float s_scale;
    if (counts > 0.f) {
        double part = 0.0;
        for (size_t i = threadIdx.x; i < npx; i += blockDim.x) part += (double)Ii[i];
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) t += red[w];
            s_scale = t > 0.0 ? (float)((double)counts / t) : 0.f;
        }
        __syncthreads();
    } else if (threadIdx.x == 0) {
        s_scale = 1.f;
    }
    __syncthreads();
    const float sc = s_scale;
    for (size_t o = threadIdx.x; o < npx; o += blockDim.x) {
        const int zz = (int)(o / ny), yy = (int)(o % ny);
        const size_t src = (size_t)((zz + nz / 2) % nz) * ny + (size_t)((yy + ny / 2) % ny);
        float a = counts < 0.f ? Ii[src] : sqrtf(sc * Ii[src]);
        if (noise) a = fmaxf(fmaf(0.5f, noise[blockIdx.x * npx + src], a), 0.f);
        x[blockIdx.x * npx + o] = gain * log1pf(a * a);
    }
}

// out[s][i0][i1][i2] = value inside any box of sample s, else 0; boxes
// [s][b] = (lo0, hi0, lo1, hi1, lo2, hi2), half-open
__global__ void k_rasterize_boxes(const int* __restrict__ boxes, int nb_per, int nsamp, int d0, int d1, int d2,
                                  float value, float* __restrict__ out) {
    const size_t per = (size_t)d0 * d1 * d2, n = per * nsamp;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const size_t smp = i / per, r = i % per;
        const int i2 = (int)(r % d2), i1 = (int)((r / d2) % d1), i0 = (int)(r / ((size_t)d1 * d2));
        const int* bx = boxes + smp * nb_per * 6;
        bool in = false;
        for (int b = 0; b < nb_per && !in; ++b, bx += 6)
            in = i0 >= bx[0] && i0 < bx[1] && i1 >= bx[2] && i1 < bx[3] && i2 >= bx[4] && i2 < bx[5];
        out[i] = in ? value : 0.f;
    }
}

unsigned nb(size_t n) {
    size_t b = (n + 255) / 256;
    return (unsigned)(b > 4096 ? 4096 : (b ? b : 1));
}

// two waves' worth of 64x64 tiles: twice the SM count of the current device
int target_ctas() {
    static int cache[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 304;
    if (cache[dev] <= 0 && cudaDeviceGetAttribute(&cache[dev], cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 304;
    return cache[dev] > 0 ? 2 * cache[dev] : 304;
}
constexpr int kMaxSplits = 64;

// split-K factor: enough CTAs to cover the GPU, at least 4 k-steps per split
int gemm_splits(int M, int N, int K) {
    const long tiles = (long)((M + kTM - 1) / kTM) * ((N + kTN - 1) / kTN);
    const int ksteps = (K + kTK - 1) / kTK;
    long s = (target_ctas() + tiles - 1) / tiles;
    s = s < ksteps / 4 ? s : ksteps / 4;
    s = s < kMaxSplits ? s : kMaxSplits;
    return s < 1 ? 1 : (int)s;
}

}  // namespace

extern "C" {

size_t mslice_nn_gemm_workspace(int M, int N, int K) {
    if (M < 1 || N < 1 || K < 1) return 0;
    const int s = gemm_splits(M, N, K);
    return s > 1 ? (size_t)s * M * N * sizeof(float) : 0;
}

int mslice_nn_gemm(int M, int N, int K, const float* A, long long sam, long long sak, const float* B, long long sbn,
                   long long sbk, float* C, long long ldc, const float* bias, int relu, float beta, void* ws,
                   size_t ws_bytes, void* stream) {
    if (M < 1 || N < 1 || K < 1 || !A || !B || !C || ldc < N) return MSLICE_EINVAL;
    const int splits = gemm_splits(M, N, K);
    dim3 grid((N + kTN - 1) / kTN, (M + kTM - 1) / kTM, splits);
    if (grid.y > 65535) return MSLICE_EUNSUPPORTED;
    cudaStream_t st = (cudaStream_t)stream;
    if (splits == 1) {
        k_gemm<<<grid, 128, 0, st>>>(M, N, K, A, sam, sak, B, sbn, sbk, C, ldc, bias, relu, beta, nullptr, K);
        return cudaGetLastError() == cudaSuccess ? MSLICE_OK : MSLICE_ELAUNCH;
    }
    if (!ws || ws_bytes < mslice_nn_gemm_workspace(M, N, K) || ((uintptr_t)ws & 15)) return MSLICE_EWORKSPACE;
    const int ksteps = (K + kTK - 1) / kTK;
    const int kchunk = ((ksteps + splits - 1) / splits) * kTK;
    grid.z = (K + kchunk - 1) / kchunk;  // splits that hold at least one k-step
    k_gemm<<<grid, 128, 0, st>>>(M, N, K, A, sam, sak, B, sbn, sbk, C, ldc, nullptr, 0, 0.f, (float*)ws, kchunk);
    k_splitk_reduce<<<nb((size_t)M * N), 256, 0, st>>>((const float*)ws, (int)grid.z, M, N, C, ldc, bias, relu,
                                                        beta);
    return cudaGetLastError() == cudaSuccess ? MSLICE_OK : MSLICE_ELAUNCH;
}

int mslice_nn_space_to_depth(const float* in, float* out, int B, int H, int W, int C, int p, int inverse,
                             void* stream) {
    if (!in || !out || B < 1 || H < 1 || W < 1 || C < 1 || p < 1 || H % p || W % p) return MSLICE_EINVAL;
    k_space_to_depth<<<nb((size_t)B * H * W * C), 256, 0, (cudaStream_t)stream>>>(in, out, B, H, W, C, p,
                                                                                   inverse);
    return cudaGetLastError() == cudaSuccess ? MSLICE_OK : MSLICE_ELAUNCH;
}

int mslice_nn_relu_backward(const float* y, const float* dy, float* dz, size_t n, void* stream) {
    if (!y || !dy || !dz) return MSLICE_EINVAL;
    if (!n) return MSLICE_OK;
    k_relu_back<<<nb(n), 256, 0, (cudaStream_t)stream>>>(y, dy, dz, n);
    return cudaGetLastError() == cudaSuccess ? MSLICE_OK : MSLICE_ELAUNCH;
}

int mslice_nn_sigmoid_mse(const float* z, const float* target, float* y, float* dz, double* row_loss, int rows,
                          int cols, float hi, void* stream) {
    if (!z || !y || rows < 1 || cols < 1) return MSLICE_EINVAL;
    k_sigmoid_mse<<<rows, 1024, 0, (cudaStream_t)stream>>>(z, target, y, dz, row_loss, rows, cols, hi);
    return cudaGetLastError() == cudaSuccess ? MSLICE_OK : MSLICE_ELAUNCH;
}

int mslice_nn_detector_features(const float* intensity, const float* noise, float* x, int nimg, int nz, int ny,
                                float counts, float gain, void* stream) {
    if (!intensity || !x || nimg < 1 || nz < 1 || ny < 1) return MSLICE_EINVAL;
    k_detector_features<<<nimg, 1024, 0, (cudaStream_t)stream>>>(intensity, noise, x, nz, ny, counts, gain);
    return cudaGetLastError() == cudaSuccess ? MSLICE_OK : MSLICE_ELAUNCH;
}

int mslice_nn_rasterize_boxes(const int* boxes, int boxes_per_sample, int nsamples, int d0, int d1, int d2,
                              float value, float* out, void* stream) {
    if (!out || nsamples < 1 || d0 < 1 || d1 < 1 || d2 < 1 || boxes_per_sample < 0 ||
        (boxes_per_sample > 0 && !boxes))
        return MSLICE_EINVAL;
    k_rasterize_boxes<<<nb((size_t)nsamples * d0 * d1 * d2), 256, 0, (cudaStream_t)stream>>>(
        boxes, boxes_per_sample, nsamples, d0, d1, d2, value, out);
    return cudaGetLastError() == cudaSuccess ? MSLICE_OK : MSLICE_ELAUNCH;
}

}  // extern "C"
