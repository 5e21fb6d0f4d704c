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

// float -> bf16, round to nearest even (finite inputs)
__device__ __forceinline__ uint16_t to_bf16(float x) {
    const uint32_t a = __float_as_uint(x);
    return (uint16_t)((a + 0x7fffu + ((a >> 16) & 1u)) >> 16);
}

// C[m][n] = sum_k A(m, k) B(n, k) (+ bias[n]) (ReLU if relu), A(m,k) = A[m*sam + k*sak],
// B(n,k) = B[n*sbn + k*sbk]; operands rounded to BF16, FP32 accumulation.
// Split-K: blockIdx.z takes k in [z*kchunk, (z+1)*kchunk); with part != NULL the
// raw partial sums go to part[z][M][N] and k_splitk_reduce finishes them.
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
    // staging order: the unit-stride index runs across neighbouring threads
    const bool a_kfast = sak == 1, b_kfast = sbk == 1;
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.f;
    for (int k0 = kbeg; k0 < kend; k0 += kTK) {
        for (int e = threadIdx.x; e < kTM * kTK; e += blockDim.x) {
            const int r = a_kfast ? e / kTK : e % kTM, c = a_kfast ? e % kTK : e / kTM;
            const int m = m0 + r, k = k0 + c;
            sA[r][c] = to_bf16((m < M && k < kend) ? A[(long long)m * sam + (long long)k * sak] : 0.f);
        }
        for (int e = threadIdx.x; e < kTN * kTK; e += blockDim.x) {
            const int r = b_kfast ? e / kTK : e % kTN, c = b_kfast ? e % kTK : e / kTN;
            const int n = n0 + r, k = k0 + c;
            sB[r][c] = to_bf16((n < N && k < kend) ? Bm[(long long)n * sbn + (long long)k * sbk] : 0.f);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kTK; kk += 16) {
            uint32_t af[2][4], bf[4][2];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int r = wm + 16 * i + g;
                af[i][0] = *reinterpret_cast<const uint32_t*>(&sA[r][kk + 2 * tq]);
                af[i][1] = *reinterpret_cast<const uint32_t*>(&sA[r + 8][kk + 2 * tq]);
                af[i][2] = *reinterpret_cast<const uint32_t*>(&sA[r][kk + 2 * tq + 8]);
                af[i][3] = *reinterpret_cast<const uint32_t*>(&sA[r + 8][kk + 2 * tq + 8]);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int c = wn + 8 * j + g;
                bf[j][0] = *reinterpret_cast<const uint32_t*>(&sB[c][kk + 2 * tq]);
                bf[j][1] = *reinterpret_cast<const uint32_t*>(&sB[c][kk + 2 * tq + 8]);
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
__global__ void k_sigmoid_mse(const float* __restrict__ z, const float* __restrict__ t, float* __restrict__ y,
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
// s = counts / sum(I) (s = 1 when counts <= 0), amplitude a = sqrt(s I), plus
// 0.5 * noise when given (the standard deviation of a Poisson amplitude), and
// x = gain * log(1 + a^2), written centred (fftshift).  One block per image.
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
        float a = sqrtf(sc * Ii[src]);
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

constexpr int kTargetCtas = 304;  // two waves' worth of 64x64 tiles on 152 SMs
constexpr int kMaxSplits = 64;

// split-K factor: enough CTAs to cover the GPU, at least 4 k-steps per split
int gemm_splits(int M, int N, int K) {
    const long tiles = (long)((M + kTM - 1) / kTM) * ((N + kTN - 1) / kTN);
    const int ksteps = (K + kTK - 1) / kTK;
    long s = (kTargetCtas + tiles - 1) / tiles;
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
    k_sigmoid_mse<<<rows, 256, 0, (cudaStream_t)stream>>>(z, target, y, dz, row_loss, rows, cols, hi);
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
