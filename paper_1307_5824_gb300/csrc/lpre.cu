// lpre.cu -- the learned Fourier-domain CG preconditioner (an addition to the paper,
// whose CG, Section 3.3, is unpreconditioned).
//
// Bins: a frequency vector q in N-grid units falls in shell s = min(63, floor(64|q|/(N/2)))
// and cone c = min(15, floor(16 |<q/|q|, a>|)), a the principal axis of the viewing
// directions; bin = 16 s + c.  The network input is the h^2-weighted density of the
// slice samples per bin; its output is a per-bin log multiplier t_b = log(p_b Ker(0))
// of the preconditioner diagonal d(q) = exp(t_b) / Ker(0).  The training target is the
// least-squares p_b = sum (kappa + lam) / sum (kappa + lam)^2 over the bin, kappa the
// spectrum of T. Chan's circulant.  MLP: 1024 -> 256 -> 256 -> 1024, ReLU, FP32
// training with Adam, BF16-weight inference, all in the kernels below.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>

#include "firm_internal.h"

namespace firm {

constexpr int kShells = 64, kCones = 16, kBins = kShells * kCones;

__device__ __forceinline__ int freq_bin_r(float q1, float q2, float q3, float r, float halfN, float a1, float a2,
                                          float a3) {
    const int s = min(kShells - 1, (int)floorf((float)kShells * r / halfN));
    const float c = r > 0.0f ? fabsf(q1 * a1 + q2 * a2 + q3 * a3) / r : 0.0f;
    const int cb = min(kCones - 1, (int)floorf((float)kCones * c));
    return kCones * s + cb;
}

__device__ __forceinline__ int freq_bin(float q1, float q2, float q3, float halfN, float a1, float a2, float a3) {
    return freq_bin_r(q1, q2, q3, sqrtf(q1 * q1 + q2 * q2 + q3 * q3), halfN, a1, a2, a3);
}

// second moment of the viewing directions d = third row of R_m (sum of d d^T)
__global__ void __launch_bounds__(1024) k_view_moment(const double* __restrict__ R, int M, double* __restrict__ out9) {
    __shared__ double s[32][9];
    double acc[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int m = threadIdx.x; m < M; m += blockDim.x) {
        const double* d = R + 9 * (size_t)m + 6;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) acc[3 * i + j] += d[i] * d[j];
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int k = 0; k < 9; ++k) {
        double v = acc[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) s[wid][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < 9) {
        double v = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += s[w][threadIdx.x];
        out9[threadIdx.x] = v;
    }
}

// h^2-weighted histogram of the half-disc samples (the mirrored half falls in the same
// bin).  A thread owns one image and walks a range of samples t (blockIdx.y picks the
// range): |xi| = |k| fixes the shell and the cone only needs |k1 <u, a> + k2 <v, a>| /
// |k| (u, v the slice axes, a the viewing axis), so the block first tabulates, per t of
// its range, the shell and k / |k|, and every point is then two FMAs, a cone index and
// one shared-memory atomic into the block's histogram.
constexpr int kFeatThreads = 256;
constexpr int kFeatT = 1024;          // samples t per block (the table: 12 B each)
__global__ void __launch_bounds__(kFeatThreads) k_pc_features(const ImgGeom* __restrict__ geom,
                                                              const int32_t* __restrict__ htab,
                                                              const int32_t* __restrict__ gid,
                                                              const float* __restrict__ h2, int M, int nH, int n_ctf,
                                                              float halfN, const float* __restrict__ axis,
                                                              float* __restrict__ hist) {
    __shared__ float s_h[kBins];
    __shared__ float2 s_k[kFeatT];        // k / |k| (0 at k = 0)
    __shared__ int s_s[kFeatT];           // shell of t
    const float a1 = axis[0], a2 = axis[1], a3 = axis[2];
    for (int i = threadIdx.x; i < kBins; i += blockDim.x) s_h[i] = 0.0f;
    const int t0 = blockIdx.y * kFeatT, t1 = min(nH, t0 + kFeatT);
    for (int t = t0 + threadIdx.x; t < t1; t += blockDim.x) {
        const int kk = __ldg(&htab[t]);
        const float k1 = (float)(int16_t)(kk & 0xffff), k2 = (float)(kk >> 16);
        const float rk = sqrtf(k1 * k1 + k2 * k2);     // |xi| in grid units, exactly |k|
        const float inv_r = rk > 0.0f ? 1.0f / rk : 0.0f;
        s_k[t - t0] = make_float2(k1 * inv_r, k2 * inv_r);
        s_s[t - t0] = min(kShells - 1, (int)floorf((float)kShells * rk / halfN));
    }
    __syncthreads();
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m < M) {
        const ImgGeom g = geom[m];
        const float ua = g.uh[0] * a1 + g.uh[1] * a2 + g.uh[2] * a3;
        const float va = g.vh[0] * a1 + g.vh[1] * a2 + g.vh[2] * a3;
        const float* h2g = h2 + (size_t)min(max(gid[m], 0), n_ctf - 1) * nH;
        for (int t = t0; t < t1; ++t) {
            const float2 kr = s_k[t - t0];
            const float c = fabsf(fmaf(kr.x, ua, kr.y * va));
            const int cb = min(kCones - 1, (int)((float)kCones * c));
            atomicAdd(&s_h[kCones * s_s[t - t0] + cb], __ldg(&h2g[t]));
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kBins; i += blockDim.x)
        if (s_h[i] != 0.0f) atomicAdd(&hist[i], s_h[i]);
}

// per-bin sums of (kappa + lam) and (kappa + lam)^2 over the half spectrum of the
// circulant (weight 2 for the interior k1 columns whose mirror is not stored)
// lam: device lam_eff (lam[0]); nullptr counts frequencies (u == nullptr too)
__global__ void __launch_bounds__(256) k_pc_target_sums(const float2* __restrict__ u, int N, const float* __restrict__ lam_p,
                                                        const float* __restrict__ axis, double* __restrict__ s1,
                                                        double* __restrict__ s2) {
    const float a1 = axis[0], a2 = axis[1], a3 = axis[2];
    const float lam = lam_p ? lam_p[0] : 0.0f;
    __shared__ float sh1[kBins], sh2[kBins];
    for (int i = threadIdx.x; i < kBins; i += blockDim.x) { sh1[i] = 0.0f; sh2[i] = 0.0f; }
    __syncthreads();
    const int H = N / 2 + 1;
    const long long total = (long long)N * N * H;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const int k1 = (int)(i % H), k2 = (int)((i / H) % N), k3 = (int)(i / ((long long)H * N));
        const float q1 = (float)k1, q2 = (float)(k2 < N / 2 ? k2 : k2 - N), q3 = (float)(k3 < N / 2 ? k3 : k3 - N);
        const float w = (k1 == 0 || k1 == N / 2) ? 1.0f : 2.0f;
        const float kap = u ? fmaxf(u[i].x, 0.0f) + lam : 1.0f;     // u == nullptr: count frequencies
        const int b = freq_bin(q1, q2, q3, 0.5f * N, a1, a2, a3);
        atomicAdd(&sh1[b], w * kap);
        atomicAdd(&sh2[b], w * kap * kap);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kBins; i += blockDim.x) {
        if (sh1[i] != 0.0f) atomicAdd(&s1[i], (double)sh1[i]);
        if (sh2[i] != 0.0f) atomicAdd(&s2[i], (double)sh2[i]);
    }
}

// d(q) = exp(table[bin(q)]) / (Ker(0) N^3) on the half spectrum
// d(q) = exp(table[bin(q)]) / (Ker(0) N^3), Ker(0) = lam[1] on the device (1 if not positive)
__global__ void __launch_bounds__(256) k_pc_from_table(const float* __restrict__ table, int N, const float* __restrict__ lam,
                                                       const float* __restrict__ axis, float* __restrict__ d) {
    const float a1 = axis[0], a2 = axis[1], a3 = axis[2];
    const float k0 = lam[1] > 0.0f ? lam[1] : 1.0f;
    const float scale = 1.0f / (k0 * (float)N * (float)N * (float)N);
    const int H = N / 2 + 1;
    const long long total = (long long)N * N * H;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const int k1 = (int)(i % H), k2 = (int)((i / H) % N), k3 = (int)(i / ((long long)H * N));
        const float q1 = (float)k1, q2 = (float)(k2 < N / 2 ? k2 : k2 - N), q3 = (float)(k3 < N / 2 ? k3 : k3 - N);
        d[i] = expf(__ldg(&table[freq_bin(q1, q2, q3, 0.5f * N, a1, a2, a3)])) * scale;
    }
}

// ---------------------------------------------------------------------------
// Principal axis: Jacobi eigenvalue iterations on the symmetric 3x3 moment, on the
// device (one thread), so that firm_kernel needs no host round trip.
// ---------------------------------------------------------------------------
__device__ static void principal_axis(const double* S, float* a) {
    double A[3][3], V[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) A[i][j] = 0.5 * (S[3 * i + j] + S[3 * j + i]);
    for (int sweep = 0; sweep < 50; ++sweep) {
        double off = fabs(A[0][1]) + fabs(A[0][2]) + fabs(A[1][2]);
        if (off < 1e-15 * (fabs(A[0][0]) + fabs(A[1][1]) + fabs(A[2][2]) + 1e-300)) break;
        for (int p = 0; p < 2; ++p)
            for (int q = p + 1; q < 3; ++q) {
                if (A[p][q] == 0.0) continue;
                const double th = 0.5 * atan2(2 * A[p][q], A[q][q] - A[p][p]);
                const double c = cos(th), s = sin(th);
                for (int k = 0; k < 3; ++k) {       // A <- J^T A J
                    const double akp = A[k][p], akq = A[k][q];
                    A[k][p] = c * akp - s * akq;
                    A[k][q] = s * akp + c * akq;
                }
                for (int k = 0; k < 3; ++k) {
                    const double apk = A[p][k], aqk = A[q][k];
                    A[p][k] = c * apk - s * aqk;
                    A[q][k] = s * apk + c * aqk;
                }
                for (int k = 0; k < 3; ++k) {
                    const double vkp = V[k][p], vkq = V[k][q];
                    V[k][p] = c * vkp - s * vkq;
                    V[k][q] = s * vkp + c * vkq;
                }
            }
    }
    int best = 0;
    for (int i = 1; i < 3; ++i)
        if (A[i][i] > A[best][best]) best = i;
    const double n = sqrt(V[0][best] * V[0][best] + V[1][best] * V[1][best] + V[2][best] * V[2][best]);
    for (int i = 0; i < 3; ++i) a[i] = (float)(V[i][best] / (n > 0 ? n : 1.0));
}

__global__ void k_view_axis(const double* __restrict__ S, float* __restrict__ axis) {
    principal_axis(S, axis);
}

cudaError_t launch_view_axis(Plan& P, const double* R, int M) {
    double* tmp = P.ws.red_b;      // 9 doubles of scratch
    k_view_moment<<<1, 1024, 0, P.stream>>>(R, M, tmp);
    k_view_axis<<<1, 1, 0, P.stream>>>(tmp, P.ws.axis);
    P.launches += 2;
    return cudaGetLastError();
}

cudaError_t launch_pc_features(Plan& P, int M, float* hist) {
    cudaError_t e = cudaMemsetAsync(hist, 0, sizeof(float) * kBins, P.stream);
    if (e != cudaSuccess || M <= 0) return e;
    const dim3 grid((M + kFeatThreads - 1) / kFeatThreads, (P.nH + kFeatT - 1) / kFeatT);
    k_pc_features<<<grid, kFeatThreads, 0, P.stream>>>(P.ws.geom, P.ws.htab, P.cur_gid, P.ws.h2, M, P.nH, P.n_ctf,
                                                       0.5f * P.N, P.ws.axis, hist);
    P.launches += 1;
    return cudaGetLastError();
}

// Features f_b = h_b / sum_b h_b (the h^2-weighted share of the samples in every bin)
// and, with x != nullptr, the network input x_b = log(1024 f_b + 1e-3).  One block of
// kBins threads; the sum is a fixed-order tree, so the result is deterministic.
__global__ void __launch_bounds__(kBins) k_pc_normalize(float* __restrict__ hist, float* __restrict__ x) {
    __shared__ double s_w[kBins / 32];
    const int i = threadIdx.x, lane = i & 31, wid = i >> 5;
    const float h = hist[i];
    double v = h;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) s_w[wid] = v;
    __syncthreads();
    if (wid == 0) {
        v = s_w[lane];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) s_w[0] = v;
    }
    __syncthreads();
    const double tot = s_w[0];
    const float f = tot > 0.0 ? (float)((double)h / tot) : 0.0f;
    hist[i] = f;
    if (x) x[i] = logf((float)kBins * f + 1e-3f);
}

cudaError_t launch_pc_normalize(Plan& P, float* hist, float* x) {
    k_pc_normalize<<<1, kBins, 0, P.stream>>>(hist, x);
    P.launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_pc_target_sums(Plan& P, double* s1, double* s2) {
    cudaError_t e = cudaMemsetAsync(s1, 0, sizeof(double) * kBins, P.stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s2, 0, sizeof(double) * kBins, P.stream);
    if (e != cudaSuccess) return e;
    k_pc_target_sums<<<P.num_sms * 2, 256, 0, P.stream>>>(P.ws.t1, P.N, P.ws.lam, P.ws.axis, s1, s2);
    P.launches += 1;
    return cudaGetLastError();
}

// Frequencies of the N^3 grid per bin (s1 = s2 = count), for bin volumes.
cudaError_t launch_pc_bin_counts(Plan& P, double* s1, double* s2) {
    cudaError_t e = cudaMemsetAsync(s1, 0, kBins * sizeof(double), P.stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s2, 0, kBins * sizeof(double), P.stream);
    if (e != cudaSuccess) return e;
    k_pc_target_sums<<<P.num_sms * 2, 256, 0, P.stream>>>(nullptr, P.N, nullptr, P.ws.axis, s1, s2);
    P.launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_pc_from_table(Plan& P, const float* table) {
    k_pc_from_table<<<P.num_sms * 4, 256, 0, P.stream>>>(table, P.N, P.ws.lam, P.ws.axis, P.ws.pc_diag);
    P.launches += 1;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// MLP 1024 -> 256 -> 256 -> 1024 (ReLU).  Row-major activations (batch x width),
// weights W (out x in).  Params: W1 b1 W2 b2 W3 b3 contiguous.
// ---------------------------------------------------------------------------
constexpr int kW0 = kBins, kW1 = 256, kW2 = 256, kW3 = kBins;
constexpr size_t kOffW1 = 0, kOffB1 = kOffW1 + (size_t)kW1 * kW0, kOffW2 = kOffB1 + kW1,
                 kOffB2 = kOffW2 + (size_t)kW2 * kW1, kOffW3 = kOffB2 + kW2, kOffB3 = kOffW3 + (size_t)kW3 * kW2,
                 kParams = kOffB3 + kW3;

// C[M x N] = op(A) op(B) (+ bias[N]) (ReLU), op by leading-dimension flags.
//   TA = false: A is M x K row-major; true: A is K x M row-major (use A^T).
//   TB = false: B is K x N row-major; true: B is N x K row-major (use B^T).
// On the tensor cores (mma.sync): a 64 x 64 output tile per block of
// four warps, each warp 32 x 32 (2 x 4 tiles of 16 x 8), K in steps of 16 staged in
// shared memory in a fixed [row][k] layout whatever the operands' transposition.
//   BF16 weights (inference): both operands as bf16 (activations rounded), m16n8k16,
//     FP32 accumulation.
//   FP32 (training and the FP32 forward pass): three TF32 products per step with each
//     operand split as x = hi + lo, hi = tf32(x), lo = tf32(x - hi) (hi*hi + hi*lo +
//     lo*hi, the small terms first), m16n8k8, FP32 accumulation: FP32-level accuracy.
constexpr int kTcTile = 64, kTcK = 16, kTcPad = 4;

__device__ __forceinline__ uint32_t bf16x2(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}
__device__ __forceinline__ uint32_t tf32_of(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ void mma_bf16(float* c, const uint32_t* a, const uint32_t* b) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}
__device__ __forceinline__ void mma_tf32(float* c, const uint32_t* a, const uint32_t* b) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

template <bool TA, bool TB, class WT>
__global__ void __launch_bounds__(128) k_gemm_tc(const float* __restrict__ A, const WT* __restrict__ B,
                                                 float* __restrict__ C, int M, int N, int K,
                                                 const float* __restrict__ bias, int relu, int accumulate) {
    constexpr bool kBf16 = sizeof(WT) == 2;
    __shared__ float As[kTcTile][kTcK + kTcPad];     // [m][k]
    __shared__ float Bs[kTcTile][kTcK + kTcPad];     // [n][k]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, t = lane & 3;
    const int m0 = blockIdx.y * kTcTile, n0 = blockIdx.x * kTcTile;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    float acc[2][4][4] = {};
    for (int k0 = 0; k0 < K; k0 += kTcK) {
        for (int i = threadIdx.x; i < kTcTile * kTcK; i += blockDim.x) {
            // A: consecutive threads along the operand's contiguous axis
            const int mm = TA ? i % kTcTile : i / kTcK, kk = TA ? i / kTcTile : i % kTcK;
            const int gm = m0 + mm, gk = k0 + kk;
            float va = 0.0f;
            if (gm < M && gk < K) va = TA ? A[(size_t)gk * M + gm] : A[(size_t)gm * K + gk];
            As[mm][kk] = va;
            const int nn = TB ? i / kTcK : i % kTcTile, kb = TB ? i % kTcK : i / kTcTile;
            const int gn = n0 + nn, gkb = k0 + kb;
            float vb = 0.0f;
            if (gn < N && gkb < K) {
                if constexpr (kBf16) vb = __bfloat162float(TB ? B[(size_t)gn * K + gkb] : B[(size_t)gkb * N + gn]);
                else vb = TB ? B[(size_t)gn * K + gkb] : B[(size_t)gkb * N + gn];
            }
            Bs[nn][kb] = vb;
        }
        __syncthreads();
        if constexpr (kBf16) {
            uint32_t af[2][4], bfr[4][2];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int r = wm + 16 * i + g;
                af[i][0] = bf16x2(As[r][2 * t], As[r][2 * t + 1]);
                af[i][1] = bf16x2(As[r + 8][2 * t], As[r + 8][2 * t + 1]);
                af[i][2] = bf16x2(As[r][2 * t + 8], As[r][2 * t + 9]);
                af[i][3] = bf16x2(As[r + 8][2 * t + 8], As[r + 8][2 * t + 9]);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int n = wn + 8 * j + g;
                bfr[j][0] = bf16x2(Bs[n][2 * t], Bs[n][2 * t + 1]);
                bfr[j][1] = bf16x2(Bs[n][2 * t + 8], Bs[n][2 * t + 9]);
            }
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], af[i], bfr[j]);
        } else {
#pragma unroll
            for (int ks = 0; ks < kTcK; ks += 8) {
                uint32_t ah[2][4], al[2][4], bh[4][2], bl[4][2];
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    const int r = wm + 16 * i + g;
                    const float v[4] = {As[r][ks + t], As[r + 8][ks + t], As[r][ks + t + 4], As[r + 8][ks + t + 4]};
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        ah[i][q] = tf32_of(v[q]);
                        al[i][q] = tf32_of(v[q] - __uint_as_float(ah[i][q]));
                    }
                }
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int n = wn + 8 * j + g;
                    const float v[2] = {Bs[n][ks + t], Bs[n][ks + t + 4]};
#pragma unroll
                    for (int q = 0; q < 2; ++q) {
                        bh[j][q] = tf32_of(v[q]);
                        bl[j][q] = tf32_of(v[q] - __uint_as_float(bh[j][q]));
                    }
                }
#pragma unroll
                for (int i = 0; i < 2; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        mma_tf32(acc[i][j], al[i], bh[j]);
                        mma_tf32(acc[i][j], ah[i], bl[j]);
                        mma_tf32(acc[i][j], ah[i], bh[j]);
                    }
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int gm = m0 + wm + 16 * i + g + (q >= 2 ? 8 : 0);
                const int gn = n0 + wn + 8 * j + 2 * t + (q & 1);
                if (gm >= M || gn >= N) continue;
                float v = acc[i][j][q];
                if (bias) v += bias[gn];
                if (relu) v = fmaxf(v, 0.0f);
                float* c = &C[(size_t)gm * N + gn];
                *c = accumulate ? *c + v : v;
            }
}

template <bool TA, bool TB, class WT>
static void gemm(cudaStream_t s, const float* A, const WT* B, float* C, int M, int N, int K, const float* bias, bool relu,
                 bool acc = false) {
    const dim3 grid((N + kTcTile - 1) / kTcTile, (M + kTcTile - 1) / kTcTile);
    k_gemm_tc<TA, TB, WT><<<grid, 128, 0, s>>>(A, B, C, M, N, K, bias, relu ? 1 : 0, acc ? 1 : 0);
}

// gy = 2 (y - t) / n, loss partials
__global__ void k_mse_grad(const float* __restrict__ y, const float* __restrict__ t, float* __restrict__ gy, size_t n,
                           double* __restrict__ loss) {
    __shared__ double s[256];
    double acc = 0.0;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float d = y[i] - t[i];
        gy[i] = 2.0f * d / (float)n;
        acc += (double)d * d;
    }
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int k = 128; k > 0; k >>= 1) {
        if ((int)threadIdx.x < k) s[threadIdx.x] += s[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(loss, s[0] / (double)n);
}

// g *= (z > 0) where the ReLU output a = max(z, 0) is stored (a > 0 <=> z > 0)
__global__ void k_relu_mask(float* __restrict__ g, const float* __restrict__ a, size_t n) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        if (!(a[i] > 0.0f)) g[i] = 0.0f;
}

// column sums: gb[j] = sum_i g[i, j]
__global__ void k_colsum(const float* __restrict__ g, float* __restrict__ gb, int rows, int cols) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= cols) return;
    float s = 0.0f;
    for (int i = 0; i < rows; ++i) s += g[(size_t)i * cols + j];
    gb[j] = s;
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       size_t n, float lr, float b1, float b2, float eps, float c1, float c2) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

__global__ void k_to_bf16(const float* __restrict__ x, __nv_bfloat16* __restrict__ y, size_t n) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        y[i] = __float2bfloat16_rn(x[i]);
}

// work layout: a1 (batch x 256), a2 (batch x 256), y (batch x 1024), g1, g2 (batch x 256), gy (batch x 1024)
static size_t mlp_work_floats(int batch) { return (size_t)batch * (2 * 256 + 1024 + 2 * 256 + 1024); }

template <class WT>
static void mlp_fwd(cudaStream_t s, const WT* P, const float* pb, int batch, const float* x, float* a1, float* a2, float* y) {
    // biases are always FP32 (pb); weights WT (float or bf16) at the same offsets as P
    gemm<false, true, WT>(s, x, P + kOffW1, a1, batch, kW1, kW0, pb + kOffB1, true);
    gemm<false, true, WT>(s, a1, P + kOffW2, a2, batch, kW2, kW1, pb + kOffB2, true);
    gemm<false, true, WT>(s, a2, P + kOffW3, y, batch, kW3, kW2, pb + kOffB3, false);
}

}  // namespace firm

using namespace firm;

extern "C" {

int firm_mlp_param_count(void) { return (int)kParams; }

size_t firm_mlp_work_floats(int batch) { return mlp_work_floats(batch); }

int firm_mlp_forward(const float* params, int batch, const float* x, float* y, float* work, void* stream) {
    if (!params || !x || !y || !work || batch <= 0) return FIRM_EINVAL;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    float* a1 = work;
    float* a2 = a1 + (size_t)batch * 256;
    mlp_fwd<float>(s, params, params, batch, x, a1, a2, y);
    return cudaGetLastError() == cudaSuccess ? FIRM_OK : FIRM_ECUDA;
}

int firm_mlp_to_bf16(const float* params, void* params_bf16, void* stream) {
    if (!params || !params_bf16) return FIRM_EINVAL;
    k_to_bf16<<<256, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(params, reinterpret_cast<__nv_bfloat16*>(params_bf16),
                                                                       kParams);
    return cudaGetLastError() == cudaSuccess ? FIRM_OK : FIRM_ECUDA;
}

int firm_mlp_forward_bf16(const void* params_bf16, const float* params, int batch, const float* x, float* y, float* work,
                          void* stream) {
    if (!params_bf16 || !params || !x || !y || !work || batch <= 0) return FIRM_EINVAL;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    float* a1 = work;
    float* a2 = a1 + (size_t)batch * 256;
    mlp_fwd<__nv_bfloat16>(s, reinterpret_cast<const __nv_bfloat16*>(params_bf16), params, batch, x, a1, a2, y);
    return cudaGetLastError() == cudaSuccess ? FIRM_OK : FIRM_ECUDA;
}

int firm_mlp_grad(const float* params, int batch, const float* x, const float* t, float* grad, float* work,
                  double* loss, void* stream) {
    if (!params || !x || !t || !grad || !work || !loss || batch <= 0) return FIRM_EINVAL;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    float* a1 = work;
    float* a2 = a1 + (size_t)batch * 256;
    float* y = a2 + (size_t)batch * 256;
    float* g1 = y + (size_t)batch * 1024;
    float* g2 = g1 + (size_t)batch * 256;
    float* gy = g2 + (size_t)batch * 256;
    mlp_fwd<float>(s, params, params, batch, x, a1, a2, y);
    if (cudaMemsetAsync(loss, 0, sizeof(double), s) != cudaSuccess) return FIRM_ECUDA;
    const size_t ny = (size_t)batch * kW3;
    k_mse_grad<<<128, 256, 0, s>>>(y, t, gy, ny, loss);
    // layer 3: gW3 = gy^T a2, gb3 = colsum gy, g2 = gy W3 masked
    gemm<true, false, float>(s, gy, a2, grad + kOffW3, kW3, kW2, batch, nullptr, false);
    k_colsum<<<(kW3 + 255) / 256, 256, 0, s>>>(gy, grad + kOffB3, batch, kW3);
    gemm<false, false, float>(s, gy, params + kOffW3, g2, batch, kW2, kW3, nullptr, false);
    k_relu_mask<<<128, 256, 0, s>>>(g2, a2, (size_t)batch * kW2);
    // layer 2
    gemm<true, false, float>(s, g2, a1, grad + kOffW2, kW2, kW1, batch, nullptr, false);
    k_colsum<<<(kW2 + 255) / 256, 256, 0, s>>>(g2, grad + kOffB2, batch, kW2);
    gemm<false, false, float>(s, g2, params + kOffW2, g1, batch, kW1, kW2, nullptr, false);
    k_relu_mask<<<128, 256, 0, s>>>(g1, a1, (size_t)batch * kW1);
    // layer 1
    gemm<true, false, float>(s, g1, x, grad + kOffW1, kW1, kW0, batch, nullptr, false);
    k_colsum<<<(kW1 + 255) / 256, 256, 0, s>>>(g1, grad + kOffB1, batch, kW1);
    return cudaGetLastError() == cudaSuccess ? FIRM_OK : FIRM_ECUDA;
}

int firm_mlp_adam(float* params, const float* grad, float* m, float* v, int step, float lr, void* stream) {
    if (!params || !grad || !m || !v || step < 1) return FIRM_EINVAL;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f - std::pow(b1, (float)step), c2 = 1.0f - std::pow(b2, (float)step);
    k_adam<<<512, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(params, grad, m, v, kParams, lr, b1, b2, 1e-8f, c1, c2);
    return cudaGetLastError() == cudaSuccess ? FIRM_OK : FIRM_ECUDA;
}

}  // extern "C"
