// fft_passes.cu -- every FFT-based stage of the FIRM hot path.
//
//   image DFT   FIRM step 1 (Section 3.4; Section 2.2 centred DFT, eq. measurement):
//               one CTA per image, row then column transforms in shared memory, the
//               half-disc samples times h_m and the shift phase written out.
//   Ker         eq. kernel: the 4N^3 fine grid (FP64) transformed along x, y, z with
//               output pruning to n in [-N, N) (n1 >= 0 by Ker(-n) = Ker(n)),
//               Ker = 2 Re(ghat) / phihat (the factor 2 adds the mirrored half disc).
//   K-hat       eq. embedding_circulant / eq. circ1: the 2N^3 circulant column gathered
//               from the Ker half box, transformed, real part kept on j1 in [0, N].
//   A*b         eq. backprojection: 2N^3 complex fine grid -> N^3, 2 Re / phihat.
//   Toeplitz    eq. property via Section 3.2: x padded to 2N^3; per z-plane, forward
//               along x (real rows, half spectrum kept) and y with the plane held in
//               shared memory; z-forward x K-hat x z-inverse in one pass; per z-plane,
//               y-inverse and x-inverse (Hermitian rows) with the crop, 1/(2N)^3 and
//               lam_eff x fused; optionally the CG update p = r + beta p in the first
//               pass and the FP64 partial sums of <p, Ap> in the last.  The first-
//               difference damping (Section 5) is added to K-hat once (k_khat_damp).
//   PCG         the Fourier-diagonal preconditioner on N^3 in the same three-launch
//               form (not in the paper).
//   A V         the forward projector's transform (type-2 NUFFT): V / phihat with the
//               centring sign, zero-padded to (2N)^3, forward along x, y, z in place.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "bulk.cuh"
#include "dw.cuh"
#include "fft.cuh"
#include "firm_internal.h"

namespace firm {


cudaError_t fft_init_constants() {
    float2 h[kTwConstTotal];
    const int sizes[] = {4, 6, 8, 10, 12, 16, 20, 24, 32};
    for (int R : sizes) {
        const int off = tw_offset(R);
        for (int j = 0; j < R; ++j) {
            const double a = -2.0 * 3.14159265358979323846 * (double)j / (double)R;
            h[off + j] = make_float2((float)cos(a), (float)sin(a));
        }
    }
    return cudaMemcpyToSymbol(c_tw, h, sizeof(h));
}

constexpr int kThreads = 256;
// Lines per tile of a column pass: enough that step 1 of the four-step FFT gives
// every thread one item (lines x L2 = kThreads).
template <int L> __host__ __device__ constexpr int TX() { return kThreads / Split<L>::L2; }

// ---------------------------------------------------------------------------
// Generic pass kernels.  An Op provides n_outer, n_inner / n_rows, tw, load, store.
// ---------------------------------------------------------------------------
template <int L, int SIGN, class Op>
__global__ void __launch_bounds__(kThreads) k_cols(const Op op) {
    extern __shared__ float2 S[];
    const int tiles = (op.n_inner + TX<L>() - 1) / TX<L>();
    const int outer = blockIdx.x / tiles;
    const int c0 = (blockIdx.x % tiles) * TX<L>();
    const int nl = min(TX<L>(), op.n_inner - c0);
    auto ld = [&](int line, int n) { return op.load(outer, n, c0 + line); };
    auto st = [&](int line, int k, float2 v) { op.store(outer, k, c0 + line, v); };
    block_fft<L, SIGN, true>(nl, ld, st, S, op.tw);
}

template <int L> __host__ __device__ constexpr int rows_per_block() { return kThreads / Split<L>::L2; }

template <int L, int SIGN, class Op>
__global__ void __launch_bounds__(kThreads) k_rows(Op op) {
    extern __shared__ float2 S[];
    constexpr int ROWS = rows_per_block<L>();
    const int r0 = blockIdx.x * ROWS;
    const int nl = min(ROWS, op.n_rows - r0);
    auto ld = [&](int line, int n) { return op.load(r0 + line, n); };
    auto st = [&](int line, int k, float2 v) { op.store(r0 + line, k, v); };
    block_fft<L, SIGN, false>(nl, ld, st, S, op.tw);
    op.finish();
}

template <int L, int SIGN, class Op>
static cudaError_t run_cols(const Op& op, cudaStream_t s) {
    const size_t smem = sizeof(float2) * smem_elems<L, true>(TX<L>());
    cudaError_t e = cudaFuncSetAttribute(k_cols<L, SIGN, Op>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int tiles = (op.n_inner + TX<L>() - 1) / TX<L>();
    k_cols<L, SIGN, Op><<<op.n_outer * tiles, kThreads, smem, s>>>(op);
    return cudaGetLastError();
}

template <int L, int SIGN, class Op>
static cudaError_t run_rows(const Op& op, cudaStream_t s) {
    constexpr int ROWS = rows_per_block<L>();
    const size_t smem = sizeof(float2) * smem_elems<L, false>(ROWS);
    cudaError_t e = cudaFuncSetAttribute(k_rows<L, SIGN, Op>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_rows<L, SIGN, Op><<<(op.n_rows + ROWS - 1) / ROWS, kThreads, smem, s>>>(op);
    return cudaGetLastError();
}

struct NoFinish {
    __device__ __forceinline__ void finish() const {}
    __device__ __forceinline__ void prepare() {}                       // per-block scalars
    __device__ __forceinline__ void post(int, int, float2) const {}    // after an item's loads
};

// Transform lengths instantiated: 2N and 4N for N in {16, 32, 48, 64, 80, 96, 128}.
#define FIRM_CASE_L(V, ...) case V: { constexpr int LL = V; __VA_ARGS__; } break;
#define FIRM_SWITCH_2N(Lval, ...)                                                             \
    switch (Lval) {                                                                          \
        FIRM_CASE_L(32, __VA_ARGS__) FIRM_CASE_L(64, __VA_ARGS__) FIRM_CASE_L(96, __VA_ARGS__)   \
        FIRM_CASE_L(128, __VA_ARGS__) FIRM_CASE_L(160, __VA_ARGS__) FIRM_CASE_L(192, __VA_ARGS__) \
        FIRM_CASE_L(256, __VA_ARGS__)                                                          \
        default: return cudaErrorInvalidValue;                                               \
    }
#define FIRM_SWITCH_4N(Lval, ...)                                                             \
    switch (Lval) {                                                                          \
        FIRM_CASE_L(64, __VA_ARGS__) FIRM_CASE_L(128, __VA_ARGS__) FIRM_CASE_L(192, __VA_ARGS__) \
        FIRM_CASE_L(256, __VA_ARGS__) FIRM_CASE_L(320, __VA_ARGS__) FIRM_CASE_L(384, __VA_ARGS__) \
        FIRM_CASE_L(512, __VA_ARGS__)                                                          \
        default: return cudaErrorInvalidValue;                                               \
    }

// ---------------------------------------------------------------------------
// Ker: 4N^3 real FP64 grid -> Ker half box
// ---------------------------------------------------------------------------
struct KerRowsOp : NoFinish {
    const double* grid; float2* out; const float2* tw; int n_rows, G, N;
    __device__ __forceinline__ float2 load(int row, int n) const {
        return make_float2((float)__ldg(&grid[(size_t)row * G + n]), 0.0f);
    }
    __device__ __forceinline__ void store(int row, int k, float2 v) const {
        if (k <= N) out[(size_t)row * (N + 1) + k] = v;
    }
};
struct KerColsYOp {
    const float2* in; float2* out; const float2* tw; int n_outer, n_inner, G, N;
    __device__ __forceinline__ float2 load(int o, int n, int i) const {
        return __ldg(&in[((size_t)o * G + n) * (N + 1) + i]);
    }
    __device__ __forceinline__ void store(int o, int k, int i, float2 v) const {
        const int n2 = k < N ? k : (k >= G - N ? k - G : G);
        if (n2 != G) out[((size_t)o * 2 * N + (n2 + N)) * (N + 1) + i] = v;
    }
};
struct KerColsZOp {
    const float2* in; float* ker; const float* dec; const float2* tw; int n_outer, n_inner, G, N;
    __device__ __forceinline__ float2 load(int, int n, int i) const { return __ldg(&in[(size_t)n * n_inner + i]); }
    __device__ __forceinline__ void store(int, int k, int i, float2 v) const {
        const int n3 = k < N ? k : (k >= G - N ? k - G : G);
        if (n3 == G) return;
        const int n2i = i / (N + 1), n1 = i - n2i * (N + 1);
        ker[(size_t)(n3 + N) * n_inner + i] = 2.0f * v.x * __ldg(&dec[n1 + N]) * __ldg(&dec[n2i]) * __ldg(&dec[n3 + N]);
    }
};

cudaError_t launch_ker_transform(Plan& P) {
    Workspace& w = P.ws;
    const int N = P.N, G = P.Gk;
    cudaError_t e = cudaSuccess;
    KerRowsOp a{{}, w.grid, w.fx1, w.tw_4n, G * G, G, N};
    KerColsYOp b{w.fx1, w.fx2, w.tw_4n, G, N + 1, G, N};
    KerColsZOp c{w.fx2, w.ker, w.dec_k, w.tw_4n, 1, 2 * N * (N + 1), G, N};
    FIRM_SWITCH_4N(G, {
        if ((e = run_rows<LL, +1>(a, P.stream)) != cudaSuccess) return e;
        if ((e = run_cols<LL, +1>(b, P.stream)) != cudaSuccess) return e;
        if ((e = run_cols<LL, +1>(c, P.stream)) != cudaSuccess) return e;
    });
    P.launches += 3;
    return e;
}

// ---------------------------------------------------------------------------
// K-hat: circulant column (reading: lag-N planes zero) -> 2N^3 forward FFT, real part
// ---------------------------------------------------------------------------
struct KhatRowsOp : NoFinish {
    const float* ker; float2* out; const float2* tw; int n_rows, N;
    __device__ __forceinline__ float2 load(int row, int i1) const {
        const int N2 = 2 * N;
        const int i3 = row / N2, i2 = row - i3 * N2;
        if (i1 == N || i2 == N || i3 == N) return make_float2(0.0f, 0.0f);
        const int d1 = i1 < N ? i1 : i1 - N2;
        const int d2 = i2 < N ? i2 : i2 - N2;
        const int d3 = i3 < N ? i3 : i3 - N2;
        size_t idx;
        if (d1 >= 0) idx = ((size_t)(d3 + N) * N2 + (d2 + N)) * (N + 1) + d1;
        else idx = ((size_t)(N - d3) * N2 + (N - d2)) * (N + 1) + (-d1);
        return make_float2(__ldg(&ker[idx]), 0.0f);
    }
    __device__ __forceinline__ void store(int row, int k, float2 v) const {
        if (k <= N) out[(size_t)row * (N + 1) + k] = v;
    }
};
struct KhatColsYOp {
    const float2* in; float2* out; const float2* tw; int n_outer, n_inner, L;
    __device__ __forceinline__ float2 load(int o, int n, int i) const {
        return __ldg(&in[((size_t)o * L + n) * n_inner + i]);
    }
    __device__ __forceinline__ void store(int o, int k, int i, float2 v) const {
        out[((size_t)o * L + k) * n_inner + i] = v;
    }
};
struct KhatColsZOp {
    const float2* in; float* khat; const float2* tw; int n_outer, n_inner;
    __device__ __forceinline__ float2 load(int, int n, int i) const { return __ldg(&in[(size_t)n * n_inner + i]); }
    __device__ __forceinline__ void store(int, int k, int i, float2 v) const { khat[(size_t)k * n_inner + i] = v.x; }
};

cudaError_t launch_khat(Plan& P) {
    Workspace& w = P.ws;
    const int N = P.N, L = 2 * N;
    cudaError_t e = cudaSuccess;
    KhatRowsOp a{{}, w.ker, w.fx1, w.tw_2n, L * L, N};
    KhatColsYOp b{w.fx1, w.fx2, w.tw_2n, L, N + 1, L};
    KhatColsZOp c{w.fx2, w.khat, w.tw_2n, 1, L * (N + 1)};
    FIRM_SWITCH_2N(L, {
        if ((e = run_rows<LL, -1>(a, P.stream)) != cudaSuccess) return e;
        if ((e = run_cols<LL, -1>(b, P.stream)) != cudaSuccess) return e;
        if ((e = run_cols<LL, -1>(c, P.stream)) != cudaSuccess) return e;
    });
    P.launches += 3;
    return e;
}

// lam_eff = lambda Ker(0) (relative reading) or lambda (absolute), on the device, so that
// the Toeplitz apply needs no host round trip; Ker(0) sits at (j3, j2, j1) = (N, N, 0).
__global__ void k_lam_eff(const float* __restrict__ ker, size_t i0, double lambda, int relative, float* lam) {
    const float k0 = ker[i0];
    lam[0] = relative ? (float)(lambda * (double)k0) : (float)lambda;
    lam[1] = k0;
}

cudaError_t launch_lam_eff(Plan& P) {
    const size_t i0 = ((size_t)P.N * 2 * P.N + P.N) * (P.N + 1);
    k_lam_eff<<<1, 1, 0, P.stream>>>(P.ws.ker, i0, P.p.lambda, P.p.lambda_mode == FIRM_LAMBDA_RELATIVE ? 1 : 0,
                                     P.ws.lam);
    P.launches += 1;
    return cudaGetLastError();
}

// High-frequency damping mu ||D V||^2 (D: first differences of V on its box, zero
// outside; a Fourier-domain regulariser of the kind Section 5 says FIRM takes in
// naturally).  D^T D is the convolution with the 7-point stencil 6 delta(n) -
// sum over a and +-1 of delta(n -+ e_a), whose support lies well inside [-N, N)^3, so it
// is added to the circulant's spectrum on the 2N grid and costs nothing per CG
// iteration: K-hat(j) += mu_eff (6 - 2 sum_a cos(pi j_a / N)), mu_eff = mu Ker(0)
// (relative reading, as lam_eff) or mu.  khat: half spectrum [j3][j2][j1], j1 in
// [0, N]; khat64 (FP64 CG mode, may be null): the full (2N)^3.
__global__ void k_khat_damp(float* __restrict__ khat, double* __restrict__ khat64, int N, double mu, int relative,
                            const float* __restrict__ lam) {
    const double m = relative ? mu * (double)lam[1] : mu;
    const long long G = 2LL * N, H = N + 1;
    const long long n_half = G * G * H, n_full = khat64 ? G * G * G : 0;
    const long long total = n_half > n_full ? n_half : n_full;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        if (i < n_half) {
            const int j1 = (int)(i % H), j2 = (int)((i / H) % G), j3 = (int)(i / (H * G));
            const double sym = 6.0 - 2.0 * (cospi((double)j1 / N) + cospi((double)j2 / N) + cospi((double)j3 / N));
            khat[i] += (float)(m * sym);
        }
        if (i < n_full) {
            const int j1 = (int)(i % G), j2 = (int)((i / G) % G), j3 = (int)(i / (G * G));
            const double sym = 6.0 - 2.0 * (cospi((double)j1 / N) + cospi((double)j2 / N) + cospi((double)j3 / N));
            khat64[i] += m * sym;
        }
    }
}

cudaError_t launch_damping(Plan& P) {
    if (!(P.mu > 0.0)) return cudaSuccess;
    const bool fp64 = (P.p.flags & FIRM_FLAG_FP64_CG) != 0;
    k_khat_damp<<<P.num_sms * 4, 256, 0, P.stream>>>(P.ws.khat, fp64 ? P.ws.khat64 : nullptr, P.N, P.mu,
                                                     P.p.lambda_mode == FIRM_LAMBDA_RELATIVE ? 1 : 0, P.ws.lam);
    P.launches += 1;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// A*b: 2N^3 complex FP64 grid -> N^3 real
// ---------------------------------------------------------------------------
struct RhsRowsOp : NoFinish {
    const double* grid; float2* out; const float2* tw; int n_rows, G, N;
    __device__ __forceinline__ float2 load(int row, int n) const {
        const double2 g = __ldg(reinterpret_cast<const double2*>(grid) + (size_t)row * G + n);
        return make_float2((float)g.x, (float)g.y);
    }
    __device__ __forceinline__ void store(int row, int k, float2 v) const {
        const int h = N / 2;
        const int n1 = k < h ? k : (k >= G - h ? k - G : G);
        if (n1 != G) out[(size_t)row * N + (n1 + h)] = v;
    }
};
struct RhsColsYOp {
    const float2* in; float2* out; const float2* tw; int n_outer, n_inner, G, N;
    __device__ __forceinline__ float2 load(int o, int n, int i) const {
        return __ldg(&in[((size_t)o * G + n) * N + i]);
    }
    __device__ __forceinline__ void store(int o, int k, int i, float2 v) const {
        const int h = N / 2;
        const int n2 = k < h ? k : (k >= G - h ? k - G : G);
        if (n2 != G) out[((size_t)o * N + (n2 + h)) * N + i] = v;
    }
};
struct RhsColsZOp {
    const float2* in; float* rhs; const float* dec; const float2* tw; int n_outer, n_inner, G, N;
    __device__ __forceinline__ float2 load(int, int n, int i) const { return __ldg(&in[(size_t)n * n_inner + i]); }
    __device__ __forceinline__ void store(int, int k, int i, float2 v) const {
        const int h = N / 2;
        const int n3 = k < h ? k : (k >= G - h ? k - G : G);
        if (n3 == G) return;
        const int n2i = i / N, n1i = i - n2i * N;
        rhs[(size_t)(n3 + h) * n_inner + i] = 2.0f * v.x * __ldg(&dec[n1i]) * __ldg(&dec[n2i]) * __ldg(&dec[n3 + h]);
    }
};

cudaError_t launch_rhs_transform(Plan& P) {
    Workspace& w = P.ws;
    const int N = P.N, G = P.Gr;
    cudaError_t e = cudaSuccess;
    RhsRowsOp a{{}, w.grid, w.fx1, w.tw_2n, G * G, G, N};
    RhsColsYOp b{w.fx1, w.fx2, w.tw_2n, G, N, G, N};
    RhsColsZOp c{w.fx2, w.rhs, w.dec_r, w.tw_2n, 1, N * N, G, N};
    FIRM_SWITCH_2N(G, {
        if ((e = run_rows<LL, +1>(a, P.stream)) != cudaSuccess) return e;
        if ((e = run_cols<LL, +1>(b, P.stream)) != cudaSuccess) return e;
        if ((e = run_cols<LL, +1>(c, P.stream)) != cudaSuccess) return e;
    });
    P.launches += 3;
    return e;
}

// A*b of the fused form: the complex A*b grid on the 4N fine grid (right after the real
// Ker grid), transformed along x, y, z with output pruning to the N modes and the
// deconvolution for oversampling 4 fused into the last pass.
cudaError_t launch_rhs_transform4(Plan& P) {
    Workspace& w = P.ws;
    const int N = P.N, G = P.Gk;
    const double* grid = w.grid + (size_t)G * G * G;
    cudaError_t e = cudaSuccess;
    RhsRowsOp a{{}, grid, w.fx1, w.tw_4n, G * G, G, N};
    RhsColsYOp b{w.fx1, w.fx2, w.tw_4n, G, N, G, N};
    RhsColsZOp c{w.fx2, w.rhs, w.dec_r4, w.tw_4n, 1, N * N, G, N};
    FIRM_SWITCH_4N(G, {
        if ((e = run_rows<LL, +1>(a, P.stream)) != cudaSuccess) return e;
        if ((e = run_cols<LL, +1>(b, P.stream)) != cudaSuccess) return e;
        if ((e = run_cols<LL, +1>(c, P.stream)) != cudaSuccess) return e;
    });
    P.launches += 3;
    return e;
}

// ---------------------------------------------------------------------------
// Forward projector (eq. forward-projector), transform half of the type-2 NUFFT: the
// volume times (-1)^n / phihat(n / 2N) per axis (dec_r; the sign centres the fine
// grid so that a slice point's fine-grid coordinate indexes it directly), zero-padded
// to (2N)^3 at n mod 2N and transformed forward along x, y, z in place.
// ---------------------------------------------------------------------------
struct FwdRowsOp : NoFinish {
    const float* V; const float* dec; float2* g; const float2* tw; int n_rows, G, N;
    __device__ __forceinline__ float2 load(int row, int n) const {      // row = i3 * N + i2
        const int h = N / 2;
        const int n1 = n < h ? n : (n >= G - h ? n - G : G);
        if (n1 == G) return make_float2(0.0f, 0.0f);
        const int i1 = n1 + h, i2 = row % N, i3 = row / N;
        const float v = __ldg(&V[(size_t)row * N + i1]) * __ldg(&dec[i1]) * __ldg(&dec[i2]) * __ldg(&dec[i3]);
        return make_float2(v, 0.0f);
    }
    __device__ __forceinline__ void store(int row, int k, float2 v) const {
        const int h = N / 2, i2 = row % N, i3 = row / N;
        const int j2 = i2 < h ? i2 - h + G : i2 - h, j3 = i3 < h ? i3 - h + G : i3 - h;
        g[((size_t)j3 * G + j2) * G + k] = v;
    }
};
struct FwdColsYOp {            // planes o = i3 (j3 = n3 mod G), columns j1
    float2* g; const float2* tw; int n_outer, n_inner, G, N;
    __device__ __forceinline__ size_t plane(int o) const {
        const int h = N / 2;
        return (size_t)(o < h ? o - h + G : o - h) * G * G;
    }
    __device__ __forceinline__ float2 load(int o, int n, int i) const {
        const int h = N / 2;
        if (n >= h && n < G - h) return make_float2(0.0f, 0.0f);          // padding rows
        return g[plane(o) + (size_t)n * G + i];
    }
    __device__ __forceinline__ void store(int o, int k, int i, float2 v) const { g[plane(o) + (size_t)k * G + i] = v; }
};
struct FwdColsZOp {            // columns (j2, j1) of all G^2
    float2* g; const float2* tw; int n_outer, n_inner, G, N;
    __device__ __forceinline__ float2 load(int, int n, int i) const {
        const int h = N / 2;
        if (n >= h && n < G - h) return make_float2(0.0f, 0.0f);          // padding planes
        return g[(size_t)n * n_inner + i];
    }
    __device__ __forceinline__ void store(int, int k, int i, float2 v) const { g[(size_t)k * n_inner + i] = v; }
};

cudaError_t launch_fwd_transform(Plan& P, const float* V, float2* ghat) {
    Workspace& w = P.ws;
    const int N = P.N, G = P.Gr;
    cudaError_t e = cudaSuccess;
    FwdRowsOp a{{}, V, w.dec_r, ghat, w.tw_2n, N * N, G, N};
    FwdColsYOp b{ghat, w.tw_2n, N, G, G, N};
    FwdColsZOp c{ghat, w.tw_2n, 1, G * G, G, N};
    FIRM_SWITCH_2N(G, {
        if ((e = run_rows<LL, -1>(a, P.stream)) != cudaSuccess) return e;
        if ((e = run_cols<LL, -1>(b, P.stream)) != cudaSuccess) return e;
        if ((e = run_cols<LL, -1>(c, P.stream)) != cudaSuccess) return e;
    });
    P.launches += 3;
    return e;
}

// ---------------------------------------------------------------------------
// Image DFT (FIRM step 1)
// ---------------------------------------------------------------------------
struct ImgArgs {
    const void* images; const double* shifts; const int32_t* gid; const int32_t* htab;
    const float* h1; float2* samples; const float2* tw; int nH, n_ctf;
    int plain;              // 1: b itself (no h, k = 0 not halved), for the data residual
    int* err;               // device failure flag (bit 2: the image copy did not land in time)
};

// A pixel of the image staged in shared memory (float32 or bfloat16 bits).
template <class T>
__device__ __forceinline__ float img_val(const T* p, int i) {
    if constexpr (sizeof(T) == 2) return __bfloat162float(__ushort_as_bfloat16(p[i]));
    else return p[i];
}

template <int N> __host__ __device__ constexpr int img_rows() { return kThreads / Split<N>::L2; }
// the N/2 + 1 columns of the half spectrum in two tiles (every thread busy in step 1)
template <int N> __host__ __device__ constexpr int img_col_tile() { return (N / 2 + 2) / 2; }
template <int N> __host__ __device__ constexpr int img_smem_elems() {
    constexpr int a = smem_elems<N, false>(img_rows<N>());
    constexpr int b = smem_elems<N, true>(img_col_tile<N>());
    return N * (N / 2 + 1) + (a > b ? a : b);
}

template <int N, class T>
__global__ void __launch_bounds__(kThreads) k_image_dft(const ImgArgs a) {
    extern __shared__ float2 sm2[];
    __shared__ __align__(8) unsigned long long s_bar;
    constexpr int H1 = N / 2 + 1;
    float2* S1 = sm2;
    float2* scr = sm2 + N * H1;
    const int m = blockIdx.x;
    const size_t img0 = (size_t)m * N * N;
    constexpr int ROWS = img_rows<N>();
    // The image arrives with one bulk copy (the tensor memory accelerator) into the tail
    // of S1: the row transforms write S1 rows 2j, 2j+1 only after reading image rows 2j,
    // 2j+1 (each batch loads all its inputs before it stores), and with the image ending
    // where S1 ends, the rows written so far never reach the rows still to be read
    // (written bytes 16 H1 p <= unread offset S1 - img + 2 N sizeof(T) p for every p <= N/2).
    constexpr uint32_t kImgBytes = (uint32_t)(N * N * sizeof(T));
    constexpr uint32_t kS1Bytes = (uint32_t)(sizeof(float2) * N * H1);
    static_assert(kImgBytes <= kS1Bytes && (kS1Bytes - kImgBytes) % 16 == 0 && kImgBytes % 16 == 0, "staging");
    const T* img = reinterpret_cast<const T*>(reinterpret_cast<const unsigned char*>(S1) + (kS1Bytes - kImgBytes));
    if (threadIdx.x == 0) mbar_init(&s_bar);
    __syncthreads();
    if (threadIdx.x == 0)
        bulk_g2s(const_cast<T*>(img), reinterpret_cast<const T*>(a.images) + img0, kImgBytes, &s_bar);
    if (!mbar_wait(&s_bar, 0)) {
        if (threadIdx.x == 0) atomicOr(a.err, 4);
        mbar_wait(&s_bar, 0);                      // the copy in flight, then leave
        return;
    }
    // rows 2j and 2j+1 (real) transformed together as z = x_2j + i x_2j+1: Z[k] for
    // k <= N/2 goes to row 2j's slots, Z[k] for k > N/2 to row 2j+1's (slot k - N/2 - 1)
    constexpr int NP = N / 2;
    for (int l0 = 0; l0 < NP; l0 += ROWS) {
        const int nl = min(ROWS, NP - l0);
        auto ld = [&](int line, int n) {
            const int i = (2 * (l0 + line)) * N + n;
            return make_float2(img_val<T>(img, i), img_val<T>(img, i + N));
        };
        auto st = [&](int line, int k, float2 v) {
            const int j = l0 + line;
            if (k < H1) S1[(2 * j) * H1 + k] = v;
            else S1[(2 * j + 1) * H1 + (k - H1)] = v;
        };
        block_fft<N, -1, false>(nl, ld, st, scr, a.tw);
    }
    // the two real rows' half spectra, in place: X_2j[k] = (Z[k] + conj Z[N-k]) / 2,
    // X_2j+1[k] = (Z[k] - conj Z[N-k]) / 2i.  Task q < N/4 owns k = q and
    // k' = N/2 - 1 - q, whose four slots hold exactly the Z values both need (Z[N-k] of
    // one is in the other's row-2j+1 slot); task q = N/4 takes k = N/2.
    for (int it = threadIdx.x; it < NP * (N / 4 + 1); it += blockDim.x) {
        const int j = it / (N / 4 + 1), q = it % (N / 4 + 1);
        float2* A = S1 + (2 * j) * H1;
        float2* B = S1 + (2 * j + 1) * H1;
        if (q == N / 4) {                                   // k = N/2: Z[N - k] = Z[k]
            const float2 z = A[N / 2];
            A[N / 2] = make_float2(z.x, 0.0f);
            B[N / 2] = make_float2(z.y, 0.0f);
            continue;
        }
        const int k2 = N / 2 - 1 - q;
        const float2 zk2 = A[k2], zm2 = B[q];               // Z[k'], Z[N - k']
        float2 xa1, xb1;
        if (q == 0) {                                       // k = 0: Z[N - k] = Z[0]
            const float2 z0 = A[0];
            xa1 = make_float2(z0.x, 0.0f);
            xb1 = make_float2(z0.y, 0.0f);
        } else {
            const float2 zk = A[q], zm = B[k2];             // Z[k], Z[N - k]
            xa1 = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
            xb1 = make_float2(0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x));
        }
        A[q] = xa1;
        B[q] = xb1;
        A[k2] = make_float2(0.5f * (zk2.x + zm2.x), 0.5f * (zk2.y - zm2.y));
        B[k2] = make_float2(0.5f * (zk2.y + zm2.y), -0.5f * (zk2.x - zm2.x));
    }
    __syncthreads();
    constexpr int CT = img_col_tile<N>();
    for (int c0 = 0; c0 < H1; c0 += CT) {
        const int nl = min(CT, H1 - c0);
        auto ld = [&](int line, int n) { return S1[n * H1 + c0 + line]; };
        auto st = [&](int line, int k, float2 v) { S1[k * H1 + c0 + line] = v; };
        block_fft<N, -1, true>(nl, ld, st, scr, a.tw);
    }
    // half-disc samples: centred index sign, CTF, shift phase, k = 0 halved.  The shift
    // phase exp(i pi (k1 s1 + k2 s2)) factors per axis: its N/2 + 1 values in k1 and N + 1
    // in k2 are formed once per image (in the scratch space, free after the columns)
    const int g = a.gid ? min(max(__ldg(&a.gid[m]), 0), a.n_ctf - 1) : 0;
    const float s1 = (float)(2.0 * a.shifts[2 * m] / N), s2 = (float)(2.0 * a.shifts[2 * m + 1] / N);
    static_assert(img_smem_elems<N>() - N * H1 >= H1 + N + 1, "phase tables fit the scratch space");
    float2* ph1 = scr;                  // k1 = 0 .. N/2
    float2* ph2 = scr + H1;             // k2 = -N/2 .. N/2 at k2 + N/2
    for (int j = threadIdx.x; j < H1 + N + 1; j += blockDim.x) {
        float sn, cs;
        if (j < H1) {
            sincospif((float)j * s1, &sn, &cs);
            ph1[j] = make_float2(cs, sn);
        } else {
            sincospif((float)(j - H1 - N / 2) * s2, &sn, &cs);
            ph2[j - H1] = make_float2(cs, sn);
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < a.nH; t += blockDim.x) {
        const int kk = __ldg(&a.htab[t]);
        const int k1 = (int16_t)(kk & 0xffff), k2 = kk >> 16;
        float2 v = S1[((k2 + N) % N) * H1 + k1];
        float hs = a.plain ? 1.0f : __ldg(&a.h1[(size_t)g * a.nH + t]);
        if ((k1 + k2) & 1) hs = -hs;
        if (t == 0 && !a.plain) hs *= 0.5f;
        const float2 p = c_mul(ph1[k1], ph2[k2 + N / 2]);
        a.samples[(size_t)m * a.nH + t] = c_mul(v, make_float2(p.x * hs, p.y * hs));
    }
}

template <int N, class T>
static cudaError_t image_dft_n(Plan& P, int M, const ImgArgs& a) {
    const size_t smem = sizeof(float2) * img_smem_elems<N>();
    cudaError_t e = cudaFuncSetAttribute(k_image_dft<N, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_image_dft<N, T><<<M, kThreads, smem, P.stream>>>(a);
    P.launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_image_dft(Plan& P, int M, const void* images, const double* shifts, const int32_t* gid,
                             bool plain) {
    if (M <= 0) return cudaSuccess;
    // each image is staged by a bulk copy, which needs a 16-byte aligned source (every
    // entry point checks this before it queues any work)
    if (reinterpret_cast<uintptr_t>(images) & 15) return cudaErrorInvalidValue;
    ImgArgs a{images, shifts, gid, P.ws.htab, P.ws.h1, P.ws.samples, P.ws.tw_n, P.nH, P.n_ctf, plain ? 1 : 0,
              P.ws.counters + 2};
    const bool bf = P.p.img_dtype == FIRM_IMG_BF16;
    switch (P.N) {
        case 16: return bf ? image_dft_n<16, uint16_t>(P, M, a) : image_dft_n<16, float>(P, M, a);
        case 32: return bf ? image_dft_n<32, uint16_t>(P, M, a) : image_dft_n<32, float>(P, M, a);
        case 48: return bf ? image_dft_n<48, uint16_t>(P, M, a) : image_dft_n<48, float>(P, M, a);
        case 64: return bf ? image_dft_n<64, uint16_t>(P, M, a) : image_dft_n<64, float>(P, M, a);
        case 80: return bf ? image_dft_n<80, uint16_t>(P, M, a) : image_dft_n<80, float>(P, M, a);
        case 96: return bf ? image_dft_n<96, uint16_t>(P, M, a) : image_dft_n<96, float>(P, M, a);
        case 128: return bf ? image_dft_n<128, uint16_t>(P, M, a) : image_dft_n<128, float>(P, M, a);
        default: return cudaErrorInvalidValue;
    }
}

// ---------------------------------------------------------------------------
// Toeplitz apply (CG-fused when cg != nullptr)
// ---------------------------------------------------------------------------
struct TRowsFwdOp : NoFinish {
    const float* x; float* p; const float2* r; const CgState* cg; float2* out; const float2* tw; int n_rows, N;
    const float* z = nullptr;   // preconditioned residual: p = z + beta p when set
    float bh = 0.0f, bl = 0.0f; // beta as a double-word, read once per block
    __device__ __forceinline__ void prepare() {
        if (cg) { bh = cg->beta_f[0]; bl = cg->beta_f[1]; }
    }
    __device__ __forceinline__ float2 load(int row, int n) const {
        if (n >= N) return make_float2(0.0f, 0.0f);
        const size_t i = (size_t)row * N + n;
        if (cg) {   // p = r + beta p (r, beta double-words) or p = z + beta p; stored by post()
            const float pv = __ldg(&p[i]);
            float ah, al;
            if (z) { ah = __ldg(&z[i]); al = 0.0f; }
            else { const float2 rv = __ldg(&r[i]); ah = rv.x; al = rv.y; }
            return make_float2(fmaf(bh, pv, ah) + fmaf(bl, pv, al), 0.0f);
        }
        return make_float2(__ldg(&x[i]), 0.0f);
    }
    __device__ __forceinline__ void post(int row, int n, float2 v) const {
        if (cg && n < N) p[(size_t)row * N + n] = v.x;
    }
    __device__ __forceinline__ void store(int row, int k, float2 v) const {
        if (k <= N) out[(size_t)row * (N + 1) + k] = v;
    }
};
struct TColsYFwdOp {
    const float2* in; float2* out; const float2* tw; int n_outer, n_inner, N;
    __device__ __forceinline__ float2 load(int o, int n, int i) const {
        return n < N ? __ldg(&in[((size_t)o * N + n) * (N + 1) + i]) : make_float2(0.0f, 0.0f);
    }
    __device__ __forceinline__ void store(int o, int k, int i, float2 v) const {
        out[((size_t)o * 2 * N + k) * (N + 1) + i] = v;
    }
};
struct TColsYInvOp {
    const float2* in; float2* out; const float2* tw; int n_outer, n_inner, N;
    __device__ __forceinline__ float2 load(int o, int n, int i) const {
        return __ldg(&in[((size_t)o * 2 * N + n) * (N + 1) + i]);
    }
    __device__ __forceinline__ void store(int o, int k, int i, float2 v) const {
        if (k < N) out[((size_t)o * N + k) * (N + 1) + i] = v;
    }
};
struct TRowsInvOp {
    const float2* in; const float* x; float* y; double* red; CgState* cg; const float2* tw;
    int n_rows, N; float scale, lam;
    const float* lam_p;   // device lam_eff (overrides lam when set)
    float2* acc;   // per-thread partial <x, y> (CG), double-word
    __device__ __forceinline__ void prepare() {
        if (lam_p) lam = __ldg(lam_p);
    }
    __device__ __forceinline__ float2 load(int row, int n) const {
        const float2* rr = in + (size_t)row * (N + 1);
        return n <= N ? __ldg(&rr[n]) : c_conj(__ldg(&rr[2 * N - n]));
    }
    __device__ __forceinline__ float pre(int row, int k) const {
        return k < N ? __ldg(&x[(size_t)row * N + k]) : 0.0f;
    }
    __device__ __forceinline__ void store(int row, int k, float2 v, float xv) const {
        if (k >= N) return;
        const float yv = fmaf(v.x, scale, lam * xv);
        y[(size_t)row * N + k] = yv;
        if (cg) *acc = dw_acc_prod(*acc, xv, yv);
    }
    __device__ __forceinline__ void finish() const {}
};

// The z pass: forward, times K-hat, inverse; tile of TX<L>() adjacent (j2, j1) columns.
template <int L>
__global__ void __launch_bounds__(kThreads) k_toep_z(float2* __restrict__ t2, const float* __restrict__ khat,
                                                     const float2* __restrict__ tw, int n_inner, int N,
                                                     const CgState* cg) {
    extern __shared__ float2 S[];
    if (cg && cg->done) return;
    const int c0 = blockIdx.x * TX<L>();
    const int nl = min(TX<L>(), n_inner - c0);
    auto ld = [&](int line, int n) {
        return n < N ? t2[(size_t)n * n_inner + c0 + line] : make_float2(0.0f, 0.0f);
    };
    auto mul = [&](int line, int k) { return __ldg(&khat[(size_t)k * n_inner + c0 + line]); };
    auto st = [&](int line, int n, float2 v) {
        if (n < N) t2[(size_t)n * n_inner + c0 + line] = v;
    };
    block_fft_mul_ifft<L>(nl, ld, mul, st, S, tw);
}

// Last pass of the apply with the CG reduction of <p, Ap> (last-block pattern).
template <int L>
__global__ void __launch_bounds__(kThreads) k_toep_rows_inv(TRowsInvOp op) {
    extern __shared__ float2 S[];
    __shared__ double s_red[kThreads / 32];
    __shared__ bool s_last;
    if (op.cg && op.cg->done) return;
    constexpr int ROWS = rows_per_block<L>();
    const int r0 = blockIdx.x * ROWS;
    const int nl = min(ROWS, op.n_rows - r0);
    float2 acc = make_float2(0.0f, 0.0f);
    op.prepare();
    op.acc = &acc;
    auto ld = [&](int line, int n) { return op.load(r0 + line, n); };
    auto pre = [&](int line, int k) { return op.pre(r0 + line, k); };
    auto st = [&](int line, int k, float2 v, float xv) { op.store(r0 + line, k, v, xv); };
    fft_step1<L, +1, false>(nl, ld, S, op.tw);
    __syncthreads();
    fft_step2_pre<L, +1, false>(nl, pre, st, S);
    if (!op.cg) return;
    // block reduction
    const float2 wsum = dw_warp_sum(acc);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = dw_to_double(wsum);
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = 0.0;
        for (int i = 0; i < kThreads / 32; ++i) b += s_red[i];
        op.red[blockIdx.x] = b;
        __threadfence();
        const unsigned t = atomicAdd(&op.cg->ticket_a, 1u);
        s_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // deterministic final sum over block partials, in block order
    double v = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) v += ((volatile double*)op.red)[i];
    // fixed-order tree over threads
    __shared__ double s_fin[kThreads];
    s_fin[threadIdx.x] = v;
    __syncthreads();
    for (int s = kThreads / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) s_fin[threadIdx.x] += s_fin[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double pq = s_fin[0];
        const double alpha = (op.cg->use_pc ? op.cg->rz : op.cg->rr) / pq;
        op.cg->pq = pq;
        op.cg->alpha = alpha;
        const float2 af = dw_from_double(isfinite(alpha) ? alpha : 0.0);
        op.cg->alpha_f[0] = af.x;
        op.cg->alpha_f[1] = af.y;
        op.cg->ticket_a = 0;
    }
}

// The Toeplitz apply's x and y transforms, one z-plane per CTA (the z pass between
// them stays a column pass): the plane's N x (N+1) half spectrum (rows of 2N padded
// samples, k1 in [0, N]) stays in shared memory between the row and the column
// transforms, so the intermediate never goes through L2 or HBM and the apply is three
// launches instead of five.  Rows and columns go in the fewest batches that fit the
// exchange buffer beside the plane in 224 KB.
template <int L> struct TPlane {
    static constexpr int N = L / 2, H = N + 1;
    static constexpr int kBudget = 224 * 1024 / (int)sizeof(float2);
    static constexpr int kPlane = N * H;
    static constexpr int kRowElems = Split<L>::L1 * (Split<L>::L2 + 1);
    static constexpr int rb0 = (kBudget - kPlane) / kRowElems < N ? (kBudget - kPlane) / kRowElems : N;
    static constexpr int RB = (N + (N + rb0 - 1) / rb0 - 1) / ((N + rb0 - 1) / rb0);     // rows per batch
    static constexpr int cb0 = (kBudget - kPlane) / L < H ? (kBudget - kPlane) / L : H;
    static constexpr int CB = (H + (H + cb0 - 1) / cb0 - 1) / ((H + cb0 - 1) / cb0);     // columns per batch
    static constexpr int kX = smem_elems<L, false>(RB) > smem_elems<L, true>(CB) ? smem_elems<L, false>(RB)
                                                                                   : smem_elems<L, true>(CB);
    static constexpr int kSmem = kPlane + kX;                                          // float2 elements
    static constexpr int kL = Split<L>::L1 > Split<L>::L2 ? Split<L>::L1 : Split<L>::L2;
    static constexpr int kItems = (RB > CB ? RB : CB) * kL;
    static constexpr int kThreadsP = kItems < 1024 ? (kItems + 31) / 32 * 32 : 1024;
};

// x rows (p = r + beta p, or p = z + beta p, when CG-fused) forward into the plane,
// then y forward (N nonzero of 2N) into t2[z][k2][k1].
template <int L>
__global__ void __launch_bounds__(TPlane<L>::kThreadsP) k_toep_plane_fwd(TRowsFwdOp op, float2* __restrict__ t2,
                                                                        const CgState* cg) {
    using T = TPlane<L>;
    constexpr int N = T::N, H = T::H;
    extern __shared__ float2 S[];
    if (cg && cg->done) return;
    float2* plane = S;                          // [y][k1]
    float2* X = S + T::kPlane;
    const int row0 = blockIdx.x * N;            // rows of this plane in [z][y] order
    op.prepare();
    for (int r0 = 0; r0 < N; r0 += T::RB) {
        const int nl = min(T::RB, N - r0);
        auto ld = [&](int line, int n) { return op.load(row0 + r0 + line, n); };
        auto post = [&](int line, int n, float2 v) { op.post(row0 + r0 + line, n, v); };
        auto st = [&](int line, int k, float2 v) {
            if (k <= N) plane[(r0 + line) * H + k] = v;
        };
        fft_step1_post<L, -1, false>(nl, ld, post, X, op.tw);
        __syncthreads();
        fft_step2<L, -1, false>(nl, st, X);
        __syncthreads();
    }
    float2* out = t2 + (size_t)blockIdx.x * 2 * N * H;
    for (int c0 = 0; c0 < H; c0 += T::CB) {
        const int nl = min(T::CB, H - c0);
        auto ld = [&](int line, int n) { return n < N ? plane[n * H + c0 + line] : make_float2(0.0f, 0.0f); };
        auto st = [&](int line, int k, float2 v) { out[(size_t)k * H + c0 + line] = v; };
        block_fft<L, -1, true>(nl, ld, st, X, op.tw);
    }
}

// y inverse of t2[z] keeping y < N into the plane, then the Hermitian x rows back to
// real with the crop, 1/(2N)^3 and + lam x (op.store); CG-fused: <x, y> reduced, the
// last CTA forms alpha (sums in CTA order).
template <int L>
__global__ void __launch_bounds__(TPlane<L>::kThreadsP) k_toep_plane_inv(TRowsInvOp op, const float2* __restrict__ t2) {
    using T = TPlane<L>;
    constexpr int N = T::N, H = T::H;
    extern __shared__ float2 S[];
    __shared__ double s_red[32];
    __shared__ bool s_last;
    if (op.cg && op.cg->done) return;
    float2* plane = S;                          // [y][k1]
    float2* X = S + T::kPlane;
    const float2* in = t2 + (size_t)blockIdx.x * 2 * N * H;
    for (int c0 = 0; c0 < H; c0 += T::CB) {
        const int nl = min(T::CB, H - c0);
        auto ld = [&](int line, int n) { return __ldg(&in[(size_t)n * H + c0 + line]); };
        auto st = [&](int line, int k, float2 v) {
            if (k < N) plane[k * H + c0 + line] = v;
        };
        block_fft<L, +1, true>(nl, ld, st, X, op.tw);
    }
    float2 acc = make_float2(0.0f, 0.0f);
    op.prepare();
    op.acc = &acc;
    const int row0 = blockIdx.x * N;
    for (int r0 = 0; r0 < N; r0 += T::RB) {
        const int nl = min(T::RB, N - r0);
        auto ld = [&](int line, int n) {
            const float2* row = plane + (r0 + line) * H;
            return n <= N ? row[n] : c_conj(row[2 * N - n]);
        };
        auto pre = [&](int line, int k) { return op.pre(row0 + r0 + line, k); };
        auto st = [&](int line, int k, float2 v, float xv) { op.store(row0 + r0 + line, k, v, xv); };
        fft_step1<L, +1, false>(nl, ld, X, op.tw);
        __syncthreads();
        fft_step2_pre<L, +1, false>(nl, pre, st, X);
        __syncthreads();
    }
    if (!op.cg) return;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    const float2 wsum = dw_warp_sum(acc);
    if (lane == 0) s_red[wid] = dw_to_double(wsum);
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = 0.0;
        for (int i = 0; i < nw; ++i) b += s_red[i];
        op.red[blockIdx.x] = b;
        __threadfence();
        const unsigned t = atomicAdd(&op.cg->ticket_a, 1u);
        s_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last || wid != 0) return;
    __threadfence();
    double v = 0.0;
    for (int i = lane; i < (int)gridDim.x; i += 32) v += ((volatile double*)op.red)[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) {
        const double pq = v;
        const double alpha = (op.cg->use_pc ? op.cg->rz : op.cg->rr) / pq;
        op.cg->pq = pq;
        op.cg->alpha = alpha;
        const float2 af = dw_from_double(isfinite(alpha) ? alpha : 0.0);
        op.cg->alpha_f[0] = af.x;
        op.cg->alpha_f[1] = af.y;
        op.cg->ticket_a = 0;
    }
}

template <int L, class Op>
__global__ void __launch_bounds__(kThreads) k_rows_cg(Op op, const CgState* cg) {
    extern __shared__ float2 S[];
    if (cg && cg->done) return;
    constexpr int ROWS = rows_per_block<L>();
    const int r0 = blockIdx.x * ROWS;
    const int nl = min(ROWS, op.n_rows - r0);
    op.prepare();
    auto ld = [&](int line, int n) { return op.load(r0 + line, n); };
    auto post = [&](int line, int n, float2 v) { op.post(r0 + line, n, v); };
    auto st = [&](int line, int k, float2 v) { op.store(r0 + line, k, v); };
    fft_step1_post<L, -1, false>(nl, ld, post, S, op.tw);
    __syncthreads();
    fft_step2<L, -1, false>(nl, st, S);
}

template <int L, int SIGN, class Op>
__global__ void __launch_bounds__(kThreads) k_cols_cg(const Op op, const CgState* cg) {
    extern __shared__ float2 S[];
    if (cg && cg->done) return;
    const int tiles = (op.n_inner + TX<L>() - 1) / TX<L>();
    const int outer = blockIdx.x / tiles;
    const int c0 = (blockIdx.x % tiles) * TX<L>();
    const int nl = min(TX<L>(), op.n_inner - c0);
    auto ld = [&](int line, int n) { return op.load(outer, n, c0 + line); };
    auto st = [&](int line, int k, float2 v) { op.store(outer, k, c0 + line, v); };
    block_fft<L, SIGN, true>(nl, ld, st, S, op.tw);
}

template <int L>
static cudaError_t toeplitz_l(Plan& P, const float* x, float* y, const float2* cg_r, CgState* cg,
                              const float* cg_z) {
    using T = TPlane<L>;
    Workspace& w = P.ws;
    const int N = P.N;
    const size_t smem_plane = sizeof(float2) * T::kSmem;
    const size_t smem_cols = sizeof(float2) * smem_elems<L, true>(TX<L>());
    cudaError_t e;
    // pass 1: per z-plane, rows of x (or p = r + beta p) forward, then y forward
    TRowsFwdOp a{{}, x, cg ? const_cast<float*>(x) : nullptr, cg_r, cg, nullptr, w.tw_2n, N * N, N, cg_z};
    if ((e = cudaFuncSetAttribute(k_toep_plane_fwd<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_plane)))
        return e;
    k_toep_plane_fwd<L><<<N, T::kThreadsP, smem_plane, P.stream>>>(a, w.t2, cg);
    // pass 2: z forward x K-hat x z inverse
    const int n_inner = 2 * N * (N + 1);
    if ((e = cudaFuncSetAttribute(k_toep_z<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_cols))) return e;
    k_toep_z<L><<<(n_inner + TX<L>() - 1) / TX<L>(), kThreads, smem_cols, P.stream>>>(w.t2, w.khat, w.tw_2n, n_inner, N, cg);
    // pass 3: per z-plane, y inverse (keep y < N), rows inverse (Hermitian), crop,
    // scale, + lam x, <x, y>
    const float scale = 1.0f / ((float)L * (float)L * (float)L);
    TRowsInvOp f{nullptr, x, y, w.red_a, cg, w.tw_2n, N * N, N, scale, 0.0f, w.lam, nullptr};
    if ((e = cudaFuncSetAttribute(k_toep_plane_inv<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_plane)))
        return e;
    k_toep_plane_inv<L><<<N, T::kThreadsP, smem_plane, P.stream>>>(f, w.t2);
    P.launches += 3;
    return cudaGetLastError();
}

cudaError_t launch_toeplitz(Plan& P, const float* x, float* y, const float2* cg_r, CgState* cg,
                            const float* cg_z) {
    FIRM_SWITCH_2N(2 * P.N, { return toeplitz_l<LL>(P, x, y, cg_r, cg, cg_z); });
    return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------
// Preconditioner z = F^-1 diag(d) F r on the N^3 grid (PCG; an addition to the
// paper, whose CG is unpreconditioned).  Three launches, like the Toeplitz apply
// without padding: per z-plane real rows forward (half spectrum) and y forward; z
// forward x d x z inverse; per z-plane y inverse and Hermitian rows inverse with
// <r, z> reduced and the flexible beta set on the device.  d already holds the 1/N^3
// of the inverse transform.
// ---------------------------------------------------------------------------
#define FIRM_SWITCH_N(Nval, ...)                                                              \
    switch (Nval) {                                                                          \
        FIRM_CASE_L(16, __VA_ARGS__) FIRM_CASE_L(32, __VA_ARGS__) FIRM_CASE_L(48, __VA_ARGS__)   \
        FIRM_CASE_L(64, __VA_ARGS__) FIRM_CASE_L(80, __VA_ARGS__) FIRM_CASE_L(96, __VA_ARGS__)   \
        FIRM_CASE_L(128, __VA_ARGS__)                                                          \
        default: return cudaErrorInvalidValue;                                               \
    }

struct PRowsFwdOp : NoFinish {
    const float2* r; float2* u; const float2* tw; int n_rows, N;     // r: double-words
    __device__ __forceinline__ float2 load(int row, int n) const {
        const float2 v = __ldg(&r[(size_t)row * N + n]);
        return make_float2(v.x + v.y, 0.0f);
    }
    __device__ __forceinline__ void store(int row, int k, float2 v) const {
        if (k <= N / 2) u[(size_t)row * (N / 2 + 1) + k] = v;
    }
};
struct PColsYOp {
    float2* u; const float2* tw; int n_outer, n_inner, N;
    __device__ __forceinline__ float2 load(int o, int n, int i) const { return u[((size_t)o * N + n) * n_inner + i]; }
    __device__ __forceinline__ void store(int o, int k, int i, float2 v) const { u[((size_t)o * N + k) * n_inner + i] = v; }
};

template <int L>
__global__ void __launch_bounds__(kThreads) k_pc_z(float2* __restrict__ u, const float* __restrict__ d,
                                                   const float2* __restrict__ tw, int n_inner, const CgState* cg) {
    extern __shared__ float2 S[];
    if (cg->done) return;
    const int c0 = blockIdx.x * TX<L>();
    const int nl = min(TX<L>(), n_inner - c0);
    auto ld = [&](int line, int n) { return u[(size_t)n * n_inner + c0 + line]; };
    auto mul = [&](int line, int k) { return __ldg(&d[(size_t)k * n_inner + c0 + line]); };
    auto st = [&](int line, int n, float2 v) { u[(size_t)n * n_inner + c0 + line] = v; };
    block_fft_mul_ifft<L>(nl, ld, mul, st, S, tw);
}

// The preconditioner's x and y transforms, one z-plane per CTA: the plane's N x (N/2+1)
// half spectrum stays in shared memory between the row and the column transforms, so
// the N^3 transform is three passes (plane forward, z with the diagonal, plane
// inverse) instead of five, and each plane is read and written once per direction.
// All rows of the plane are one batch and all columns one batch, with up to 1024
// threads, so a CTA has the whole plane's loads in flight at once (214 KB of shared
// memory at N = 128).
template <int L> __host__ __device__ constexpr int plane_threads() {
    return L * Split<L>::L2 < 1024 ? L * Split<L>::L2 : 1024;
}
template <int L> __host__ __device__ constexpr int pc_plane_smem_elems() {
    constexpr int a = smem_elems<L, false>(L), b = smem_elems<L, true>(L / 2 + 1);
    return L * (L / 2 + 1) + (a > b ? a : b);
}

// u[z][k2][k1] = forward 2D DFT over (x, y) of plane z of r (double-word, summed to FP32)
template <int L>
__global__ void __launch_bounds__(plane_threads<L>()) k_pc_plane_fwd(const float2* __restrict__ r,
                                                                    float2* __restrict__ u,
                                                                    const float2* __restrict__ tw, const CgState* cg) {
    extern __shared__ float2 S[];
    if (cg->done) return;
    constexpr int N = L, H = L / 2 + 1;
    float2* plane = S;                          // [y][k1]
    float2* X = S + N * H;                      // exchange buffer of the transforms
    const float2* rz = r + (size_t)blockIdx.x * N * N;
    auto ld_r = [&](int line, int n) {
        const float2 v = __ldg(&rz[(size_t)line * N + n]);
        return make_float2(v.x + v.y, 0.0f);
    };
    auto st_r = [&](int line, int k, float2 v) {
        if (k <= N / 2) plane[line * H + k] = v;
    };
    block_fft<L, -1, false>(N, ld_r, st_r, X, tw);
    float2* uz = u + (size_t)blockIdx.x * N * H;
    auto ld_c = [&](int line, int n) { return plane[n * H + line]; };
    auto st_c = [&](int line, int k, float2 v) { uz[(size_t)k * H + line] = v; };
    block_fft<L, -1, true>(H, ld_c, st_c, X, tw);
}

// Plane z of the inverse 2D DFT of u (Hermitian along x) is the new z = P r; the CTA
// also reduces <r, z_new> and <r, z_old> for the flexible (Polak-Ribiere)
// beta = (<r,z_new> - <r,z_old>) / <r_old,z_old>, which tolerates the FP32 rounding of
// the preconditioner apply; the last CTA forms beta (sums in CTA order).
template <int L>
__global__ void __launch_bounds__(plane_threads<L>()) k_pc_plane_inv(const float2* __restrict__ u,
                                                                    const float2* __restrict__ r,
                                                                    float* __restrict__ z, double* red, CgState* cg,
                                                                    const float2* __restrict__ tw) {
    extern __shared__ float2 S[];
    __shared__ double s_red[2][32];
    __shared__ bool s_last;
    if (cg->done) return;
    constexpr int N = L, H = L / 2 + 1;
    float2* plane = S;                          // [y][k1]
    float2* X = S + N * H;
    const float2* uz = u + (size_t)blockIdx.x * N * H;
    auto ld_c = [&](int line, int n) { return uz[(size_t)n * H + line]; };
    auto st_c = [&](int line, int k, float2 v) { plane[k * H + line] = v; };
    block_fft<L, +1, true>(H, ld_c, st_c, X, tw);
    float2 acc = make_float2(0.0f, 0.0f), acc_old = make_float2(0.0f, 0.0f);
    const size_t zbase = (size_t)blockIdx.x * N * N;
    auto ld = [&](int line, int n) {
        const float2* row = plane + line * H;
        return n <= N / 2 ? row[n] : c_conj(row[N - n]);
    };
    auto pre = [&](int line, int k) {           // r (double-word) and the previous z
        const size_t i = zbase + (size_t)line * N + k;
        const float2 ri = __ldg(&r[i]);
        return make_float3(ri.x, ri.y, z[i]);
    };
    auto st = [&](int line, int k, float2 v, float3 rzv) {
        const float2 ri = make_float2(rzv.x, rzv.y);
        acc_old = dw_acc_mul(acc_old, ri, rzv.z);
        z[zbase + (size_t)line * N + k] = v.x;
        acc = dw_acc_mul(acc, ri, v.x);
    };
    fft_step1<L, +1, false>(N, ld, X, tw);
    __syncthreads();
    fft_step2_pre<L, +1, false>(N, pre, st, X);
    const float2 w0 = dw_warp_sum(acc), w1 = dw_warp_sum(acc_old);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    if (lane == 0) {
        s_red[0][wid] = dw_to_double(w0);
        s_red[1][wid] = dw_to_double(w1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double b0 = 0.0, b1 = 0.0;
        for (int i = 0; i < nw; ++i) { b0 += s_red[0][i]; b1 += s_red[1][i]; }
        red[2 * blockIdx.x] = b0;
        red[2 * blockIdx.x + 1] = b1;
        __threadfence();
        const unsigned t = atomicAdd(&cg->ticket_c, 1u);
        s_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last || wid != 0) return;
    __threadfence();
    double v0 = 0.0, v1 = 0.0;
    for (int i = lane; i < (int)gridDim.x; i += 32) {
        v0 += ((volatile double*)red)[2 * i];
        v1 += ((volatile double*)red)[2 * i + 1];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v0 += __shfl_xor_sync(0xffffffffu, v0, o);
        v1 += __shfl_xor_sync(0xffffffffu, v1, o);
    }
    if (lane == 0) {
        const double rz_new = v0, rz_old_new_r = v1;
        cg->beta = cg->first ? 0.0 : fmax(0.0, (rz_new - rz_old_new_r) / cg->rz);
        const float2 bf = dw_from_double(cg->beta);
        cg->beta_f[0] = bf.x;
        cg->beta_f[1] = bf.y;
        cg->rz = rz_new;
        cg->first = 0;
        cg->ticket_c = 0;
        if (!(rz_new > 0.0) || !isfinite(rz_new)) {     // P must be positive definite
            if (!(rz_new == 0.0)) cg->status = FIRM_EBREAKDOWN;
            cg->done = 1;
        }
    }
}

template <int L>
static cudaError_t precond_l(Plan& P, const float2* r, float* z, CgState* cg) {
    Workspace& w = P.ws;
    constexpr int N = L, H = L / 2 + 1;
    const size_t smem_plane = sizeof(float2) * pc_plane_smem_elems<L>();
    const size_t smem_cols = sizeof(float2) * smem_elems<L, true>(TX<L>());
    float2* u = w.t1;                       // N x N x (N/2+1) complex
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_pc_plane_fwd<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_plane)))
        return e;
    k_pc_plane_fwd<L><<<N, plane_threads<L>(), smem_plane, P.stream>>>(r, u, w.tw_n, cg);
    const int n_inner = N * H;
    if ((e = cudaFuncSetAttribute(k_pc_z<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_cols))) return e;
    k_pc_z<L><<<(n_inner + TX<L>() - 1) / TX<L>(), kThreads, smem_cols, P.stream>>>(u, w.pc_diag, w.tw_n, n_inner, cg);
    if ((e = cudaFuncSetAttribute(k_pc_plane_inv<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_plane)))
        return e;
    k_pc_plane_inv<L><<<N, plane_threads<L>(), smem_plane, P.stream>>>(u, r, z, w.red_a, cg, w.tw_n);
    P.launches += 3;
    return cudaGetLastError();
}

cudaError_t launch_precond(Plan& P, const float2* r, float* z, CgState* cg) {
    FIRM_SWITCH_N(P.N, { return precond_l<LL>(P, r, z, cg); });
    return cudaErrorInvalidValue;
}

// T. Chan's optimal circulant of the Toeplitz operator (the circulant nearest to it in
// Frobenius norm): column c(m) = sum over n = m (mod N), n in (-N, N)^3, of
// Ker(n) prod_a (N - |n_a|) / N, read from the Ker half box (Ker(-n) = Ker(n)).
__global__ void k_chan_column(const float* __restrict__ ker, float2* __restrict__ c, int N) {
    const long long total = (long long)N * N * N;
    const int N2 = 2 * N;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const int m1 = (int)(i % N), m2 = (int)((i / N) % N), m3 = (int)(i / ((long long)N * N));
        double acc = 0.0;
        for (int a = 0; a < 2; ++a) {
            if (a && m1 == 0) continue;                 // n1 = -N: weight 0
            const int n1 = m1 - a * N;
            const double w1 = (double)(N - abs(n1)) / N;
            for (int b = 0; b < 2; ++b) {
                if (b && m2 == 0) continue;
                const int n2 = m2 - b * N;
                const double w2 = w1 * (double)(N - abs(n2)) / N;
                for (int d = 0; d < 2; ++d) {
                    if (d && m3 == 0) continue;
                    const int n3 = m3 - d * N;
                    const double w3 = w2 * (double)(N - abs(n3)) / N;
                    const size_t idx = n1 >= 0 ? ((size_t)(n3 + N) * N2 + (n2 + N)) * (N + 1) + n1
                                               : ((size_t)(N - n3) * N2 + (N - n2)) * (N + 1) + (-n1);
                    acc += w3 * (double)__ldg(&ker[idx]);
                }
            }
        }
        c[i] = dw_from_double(acc);
    }
}

struct PColsZOp {
    float2* u; const float2* tw; int n_outer, n_inner;
    __device__ __forceinline__ float2 load(int, int n, int i) const { return u[(size_t)n * n_inner + i]; }
    __device__ __forceinline__ void store(int, int k, int i, float2 v) const { u[(size_t)k * n_inner + i] = v; }
};

// d = 1 / ((max(kappa, 0) + floor) N^3), floor = lam_eff (device lam[0]) or 1e-6 kappa(0)
__global__ void k_pc_diag(const float2* __restrict__ u, float* __restrict__ d, long long total, const float* lam_p,
                          float n3) {
    const float lam = lam_p[0];
    const float floor_v = lam > 0.0f ? lam : 1e-6f * fmaxf(u[0].x, 1e-30f);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x)
        d[i] = 1.0f / ((fmaxf(u[i].x, 0.0f) + floor_v) * n3);
}

template <int L>
static cudaError_t chan_spectrum_l(Plan& P) {
    Workspace& w = P.ws;
    constexpr int N = L, H = L / 2 + 1;
    constexpr int ROWS = rows_per_block<L>();
    const size_t smem_rows = sizeof(float2) * smem_elems<L, false>(ROWS);
    const size_t smem_cols = sizeof(float2) * smem_elems<L, true>(TX<L>());
    float2* u = w.t1;
    cudaError_t e;
    k_chan_column<<<P.num_sms * 4, 256, 0, P.stream>>>(w.ker, w.r, N);
    PRowsFwdOp a{{}, w.r, u, w.tw_n, N * N, N};
    if ((e = cudaFuncSetAttribute(k_rows_cg<L, PRowsFwdOp>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_rows)))
        return e;
    k_rows_cg<L, PRowsFwdOp><<<(N * N + ROWS - 1) / ROWS, kThreads, smem_rows, P.stream>>>(a, nullptr);
    PColsYOp b{u, w.tw_n, N, H, N};
    if ((e = cudaFuncSetAttribute(k_cols_cg<L, -1, PColsYOp>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_cols)))
        return e;
    k_cols_cg<L, -1, PColsYOp><<<N * ((H + TX<L>() - 1) / TX<L>()), kThreads, smem_cols, P.stream>>>(b, nullptr);
    PColsZOp c{u, w.tw_n, 1, N * H};
    if ((e = cudaFuncSetAttribute(k_cols_cg<L, -1, PColsZOp>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_cols)))
        return e;
    k_cols_cg<L, -1, PColsZOp><<<(N * H + TX<L>() - 1) / TX<L>(), kThreads, smem_cols, P.stream>>>(c, nullptr);
    P.launches += 4;
    return cudaGetLastError();
}

cudaError_t launch_chan_spectrum(Plan& P) {
    FIRM_SWITCH_N(P.N, { return chan_spectrum_l<LL>(P); });
    return cudaErrorInvalidValue;
}

cudaError_t launch_pc_build_circulant(Plan& P) {
    const long long total = (long long)P.N * P.N * (P.N / 2 + 1);
    const float n3 = (float)P.N * (float)P.N * (float)P.N;
    k_pc_diag<<<P.num_sms * 4, 256, 0, P.stream>>>(P.ws.t1, P.ws.pc_diag, total, P.ws.lam, n3);
    P.launches += 1;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Toeplitz apply without any device allocation.
//
// For callers that cannot call cudaMalloc and have no workspace to lend: for
// example a host application whose allocator already owns all device memory, or a
// real-time path that must not change the device memory footprint while it runs.
// The scratch of the five Toeplitz passes (and the FFT twiddle table) lives in
// the file-scope array below instead; the caller still passes K-hat, x and y.
// ---------------------------------------------------------------------------
constexpr int kStaticMaxN = 64;
constexpr size_t kStaticT1 = (size_t)kStaticMaxN * kStaticMaxN * (kStaticMaxN + 1);       // N x N x (N+1)
constexpr size_t kStaticT2 = (size_t)kStaticMaxN * 2 * kStaticMaxN * (kStaticMaxN + 1);   // N x 2N x (N+1)
// One twiddle slot per transform length L = 2N (32, 64, 96, 128), back to back:
// slot(L) starts at 32 + 64 + ... + (L - 32), 320 float2 in all.
constexpr size_t kStaticTw = 32 + 64 + 96 + 128;
static __device__ __align__(256) float2 g_static_scratch[kStaticT1 + kStaticT2 + kStaticTw];

static constexpr size_t static_tw_slot(int L) {
    return kStaticT1 + kStaticT2 + (size_t)(L / 32 - 1) * (L / 32) / 2 * 32;
}

// Device address of g_static_scratch on the current device.  Host code cannot use
// the symbol itself as a device pointer, so the address is looked up once per
// device, under a lock, and the twiddle slots are written then, with a synchronous
// copy: later calls queue kernels only.
static int static_scratch(float2** out) {
    static std::mutex mu;
    static void* addr[256] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return FIRM_ECUDA;
    if (dev < 0 || dev >= 256) return FIRM_EINVAL;
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess) return FIRM_ECUDA;
        float2 tw_h[kStaticTw];           // on the stack: no heap either
        for (int L = 32; L <= 2 * kStaticMaxN; L += 32) {
            float2* slot = tw_h + (static_tw_slot(L) - kStaticT1 - kStaticT2);
            for (int j = 0; j < L; ++j) {
                const double a = -2.0 * 3.14159265358979323846 * j / L;
                slot[j] = make_float2((float)std::cos(a), (float)std::sin(a));
            }
        }
        float2* tw_d = reinterpret_cast<float2*>(p) + kStaticT1 + kStaticT2;
        if (cudaMemcpy(tw_d, tw_h, sizeof(tw_h), cudaMemcpyHostToDevice) != cudaSuccess) return FIRM_ECUDA;
        addr[dev] = p;
    }
    *out = reinterpret_cast<float2*>(addr[dev]);
    return FIRM_OK;
}

template <int L>
static cudaError_t toeplitz_static_l(float2* scratch, const float* khat, const float* x, float* y, float lam, int N,
                                     cudaStream_t s) {
    float2* t1 = scratch;
    float2* t2 = scratch + kStaticT1;
    const float2* tw = scratch + static_tw_slot(L);
    cudaError_t e;
    constexpr int ROWS = rows_per_block<L>();
    const size_t smem_rows = sizeof(float2) * smem_elems<L, false>(ROWS);
    const size_t smem_cols = sizeof(float2) * smem_elems<L, true>(TX<L>());
    TRowsFwdOp a{{}, x, nullptr, nullptr, nullptr, t1, tw, N * N, N};
    if ((e = cudaFuncSetAttribute(k_rows_cg<L, TRowsFwdOp>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_rows)))
        return e;
    k_rows_cg<L, TRowsFwdOp><<<(N * N + ROWS - 1) / ROWS, kThreads, smem_rows, s>>>(a, nullptr);
    TColsYFwdOp b{t1, t2, tw, N, N + 1, N};
    if ((e = cudaFuncSetAttribute(k_cols_cg<L, -1, TColsYFwdOp>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_cols)))
        return e;
    const int tiles_b = (N + 1 + TX<L>() - 1) / TX<L>();
    k_cols_cg<L, -1, TColsYFwdOp><<<N * tiles_b, kThreads, smem_cols, s>>>(b, nullptr);
    const int n_inner = 2 * N * (N + 1);
    if ((e = cudaFuncSetAttribute(k_toep_z<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_cols))) return e;
    k_toep_z<L><<<(n_inner + TX<L>() - 1) / TX<L>(), kThreads, smem_cols, s>>>(t2, khat, tw, n_inner, N, nullptr);
    TColsYInvOp d{t2, t1, tw, N, N + 1, N};
    if ((e = cudaFuncSetAttribute(k_cols_cg<L, +1, TColsYInvOp>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_cols)))
        return e;
    k_cols_cg<L, +1, TColsYInvOp><<<N * tiles_b, kThreads, smem_cols, s>>>(d, nullptr);
    const float scale = 1.0f / ((float)L * (float)L * (float)L);
    TRowsInvOp f{t1, x, y, nullptr, nullptr, tw, N * N, N, scale, lam, nullptr, nullptr};
    if ((e = cudaFuncSetAttribute(k_toep_rows_inv<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_rows)))
        return e;
    k_toep_rows_inv<L><<<(N * N + ROWS - 1) / ROWS, kThreads, smem_rows, s>>>(f);
    return cudaGetLastError();
}

}  // namespace firm

// True when p is device (or managed) memory of the current device: the static
// array used with it is the current device's copy.
static bool on_device(const void* p) {
    cudaPointerAttributes a;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    return a.type == cudaMemoryTypeDevice && a.device == dev;
}

extern "C" int firm_toeplitz_apply_static(int N, const float* khat, double lam_eff, const float* x, float* y,
                                          void* stream) {
    using namespace firm;
    if (N != 16 && N != 32 && N != 48 && N != 64) return FIRM_EINVAL;   // 64 is the static maximum
    if (!khat || !x || !y || x == y || !(lam_eff >= 0.0)) return FIRM_EINVAL;
    if (!on_device(khat) || !on_device(x) || !on_device(y)) return FIRM_EINVAL;
    float2* scratch = nullptr;
    const int st = static_scratch(&scratch);
    if (st != FIRM_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaErrorInvalidValue;
    switch (2 * N) {
        case 32: e = toeplitz_static_l<32>(scratch, khat, x, y, (float)lam_eff, N, s); break;
        case 64: e = toeplitz_static_l<64>(scratch, khat, x, y, (float)lam_eff, N, s); break;
        case 96: e = toeplitz_static_l<96>(scratch, khat, x, y, (float)lam_eff, N, s); break;
        case 128: e = toeplitz_static_l<128>(scratch, khat, x, y, (float)lam_eff, N, s); break;
        default: break;
    }
    return e == cudaSuccess ? FIRM_OK : FIRM_ECUDA;
}
