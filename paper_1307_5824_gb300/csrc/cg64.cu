// cg64.cu -- the FP64 CG mode (FIRM_FLAG_FP64_CG): CG of Section 3.3 with FP64
// vectors and an FP64 Toeplitz apply (eq. property through the 2N circulant of
// Section 3.2, K-hat recomputed in FP64 from the Ker half box).  For N in {16, 32, 64}:
// plain radix-2 FFTs in shared memory, one line per L/2 threads, no pruning.  Its
// purpose is precision, not speed: a long fixed-count CG iterate is sensitive to the
// ~1e-7 rounding of FP32 FFTs, and this mode removes that rounding from the solve
// (Ker and A*b still come from the FP32 NUFFT).
#include <cuda_runtime.h>

#include "firm_internal.h"

namespace firm {

namespace {

constexpr int kT = 256;

__device__ __forceinline__ double2 cmul64(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// Sum over the block (valid in thread 0).
__device__ __forceinline__ double blk_sum(double v, double* sw) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = v;
    __syncthreads();
    double b = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) b += sw[i];
    return b;
}

// Last block to finish gets true (all threads); then the partials in block order.
__device__ __forceinline__ bool last_blk(unsigned int* ticket, bool* s_last) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        *s_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (*s_last) __threadfence();
    return *s_last;
}

__device__ __forceinline__ double fin_sum(const double* red, double* s_fin) {
    double v = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) v += ((volatile const double*)red)[i];
    s_fin[threadIdx.x] = v;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) s_fin[threadIdx.x] += s_fin[threadIdx.x + s];
        __syncthreads();
    }
    return s_fin[0];
}

// Lines of length L through the (2N)^3 array: element k of line l is
// data[(l / inner) * s_outer + (l % inner) * s_inner + k * s_elem].
template <int L>
__global__ void __launch_bounds__(kT) k_fft64(double2* __restrict__ data, int n_lines, int inner, long long s_outer,
                                               long long s_inner, long long s_elem, const double2* __restrict__ tw,
                                               int sign, const CgState* cg) {
    constexpr int TPL = L / 2;
    constexpr int LPB = kT / TPL;
    constexpr int LOG = L == 32 ? 5 : L == 64 ? 6 : 7;
    static_assert(L == 32 || L == 64 || L == 128, "FP64 mode: 2N in {32, 64, 128}");
    __shared__ double2 s[LPB][L];
    if (cg && cg->done) return;
    const int lt = threadIdx.x / TPL, t = threadIdx.x % TPL;
    const int line = blockIdx.x * LPB + lt;
    const bool active = line < n_lines;
    const long long base = active ? (long long)(line / inner) * s_outer + (long long)(line % inner) * s_inner : 0;
    if (active)
        for (int k = t; k < L; k += TPL) s[lt][__brev((unsigned)k) >> (32 - LOG)] = data[base + k * s_elem];
    __syncthreads();
    for (int half = 1; half < L; half <<= 1) {
        if (active) {
            const int j = t % half, grp = t / half;
            const int i0 = grp * 2 * half + j, i1 = i0 + half;
            double2 w = tw[j * (L / (2 * half))];
            if (sign > 0) w.y = -w.y;
            const double2 a = s[lt][i0], bw = cmul64(s[lt][i1], w);
            s[lt][i0] = make_double2(a.x + bw.x, a.y + bw.y);
            s[lt][i1] = make_double2(a.x - bw.x, a.y - bw.y);
        }
        __syncthreads();
    }
    if (active)
        for (int k = t; k < L; k += TPL) data[base + k * s_elem] = s[lt][k];
}

// First column of the circulant (reading 2: 0-based lags, lag-N planes zero) from the
// Ker half box [n3+N][n2+N][n1], n1 in [0, N], using Ker(-n) = Ker(n).
__global__ void k_circ64(const float* __restrict__ ker, double2* __restrict__ C, int N) {
    const int L = 2 * N;
    const long long total = (long long)L * L * L;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const int i1 = (int)(i % L), i2 = (int)((i / L) % L), i3 = (int)(i / ((long long)L * L));
        double v = 0.0;
        if (i1 != N && i2 != N && i3 != N) {
            int d1 = i1 < N ? i1 : i1 - L, d2 = i2 < N ? i2 : i2 - L, d3 = i3 < N ? i3 : i3 - L;
            if (d1 < 0) { d1 = -d1; d2 = -d2; d3 = -d3; }
            v = (double)ker[((size_t)(d3 + N) * L + (d2 + N)) * (N + 1) + d1];
        }
        C[i] = make_double2(v, 0.0);
    }
}

__global__ void k_real64(const double2* __restrict__ C, double* __restrict__ kh, long long total) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x)
        kh[i] = C[i].x;
}

// C = p zero-padded to (2N)^3 (p at indices [0, N)^3)
__global__ void k_pad64(const double* __restrict__ p, double2* __restrict__ C, int N, const CgState* cg) {
    if (cg->done) return;
    const int L = 2 * N;
    const long long total = (long long)L * L * L;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const int i1 = (int)(i % L), i2 = (int)((i / L) % L), i3 = (int)(i / ((long long)L * L));
        const double v = (i1 < N && i2 < N && i3 < N) ? p[((size_t)i3 * N + i2) * N + i1] : 0.0;
        C[i] = make_double2(v, 0.0);
    }
}

__global__ void k_mul64(double2* __restrict__ C, const double* __restrict__ kh, long long total, const CgState* cg) {
    if (cg->done) return;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const double k = kh[i];
        C[i] = make_double2(C[i].x * k, C[i].y * k);
    }
}

// q = crop(C) / (2N)^3 + lam_eff p;  <p, q> -> pq, alpha = rr / pq
__global__ void __launch_bounds__(kT) k_crop64(const double2* __restrict__ C, const double* __restrict__ p,
                                                double* __restrict__ q, int N, const float* __restrict__ lam,
                                                CgState* cg, double* red) {
    __shared__ double sw[kT / 32];
    __shared__ double s_fin[kT];
    __shared__ bool s_last;
    if (cg->done) return;
    const int L = 2 * N;
    const double scale = 1.0 / ((double)L * L * L), lv = (double)lam[0];
    const long long n = (long long)N * N * N;
    double acc = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int i1 = (int)(i % N), i2 = (int)((i / N) % N), i3 = (int)(i / ((long long)N * N));
        const double pv = p[i];
        const double qv = C[((size_t)i3 * L + i2) * L + i1].x * scale + lv * pv;
        q[i] = qv;
        acc += pv * qv;
    }
    const double b = blk_sum(acc, sw);
    if (threadIdx.x == 0) red[blockIdx.x] = b;
    if (!last_blk(&cg->ticket_a, &s_last)) return;
    const double pq = fin_sum(red, s_fin);
    if (threadIdx.x == 0) {
        cg->pq = pq;
        cg->alpha = cg->rr / pq;
        cg->ticket_a = 0;
    }
}

__global__ void __launch_bounds__(kT) k_cg64_init(const float* __restrict__ rhs, double* __restrict__ x,
                                                   double* __restrict__ r, double* __restrict__ p, long long n,
                                                   CgState* cg, double* red, double* hist, int max_iter,
                                                   double rel_tol) {
    __shared__ double sw[kT / 32];
    __shared__ double s_fin[kT];
    __shared__ bool s_last;
    double acc = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double b = (double)rhs[i];
        x[i] = 0.0;
        r[i] = b;
        p[i] = b;
        acc += b * b;
    }
    const double bs = blk_sum(acc, sw);
    if (threadIdx.x == 0) red[blockIdx.x] = bs;
    if (!last_blk(&cg->ticket_b, &s_last)) return;
    const double rr = fin_sum(red, s_fin);
    if (threadIdx.x == 0) {
        cg->rr = rr;
        cg->pq = 0.0;
        cg->beta = 0.0;
        cg->alpha = 0.0;
        cg->bnorm = sqrt(rr);
        cg->tol = rel_tol > 0.0 ? rel_tol * sqrt(rr) : 0.0;
        cg->it = 0;
        cg->max_iter = max_iter;
        cg->status = FIRM_OK;
        cg->rz = 0.0;
        cg->use_pc = 0;
        cg->first = 1;
        cg->done = (rr == 0.0 || max_iter <= 0 || (cg->tol > 0.0 && sqrt(rr) <= cg->tol)) ? 1 : 0;
        if (!(rr == rr) || rr > 1.7e308) { cg->done = 1; cg->status = FIRM_EBREAKDOWN; }
        hist[0] = sqrt(rr);
        cg->ticket_b = 0;
    }
}

// p = r + beta p
__global__ void k_cg64_p(double* __restrict__ p, const double* __restrict__ r, long long n, const CgState* cg) {
    if (cg->done) return;
    const double beta = cg->beta;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        p[i] = fma(beta, p[i], r[i]);
}

__global__ void __launch_bounds__(kT) k_cg64_update(double* __restrict__ x, double* __restrict__ r,
                                                     const double* __restrict__ p, const double* __restrict__ q,
                                                     long long n, CgState* cg, double* red, double* hist) {
    __shared__ double sw[kT / 32];
    __shared__ double s_fin[kT];
    __shared__ bool s_last;
    if (cg->done) return;
    const double pq = cg->pq, rr = cg->rr, alpha = cg->alpha;
    const bool ok = pq > 0.0 && isfinite(alpha);
    double acc = 0.0;
    if (ok) {
        for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
            x[i] = fma(alpha, p[i], x[i]);
            const double rv = fma(-alpha, q[i], r[i]);
            r[i] = rv;
            acc += rv * rv;
        }
    }
    const double bs = blk_sum(acc, sw);
    if (threadIdx.x == 0) red[blockIdx.x] = bs;
    if (!last_blk(&cg->ticket_b, &s_last)) return;
    const double rr_new = fin_sum(red, s_fin);
    if (threadIdx.x == 0) {
        cg->ticket_b = 0;
        if (!ok || !(rr_new == rr_new)) {
            cg->status = FIRM_EBREAKDOWN;
            cg->done = 1;
        } else {
            const int it = cg->it + 1;
            cg->it = it;
            hist[it < kMaxHist ? it : kMaxHist - 1] = sqrt(rr_new);
            cg->beta = rr_new / rr;
            cg->rr = rr_new;
            if (cg->tol > 0.0 && sqrt(rr_new) <= cg->tol) cg->done = 1;
            if (it >= cg->max_iter) cg->done = 1;
        }
    }
}

__global__ void k_d2f(const double* __restrict__ a, float* __restrict__ b, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        b[i] = (float)a[i];
}

int blocks_for(long long n, const Plan& P) {
    long long b = (n + kT - 1) / kT;
    const long long cap = (long long)P.num_sms * 8;
    return (int)(b < cap ? (b > 0 ? b : 1) : cap);
}

template <int L>
cudaError_t fft3_64(Plan& P, double2* C, int sign, const CgState* cg) {
    constexpr int LPB = kT / (L / 2);
    const int lines = L * L;
    const int grid = (lines + LPB - 1) / LPB;
    const long long L2 = (long long)L * L;
    const double2* tw = P.ws.tw64;
    // x (i1): line l = (i3, i2) -> base l * L;  y (i2): base i3 * L^2 + i1;  z (i3): base l
    k_fft64<L><<<grid, kT, 0, P.stream>>>(C, lines, 1, L, 0, 1, tw, sign, cg);
    k_fft64<L><<<grid, kT, 0, P.stream>>>(C, lines, L, L2, 1, L, tw, sign, cg);
    k_fft64<L><<<grid, kT, 0, P.stream>>>(C, lines, lines, 0, 1, L2, tw, sign, cg);
    P.launches += 3;
    return cudaGetLastError();
}

cudaError_t fft3_64_any(Plan& P, double2* C, int sign, const CgState* cg) {
    switch (2 * P.N) {
        case 32: return fft3_64<32>(P, C, sign, cg);
        case 64: return fft3_64<64>(P, C, sign, cg);
        case 128: return fft3_64<128>(P, C, sign, cg);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_khat64(Plan& P) {
    Workspace& w = P.ws;
    const long long total = 8LL * P.N * P.N * P.N;
    k_circ64<<<blocks_for(total, P), kT, 0, P.stream>>>(w.ker, w.c64, P.N);
    cudaError_t e = fft3_64_any(P, w.c64, -1, nullptr);
    if (e != cudaSuccess) return e;
    k_real64<<<blocks_for(total, P), kT, 0, P.stream>>>(w.c64, w.khat64, total);
    P.launches += 2;
    return cudaGetLastError();
}

cudaError_t launch_cg64(Plan& P, const float* rhs, int max_iter, double rel_tol, int first_iter, int n_iter) {
    Workspace& w = P.ws;
    const long long n = (long long)P.N * P.N * P.N, total = 8 * n;
    const int gb = blocks_for(n, P) < kRedSlots ? blocks_for(n, P) : kRedSlots;
    if (first_iter == 0) {
        cudaError_t e = cudaMemsetAsync(w.cg, 0, sizeof(CgState), P.stream);   // tickets start at zero
        if (e != cudaSuccess) return e;
        k_cg64_init<<<gb, kT, 0, P.stream>>>(rhs, w.x64, w.r64, w.p64, n, w.cg, w.red_b, w.hist, max_iter, rel_tol);
        P.launches += 1;
    }
    for (int k = 0; k < n_iter; ++k) {
        k_cg64_p<<<blocks_for(n, P), kT, 0, P.stream>>>(w.p64, w.r64, n, w.cg);
        k_pad64<<<blocks_for(total, P), kT, 0, P.stream>>>(w.p64, w.c64, P.N, w.cg);
        cudaError_t e = fft3_64_any(P, w.c64, -1, w.cg);
        if (e != cudaSuccess) return e;
        k_mul64<<<blocks_for(total, P), kT, 0, P.stream>>>(w.c64, w.khat64, total, w.cg);
        e = fft3_64_any(P, w.c64, +1, w.cg);
        if (e != cudaSuccess) return e;
        k_crop64<<<gb, kT, 0, P.stream>>>(w.c64, w.p64, w.q64, P.N, w.lam, w.cg, w.red_a);
        k_cg64_update<<<gb, kT, 0, P.stream>>>(w.x64, w.r64, w.p64, w.q64, n, w.cg, w.red_b, w.hist);
        P.launches += 5;
    }
    return cudaGetLastError();
}

cudaError_t launch_cg64_result(Plan& P) {
    const long long n = (long long)P.N * P.N * P.N;
    k_d2f<<<blocks_for(n, P), kT, 0, P.stream>>>(P.ws.x64, P.ws.x, n);
    P.launches += 1;
    return cudaGetLastError();
}

}  // namespace firm
