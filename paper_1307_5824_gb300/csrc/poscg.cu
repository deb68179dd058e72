// poscg.cu -- the positivity-constrained solve (Section 5 names positivity constraints
// among the prior knowledge FIRM can take in).  Reading: the quadratic of Section 3.3,
// min 1/2 <V, H V> - <A*b, V> over V >= 0 with H = A*A + lam_eff I (plus the damping
// when set), by conjugate gradients on the free voxels with projection and restarts
// (Polyak's method for bound-constrained quadratics):
//
//   restart: free = {V > 0 or r > 0} (r = A*b - H V), p = r on the free voxels;
//   step:    q = H p (the Toeplitz apply), alpha = <r_f, r_f> / <p, q>, and the
//            largest feasible step amax = min over p_i < 0 of V_i / -p_i;
//            amax < alpha: V += amax p, r -= amax q, the blocking voxels set to 0,
//            V projected onto V >= 0, restart;
//            else V += alpha p, r -= alpha q; once ||r_f|| <= rel_tol ||A*b|| restart
//            (a voxel held at 0 whose residual turned positive becomes free); stop
//            when a restart finds the free residual that small; otherwise
//            p = r_f + beta p, beta = <r_f, r_f>_new / <r_f, r_f>.
//
// Vectors are FP32; every inner product, norm and minimum is reduced in FP64 over a
// fixed grid (block partials summed in block order: repeatable), and the host reads
// two small scalar sets per step to take the branch.  Convergence is accepted only on
// the true residual: when the free residual of the FP32 recurrence is small, r is
// recomputed as A*b - H V (one more apply) and the free set re-derived from it; with
// every voxel of positive residual free, a small free residual is then the KKT point.
#include <cuda_runtime.h>

#include <cmath>

#include "firm_internal.h"

namespace firm {

namespace {

constexpr int kT = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_min(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Block reduction of (a: sum, b: sum or min) into part[blockIdx.x], part[nb + blockIdx.x].
template <bool B_MIN>
__device__ __forceinline__ void block_out(double a, double b, double* part) {
    __shared__ double s[2][kT / 32];
    a = warp_sum(a);
    b = B_MIN ? warp_min(b) : warp_sum(b);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        s[0][wid] = a;
        s[1][wid] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double x = s[0][0], y = s[1][0];
        for (int i = 1; i < kT / 32; ++i) {
            x += s[0][i];
            y = B_MIN ? fmin(y, s[1][i]) : y + s[1][i];
        }
        part[blockIdx.x] = x;
        part[gridDim.x + blockIdx.x] = y;
    }
}

__global__ void __launch_bounds__(kT) k_pos_init(float* __restrict__ x, float* __restrict__ r,
                                                 const float* __restrict__ rhs, long long n, double* part) {
    double bb = 0.0;
    for (long long i = (long long)blockIdx.x * kT + threadIdx.x; i < n; i += (long long)gridDim.x * kT) {
        const float b = rhs[i];
        x[i] = 0.0f;
        r[i] = b;
        bb += (double)b * b;
    }
    block_out<false>(bb, 0.0, part);
}

// free set and p = r on it; partial <r_f, r_f>
__global__ void __launch_bounds__(kT) k_pos_restart(const float* __restrict__ x, const float* __restrict__ r,
                                                    float* __restrict__ p, uint8_t* __restrict__ freev, long long n,
                                                    double* part) {
    double rr = 0.0;
    for (long long i = (long long)blockIdx.x * kT + threadIdx.x; i < n; i += (long long)gridDim.x * kT) {
        const float ri = r[i];
        const bool f = x[i] > 0.0f || ri > 0.0f;
        freev[i] = f ? 1 : 0;
        const float pi = f ? ri : 0.0f;
        p[i] = pi;
        rr += (double)pi * pi;
    }
    block_out<false>(rr, 0.0, part);
}

// partial <p, q> and min over p_i < 0 of x_i / -p_i
__global__ void __launch_bounds__(kT) k_pos_pq(const float* __restrict__ x, const float* __restrict__ p,
                                               const float* __restrict__ q, long long n, double* part) {
    double pq = 0.0, am = INFINITY;
    for (long long i = (long long)blockIdx.x * kT + threadIdx.x; i < n; i += (long long)gridDim.x * kT) {
        const float pi = p[i];
        pq += (double)pi * q[i];
        if (pi < 0.0f) am = fmin(am, (double)x[i] / -(double)pi);
    }
    block_out<true>(pq, am, part);
}

// x += step p, r -= step q; on a bound hit the blocking voxels (ratio <= amax) go to 0
// and x is projected; partial <r_f, r_f>
__global__ void __launch_bounds__(kT) k_pos_update(float* __restrict__ x, float* __restrict__ r,
                                                   const float* __restrict__ p, const float* __restrict__ q,
                                                   const uint8_t* __restrict__ freev, long long n, float step,
                                                   int hit, double amax, double* part) {
    double rr = 0.0;
    for (long long i = (long long)blockIdx.x * kT + threadIdx.x; i < n; i += (long long)gridDim.x * kT) {
        const float pi = p[i], xi = x[i];
        float xn = fmaf(step, pi, xi);
        const float rn = fmaf(-step, q[i], r[i]);
        if (hit) {
            if (pi < 0.0f && (double)xi / -(double)pi <= amax) xn = 0.0f;
            xn = fmaxf(xn, 0.0f);
        }
        x[i] = xn;
        r[i] = rn;
        if (freev[i]) rr += (double)rn * rn;
    }
    block_out<false>(rr, 0.0, part);
}

// r = rhs - q (q = H x): the true residual, replacing the FP32 recurrence
__global__ void __launch_bounds__(kT) k_pos_refresh(float* __restrict__ r, const float* __restrict__ q,
                                                    const float* __restrict__ rhs, long long n) {
    for (long long i = (long long)blockIdx.x * kT + threadIdx.x; i < n; i += (long long)gridDim.x * kT)
        r[i] = rhs[i] - q[i];
}

__global__ void __launch_bounds__(kT) k_pos_dir(float* __restrict__ p, const float* __restrict__ r,
                                                const uint8_t* __restrict__ freev, long long n, float beta) {
    for (long long i = (long long)blockIdx.x * kT + threadIdx.x; i < n; i += (long long)gridDim.x * kT)
        p[i] = freev[i] ? fmaf(beta, p[i], r[i]) : 0.0f;
}

// out[0] = sum of part[0..nb), out[1] = sum or min of part[nb..2nb), in block order
template <bool B_MIN>
__global__ void k_pos_fold(const double* __restrict__ part, int nb, double* __restrict__ out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double a = 0.0, b = B_MIN ? INFINITY : 0.0;
    for (int i = 0; i < nb; ++i) {
        a += part[i];
        b = B_MIN ? fmin(b, part[nb + i]) : b + part[nb + i];
    }
    out[0] = a;
    out[1] = b;
}

}  // namespace

// Runs the solve on the plan's A*b and K-hat; x (device, N^3) receives the iterate.
int pos_solve(Plan& P, float* x, int max_iter, double rel_tol, int* iters_out) {
    Workspace& w = P.ws;
    const long long n = (long long)P.N * P.N * P.N;
    int nb = P.num_sms * 4;
    if (nb > kRedSlots / 2) nb = kRedSlots / 2;
    float* r = w.z;
    float* p = w.p;
    float* q = w.q;
    uint8_t* freev = reinterpret_cast<uint8_t*>(w.t1);
    double* part = w.red_a;
    double* sc = w.red_b;        // two finished scalars
    double h[2];
    cudaStream_t s = P.stream;
    auto fold = [&](bool bmin) -> cudaError_t {
        if (bmin) k_pos_fold<true><<<1, 32, 0, s>>>(part, nb, sc);
        else k_pos_fold<false><<<1, 32, 0, s>>>(part, nb, sc);
        cudaError_t e = cudaMemcpyAsync(h, sc, sizeof(h), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        P.launches += 1;
        return e;
    };
#define POS_CK(x)                                 \
    do {                                          \
        if ((x) != cudaSuccess) return FIRM_ECUDA; \
    } while (0)
    k_pos_init<<<nb, kT, 0, s>>>(x, r, w.rhs, n, part);
    P.launches += 1;
    POS_CK(fold(false));
    const double tol = rel_tol * std::sqrt(h[0]);
    int its = 0;
    bool restart = true, fresh = true;      // fresh: r is b - H x computed at this x
    double rz = 0.0;
    int status = FIRM_ENOTCONV;
    for (;;) {
        if (restart) {
            k_pos_restart<<<nb, kT, 0, s>>>(x, r, p, freev, n, part);
            P.launches += 1;
            POS_CK(fold(false));
            rz = h[0];
            if (std::sqrt(rz) <= tol) {
                // every voxel with r > 0 is free, so a small free residual is the KKT
                // point once r is the true residual
                if (fresh) { status = FIRM_OK; break; }
                if (its >= max_iter) break;
                POS_CK(launch_toeplitz(P, x, q, nullptr, nullptr, nullptr));
                ++its;
                k_pos_refresh<<<nb, kT, 0, s>>>(r, q, w.rhs, n);
                P.launches += 1;
                fresh = true;
                continue;                    // restart again on the true residual
            }
            restart = false;
        }
        if (its >= max_iter) break;
        POS_CK(launch_toeplitz(P, p, q, nullptr, nullptr, nullptr));
        ++its;
        k_pos_pq<<<nb, kT, 0, s>>>(x, p, q, n, part);
        P.launches += 1;
        POS_CK(fold(true));
        const double pq = h[0], amax = h[1];
        if (!(pq > 0.0) || !std::isfinite(pq)) { status = FIRM_EBREAKDOWN; break; }
        const double alpha = rz / pq;
        const bool hit = amax < alpha;
        k_pos_update<<<nb, kT, 0, s>>>(x, r, p, q, freev, n, (float)(hit ? amax : alpha), hit ? 1 : 0, amax, part);
        P.launches += 1;
        fresh = false;
        if (hit) {
            restart = true;
            continue;
        }
        POS_CK(fold(false));
        const double rz_new = h[0];
        if (std::sqrt(rz_new) <= tol) {      // the free subspace is solved: check on restart
            restart = true;
            continue;
        }
        k_pos_dir<<<nb, kT, 0, s>>>(p, r, freev, n, (float)(rz_new / rz));
        P.launches += 1;
        rz = rz_new;
    }
#undef POS_CK
    if (iters_out) *iters_out = its;
    if (cudaGetLastError() != cudaSuccess) return FIRM_ECUDA;
    return status;
}

}  // namespace firm
