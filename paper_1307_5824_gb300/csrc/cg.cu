// cg.cu -- conjugate gradients of FIRM step 4 (Section 3.3) on
// (A*A + lam_eff I) x = A*b from x = 0, vectors FP32, scalars FP64.
//
// One iteration is the Toeplitz apply (whose first pass forms p = r + beta p and
// whose last pass reduces <p, q>) followed by k_cg_update below.  Reductions are
// two-level and deterministic: every block writes one FP64 partial, the last block
// to finish (ticket counter) sums the partials in block order.  All scalar logic
// (alpha, beta, the stop test, breakdown) runs on the device; a kernel that finds
// the `done` flag set returns at once, so batches of iterations can be queued
// without reading anything back.  Scalars are FP64; the residual vector and the
// per-thread parts of the inner products are double-words (dw.cuh), so no kernel
// does FP64 arithmetic per element.
#include <cuda_runtime.h>

#include "dw.cuh"
#include "firm_internal.h"

namespace firm {

constexpr int kCgThreads = 256;

__device__ __forceinline__ double block_sum(float2 v2, double* s_warp) {
    const double v = dw_to_double(dw_warp_sum(v2));
    if ((threadIdx.x & 31) == 0) s_warp[threadIdx.x >> 5] = v;
    __syncthreads();
    double b = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) b += s_warp[i];
    return b;   // valid in thread 0
}

// Sum of the gridDim.x partials in a fixed order (thread-strided, then a tree).
__device__ __forceinline__ double final_sum(const double* red, double* s_fin) {
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

// Returns true in every thread of the last block to finish.
__device__ __forceinline__ bool last_block(unsigned int* ticket, bool* s_last) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned t = atomicAdd(ticket, 1u);
        *s_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (*s_last) __threadfence();
    return *s_last;
}

__global__ void __launch_bounds__(kCgThreads) k_cg_init(const float* __restrict__ rhs, float* __restrict__ x,
                                                        float2* __restrict__ r, float* __restrict__ p, size_t n,
                                                        CgState* cg, double* red, double* hist, int max_iter,
                                                        double rel_tol, int use_pc) {
    __shared__ double s_warp[kCgThreads / 32];
    __shared__ double s_fin[kCgThreads];
    __shared__ bool s_last;
    float2 acc = make_float2(0.0f, 0.0f);
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float b = rhs[i];
        x[i] = 0.0f;
        r[i] = make_float2(b, 0.0f);
        p[i] = b;
        acc = dw_acc_prod(acc, b, b);
    }
    const double bs = block_sum(acc, s_warp);
    if (threadIdx.x == 0) red[blockIdx.x] = bs;
    if (!last_block(&cg->ticket_b, &s_last)) return;
    const double rr = final_sum(red, s_fin);
    if (threadIdx.x == 0) {
        cg->rr = rr;
        cg->pq = 0.0;
        cg->beta = 0.0;
        cg->beta_f[0] = cg->beta_f[1] = 0.0f;
        cg->alpha = 0.0;
        cg->alpha_f[0] = cg->alpha_f[1] = 0.0f;
        cg->bnorm = sqrt(rr);
        cg->tol = rel_tol > 0.0 ? rel_tol * sqrt(rr) : 0.0;
        cg->it = 0;
        cg->max_iter = max_iter;
        cg->status = FIRM_OK;
        cg->rz = 0.0;
        cg->use_pc = use_pc;
        cg->first = 1;
        cg->done = (rr == 0.0 || max_iter <= 0 || (cg->tol > 0.0 && sqrt(rr) <= cg->tol)) ? 1 : 0;
        if (!(rr == rr) || rr > 1.7e308) { cg->done = 1; cg->status = FIRM_EBREAKDOWN; }
        hist[0] = sqrt(rr);
        cg->ticket_b = 0;
    }
}

// x += alpha p, r -= alpha q (alpha from the Toeplitz apply's last block), then
// <r, r> and the next beta.
__global__ void __launch_bounds__(kCgThreads) k_cg_update(float* __restrict__ x, float2* __restrict__ r,
                                                          const float* __restrict__ p, const float* __restrict__ q,
                                                          size_t n4, CgState* cg, double* red, double* hist) {
    __shared__ double s_warp[kCgThreads / 32];
    __shared__ double s_fin[kCgThreads];
    __shared__ bool s_last;
    if (cg->done) return;
    const double pq = cg->pq, rr = cg->rr;
    const bool ok = pq > 0.0 && isfinite(cg->alpha);
    float2 acc = make_float2(0.0f, 0.0f);
    if (ok) {
        const float2 a = make_float2(cg->alpha_f[0], cg->alpha_f[1]);
        float4* x4 = reinterpret_cast<float4*>(x);
        float4* r4 = reinterpret_cast<float4*>(r);
        const float4* p4 = reinterpret_cast<const float4*>(p);
        const float4* q4 = reinterpret_cast<const float4*>(q);
        for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (size_t)gridDim.x * blockDim.x) {
            float4 xv = x4[i];
            const float4 pv = p4[i], qv = q4[i];
            const float4 ra = r4[2 * i], rb = r4[2 * i + 1];      // (hi, lo) of 4 elements
            xv.x = fmaf(a.x, pv.x, xv.x); xv.y = fmaf(a.x, pv.y, xv.y);
            xv.z = fmaf(a.x, pv.z, xv.z); xv.w = fmaf(a.x, pv.w, xv.w);
            const float2 r0 = dw_sub_mul(make_float2(ra.x, ra.y), a, qv.x);
            const float2 r1 = dw_sub_mul(make_float2(ra.z, ra.w), a, qv.y);
            const float2 r2 = dw_sub_mul(make_float2(rb.x, rb.y), a, qv.z);
            const float2 r3 = dw_sub_mul(make_float2(rb.z, rb.w), a, qv.w);
            x4[i] = xv;
            r4[2 * i] = make_float4(r0.x, r0.y, r1.x, r1.y);
            r4[2 * i + 1] = make_float4(r2.x, r2.y, r3.x, r3.y);
            acc = dw_acc_sq(acc, r0);
            acc = dw_acc_sq(acc, r1);
            acc = dw_acc_sq(acc, r2);
            acc = dw_acc_sq(acc, r3);
        }
    }
    const double bs = block_sum(acc, s_warp);
    if (threadIdx.x == 0) red[blockIdx.x] = bs;
    if (!last_block(&cg->ticket_b, &s_last)) return;
    const double rr_new = final_sum(red, s_fin);
    if (threadIdx.x == 0) {
        cg->ticket_b = 0;
        if (!ok || !(rr_new == rr_new)) {
            cg->status = FIRM_EBREAKDOWN;
            cg->done = 1;
        } else {
            const int it = cg->it + 1;
            cg->it = it;
            hist[it < kMaxHist ? it : kMaxHist - 1] = sqrt(rr_new);
            if (!cg->use_pc) {                        // else set by the preconditioner pass
                const double beta = rr_new / rr;
                cg->beta = beta;
                const float2 bf = dw_from_double(beta);
                cg->beta_f[0] = bf.x;
                cg->beta_f[1] = bf.y;
            }
            cg->rr = rr_new;
            if (cg->tol > 0.0 && sqrt(rr_new) <= cg->tol) cg->done = 1;
            if (it >= cg->max_iter) cg->done = 1;
        }
    }
}

// Four blocks per SM: enough loads in flight, and few enough blocks that the
// last-block ticket (one atomic per block on one address) stays cheap.
static int cg_blocks(const Plan& P) {
    const int b = P.num_sms * 4;
    return b < kRedSlots ? b : kRedSlots;
}

cudaError_t launch_cg_init(Plan& P, const float* rhs, int max_iter, double rel_tol, bool use_pc) {
    Workspace& w = P.ws;
    const size_t n = (size_t)P.N * P.N * P.N;
    cudaError_t e = cudaMemsetAsync(w.cg, 0, sizeof(CgState), P.stream);
    if (e != cudaSuccess) return e;
    k_cg_init<<<cg_blocks(P), kCgThreads, 0, P.stream>>>(rhs, w.x, w.r, w.p, n, w.cg, w.red_b, w.hist, max_iter,
                                                         rel_tol, use_pc ? 1 : 0);
    P.launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_cg_update(Plan& P) {
    Workspace& w = P.ws;
    const size_t n4 = (size_t)P.N * P.N * P.N / 4;
    k_cg_update<<<cg_blocks(P), kCgThreads, 0, P.stream>>>(w.x, w.r, w.p, w.q, n4, w.cg, w.red_b, w.hist);
    P.launches += 1;
    return cudaGetLastError();
}

}  // namespace firm
