// fft.cuh -- hand-written FFT building blocks for sm_103a.
//
// Register DFTs of small radix (2, 3, 4, 5, 8 written out; composite sizes by a
// two-level Cooley-Tukey split), and a CTA-level "four-step" transform of length
// L = L1 * L2 over a tile of lines: step 1 runs an L1-point DFT per (line, n2) in
// registers, twiddles by W_L^{n2 k1} and exchanges through shared memory; step 2
// runs an L2-point DFT per (line, k1).  One shared-memory exchange per transform.
//
// Index algebra (forward, W = exp(SIGN 2 pi i / L)):
//   x[n], n = L2 n1 + n2;  X[k], k = k1 + L1 k2
//   X[k1 + L1 k2] = sum_{n2} W_{L2}^{n2 k2} W_L^{n2 k1} sum_{n1} W_{L1}^{n1 k1} x[L2 n1 + n2]
// The same split read backwards (input k = k1 + L1 k2 owned per k1, output
// n = na + L2 nb) gives the transform that starts from the step-2 layout, which the
// Toeplitz pass uses to go forward, multiply and back without an extra exchange.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace firm {

__device__ __forceinline__ float2 c_add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 c_sub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 c_mul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 c_conj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 c_scale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// a * (SIGN * i)
template <int SIGN> __device__ __forceinline__ float2 c_mul_i(float2 a) {
    return SIGN > 0 ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}
// a * w where w is a forward twiddle exp(-2 pi i j / R); SIGN > 0 uses conj(w)
template <int SIGN> __device__ __forceinline__ float2 c_mul_tw(float2 a, float2 w) {
    return c_mul(a, SIGN > 0 ? c_conj(w) : w);
}

// ---------------------------------------------------------------------------
// Constant twiddles exp(-2 pi i j / R) for the composite register DFT sizes.
// Filled from the host (double precision) by firm_fft_init_constants().
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int tw_offset(int R) {
    return R == 4 ? 0 : R == 6 ? 4 : R == 8 ? 10 : R == 10 ? 18 : R == 12 ? 28 : R == 16 ? 40
         : R == 20 ? 56 : R == 24 ? 76 : R == 32 ? 100 : -1;
}
constexpr int kTwConstTotal = 132;
static __constant__ float2 c_tw[kTwConstTotal];   // one copy per translation unit

template <int R> __device__ __forceinline__ float2 tw_c(int j) { return c_tw[tw_offset(R) + j]; }

// ---------------------------------------------------------------------------
// Register DFTs, in place, natural order.  SIGN = -1 forward, +1 inverse (unnormalised).
// ---------------------------------------------------------------------------
template <int R, int SIGN> struct Dft;

template <int SIGN> struct Dft<1, SIGN> {
    __device__ __forceinline__ static void run(float2*) {}
};
template <int SIGN> struct Dft<2, SIGN> {
    __device__ __forceinline__ static void run(float2* x) {
        float2 a = x[0], b = x[1];
        x[0] = c_add(a, b);
        x[1] = c_sub(a, b);
    }
};
template <int SIGN> struct Dft<3, SIGN> {
    __device__ __forceinline__ static void run(float2* x) {
        const float c = -0.5f, s = 0.86602540378443864676f;   // cos, sin of 2 pi / 3
        float2 t = c_add(x[1], x[2]), d = c_sub(x[1], x[2]);
        float2 m = make_float2(fmaf(c, t.x, x[0].x), fmaf(c, t.y, x[0].y));
        float2 r = c_mul_i<SIGN>(c_scale(d, s));
        x[0] = c_add(x[0], t);
        x[1] = c_add(m, r);
        x[2] = c_sub(m, r);
    }
};
template <int SIGN> struct Dft<4, SIGN> {
    __device__ __forceinline__ static void run(float2* x) {
        float2 a0 = c_add(x[0], x[2]), a1 = c_sub(x[0], x[2]);
        float2 b0 = c_add(x[1], x[3]), b1 = c_mul_i<SIGN>(c_sub(x[1], x[3]));
        x[0] = c_add(a0, b0);
        x[2] = c_sub(a0, b0);
        x[1] = c_add(a1, b1);
        x[3] = c_sub(a1, b1);
    }
};
template <int SIGN> struct Dft<5, SIGN> {
    __device__ __forceinline__ static void run(float2* x) {
        // cos and sin of 2 pi / 5 and 4 pi / 5
        const float c1 = 0.30901699437494742410f, c2 = -0.80901699437494742410f;
        const float s1 = 0.95105651629515357212f, s2 = 0.58778525229247312917f;
        float2 t1 = c_add(x[1], x[4]), t2 = c_add(x[2], x[3]);
        float2 d1 = c_sub(x[1], x[4]), d2 = c_sub(x[2], x[3]);
        float2 m1 = make_float2(x[0].x + c1 * t1.x + c2 * t2.x, x[0].y + c1 * t1.y + c2 * t2.y);
        float2 m2 = make_float2(x[0].x + c2 * t1.x + c1 * t2.x, x[0].y + c2 * t1.y + c1 * t2.y);
        float2 r1 = c_mul_i<SIGN>(make_float2(s1 * d1.x + s2 * d2.x, s1 * d1.y + s2 * d2.y));
        float2 r2 = c_mul_i<SIGN>(make_float2(s2 * d1.x - s1 * d2.x, s2 * d1.y - s1 * d2.y));
        x[0] = c_add(x[0], c_add(t1, t2));
        x[1] = c_add(m1, r1);
        x[4] = c_sub(m1, r1);
        x[2] = c_add(m2, r2);
        x[3] = c_sub(m2, r2);
    }
};
template <int SIGN> struct Dft<8, SIGN> {
    __device__ __forceinline__ static void run(float2* x) {
        const float h = 0.70710678118654752440f;
        float2 a[4] = {x[0], x[2], x[4], x[6]};
        float2 b[4] = {x[1], x[3], x[5], x[7]};
        Dft<4, SIGN>::run(a);
        Dft<4, SIGN>::run(b);
        // twiddles exp(SIGN 2 pi i k / 8), k = 0..3
        float2 b1 = make_float2(h * (b[1].x - SIGN * b[1].y), h * (b[1].y + SIGN * b[1].x));
        float2 b2 = c_mul_i<SIGN>(b[2]);
        float2 b3 = make_float2(h * (-b[3].x - SIGN * b[3].y), h * (-b[3].y + SIGN * b[3].x));
        x[0] = c_add(a[0], b[0]);
        x[4] = c_sub(a[0], b[0]);
        x[1] = c_add(a[1], b1);
        x[5] = c_sub(a[1], b1);
        x[2] = c_add(a[2], b2);
        x[6] = c_sub(a[2], b2);
        x[3] = c_add(a[3], b3);
        x[7] = c_sub(a[3], b3);
    }
};

// Composite R = A * B in registers.
template <int A, int B, int SIGN> struct DftComp {
    __device__ __forceinline__ static void run(float2* x) {
        constexpr int R = A * B;
        float2 u[B][A];
#pragma unroll
        for (int n2 = 0; n2 < B; ++n2) {
            float2 t[A];
#pragma unroll
            for (int n1 = 0; n1 < A; ++n1) t[n1] = x[B * n1 + n2];
            Dft<A, SIGN>::run(t);
#pragma unroll
            for (int k1 = 0; k1 < A; ++k1)
                u[n2][k1] = (n2 * k1 == 0) ? t[k1] : c_mul_tw<SIGN>(t[k1], tw_c<R>((n2 * k1) % R));
        }
#pragma unroll
        for (int k1 = 0; k1 < A; ++k1) {
            float2 t[B];
#pragma unroll
            for (int n2 = 0; n2 < B; ++n2) t[n2] = u[n2][k1];
            Dft<B, SIGN>::run(t);
#pragma unroll
            for (int k2 = 0; k2 < B; ++k2) x[k1 + A * k2] = t[k2];
        }
    }
};
template <int SIGN> struct Dft<6, SIGN> : DftComp<2, 3, SIGN> {};
template <int SIGN> struct Dft<10, SIGN> : DftComp<2, 5, SIGN> {};
template <int SIGN> struct Dft<12, SIGN> : DftComp<4, 3, SIGN> {};
template <int SIGN> struct Dft<16, SIGN> : DftComp<4, 4, SIGN> {};
template <int SIGN> struct Dft<20, SIGN> : DftComp<4, 5, SIGN> {};
template <int SIGN> struct Dft<24, SIGN> : DftComp<8, 3, SIGN> {};
template <int SIGN> struct Dft<32, SIGN> : DftComp<8, 4, SIGN> {};

// ---------------------------------------------------------------------------
// Factorisation L = L1 * L2 used for each supported transform length.
// ---------------------------------------------------------------------------
template <int L> struct Split;
template <> struct Split<16> { static constexpr int L1 = 4, L2 = 4; };
template <> struct Split<32> { static constexpr int L1 = 8, L2 = 4; };
template <> struct Split<48> { static constexpr int L1 = 12, L2 = 4; };
template <> struct Split<64> { static constexpr int L1 = 8, L2 = 8; };
template <> struct Split<80> { static constexpr int L1 = 10, L2 = 8; };
template <> struct Split<96> { static constexpr int L1 = 12, L2 = 8; };
template <> struct Split<128> { static constexpr int L1 = 16, L2 = 8; };
template <> struct Split<160> { static constexpr int L1 = 20, L2 = 8; };
template <> struct Split<192> { static constexpr int L1 = 24, L2 = 8; };
template <> struct Split<256> { static constexpr int L1 = 16, L2 = 16; };
template <> struct Split<320> { static constexpr int L1 = 20, L2 = 16; };
template <> struct Split<384> { static constexpr int L1 = 24, L2 = 16; };
template <> struct Split<512> { static constexpr int L1 = 32, L2 = 16; };

// ---------------------------------------------------------------------------
// Block-level transforms.  `tw` is the table exp(-2 pi i j / L), j < L.
//
// block_fft: length-L transforms of nl lines with all threads of the block.
//   ld(line, n) -> float2 input sample n of a line (the functor does any zero padding);
//   st(line, k, v) receives output k.  LINE_FAST selects the thread order: line index
//   fastest (lines adjacent in memory, transform axis strided) or sample index fastest
//   (each line contiguous).  S must hold smem_elems<L, LINE_FAST>(nl) float2.
// ---------------------------------------------------------------------------
template <int L, bool LINE_FAST> __host__ __device__ constexpr int smem_elems(int nl) {
    return LINE_FAST ? L * nl : nl * Split<L>::L1 * (Split<L>::L2 + 1);
}

template <int L, bool LINE_FAST> __device__ __forceinline__ int sidx(int line, int k1, int n2, int nl) {
    constexpr int L1 = Split<L>::L1, L2 = Split<L>::L2;
    return LINE_FAST ? ((k1 * L2 + n2) * nl + line) : (line * (L1 * (L2 + 1)) + k1 * (L2 + 1) + n2);
}

template <int L, int SIGN, bool LINE_FAST, class Ld>
__device__ __forceinline__ void fft_step1(int nl, Ld& ld, float2* S, const float2* __restrict__ tw) {
    constexpr int L1 = Split<L>::L1, L2 = Split<L>::L2;
    for (int it = threadIdx.x; it < nl * L2; it += blockDim.x) {
        const int line = LINE_FAST ? it % nl : it / L2;
        const int n2 = LINE_FAST ? it / nl : it % L2;
        float2 a[L1];
#pragma unroll
        for (int n1 = 0; n1 < L1; ++n1) a[n1] = ld(line, L2 * n1 + n2);
        Dft<L1, SIGN>::run(a);
#pragma unroll
        for (int k1 = 0; k1 < L1; ++k1) {
            float2 v = a[k1];
            if (k1 != 0 && n2 != 0) v = c_mul_tw<SIGN>(v, __ldg(&tw[n2 * k1]));
            S[sidx<L, LINE_FAST>(line, k1, n2, nl)] = v;
        }
    }
}

template <int L, int SIGN, bool LINE_FAST, class St>
__device__ __forceinline__ void fft_step2(int nl, St& st, const float2* S) {
    constexpr int L1 = Split<L>::L1, L2 = Split<L>::L2;
    for (int it = threadIdx.x; it < nl * L1; it += blockDim.x) {
        const int line = LINE_FAST ? it % nl : it / L1;
        const int k1 = LINE_FAST ? it / nl : it % L1;
        float2 b[L2];
#pragma unroll
        for (int n2 = 0; n2 < L2; ++n2) b[n2] = S[sidx<L, LINE_FAST>(line, k1, n2, nl)];
        Dft<L2, SIGN>::run(b);
#pragma unroll
        for (int k2 = 0; k2 < L2; ++k2) st(line, k1 + L1 * k2, b[k2]);
    }
}

// Step 1 with a hook run once per item after all of its loads: a loader that also
// writes back (the CG direction update) keeps its loads pure, so they are all in
// flight together, and does its stores in the hook.
template <int L, int SIGN, bool LINE_FAST, class Ld, class Post>
__device__ __forceinline__ void fft_step1_post(int nl, Ld& ld, Post& post, float2* S, const float2* __restrict__ tw) {
    constexpr int L1 = Split<L>::L1, L2 = Split<L>::L2;
    for (int it = threadIdx.x; it < nl * L2; it += blockDim.x) {
        const int line = LINE_FAST ? it % nl : it / L2;
        const int n2 = LINE_FAST ? it / nl : it % L2;
        float2 a[L1];
#pragma unroll
        for (int n1 = 0; n1 < L1; ++n1) a[n1] = ld(line, L2 * n1 + n2);
#pragma unroll
        for (int n1 = 0; n1 < L1; ++n1) post(line, L2 * n1 + n2, a[n1]);
        Dft<L1, SIGN>::run(a);
#pragma unroll
        for (int k1 = 0; k1 < L1; ++k1) {
            float2 v = a[k1];
            if (k1 != 0 && n2 != 0) v = c_mul_tw<SIGN>(v, __ldg(&tw[n2 * k1]));
            S[sidx<L, LINE_FAST>(line, k1, n2, nl)] = v;
        }
    }
}

// Step 2 with per-output operands fetched before the DFT: pre(line, k) is issued for
// all L2 outputs of an item first (independent loads in flight together), then
// st(line, k, value, pre(line, k)).
template <int L, int SIGN, bool LINE_FAST, class Pre, class St>
__device__ __forceinline__ void fft_step2_pre(int nl, Pre& pre, St& st, const float2* S) {
    constexpr int L1 = Split<L>::L1, L2 = Split<L>::L2;
    using PV = decltype(pre(0, 0));
    for (int it = threadIdx.x; it < nl * L1; it += blockDim.x) {
        const int line = LINE_FAST ? it % nl : it / L1;
        const int k1 = LINE_FAST ? it / nl : it % L1;
        PV pv[L2];
#pragma unroll
        for (int k2 = 0; k2 < L2; ++k2) pv[k2] = pre(line, k1 + L1 * k2);
        float2 b[L2];
#pragma unroll
        for (int n2 = 0; n2 < L2; ++n2) b[n2] = S[sidx<L, LINE_FAST>(line, k1, n2, nl)];
        Dft<L2, SIGN>::run(b);
#pragma unroll
        for (int k2 = 0; k2 < L2; ++k2) st(line, k1 + L1 * k2, b[k2], pv[k2]);
    }
}

template <int L, int SIGN, bool LINE_FAST, class Ld, class St>
__device__ __forceinline__ void block_fft(int nl, Ld& ld, St& st, float2* S, const float2* __restrict__ tw) {
    fft_step1<L, SIGN, LINE_FAST>(nl, ld, S, tw);
    __syncthreads();
    fft_step2<L, SIGN, LINE_FAST>(nl, st, S);
    __syncthreads();
}

// Forward transform, pointwise multiply, inverse transform, in one pass with two
// exchanges (used along the last axis of the Toeplitz apply).  Lines are adjacent in
// memory (line index fastest).  ld(line, n) gives the input (zero-padded by the
// functor), mul(line, k) the real multiplier of frequency k, st(line, n, v) receives
// the unnormalised inverse at n (the functor keeps the samples it needs).
template <int L, class Ld, class Mul, class St>
__device__ __forceinline__ void block_fft_mul_ifft(int nl, Ld& ld, Mul& mul, St& st, float2* S,
                                                   const float2* __restrict__ tw) {
    constexpr int L1 = Split<L>::L1, L2 = Split<L>::L2;
    fft_step1<L, -1, true>(nl, ld, S, tw);
    __syncthreads();
    // forward step 2, multiply, inverse step 1, all in registers per (line, k1)
    for (int it = threadIdx.x; it < nl * L1; it += blockDim.x) {
        const int line = it % nl, k1 = it / nl;
        float2 b[L2];
#pragma unroll
        for (int n2 = 0; n2 < L2; ++n2) b[n2] = S[sidx<L, true>(line, k1, n2, nl)];
        Dft<L2, -1>::run(b);
#pragma unroll
        for (int k2 = 0; k2 < L2; ++k2) b[k2] = c_scale(b[k2], mul(line, k1 + L1 * k2));
        Dft<L2, +1>::run(b);   // over k2 -> index na
        // only this thread touches the (line, k1) slots, so they can be overwritten
#pragma unroll
        for (int na = 0; na < L2; ++na) {
            float2 v = b[na];
            if (k1 != 0 && na != 0) v = c_mul_tw<+1>(v, __ldg(&tw[na * k1]));
            S[sidx<L, true>(line, k1, na, nl)] = v;
        }
    }
    __syncthreads();
    // inverse step 2: per (line, na), DFT over k1 -> n = na + L2 nb
    for (int it = threadIdx.x; it < nl * L2; it += blockDim.x) {
        const int line = it % nl, na = it / nl;
        float2 c[L1];
#pragma unroll
        for (int k1 = 0; k1 < L1; ++k1) c[k1] = S[sidx<L, true>(line, k1, na, nl)];
        Dft<L1, +1>::run(c);
#pragma unroll
        for (int nb = 0; nb < L1; ++nb) st(line, na + L2 * nb, c[nb]);
    }
    __syncthreads();
}

}  // namespace firm
