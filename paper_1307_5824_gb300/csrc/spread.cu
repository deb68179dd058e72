// spread.cu -- type-1 NUFFT spreading of the central-slice samples (FIRM steps 2-3,
// Section 3.4; eq. kernel and eq. backprojection).
//
// The samples of image m sit at xi = R_m^T (2 pi k / N, 0) for k in the half disc H
// (the other half follows by the symmetry xi(-k) = -xi(k); the transform stage adds
// the mirror image as 2 Re(.)).  On a fine grid of G = 2 sigma * (modes) cells per
// axis the sample lands at y = G/2 + (G/N)(k1 u_m + k2 v_m), u_m and v_m the first
// two rows of R_m.
//
// Pipeline per channel (kernel: weights h^2 on G = 4N; right-hand side: weights
// h b on G = 2N):
//   1. bin:    count points per 16^3 brick (warp-aggregated atomics), scan, and
//              scatter point ids into per-brick segments; cut segments into work
//              items of at most kChunk points.
//   2. spread: persistent CTAs take work items; each accumulates its points into a
//              (16 + W)^3 shared-memory region with shared atomics (FP32), then adds
//              the region into the FP64 global grid with FP64 atomics.
#include <cuda_runtime.h>

#include "firm_internal.h"

namespace firm {

// ---------------------------------------------------------------------------
// Geometry
// ---------------------------------------------------------------------------
__global__ void k_geom(const double* __restrict__ R, int M, ImgGeom* __restrict__ g) {
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    const double* r = R + 9 * (size_t)m;
    ImgGeom o;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        double u = r[d], v = r[3 + d];
        float uh = (float)u, vh = (float)v;
        o.uh[d] = uh;
        o.ul[d] = (float)(u - (double)uh);
        o.vh[d] = vh;
        o.vl[d] = (float)(v - (double)vh);
    }
    g[m] = o;
}

cudaError_t launch_geom(const double* R, int M, ImgGeom* geom, cudaStream_t s) {
    if (M <= 0) return cudaSuccess;
    k_geom<<<(M + 255) / 256, 256, 0, s>>>(R, M, geom);
    return cudaGetLastError();
}

// Integer cell I in [0, G) and fraction f in [0, 1) of the coordinate
// y = G/2 + sk1 * u + sk2 * v along one axis, with sk1 = (G/N) k1 and sk2 = (G/N) k2
// exact small integers.  The products are split exactly (FMA error terms) and the
// integer parts removed before the fractions are summed, so y is formed to ~1e-7.
__device__ __forceinline__ void cell_coord(float sk1, float sk2, float uh, float ul, float vh, float vl,
                                           int halfG, int G, int& I, float& f) {
    // explicit rounding intrinsics: no contraction, so every kernel that calls this
    // (binning and spreading) gets bit-identical cells
    const float a = __fmul_rn(sk1, uh), ea = fmaf(sk1, uh, -a);
    const float b = __fmul_rn(sk2, vh), eb = fmaf(sk2, vh, -b);
    const float ra = rintf(a), rb = rintf(b);
    const float lo = __fadd_rn(__fadd_rn(ea, eb), fmaf(sk1, ul, __fmul_rn(sk2, vl)));
    const float fr = __fadd_rn(__fadd_rn(__fsub_rn(a, ra), __fsub_rn(b, rb)), lo);
    const float fl = floorf(fr);
    float ff = __fsub_rn(fr, fl);
    int ii = (int)ra + (int)rb + (int)fl + halfG;
    if (ff >= 1.0f) { ff = 0.0f; ii += 1; }
    ii %= G;
    if (ii < 0) ii += G;
    I = ii;
    f = ff;
}

struct PointPos {
    int I[3];
    float f[3];
};

__device__ __forceinline__ PointPos point_pos(const ImgGeom& g, int32_t kk, float scale, int halfG, int G) {
    const float k1 = (float)(int16_t)(kk & 0xffff), k2 = (float)(kk >> 16);
    const float sk1 = scale * k1, sk2 = scale * k2;
    PointPos p;
#pragma unroll
    for (int d = 0; d < 3; ++d) cell_coord(sk1, sk2, g.uh[d], g.ul[d], g.vh[d], g.vl[d], halfG, G, p.I[d], p.f[d]);
    return p;
}

// ---------------------------------------------------------------------------
// Binning
// ---------------------------------------------------------------------------
struct BinArgs {
    const ImgGeom* geom;
    const int32_t* htab;
    uint32_t* count;       // count pass: per-brick counters; scatter pass: cursors
    uint32_t* payload;     // scatter pass output
    long long npts;        // M * nH
    int nH, G, halfG, nb;  // nb = bricks per axis
    float scale;
};

template <bool SCATTER>
__global__ void __launch_bounds__(256) k_bin(BinArgs a) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = idx < a.npts;
    int key = -1;
    if (valid) {
        const int m = (int)(idx / a.nH);
        const int t = (int)(idx - (long long)m * a.nH);
        const PointPos p = point_pos(a.geom[m], __ldg(&a.htab[t]), a.scale, a.halfG, a.G);
        key = ((p.I[2] / kBrick) * a.nb + p.I[1] / kBrick) * a.nb + p.I[0] / kBrick;
    }
    // warp aggregation: lanes with equal keys add once
    const unsigned peers = __match_any_sync(0xffffffffu, key);
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(peers) - 1;
    const int rank = __popc(peers & ((1u << lane) - 1u));
    if (!SCATTER) {
        if (valid && lane == leader) atomicAdd(&a.count[key], (uint32_t)__popc(peers));
    } else {
        uint32_t base = 0;
        if (valid && lane == leader) base = atomicAdd(&a.count[key], (uint32_t)__popc(peers));
        base = __shfl_sync(peers, base, leader);
        if (valid) a.payload[base + rank] = (uint32_t)idx;
    }
}

// Single-block scan: cursor[b] = exclusive prefix of count; work items for each brick.
__global__ void __launch_bounds__(1024) k_scan_work(const uint32_t* __restrict__ count, uint32_t* __restrict__ cursor,
                                                    int nbricks, int4* __restrict__ work, int* __restrict__ counters,
                                                    int max_work) {
    __shared__ unsigned long long s_pts[32];
    __shared__ int s_items[32];
    const int T = blockDim.x, tid = threadIdx.x;
    const int per = (nbricks + T - 1) / T;
    const int b0 = min(nbricks, tid * per), b1 = min(nbricks, b0 + per);
    unsigned long long pts = 0;
    int items = 0;
    for (int b = b0; b < b1; ++b) {
        const uint32_t c = count[b];
        pts += c;
        items += (int)((c + kChunk - 1) / kChunk);
    }
    // block exclusive scan of (pts, items)
    const int lane = tid & 31, wid = tid >> 5;
    unsigned long long ip = pts;
    int ii = items;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned long long vp = __shfl_up_sync(0xffffffffu, ip, o);
        int vi = __shfl_up_sync(0xffffffffu, ii, o);
        if (lane >= o) { ip += vp; ii += vi; }
    }
    if (lane == 31) { s_pts[wid] = ip; s_items[wid] = ii; }
    __syncthreads();
    if (wid == 0) {
        const int nw = T / 32;
        unsigned long long vp = lane < nw ? s_pts[lane] : 0ull;
        int vi = lane < nw ? s_items[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned long long tp = __shfl_up_sync(0xffffffffu, vp, o);
            int ti = __shfl_up_sync(0xffffffffu, vi, o);
            if (lane >= o) { vp += tp; vi += ti; }
        }
        if (lane < nw) { s_pts[lane] = vp; s_items[lane] = vi; }
    }
    __syncthreads();
    unsigned long long off = ip - pts + (wid ? s_pts[wid - 1] : 0ull);
    int woff = ii - items + (wid ? s_items[wid - 1] : 0);
    for (int b = b0; b < b1; ++b) {
        const uint32_t c = count[b];
        cursor[b] = (uint32_t)off;
        for (uint32_t s = 0; s < c; s += kChunk) {
            if (woff < max_work) work[woff] = make_int4(b, (int)(off + s), (int)min((uint32_t)kChunk, c - s), 0);
            ++woff;
        }
        off += c;
    }
    if (tid == T - 1) {
        counters[0] = min(woff, max_work);
        counters[1] = 0;
    }
}

cudaError_t launch_bin(Plan& P, int M, bool kc) {
    Workspace& w = P.ws;
    const int G = kc ? P.Gk : P.Gr;
    const int nb = kc ? P.nbk : P.nbr;
    const int nbricks = nb * nb * nb;
    cudaError_t e = cudaMemsetAsync(w.count, 0, sizeof(uint32_t) * nbricks, P.stream);
    if (e != cudaSuccess) return e;
    BinArgs a;
    a.geom = w.geom;
    a.htab = w.htab;
    a.count = w.count;
    a.payload = w.payload;
    a.npts = (long long)M * P.nH;
    a.nH = P.nH;
    a.G = G;
    a.halfG = G / 2;
    a.nb = nb;
    a.scale = (float)(G / P.N);
    const long long blocks = (a.npts + 255) / 256;
    if (blocks == 0) {
        k_scan_work<<<1, 1024, 0, P.stream>>>(w.count, w.cursor, nbricks, w.work, w.counters, (int)P.max_work);
        return cudaGetLastError();
    }
    k_bin<false><<<(unsigned)blocks, 256, 0, P.stream>>>(a);
    k_scan_work<<<1, 1024, 0, P.stream>>>(w.count, w.cursor, nbricks, w.work, w.counters, (int)P.max_work);
    a.count = w.cursor;
    k_bin<true><<<(unsigned)blocks, 256, 0, P.stream>>>(a);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Spreading
// ---------------------------------------------------------------------------
struct SpreadArgs {
    const uint32_t* payload;
    const int4* work;
    int* counters;
    const ImgGeom* geom;
    const int32_t* htab;
    const int32_t* gid;
    const float* h2;          // kernel channel weights [group][t]
    const float2* samples;    // right-hand-side weights [m][t]
    double* grid;             // G^3 real, or G^3 complex interleaved (re, im)
    int G, halfG, nb, nH, n_ctf;
    float scale;
    KbPoly poly;
};

constexpr int kSpreadThreads = 256;

template <int W>
__device__ __forceinline__ void window_taps(const KbPoly& P, float f, int& c, float* w) {
    // first tap offset u in [0,1): taps at u + l - W/2, l = 0..W-1
    constexpr float h = (W & 1) ? 0.5f : 0.0f;
    const float t0 = f - h;
    const float cf = ceilf(t0);
    c = (int)cf;
    const float z = 2.0f * (cf - t0) - 1.0f;
#pragma unroll
    for (int l = 0; l < W; ++l) {
        float acc = P.c[l][kKbDeg];
#pragma unroll
        for (int j = kKbDeg - 1; j >= 0; --j) acc = fmaf(acc, z, P.c[l][j]);
        w[l] = acc;
    }
}

template <int W, bool CPLX>
__global__ void __launch_bounds__(kSpreadThreads) k_spread(const SpreadArgs a) {
    constexpr int RG = kBrick + W;
    constexpr int RG3 = RG * RG * RG;
    extern __shared__ float sm[];           // CPLX: [re plane][im plane]
    __shared__ int s_item;
    const int n_work = a.counters[0];
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(&a.counters[1], 1);
        for (int i = threadIdx.x; i < RG3 * (CPLX ? 2 : 1); i += blockDim.x) sm[i] = 0.0f;
        __syncthreads();
        const int item = s_item;
        if (item >= n_work) break;
        const int4 wk = a.work[item];
        const int b = wk.x;
        const int bx = b % a.nb, by = (b / a.nb) % a.nb, bz = b / (a.nb * a.nb);
        const int lo0 = bx * kBrick, lo1 = by * kBrick, lo2 = bz * kBrick;
        for (int j = threadIdx.x; j < wk.z; j += blockDim.x) {
            const uint32_t id = __ldg(&a.payload[wk.y + j]);
            const int m = (int)(id / (uint32_t)a.nH);
            const int t = (int)(id - (uint32_t)m * (uint32_t)a.nH);
            const PointPos p = point_pos(a.geom[m], __ldg(&a.htab[t]), a.scale, a.halfG, a.G);
            float wr, wi = 0.0f;
            if (CPLX) {
                const float2 s = __ldg(&a.samples[(size_t)m * a.nH + t]);
                wr = s.x;
                wi = s.y;
            } else {
                const int g = min(max(__ldg(&a.gid[m]), 0), a.n_ctf - 1);
                wr = __ldg(&a.h2[(size_t)g * a.nH + t]);
            }
            float wx[W], wy[W], wz[W];
            int cx, cy, cz;
            window_taps<W>(a.poly, p.f[0], cx, wx);
            window_taps<W>(a.poly, p.f[1], cy, wy);
            window_taps<W>(a.poly, p.f[2], cz, wz);
            const int r0 = p.I[0] - lo0 + cx, r1 = p.I[1] - lo1 + cy, r2 = p.I[2] - lo2 + cz;
            if ((unsigned)r0 > (unsigned)kBrick || (unsigned)r1 > (unsigned)kBrick || (unsigned)r2 > (unsigned)kBrick) {
                atomicOr(&a.counters[2], 1);   // point outside its brick: reported, never written
                continue;
            }
            const int base = (r2 * RG + r1) * RG + r0;
#pragma unroll
            for (int dz = 0; dz < W; ++dz) {
                const float az = wr * wz[dz];
                const float bzw = wi * wz[dz];
#pragma unroll
                for (int dy = 0; dy < W; ++dy) {
                    const float ayz = az * wy[dy];
                    const float byz = bzw * wy[dy];
                    float* row = sm + base + (dz * RG + dy) * RG;
#pragma unroll
                    for (int dx = 0; dx < W; ++dx) {
                        atomicAdd(row + dx, ayz * wx[dx]);
                        if (CPLX) atomicAdd(row + RG3 + dx, byz * wx[dx]);
                    }
                }
            }
        }
        __syncthreads();
        // flush the region into the FP64 grid (periodic wrap)
        const int o0 = lo0 - W / 2, o1 = lo1 - W / 2, o2 = lo2 - W / 2;
        for (int i = threadIdx.x; i < RG3; i += blockDim.x) {
            const float vr = sm[i];
            const float vi = CPLX ? sm[RG3 + i] : 0.0f;
            if (vr == 0.0f && vi == 0.0f) continue;
            const int rx = i % RG, ry = (i / RG) % RG, rz = i / (RG * RG);
            int gx = o0 + rx, gy = o1 + ry, gz = o2 + rz;
            gx += (gx < 0) ? a.G : 0;
            gx -= (gx >= a.G) ? a.G : 0;
            gy += (gy < 0) ? a.G : 0;
            gy -= (gy >= a.G) ? a.G : 0;
            gz += (gz < 0) ? a.G : 0;
            gz -= (gz >= a.G) ? a.G : 0;
            const size_t cell = ((size_t)gz * a.G + gy) * a.G + gx;
            if (CPLX) {
                atomicAdd(&a.grid[2 * cell], (double)vr);
                atomicAdd(&a.grid[2 * cell + 1], (double)vi);
            } else {
                atomicAdd(&a.grid[cell], (double)vr);
            }
        }
        __syncthreads();
    }
}

template <int W, bool CPLX>
static cudaError_t spread_w(Plan& P, const SpreadArgs& a) {
    constexpr int RG = kBrick + W;
    const size_t smem = sizeof(float) * RG * RG * RG * (CPLX ? 2 : 1);
    cudaError_t e = cudaFuncSetAttribute(k_spread<W, CPLX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_spread<W, CPLX>, kSpreadThreads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    k_spread<W, CPLX><<<P.num_sms * per_sm, kSpreadThreads, smem, P.stream>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_spread(Plan& P, int M, bool kc) {
    Workspace& w = P.ws;
    const int G = kc ? P.Gk : P.Gr;
    const size_t cells = (size_t)G * G * G * (kc ? 1 : 2);
    cudaError_t e = cudaMemsetAsync(w.grid, 0, sizeof(double) * cells, P.stream);
    if (e != cudaSuccess || M <= 0) return e;
    SpreadArgs a;
    a.payload = w.payload;
    a.work = w.work;
    a.counters = w.counters;
    a.geom = w.geom;
    a.htab = w.htab;
    a.gid = P.cur_gid;
    a.h2 = w.h2;
    a.samples = w.samples;
    a.grid = w.grid;
    a.G = G;
    a.halfG = G / 2;
    a.nb = kc ? P.nbk : P.nbr;
    a.nH = P.nH;
    a.n_ctf = P.n_ctf;
    a.scale = (float)(G / P.N);
    a.poly = P.poly;
    switch (P.p.W) {
        case 6: return kc ? spread_w<6, false>(P, a) : spread_w<6, true>(P, a);
        case 7: return kc ? spread_w<7, false>(P, a) : spread_w<7, true>(P, a);
        case 8: return kc ? spread_w<8, false>(P, a) : spread_w<8, true>(P, a);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace firm
