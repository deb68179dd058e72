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
//   1. bin:    count points per 8^3 brick (warp-aggregated atomics), scan, scatter
//              point ids into per-brick segments cut into work items of at most
//              `chunk` points, and order each item round-robin over bank classes.
//   2. spread: persistent CTAs take work items; each accumulates its points into an
//              (8 + W)^3 shared-memory region in int32 fixed point (native shared
//              atomics), folds it into FP32 every 512 or 1024 points, then adds the region
//              into the FP64 global grid with FP64 atomics.
// The forward projector's interpolation (k_interp, at the end of this file) is the
// transpose of step 2 on the same binning: a CTA stages its brick's region of the
// transformed grid and gathers the W^3 taps of each point, with no atomics.
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
    // (binning and spreading) gets bit-identical cells.  Round-to-nearest integers by
    // adding 1.5 * 2^23 (|a|, |b| <= G/2 < 2^22); the bit pattern then holds the integer.
    constexpr float kMagic = 12582912.0f;
    constexpr int kMagicBits = 0x4B400000;
    const float a = __fmul_rn(sk1, uh), ea = fmaf(sk1, uh, -a);
    const float b = __fmul_rn(sk2, vh), eb = fmaf(sk2, vh, -b);
    const float ma = __fadd_rn(a, kMagic), mb = __fadd_rn(b, kMagic);
    const float ra = __fsub_rn(ma, kMagic), rb = __fsub_rn(mb, kMagic);
    const float lo = __fadd_rn(__fadd_rn(ea, eb), fmaf(sk1, ul, __fmul_rn(sk2, vl)));
    const float fr = __fadd_rn(__fadd_rn(__fsub_rn(a, ra), __fsub_rn(b, rb)), lo);
    const float fl = floorf(fr);
    float ff = __fsub_rn(fr, fl);
    int ii = (__float_as_int(ma) - kMagicBits) + (__float_as_int(mb) - kMagicBits) +
             (__float_as_int(__fadd_rn(fl, kMagic)) - kMagicBits) + halfG;
    if (ff >= 1.0f) { ff = 0.0f; ii += 1; }
    // |k1 u + k2 v| <= |k| <= N/2 (u, v: parts of a unit column of R), so ii lies in
    // [-1, G + 1]: one wrap either way is the periodic index
    if (ii >= G) ii -= G;
    else if (ii < 0) ii += G;
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
// Window taps and the region base of a point
// ---------------------------------------------------------------------------
template <int W>
__device__ __forceinline__ int tap_shift(float f) {
    // first tap offset u = c - (f - h) in [0, 1), h = 1/2 for odd W, 0 for even W
    constexpr float h = (W & 1) ? 0.5f : 0.0f;
    return (int)ceilf(f - h);
}

template <int W>
__device__ __forceinline__ void window_taps(const KbPoly& P, float f, float* w) {
    constexpr float h = (W & 1) ? 0.5f : 0.0f;
    const float t0 = f - h;
    const float z = 2.0f * (ceilf(t0) - t0) - 1.0f;
#pragma unroll
    for (int l = 0; l < W; ++l) {
        float acc = P.c[l][kKbDeg];
#pragma unroll
        for (int j = kKbDeg - 1; j >= 0; --j) acc = fmaf(acc, z, P.c[l][j]);
        w[l] = acc;
    }
}

// Dither of the kernel channel's fixed-point rounding: a value in [-1/2, 1/2) fixed by
// the point id (a 32-bit integer hash), added to every tap of the point before it is
// rounded to an integer.  Rounding to nearest drops every tap below half a unit, and
// the far taps of the window are that small: without the dither the kernel's sums come
// out biased low (~1e-6 relative, a smooth error that moves a 10-iteration CG volume by
// 1e-4 on the N=64 workload).  With it the rounding is unbiased, E[round(v + d)] = v
// for d uniform, and its error is white (a 1e-6 white error in Ker moves that volume by
// ~4e-7).
__device__ __forceinline__ float point_dither(uint32_t id) {
    uint32_t h = id * 2654435761u;
    h ^= h >> 15;
    h *= 2246822519u;
    h ^= h >> 13;
    return (float)(h >> 8) * (1.0f / 16777216.0f) - 0.5f;
}

// Rank (mod W) of this lane's point among the lanes of its warp with the same bank
// class (base mod 32; base < 0: no point).  Called by all 32 lanes.  Most warp steps of
// a round-robin piece hold 32 distinct classes: one OR-reduction of the class bits
// finds those, and only the others pay for the match.
template <int W>
__device__ __forceinline__ int class_rank(int base, int lane) {
    const bool pt = base >= 0;
    const unsigned bits = __reduce_or_sync(0xffffffffu, pt ? 1u << (base & 31) : 0u);
    const unsigned pts = __ballot_sync(0xffffffffu, pt);
    if (__popc(bits) == __popc(pts)) return 0;
    const unsigned same = __match_any_sync(0xffffffffu, pt ? (base & 31) : -1 - lane);
    const int r = __popc(same & ((1u << lane) - 1u));
    return r < W ? r : r % W;
}

// Bricks: 8 x 8 x BZ cells (BZ = kBrickZk for the kernel channel, 8 for A*b).
template <bool KC> struct Brick { static constexpr int BZ = KC ? kBrickZk : kBrick; };

// Index of the first tap of a point inside its brick's (8 + W) x (8 + W) x (BZ + W)
// region (x fastest), or -1 if the point is not inside the brick (never expected:
// binning uses the same code).
template <int W, int BZ>
__device__ __forceinline__ int region_base(const PointPos& p, int lo0, int lo1, int lo2) {
    constexpr int RG = kBrick + W;
    const int r0 = p.I[0] - lo0 + tap_shift<W>(p.f[0]);
    const int r1 = p.I[1] - lo1 + tap_shift<W>(p.f[1]);
    const int r2 = p.I[2] - lo2 + tap_shift<W>(p.f[2]);
    if ((unsigned)r0 > (unsigned)kBrick || (unsigned)r1 > (unsigned)kBrick || (unsigned)r2 > (unsigned)BZ)
        return -1;
    return (r2 * RG + r1) * RG + r0;
}

// ---------------------------------------------------------------------------
// Binning.  Points are counted and scattered by brick (warp-aggregated atomics: lanes
// hold consecutive samples of one image, which mostly share a brick).  Each brick's
// segment is cut into pieces of at most kChunk points (the work items), and every
// piece is then counting-sorted in shared memory by bank class = region base mod 32:
// lane l of a spreading warp takes points of class l, so the 32 lanes of every tap
// step touch 32 different shared-memory banks.
// ---------------------------------------------------------------------------
struct BinArgs {
    const ImgGeom* geom;
    const int32_t* htab;
    uint32_t* count;       // count pass: per-brick counters; scatter pass: cursors
    uint32_t* payload;     // scatter pass output: point ids m * nH + t
    uint8_t* cls;          // scatter pass output: bank class of each point
    const float2* samples; // A*b channel: weights [m][t], copied to samples_b[slot] by the scatter
    float2* samples_b;     //   (consecutive lanes read consecutive t: coalesced)
    long long npts;        // M * nH
    int nH, G, halfG, nb;  // nb = bricks per axis
    float scale;
};

template <int W, bool SCATTER, bool KC>
__global__ void __launch_bounds__(256) k_bin(BinArgs a, int M) {
    constexpr int BZ = Brick<KC>::BZ;
    // x: samples t of one image (consecutive lanes walk a column of the half disc);
    // y: images.  Runs of equal bricks among consecutive lanes are aggregated.
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    for (int m = blockIdx.y; m < M; m += gridDim.y) {
        const bool valid = t < a.nH;
        int key = -1, c = 0;
        if (valid) {
            const PointPos p = point_pos(a.geom[m], __ldg(&a.htab[t]), a.scale, a.halfG, a.G);
            const int bx = p.I[0] / kBrick, by = p.I[1] / kBrick, bz = p.I[2] / BZ;
            key = (bz * a.nb + by) * a.nb + bx;
            if (SCATTER) c = region_base<W, BZ>(p, bx * kBrick, by * kBrick, bz * BZ) & 31;
        }
        const int prev = __shfl_up_sync(0xffffffffu, key, 1);
        const bool head = (lane == 0) || (prev != key);
        const unsigned heads = __ballot_sync(0xffffffffu, head);
        // run of this lane: from its head to the lane before the next head
        const int my_head = 31 - __clz(heads & ((2u << lane) - 1u));
        const unsigned later = heads & ~((2u << lane) - 1u);
        const int next_head = later ? __ffs(later) - 1 : 32;
        uint32_t base = 0;
        if (valid && head) {
            const int run = next_head - lane;
            base = atomicAdd(&a.count[key], (uint32_t)run);
        }
        if (SCATTER) {
            base = __shfl_sync(0xffffffffu, base, my_head);
            if (valid) {
                const uint32_t slot = base + (uint32_t)(lane - my_head);
                a.payload[slot] = ((uint32_t)m << kTBits) | (uint32_t)t;
                a.cls[slot] = (uint8_t)c;
                if (a.samples) a.samples_b[slot] = __ldg(&a.samples[(size_t)m * a.nH + t]);
            }
        }
    }
}

// Scatter pass with 2D patches: each warp takes a 4 x 8 patch of (k1, k2) of one image
// (4 columns of the half disc, 8 consecutive k2 in each), so its 32 points cover a small
// 2D piece of the slice and fall in few bricks; lanes with equal bricks are grouped
// with __match_any_sync, one cursor atomic per group (about half as many as runs along
// one column give).  col[k1] = (first index t of column k1, its lowest k2, its highest k2).
template <int W, bool KC>
__global__ void __launch_bounds__(256) k_bin_scatter2d(BinArgs a, int M, int hN, const int4* __restrict__ col,
                                                       int tiles_x, int n_tiles) {
    constexpr int BZ = Brick<KC>::BZ;
    const int lane = threadIdx.x & 31;
    const int tile = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (tile >= n_tiles) return;                       // uniform over the warp
    const int k1 = (tile % tiles_x) * 4 + (lane >> 3);
    const int k2 = -hN + (tile / tiles_x) * 8 + (lane & 7);
    int t = -1;
    if (k1 <= hN) {
        const int4 c = __ldg(&col[k1]);
        if (k2 >= c.y && k2 <= c.z) t = c.x + (k2 - c.y);
    }
    const bool valid = t >= 0;
    const int32_t kk = (int32_t)((uint32_t)(k1 & 0xffff) | ((uint32_t)k2 << 16));
    for (int m = blockIdx.y; m < M; m += gridDim.y) {
        int key = -1, c = 0;
        if (valid) {
            const PointPos p = point_pos(a.geom[m], kk, a.scale, a.halfG, a.G);
            const int bx = p.I[0] / kBrick, by = p.I[1] / kBrick, bz = p.I[2] / BZ;
            key = (bz * a.nb + by) * a.nb + bx;
            c = region_base<W, BZ>(p, bx * kBrick, by * kBrick, bz * BZ) & 31;
        }
        const unsigned grp = __match_any_sync(0xffffffffu, key);
        const int leader = __ffs(grp) - 1;
        uint32_t base = 0;
        if (valid && lane == leader) base = atomicAdd(&a.count[key], (uint32_t)__popc(grp));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (valid) {
            const uint32_t slot = base + (uint32_t)__popc(grp & ((1u << lane) - 1u));
            a.payload[slot] = ((uint32_t)m << kTBits) | (uint32_t)t;
            a.cls[slot] = (uint8_t)c;
            if (a.samples) a.samples_b[slot] = __ldg(&a.samples[(size_t)m * a.nH + t]);
        }
    }
}

// Scan over bricks: cursor = exclusive prefix of count; work items (brick, start,
// length) of at most `chunk` points (chunk <= kChunk), numbered in brick order.  Three
// launches: per-block totals of points and items over kScanSpan bricks, an exclusive
// scan of those totals (one block), and the per-block scan that writes cursors and
// items from its block's offsets.  nbricks is a multiple of 4.
constexpr int kScanThreads = kScanSpan / 4;     // one uint4 of counts per thread
struct ScanPart {
    unsigned long long pts;
    long long items;
};

// Block-wide inclusive scan of (pts, items); returns the block totals in thread 0's view
// through s_tot.
__device__ __forceinline__ void block_scan2(unsigned long long& ip, long long& ii, ScanPart* s_w, ScanPart* s_tot) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long vp = __shfl_up_sync(0xffffffffu, ip, o);
        const long long vi = __shfl_up_sync(0xffffffffu, ii, o);
        if (lane >= o) { ip += vp; ii += vi; }
    }
    if (lane == 31) s_w[wid] = ScanPart{ip, ii};
    __syncthreads();
    if (wid == 0) {
        const int nw = blockDim.x / 32;
        unsigned long long vp = lane < nw ? s_w[lane].pts : 0ull;
        long long vi = lane < nw ? s_w[lane].items : 0ll;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long tp = __shfl_up_sync(0xffffffffu, vp, o);
            const long long ti = __shfl_up_sync(0xffffffffu, vi, o);
            if (lane >= o) { vp += tp; vi += ti; }
        }
        if (lane < nw) s_w[lane] = ScanPart{vp, vi};
        if (lane == nw - 1) *s_tot = ScanPart{vp, vi};
    }
    __syncthreads();
    if (wid > 0) { ip += s_w[wid - 1].pts; ii += s_w[wid - 1].items; }
}

template <bool WRITE>
__global__ void __launch_bounds__(kScanThreads) k_scan_bricks(const uint32_t* __restrict__ count,
                                                              uint32_t* __restrict__ cursor, int nbricks,
                                                              ScanPart* __restrict__ part, int4* __restrict__ work,
                                                              int* __restrict__ counters, int max_work, int chunk) {
    __shared__ ScanPart s_w[32], s_tot;
    const int b = blockIdx.x * kScanSpan + 4 * threadIdx.x;
    uint4 c4 = make_uint4(0, 0, 0, 0);
    if (b < nbricks) c4 = *reinterpret_cast<const uint4*>(count + b);
    const uint32_t c[4] = {c4.x, c4.y, c4.z, c4.w};
    unsigned long long pts = 0;
    long long items = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        pts += c[k];
        items += (c[k] + chunk - 1) / chunk;
    }
    unsigned long long ip = pts;
    long long ii = items;
    block_scan2(ip, ii, s_w, &s_tot);
    if (!WRITE) {
        if (threadIdx.x == 0) part[blockIdx.x] = s_tot;
        return;
    }
    unsigned long long off = part[blockIdx.x].pts + ip - pts;      // part: exclusive block offsets
    long long woff = part[blockIdx.x].items + ii - items;
    if (b < nbricks) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            cursor[b + k] = (uint32_t)off;
            for (uint32_t s = 0; s < c[k]; s += (uint32_t)chunk) {
                if (woff < max_work) work[woff] = make_int4(b + k, (int)(off + s), (int)min((uint32_t)chunk, c[k] - s), 0);
                ++woff;
            }
            off += c[k];
        }
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == blockDim.x - 1) {
        counters[0] = (int)min(woff, (long long)max_work);
        counters[1] = 0;
    }
}

// Exclusive scan of the per-block totals in place (one block; n <= 32 * kScanThreads).
__global__ void __launch_bounds__(kScanThreads) k_scan_parts(ScanPart* __restrict__ part, int n) {
    __shared__ ScanPart s_w[32], s_tot;
    const int per = (n + kScanThreads - 1) / kScanThreads;
    const int i0 = min(n, (int)threadIdx.x * per), i1 = min(n, i0 + per);
    unsigned long long pts = 0;
    long long items = 0;
    for (int i = i0; i < i1; ++i) { pts += part[i].pts; items += part[i].items; }
    unsigned long long ip = pts;
    long long ii = items;
    block_scan2(ip, ii, s_w, &s_tot);
    unsigned long long op = ip - pts;
    long long oi = ii - items;
    for (int i = i0; i < i1; ++i) {
        const ScanPart v = part[i];
        part[i] = ScanPart{op, oi};
        op += v.pts;
        oi += v.items;
    }
}

static void launch_scan(Plan& P, int nbricks) {
    Workspace& w = P.ws;
    const int nblk = (nbricks + kScanSpan - 1) / kScanSpan;
    ScanPart* part = reinterpret_cast<ScanPart*>(w.scan_part);
    k_scan_bricks<false><<<nblk, kScanThreads, 0, P.stream>>>(w.count, w.cursor, nbricks, part, w.work,
                                                               w.counters, (int)P.max_work, P.chunk);
    k_scan_parts<<<1, kScanThreads, 0, P.stream>>>(part, nblk);
    k_scan_bricks<true><<<nblk, kScanThreads, 0, P.stream>>>(w.count, w.cursor, nbricks, part, w.work,
                                                              w.counters, (int)P.max_work, P.chunk);
    P.launches += 3;
}

// Orders each piece round-robin over bank classes, in place: the point of rank r in
// class c (order within a class is arbitrary) goes to position A(r) + #{c' < c : n_c' > r},
// A(r) = sum over r' < r of #{c : n_c > r'}.  Any 32 consecutive points then belong to
// (almost always) 32 different classes, so the spreading threads can take the piece
// in order -- every thread the same number of points -- and a warp's 32 atomics of a
// tap step still hit 32 different banks.  A piece whose largest class exceeds
// kSortLevels points (a very skewed piece) is only grouped by class: any order is
// correct, this one just conflicts more.
constexpr int kSortLevels = 1024;
constexpr int kSortSmem = kChunk * (4 + 1) + kSortLevels * (4 + 4);   // ids, classes, masks, prefix
// With perm != nullptr (A*b channel) the piece's pre-sort index of each point is kept
// in perm at its new position: the A*b weights stay where the scatter put them (in
// scatter order, samples_b), and the spreading pass reads them through perm from
// within the piece's own 64 KB window instead of one scattered sector per point.
// With in != nullptr the ids are read from `in` (scatter order, kept) and written sorted
// to payload; inv_perm != nullptr receives, at each point's scatter position, its
// position in the sorted piece (the fused form's weight gather walks the points in
// scatter order, where the points of one image sit together).
__global__ void __launch_bounds__(256) k_class_sort(uint32_t* __restrict__ payload, const uint8_t* __restrict__ cls,
                                                    const int4* __restrict__ work, const int* __restrict__ counters,
                                                    uint16_t* __restrict__ perm, const uint32_t* __restrict__ in,
                                                    uint16_t* __restrict__ inv_perm) {
    extern __shared__ uint32_t sm_u[];
    uint32_t* s_ids = sm_u;                                         // kChunk
    uint32_t* s_mask = s_ids + kChunk;                              // kSortLevels: classes with n_c > r
    int* s_pre = reinterpret_cast<int*>(s_mask + kSortLevels);      // kSortLevels: A(r)
    uint8_t* s_cls = reinterpret_cast<uint8_t*>(s_pre + kSortLevels);
    __shared__ int s_hist[32], s_cur[32], s_off[32], s_maxn;
    __shared__ int s_part[8];
    const int n_work = counters[0];
    for (int item = blockIdx.x; item < n_work; item += gridDim.x) {
        const int4 wk = work[item];
        const int len = wk.z;
        if (threadIdx.x < 32) s_hist[threadIdx.x] = 0;
        __syncthreads();
        // four points per thread per step, all loads issued before the shared stores
        for (int i0 = threadIdx.x; i0 < len; i0 += 4 * blockDim.x) {
            uint8_t c[4];
            uint32_t id[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int i = i0 + u * blockDim.x;
                if (i < len) { c[u] = cls[wk.y + i]; id[u] = in ? in[wk.y + i] : payload[wk.y + i]; }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int i = i0 + u * blockDim.x;
                if (i < len) {
                    s_ids[i] = id[u];
                    s_cls[i] = c[u];
                    atomicAdd(&s_hist[c[u]], 1);
                }
            }
        }
        __syncthreads();
        if (threadIdx.x < 32) {
            const int h = s_hist[threadIdx.x];
            int v = h, mx = h;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_up_sync(0xffffffffu, v, o);
                if ((int)threadIdx.x >= o) v += u;
                mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            }
            s_off[threadIdx.x] = v - h;
            s_cur[threadIdx.x] = v - h;
            if (threadIdx.x == 0) s_maxn = mx;
        }
        __syncthreads();
        const int maxn = s_maxn;
        const bool interleave = maxn <= kSortLevels;
        if (interleave) {
            // masks and per-thread partial sums of their popcounts (contiguous r ranges)
            const int per = (maxn + blockDim.x - 1) / blockDim.x;
            const int r0 = threadIdx.x * per, r1 = min(maxn, r0 + per);
            int part = 0;
            for (int r = r0; r < r1; ++r) {
                uint32_t m = 0;
#pragma unroll 8
                for (int c = 0; c < 32; ++c) m |= (uint32_t)(s_hist[c] > r) << c;
                s_mask[r] = m;
                part += __popc(m);
            }
            // exclusive block scan of the partial sums (warp scans, then the 8 warp totals)
            const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
            int incl = part;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += u;
            }
            if (lane == 31) s_part[wid] = incl;
            __syncthreads();
            int wbase = 0;
            for (int i = 0; i < wid; ++i) wbase += s_part[i];
            int acc = wbase + incl - part;
            for (int r = r0; r < r1; ++r) { s_pre[r] = acc; acc += __popc(s_mask[r]); }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < len; i += blockDim.x) {
            const int c = s_cls[i];
            const int k = atomicAdd(&s_cur[c], 1);
            int pos = k;                                        // grouped by class
            if (interleave) {
                const int r = k - s_off[c];
                pos = s_pre[r] + __popc(s_mask[r] & ((1u << c) - 1u));
            }
            payload[wk.y + pos] = s_ids[i];
            if (perm) perm[wk.y + pos] = (uint16_t)i;
            if (inv_perm) inv_perm[wk.y + i] = (uint16_t)pos;
        }
        __syncthreads();
    }
}

template <int W>
static void bin_w(Plan& P, const BinArgs& a0, int nbricks, bool kc) {
    Workspace& w = P.ws;
    BinArgs a = a0;
    const int M = (int)(a.npts / a.nH);
    const dim3 grid((a.nH + 255) / 256, (unsigned)(M < 65535 ? M : 65535));
    if (kc) k_bin<W, false, true><<<grid, 256, 0, P.stream>>>(a, M);
    else k_bin<W, false, false><<<grid, 256, 0, P.stream>>>(a, M);
    launch_scan(P, nbricks);
    a.count = w.cursor;
    const int hN = P.N / 2, tiles_x = (hN + 1 + 3) / 4, n_tiles = tiles_x * ((P.N + 1 + 7) / 8);
    const dim3 grid2((n_tiles + 7) / 8, (unsigned)(M < 65535 ? M : 65535));
    if (kc) k_bin_scatter2d<W, true><<<grid2, 256, 0, P.stream>>>(a, M, hN, w.colinfo, tiles_x, n_tiles);
    else k_bin_scatter2d<W, false><<<grid2, 256, 0, P.stream>>>(a, M, hN, w.colinfo, tiles_x, n_tiles);
    cudaFuncSetAttribute(k_class_sort, cudaFuncAttributeMaxDynamicSharedMemorySize, kSortSmem);
    const bool keep = kc && w.payload_scat;       // fused plans keep the scatter order
    k_class_sort<<<P.num_sms * 4, 256, kSortSmem, P.stream>>>(w.payload, w.cls, w.work, w.counters,
                                                               kc ? nullptr : w.perm, keep ? w.payload_scat : nullptr,
                                                               keep ? w.inv_perm : nullptr);
}

cudaError_t launch_bin(Plan& P, int M, bool kc) {
    Workspace& w = P.ws;
    const int G = kc ? P.Gk : P.Gr;
    const int nb = kc ? P.nbk : P.nbr;
    const int nbricks = nb * nb * (kc ? P.nbkz : P.nbr);
    cudaError_t e = cudaMemsetAsync(w.count, 0, sizeof(uint32_t) * nbricks, P.stream);
    if (e != cudaSuccess) return e;
    BinArgs a;
    a.geom = w.geom;
    a.htab = w.htab;
    a.count = w.count;
    a.payload = kc && w.payload_scat ? w.payload_scat : w.payload;
    a.cls = w.cls;
    a.samples = kc ? nullptr : w.samples;
    a.samples_b = w.samples_b;
    a.npts = (long long)M * P.nH;
    a.nH = P.nH;
    a.G = G;
    a.halfG = G / 2;
    a.nb = nb;
    a.scale = (float)(G / P.N);
    const long long blocks = (a.npts + 255) / 256;
    if (blocks == 0) {
        launch_scan(P, nbricks);
        return cudaGetLastError();
    }
    switch (P.p.W) {
        case 6: bin_w<6>(P, a, nbricks, kc); break;
        case 7: bin_w<7>(P, a, nbricks, kc); break;
        case 8: bin_w<8>(P, a, nbricks, kc); break;
        default: return cudaErrorInvalidValue;
    }
    P.launches += 3;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Spreading
//
// Level 1: int32 fixed point in shared memory, one native shared-memory atomic add
// per tap (v * S rounded to nearest through the FMA with 1.5 * 2^23; the kernel
// channel adds the point's dither first, see point_dither).  S is a power
// of two with max|w| * S <= 2^21 (A*b) or 2^20 (kernel), and level 1 is folded into
// the FP32 level-2 region after every 512 (A*b) or 1024 (kernel) points of the block,
// so a cell can never exceed 2^30.  Level 2 is added into the FP64 grid when the work
// item ends.
// ---------------------------------------------------------------------------
struct SpreadArgs {
    const uint32_t* payload;
    const int4* work;
    int* counters;
    const ImgGeom* geom;
    const int32_t* htab;
    const int32_t* gid;
    const float* h2;          // kernel channel weights [group][t]
    const float2* samples_b;  // right-hand-side weights in scatter order
    const float2* samples;    // fused form: the weights h b at [m][t]
    const uint16_t* perm;     // per payload position: the point's index in scatter order
    double* grid;             // G^3 real, or G^3 complex interleaved (re, im)
    int G, halfG, nb, nH, n_ctf;
    float scale;
    float wmax_fixed;         // > 0: bound on |w| known in advance (no pre-pass)
    const float* wmax_item;   // fused form: per work item, the largest |h b| of its points
    KbPoly poly;
};

constexpr int kSpreadThreads = 256;
constexpr int kSpreadWarps = kSpreadThreads / 32;

// Weight of the point at payload position pos (image m, sample t) of the piece
// starting at p0.
__device__ __forceinline__ float2 point_weight(const SpreadArgs& a, bool cplx, int m, int t, uint32_t p0,
                                               uint32_t pos) {
    if (cplx) return __ldg(&a.samples_b[p0 + __ldg(&a.perm[pos])]);
    const int g = min(max(__ldg(&a.gid[m]), 0), a.n_ctf - 1);
    return make_float2(__ldg(&a.h2[(size_t)g * a.nH + t]), 0.0f);
}

// Points each thread spreads between two folds of level 1 into level 2.  A fold is a
// block-wide barrier; with PPR points per thread a cell can receive at most 256 * PPR
// taps between folds, so a tap is scaled to at most 2^30 / (256 * PPR): 2^21 for the
// A*b channel (PPR 2) and 2^20 for the kernel channel (PPR 4, half the barriers; the
// extra bit of rounding is white noise under the dither, which CG does not amplify;
// for A*b it would double the fixed-point error to ~3e-6 for a 1% gain, so A*b keeps
// PPR 2).
template <bool CPLX> struct SpreadRound { static constexpr int PPR = CPLX ? 2 : 4; static constexpr int kScaleBits = CPLX ? 21 : 20; };

// One work item (a piece of one brick's points) into the brick's shared-memory region,
// then the region into the FP64 grid.  lev1/lev2 are zero on entry and on return.
template <int W, bool CPLX>
__device__ __forceinline__ void spread_piece(const SpreadArgs& a, const KbPoly& poly, const int4 wk, int* lev1,
                                             float* lev2, float* s_red) {
    constexpr int BZ = Brick<!CPLX>::BZ;           // the kernel channel is the real one
    constexpr int RG = kBrick + W;
    constexpr int RG3 = RG * RG * (BZ + W);
    constexpr int NC = CPLX ? 2 : 1;
    constexpr float kMagic = 12582912.0f;          // 1.5 * 2^23
    constexpr int kMagicBits = 0x4B400000;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int b = wk.x;
    const int bx = b % a.nb, by = (b / a.nb) % a.nb, bz = b / (a.nb * a.nb);
    const int lo0 = bx * kBrick, lo1 = by * kBrick, lo2 = bz * BZ;
    // the piece is ordered round-robin over bank classes: thread i takes points
    // i, i + 256, ... (every thread the same count, up to one)
    const uint32_t s0 = (uint32_t)wk.y + threadIdx.x;
    const int my_n = wk.z > (int)threadIdx.x ? (wk.z - (int)threadIdx.x + kSpreadThreads - 1) / kSpreadThreads : 0;
    float wmax = a.wmax_fixed;
    if (wmax <= 0.0f) {
        if (CPLX) {
            // the piece's A*b weights sit in its own window of samples_b (scatter order):
            // read it straight, coalesced, instead of through the ids and permutation
            for (int j = threadIdx.x; j < wk.z; j += kSpreadThreads) {
                const float2 wv = __ldg(&a.samples_b[wk.y + j]);
                wmax = fmaxf(wmax, fmaxf(fabsf(wv.x), fabsf(wv.y)));
            }
        } else {
            for (int i = 0; i < my_n; ++i) {
                const uint32_t id = __ldg(&a.payload[s0 + kSpreadThreads * i]);
                const float2 wv = point_weight(a, CPLX, (int)(id >> kTBits), (int)(id & ((1u << kTBits) - 1u)),
                                               (uint32_t)wk.y, s0 + kSpreadThreads * i);
                wmax = fmaxf(wmax, fmaxf(fabsf(wv.x), fabsf(wv.y)));
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) wmax = fmaxf(wmax, __shfl_xor_sync(0xffffffffu, wmax, o));
        if (lane == 0) s_red[warp] = wmax;
        __syncthreads();
        wmax = s_red[0];
#pragma unroll
        for (int i = 1; i < kSpreadWarps; ++i) wmax = fmaxf(wmax, s_red[i]);
    }
    constexpr int PPR = SpreadRound<CPLX>::PPR, SB = SpreadRound<CPLX>::kScaleBits;
    const int rounds = (((wk.z + kSpreadThreads - 1) / kSpreadThreads) + PPR - 1) / PPR;
    int ex = 0;
    if (wmax > 0.0f) frexpf(wmax, &ex);                // wmax <= 2^ex
    const float S = ldexpf(1.0f, SB - ex), invS = ldexpf(1.0f, ex - SB);
    for (int r = 0; r < rounds; ++r) {
#pragma unroll 2
        for (int q = 0; q < PPR; ++q) {
            const int i = PPR * r + q;
            // the warp's 32 lanes take 32 consecutive points of the piece (one warp step)
            const bool live = i < my_n;
            uint32_t id = 0;
            PointPos p{};
            int base = -1;
            if (live) {
                id = __ldg(&a.payload[s0 + kSpreadThreads * i]);
                p = point_pos(a.geom[id >> kTBits], __ldg(&a.htab[id & ((1u << kTBits) - 1u)]), a.scale, a.halfG,
                              a.G);
                base = region_base<W, BZ>(p, lo0, lo1, lo2);
                if (base < 0) atomicOr(&a.counters[2], 1);   // point outside its brick: reported, never written
            }
            // rank among the lanes of this step with the same bank class (base mod 32):
            // a point of rank s starts at window plane s (mod W), so points of one class
            // take different planes (offset RG^2 = 4 banks at W = 6) at every tap step
            // instead of repeating one bank together
            const int sh = class_rank<W>(base, lane);
            if (base < 0) continue;
            const int m = (int)(id >> kTBits);
            const int t = (int)(id & ((1u << kTBits) - 1u));
            const float2 wv = point_weight(a, CPLX, m, t, (uint32_t)wk.y, s0 + kSpreadThreads * i);
            float wx[W], wy[W], wz[W];
            window_taps<W>(poly, p.f[0], wx);
            window_taps<W>(poly, p.f[1], wy);
            window_taps<W>(poly, p.f[2], wz);
            const float dth = CPLX ? 0.0f : point_dither(id);
#pragma unroll
            for (int r = 1; r < W; ++r)
                if (r <= sh) {
                    const float t0 = wz[0];
#pragma unroll
                    for (int k = 0; k < W - 1; ++k) wz[k] = wz[k + 1];
                    wz[W - 1] = t0;
                }
            const float2 w2 = make_float2(wv.x * S, wv.y * S);
            const float2 magic2 = make_float2(kMagic, kMagic);
            const float2 d2 = make_float2(dth, dth);
#pragma unroll
            for (int k = 0; k < W; ++k) {
                const int dz = k + sh < W ? k + sh : k + sh - W;
                const float2 abz = __fmul2_rn(w2, make_float2(wz[k], wz[k]));
                int* plane = lev1 + base + dz * (RG * RG);
#pragma unroll
                for (int dy = 0; dy < W; ++dy) {
                    const float2 abyz = __fmul2_rn(abz, make_float2(wy[dy], wy[dy]));
                    int* row = plane + dy * RG;
                    if (CPLX) {
#pragma unroll
                        for (int dx = 0; dx < W; ++dx) {
                            const float2 v = __ffma2_rn(abyz, make_float2(wx[dx], wx[dx]), magic2);
                            atomicAdd(row + dx, __float_as_int(v.x) - kMagicBits);
                            atomicAdd(row + RG3 + dx, __float_as_int(v.y) - kMagicBits);
                        }
                    } else {
                        const float2 a2 = make_float2(abyz.x, abyz.x);
#pragma unroll
                        for (int dx = 0; dx + 1 < W; dx += 2) {
                            const float2 v = __fadd2_rn(__ffma2_rn(a2, make_float2(wx[dx], wx[dx + 1]), d2), magic2);
                            atomicAdd(row + dx, __float_as_int(v.x) - kMagicBits);
                            atomicAdd(row + dx + 1, __float_as_int(v.y) - kMagicBits);
                        }
                        if (W & 1)
                            atomicAdd(row + W - 1,
                                      __float_as_int(__fadd_rn(fmaf(abyz.x, wx[W - 1], dth), kMagic)) - kMagicBits);
                    }
                }
            }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < NC * RG3; i += blockDim.x) {
            const int v = lev1[i];
            if (v != 0) {
                lev2[i] = fmaf((float)v, invS, lev2[i]);
                lev1[i] = 0;
            }
        }
        __syncthreads();
    }
    // add level 2 into the FP64 grid (periodic wrap) and clear it
    const int o0 = lo0 - W / 2, o1 = lo1 - W / 2, o2 = lo2 - W / 2;
    for (int i = threadIdx.x; i < RG3; i += blockDim.x) {
        const float vr = lev2[i];
        const float vi = CPLX ? lev2[RG3 + i] : 0.0f;
        lev2[i] = 0.0f;
        if (CPLX) lev2[RG3 + i] = 0.0f;
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

template <int W, bool CPLX>
__global__ void __launch_bounds__(kSpreadThreads, CPLX ? 5 : 6) k_spread(const SpreadArgs a) {
    constexpr int NC = CPLX ? 2 : 1;
    constexpr int R3 = (kBrick + W) * (kBrick + W) * (Brick<!CPLX>::BZ + W);
    extern __shared__ int sm_i[];
    int* lev1 = sm_i;                                  // NC * R3 int32
    float* lev2 = reinterpret_cast<float*>(sm_i + NC * R3);   // NC * R3 float
    __shared__ int s_item;
    __shared__ float s_red[kSpreadWarps];
    for (int i = threadIdx.x; i < 2 * NC * R3; i += blockDim.x) sm_i[i] = 0;
    const int n_work = a.counters[0];
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = atomicAdd(&a.counters[1], 1);
        __syncthreads();
        const int item = s_item;
        if (item >= n_work) break;
        spread_piece<W, CPLX>(a, a.poly, a.work[item], lev1, lev2, s_red);
    }
}

// Persistent spreading over the work items of several plans: one queue, items of plan
// p numbered item_off[p] .. item_off[p + 1] - 1 (plans in the order given).
template <int W, bool CPLX>
__global__ void __launch_bounds__(kSpreadThreads, CPLX ? 5 : 6) k_spread_batch(const SpreadArgs* __restrict__ desc, int n,
                                                                 const int* __restrict__ item_off, int* queue,
                                                                 const KbPoly poly) {
    constexpr int NC = CPLX ? 2 : 1;
    constexpr int R3 = (kBrick + W) * (kBrick + W) * (Brick<!CPLX>::BZ + W);
    extern __shared__ int sm_i[];
    int* lev1 = sm_i;
    float* lev2 = reinterpret_cast<float*>(sm_i + NC * R3);
    __shared__ int s_item, s_prob;
    __shared__ float s_red[kSpreadWarps];
    for (int i = threadIdx.x; i < 2 * NC * R3; i += blockDim.x) sm_i[i] = 0;
    const int total = item_off[n];
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) {
            const int g = atomicAdd(queue, 1);
            int lo = 0, hi = n;                        // last p with item_off[p] <= g
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (__ldg(&item_off[mid]) <= g) lo = mid; else hi = mid;
            }
            s_item = g;
            s_prob = lo;
        }
        __syncthreads();
        const int g = s_item;
        if (g >= total) break;
        const int pi = s_prob;
        const SpreadArgs a = desc[pi];
        spread_piece<W, CPLX>(a, poly, a.work[g - __ldg(&item_off[pi])], lev1, lev2, s_red);
    }
}

// item_off = exclusive prefix of the plans' work-item counts; queue = 0.  One warp.
__global__ void k_batch_items(const SpreadArgs* __restrict__ desc, int n, int* __restrict__ item_off, int* queue) {
    const int lane = threadIdx.x;
    int carry = 0;
    for (int p0 = 0; p0 < n; p0 += 32) {
        const int p = p0 + lane;
        const int c = p < n ? desc[p].counters[0] : 0;
        int v = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += u;
        }
        if (p < n) item_off[p] = carry + v - c;
        carry += __shfl_sync(0xffffffffu, v, 31);
    }
    if (lane == 0) {
        item_off[n] = carry;
        *queue = 0;
    }
}

// ---------------------------------------------------------------------------
// Both channels in one pass (the fused form of FIRM steps 2-3): the points of the
// kernel channel's binning on the 4N grid (which needs the poses only, so it can run
// while the images are still uploading) carry both weights, h^2 (eq. kernel) and h b
// (eq. backprojection: the image DFT's [m][t] samples, put in the binning's order by
// k_fused_gather), and every window tap is formed once and added to three shared-memory
// planes (Ker; A*b real and imaginary).  Level 2 goes to the FP64 Ker
// grid (real, G^3) and the FP64 A*b grid (complex, G^3, right after it); A*b is then
// read from the 4N grid (oversampling 4 for its N modes).  Fixed point as in
// spread_piece: the kernel channel's scale comes from the largest h^2 of the CTF table,
// the A*b scale from the piece's own largest |h b| (recorded by the gather); PPR points
// per thread between folds.
// ---------------------------------------------------------------------------
// T threads per block (256; the three planes take 66 KB at W = 6, three blocks per SM:
// 512-thread blocks, twice the warps per SM, measured 10% slower); with PPR points per
// thread between folds a cell takes at most T * PPR taps, each at most 2^kScaleBits:
// T * PPR * 2^kScaleBits <= 2^30.  PPR 4 with 20 bits (half the folds of PPR 2 with 21
// bits) measured 2% faster; the Ker plane is dithered, the A*b planes keep their
// per-piece scale.  The points of a thread are taken one at a time (unrolling two
// measured 3% slower).
constexpr int kFusedThreads = 256;
template <int T> struct FusedRound {
    static constexpr int PPR = T >= 512 ? 1 : 4;
    static constexpr int kScaleBits = 20;
    static_assert((long long)T * PPR << kScaleBits <= (1ll << 30), "fold bound");
};

template <int W, int T>
__device__ __forceinline__ void spread_piece_fused(const SpreadArgs& a, const KbPoly& poly, const int item,
                                                   const int4 wk, int* lev1, float* lev2) {
    constexpr int BZ = kBrickZk;
    constexpr int RG = kBrick + W;
    constexpr int RG3 = RG * RG * (BZ + W);
    constexpr float kMagic = 12582912.0f;          // 1.5 * 2^23
    constexpr int kMagicBits = 0x4B400000;
    const int lane = threadIdx.x & 31;
    const int b = wk.x;
    const int bx = b % a.nb, by = (b / a.nb) % a.nb, bz = b / (a.nb * a.nb);
    const int lo0 = bx * kBrick, lo1 = by * kBrick, lo2 = bz * BZ;
    const uint32_t s0 = (uint32_t)wk.y + threadIdx.x;
    const int my_n = wk.z > (int)threadIdx.x ? (wk.z - (int)threadIdx.x + T - 1) / T : 0;
    // largest |h b| of the piece (the A*b scale), found by the gather pass
    const float wmax = __ldg(&a.wmax_item[item]);
    constexpr int PPR = FusedRound<T>::PPR, SB = FusedRound<T>::kScaleBits;
    const int rounds = (((wk.z + T - 1) / T) + PPR - 1) / PPR;
    int ek = 0, eb = 0;
    if (a.wmax_fixed > 0.0f) frexpf(a.wmax_fixed, &ek);
    if (wmax > 0.0f) frexpf(wmax, &eb);
    const float Sk = ldexpf(1.0f, SB - ek), invSk = ldexpf(1.0f, ek - SB);
    const float Sb = ldexpf(1.0f, SB - eb), invSb = ldexpf(1.0f, eb - SB);
    for (int r = 0; r < rounds; ++r) {
#pragma unroll 1
        for (int q = 0; q < PPR; ++q) {
            const int i = PPR * r + q;
            const bool live = i < my_n;
            uint32_t id = 0;
            PointPos p{};
            int base = -1;
            if (live) {
                id = __ldg(&a.payload[s0 + T * i]);
                p = point_pos(a.geom[id >> kTBits], __ldg(&a.htab[id & ((1u << kTBits) - 1u)]), a.scale, a.halfG,
                              a.G);
                base = region_base<W, BZ>(p, lo0, lo1, lo2);
                if (base < 0) atomicOr(&a.counters[2], 1);   // point outside its brick: reported, never written
            }
            // repeated bank classes in a warp step start at different window planes, as
            // in spread_piece
            const int sh = class_rank<W>(base, lane);
            if (base < 0) continue;
            const int m = (int)(id >> kTBits);
            const int t = (int)(id & ((1u << kTBits) - 1u));
            const int g = min(max(__ldg(&a.gid[m]), 0), a.n_ctf - 1);
            const float wk2 = __ldg(&a.h2[(size_t)g * a.nH + t]) * Sk;
            const float2 wv = __ldg(&a.samples_b[s0 + T * i]);     // gathered in payload order
            const float2 w2 = make_float2(wv.x * Sb, wv.y * Sb);
            const float dth = point_dither(id);
            float wx[W], wy[W], wz[W];
            window_taps<W>(poly, p.f[0], wx);
            window_taps<W>(poly, p.f[1], wy);
            window_taps<W>(poly, p.f[2], wz);
#pragma unroll
            for (int rr = 1; rr < W; ++rr)
                if (rr <= sh) {
                    const float t0 = wz[0];
#pragma unroll
                    for (int k = 0; k < W - 1; ++k) wz[k] = wz[k + 1];
                    wz[W - 1] = t0;
                }
            const float2 magic2 = make_float2(kMagic, kMagic);
            const float2 d2 = make_float2(dth, dth);
#pragma unroll
            for (int k = 0; k < W; ++k) {
                const int dz = k + sh < W ? k + sh : k + sh - W;
                const float kz = wk2 * wz[k];
                const float2 abz = __fmul2_rn(w2, make_float2(wz[k], wz[k]));
                int* plane = lev1 + base + dz * (RG * RG);
#pragma unroll
                for (int dy = 0; dy < W; ++dy) {
                    const float kyz = kz * wy[dy];
                    const float2 abyz = __fmul2_rn(abz, make_float2(wy[dy], wy[dy]));
                    int* row = plane + dy * RG;
                    const float2 k2 = make_float2(kyz, kyz);
#pragma unroll
                    for (int dx = 0; dx + 1 < W; dx += 2) {
                        const float2 v = __fadd2_rn(__ffma2_rn(k2, make_float2(wx[dx], wx[dx + 1]), d2), magic2);
                        atomicAdd(row + dx, __float_as_int(v.x) - kMagicBits);
                        atomicAdd(row + dx + 1, __float_as_int(v.y) - kMagicBits);
                    }
                    if (W & 1)
                        atomicAdd(row + W - 1, __float_as_int(__fadd_rn(fmaf(kyz, wx[W - 1], dth), kMagic)) - kMagicBits);
#pragma unroll
                    for (int dx = 0; dx < W; ++dx) {
                        const float2 v = __ffma2_rn(abyz, make_float2(wx[dx], wx[dx]), magic2);
                        atomicAdd(row + RG3 + dx, __float_as_int(v.x) - kMagicBits);
                        atomicAdd(row + 2 * RG3 + dx, __float_as_int(v.y) - kMagicBits);
                    }
                }
            }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < 3 * RG3; i += blockDim.x) {
            const int v = lev1[i];
            if (v != 0) {
                lev2[i] = fmaf((float)v, i < RG3 ? invSk : invSb, lev2[i]);
                lev1[i] = 0;
            }
        }
        __syncthreads();
    }
    // level 2 into the FP64 grids (periodic wrap) and cleared
    const int o0 = lo0 - W / 2, o1 = lo1 - W / 2, o2 = lo2 - W / 2;
    double* gk = a.grid;
    double* gb = a.grid + (size_t)a.G * a.G * a.G;
    for (int i = threadIdx.x; i < RG3; i += blockDim.x) {
        const float vk = lev2[i], vr = lev2[RG3 + i], vi = lev2[2 * RG3 + i];
        lev2[i] = 0.0f;
        lev2[RG3 + i] = 0.0f;
        lev2[2 * RG3 + i] = 0.0f;
        if (vk == 0.0f && vr == 0.0f && vi == 0.0f) continue;
        const int rx = i % RG, ry = (i / RG) % RG, rz = i / (RG * RG);
        int gx = o0 + rx, gy = o1 + ry, gz = o2 + rz;
        gx += (gx < 0) ? a.G : 0;
        gx -= (gx >= a.G) ? a.G : 0;
        gy += (gy < 0) ? a.G : 0;
        gy -= (gy >= a.G) ? a.G : 0;
        gz += (gz < 0) ? a.G : 0;
        gz -= (gz >= a.G) ? a.G : 0;
        const size_t cell = ((size_t)gz * a.G + gy) * a.G + gx;
        if (vk != 0.0f) atomicAdd(&gk[cell], (double)vk);
        if (vr != 0.0f) atomicAdd(&gb[2 * cell], (double)vr);
        if (vi != 0.0f) atomicAdd(&gb[2 * cell + 1], (double)vi);
    }
    __syncthreads();
}

template <int W>
__global__ void __launch_bounds__(kFusedThreads) k_spread_fused(const SpreadArgs a) {
    constexpr int R3 = (kBrick + W) * (kBrick + W) * (kBrickZk + W);
    extern __shared__ int sm_i[];
    int* lev1 = sm_i;                                          // 3 * R3 int32
    float* lev2 = reinterpret_cast<float*>(sm_i + 3 * R3);     // 3 * R3 float
    __shared__ int s_item;
    for (int i = threadIdx.x; i < 6 * R3; i += blockDim.x) sm_i[i] = 0;
    const int n_work = a.counters[0];
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = atomicAdd(&a.counters[1], 1);
        __syncthreads();
        const int item = s_item;
        if (item >= n_work) break;
        spread_piece_fused<W, kFusedThreads>(a, a.poly, item, a.work[item], lev1, lev2);
    }
}

// The fused pass's A*b weights in payload order (samples_b[pos] = h b of the point at
// pos, one gathered 8-byte read per point) and each work item's largest |h b| (its
// fixed-point scale), so the spreading pass reads both coalesced.
__global__ void __launch_bounds__(256) k_fused_gather(const uint32_t* __restrict__ scat,
                                                      const uint16_t* __restrict__ inv_perm,
                                                      const int4* __restrict__ work, const int* __restrict__ counters,
                                                      const float2* __restrict__ samples, int nH,
                                                      float2* __restrict__ samples_b, float* __restrict__ wmax_item) {
    __shared__ float s_red[8];
    const int n_work = counters[0];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int item = blockIdx.x; item < n_work; item += gridDim.x) {
        const int4 wk = work[item];
        float wmax = 0.0f;
        // the points in scatter order (an image's points of this brick together: their
        // weights share sectors), each written to its sorted position
        for (int i = threadIdx.x; i < wk.z; i += blockDim.x) {
            const uint32_t id = __ldg(&scat[wk.y + i]);
            const float2 v = __ldg(&samples[(size_t)(id >> kTBits) * nH + (id & ((1u << kTBits) - 1u))]);
            samples_b[wk.y + __ldg(&inv_perm[wk.y + i])] = v;
            wmax = fmaxf(wmax, fmaxf(fabsf(v.x), fabsf(v.y)));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) wmax = fmaxf(wmax, __shfl_xor_sync(0xffffffffu, wmax, o));
        if (lane == 0) s_red[warp] = wmax;
        __syncthreads();
        if (threadIdx.x == 0) {
            float m = s_red[0];
            for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, s_red[w]);
            wmax_item[item] = m;
        }
        __syncthreads();
    }
}

template <int W>
static cudaError_t spread_fused_w(Plan& P, const SpreadArgs& a) {
    constexpr int R3 = (kBrick + W) * (kBrick + W) * (kBrickZk + W);
    const size_t smem = sizeof(int) * 6 * R3;
    cudaError_t e = cudaFuncSetAttribute(k_spread_fused<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_spread_fused<W>, kFusedThreads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    k_spread_fused<W><<<P.num_sms * per_sm, kFusedThreads, smem, P.stream>>>(a);
    P.launches += 1;
    return cudaGetLastError();
}

template <int W, bool CPLX>
static size_t spread_smem() {
    constexpr int R3 = (kBrick + W) * (kBrick + W) * (Brick<!CPLX>::BZ + W);
    return sizeof(int) * R3 * (CPLX ? 2 : 1) * 2;
}

template <int W, bool CPLX>
static cudaError_t spread_w(Plan& P, const SpreadArgs& a) {
    const size_t smem = spread_smem<W, CPLX>();
    cudaError_t e = cudaFuncSetAttribute(k_spread<W, CPLX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_spread<W, CPLX>, kSpreadThreads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    k_spread<W, CPLX><<<P.num_sms * per_sm, kSpreadThreads, smem, P.stream>>>(a);
    P.launches += 1;
    return cudaGetLastError();
}

template <int W, bool CPLX>
static cudaError_t spread_batch_w(int n, const SpreadArgs* desc, int* item_off, int* queue, const KbPoly& poly,
                                  int num_sms, cudaStream_t s) {
    const size_t smem = spread_smem<W, CPLX>();
    cudaError_t e = cudaFuncSetAttribute(k_spread_batch<W, CPLX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_spread_batch<W, CPLX>, kSpreadThreads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    k_batch_items<<<1, 32, 0, s>>>(desc, n, item_off, queue);
    k_spread_batch<W, CPLX><<<num_sms * per_sm, kSpreadThreads, smem, s>>>(desc, n, item_off, queue, poly);
    return cudaGetLastError();
}

static SpreadArgs spread_args(Plan& P, bool kc) {
    Workspace& w = P.ws;
    const int G = kc ? P.Gk : P.Gr;
    SpreadArgs a;
    a.payload = w.payload;
    a.work = w.work;
    a.counters = w.counters;
    a.geom = w.geom;
    a.htab = w.htab;
    a.gid = P.cur_gid;
    a.h2 = w.h2;
    a.samples_b = w.samples_b;
    a.samples = w.samples;
    a.perm = w.perm;
    a.grid = w.grid;
    a.G = G;
    a.halfG = G / 2;
    a.nb = kc ? P.nbk : P.nbr;
    a.nH = P.nH;
    a.n_ctf = P.n_ctf;
    a.scale = (float)(G / P.N);
    a.wmax_fixed = kc ? P.h2_max : 0.0f;
    a.wmax_item = nullptr;
    a.poly = P.poly;
    return a;
}

cudaError_t launch_spread_clear(Plan& P, bool kc) {
    const int G = kc ? P.Gk : P.Gr;
    const size_t cells = (size_t)G * G * G * (kc ? 1 : 2);
    return cudaMemsetAsync(P.ws.grid, 0, sizeof(double) * cells, P.stream);
}

cudaError_t launch_spread_only(Plan& P, int M, bool kc) {
    if (M <= 0) return cudaSuccess;
    const SpreadArgs a = spread_args(P, kc);
    switch (P.p.W) {
        case 6: return kc ? spread_w<6, false>(P, a) : spread_w<6, true>(P, a);
        case 7: return kc ? spread_w<7, false>(P, a) : spread_w<7, true>(P, a);
        case 8: return kc ? spread_w<8, false>(P, a) : spread_w<8, true>(P, a);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_spread(Plan& P, int M, bool kc) {
    cudaError_t e = launch_spread_clear(P, kc);
    if (e != cudaSuccess) return e;
    return launch_spread_only(P, M, kc);
}

cudaError_t launch_fused_gather(Plan& P, int M) {
    if (M <= 0) return cudaSuccess;
    Workspace& w = P.ws;
    if (!w.payload_scat) return cudaErrorInvalidValue;      // fused plans only
    k_fused_gather<<<P.num_sms * 8, 256, 0, P.stream>>>(w.payload_scat, w.inv_perm, w.work, w.counters, w.samples,
                                                       P.nH, w.samples_b, w.wmax_item);
    P.launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_spread_fused(Plan& P, int M) {
    const size_t cells = (size_t)P.Gk * P.Gk * P.Gk;
    cudaError_t e = cudaMemsetAsync(P.ws.grid, 0, sizeof(double) * 3 * cells, P.stream);
    if (e != cudaSuccess || M <= 0) return e;
    SpreadArgs a = spread_args(P, true);
    a.samples_b = P.ws.samples_b;
    a.wmax_item = P.ws.wmax_item;
    switch (P.p.W) {
        case 6: return spread_fused_w<6>(P, a);
        case 7: return spread_fused_w<7>(P, a);
        case 8: return spread_fused_w<8>(P, a);
        default: return cudaErrorInvalidValue;
    }
}

size_t spread_batch_desc_bytes() { return sizeof(SpreadArgs); }

void spread_batch_fill_desc(Plan& P, bool kc, void* host_desc) {
    *reinterpret_cast<SpreadArgs*>(host_desc) = spread_args(P, kc);
}

cudaError_t launch_spread_batch(int n, bool kc, int W, const KbPoly& poly, const void* dev_desc, int* item_off,
                                int* queue, int num_sms, cudaStream_t s) {
    const SpreadArgs* d = reinterpret_cast<const SpreadArgs*>(dev_desc);
    switch (W) {
        case 6: return kc ? spread_batch_w<6, false>(n, d, item_off, queue, poly, num_sms, s)
                          : spread_batch_w<6, true>(n, d, item_off, queue, poly, num_sms, s);
        case 7: return kc ? spread_batch_w<7, false>(n, d, item_off, queue, poly, num_sms, s)
                          : spread_batch_w<7, true>(n, d, item_off, queue, poly, num_sms, s);
        case 8: return kc ? spread_batch_w<8, false>(n, d, item_off, queue, poly, num_sms, s)
                          : spread_batch_w<8, true>(n, d, item_off, queue, poly, num_sms, s);
        default: return cudaErrorInvalidValue;
    }
}


// ---------------------------------------------------------------------------
// Interpolation (the forward projector's type-2 NUFFT, the transpose of spreading):
// (A V)(xi) = sum over the W^3 cells j around the point of phi(j - y) g[j], g the
// forward-transformed, deconvolved volume on the centred 2N grid.  Per work item (one
// 8^3 brick of the A*b binning) the brick's (8+W)^3 region of g is staged in shared
// memory (real and imaginary planes; the bank-class order of the piece keeps a warp's
// lanes on distinct banks) and each thread gathers its points' taps.  Forward mode
// writes h_m(k) (A V) at [m][t]; residual mode reads b (the unweighted image DFT in
// scatter order) and sums c |b - h A V|^2 and c |b|^2 per work item (c = 2 off the
// origin: the other half of the disc is the complex conjugate).
// ---------------------------------------------------------------------------
struct InterpArgs {
    const uint32_t* payload;
    const int4* work;
    int* counters;
    const ImgGeom* geom;
    const int32_t* htab;
    const int32_t* gid;
    const float* h1;          // [group][t] h
    const float2* ghat;       // G^3 complex, [j3][j2][j1] on the centred grid
    const float2* samples_b;  // residual mode: b in scatter order
    const uint16_t* perm;
    float2* out;              // forward mode: [m][t]
    double* item_part;        // residual mode: per work item (sum c|r|^2, sum c|b|^2)
    int G, halfG, nb, nH, n_ctf;
    float scale;
    KbPoly poly;
};

template <int W, bool RESID>
__global__ void __launch_bounds__(kSpreadThreads) k_interp(const InterpArgs a) {
    constexpr int BZ = kBrick;
    constexpr int RG = kBrick + W;
    constexpr int RG3 = RG * RG * (BZ + W);
    extern __shared__ float s_f[];
    float* s_re = s_f;
    float* s_im = s_f + RG3;
    __shared__ int s_item;
    __shared__ double s_red[2][kSpreadWarps];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int n_work = a.counters[0];
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = atomicAdd(&a.counters[1], 1);
        __syncthreads();
        const int item = s_item;
        if (item >= n_work) break;
        const int4 wk = a.work[item];
        const int b = wk.x;
        const int bx = b % a.nb, by = (b / a.nb) % a.nb, bz = b / (a.nb * a.nb);
        const int lo0 = bx * kBrick, lo1 = by * kBrick, lo2 = bz * BZ;
        const int o0 = lo0 - W / 2, o1 = lo1 - W / 2, o2 = lo2 - W / 2;
        for (int i = threadIdx.x; i < RG3; i += blockDim.x) {
            const int rx = i % RG, ry = (i / RG) % RG, rz = i / (RG * RG);
            int gx = o0 + rx, gy = o1 + ry, gz = o2 + rz;
            gx += (gx < 0) ? a.G : 0;
            gx -= (gx >= a.G) ? a.G : 0;
            gy += (gy < 0) ? a.G : 0;
            gy -= (gy >= a.G) ? a.G : 0;
            gz += (gz < 0) ? a.G : 0;
            gz -= (gz >= a.G) ? a.G : 0;
            const float2 v = __ldg(&a.ghat[((size_t)gz * a.G + gy) * a.G + gx]);
            s_re[i] = v.x;
            s_im[i] = v.y;
        }
        __syncthreads();
        double acc_r = 0.0, acc_b = 0.0;
        for (int i = threadIdx.x; i < wk.z; i += blockDim.x) {
            const uint32_t pos = (uint32_t)wk.y + i;
            const uint32_t id = __ldg(&a.payload[pos]);
            const int m = (int)(id >> kTBits);
            const int t = (int)(id & ((1u << kTBits) - 1u));
            const PointPos p = point_pos(a.geom[m], __ldg(&a.htab[t]), a.scale, a.halfG, a.G);
            const int base = region_base<W, BZ>(p, lo0, lo1, lo2);
            if (base < 0) {
                atomicOr(&a.counters[2], 1);   // point outside its brick: reported, never read
                continue;
            }
            float wx[W], wy[W], wz[W];
            window_taps<W>(a.poly, p.f[0], wx);
            window_taps<W>(a.poly, p.f[1], wy);
            window_taps<W>(a.poly, p.f[2], wz);
            float fr = 0.0f, fi = 0.0f;
#pragma unroll
            for (int dz = 0; dz < W; ++dz) {
#pragma unroll
                for (int dy = 0; dy < W; ++dy) {
                    const int row = base + (dz * RG + dy) * RG;
                    float rr = 0.0f, ri = 0.0f;
#pragma unroll
                    for (int dx = 0; dx < W; ++dx) {
                        rr = fmaf(wx[dx], s_re[row + dx], rr);
                        ri = fmaf(wx[dx], s_im[row + dx], ri);
                    }
                    const float wyz = wz[dz] * wy[dy];
                    fr = fmaf(wyz, rr, fr);
                    fi = fmaf(wyz, ri, fi);
                }
            }
            const int g = a.gid ? min(max(__ldg(&a.gid[m]), 0), a.n_ctf - 1) : 0;
            const float h = __ldg(&a.h1[(size_t)g * a.nH + t]);
            if (!RESID) {
                a.out[(size_t)m * a.nH + t] = make_float2(h * fr, h * fi);
            } else {
                const float2 bv = __ldg(&a.samples_b[wk.y + __ldg(&a.perm[pos])]);
                const double dr = (double)bv.x - (double)h * fr, di = (double)bv.y - (double)h * fi;
                const double c = t == 0 ? 1.0 : 2.0;
                acc_r += c * (dr * dr + di * di);
                acc_b += c * ((double)bv.x * bv.x + (double)bv.y * bv.y);
            }
        }
        if (RESID) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                acc_r += __shfl_xor_sync(0xffffffffu, acc_r, o);
                acc_b += __shfl_xor_sync(0xffffffffu, acc_b, o);
            }
            if (lane == 0) {
                s_red[0][warp] = acc_r;
                s_red[1][warp] = acc_b;
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                double r = 0.0, bb = 0.0;
                for (int w = 0; w < kSpreadWarps; ++w) { r += s_red[0][w]; bb += s_red[1][w]; }
                a.item_part[2 * item] = r;
                a.item_part[2 * item + 1] = bb;
            }
        }
    }
}

// out[0..1] = sums over the work items, in item order (one CTA: fixed order).
__global__ void __launch_bounds__(1024) k_item_sum(const double* __restrict__ part, const int* __restrict__ counters,
                                                   double* __restrict__ out) {
    __shared__ double s[2][1024];
    const int n = counters[0];
    double r = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        r += part[2 * i];
        b += part[2 * i + 1];
    }
    s[0][threadIdx.x] = r;
    s[1][threadIdx.x] = b;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if ((int)threadIdx.x < k) {
            s[0][threadIdx.x] += s[0][threadIdx.x + k];
            s[1][threadIdx.x] += s[1][threadIdx.x + k];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = s[0][0];
        out[1] = s[1][0];
    }
}

template <int W, bool RESID>
static cudaError_t interp_w(Plan& P, const InterpArgs& a) {
    constexpr int RG3 = (kBrick + W) * (kBrick + W) * (kBrick + W);
    const size_t smem = sizeof(float) * 2 * RG3;
    cudaError_t e = cudaFuncSetAttribute(k_interp<W, RESID>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_interp<W, RESID>, kSpreadThreads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    k_interp<W, RESID><<<P.num_sms * per_sm, kSpreadThreads, smem, P.stream>>>(a);
    P.launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_interp(Plan& P, int M, const float2* ghat, float2* out, double* item_part, double* sums) {
    if (M <= 0) return cudaSuccess;
    Workspace& w = P.ws;
    InterpArgs a;
    a.payload = w.payload;
    a.work = w.work;
    a.counters = w.counters;
    a.geom = w.geom;
    a.htab = w.htab;
    a.gid = P.cur_gid;
    a.h1 = w.h1;
    a.ghat = ghat;
    a.samples_b = w.samples_b;
    a.perm = w.perm;
    a.out = out;
    a.item_part = item_part;
    a.G = P.Gr;
    a.halfG = P.Gr / 2;
    a.nb = P.nbr;
    a.nH = P.nH;
    a.n_ctf = P.n_ctf;
    a.scale = (float)(P.Gr / P.N);
    a.poly = P.poly;
    const bool resid = item_part != nullptr;
    cudaError_t e;
    switch (P.p.W) {
        case 6: e = resid ? interp_w<6, true>(P, a) : interp_w<6, false>(P, a); break;
        case 7: e = resid ? interp_w<7, true>(P, a) : interp_w<7, false>(P, a); break;
        case 8: e = resid ? interp_w<8, true>(P, a) : interp_w<8, false>(P, a); break;
        default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess || !resid) return e;
    k_item_sum<<<1, 1024, 0, P.stream>>>(item_part, w.counters, sums);
    P.launches += 1;
    return cudaGetLastError();
}

}  // namespace firm
