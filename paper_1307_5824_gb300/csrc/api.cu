// api.cu -- the C ABI of include/firm.h: plan, workspace layout, host tables, staging
// of host inputs, and the FIRM steps (Section 3.4) in stream order.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "firm_internal.h"

namespace firm {

static const double kPi = 3.14159265358979323846;

// ---------------------------------------------------------------------------
// Host tables
// ---------------------------------------------------------------------------

// Modified Bessel function I0 by its defining power series sum (x^2/4)^k / (k!)^2.
static double bessel_i0(double x) {
    const double q = 0.25 * x * x;
    double term = 1.0, sum = 1.0;
    for (int k = 1; k < 200; ++k) {
        term *= q / ((double)k * (double)k);
        sum += term;
        if (term < 1e-17 * sum) break;
    }
    return sum;
}

static double kb_beta(int W, double sigma) {
    // Beatty, Nishimura & Pauly (2005): beta = pi sqrt((W/sigma)^2 (sigma - 1/2)^2 - 0.8)
    const double a = (double)W / sigma * (sigma - 0.5);
    return kPi * std::sqrt(a * a - 0.8);
}

static double kb_phi(double t, int W, double beta, double norm) {
    const double s = 2.0 * t / W;
    if (std::fabs(s) > 1.0) return 0.0;
    return bessel_i0(beta * std::sqrt(1.0 - s * s)) / norm;
}

// Chebyshev interpolation of each tap's weight phi(u + l - W/2), u = (z+1)/2, on
// kKbDeg+1 Chebyshev nodes, converted to monomials in z (Horner on the device).
void kb_build(int W, double sigma, KbPoly& poly, double* beta_out) {
    const double beta = kb_beta(W, sigma);
    const double norm = bessel_i0(beta);
    constexpr int D = kKbDeg;
    std::memset(&poly, 0, sizeof(poly));
    for (int l = 0; l < W; ++l) {
        double f[D + 1], cheb[D + 1];
        for (int j = 0; j <= D; ++j) {
            const double z = std::cos(kPi * (j + 0.5) / (D + 1));
            f[j] = kb_phi(0.5 * (z + 1.0) + l - 0.5 * W, W, beta, norm);
        }
        for (int k = 0; k <= D; ++k) {
            double s = 0.0;
            for (int j = 0; j <= D; ++j) s += f[j] * std::cos(kPi * k * (j + 0.5) / (D + 1));
            cheb[k] = (k == 0 ? 1.0 : 2.0) * s / (D + 1);
        }
        // T_k -> monomials: T_0 = 1, T_1 = z, T_{k+1} = 2 z T_k - T_{k-1}
        double Tm1[D + 1] = {0}, T0[D + 1] = {0}, T1[D + 1] = {0}, mono[D + 1] = {0};
        T0[0] = 1.0;
        for (int k = 0; k <= D; ++k) {
            const double* Tk = (k == 0) ? T0 : T1;
            for (int j = 0; j <= D; ++j) mono[j] += cheb[k] * Tk[j];
            if (k == 0) {
                std::memset(T1, 0, sizeof(T1));
                T1[1] = 1.0;
                std::memcpy(Tm1, T0, sizeof(T0));
            } else {
                double Tn[D + 1] = {0};
                for (int j = 0; j < D; ++j) Tn[j + 1] += 2.0 * T1[j];
                for (int j = 0; j <= D; ++j) Tn[j] -= Tm1[j];
                std::memcpy(Tm1, T1, sizeof(T1));
                std::memcpy(T1, Tn, sizeof(Tn));
            }
        }
        for (int j = 0; j <= D; ++j) poly.c[l][j] = (float)mono[j];
    }
    if (beta_out) *beta_out = beta;
}

// Fourier transform of the normalised window, int phi(t) exp(-2 pi i u t) dt
//   = W sinh(sqrt(beta^2 - (pi W u)^2)) / sqrt(beta^2 - (pi W u)^2) / I0(beta).
double kb_phihat(double u, int W, double beta) {
    const double a = beta * beta - (kPi * W * u) * (kPi * W * u);
    double v;
    if (a > 1e-12) { const double s = std::sqrt(a); v = std::sinh(s) / s; }
    else if (a < -1e-12) { const double s = std::sqrt(-a); v = std::sin(s) / s; }
    else v = 1.0;
    return W * v / bessel_i0(beta);
}

std::vector<int32_t> half_disc(int N) {
    // k = (0,0); (0, k2) for k2 = 1..N/2; then k1 = 1..N/2 with all k2 in the disc
    std::vector<int32_t> h;
    const int hN = N / 2;
    auto pack = [](int k1, int k2) { return (int32_t)((uint32_t)(k1 & 0xffff) | ((uint32_t)k2 << 16)); };
    for (int k2 = 0; k2 <= hN; ++k2) h.push_back(pack(0, k2));
    for (int k1 = 1; k1 <= hN; ++k1)
        for (int k2 = -hN; k2 <= hN; ++k2)
            if (k1 * k1 + k2 * k2 <= hN * hN) h.push_back(pack(k1, k2));
    return h;
}

double wavelength_A(double kV) {
    const double U = kV * 1e3, h = 6.62607015e-34, m = 9.1093837015e-31, e = 1.602176634e-19, c = 299792458.0;
    return h / std::sqrt(2.0 * m * e * U * (1.0 + e * U / (2.0 * m * c * c))) * 1e10;
}

double ctf_value(const firm_ctf_group& g, double r) {
    const double lam = wavelength_A(g.kV);
    const double cs = g.Cs_mm * 1e7;
    const double r2 = r * r;
    const double chi = kPi * lam * g.defocus_A * r2 - 0.5 * kPi * cs * lam * lam * lam * r2 * r2;
    return -std::sin(chi + g.amp_contrast) * std::exp(-g.bfactor_A2 * r2 / 4.0);
}

// ---------------------------------------------------------------------------
// Workspace layout
// ---------------------------------------------------------------------------
static int disc_size(int N) {
    int c = 0;
    const int h = N / 2;
    for (int k1 = -h; k1 <= h; ++k1)
        for (int k2 = -h; k2 <= h; ++k2) c += (k1 * k1 + k2 * k2 <= h * h);
    return c;
}

struct Carver {
    char* base;
    size_t off = 0;
    template <class T> T* take(size_t count) {
        off = (off + 255) & ~(size_t)255;
        T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
        off += count * sizeof(T);
        return p;
    }
};

size_t layout_workspace(const firm_params& p, char* base, Workspace& w) {
    const size_t N = p.N, M = p.M;
    const size_t nH = (size_t)(disc_size(p.N) + 1) / 2;
    const size_t n_ctf = p.n_groups > 0 ? (size_t)p.n_groups : 1;
    const size_t Gk = 4 * N, Gr = 2 * N;
    const size_t nbk = Gk / kBrick;
    const size_t nb3 = nbk * nbk * nbk;
    const size_t max_work = nb3 + M * nH / kMinChunk + 2;
    const size_t esz = p.img_dtype == FIRM_IMG_BF16 ? 2 : 4;
    const size_t N3 = N * N * N, H3 = 2 * N * 2 * N * (N + 1);
    Carver c{base};
    w.R = c.take<double>(M * 9);
    w.shifts = c.take<double>(M * 2);
    w.gid = c.take<int32_t>(M);
    w.geom = c.take<ImgGeom>(M);
    w.htab = c.take<int32_t>(nH);
    w.colinfo = c.take<int4>(N / 2 + 1);
    w.h2 = c.take<float>(n_ctf * nH);
    w.h1 = c.take<float>(n_ctf * nH);
    w.tw_n = c.take<float2>(N);
    w.tw_2n = c.take<float2>(2 * N);
    w.tw_4n = c.take<float2>(4 * N);
    w.dec_k = c.take<float>(2 * N);
    w.dec_r = c.take<float>(N);
    w.dec_r4 = c.take<float>(N);
    w.samples = c.take<float2>(M * nH);
    w.count = c.take<uint32_t>(nb3);
    w.cursor = c.take<uint32_t>(nb3);
    w.work = c.take<int4>(max_work);
    w.wmax_item = c.take<float>(max_work);
    w.scan_part = c.take<unsigned long long>(2 * (nb3 / kScanSpan + 1));
    w.item_part = c.take<double>(2 * max_work);
    w.counters = c.take<int>(8);
    // FP64 fine grid: Ker (4N^3 real) or A*b (2N^3 complex); the fused form holds both
    // channels on the 4N grid (real Ker, then complex A*b)
    const bool fused = (p.flags & FIRM_FLAG_FUSED) != 0;
    const size_t grid_bytes = std::max(Gk * Gk * Gk * sizeof(double) * (fused ? 3 : 1),
                                       Gr * Gr * Gr * 2 * sizeof(double));
    w.grid = c.take<double>(grid_bytes / sizeof(double));
    // fused plans keep the kernel channel's ids in scatter order for the weight gather
    w.payload_scat = fused ? c.take<uint32_t>(M * nH) : nullptr;
    w.inv_perm = fused ? c.take<uint16_t>(M * nH) : nullptr;
    // union: staged images | point ids | FFT intermediates (never live together)
    const size_t fx1 = std::max({Gk * Gk * (N + 1), Gr * Gr * N, H3});
    const size_t fx2 = std::max({Gk * 2 * N * (N + 1), Gr * N * N, H3});
    // point ids, bank bytes, the A*b weights in scatter order and the sort's permutation
    const size_t ids_bytes = (M * nH * sizeof(uint32_t) + 255) & ~(size_t)255;
    const size_t cls_bytes = (M * nH + 255) & ~(size_t)255;
    const size_t smp_bytes = (M * nH * sizeof(float2) + 255) & ~(size_t)255;
    const size_t pay_bytes = ids_bytes + cls_bytes + smp_bytes + M * nH * sizeof(uint16_t);
    const size_t u_bytes = std::max({M * N * N * esz, pay_bytes, (fx1 + fx2) * sizeof(float2) + 256});
    char* u = c.take<char>(u_bytes);
    w.images = u;
    w.payload = reinterpret_cast<uint32_t*>(u);
    w.cls = u ? reinterpret_cast<uint8_t*>(u + ids_bytes) : nullptr;
    w.samples_b = u ? reinterpret_cast<float2*>(u + ids_bytes + cls_bytes) : nullptr;
    w.perm = u ? reinterpret_cast<uint16_t*>(u + ids_bytes + cls_bytes + smp_bytes) : nullptr;
    w.fx1 = reinterpret_cast<float2*>(u);
    w.fx2 = u ? reinterpret_cast<float2*>(u + ((fx1 * sizeof(float2) + 255) & ~(size_t)255)) : nullptr;
    w.ker = c.take<float>(H3);
    w.khat = c.take<float>(H3);
    w.rhs = c.take<float>(N3);
    w.x = c.take<float>(N3);
    w.r = c.take<float2>(N3);
    w.p = c.take<float>(N3);
    w.q = c.take<float>(N3);
    w.t1 = c.take<float2>(N * N * (N + 1));
    w.t2 = c.take<float2>(N * 2 * N * (N + 1));
    w.z = c.take<float>(N3);
    w.pc_diag = c.take<float>(N * N * (N / 2 + 1) + 1);
    w.pc_feat = c.take<float>(1024);
    w.pc_table = c.take<float>(1024);
    w.pc_s1 = c.take<double>(1024);
    w.pc_s2 = c.take<double>(1024);
    w.red_a = c.take<double>(kRedSlots);
    w.red_b = c.take<double>(kRedSlots);
    w.hist = c.take<double>(kMaxHist);
    w.cg = c.take<CgState>(1);
    w.lam = c.take<float>(2);
    w.axis = c.take<float>(4);
    const bool fp64 = (p.flags & FIRM_FLAG_FP64_CG) != 0;
    const size_t L3 = fp64 ? 8 * N3 : 0, n64 = fp64 ? N3 : 0;
    w.tw64 = c.take<double2>(fp64 ? N : 0);
    w.khat64 = c.take<double>(L3);
    w.c64 = c.take<double2>(L3);
    w.x64 = c.take<double>(n64);
    w.r64 = c.take<double>(n64);
    w.p64 = c.take<double>(n64);
    w.q64 = c.take<double>(n64);
    w.total = c.off + 256;
    return w.total;
}

static bool supported_N(int N) {
    return N == 16 || N == 32 || N == 48 || N == 64 || N == 80 || N == 96 || N == 128;
}

static int check_params(const firm_params* p) {
    if (!p) return FIRM_EINVAL;
    if (!supported_N(p->N)) return FIRM_EINVAL;
    if (p->M < 0 || p->n_groups < 0) return FIRM_EINVAL;
    if (p->W < 6 || p->W > 8) return FIRM_EINVAL;
    if (p->sigma != 2.0) return FIRM_EINVAL;
    if (p->disc_mode != 0 || (p->flags & ~(FIRM_FLAG_FP64_CG | FIRM_FLAG_FUSED)) != 0) return FIRM_EINVAL;
    if ((p->flags & FIRM_FLAG_FP64_CG) && p->N != 16 && p->N != 32 && p->N != 64) return FIRM_EINVAL;
    if (p->img_dtype != FIRM_IMG_F32 && p->img_dtype != FIRM_IMG_BF16) return FIRM_EINVAL;
    if (p->lambda_mode != FIRM_LAMBDA_RELATIVE && p->lambda_mode != FIRM_LAMBDA_ABSOLUTE) return FIRM_EINVAL;
    if (!(p->lambda >= 0.0)) return FIRM_EINVAL;
    // point ids are m << 13 | t: t < 8192 and m < 2^19
    if ((disc_size(p->N) + 1) / 2 >= (1 << kTBits) || p->M >= (1 << (32 - kTBits))) return FIRM_EINVAL;
    // positions in the binned id array (work items, cursors) are 32-bit signed
    if ((long long)p->M * ((disc_size(p->N) + 1) / 2) >= (1ll << 31)) return FIRM_EINVAL;
    return FIRM_OK;
}

// ---------------------------------------------------------------------------
// Helpers
// ---------------------------------------------------------------------------
static bool is_device(const void* ptr) {
    if (!ptr) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Device pointer for an input: the caller's own if it is device memory, else a copy.
template <class T>
static const T* stage(const T* src, T* dst, size_t count, cudaStream_t s, cudaError_t& e) {
    if (is_device(src)) return src;
    e = cudaMemcpyAsync(dst, src, count * sizeof(T), cudaMemcpyHostToDevice, s);
    return dst;
}

static int put_out(void* dst, const void* src, size_t bytes, cudaStream_t s) {
    if (!dst) return FIRM_OK;
    const bool dev = is_device(dst);
    if (cudaMemcpyAsync(dst, src, bytes, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return FIRM_ECUDA;
    if (!dev && cudaStreamSynchronize(s) != cudaSuccess) return FIRM_ECUDA;
    return FIRM_OK;
}

// Records a start / stop event pair per stage slot on the plan's stream; nothing
// waits here, firm_stage_times synchronises when it reads them.
struct StageTimer {
    Plan& P;
    int slot = -1;
    explicit StageTimer(Plan& p) : P(p) {}
    void start(int s) {
        if (!P.timing) return;
        slot = s;
        if (!P.ev_a[s]) {
            cudaEventCreate(&P.ev_a[s]);
            cudaEventCreate(&P.ev_b[s]);
        }
        cudaEventRecord(P.ev_a[s], P.stream);
    }
    void stop() {
        if (!P.timing || slot < 0) return;
        cudaEventRecord(P.ev_b[slot], P.stream);
        P.ev_used[slot] = true;
        slot = -1;
    }
};

#define FIRM_CK(x)                                     \
    do {                                               \
        if ((x) != cudaSuccess) { return FIRM_ECUDA; } \
    } while (0)

// The spreading and interpolation kernels set counters[2] when a binned point falls
// outside its brick (an internal invariant; never expected).  Entry points do not wait
// for it: it is read, and cleared, where the host waits for the stream anyway (a host
// output, the end of a CG solve, a query of device scalars).
static int take_device_flag(Plan& P) {
    int flag = 0;
    FIRM_CK(cudaMemcpyAsync(&flag, P.ws.counters + 2, sizeof(int), cudaMemcpyDeviceToHost, P.stream));
    FIRM_CK(cudaStreamSynchronize(P.stream));
    if (!flag) return FIRM_OK;
    FIRM_CK(cudaMemsetAsync(P.ws.counters + 2, 0, sizeof(int), P.stream));
    return FIRM_EINTERNAL;
}

// An output to dst: device memory is written in stream order; host memory waits for
// the copy (and reports the device flag).
static int put_out_checked(Plan& P, void* dst, const void* src, size_t bytes) {
    if (!dst) return FIRM_OK;
    if (is_device(dst)) return put_out(dst, src, bytes, P.stream);
    const int st = put_out(dst, src, bytes, P.stream);
    return st != FIRM_OK ? st : take_device_flag(P);
}

// lam_eff and Ker(0) of the last firm_kernel, read from the device (waits for the stream).
static int read_lam(Plan& P, double* lam_eff, double* ker0) {
    float lam[2] = {0.f, 0.f};
    FIRM_CK(cudaMemcpyAsync(lam, P.ws.lam, sizeof(lam), cudaMemcpyDeviceToHost, P.stream));
    const int st = take_device_flag(P);
    if (st != FIRM_OK) return st;
    if (ker0) *ker0 = lam[1] > 0.0f ? lam[1] : 1.0;
    if (lam_eff) *lam_eff = P.p.lambda_mode == FIRM_LAMBDA_RELATIVE ? P.p.lambda * (double)lam[1] : P.p.lambda;
    return FIRM_OK;
}


// Per-bin log target t_b = log(p_b Ker(0)), p_b = s1 / s2; empty bins take the value of
// the nearest non-empty shell of the same cone (all empty: the mean of the others).
static void finalize_target(const double* s1, const double* s2, double ker0, float* t) {
    const int S = 64, C = 16;
    std::vector<double> v(1024, NAN);
    double sum = 0.0;
    int cnt = 0;
    for (int b = 0; b < 1024; ++b)
        if (s2[b] > 0.0) { v[b] = std::log(s1[b] / s2[b] * ker0); sum += v[b]; ++cnt; }
    const double mean = cnt ? sum / cnt : 0.0;
    for (int c = 0; c < C; ++c)
        for (int s = 0; s < S; ++s) {
            if (!std::isnan(v[C * s + c])) { t[C * s + c] = (float)v[C * s + c]; continue; }
            int best = -1;
            for (int d = 1; d < S && best < 0; ++d) {
                if (s - d >= 0 && !std::isnan(v[C * (s - d) + c])) best = s - d;
                else if (s + d < S && !std::isnan(v[C * (s + d) + c])) best = s + d;
            }
            t[C * s + c] = (float)(best >= 0 ? v[C * best + c] : mean);
        }
}

static int compute_target(Plan& P, float* t_host) {
    FIRM_CK(launch_chan_spectrum(P));
    FIRM_CK(launch_pc_target_sums(P, P.ws.pc_s1, P.ws.pc_s2));
    std::vector<double> s1(1024), s2(1024);
    FIRM_CK(cudaMemcpyAsync(s1.data(), P.ws.pc_s1, 1024 * sizeof(double), cudaMemcpyDeviceToHost, P.stream));
    FIRM_CK(cudaMemcpyAsync(s2.data(), P.ws.pc_s2, 1024 * sizeof(double), cudaMemcpyDeviceToHost, P.stream));
    double ker0 = 1.0;
    const int st = read_lam(P, nullptr, &ker0);
    if (st != FIRM_OK) return st;
    finalize_target(s1.data(), s2.data(), ker0, t_host);
    return FIRM_OK;
}

static int build_preconditioner(Plan& P) {
    if (P.pc_mode == FIRM_PRECOND_CIRCULANT) {
        FIRM_CK(launch_chan_spectrum(P));
        FIRM_CK(launch_pc_build_circulant(P));
        return FIRM_OK;
    }
    if (P.pc_mode == FIRM_PRECOND_BINNED) {
        std::vector<float> t(1024);
        const int st = compute_target(P, t.data());
        if (st != FIRM_OK) return st;
        FIRM_CK(cudaMemcpyAsync(P.ws.pc_table, t.data(), 1024 * sizeof(float), cudaMemcpyHostToDevice, P.stream));
    }
    // FIRM_PRECOND_TABLE: pc_table was set by firm_set_precond_table
    FIRM_CK(launch_pc_from_table(P, P.ws.pc_table));
    return FIRM_OK;
}

// CG in the FP64 mode (FIRM_FLAG_FP64_CG): plain CG only; same stopping rule and
// outputs as the FP32 path.
static int cg_solve_fp64(Plan& P, const float* rd, float* x, int max_iter, double rel_tol, double* resid_hist,
                         int* iters_out, StageTimer& tm) {
    if (P.pc_mode != FIRM_PRECOND_NONE) return FIRM_EINVAL;
    Workspace& w = P.ws;
    const size_t n = (size_t)P.N * P.N * P.N;
    const int batch = 8;
    FIRM_CK(launch_cg64(P, rd, max_iter, rel_tol, 0, 0));
    for (int it = 0; it < max_iter; it += batch) {
        FIRM_CK(launch_cg64(P, rd, max_iter, rel_tol, 1, std::min(batch, max_iter - it)));
        if (rel_tol > 0.0 && it + batch < max_iter) {
            int done = 0;
            FIRM_CK(cudaMemcpyAsync(&done, &w.cg->done, sizeof(int), cudaMemcpyDeviceToHost, P.stream));
            FIRM_CK(cudaStreamSynchronize(P.stream));
            if (done) break;
        }
    }
    FIRM_CK(launch_cg64_result(P));
    tm.stop();
    CgState s;
    FIRM_CK(cudaMemcpyAsync(&s, w.cg, sizeof(CgState), cudaMemcpyDeviceToHost, P.stream));
    FIRM_CK(cudaStreamSynchronize(P.stream));
    P.cg_iters = s.it;
    if (resid_hist) {
        const bool dev = is_device(resid_hist);
        FIRM_CK(cudaMemcpyAsync(resid_hist, w.hist, sizeof(double) * (s.it + 1),
                                dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, P.stream));
    }
    if (iters_out) *iters_out = s.it;
    int st = put_out(x, w.x, n * sizeof(float), P.stream);
    if (st != FIRM_OK) return st;
    st = take_device_flag(P);
    if (st != FIRM_OK) return st;
    if (s.status != FIRM_OK) return s.status;
    if (rel_tol > 0.0 && !(s.rr >= 0.0 && std::sqrt(s.rr) <= s.tol)) return FIRM_ENOTCONV;
    return FIRM_OK;
}

}  // namespace firm

using namespace firm;

extern "C" {

int firm_workspace_size(const firm_params* p, size_t* bytes) {
    const int st = check_params(p);
    if (st != FIRM_OK) return st;
    if (!bytes) return FIRM_EINVAL;
    Workspace w;
    *bytes = layout_workspace(*p, nullptr, w);
    return FIRM_OK;
}

int firm_plan(firm_plan_t* out, const firm_params* p, const firm_ctf_group* groups, void* workspace,
              size_t workspace_bytes, void* stream) {
    if (!out) return FIRM_EINVAL;
    *out = nullptr;
    int st = check_params(p);
    if (st != FIRM_OK) return st;
    if (p->n_groups > 0 && !groups) return FIRM_EINVAL;
    Workspace probe;
    const size_t need = layout_workspace(*p, nullptr, probe);
    if (!workspace || workspace_bytes < need) return FIRM_ENOMEM;
    if ((reinterpret_cast<uintptr_t>(workspace) & 255) != 0) return FIRM_EINVAL;
    if (!is_device(workspace)) return FIRM_EINVAL;

    firm_plan_s* h = new (std::nothrow) firm_plan_s();
    if (!h) return FIRM_ENOMEM;
    Plan& P = h->P;
    P.p = *p;
    P.stream = reinterpret_cast<cudaStream_t>(stream);
    P.base = reinterpret_cast<char*>(workspace);
    layout_workspace(*p, P.base, P.ws);
    P.N = p->N;
    P.Gk = 4 * p->N;
    P.Gr = 2 * p->N;
    P.nbk = P.Gk / kBrick;
    P.nbkz = P.Gk / kBrickZk;
    P.nbr = P.Gr / kBrick;
    P.nK = disc_size(p->N);
    P.nH = (P.nK + 1) / 2;
    P.n_ctf = p->n_groups > 0 ? p->n_groups : 1;
    P.max_work = (size_t)P.nbk * P.nbk * P.nbk + (size_t)p->M * P.nH / kMinChunk + 2;
    for (int g = 0; g < p->n_groups; ++g) P.groups.push_back(groups[g]);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&P.num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        delete h;
        return FIRM_ECUDA;
    }
    if (fft_init_constants() != cudaSuccess) { delete h; return FIRM_ECUDA; }

    double beta = 0.0;
    kb_build(p->W, p->sigma, P.poly, &beta);

    // tables
    const int N = P.N, nH = P.nH;
    P.htab_host = half_disc(N);
    std::vector<float> h1((size_t)P.n_ctf * nH), h2((size_t)P.n_ctf * nH);
    P.h2_max = 0.0f;
    for (int g = 0; g < P.n_ctf; ++g) {
        for (int t = 0; t < nH; ++t) {
            const int32_t kk = P.htab_host[t];
            const int k1 = (int16_t)(kk & 0xffff), k2 = kk >> 16;
            double hv = 1.0;
            if (p->n_groups > 0) hv = ctf_value(P.groups[g], std::sqrt((double)(k1 * k1 + k2 * k2)) / (N * P.groups[g].pixel_A));
            h1[(size_t)g * nH + t] = (float)hv;
            h2[(size_t)g * nH + t] = (float)(hv * hv * (t == 0 ? 0.5 : 1.0));
            P.h2_max = std::max(P.h2_max, h2[(size_t)g * nH + t]);
        }
    }
    auto tw = [](int L) {
        std::vector<float2> v(L);
        for (int j = 0; j < L; ++j) {
            const double a = -2.0 * kPi * j / L;
            v[j] = make_float2((float)std::cos(a), (float)std::sin(a));
        }
        return v;
    };
    // deconvolution: (-1)^n / phihat(n / G) for the centred fine grid
    std::vector<float> dk(2 * N), dr(N), dr4(N);
    for (int i = 0; i < 2 * N; ++i) {
        const int n = i - N;
        dk[i] = (float)(((n & 1) ? -1.0 : 1.0) / kb_phihat((double)n / P.Gk, p->W, beta));
    }
    for (int i = 0; i < N; ++i) {
        const int n = i - N / 2;
        dr[i] = (float)(((n & 1) ? -1.0 : 1.0) / kb_phihat((double)n / P.Gr, p->W, beta));
        dr4[i] = (float)(((n & 1) ? -1.0 : 1.0) / kb_phihat((double)n / P.Gk, p->W, beta));
    }
    const std::vector<float2> t1 = tw(N), t2 = tw(2 * N), t4 = tw(4 * N);
    Workspace& w = P.ws;
    cudaError_t e = cudaSuccess;
    auto cp = [&](void* d, const void* s, size_t b) {
        if (e == cudaSuccess) e = cudaMemcpyAsync(d, s, b, cudaMemcpyHostToDevice, P.stream);
    };
    cp(w.htab, P.htab_host.data(), sizeof(int32_t) * nH);
    // columns of the half disc in the order of htab: k1 = 0 holds k2 = 0..N/2, k1 > 0 holds -km..km
    std::vector<int4> colv(N / 2 + 1);
    {
        int t0 = 0;
        for (int k1 = 0; k1 <= N / 2; ++k1) {
            int km = 0;
            while ((km + 1) * (km + 1) + k1 * k1 <= (N / 2) * (N / 2)) ++km;
            const int lo = k1 == 0 ? 0 : -km;
            colv[k1] = make_int4(t0, lo, km, 0);
            t0 += km - lo + 1;
        }
        if (t0 != nH) e = cudaErrorInvalidValue;
    }
    cp(w.colinfo, colv.data(), sizeof(int4) * colv.size());
    cp(w.h1, h1.data(), sizeof(float) * h1.size());
    cp(w.h2, h2.data(), sizeof(float) * h2.size());
    cp(w.tw_n, t1.data(), sizeof(float2) * N);
    cp(w.tw_2n, t2.data(), sizeof(float2) * 2 * N);
    cp(w.tw_4n, t4.data(), sizeof(float2) * 4 * N);
    cp(w.dec_k, dk.data(), sizeof(float) * dk.size());
    cp(w.dec_r, dr.data(), sizeof(float) * dr.size());
    cp(w.dec_r4, dr4.data(), sizeof(float) * dr4.size());
    std::vector<double2> t64;
    if (p->flags & FIRM_FLAG_FP64_CG) {
        for (int j = 0; j < N; ++j) {
            const double a = -2.0 * kPi * j / (2 * N);
            t64.push_back(make_double2(std::cos(a), std::sin(a)));
        }
        cp(w.tw64, t64.data(), sizeof(double2) * t64.size());
    }
    const float axis0[4] = {0.f, 0.f, 1.f, 0.f};
    cp(w.axis, axis0, sizeof(axis0));
    if (e == cudaSuccess) e = cudaMemsetAsync(w.counters, 0, 8 * sizeof(int), P.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(P.stream);
    if (e != cudaSuccess) {
        delete h;
        return FIRM_ECUDA;
    }
    *out = h;
    return FIRM_OK;
}

// Issues a recorded image upload on the copy stream, after everything queued so far on
// the plan's stream (the calling entry point's own small uploads come first: a copy
// engine serves queued copies in order, so poses queued behind 1.6 GB of images would
// hold the kernel channel back for the whole upload).
static cudaError_t start_stage(Plan& P) {
    if (!P.staged_host || P.stage_started) return cudaSuccess;
    cudaError_t e = cudaEventRecord(P.ev_inputs, P.stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(P.copy_stream, P.ev_inputs, 0);
    // an earlier staged upload must have been read by its image DFT (an event never
    // recorded counts as complete)
    if (e == cudaSuccess) e = cudaStreamWaitEvent(P.copy_stream, P.ev_stage_read, 0);
    if (e == cudaSuccess && P.staged_bytes > 0)
        e = cudaMemcpyAsync(P.staged_dev, P.staged_host, P.staged_bytes, cudaMemcpyHostToDevice, P.copy_stream);
    if (e == cudaSuccess) e = cudaEventRecord(P.ev_staged, P.copy_stream);
    if (e == cudaSuccess) P.stage_started = true;
    return e;
}

int firm_kernel(firm_plan_t plan, int M, const double* R, const int32_t* group, float* khat_out) {
    if (!plan || M < 0 || M > plan->P.p.M || (M > 0 && !R)) return FIRM_EINVAL;
    Plan& P = plan->P;
    Workspace& w = P.ws;
    cudaError_t e = cudaSuccess;
    StageTimer tm(P);
    P.cur_R = stage(R, w.R, (size_t)M * 9, P.stream, e);
    if (group) P.cur_gid = stage(group, w.gid, (size_t)M, P.stream, e);
    else { e = cudaMemsetAsync(w.gid, 0, sizeof(int32_t) * (M > 0 ? M : 1), P.stream); P.cur_gid = w.gid; }
    FIRM_CK(e);
    P.ev_used[10] = false;                     // no fused weight gather in this form
    FIRM_CK(start_stage(P));                   // a staged image upload runs beside the kernel channel
    P.bin_M = -1;
    tm.start(0);
    FIRM_CK(launch_geom(P.cur_R, M, w.geom, P.stream));
    P.launches += M > 0 ? 1 : 0;
    FIRM_CK(launch_bin(P, M, true));
    tm.stop();
    tm.start(1);
    FIRM_CK(launch_spread(P, M, true));
    tm.stop();
    tm.start(2);
    FIRM_CK(launch_ker_transform(P));
    tm.stop();
    tm.start(3);
    FIRM_CK(launch_khat(P));
    FIRM_CK(launch_lam_eff(P));
    if (P.p.flags & FIRM_FLAG_FP64_CG) FIRM_CK(launch_khat64(P));
    FIRM_CK(launch_damping(P));
    tm.stop();
    P.last_M = M;
    if (M > 0) FIRM_CK(launch_view_axis(P, P.cur_R, M));
    P.have_kernel = true;
    P.pc_ready = false;
    return put_out_checked(P, khat_out, w.khat, sizeof(float) * 2 * P.N * 2 * P.N * (P.N + 1));
}

static bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

int firm_backproject(firm_plan_t plan, int M, const void* images, const double* shifts, const double* R,
                     const int32_t* group, float* rhs_out) {
    if (!plan || M < 0 || M > plan->P.p.M || (M > 0 && (!R || !images || !aligned16(images)))) return FIRM_EINVAL;
    Plan& P = plan->P;
    Workspace& w = P.ws;
    cudaError_t e = cudaSuccess;
    StageTimer tm(P);
    const size_t esz = P.p.img_dtype == FIRM_IMG_BF16 ? 2 : 4;
    P.cur_R = stage(R, w.R, (size_t)M * 9, P.stream, e);
    if (group) P.cur_gid = stage(group, w.gid, (size_t)M, P.stream, e);
    else { e = cudaMemsetAsync(w.gid, 0, sizeof(int32_t) * (M > 0 ? M : 1), P.stream); P.cur_gid = w.gid; }
    if (shifts) P.cur_shifts = stage(shifts, w.shifts, (size_t)M * 2, P.stream, e);
    else { if (e == cudaSuccess) e = cudaMemsetAsync(w.shifts, 0, sizeof(double) * 2 * (M > 0 ? M : 1), P.stream); P.cur_shifts = w.shifts; }
    FIRM_CK(e);
    bool from_stage = false;
    if (M > 0 && P.staged_host == images && P.staged_M == M) {
        FIRM_CK(start_stage(P));                                     // unless firm_kernel started it
        FIRM_CK(cudaStreamWaitEvent(P.stream, P.ev_staged, 0));     // the upload has landed
        P.cur_images = P.staged_dev;
        P.staged_host = nullptr;
        P.staged_M = -1;
        from_stage = true;
    } else if (M > 0 && !is_device(images)) {
        FIRM_CK(cudaMemcpyAsync(w.images, images, (size_t)M * P.N * P.N * esz, cudaMemcpyHostToDevice, P.stream));
        P.cur_images = w.images;
    } else {
        P.cur_images = images;
    }
    P.bin_M = -1;
    tm.start(4);
    FIRM_CK(launch_geom(P.cur_R, M, w.geom, P.stream));
    P.launches += M > 0 ? 1 : 0;
    FIRM_CK(launch_image_dft(P, M, P.cur_images, P.cur_shifts, P.cur_gid));
    if (from_stage) FIRM_CK(cudaEventRecord(P.ev_stage_read, P.stream));   // staging free again
    tm.stop();
    tm.start(5);
    FIRM_CK(launch_bin(P, M, false));
    tm.stop();
    tm.start(6);
    FIRM_CK(launch_spread(P, M, false));
    tm.stop();
    tm.start(7);
    FIRM_CK(launch_rhs_transform(P));
    tm.stop();
    P.have_rhs = true;
    return put_out_checked(P, rhs_out, w.rhs, sizeof(float) * P.N * P.N * P.N);
}

int firm_kernel_backproject(firm_plan_t plan, int M, const void* images, const double* shifts, const double* R,
                            const int32_t* group, float* khat_out, float* rhs_out) {
    if (!plan || M < 0 || M > plan->P.p.M || (M > 0 && (!R || !images || !aligned16(images)))) return FIRM_EINVAL;
    Plan& P = plan->P;
    if (!(P.p.flags & FIRM_FLAG_FUSED)) return FIRM_EINVAL;
    Workspace& w = P.ws;
    cudaError_t e = cudaSuccess;
    StageTimer tm(P);
    const size_t esz = P.p.img_dtype == FIRM_IMG_BF16 ? 2 : 4;
    P.cur_R = stage(R, w.R, (size_t)M * 9, P.stream, e);
    if (group) P.cur_gid = stage(group, w.gid, (size_t)M, P.stream, e);
    else { e = cudaMemsetAsync(w.gid, 0, sizeof(int32_t) * (M > 0 ? M : 1), P.stream); P.cur_gid = w.gid; }
    if (shifts) P.cur_shifts = stage(shifts, w.shifts, (size_t)M * 2, P.stream, e);
    else { if (e == cudaSuccess) e = cudaMemsetAsync(w.shifts, 0, sizeof(double) * 2 * (M > 0 ? M : 1), P.stream); P.cur_shifts = w.shifts; }
    FIRM_CK(e);
    P.ev_used[5] = P.ev_used[6] = false;      // no separate A*b binning or spreading stage here
    const bool staged = M > 0 && P.staged_host == images && P.staged_M == M;
    // host images not staged ahead are copied into the workspace region the point ids
    // use, so they are transformed before the binning; otherwise the binning (poses
    // only) goes first, beside a staged upload
    const bool host_copy = M > 0 && !staged && !is_device(images);
    if (staged) FIRM_CK(start_stage(P));
    P.bin_M = -1;
    FIRM_CK(launch_geom(P.cur_R, M, w.geom, P.stream));
    P.launches += M > 0 ? 1 : 0;
    if (!host_copy) {
        tm.start(0);
        FIRM_CK(launch_bin(P, M, true));
        tm.stop();
    }
    if (staged) {
        FIRM_CK(cudaStreamWaitEvent(P.stream, P.ev_staged, 0));     // the upload has landed
        P.cur_images = P.staged_dev;
        P.staged_host = nullptr;
        P.staged_M = -1;
    } else if (host_copy) {
        FIRM_CK(cudaMemcpyAsync(w.images, images, (size_t)M * P.N * P.N * esz, cudaMemcpyHostToDevice, P.stream));
        P.cur_images = w.images;
    } else {
        P.cur_images = images;
    }
    tm.start(4);
    FIRM_CK(launch_image_dft(P, M, P.cur_images, P.cur_shifts, P.cur_gid));
    if (staged) FIRM_CK(cudaEventRecord(P.ev_stage_read, P.stream));   // staging free again
    tm.stop();
    if (host_copy) {
        tm.start(0);
        FIRM_CK(launch_bin(P, M, true));
        tm.stop();
    }
    tm.start(10);
    FIRM_CK(launch_fused_gather(P, M));
    tm.stop();
    tm.start(1);
    FIRM_CK(launch_spread_fused(P, M));
    tm.stop();
    tm.start(2);
    FIRM_CK(launch_ker_transform(P));
    tm.stop();
    tm.start(3);
    FIRM_CK(launch_khat(P));
    FIRM_CK(launch_lam_eff(P));
    if (P.p.flags & FIRM_FLAG_FP64_CG) FIRM_CK(launch_khat64(P));
    FIRM_CK(launch_damping(P));
    tm.stop();
    tm.start(7);
    FIRM_CK(launch_rhs_transform4(P));
    tm.stop();
    P.last_M = M;
    if (M > 0) FIRM_CK(launch_view_axis(P, P.cur_R, M));
    P.have_kernel = P.have_rhs = true;
    P.pc_ready = false;
    const int st = put_out_checked(P, khat_out, w.khat, sizeof(float) * 2 * P.N * 2 * P.N * (P.N + 1));
    if (st != FIRM_OK) return st;
    return put_out_checked(P, rhs_out, w.rhs, sizeof(float) * P.N * P.N * P.N);
}

int firm_load_sums(firm_plan_t plan, const float* ker_half, const float* rhs) {
    if (!plan || (!ker_half && !rhs)) return FIRM_EINVAL;
    Plan& P = plan->P;
    Workspace& w = P.ws;
    const size_t H3 = (size_t)2 * P.N * 2 * P.N * (P.N + 1), N3 = (size_t)P.N * P.N * P.N;
    auto in = [&](const float* src, float* dst, size_t n) -> cudaError_t {
        return cudaMemcpyAsync(dst, src, n * sizeof(float), is_device(src) ? cudaMemcpyDeviceToDevice
                                                                          : cudaMemcpyHostToDevice, P.stream);
    };
    StageTimer tm(P);
    if (ker_half) {
        FIRM_CK(in(ker_half, w.ker, H3));
        tm.start(3);
        FIRM_CK(launch_khat(P));
        FIRM_CK(launch_lam_eff(P));
        if (P.p.flags & FIRM_FLAG_FP64_CG) FIRM_CK(launch_khat64(P));
        FIRM_CK(launch_damping(P));
        tm.stop();
        P.have_kernel = true;
        P.pc_ready = false;
    }
    if (rhs) {
        FIRM_CK(in(rhs, w.rhs, N3));
        P.have_rhs = true;
    }
    return FIRM_OK;
}

int firm_stage_images(firm_plan_t plan, int M, const void* images, void* staging, size_t staging_bytes) {
    if (!plan || M < 0 || M > plan->P.p.M || (M > 0 && (!images || !staging))) return FIRM_EINVAL;
    Plan& P = plan->P;
    const size_t esz = P.p.img_dtype == FIRM_IMG_BF16 ? 2 : 4;
    const size_t bytes = (size_t)M * P.N * P.N * esz;
    if (M > 0 && (is_device(images) || !is_device(staging) || staging_bytes < bytes || !aligned16(staging)))
        return FIRM_EINVAL;
    if (!P.copy_stream) {
        FIRM_CK(cudaStreamCreateWithFlags(&P.copy_stream, cudaStreamNonBlocking));
        FIRM_CK(cudaEventCreateWithFlags(&P.ev_inputs, cudaEventDisableTiming));
        FIRM_CK(cudaEventCreateWithFlags(&P.ev_staged, cudaEventDisableTiming));
        FIRM_CK(cudaEventCreateWithFlags(&P.ev_stage_read, cudaEventDisableTiming));
    }
    P.staged_host = images;
    P.staged_dev = staging;
    P.staged_bytes = bytes;
    P.staged_M = M;
    P.stage_started = false;
    return FIRM_OK;
}

// Poses, groups and the volume of a forward-projector call staged on the plan's stream.
static cudaError_t stage_forward_inputs(Plan& P, int M, const float* V, const double* R, const int32_t* group,
                                        const float*& Vd) {
    Workspace& w = P.ws;
    cudaError_t e = cudaSuccess;
    P.cur_R = stage(R, w.R, (size_t)M * 9, P.stream, e);
    if (group) P.cur_gid = stage(group, w.gid, (size_t)M, P.stream, e);
    else if (e == cudaSuccess) { e = cudaMemsetAsync(w.gid, 0, sizeof(int32_t) * (M > 0 ? M : 1), P.stream); P.cur_gid = w.gid; }
    Vd = stage(V, w.q, (size_t)P.N * P.N * P.N, P.stream, e);
    P.bin_M = -1;
    return e;
}

int firm_forward(firm_plan_t plan, int M, const float* V, const double* R, const int32_t* group, float* out) {
    if (!plan || M < 0 || M > plan->P.p.M || (M > 0 && (!R || !V || !out))) return FIRM_EINVAL;
    Plan& P = plan->P;
    Workspace& w = P.ws;
    if (M == 0) return FIRM_OK;
    const float* Vd = nullptr;
    FIRM_CK(stage_forward_inputs(P, M, V, R, group, Vd));
    FIRM_CK(launch_geom(P.cur_R, M, w.geom, P.stream));
    P.launches += 1;
    FIRM_CK(launch_bin(P, M, false));
    float2* ghat = reinterpret_cast<float2*>(w.grid);
    FIRM_CK(launch_fwd_transform(P, Vd, ghat));
    const bool odev = is_device(out);
    float2* od = odev ? reinterpret_cast<float2*>(out) : w.samples;
    FIRM_CK(launch_interp(P, M, ghat, od, nullptr, nullptr));
    if (!odev) return put_out_checked(P, out, od, sizeof(float2) * (size_t)M * P.nH);
    return FIRM_OK;
}

int firm_data_residual(firm_plan_t plan, int M, const float* V, const void* images, const double* shifts,
                       const double* R, const int32_t* group, double* out2) {
    if (!plan || !out2 || M < 0 || M > plan->P.p.M || (M > 0 && (!R || !V || !images || !aligned16(images))))
        return FIRM_EINVAL;
    Plan& P = plan->P;
    Workspace& w = P.ws;
    if (M == 0) {
        const double z[2] = {0.0, 0.0};
        if (is_device(out2)) FIRM_CK(cudaMemcpyAsync(out2, z, sizeof(z), cudaMemcpyHostToDevice, P.stream));
        else { out2[0] = 0.0; out2[1] = 0.0; }
        return FIRM_OK;
    }
    const float* Vd = nullptr;
    FIRM_CK(stage_forward_inputs(P, M, V, R, group, Vd));
    cudaError_t e = cudaSuccess;
    const double* sh = shifts ? stage(shifts, w.shifts, (size_t)M * 2, P.stream, e) : nullptr;
    FIRM_CK(e);
    if (!shifts) { FIRM_CK(cudaMemsetAsync(w.shifts, 0, sizeof(double) * 2 * M, P.stream)); sh = w.shifts; }
    const size_t esz = P.p.img_dtype == FIRM_IMG_BF16 ? 2 : 4;
    const void* img = images;
    if (!is_device(images)) {
        FIRM_CK(cudaMemcpyAsync(w.images, images, (size_t)M * P.N * P.N * esz, cudaMemcpyHostToDevice, P.stream));
        img = w.images;
    }
    FIRM_CK(launch_geom(P.cur_R, M, w.geom, P.stream));
    P.launches += 1;
    FIRM_CK(launch_image_dft(P, M, img, sh, P.cur_gid, true));    // b itself into samples
    FIRM_CK(launch_bin(P, M, false));                                // b copied in scatter order
    float2* ghat = reinterpret_cast<float2*>(w.grid);
    FIRM_CK(launch_fwd_transform(P, Vd, ghat));
    FIRM_CK(launch_interp(P, M, ghat, nullptr, w.item_part, w.red_a));
    return put_out_checked(P, out2, w.red_a, 2 * sizeof(double));
}

int firm_solve_nonneg(firm_plan_t plan, float* x, int max_iter, double rel_tol, int* iters_out) {
    if (!plan || !x || max_iter < 0 || !(rel_tol >= 0.0) || !std::isfinite(rel_tol)) return FIRM_EINVAL;
    Plan& P = plan->P;
    if (!P.have_kernel || !P.have_rhs) return FIRM_ESTATE;
    const bool xdev = is_device(x);
    float* xd = xdev ? x : P.ws.x;
    const int st = pos_solve(P, xd, max_iter, rel_tol, iters_out);
    if (st == FIRM_ECUDA) return st;
    if (!xdev) {
        const int s2 = put_out(x, xd, sizeof(float) * P.N * P.N * P.N, P.stream);
        if (s2 != FIRM_OK) return s2;
    }
    return st;
}

int firm_set_damping(firm_plan_t plan, double mu) {
    if (!plan || !(mu >= 0.0) || !std::isfinite(mu)) return FIRM_EINVAL;
    plan->P.mu = mu;
    return FIRM_OK;
}

int firm_toeplitz_apply(firm_plan_t plan, const float* x, float* y) {
    if (!plan || !x || !y) return FIRM_EINVAL;
    Plan& P = plan->P;
    if (!P.have_kernel) return FIRM_ESTATE;
    Workspace& w = P.ws;
    const size_t n = (size_t)P.N * P.N * P.N;
    cudaError_t e = cudaSuccess;
    const float* xd = stage(x, w.x, n, P.stream, e);
    FIRM_CK(e);
    const bool ydev = is_device(y);
    float* yd = ydev ? y : w.q;
    if (xd == yd) return FIRM_EINVAL;
    FIRM_CK(launch_toeplitz(P, xd, yd, nullptr, nullptr));
    if (!ydev) return put_out(y, yd, n * sizeof(float), P.stream);
    return FIRM_OK;
}

int firm_cg_solve(firm_plan_t plan, const float* rhs, float* x, int max_iter, double rel_tol, double* resid_hist,
                  int* iters_out) {
    if (!plan || !x || max_iter < 0 || max_iter >= kMaxHist || !(rel_tol >= 0.0)) return FIRM_EINVAL;
    Plan& P = plan->P;
    if (!P.have_kernel) return FIRM_ESTATE;
    if (!rhs && !P.have_rhs) return FIRM_ESTATE;
    Workspace& w = P.ws;
    const size_t n = (size_t)P.N * P.N * P.N;
    cudaError_t e = cudaSuccess;
    const float* rd = rhs ? stage(rhs, w.q, n, P.stream, e) : w.rhs;
    FIRM_CK(e);
    StageTimer tm(P);
    tm.start(8);
    const bool use_pc = P.pc_mode != FIRM_PRECOND_NONE;
    if (P.p.flags & FIRM_FLAG_FP64_CG) return cg_solve_fp64(P, rd, x, max_iter, rel_tol, resid_hist, iters_out, tm);
    if (use_pc && !P.pc_ready) {
        int st = build_preconditioner(P);
        if (st != FIRM_OK) return st;
        P.pc_ready = true;
    }
    FIRM_CK(launch_cg_init(P, rd, max_iter, rel_tol, use_pc));
    if (use_pc) FIRM_CK(launch_precond(P, w.r, w.z, w.cg));
    const int batch = 8;
    for (int it = 0; it < max_iter; ++it) {
        FIRM_CK(launch_toeplitz(P, w.p, w.q, w.r, w.cg, use_pc ? w.z : nullptr));
        FIRM_CK(launch_cg_update(P));
        if (use_pc) FIRM_CK(launch_precond(P, w.r, w.z, w.cg));
        if (rel_tol > 0.0 && ((it + 1) % batch == 0) && it + 1 < max_iter) {
            int done = 0;
            FIRM_CK(cudaMemcpyAsync(&done, &w.cg->done, sizeof(int), cudaMemcpyDeviceToHost, P.stream));
            FIRM_CK(cudaStreamSynchronize(P.stream));
            if (done) break;
        }
    }
    tm.stop();
    CgState s;
    FIRM_CK(cudaMemcpyAsync(&s, w.cg, sizeof(CgState), cudaMemcpyDeviceToHost, P.stream));
    FIRM_CK(cudaStreamSynchronize(P.stream));
    P.cg_iters = s.it;
    if (resid_hist) {
        const bool dev = is_device(resid_hist);
        FIRM_CK(cudaMemcpyAsync(resid_hist, w.hist, sizeof(double) * (s.it + 1),
                                dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, P.stream));
    }
    if (iters_out) *iters_out = s.it;
    int st = put_out(x, w.x, n * sizeof(float), P.stream);
    if (st != FIRM_OK) return st;
    st = take_device_flag(P);
    if (st != FIRM_OK) return st;
    if (s.status != FIRM_OK) return s.status;
    if (rel_tol > 0.0 && !(s.rr >= 0.0 && std::sqrt(s.rr) <= s.tol)) return FIRM_ENOTCONV;
    return FIRM_OK;
}

int firm_set_precond(firm_plan_t plan, int mode) {
    if (!plan) return FIRM_EINVAL;
    if (mode != FIRM_PRECOND_NONE && mode != FIRM_PRECOND_CIRCULANT && mode != FIRM_PRECOND_BINNED &&
        mode != FIRM_PRECOND_TABLE)
        return FIRM_EINVAL;
    plan->P.pc_mode = mode;
    plan->P.pc_ready = false;
    return FIRM_OK;
}

int firm_set_precond_table(firm_plan_t plan, const float* table_log) {
    if (!plan || !table_log) return FIRM_EINVAL;
    Plan& P = plan->P;
    cudaError_t e = cudaSuccess;
    const float* d = stage(table_log, P.ws.pc_table, 1024, P.stream, e);
    FIRM_CK(e);
    if (d != P.ws.pc_table) FIRM_CK(cudaMemcpyAsync(P.ws.pc_table, d, 1024 * sizeof(float), cudaMemcpyDeviceToDevice, P.stream));
    P.pc_mode = FIRM_PRECOND_TABLE;
    P.pc_ready = false;
    return FIRM_OK;
}

int firm_pc_features(firm_plan_t plan, float* out) {
    if (!plan || !out) return FIRM_EINVAL;
    Plan& P = plan->P;
    if (!P.have_kernel) return FIRM_ESTATE;
    FIRM_CK(launch_pc_features(P, P.last_M, P.ws.pc_feat));
    FIRM_CK(launch_pc_normalize(P, P.ws.pc_feat, nullptr));
    return put_out_checked(P, out, P.ws.pc_feat, 1024 * sizeof(float));
}

int firm_pc_net_input(firm_plan_t plan, float* out) {
    if (!plan || !out) return FIRM_EINVAL;
    Plan& P = plan->P;
    if (!P.have_kernel) return FIRM_ESTATE;
    float* x = reinterpret_cast<float*>(P.ws.pc_s2);       // 1024 floats of scratch
    FIRM_CK(launch_pc_features(P, P.last_M, P.ws.pc_feat));
    FIRM_CK(launch_pc_normalize(P, P.ws.pc_feat, x));
    return put_out_checked(P, out, x, 1024 * sizeof(float));
}

int firm_pc_target(firm_plan_t plan, float* out) {
    if (!plan || !out) return FIRM_EINVAL;
    Plan& P = plan->P;
    if (!P.have_kernel) return FIRM_ESTATE;
    std::vector<float> t(1024);
    const int st = compute_target(P, t.data());
    if (st != FIRM_OK) return st;
    P.pc_ready = false;                 // ws.t1 was used as scratch
    FIRM_CK(cudaMemcpyAsync(P.ws.pc_s1, t.data(), 1024 * sizeof(float), cudaMemcpyHostToDevice, P.stream));
    return put_out(out, P.ws.pc_s1, 1024 * sizeof(float), P.stream);
}

// Density-per-volume baseline of the log table: the mean eigenvalue of a sampling
// operator over a bin is about Ker(0) f_b / v_b, so log(p_b Ker(0)) ~ -log(f_b / v_b +
// lambda / Ker(0)) with lambda / Ker(0) = 1e-3 (the relative Tikhonov weight).
int firm_pc_baseline(firm_plan_t plan, float* out) {
    if (!plan || !out) return FIRM_EINVAL;
    Plan& P = plan->P;
    if (!P.have_kernel) return FIRM_ESTATE;
    std::vector<float> f(1024), v(1024), t(1024);
    int st = firm_pc_features(plan, f.data());
    if (st != FIRM_OK) return st;
    st = firm_pc_bin_volumes(plan, v.data());
    if (st != FIRM_OK) return st;
    double ker0 = 1.0;
    st = read_lam(P, nullptr, &ker0);
    if (st != FIRM_OK) return st;
    const double rl = P.p.lambda_mode == FIRM_LAMBDA_RELATIVE ? P.p.lambda : P.p.lambda / ker0;
    for (int b = 0; b < 1024; ++b)
        t[b] = (float)-std::log((v[b] > 0.0f ? (double)f[b] / (double)v[b] : 0.0) + (rl > 0.0 ? rl : 1e-6));
    if (is_device(out)) {
        FIRM_CK(cudaMemcpyAsync(out, t.data(), 1024 * sizeof(float), cudaMemcpyHostToDevice, P.stream));
        FIRM_CK(cudaStreamSynchronize(P.stream));
    } else {
        std::memcpy(out, t.data(), 1024 * sizeof(float));
    }
    return FIRM_OK;
}

static int to_host(const float* src, float* dst, size_t n, cudaStream_t s) {
    if (is_device(src)) {
        FIRM_CK(cudaMemcpyAsync(dst, src, n * sizeof(float), cudaMemcpyDeviceToHost, s));
        FIRM_CK(cudaStreamSynchronize(s));
    } else {
        std::memcpy(dst, src, n * sizeof(float));
    }
    return FIRM_OK;
}

static int from_host(const float* src, float* dst, size_t n, cudaStream_t s) {
    if (is_device(dst)) {
        FIRM_CK(cudaMemcpyAsync(dst, src, n * sizeof(float), cudaMemcpyHostToDevice, s));
        FIRM_CK(cudaStreamSynchronize(s));
    } else {
        std::memcpy(dst, src, n * sizeof(float));
    }
    return FIRM_OK;
}

int firm_pc_residual_target(firm_plan_t plan, float* out) {
    if (!plan || !out) return FIRM_EINVAL;
    std::vector<float> t(1024), b(1024);
    int st = firm_pc_target(plan, t.data());
    if (st == FIRM_OK) st = firm_pc_baseline(plan, b.data());
    if (st != FIRM_OK) return st;
    for (int k = 0; k < 1024; ++k) t[k] -= b[k];
    return from_host(t.data(), out, 1024, plan->P.stream);
}

int firm_set_precond_residual(firm_plan_t plan, const float* delta) {
    if (!plan || !delta) return FIRM_EINVAL;
    std::vector<float> d(1024), b(1024);
    int st = to_host(delta, d.data(), 1024, plan->P.stream);
    if (st == FIRM_OK) st = firm_pc_baseline(plan, b.data());
    if (st != FIRM_OK) return st;
    for (int k = 0; k < 1024; ++k) b[k] += d[k];
    return firm_set_precond_table(plan, b.data());
}

int firm_pc_bin_volumes(firm_plan_t plan, float* out) {
    if (!plan || !out) return FIRM_EINVAL;
    Plan& P = plan->P;
    if (!P.have_kernel) return FIRM_ESTATE;
    FIRM_CK(launch_pc_bin_counts(P, P.ws.pc_s1, P.ws.pc_s2));
    std::vector<double> c(1024);
    FIRM_CK(cudaMemcpyAsync(c.data(), P.ws.pc_s1, 1024 * sizeof(double), cudaMemcpyDeviceToHost, P.stream));
    FIRM_CK(cudaStreamSynchronize(P.stream));
    const double n3 = (double)P.N * P.N * P.N;
    std::vector<float> v(1024);
    for (int b = 0; b < 1024; ++b) v[b] = (float)(c[b] / n3);
    if (is_device(out)) {
        FIRM_CK(cudaMemcpyAsync(out, v.data(), 1024 * sizeof(float), cudaMemcpyHostToDevice, P.stream));
        FIRM_CK(cudaStreamSynchronize(P.stream));
    } else {
        std::memcpy(out, v.data(), 1024 * sizeof(float));
    }
    return FIRM_OK;
}

int firm_pc_axis(firm_plan_t plan, float* out3) {
    if (!plan || !out3) return FIRM_EINVAL;
    Plan& P = plan->P;
    if (!P.have_kernel) return FIRM_ESTATE;
    float a[4];
    FIRM_CK(cudaMemcpyAsync(a, P.ws.axis, sizeof(a), cudaMemcpyDeviceToHost, P.stream));
    const int st = take_device_flag(P);
    if (st != FIRM_OK) return st;
    for (int i = 0; i < 3; ++i) out3[i] = a[i];
    return FIRM_OK;
}

int firm_lambda_eff(firm_plan_t plan, double* out) {
    if (!plan || !out) return FIRM_EINVAL;
    if (!plan->P.have_kernel) return FIRM_ESTATE;
    return read_lam(plan->P, out, nullptr);
}

int firm_copy_out(firm_plan_t plan, int which, void* dst) {
    if (!plan || !dst) return FIRM_EINVAL;
    Plan& P = plan->P;
    const size_t N = P.N, H3 = 2 * N * 2 * N * (N + 1);
    switch (which) {
        case FIRM_OUT_KER: return P.have_kernel ? put_out(dst, P.ws.ker, H3 * sizeof(float), P.stream) : FIRM_ESTATE;
        case FIRM_OUT_KHAT: return P.have_kernel ? put_out(dst, P.ws.khat, H3 * sizeof(float), P.stream) : FIRM_ESTATE;
        case FIRM_OUT_RHS: return P.have_rhs ? put_out(dst, P.ws.rhs, N * N * N * sizeof(float), P.stream) : FIRM_ESTATE;
        case FIRM_OUT_SAMPLES:
            return P.have_rhs ? put_out(dst, P.ws.samples, (size_t)P.p.M * P.nH * sizeof(float2), P.stream) : FIRM_ESTATE;
        case FIRM_OUT_BIN_IDS:
            if (P.bin_M < 0) return FIRM_ESTATE;
            return put_out(dst, P.ws.payload, (size_t)P.bin_M * P.nH * sizeof(uint32_t), P.stream);
        case FIRM_OUT_BIN_WORK: {
            if (P.bin_M < 0) return FIRM_ESTATE;
            int nw = 0;
            FIRM_CK(cudaMemcpyAsync(&nw, P.ws.counters, sizeof(int), cudaMemcpyDeviceToHost, P.stream));
            FIRM_CK(cudaStreamSynchronize(P.stream));
            return put_out(dst, P.ws.work, (size_t)nw * sizeof(int4), P.stream);
        }
        default: return FIRM_EINVAL;
    }
}

int firm_bin(firm_plan_t plan, int M, const double* R, int channel) {
    if (!plan || M < 0 || M > plan->P.p.M || (M > 0 && !R) || (channel != 0 && channel != 1)) return FIRM_EINVAL;
    Plan& P = plan->P;
    Workspace& w = P.ws;
    cudaError_t e = cudaSuccess;
    const double* Rd = stage(R, w.R, (size_t)M * 9, P.stream, e);
    FIRM_CK(e);
    FIRM_CK(launch_geom(Rd, M, w.geom, P.stream));
    P.launches += M > 0 ? 1 : 0;
    FIRM_CK(launch_bin(P, M, channel == 0));
    P.bin_M = M;
    P.bin_kc = channel == 0;
    P.have_kernel = P.have_rhs = false;      // the ids share memory with the other stages' buffers
    FIRM_CK(cudaStreamSynchronize(P.stream));
    return FIRM_OK;
}

int firm_bin_info(firm_plan_t plan, int* n_work, int* n_points, int* bricks_per_axis, int* brick_depth, int* chunk) {
    if (!plan) return FIRM_EINVAL;
    Plan& P = plan->P;
    if (P.bin_M < 0) return FIRM_ESTATE;
    int nw = 0;
    FIRM_CK(cudaMemcpyAsync(&nw, P.ws.counters, sizeof(int), cudaMemcpyDeviceToHost, P.stream));
    FIRM_CK(cudaStreamSynchronize(P.stream));
    if (n_work) *n_work = nw;
    if (n_points) *n_points = P.bin_M * P.nH;
    if (bricks_per_axis) *bricks_per_axis = P.bin_kc ? P.nbk : P.nbr;
    if (brick_depth) *brick_depth = P.bin_kc ? kBrickZk : kBrick;
    if (chunk) *chunk = P.chunk;
    return FIRM_OK;
}

int firm_launch_count(firm_plan_t plan, long long* out) {
    if (!plan || !out) return FIRM_EINVAL;
    *out = plan->P.launches;
    return FIRM_OK;
}

int firm_set_timing(firm_plan_t plan, int on) {
    if (!plan) return FIRM_EINVAL;
    plan->P.timing = on != 0;
    return FIRM_OK;
}

int firm_stage_times(firm_plan_t plan, double* out, int n) {
    if (!plan || !out || n < 0) return FIRM_EINVAL;
    Plan& P = plan->P;
    for (int i = 0; i < n; ++i) out[i] = 0.0;
    for (int i = 0; i < n && i < Plan::kSlots - 1; ++i) {
        if (!P.ev_used[i]) continue;
        if (cudaEventSynchronize(P.ev_b[i]) != cudaSuccess) return FIRM_ECUDA;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, P.ev_a[i], P.ev_b[i]) != cudaSuccess) return FIRM_ECUDA;
        out[i] = ms;
    }
    if (n > 9) out[9] = P.cg_iters;
    return FIRM_OK;
}

void firm_destroy(firm_plan_t plan) {
    if (!plan) return;
    if (plan->P.copy_stream) {
        cudaStreamSynchronize(plan->P.copy_stream);        // a pending upload finishes first
        cudaStreamDestroy(plan->P.copy_stream);
        cudaEventDestroy(plan->P.ev_inputs);
        cudaEventDestroy(plan->P.ev_staged);
        cudaEventDestroy(plan->P.ev_stage_read);
    }
    for (int i = 0; i < Plan::kSlots; ++i) {
        if (plan->P.ev_a[i]) cudaEventDestroy(plan->P.ev_a[i]);
        if (plan->P.ev_b[i]) cudaEventDestroy(plan->P.ev_b[i]);
    }
    delete plan;
}

const char* firm_strerror(int code) {
    switch (code) {
        case FIRM_OK: return "ok";
        case FIRM_EINVAL: return "invalid argument";
        case FIRM_ENOMEM: return "workspace too small";
        case FIRM_ECUDA: return "CUDA error";
        case FIRM_ENOTCONV: return "CG did not reach the relative tolerance";
        case FIRM_EBREAKDOWN: return "CG breakdown";
        case FIRM_ETIMEOUT: return "device wait timed out";
        case FIRM_ESTATE: return "call order (kernel or right-hand side missing)";
        case FIRM_EINTERNAL: return "internal invariant failed on the device (a binned point outside its brick or a copy wait that gave up)";
        default: return "unknown status";
    }
}

}  // extern "C"
