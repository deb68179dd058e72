// firm_internal.h -- plan state, workspace layout and kernel launchers shared by the
// translation units of the CUDA library.  Not part of the public ABI (include/firm.h).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <vector>

#include "../../include/firm.h"

namespace firm {

constexpr int kBrick = 8;             // spreading brick edge in fine-grid cells (x, y; z of A*b)
constexpr int kBrickZk = 8;           // kernel channel: brick depth along z (16 was measured 8% slower:
                                      // fewer bank conflicts, but a 57% larger region to fold)
constexpr int kKbDeg = 7;             // degree of the per-tap window polynomials
constexpr int kMaxW = 8;              // widest Kaiser-Bessel window supported
constexpr int kChunk = 8192;          // most points one spreading work item takes
constexpr int kMinChunk = 1024;       // smallest work-item size a plan may be tuned to
constexpr int kMaxBatch = 1024;       // most plans one batch holds
constexpr int kTBits = 13;            // point id = m << kTBits | t (t < 8192)
constexpr int kMaxHist = 20001;       // residual history capacity (iterations + 1)
constexpr int kRedSlots = 4096;       // per-block partial sums of a reduction
constexpr int kScanSpan = 1024;       // bricks per block of the brick scan

// Window polynomials: tap l of a point with fractional tap offset u in [0,1) has
// weight phi(u + l - W/2) = sum_j c[l][j] z^j, z = 2u - 1 (Horner in z).
struct KbPoly {
    float c[kMaxW][kKbDeg + 1];
};

// Per-image slice geometry: rows 0 and 1 of R_m (the in-plane axes u, v of the slice,
// xi = w1 u + w2 v) split into float hi + lo parts so that positions on the fine
// grid are formed to ~1e-7 cells.
struct ImgGeom {
    float uh[3], ul[3], vh[3], vl[3];
};

// CG state on the device (FP64 scalars; Section 3.3).
struct CgState {
    double rr;        // <r, z> of the current iterate (z = r unpreconditioned)
    double pq;        // <p, A p>
    double beta;      // next p = z + beta p
    double bnorm;     // ||rhs||
    double tol;       // rel_tol * ||rhs|| (0: none)
    int it;           // iterations done
    int max_iter;
    int done;         // 1: stop (converged, max_iter or breakdown)
    int status;       // firm_status of the solve
    unsigned int ticket_a, ticket_b;   // last-block counters of the two reductions
    double rz;        // <r, z> with z = P r (preconditioned solve)
    int use_pc;       // 1: preconditioned CG
    int first;        // 1 until the first preconditioner application
    unsigned int ticket_c;
    int pad_;
    double alpha;     // step length of the current iteration (set with pq)
    float alpha_f[2]; // alpha and beta as double-words (hi, lo) for the vector updates
    float beta_f[2];
};

struct Workspace {
    // inputs staged from host memory
    double* R = nullptr;
    double* shifts = nullptr;
    int32_t* gid = nullptr;
    void* images = nullptr;
    // tables
    ImgGeom* geom = nullptr;
    int32_t* htab = nullptr;        // half-disc (k1, k2) packed as k1 | k2 << 16
    int4* colinfo = nullptr;        // per k1 = 0..N/2: (first t of the column, lowest k2, highest k2, 0)
    float* h2 = nullptr;            // [group][t] h^2 (t = 0 halved)
    float* h1 = nullptr;            // [group][t] h
    float2* tw_n = nullptr;         // exp(-2 pi i j / L) for L = N, 2N, 4N
    float2* tw_2n = nullptr;
    float2* tw_4n = nullptr;
    float* dec_k = nullptr;         // deconvolution factors, Ker (2N) and A*b (N)
    float* dec_r = nullptr;
    float* dec_r4 = nullptr;        // A*b from the 4N grid (fused form): (-1)^n / phihat(n / 4N)
    // spreading
    float2* samples = nullptr;      // [m][t] h b (t = 0 halved)
    uint32_t* count = nullptr;      // per brick
    uint32_t* cursor = nullptr;
    uint32_t* payload = nullptr;    // point ids m * nH + t sorted by brick, then bank class
    uint32_t* payload_scat = nullptr;   // fused plans: the kernel channel's ids in scatter order
    uint16_t* inv_perm = nullptr;   //   and each one's position in its sorted piece
    uint8_t* cls = nullptr;         // bank class of each binned point
    float2* samples_b = nullptr;    // A*b weights in scatter order (written by the scatter pass)
    uint16_t* perm = nullptr;       // per payload position: index in scatter order within its piece
    int4* work = nullptr;           // (brick, start, count, -)
    float* wmax_item = nullptr;     // fused form: per work item, the largest |h b| of its points
    unsigned long long* scan_part = nullptr;   // brick scan: per-block (points, items) totals
    double* item_part = nullptr;    // per work item: two FP64 partial sums (data residual)
    int* counters = nullptr;        // [0] work items, [1] work cursor, [2] error flag
    double* grid = nullptr;         // fine grid, FP64 (real for Ker, complex for A*b)
    float2* fx1 = nullptr;          // FFT intermediates
    float2* fx2 = nullptr;
    // results
    float* ker = nullptr;           // Ker half box
    float* khat = nullptr;          // K-hat half spectrum
    float* rhs = nullptr;           // A*b
    // CG
    float* x = nullptr;
    float2* r = nullptr;            // residual recurrence, double-word (hi, lo) per element
    float* p = nullptr;
    float* q = nullptr;
    float2* t1 = nullptr;           // N x N x (N+1)
    float2* t2 = nullptr;           // N x 2N x (N+1)
    float* z = nullptr;             // preconditioned residual (N^3)
    float* pc_diag = nullptr;       // preconditioner, Fourier diagonal N x N x (N/2+1)
    float* pc_feat = nullptr;       // 1024-bin density histogram
    float* pc_table = nullptr;      // 1024-bin log table of the TABLE / BINNED preconditioner
    double* pc_s1 = nullptr;        // per-bin sums for the binned target
    double* pc_s2 = nullptr;
    double* red_a = nullptr;        // partial sums
    double* red_b = nullptr;
    double* hist = nullptr;
    CgState* cg = nullptr;
    float* lam = nullptr;           // device: [0] lam_eff, [1] Ker(0) of the last kernel
    float* axis = nullptr;          // device: principal viewing axis of the last kernel (3 floats)
    // FP64 CG mode only (FIRM_FLAG_FP64_CG; empty otherwise)
    double2* tw64 = nullptr;        // exp(-2 pi i k / 2N), k < N
    double* khat64 = nullptr;       // Re K-hat, full (2N)^3
    double2* c64 = nullptr;         // (2N)^3 FFT buffer
    double* x64 = nullptr;
    double* r64 = nullptr;
    double* p64 = nullptr;
    double* q64 = nullptr;
    size_t total = 0;
};

struct Plan {
    firm_params p{};
    std::vector<firm_ctf_group> groups;
    cudaStream_t stream = nullptr;
    char* base = nullptr;
    Workspace ws;
    int N = 0, Gk = 0, Gr = 0, nH = 0, nK = 0, nbk = 0, nbkz = 0, nbr = 0, n_ctf = 1;
    size_t max_work = 0;
    int chunk = kChunk;             // points per spreading work item (kMinChunk..kChunk)
    KbPoly poly{};
    double mu = 0.0;                // high-frequency damping weight (firm_set_damping)
    float h2_max = 1.0f;           // largest kernel-channel weight (bounds the fixed-point scale)
    bool have_kernel = false, have_rhs = false;
    bool timing = false;
    // stage timing: events recorded around each stage when timing is on; read lazily
    static constexpr int kSlots = 12;
    cudaEvent_t ev_a[kSlots] = {}, ev_b[kSlots] = {};
    bool ev_used[kSlots] = {};
    double cg_iters = 0;
    int num_sms = 0;
    long long launches = 0;         // kernels launched by this plan
    int pc_mode = 0;                // FIRM_PRECOND_*
    bool pc_ready = false;          // pc_diag built for the current K-hat and mode
    int last_M = 0;                 // images of the last firm_kernel
    int bin_M = -1;                 // images of the last firm_bin (its ids and items still held); -1 none
    bool bin_kc = true;             // channel of the last firm_bin (true: kernel, 4N grid)
    // device pointers of the current call's inputs (caller's or staged copies)
    const double* cur_R = nullptr;
    const double* cur_shifts = nullptr;
    const int32_t* cur_gid = nullptr;
    const void* cur_images = nullptr;
    std::vector<int32_t> htab_host;
    // images uploaded ahead of firm_backproject (firm_stage_images): copy stream,
    // events (inputs queued, copy done, staging read), and the pending upload
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t ev_inputs = nullptr, ev_staged = nullptr, ev_stage_read = nullptr;
    const void* staged_host = nullptr;
    void* staged_dev = nullptr;
    size_t staged_bytes = 0;
    int staged_M = -1;
    bool stage_started = false;
};

// Workspace layout (also used by firm_workspace_size with base = nullptr).
size_t layout_workspace(const firm_params& p, char* base, Workspace& ws);

// Host-side tables (double precision, from the definitions).
void kb_build(int W, double sigma, KbPoly& poly, double* beta_out);
double kb_phihat(double u, int W, double beta);     // FT of the normalised window
std::vector<int32_t> half_disc(int N);               // (k1, k2) packed, ordered as in firm.h
double wavelength_A(double kV);
double ctf_value(const firm_ctf_group& g, double r_invA);

// ---- launchers (spread.cu) ----
cudaError_t launch_geom(const double* R, int M, ImgGeom* geom, cudaStream_t s);
cudaError_t launch_bin(Plan& P, int M, bool kernel_channel);
cudaError_t launch_spread(Plan& P, int M, bool kernel_channel);        // clear + spread
cudaError_t launch_spread_clear(Plan& P, bool kernel_channel);          // zero the fine grid
cudaError_t launch_spread_only(Plan& P, int M, bool kernel_channel);    // spread (grid cleared)
// Both channels onto the 4N grid in one pass (clears the Ker and A*b grids first): the
// points of the kernel channel's binning (launch_bin(P, M, true)), the A*b weights read
// from ws.samples.  FIRM_FLAG_FUSED plans only.
cudaError_t launch_spread_fused(Plan& P, int M);
// The fused pass's A*b weights gathered into payload order (ws.samples_b) and each work
// item's largest |h b| (ws.wmax_item); after the image DFT, before launch_spread_fused.
cudaError_t launch_fused_gather(Plan& P, int M);
// One persistent launch spreading the binned points of n plans (same W) into their own
// fine grids; each plan's grid cleared and its points binned beforehand.  args: device
// array of n per-plan descriptors; item_off: device (n + 1) ints; queue: device int.
size_t spread_batch_desc_bytes();
void spread_batch_fill_desc(Plan& P, bool kernel_channel, void* host_desc);
cudaError_t launch_spread_batch(int n, bool kernel_channel, int W, const KbPoly& poly, const void* dev_desc,
                                int* item_off, int* queue, int num_sms, cudaStream_t s);

// ---- launchers (fft_passes.cu) ----
cudaError_t fft_init_constants();
// plain: b itself (no CTF weight, k = 0 not halved) instead of the A*b weights
cudaError_t launch_image_dft(Plan& P, int M, const void* images, const double* shifts, const int32_t* gid,
                             bool plain = false);
// Forward projector (type-2 NUFFT): the deconvolved, centred, zero-padded volume
// transformed forward on the (2N)^3 grid (ghat, G^3 complex), then interpolated at
// the A*b channel's binned points.  Forward mode (item_part == nullptr): out[m][t] =
// h_m(k_t) (A V)(xi_mt).  Residual mode: per work item sums of c |b - h A V|^2 and
// c |b|^2 into item_part, then their item-order sums into sums[0..1] (device).
cudaError_t launch_fwd_transform(Plan& P, const float* V, float2* ghat);
cudaError_t launch_interp(Plan& P, int M, const float2* ghat, float2* out, double* item_part, double* sums);
cudaError_t launch_ker_transform(Plan& P);     // grid -> Ker half box
cudaError_t launch_khat(Plan& P);              // Ker -> K-hat
cudaError_t launch_rhs_transform(Plan& P);     // grid -> A*b
cudaError_t launch_rhs_transform4(Plan& P);    // the fused form's 4N A*b grid -> A*b
cudaError_t launch_lam_eff(Plan& P);           // ws.lam from Ker(0) on the device
// Toeplitz apply y = Ker * x + lam_eff x (lam_eff read from ws.lam).  With cg != nullptr
// the first pass forms p = r + beta p in place (x = p, r given) and the last pass
// reduces <p, y>.
cudaError_t launch_toeplitz(Plan& P, const float* x, float* y, const float2* cg_r, CgState* cg,
                            const float* cg_z = nullptr);

// Preconditioner: z = P r through N^3 FFTs with the Fourier diagonal pc_diag; the last
// pass reduces <r, z> and sets beta (fft_passes.cu).
cudaError_t launch_precond(Plan& P, const float2* r, float* z, CgState* cg);
cudaError_t launch_chan_spectrum(Plan& P);       // T. Chan circulant spectrum into ws.t1 (half spectrum)
cudaError_t launch_pc_build_circulant(Plan& P);  // pc_diag = 1 / ((kappa + lam_eff) N^3) from ws.t1

// ---- launchers (lpre.cu) ----
cudaError_t launch_view_axis(Plan& P, const double* R, int M);
cudaError_t launch_pc_features(Plan& P, int M, float* hist);
// hist <- hist / sum(hist); x (nullable) <- log(1024 hist + 1e-3), the network input
cudaError_t launch_pc_normalize(Plan& P, float* hist, float* x);
cudaError_t launch_pc_target_sums(Plan& P, double* s1, double* s2);
cudaError_t launch_pc_bin_counts(Plan& P, double* s1, double* s2);     // grid frequencies per bin
cudaError_t launch_pc_from_table(Plan& P, const float* table);

// ---- launchers (cg64.cu): the FP64 CG mode ----
cudaError_t launch_khat64(Plan& P);                 // khat64 from the Ker half box
cudaError_t launch_damping(Plan& P);                // mu D^T D added to K-hat (and khat64); no-op at mu = 0
// Positivity-constrained solve (poscg.cu) on the plan's A*b and K-hat; x: device N^3.
// Returns a firm_status (FIRM_ENOTCONV at max_iter).
int pos_solve(Plan& P, float* x, int max_iter, double rel_tol, int* iters_out);
// CG from x0 = 0 (first_iter == 0 queues the initialisation), then n_iter iterations.
cudaError_t launch_cg64(Plan& P, const float* rhs, int max_iter, double rel_tol, int first_iter, int n_iter);
cudaError_t launch_cg64_result(Plan& P);            // x64 -> ws.x (float)

// ---- launchers (cg.cu) ----
cudaError_t launch_cg_init(Plan& P, const float* rhs, int max_iter, double rel_tol, bool use_pc);
cudaError_t launch_cg_update(Plan& P);

}  // namespace firm

// The opaque plan handle of include/firm.h.
struct firm_plan_s {
    firm::Plan P;
};
