/*
 * firm.h -- C ABI of the GB300 FIRM hot path.
 *
 * FIRM (Wang, Shkolnisky & Singer, "A Fourier-based Approach for Iterative 3D
 * Reconstruction from Cryo-EM Images") reconstructs a volume V from M projection
 * images with known rotations R_m, shifts s_m and CTFs h_m by solving
 *     (A*A + lam_eff I) V = A*b                                  (Section 3.3)
 * with conjugate gradients, where A*A is applied as a convolution with the kernel
 * Ker through a 2N circulant embedding (Section 3.2, eq. property,
 * eq. embedding_circulant) and Ker and A*b are computed once by type-1 NUFFT
 * (Section 3.4, steps 2-3; eq. kernel, eq. backprojection).
 *
 * Conventions (shared by every entry point):
 *   - A volume is N^3 float32, row-major [i3][i2][i1] (i1 = x fastest), voxel index
 *     i_j <-> centred coordinate n_j = i_j - N/2 (Section 3.1).
 *   - Images are M x N x N, [m][i2][i1], float32 or bfloat16 (firm_params.img_dtype),
 *     starting at a 16-byte aligned address (each image is moved into shared memory by
 *     one bulk copy); a misaligned image array is rejected with FIRM_EINVAL.
 *   - R is M x 9 float64, each rotation row-major.  The slice of image m samples
 *     the points xi = R_m^T (2 pi k1 / N, 2 pi k2 / N, 0) for |k| <= N/2
 *     (eq. forward-projector, eq. truncation: the symmetric disc).
 *   - shifts is M x 2 float64 (x, y) in pixels; the samples of image m are
 *     multiplied by exp(+2 pi i <k, s_m> / N) before back-projection.
 *   - group is M int32 defocus-group indices into the plan's CTF table.
 *   - K-hat (the eigenvalues of the circulant, eq. circ1) is real; it is stored as
 *     the half spectrum 2N x 2N x (N+1) float32, [j3][j2][j1] with j1 in [0, N].
 *   - Ker is stored the same way: [n3+N][n2+N][n1], n1 in [0, N], n2, n3 in [-N, N)
 *     (Ker(-n) = Ker(n), so the half holds every value).
 *
 * Pointers: every array argument may be host or device memory (the library asks
 * the CUDA runtime which).  Host inputs are copied into the plan's workspace; host
 * outputs are copied back before the call returns.  Device arrays are read or
 * written in stream order on the plan's stream; the call returns without waiting
 * unless a host output, a host residual history or a relative tolerance needs it.
 * In particular firm_kernel and firm_backproject with device inputs and outputs (or
 * null outputs) queue their work and return: lam_eff, Ker(0) and the principal viewing
 * axis stay on the device until a query (firm_lambda_eff, firm_pc_axis) reads them.
 *
 * Ownership: the caller owns every array it passes, including the plan's
 * workspace (firm_workspace_size / firm_plan); the library allocates no device
 * memory of its own.  Buffers must not be freed while work queued on the stream may
 * still use them.
 *
 * Errors: every call returns a firm_status; nothing aborts or throws.  A call that
 * fails leaves its outputs unspecified; the plan stays usable unless the status is
 * FIRM_ECUDA (a CUDA error: the context may be lost).
 */
#ifndef FIRM_H
#define FIRM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FIRM_OK = 0,
    FIRM_EINVAL = 1,      /* bad argument: size, null pointer, unsupported option */
    FIRM_ENOMEM = 2,      /* workspace smaller than firm_workspace_size() */
    FIRM_ECUDA = 3,       /* a CUDA runtime call or kernel launch failed */
    FIRM_ENOTCONV = 4,    /* CG reached max_iter above rel_tol */
    FIRM_EBREAKDOWN = 5,  /* CG breakdown: <p, Ap> <= 0 or a non-finite scalar */
    FIRM_ETIMEOUT = 6,    /* a bounded device wait gave up (never expected) */
    FIRM_ESTATE = 7,      /* call order: e.g. firm_cg_solve before firm_kernel */
    FIRM_EINTERNAL = 8    /* an internal invariant failed on the device (a binned point
                           * outside its brick, or a bounded wait for an asynchronous copy
                           * that gave up; never expected).  Device kernels record it
                           * in the plan; it is reported, and cleared, by the next call that
                           * waits for the stream (a host output, firm_cg_solve,
                           * firm_lambda_eff, firm_pc_axis), not by the call that queued it. */
} firm_status;

enum { FIRM_IMG_F32 = 0, FIRM_IMG_BF16 = 1 };
enum { FIRM_LAMBDA_RELATIVE = 0, FIRM_LAMBDA_ABSOLUTE = 1 };

/* One defocus group of the CTF of Section 3.1, read as
 *   h(r) = -sin(chi(r) + amp_contrast) * exp(-bfactor_A2 * r^2 / 4),
 *   chi(r) = pi * lambda * defocus_A * r^2 - (pi/2) * Cs * lambda^3 * r^4,
 * r = |k| / (N * pixel_A) in 1/Angstrom, lambda the relativistic wavelength at kV,
 * Cs = Cs_mm * 1e7 Angstrom.  amp_contrast enters as a phase in radians. */
typedef struct {
    double defocus_A, kV, Cs_mm, amp_contrast, pixel_A, bfactor_A2;
} firm_ctf_group;

typedef struct {
    int N;            /* volume edge: 16, 32, 48, 64, 80, 96 or 128 */
    int M;            /* largest image count any call on the plan will pass; M < 2^19 and
                         M * (|K| + 1) / 2 < 2^31 (|K| = the disc size), else FIRM_EINVAL */
    int n_groups;     /* defocus groups in the CTF table; 0 means no CTF (h = 1) */
    int W;            /* Kaiser-Bessel window width in fine-grid cells: 6, 7 or 8 */
    double sigma;     /* NUFFT oversampling; only 2 is supported */
    double lambda;    /* Tikhonov weight */
    int lambda_mode;  /* FIRM_LAMBDA_RELATIVE: lam_eff = lambda * Ker(0); ABSOLUTE: lambda */
    int disc_mode;    /* 0: symmetric disc |k| <= N/2 (the only mode of the CUDA path) */
    int img_dtype;    /* FIRM_IMG_F32 or FIRM_IMG_BF16 */
    int flags;        /* 0, or FIRM_FLAG_FP64_CG and / or FIRM_FLAG_FUSED */
} firm_params;

/* FIRM_FLAG_FP64_CG: firm_cg_solve runs CG (Section 3.3) with FP64 vectors and an FP64
 * Toeplitz apply (eq. property through the 2N circulant of Section 3.2, K-hat recomputed
 * in FP64 by firm_kernel).  N must be 16, 32 or 64; plain CG only (a preconditioner
 * set with firm_set_precond makes firm_cg_solve return FIRM_EINVAL); not accepted by
 * firm_batch_create.  Ker and A*b still come from the FP32 NUFFT.  A long fixed-count
 * CG iterate is sensitive to the ~1e-7 rounding of FP32 FFTs; this mode removes that
 * rounding from the solve, at FP64 speed.  The workspace grows by about
 * (2N)^3 * 24 + N^3 * 32 bytes. */
enum { FIRM_FLAG_FP64_CG = 1 };

/* FIRM_FLAG_FUSED: the plan can run firm_kernel_backproject, which spreads both
 * channels of FIRM steps 2-3 (eq. kernel, eq. backprojection) onto the one 4N^3 fine
 * grid in a single pass over the slice points.  The workspace grows by 2 (4N)^3
 * doubles (the complex A*b grid beside the real Ker grid: 2.1 GB at N = 128).  May be
 * combined with FIRM_FLAG_FP64_CG; not accepted by firm_batch_create. */
enum { FIRM_FLAG_FUSED = 2 };

typedef struct firm_plan_s* firm_plan_t;

/* Bytes of device workspace a plan with these parameters needs (the layout of
 * firm_plan: fine grid, FFT intermediates, CG vectors; Section 3.4 steps 1-4). */
int firm_workspace_size(const firm_params* p, size_t* bytes);

/* Create a plan for FIRM's precomputation and CG (Section 3.4, steps 1-4; the CTF of
 * Section 3.1, the window and deconvolution of the type-1 NUFFT of Section 3.4, the
 * FFTs of the circulant embedding of Section 3.2): validates p, copies the CTF table
 * (n_groups entries; may be NULL
 * when n_groups == 0), precomputes the Kaiser-Bessel window polynomials, the
 * deconvolution factors and the FFT tables, and carves `workspace` (device memory,
 * at least firm_workspace_size bytes, 256-byte aligned) into its buffers.  stream is
 * a cudaStream_t (NULL = legacy default stream).  On success *out owns no device
 * memory; firm_destroy releases its host state. */
int firm_plan(firm_plan_t* out, const firm_params* p, const firm_ctf_group* groups,
              void* workspace, size_t workspace_bytes, void* stream);

/* FIRM step 3 (Section 3.4; eq. kernel, eq. embedding_circulant, eq. circ1).
 * Spreads the CTF^2-weighted slice samples of M <= p.M images onto the 4N^3 fine
 * grid, transforms and deconvolves it to Ker on [-N, N)^3, embeds Ker in the 2N^3
 * circulant and transforms it to K-hat, which the plan keeps for firm_cg_solve and
 * firm_toeplitz_apply.  khat_out (nullable) receives a copy of K-hat (half
 * spectrum, see above).  Also fixes lam_eff (firm_lambda_eff). */
int firm_kernel(firm_plan_t plan, int M, const double* R, const int32_t* group, float* khat_out);

/* FIRM steps 1-2 (Section 3.4; eq. measurement, eq. backprojection).  Takes the
 * centred 2D DFT of each image on the disc, applies the shift phase and h_m, spreads
 * the samples onto the 2N^3 fine grid, transforms and deconvolves to A*b on N^3.
 * The plan keeps A*b; rhs_out (nullable) receives a copy (N^3 float32). */
int firm_backproject(firm_plan_t plan, int M, const void* images, const double* shifts,
                     const double* R, const int32_t* group, float* rhs_out);

/* FIRM steps 1-3 in one call, the two spreading channels fused (Section 3.4; eq.
 * measurement, eq. backprojection, eq. kernel, eq. embedding_circulant, eq. circ1).
 * Both sums run over the same slice points xi_{m,k} with the same window, so the
 * points are binned once on the 4N^3 grid (poses only: this runs while a staged image
 * upload, firm_stage_images, is still landing), the images are transformed to h b on
 * the disc, the h b of every point is gathered into the binning's order, and one
 * spreading pass adds h^2 phi to the Ker grid and h b phi to the A*b grid (complex,
 * 4N^3); Ker (on [-N, N)^3), K-hat, lam_eff and A*b (on N^3, from the
 * 4N grid: oversampling 4 for its N modes) follow as in firm_kernel and
 * firm_backproject, whose results it replaces.  Arguments as those two calls;
 * khat_out and rhs_out are nullable.  FIRM_EINVAL unless the plan was made with
 * FIRM_FLAG_FUSED.  Host images not staged ahead are copied into the workspace and
 * transformed before the binning (no overlap). */
int firm_kernel_backproject(firm_plan_t plan, int M, const void* images, const double* shifts,
                            const double* R, const int32_t* group, float* khat_out, float* rhs_out);

/* Sums formed elsewhere, loaded into the plan.  Ker and A*b are sums over the images
 * (eq. kernel, eq. backprojection; Section 3.4), so a reconstruction can be split by
 * images: every process runs firm_kernel and firm_backproject (or
 * firm_kernel_backproject) on its own images, copies out FIRM_OUT_KER and FIRM_OUT_RHS,
 * the copies are summed across processes (one all-reduce), and each process loads the
 * sums here.  ker_half (nullable): the Ker half box, 2N x 2N x (N+1) float32 as
 * FIRM_OUT_KER; K-hat (eq. embedding_circulant, eq. circ1), lam_eff and the damping
 * are formed from it as firm_kernel does.  rhs (nullable): A*b, N^3 float32.  Host or
 * device memory.  The learned and binned preconditioners also use the viewing axis,
 * which only firm_kernel forms from the poses.  FIRM_EINVAL if both are NULL. */
int firm_load_sums(firm_plan_t plan, const float* ker_half, const float* rhs);

/* Forward projector A (Section 3.1, eq. forward-projector; with eq. truncation's disc):
 *     (A V)_m(k) = h_m(|w_k|) sum_n V_n exp(-i <n, xi_{m,k}>),  xi = R_m^T (2 pi k / N, 0),
 * for the half disc of every image (the order of FIRM_OUT_SAMPLES: (0, k2) for
 * k2 = 0..N/2, then k1 = 1..N/2 with every k2 of the disc; the other half is the
 * complex conjugate for a real V).  Computed as a type-2 NUFFT: V divided by the
 * window's transform, zero-padded to the (2N)^3 fine grid, transformed, and
 * interpolated with the same Kaiser-Bessel window at each slice point.  V: N^3
 * float32 (host or device).  out: M x |K|/2 complex float32 (interleaved re, im; host
 * or device).  group may be NULL (group 0).  Uses the fine grid and the binning
 * buffers of the plan (its kept Ker, K-hat and A*b are not touched).  FIRM_EINVAL:
 * M < 0 or above the plan's M, or a null pointer with M > 0. */
int firm_forward(firm_plan_t plan, int M, const float* V, const double* R, const int32_t* group, float* out);

/* Data term of the reconstruction (Section 3.3: the least-squares residual the
 * solution minimises, used for the L-curve of Section 3.3): with b_m(k) the centred
 * DFT of image m with its shift phase (eq. measurement, as firm_backproject takes it)
 * and A the forward projector above, out2[0] = sum over m and the whole disc K of
 * |b_m(k) - (A V)_m(k)|^2 and out2[1] = sum of |b_m(k)|^2, both in FP64 (the half
 * disc counted twice except k = 0).  Sums go through one FP64 partial per binning
 * work item (no floating-point atomics); the points' order within the binning varies
 * between calls, so repeated calls agree to FP64 rounding.  Arguments as firm_backproject
 * plus V (N^3 float32, host or device); out2: 2 doubles (host or device).  M = 0
 * gives zeros.  FIRM_EINVAL as firm_forward, or out2 NULL. */
int firm_data_residual(firm_plan_t plan, int M, const float* V, const void* images, const double* shifts,
                       const double* R, const int32_t* group, double* out2);

/* Upload of host images ahead of firm_backproject (Section 3.4, step 1's input), so
 * that the copy overlaps firm_kernel, which does not read the images.  Records an
 * upload of M host images (images: host memory, M x N x N in the plan's image type,
 * row major; page-locked for the copy to run asynchronously) into `staging` (device
 * memory owned by the caller, at least M * N * N * element-size bytes) and returns.
 * The copy runs on a copy stream of the plan; it is issued by the plan's next
 * firm_kernel once that call has queued its own small uploads (so they do not wait
 * behind the images), or by firm_backproject if no firm_kernel comes first.  The next
 * firm_backproject called with the same host pointer and the same M orders itself
 * after the copy and reads the staged images; any other call copies as usual.  The
 * caller keeps `images` and `staging` unchanged until that firm_backproject has
 * returned.  A later upload waits for the previous staged images to be read.
 * firm_destroy waits for a copy in flight.  FIRM_EINVAL: M < 0 or above the plan's
 * M, a null pointer with M > 0, images in device memory, staging not in device memory
 * or too small. */
int firm_stage_images(firm_plan_t plan, int M, const void* images, void* staging, size_t staging_bytes);

/* FIRM step 4 (Section 3.3): conjugate gradients on (A*A + lam_eff I) x = rhs from
 * x = 0, with FP64 step lengths and residual recurrence.  rhs may be NULL (use the
 * A*b kept by firm_backproject).  Runs max_iter iterations, or stops once the
 * recurrence residual ||r_k|| <= rel_tol ||rhs|| (rel_tol > 0; the check reads one
 * flag per batch of iterations).  x receives the iterate (N^3).  resid_hist
 * (nullable, max_iter+1 doubles) receives ||r_k|| for k = 0..iters; *iters_out
 * (nullable) the iterations run.  Returns FIRM_ENOTCONV if rel_tol > 0 was not met,
 * FIRM_EBREAKDOWN on <p, Ap> <= 0 or a non-finite scalar (x then holds the last
 * good iterate). */
int firm_cg_solve(firm_plan_t plan, const float* rhs, float* x, int max_iter, double rel_tol,
                  double* resid_hist, int* iters_out);

/* Positivity constraint (Section 5 names positivity among the prior knowledge FIRM can
 * take in; the paper gives no method, and this reading is the quadratic of Section 3.3
 * restricted to V >= 0):
 *     min 1/2 <V, H V> - <A*b, V>  subject to V >= 0,  H = A*A + lam_eff I (+ the damping),
 * solved from V = 0 by conjugate gradients on the free voxels with projection and
 * restarts (Polyak's method for bound-constrained quadratics: a step is capped where a
 * voxel would cross zero, the blocking voxels are set to 0 and CG restarts; a voxel held
 * at 0 is released when its residual turns positive).  Uses the plan's A*b and K-hat
 * (firm_backproject and firm_kernel first).  Stops when the residual on the free voxels
 * is <= rel_tol ||A*b|| and no voxel held at 0 has a positive residual (the KKT
 * conditions), or after max_iter Toeplitz applies (FIRM_ENOTCONV; x then holds the last
 * feasible iterate).  x: N^3 float32 (host or device), x >= 0 on return.  *iters_out
 * (nullable): Toeplitz applies.  The host reads two scalars per step.  FIRM_ESTATE:
 * no K-hat or A*b yet; FIRM_EINVAL: x NULL, max_iter < 0, rel_tol < 0 or not finite;
 * FIRM_EBREAKDOWN: <p, H p> <= 0. */
int firm_solve_nonneg(firm_plan_t plan, float* x, int max_iter, double rel_tol, int* iters_out);

/* High-frequency damping (Section 5: FIRM can take regularisers that are natural in
 * Fourier space, damping high frequencies among them; the paper gives no formula, and
 * this reading is the first-difference penalty).  From the next firm_kernel on, the
 * system solved by firm_cg_solve (and applied by firm_toeplitz_apply) is
 *     (A*A + mu_eff D^T D + lam_eff I) V = A*b,
 * D the first differences of V along x, y, z on its box (V = 0 outside), i.e. the
 * kernel Ker gains the 7-point stencil 6 delta(n) - sum of delta(n -+ e_a); it is added
 * to K-hat (spectrum 6 - 2 sum_a cos(pi j_a / N) on the 2N grid), so a CG iteration
 * costs the same.  mu_eff = mu * Ker(0) under FIRM_LAMBDA_RELATIVE, mu under
 * FIRM_LAMBDA_ABSOLUTE.  K-hat-based preconditioners see the damped spectrum.
 * mu = 0 (the default) switches it off.  FIRM_EINVAL: mu < 0 or not finite. */
int firm_set_damping(firm_plan_t plan, double mu);

/* Preconditioner used by firm_cg_solve from its next call on (an addition to the
 * paper, whose CG is unpreconditioned).  FIRM_PRECOND_NONE: plain CG (Section 3.3).
 * FIRM_PRECOND_CIRCULANT: z = F^-1 diag(1 / (kappa(k) + lam_eff)) F r on the N^3 grid,
 * kappa the spectrum of T. Chan's optimal circulant of the Toeplitz operator (the
 * circulant nearest to it in Frobenius norm; column sum over n = m mod N of
 * Ker(n) prod_a (N - |n_a|)/N), built on the circulant diagonalisation of Section 2.3.
 * kappa >= 0 for A*A; the floor is lam_eff (or 1e-6 kappa(0) when lam_eff = 0).  The
 * stopping test stays ||r_k|| <= rel_tol ||rhs||; beta is the flexible (Polak-Ribiere)
 * form, equal to the textbook one in exact arithmetic.
 * FIRM_PRECOND_BINNED: the same Fourier diagonal averaged per radial-angular bin (64 shells
 * of |q|/(N/2) x 16 cones of |cos| to the principal viewing axis; see firm_pc_target) --
 * the direct, network-free control of the learned preconditioner.
 * FIRM_PRECOND_TABLE: the per-bin table given to firm_set_precond_table (for example the
 * learned network's output). */
enum { FIRM_PRECOND_NONE = 0, FIRM_PRECOND_CIRCULANT = 1, FIRM_PRECOND_BINNED = 2, FIRM_PRECOND_TABLE = 3 };
int firm_set_precond(firm_plan_t plan, int mode);

/* Learned-preconditioner interface (no counterpart in the paper).  Bins: a
 * frequency q (N-grid units) is in shell s = min(63, floor(64 |q| / (N/2))) and cone
 * c = min(15, floor(16 |<q/|q|, a>|)), bin = 16 s + c, a = firm_pc_axis (eigenvector of
 * the largest eigenvalue of the second moment of the viewing directions R_m^T e3 of
 * the last firm_kernel).
 * firm_pc_features: h^2-weighted density of the slice samples per bin, summing to 1
 *   (1024 floats, host or device).
 * firm_pc_target: t_b = log(p_b Ker(0)), p_b = sum (kappa + lam_eff) / sum (kappa +
 *   lam_eff)^2 over the bin, kappa the spectrum of FIRM_PRECOND_CIRCULANT (least-squares
 *   fit of 1/(kappa + lam_eff) by one value per bin); empty bins copy the nearest
 *   non-empty shell of the same cone.
 * firm_set_precond_table: use d(q) = exp(table_log[bin(q)]) / Ker(0) as the
 *   preconditioner (selects FIRM_PRECOND_TABLE). */
int firm_pc_features(firm_plan_t plan, float* out1024);

/* The learned network's input for the plan's last kernel, on the device: the features
 * of firm_pc_features (the h^2-weighted share of the slice samples in each of the 1024
 * shell x cone bins) mapped to x_b = log(1024 f_b + 1e-3).  out: 1024 float32, host
 * or device.  Not in the paper (the learned preconditioner is an addition to its CG,
 * Section 3.3).  FIRM_ESTATE before firm_kernel. */
int firm_pc_net_input(firm_plan_t plan, float* out);
int firm_pc_target(firm_plan_t plan, float* out1024);
int firm_pc_axis(firm_plan_t plan, float* out3);
/* Fraction of the N^3 frequency grid (FFT index order, q in [-N/2, N/2)) falling in each
 * of the 1024 (shell, cone) bins of the last firm_kernel's principal axis: 1024 float32,
 * summing to 1.  With the density features f this gives the density per unit volume
 * f_b / v_b, which for a sampling operator is the bin's mean eigenvalue / Ker(0). */
int firm_pc_bin_volumes(firm_plan_t plan, float* out);
/* A per-bin log table from the sampling density alone: t_b = -log(f_b / v_b + r), f the
 * features (firm_pc_features), v the bin volumes, r the relative Tikhonov weight
 * lambda_eff / Ker(0).  A closed-form estimate of the target of firm_pc_target (the
 * bin's mean eigenvalue / Ker(0) is about f_b / v_b for a sampling operator); the
 * learned preconditioner predicts the difference from it.  1024 float32. */
int firm_pc_baseline(firm_plan_t plan, float* out);
/* firm_pc_target minus firm_pc_baseline (what the learned preconditioner is trained on),
 * and FIRM_PRECOND_TABLE set from baseline + delta (its prediction added back). */
int firm_pc_residual_target(firm_plan_t plan, float* out);
int firm_set_precond_residual(firm_plan_t plan, const float* delta);
int firm_set_precond_table(firm_plan_t plan, const float* table_log1024);

/* The network of the learned preconditioner: 1024 -> 256 -> 256 -> 1024 with ReLU, input
 * x_b = log(1024 f_b + 1e-3) of the features, output the log table t.  Parameters are one
 * float32 array of firm_mlp_param_count() values: W1 (256 x 1024), b1, W2 (256 x 256),
 * b2, W3 (1024 x 256), b3 (W row-major, out x in).  All arrays are device memory; work
 * holds firm_mlp_work_floats(batch) floats; calls are queued on `stream`.
 *   forward:   y (batch x 1024) from x (batch x 1024), FP32.
 *   to_bf16 / forward_bf16: BF16 copy of the weights (2 bytes each) and the forward pass
 *              with BF16 weights, FP32 biases and FP32 accumulation (inference).
 *   grad:      mean squared error of y against t and its gradient (same layout as the
 *              parameters); *loss is device memory.
 *   adam:      one Adam step (beta1 0.9, beta2 0.999, eps 1e-8, step counted from 1). */
int firm_mlp_param_count(void);
size_t firm_mlp_work_floats(int batch);
int firm_mlp_forward(const float* params, int batch, const float* x, float* y, float* work, void* stream);
int firm_mlp_to_bf16(const float* params, void* params_bf16, void* stream);
int firm_mlp_forward_bf16(const void* params_bf16, const float* params, int batch, const float* x, float* y,
                          float* work, void* stream);
int firm_mlp_grad(const float* params, int batch, const float* x, const float* t, float* grad, float* work,
                  double* loss, void* stream);
int firm_mlp_adam(float* params, const float* grad, float* m, float* v, int step, float lr, void* stream);

/* One application of the regularised normal operator, y = Ker * x + lam_eff x
 * (eq. property through the circulant embedding of Section 3.2), using the K-hat of
 * the last firm_kernel.  x and y are N^3 and must not overlap. */
int firm_toeplitz_apply(firm_plan_t plan, const float* x, float* y);

/* The same operator as firm_toeplitz_apply, y = Ker * x + lam_eff x, for callers that
 * cannot allocate device memory and have no plan workspace to lend (for example a host
 * application whose own allocator holds all device memory, or a code path that must not
 * change the device memory footprint).  The paper has no counterpart: this is an
 * interface variant.  It allocates nothing: the FFT scratch lives in one static device
 * array inside the library, sized for N <= 64 (about 6.4 MB, resident on every device
 * that loads the library until the process exits).
 *   N       16, 32, 48 or 64; larger N is rejected with FIRM_EINVAL.
 *   khat    K-hat half spectrum, 2N x 2N x (N+1) float32, device memory
 *           (from firm_kernel(..., khat_out) or firm_copy_out(FIRM_OUT_KHAT)).
 *   lam_eff Tikhonov weight added (>= 0), e.g. firm_lambda_eff of that plan.
 *   x, y    N^3 float32 device arrays, distinct.
 *   stream  cudaStream_t the passes are queued on; the call does not wait.
 * All four pointers must be memory of the current device; anything else is rejected
 * with FIRM_EINVAL.  The first call on a device does a one-time set-up: it looks up the
 * array's device address and writes the FFT twiddles of every supported N into it with
 * a synchronous copy (once per device, under a lock), so that first call waits for the
 * device.  Later calls only queue kernels.  All calls share the one array:
 * calls whose work overlaps on the GPU (other streams, other threads) race and must be
 * serialised by the caller.  Every pass writes its scratch before reading it, so
 * nothing has to start at zero. */
int firm_toeplitz_apply_static(int N, const float* khat, double lam_eff, const float* x, float* y, void* stream);

/* lam_eff of the last firm_kernel (Tikhonov weight actually added to A*A). */
int firm_lambda_eff(firm_plan_t plan, double* out);

/* Copies of intermediate results kept by the plan (for verification):
 *   FIRM_OUT_KER   Ker half box, 2N x 2N x (N+1) float32 (eq. kernel)
 *   FIRM_OUT_KHAT  K-hat half spectrum, 2N x 2N x (N+1) float32 (eq. circ1)
 *   FIRM_OUT_RHS   A*b, N^3 float32 (eq. backprojection)
 *   FIRM_OUT_SAMPLES  h_m b_m(k) on the half disc, M x |H| complex float32, with the
 *                  k = 0 sample halved (the symmetric completion doubles it back).
 *                  |H| = (|K| + 1) / 2, ordered by k1 = 0..N/2 then k2 ascending,
 *                  starting (0,0), (0,1), ... (0,N/2), (1,-..), ... */
enum { FIRM_OUT_KER = 0, FIRM_OUT_KHAT = 1, FIRM_OUT_RHS = 2, FIRM_OUT_SAMPLES = 3,
       FIRM_OUT_BIN_IDS = 4, FIRM_OUT_BIN_WORK = 5 };
int firm_copy_out(firm_plan_t plan, int which, void* dst);

/* The binning step of the spreading (slice geometry of eq. forward-projector, points
 * grouped per brick of the fine grid; Section 3.4 steps 2-3) run alone, for
 * verification: the points of images 0..M-1 (R: M x 9 float64) are binned for the
 * kernel channel (channel 0: fine grid 4N, bricks of 8^3 cells) or the A*b channel
 * (channel 1: fine grid 2N).  Afterwards
 *   FIRM_OUT_BIN_IDS   M * |H| uint32 point ids (m << 13 | t, t the half-disc index of
 *                      FIRM_OUT_SAMPLES), grouped by work item;
 *   FIRM_OUT_BIN_WORK  n_work work items, 4 int32 each: (brick, first id position,
 *                      point count, 0); brick = (bz * nb + by) * nb + bx;
 * and firm_bin_info gives n_work, M * |H|, nb (bricks per axis along x and y), the
 * brick depth along z in cells (bricks are 8 x 8 x depth) and the most points of an
 * item.  Within an item the points are ordered round-robin over the 32 bank
 * classes of their first tap.  firm_bin reuses the memory of the kernel and A*b
 * results: call firm_kernel / firm_backproject again before using those. */
int firm_bin(firm_plan_t plan, int M, const double* R, int channel);
int firm_bin_info(firm_plan_t plan, int* n_work, int* n_points, int* bricks_per_axis, int* brick_depth, int* chunk);

/* Device time of the last call of each stage, in milliseconds between CUDA events
 * recorded on the plan's stream around the stage (recorded only while timing is on,
 * firm_set_timing(plan, 1); recording adds no host synchronisation).  Slots:
 *   0 geometry + binning (kernel channel)   1 spreading (kernel channel)
 *   2 4N^3 transform + deconvolution (Ker) 3 circulant K-hat
 *   4 geometry + image DFT                  5 binning (A*b channel)
 *   6 spreading (A*b channel)               7 2N^3 transform + deconvolution (A*b)
 *   8 CG total                              9 CG iterations of the last solve
 *  10 the fused form's weight gather (firm_kernel_backproject; its spreading is slot 1)
 * firm_stage_times waits for the recorded events and fills out[0..n-1]. */
int firm_set_timing(firm_plan_t plan, int on);
int firm_stage_times(firm_plan_t plan, double* out, int n);

/* Number of CUDA kernels this plan has launched since firm_plan (for accounting). */
int firm_launch_count(firm_plan_t plan, long long* out);

void firm_destroy(firm_plan_t plan);
const char* firm_strerror(int code);

/* ---- Batched reconstructions ------------------------------------------------------
 * Many independent FIRM reconstructions (Section 3.4, steps 1-4 each: Ker, A*b, K-hat,
 * then a fixed number of CG iterations from x0 = 0) run as one unit of work.  Each
 * reconstruction is a plan of its own (its own N, image count, CTF table and
 * workspace); all plans of a batch share W and the device.  The paper reconstructs
 * one volume at a time: batching is an execution form of the same steps, and each
 * volume equals what firm_kernel + firm_backproject + firm_cg_solve(max_iter = iters,
 * rel_tol = 0) give for that plan, up to the order of floating-point additions.
 *
 * Execution: the plans' stages are queued on n_streams worker streams forked from
 * the batch's stream (plans dealt out largest first).  With FIRM_BATCH_PERSISTENT the
 * spreading of every plan (each channel) is one persistent launch over one shared
 * queue of work items; otherwise each plan spreads on its own stream.  With
 * FIRM_BATCH_GRAPH the whole batch is captured once into a CUDA graph and replayed
 * while the items, iteration count, flags and tuning stay the same (changing any of
 * them captures a new graph).
 *
 * The batch needs a small device workspace from the caller (descriptors and work
 * queues): firm_batch_workspace_size.  It creates its own CUDA streams and events. */
typedef struct firm_batch_s* firm_batch_t;

typedef struct {
    int M;                  /* images of this reconstruction, 0 <= M <= the plan's M */
    const double* R;        /* device, M x 9 float64 */
    const int32_t* group;   /* device, M int32, or NULL (every image in group 0) */
    const void* images;     /* device, M x N x N in the plan's image dtype */
    const double* shifts;   /* device, M x 2 float64, or NULL (no shifts) */
    float* x;               /* device, N^3 float32: the reconstructed volume */
} firm_batch_item;

enum { FIRM_BATCH_GRAPH = 1, FIRM_BATCH_PERSISTENT = 2, FIRM_BATCH_LEARNED = 4 };

int firm_batch_workspace_size(int n_plans, size_t* bytes);
/* plans: n_plans distinct plans (not destroyed while the batch lives).  n_streams in
 * 1..64 (worker streams; the tuner may lower it).  stream: the batch's cudaStream_t;
 * plans' own streams are not used by batch runs. */
int firm_batch_create(firm_batch_t* out, int n_plans, const firm_plan_t* plans, int n_streams, void* workspace,
                      size_t workspace_bytes, void* stream);
/* Queues every reconstruction (items[i] for plans[i]) on the batch's stream and
 * returns without waiting.  iters in 0..20000; flags: FIRM_BATCH_*. */
int firm_batch_run(firm_batch_t batch, const firm_batch_item* items, int iters, int flags);
/* Every reconstruction solved to a relative residual (Section 3.3 with the stopping rule
 * of firm_cg_solve): steps 1-3 as firm_batch_run (graph-captured with FIRM_BATCH_GRAPH,
 * persistent spreading with FIRM_BATCH_PERSISTENT), then preconditioned CG from x0 = 0
 * until ||r|| <= rel_tol ||A*b|| or max_iter, every plan on its own.  Preconditioner of
 * plan i: with FIRM_BATCH_LEARNED the batch's network (firm_batch_set_network) maps the
 * plans' density features (firm_pc_net_input), all plans in one forward pass, to their
 * FIRM_PRECOND_TABLE tables; otherwise the plan's own mode (firm_set_precond; NONE,
 * CIRCULANT or a TABLE set with firm_set_precond_table; BINNED needs the host per plan
 * and gives FIRM_EINVAL).  The iterations run in chunks of 8 per plan (one CUDA graph
 * per chunk with FIRM_BATCH_GRAPH); between chunks the host reads one count of the plans
 * not yet stopped, so the call returns when every plan has stopped.  The volumes are in
 * items[i].x; firm_batch_wait reports per plan FIRM_OK, FIRM_ENOTCONV (rel_tol not met
 * at max_iter) or FIRM_EBREAKDOWN and the iterations.  Not in the paper (an execution
 * form and an addition to its CG).  FIRM_ESTATE: FIRM_BATCH_LEARNED without a network. */
int firm_batch_solve(firm_batch_t batch, const firm_batch_item* items, int max_iter, double rel_tol, int flags);
/* The learned preconditioner's network for firm_batch_solve: params_bf16 (the BF16
 * weights of firm_mlp_to_bf16) and params (FP32, for the biases), device memory the
 * caller keeps alive; NULL, NULL removes it. */
int firm_batch_set_network(firm_batch_t batch, const void* params_bf16, const float* params);
/* Waits for the batch, then reports per plan the CG status (firm_status) and the
 * iterations run; also leaves each plan as after its own firm_kernel /
 * firm_backproject (lam_eff, Ker, K-hat and A*b readable).  Returns FIRM_OK when every
 * plan is OK, else the first failing status.  status, iters: n_plans entries or NULL. */
int firm_batch_wait(firm_batch_t batch, int* status, int* iters);
/* Tuning knobs: active worker streams (1..n_streams of create) and the points per
 * spreading work item of every plan (1024..8192, a multiple of 256).  firm_batch_tune
 * times the candidates on the given items (each candidate run twice, the second
 * timed with CUDA events) and keeps the fastest; ms_out (nullable) gets its time. */
int firm_batch_set_config(firm_batch_t batch, int n_streams, int chunk);
int firm_batch_get_config(firm_batch_t batch, int* n_streams, int* chunk);
int firm_batch_tune(firm_batch_t batch, const firm_batch_item* items, int iters, int flags, double* ms_out);
/* Kernels one run of the batch launches (graph or not), counted when queued. */
int firm_batch_launch_count(firm_batch_t batch, long long* out);
void firm_batch_destroy(firm_batch_t batch);

#ifdef __cplusplus
}
#endif
#endif /* FIRM_H */
