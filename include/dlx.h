/*
 * dlx.h - C ABI of the GB300 (sm_103a) differentiable-optics hot path.
 *
 * The library evaluates, on one GPU, the forward model and gradient of
 * arXiv:2406.08703 (Sec. 3-4):
 *
 *   OPD   = OPD_fixed + sum_j c_j Z_j + OPD_pix                   (Sec. 3, BasisOptic + mask)
 *   P     = T_hat exp(i 2 pi / lambda (OPD + x th_x + y th_y))       (Sec. 3, normalise=True)
 *   E     = A(lambda) P A(lambda)^T                                   (Sec. 3, two-sided MFT)
 *           A[k][n] = sqrt(dx du / lambda) exp(-2 pi i x_n u_k / lambda)
 *   I_e   = sum_s F_s sum_l w_l |E_{l,s,e}|^2    (w normalised to sum 1)
 *   m_e   = FF * (os x os block sums of I_e)                          (Sec. 3, pixel response)
 *   L     = sum_e sum_p (m - d ln m)                                  (Sec. 4, Poisson likelihood)
 *
 * and the gradient of L with respect to the Zernike coefficients, the pixel
 * OPD map, the flat field, the source fluxes and the source positions (the
 * parameter groups of Sec. 3-4).
 *
 * Grids are pixel-centred: x_n = (n - (N-1)/2) D/N_pupil, u_k = (k - (No-1)/2)
 * pixscale/oversample with No = n_det * oversample.  A source at +theta lands
 * at u = +theta.  Arrays are row-major [y][x], float32, contiguous, on the
 * plan's device unless stated otherwise.  Angles are radians.
 *
 * Ownership: the caller owns every array it passes and the CUDA stream; the
 * library owns plans (MFT matrices + workspaces) and servers.  Device-pointer
 * calls are asynchronous on the given stream (NULL = legacy default stream):
 * outputs are valid once the stream has completed.  Every call returns a
 * dlx_status; no exception crosses the ABI.  dlx_last_error() gives a
 * thread-local message for the last failing call on the calling thread.
 *
 * A plan holds one evaluation's workspaces: calls on the same plan must be
 * issued by one host thread at a time and on one stream (or with the caller
 * ordering the streams), since each call's work reuses them; different plans
 * are independent.  The server (dlx_server_*) is thread-safe.
 */
#ifndef DLX_H
#define DLX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    DLX_OK = 0,
    DLX_PENDING = 1,             /* dlx_poll: request not finished yet */
    DLX_ERR_INVALID_ARG = -1,    /* bad pointer, size, or enum value */
    DLX_ERR_NOMEM = -2,          /* device allocation or admission budget failed */
    DLX_ERR_CUDA = -3,           /* a CUDA runtime call failed (message has the CUDA error) */
    DLX_ERR_NONFINITE = -4,      /* loss or gradient is NaN/Inf (server path) */
    DLX_ERR_TIMEOUT = -5,        /* dlx_poll deadline, or a device-side bounded wait expired */
    DLX_ERR_RANGE = -6,          /* size beyond a supported maximum */
    DLX_ERR_UNSUPPORTED = -7     /* precision form not available for this shape or device */
} dlx_status;

/* Arithmetic form of the four MFT contractions (Sec. 3 "two-sided MFT").
 * All forms accumulate in FP32; phase arguments are reduced in FP64 and the
 * loss and gradient reductions are FP64. */
typedef enum {
    DLX_FP32_SIMT = 0, /* FP32 FMA on CUDA cores */
    DLX_TF32X3 = 1,    /* tcgen05 kind::tf32, operands split hi + lo, 3 products (forward
                          contractions accumulate hi*hi apart from the corrections) */
    DLX_BF16X3 = 2,    /* tcgen05 kind::f16 (BF16), operands split hi + lo, 3 products; the forward
                          operands are split by stochastic rounding (hash-seeded, reproducible)
                          so that the dropped lo*lo term and the rounding errors are zero-mean,
                          and stage 2 (stage 1 too above 256-long contractions) accumulates the
                          hi*hi products apart */
    DLX_BF16 = 3,      /* tcgen05 kind::f16 (BF16), hi only */
    DLX_BF16X4 = 4,    /* as BF16X3, plus the lo*lo product, and in the forward contractions the
                          hi*hi products accumulate apart from the correction products */
    DLX_F16X3 = 5,     /* tcgen05 kind::f16 (FP16), operands split hi + lo (22 significant bits),
                          3 products (forward contractions accumulate hi*hi apart); every
                          operand is stored times an exact power of two chosen from a bound on
                          its magnitude, so it stays inside FP16's exponent range */
    DLX_BF16X3SA = 6   /* forward as DLX_BF16X3; the adjoint contractions use the stochastically
                          rounded hi parts alone (one BF16 product per real product): each hi is
                          an unbiased estimate of its value, so the gradient carries zero-mean
                          noise of about 2^-8 / sqrt(K) of each contraction's terms instead of
                          the split's bias-free 2^-16; the PSF and loss are those of DLX_BF16X3 */
} dlx_prec;
/* The BF16 split forms (BF16X3, BF16X4, BF16X3SA) keep about 17 significant bits per operand,
 * whose representation error a contraction averages down over its terms only: below 32 pupil
 * samples per side their PSF misses 1e-5 of its peak, so plans of such pupils run DLX_F16X3
 * (22 bits) instead, and dlx_plan_info.precision reports the form that runs. */

typedef struct dlx_plan dlx_plan;
typedef struct dlx_server dlx_server;

/* Shape of one optical model (Sec. 3, Listing 1: AngularOpticalSystem(wf_npix,
 * diameter, layers, det_npix, det_pixsize) over a set of wavelengths). */
typedef struct {
    int n_pupil;             /* pupil samples per side, Ni >= 2 */
    double diameter_m;       /* aperture diameter D; pupil spacing dx = D / Ni */
    int n_det;               /* detector pixels per side, Nd >= 1 */
    double pixscale_rad;     /* detector pixel scale p; MFT spacing du = p / oversample */
    int oversample;          /* os >= 1; MFT output No = Nd * os */
    int n_lambda;            /* number of wavelengths, >= 1 */
    const double *lambda_m;  /* HOST array [n_lambda], metres; copied */
    int n_src;               /* point sources, 1 .. 32 */
    int n_exp;               /* exposures (known dithers), >= 1 */
    int n_zern;              /* Zernike basis terms, >= 0 */
    int precision;           /* dlx_prec */
    int psf_chunk;           /* PSFs per adjoint pass (per-wavelength recomputation batch;
                                all PSFs at once lets the BF16 split forms keep stage 2's fields);
                                0 = automatic from workspace_limit_bytes */
    size_t workspace_limit_bytes; /* 0 = no limit; bounds the adjoint workspace */
    double prf_prior_sigma;  /* > 0: the loss adds the chi^2 log prior on the pixel response
                                (Sec. 4) sum_p (FF_p - 1)^2 / (2 sigma^2), and dL/dFF its
                                gradient (FF_p - 1) / sigma^2; 0 = none */
    const int32_t *dither_px;/* NULL: the exposures' dithers are params->dither (any angle).
                                Else HOST [n_exp][2] integer-pixel dithers (x, y), copied, each
                                |dither| <= 4096: every source's PSF is computed once on a
                                (Nd + 2 max|dither_px|)^2 detector and image e is the Nd x Nd
                                window of it shifted by dither_px[e] (Sec. 3's integer dithers),
                                which equals the model with params->dither = dither_px * pixscale
                                (times f / z in the Fresnel regime below: the pointing offset that
                                moves the image by whole pixels) at 1/n_exp of the MFT work;
                                params->dither is then not read (nor a request's dither
                                in dlx_submit). */
    double focal_length_m;   /* 0: Fraunhofer regime (the detector at focus; the model is angular).
                                > 0: Fresnel regime (Sec. 1: a detector slightly out of focus adds
                                quadratic phase factors before and after the transform): a lens of
                                focal length f with the detector at z = f + focal_shift_m > 0;
                                pixscale_rad is then the detector pitch over f.  The pupil gets
                                exp(i pi |x|^2 (1/z - 1/f) / lambda) and the transform is taken at
                                the angles r / z of the detector positions r; the factor after the
                                transform, exp(i pi |r|^2 / (lambda z)), has modulus 1 and leaves
                                every intensity, so it is not applied. */
    double focal_shift_m;    /* z - f, metres; must be 0 when focal_length_m is 0 */
} dlx_mft_desc;

/* Parameters and fixed inputs of one evaluation.  Device pointers. */
typedef struct {
    const float *transmission; /* [Ni][Ni] aperture transmission T (>= 0) */
    const float *opd_fixed;    /* [Ni][Ni] fixed OPD (mask), metres; NULL = 0 */
    const float *zern_basis;   /* [n_zern][Ni][Ni] basis images; NULL iff n_zern == 0 */
    const float *zern_coeff;   /* [n_zern] coefficients, metres RMS; NULL iff n_zern == 0 */
    const float *opd_pix;      /* [Ni][Ni] free pixel OPD map, metres; NULL = not a parameter */
    const float *weights;      /* [n_lambda] spectral weights (normalised internally) */
    const float *flux;         /* [n_src] photons per source per exposure */
    const float *pos;          /* [n_src][2] (theta_x, theta_y), rad */
    const float *dither;       /* [n_exp][2] known offsets added to every source, rad; NULL = 0 */
    const float *flat;         /* [Nd][Nd] pixel response FF */
} dlx_params;

/* Gradient outputs (device, caller-owned).  Any pointer may be NULL to skip it. */
typedef struct {
    float *d_zern;    /* [n_zern]   dL/dc_j */
    float *d_opd_pix; /* [Ni][Ni]   dL/dOPD_pix */
    float *d_flat;    /* [Nd][Nd]   dL/dFF */
    float *d_flux;    /* [n_src]    dL/dF_s */
    float *d_pos;     /* [n_src][2] dL/dtheta */
} dlx_grads;

typedef struct {
    int n_pupil, n_det, oversample, n_out, n_lambda, n_src, n_exp, n_zern, n_psf;
    int precision;
    int psf_chunk;             /* PSFs per adjoint pass */
    size_t workspace_bytes;    /* device memory held by the plan */
    double flop_forward;       /* algorithmic MFT FLOP of one forward (8 per complex MAC) */
    double flop_loss_grad;     /* algorithmic MFT FLOP of one loss+gradient, with the field's
                                  recomputation where the plan does not keep stage 2's fields */
    int gemm_tiles_stage2;     /* output tiles of the dominant contraction */
    int n_mft_out;             /* the MFT's output grid per side: n_out, or (Nd + 2 max|dither_px|) * os */
} dlx_plan_info;

/* Build a plan: validates the shape, allocates the MFT matrices A(lambda) and
 * A(lambda)^H for every wavelength in the chosen operand form (phase arguments
 * x_n u_k / lambda reduced in FP64 before sin/cos) and the workspaces, on
 * `device`.  Synchronous.  Errors: INVALID_ARG (bad shape), UNSUPPORTED
 * (tensor-core form on a device that is not sm_103), NOMEM, CUDA. */
int dlx_make_mft(const dlx_mft_desc *desc, int device, dlx_plan **out);
int dlx_destroy_plan(dlx_plan *plan);
int dlx_plan_get_info(const dlx_plan *plan, dlx_plan_info *out);

/* Forward model (Sec. 3): model[e][py][px] = FF * bin_os(sum_s F_s sum_l w_l |E|^2).
 * `model` is device [n_exp][Nd][Nd]. */
int dlx_forward(dlx_plan *plan, const dlx_params *params, float *model, void *cuda_stream);

/* Directional derivative of the model (forward mode), for the Laplace
 * approximation of the parameter errors (Sec. 4): jvp = dm/dalpha at alpha = 0
 * for the phasors of the sources whose bit is set in `src_mask` (bit s = source
 * s, every exposure) multiplied by exp(i alpha (2 pi / lambda) t[n]), i.e. the
 * derivative along a change of optical path t (metres, device float [Ni][Ni]).
 * t = a Zernike basis map with every bit set gives dm/dc_j; t = the pupil x or y
 * coordinate (n - (Ni-1)/2) D/Ni for one source gives dm/dtheta_x or theta_y of
 * that source.  The model is a quadratic form of the phasor, so the central
 * difference (m(P (1 + i a)) - m(P (1 - i a))) / (2 alpha), a = alpha (2 pi /
 * lambda) t, is the derivative itself for any alpha > 0; alpha only sets the
 * size of the two models against their rounding (alpha max |a| near 1 is a good
 * choice).  `jvp` and `work` are device float [n_exp][Nd][Nd]; `work` is
 * overwritten.  Asynchronous on the stream; t_map must stay valid until the
 * work has run.  Errors: INVALID_ARG (NULL pointers, alpha not > 0), those of
 * dlx_forward. */
int dlx_model_jvp(dlx_plan *plan, const dlx_params *params, const float *t_map, uint32_t src_mask, double alpha,
                  float *jvp, float *work, void *cuda_stream);

/* Vector-Jacobian product (reverse mode): grads = J^T cot, the gradient of
 * sum_p cot[p] m[p] with respect to every parameter, where `cot` is a device
 * float [n_exp][Nd][Nd] weight on the model pixels.  With cot = 1 - d/m it is
 * the likelihood gradient of dlx_loss_grad without the prior term.  Arrays of
 * `grads` left NULL are not computed.  Asynchronous on the stream. */
int dlx_model_vjp(dlx_plan *plan, const dlx_params *params, const float *cot, const dlx_grads *grads,
                  void *cuda_stream);

/* Derivative of J^T cot along the phasor tangent of dlx_model_jvp, with cot
 * held fixed: grads[i] = sum_p cot[p] d^2 m[p] / (d theta_i d alpha).  This is
 * the term of the likelihood Hessian that the Fisher matrix J^T diag(d/m^2) J
 * leaves out (Laplace approximation, Sec. 4): with cot = 1 - d/m it gives, for a
 * tangent t = dOPD/dtheta_j, column j of sum_p (1 - d_p/m_p) d^2 m_p.  J^T cot
 * is a quadratic form of the phasor, so the central difference over 2 alpha is
 * exact, as in dlx_model_jvp.  `work` needs every array that `grads` has (same
 * sizes; overwritten).  Errors: INVALID_ARG, those of dlx_model_vjp. */
int dlx_model_vjp_jvp(dlx_plan *plan, const dlx_params *params, const float *cot, const float *t_map,
                      uint32_t src_mask, double alpha, const dlx_grads *grads, const dlx_grads *work,
                      void *cuda_stream);

/* The weights dL/dm of the Poisson negative log-likelihood sum (m - d ln m)
 * (Sec. 4): cot[i] = 1 - data[i] / max(model[i], 1e-30), all device arrays of
 * n elements (model float, data int32, cot float).  The cotangent that turns
 * dlx_model_vjp into the likelihood gradient and dlx_model_vjp_jvp into the
 * second-order part of its Hessian.  Asynchronous on the stream. */
int dlx_nll_cotangent(const float *model, const int32_t *data, size_t n, float *cot, void *cuda_stream);

/* Weighted Gram matrix of Jacobian rows, the information matrix of the Poisson
 * likelihood (Laplace approximation, Sec. 4):
 *   F[i][j] = sum_p J[i][p] J[j][p] w_p,
 *   w_p = 1 / max(m_p, 1e-30)               (data == NULL: expected Fisher information)
 *   w_p = d_p / max(m_p, 1e-30)^2           (observed Gauss-Newton term of the Hessian).
 * J: device float [n_par][n_pix] row-major; model: device float [n_pix];
 * data: device int32 [n_pix] or NULL; F: device double [n_par][n_par] (both
 * triangles written); work: device double scratch of at least
 * DLX_GRAM_BLOCKS * n_par (n_par + 1) / 2 elements.  Products are summed in
 * FP32 over 32-pixel chunks and in FP64 beyond; the result is the same on every
 * run.  Errors: INVALID_ARG (NULL, n_pix = 0), RANGE (n_par outside
 * 1..DLX_GRAM_MAX_PAR). */
#define DLX_GRAM_MAX_PAR 128
#define DLX_GRAM_BLOCKS 256
int dlx_fisher_gram(const float *J, int n_par, size_t n_pix, const float *model, const int32_t *data, double *F,
                    double *work, void *cuda_stream);

/* The paper has no counterpart of this entry point; it exists for callers that
 * cannot allocate device memory -- host applications that reserve all of the
 * GPU's memory through their own allocator at start-up and forbid further
 * allocation at run time (for example an instrument-control or real-time
 * reduction loop that must never stall or fail on an allocation).
 * It computes the same model as dlx_forward in the FP32 CUDA-core form
 * (desc->precision is ignored) without a plan and without calling cudaMalloc,
 * cudaFree or any allocating routine: all working memory comes from one
 * file-scope device array of 16 MiB that every GPU loading the library holds
 * until the process exits.  Arguments are dlx_forward's, with `desc` in place
 * of a plan (desc->lambda_m is host memory, read during the call).
 * Limits: dlx_make_mft's checks of the descriptor (INVALID_ARG, RANGE), at most
 * 32 sources and 256 wavelengths, no dither_px windows (UNSUPPORTED), and the
 * working memory of
 *   8*nl + 8*nl + 8*B*Ni + 4*Ni^2 + 8*nl*No*Ni8 + 8*nl*Ni*No8 + 8*B*Ni*Ni8
 *   + 8*B*No*Ni8 + 4*nS*nE*No^2 + reduction partials   (bytes, Ni8/No8 = sizes rounded up to 8,
 *   each of the 16 regions starting on a 256-byte boundary)
 * must fit in 16 MiB; larger shapes return DLX_ERR_RANGE with the byte count.
 * Under dlx_set_checks(1) the parameter arrays and `model` are checked as for
 * dlx_forward before anything runs.
 * When memory is taken: CUDA loads a library's device code and its device arrays
 * when they are first used (lazy loading, the default), so the first call on a
 * device loads the 16 MiB array and the kernels the call runs; a later call that
 * needs a kernel no earlier call ran (more than 8 sources, for one) loads that
 * kernel too.  Make the first calls, with the shapes the caller will use, before
 * reserving the device's memory, or have everything loaded when the context is
 * created by setting CUDA_MODULE_LOADING=EAGER in the environment.  Every call
 * looks up the array's device address (cudaGetSymbolAddress) on the calling
 * thread's current device, which must be the device of the arrays passed in.
 * Every call on a device
 * shares the array and overwrites it, so calls whose work overlaps on the GPU
 * (other streams or threads) race: serialise them.  Asynchronous on the stream
 * like dlx_forward. */
int dlx_forward_noalloc(const dlx_mft_desc *desc, const dlx_params *params, float *model, void *cuda_stream);

/* The flux-weighted oversampled intensity before binning and flat field,
 * psf_os[e][ky][kx] = sum_s F_s sum_l w_l |E_{l,s,e}|^2, device [n_exp][No][No]. */
int dlx_psf(dlx_plan *plan, const dlx_params *params, float *psf_os, void *cuda_stream);

/* Loss and gradient (Sec. 4): *loss (device, one double) = sum (m - d ln max(m, 1e-30)),
 * gradients into `grads`, and the model into `model_opt` ([n_exp][Nd][Nd], may be NULL).
 * `data` is device int32 [n_exp][Nd][Nd] photon counts.  When a pupil gradient is
 * wanted, the BF16 split forms (BF16x3, BF16x4) whose adjoint takes every PSF in one
 * pass (psf_chunk at least the PSF count, with the workspace to hold them) keep each
 * PSF's field from stage 2 and form the adjoint field from it; the other forms and
 * smaller psf_chunk recompute each PSF's field from the stored first-stage product,
 * psf_chunk PSFs at a time. */
int dlx_loss_grad(dlx_plan *plan, const dlx_params *params, const int32_t *data, double *loss,
                  const dlx_grads *grads, float *model_opt, void *cuda_stream);

/* Synchronous diagnostics of the last evaluation on this plan: pixels whose
 * model was clamped at 1e-30 before the log, and the device error flag (non-zero
 * when a device-side bounded wait expired; the flag is cleared by this call). */
int dlx_plan_diagnostics(dlx_plan *plan, int64_t *clamped, int32_t *device_error);

/* Checked mode, a stand-in for a device memory checker (the library checks its own
 * calls).  Level 1: before any launch, every device array an entry point reads or
 * writes must be device memory of the plan's device (or managed memory), aligned
 * for its element type (4 bytes; 8 for doubles) and, where the driver reports the
 * allocation holding it, lie inside that allocation for the full size the shapes
 * imply (a sub-allocation of a caching allocator is checked against its whole
 * block); a failure returns INVALID_ARG naming the argument and launches nothing.
 * Level 2 also synchronises the stream after each kernel class (not while the
 * stream is being captured) and returns CUDA, or TIMEOUT when a device-side
 * bounded wait expired, naming the class.  0 (the default) checks nothing.  The
 * level is process-wide; the environment variable DLX_CHECKS sets it when the
 * library is first used.  Errors: INVALID_ARG (level outside 0..2). */
int dlx_set_checks(int level);
int dlx_get_checks(void);
/* Level 1's test of one array: device memory of `device`, 4-byte aligned, and
 * `bytes` inside its allocation.  Launches nothing. */
int dlx_check_buffer(const void *ptr, size_t bytes, int device);
/* The level-1 checks of a dlx_loss_grad call with these arguments, whatever the
 * level; launches nothing. */
int dlx_check_loss_grad_args(dlx_plan *plan, const dlx_params *params, const int32_t *data, const double *loss,
                             const dlx_grads *grads, const float *model_opt);

/* Test hook for the device-side bounded waits (no fault, no hang): kind 1 makes
 * CTA 0 of the plan's next tensor-core contraction withhold its first operand
 * copy, so the wait for it expires after 1 s; the CTA stops its work, frees its
 * tensor memory and returns, the device error flag is raised
 * (dlx_plan_diagnostics), and that call's results are undefined.  The plan and
 * the context stay usable.  Errors: INVALID_ARG (other kinds, the FP32 form,
 * which has no such waits). */
int dlx_plan_inject_fault(dlx_plan *plan, int kind);

/* Per-kernel-class device time of the evaluations issued on this plan while
 * timing is enabled: CUDA events are recorded on the launching stream around
 * each timed class of launch (so the times include no host gaps), and every
 * kernel launch is counted whether timing is on or not.  `class_mask` selects
 * the timed classes: bit c times class c (the order of dlx_kernel_times.name),
 * -1 times all of them and 0 turns timing off; each timed launch group costs
 * two event records on the stream, so timing one class disturbs an evaluation
 * far less than timing all.  dlx_plan_get_timing is synchronous and resets the
 * accumulators and counters. */
typedef struct {
    int n_classes;
    const char *name[16];   /* e.g. "stage2_intensity", "adjoint_field" */
    double ms[16];          /* total device milliseconds (0 when timing was off) */
    int64_t events[16];     /* timed scopes (one per launch or launch group) */
    int64_t launches[16];   /* kernel launches */
    int64_t total_launches;
} dlx_kernel_times;
int dlx_plan_set_timing(dlx_plan *plan, int class_mask);
int dlx_plan_get_timing(dlx_plan *plan, dlx_kernel_times *out);

/* Adam update (Kingma & Ba; the optimiser of Sec. 4) of n parameters in place:
 * m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2; theta -= lr mhat / (sqrt(vhat) + eps),
 * with bias correction for 1-based step `t`.  All arrays device float32. */
int dlx_adam(float *theta, const float *grad, float *m, float *v, size_t n, float lr, float beta1, float beta2,
             float eps, int t, void *cuda_stream);

/* ---------------------------------------------------------------- serving */

/* One fit request: the model shape, host copies of the fixed inputs, a starting
 * point, the data, and K Adam steps (K = 0: one loss+gradient evaluation). */
typedef struct {
    dlx_mft_desc desc;          /* desc.precision selects the form; lambda_m is host */
    const float *transmission;  /* host [Ni][Ni] */
    const float *opd_fixed;     /* host [Ni][Ni] or NULL */
    const float *zern_basis;    /* host [n_zern][Ni][Ni] or NULL iff n_zern == 0 */
    const float *weights;       /* host [n_lambda] */
    const float *dither;        /* host [n_exp][2] or NULL */
    const float *zern_coeff;    /* host [n_zern] start */
    const float *opd_pix;       /* host [Ni][Ni] start, or NULL (not fitted) */
    const float *flux;          /* host [n_src] start */
    const float *pos;           /* host [n_src][2] start */
    const float *flat;          /* host [Nd][Nd] start */
    const int32_t *data;        /* host [n_exp][Nd][Nd] */
    int n_steps;                /* K Adam steps */
    float lr[5];                /* learning rates: zern, opd_pix, flat, flux, pos (0 freezes a group) */
    /* Optional resume state; NULL / 0 start a fresh fit.  The Adam moments are in
     * the packed parameter order [zern_coeff | opd_pix (only when fitted) | flat |
     * flux | pos], n_state = n_zern + (opd_pix ? Ni*Ni : 0) + Nd*Nd + 3 n_src
     * floats each (NULL = zeros); adam_step >= 0 is the number of Adam steps
     * already taken, which sets the bias correction of the next one.  Fed the
     * parameters, moments and step count of a dlx_result, a request continues
     * that fit bit for bit: K1 steps and then K2 more equal K1 + K2 in one. */
    const float *adam_m;        /* host [n_state] or NULL */
    const float *adam_v;        /* host [n_state] or NULL */
    int adam_step;
} dlx_request;

/* Result of a finished request, copied into caller-owned HOST buffers (any may be NULL). */
typedef struct {
    double loss;                /* loss at the final parameters' last evaluation */
    float *zern_coeff, *opd_pix, *flux, *pos, *flat;          /* final parameters */
    float *g_zern, *g_opd_pix, *g_flux, *g_pos, *g_flat;      /* gradient of the last evaluation */
    double queued_s, latency_s; /* submit -> admit, submit -> done */
    int steps_done;
    float *adam_m, *adam_v;     /* Adam moments after the last step, packed as in dlx_request, or NULL */
    int adam_step;              /* the request's adam_step + K: feed back to continue the fit */
} dlx_result;

typedef struct {
    uint64_t submitted, admitted, completed, rejected;
    int active, queued;
    size_t hbm_in_use, hbm_budget;
    uint64_t evals, graph_launches, grouped_launches;
    /* admissions into a bucket where another request had already taken steps (a slot
     * refilled mid-flight), and finished slots refilled by moving the bucket's last
     * active slot down into them */
    uint64_t midflight_admits, slot_moves;
} dlx_server_stats;

/* Create a continuous-batching fit server on `device` with its own stream and
 * scheduler thread.  `hbm_budget` bounds the device memory of admitted
 * requests (0 = 90% of free memory); `max_slots` bounds concurrent fits. */
int dlx_server_create(int device, size_t hbm_budget, int max_slots, dlx_server **out);
int dlx_server_destroy(dlx_server *server);

/* Non-blocking: copies the request's host inputs and queues it.  Returns
 * NOMEM if the request alone exceeds the budget, INVALID_ARG on a bad shape. */
int dlx_submit(dlx_server *server, const dlx_request *request, uint64_t *ticket);

/* Wait up to timeout_s (0 = just test) for a ticket.  Returns OK and fills
 * `out` once, PENDING while running, TIMEOUT if the deadline passed, or the
 * request's error status (NONFINITE, NOMEM, CUDA...).  A finished ticket is
 * released after a successful poll. */
int dlx_poll(dlx_server *server, uint64_t ticket, double timeout_s, dlx_result *out);
int dlx_server_get_stats(dlx_server *server, dlx_server_stats *out);

/* Host-side fault injection for tests: 1 = fail the next admission with NOMEM,
 * 2 = poison the next admitted request's first gradient with NaN. */
int dlx_server_inject_fault(dlx_server *server, int kind);

const char *dlx_last_error(void);
const char *dlx_version(void);

#ifdef __cplusplus
}
#endif
#endif /* DLX_H */
