/*
 * FP64 CPU oracle for the differentiable-optics forward model, Poisson
 * likelihood and gradient of arXiv:2406.08703 (Sec. 3 and Sec. 4).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plainly written
 * definition that the CUDA path is checked against.  It may be built, loaded
 * and called only by the tests, by the package smoke check and by the CPU
 * baseline leg of the benchmark.  It shares no code, header, table or helper
 * with the CUDA library, and the library never calls it.
 *
 * What it computes, in the paper's order:
 *   OPD   = OPD_fixed + sum_j c_j Z_j + OPD_pix           (BasisOptic + mask, Sec. 3)
 *   P     = T_hat exp(i 2 pi/lambda (OPD + x th_x + y th_y)),
 *           T_hat = T / sqrt(sum T^2)                        (normalise=True, Sec. 3)
 *   E     = A_y P A_x^T,  A[k][n] = sqrt(dx du/lambda) exp(-2 pi i x_n u_k/lambda)
 *                                                            (two-sided MFT, Sec. 3)
 *   I_e   = sum_s F_s sum_l w_l |E_{l,s,e}|^2, w normalised to sum 1
 *   B_e   = os x os block sums of I_e;  m = FF * B_e         (pixel response, Sec. 3)
 *   L     = sum_e sum_p (m - d ln m)                         (Poisson likelihood, Sec. 4)
 *           + sum_p (FF_p - 1)^2 / (2 sigma^2)                 (chi^2 log prior on the pixel
 *                                                              response, Sec. 4; sigma = 0: none)
 * In the Fresnel regime (Sec. 1: a detector slightly out of focus adds
 * quadratic phase factors before and after the transform), with a lens of
 * focal length f and the detector at z = f + dz, the field at detector
 * position r (pitch pixscale * f) is
 *   E(r) = exp(i pi |r|^2 / (lambda z)) * MFT[ exp(i pi |x|^2 (1/z - 1/f) / lambda) P ](r / z),
 * the transform taken at angles r / z, i.e. with du = (pixscale / os) f / z;
 * focal_length = 0 is the Fraunhofer model above.
 * and the analytic adjoint of L with respect to the Zernike coefficients, the
 * pixel OPD map, the flat field, the source fluxes and the source positions
 * (Sec. 4 takes gradients of this loss with respect to exactly these groups).
 *
 * Conventions (readings of the paper where it is silent):
 *   - grids are pixel-centred: x_n = (n - (N-1)/2) dx with dx = D/N_pupil,
 *     u_k = (k - (N_out-1)/2) du with du = pixscale/oversample;
 *   - the MFT normalisation sqrt(dx du / lambda) per axis conserves energy;
 *   - a source at +theta adds the pupil phase +2 pi x theta / lambda, so its
 *     image lands at u = +theta;
 *   - binning sums the os x os block; ln m is taken of max(m, 1e-30).
 * Every function below is pinned by a CPU test against closed forms,
 * library routines or brute force (Airy pattern, zero-padded FFT, Parseval,
 * shift theorem, centrosymmetry, twin image, Euler identities, central finite
 * differences, the adjoint dot-product identity).
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

/* Threads of the OpenMP loops below (n < 1: one per processor); returns the number the next
 * parallel loop will use.  Timing control for the benchmark's CPU baseline, no arithmetic. */
int orc_set_threads(int n) {
#ifdef _OPENMP
    omp_set_num_threads(n > 0 ? n : omp_get_num_procs());
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

typedef struct {
    int n_pupil;
    double diameter;
    int n_det;
    double pixscale;
    int oversample;
    int n_lambda;
    const double *lambdas;
    const double *weights;
    int n_src;
    const double *flux; /* photons per source per exposure */
    const double *pos;  /* [n_src][2] = (theta_x, theta_y) rad */
    int n_exp;
    const double *dither; /* [n_exp][2] rad, added to every source position */
    int n_zern;
    const double *basis; /* [n_zern][n][n] */
    const double *coeff; /* [n_zern] */
    const double *transmission; /* [n][n] */
    const double *opd_fixed;    /* [n][n] */
    const double *opd_pix;      /* [n][n] or NULL */
    const double *flat;         /* [n_det][n_det] */
    double prf_sigma;           /* s.d. of the chi^2 prior on the flat field about 1; 0 = no prior */
    double focal_length;        /* f > 0: Fresnel regime with the detector at f + focal_shift; 0: Fraunhofer */
    double focal_shift;
} orc_problem;

static const double TWO_PI = 6.283185307179586476925286766559;

/* Pixel-centred coordinate i of an n-point grid with the given spacing. */
static double coord(int i, int n, double spacing) { return ((double)i - 0.5 * (double)(n - 1)) * spacing; }

void orc_coords(int n, double spacing, double *out) {
    for (int i = 0; i < n; ++i) out[i] = coord(i, n, spacing);
}

/* Angle step of the transform's output samples: pixscale / os, times f / z in the Fresnel regime. */
static double mft_du(const orc_problem *q) {
    double du = q->pixscale / q->oversample;
    if (q->focal_length > 0) du *= q->focal_length / (q->focal_length + q->focal_shift);
    return du;
}

/* Fresnel factor before the transform: P *= exp(sgn i pi |x|^2 (1/z - 1/f) / lambda). */
static void fresnel_pre(const orc_problem *q, double lam, int sgn, cplx *P) {
    if (!(q->focal_length > 0)) return;
    int n = q->n_pupil;
    double dx = q->diameter / n, f = q->focal_length, z = f + q->focal_shift;
    for (int ny = 0; ny < n; ++ny)
        for (int nx = 0; nx < n; ++nx) {
            double x = coord(nx, n, dx), y = coord(ny, n, dx);
            double ph = sgn * (0.5 * TWO_PI) * (x * x + y * y) * (1.0 / z - 1.0 / f) / lam;
            P[(size_t)ny * n + nx] *= cos(ph) + I * sin(ph);
        }
}

/* Fresnel factor after the transform: E *= exp(sgn i pi |r|^2 / (lambda z)), r the detector
 * position of each output sample (pitch pixscale * f / os). */
static void fresnel_post(const orc_problem *q, double lam, int sgn, cplx *E) {
    if (!(q->focal_length > 0)) return;
    int no = q->n_det * q->oversample;
    double f = q->focal_length, z = f + q->focal_shift, dr = q->pixscale * f / q->oversample;
    for (int ky = 0; ky < no; ++ky)
        for (int kx = 0; kx < no; ++kx) {
            double rx = coord(kx, no, dr), ry = coord(ky, no, dr);
            double ph = sgn * (0.5 * TWO_PI) * (rx * rx + ry * ry) / (lam * z);
            E[(size_t)ky * no + kx] *= cos(ph) + I * sin(ph);
        }
}

/* Two-sided MFT matrix (Sec. 3, Soummer et al. 2007):
 * A[k][n] = sqrt(dx du / lambda) exp(-2 pi i x_n u_k / lambda), n_out x n_in. */
void orc_mft_matrix(int n_out, int n_in, double dx, double du, double lam, cplx *A) {
    double s = sqrt(dx * du / lam);
    for (int k = 0; k < n_out; ++k) {
        double u = coord(k, n_out, du);
        for (int n = 0; n < n_in; ++n) {
            double x = coord(n, n_in, dx);
            double ph = -TWO_PI * x * u / lam;
            A[(size_t)k * n_in + n] = s * (cos(ph) + I * sin(ph));
        }
    }
}

/* E = A P A^T with the matrix of orc_mft_matrix, evaluated as two direct
 * sums: T[ny][kx] = sum_nx P[ny][nx] A[kx][nx], then E[ky][kx] = sum_ny A[ky][ny] T[ny][kx]. */
static void mft_with(const cplx *A, int n_in, int n_out, const cplx *P, cplx *E) {
    cplx *T = (cplx *)calloc((size_t)n_in * n_out, sizeof(cplx));
#pragma omp parallel for schedule(static)
    for (int ny = 0; ny < n_in; ++ny)
        for (int kx = 0; kx < n_out; ++kx) {
            cplx acc = 0;
            const cplx *p = P + (size_t)ny * n_in, *a = A + (size_t)kx * n_in;
            for (int nx = 0; nx < n_in; ++nx) acc += p[nx] * a[nx];
            T[(size_t)ny * n_out + kx] = acc;
        }
#pragma omp parallel for schedule(static)
    for (int ky = 0; ky < n_out; ++ky) {
        cplx *e = E + (size_t)ky * n_out;
        for (int kx = 0; kx < n_out; ++kx) e[kx] = 0;
        for (int ny = 0; ny < n_in; ++ny) {
            cplx a = A[(size_t)ky * n_in + ny];
            const cplx *t = T + (size_t)ny * n_out;
            for (int kx = 0; kx < n_out; ++kx) e[kx] += a * t[kx];
        }
    }
    free(T);
}

/* Adjoint of P -> A P A^T: out = A^H G conj(A), i.e.
 * out[ny][nx] = sum_ky conj(A[ky][ny]) sum_kx G[ky][kx] conj(A[kx][nx]). */
static void mft_adjoint_with(const cplx *A, int n_in, int n_out, const cplx *G, cplx *out) {
    cplx *U = (cplx *)calloc((size_t)n_out * n_in, sizeof(cplx));
#pragma omp parallel for schedule(static)
    for (int ky = 0; ky < n_out; ++ky) {
        cplx *u = U + (size_t)ky * n_in;
        for (int kx = 0; kx < n_out; ++kx) {
            cplx g = G[(size_t)ky * n_out + kx];
            const cplx *a = A + (size_t)kx * n_in;
            for (int nx = 0; nx < n_in; ++nx) u[nx] += g * conj(a[nx]);
        }
    }
#pragma omp parallel for schedule(static)
    for (int ny = 0; ny < n_in; ++ny) {
        cplx *o = out + (size_t)ny * n_in;
        for (int nx = 0; nx < n_in; ++nx) o[nx] = 0;
        for (int ky = 0; ky < n_out; ++ky) {
            cplx a = conj(A[(size_t)ky * n_in + ny]);
            const cplx *u = U + (size_t)ky * n_in;
            for (int nx = 0; nx < n_in; ++nx) o[nx] += a * u[nx];
        }
    }
    free(U);
}

/* Fraunhofer propagation of a pupil field to the angular detector grid by the
 * two-sided MFT (Sec. 3).  P is n_in x n_in, E is n_out x n_out. */
void orc_mft(int n_in, double dx, int n_out, double du, double lam, const cplx *P, cplx *E) {
    cplx *A = (cplx *)malloc((size_t)n_out * n_in * sizeof(cplx));
    orc_mft_matrix(n_out, n_in, dx, du, lam, A);
    mft_with(A, n_in, n_out, P, E);
    free(A);
}

/* The same transform as one four-fold sum straight from the exponent, for tiny sizes. */
void orc_mft_direct(int n_in, double dx, int n_out, double du, double lam, const cplx *P, cplx *E) {
    double s2 = dx * du / lam;
    for (int ky = 0; ky < n_out; ++ky)
        for (int kx = 0; kx < n_out; ++kx) {
            double u = coord(kx, n_out, du), v = coord(ky, n_out, du);
            cplx acc = 0;
            for (int ny = 0; ny < n_in; ++ny)
                for (int nx = 0; nx < n_in; ++nx) {
                    double x = coord(nx, n_in, dx), y = coord(ny, n_in, dx);
                    double ph = -TWO_PI * (x * u + y * v) / lam;
                    acc += P[(size_t)ny * n_in + nx] * (cos(ph) + I * sin(ph));
                }
            E[(size_t)ky * n_out + kx] = s2 * acc;
        }
}

void orc_mft_adjoint(int n_in, double dx, int n_out, double du, double lam, const cplx *G, cplx *out) {
    cplx *A = (cplx *)malloc((size_t)n_out * n_in * sizeof(cplx));
    orc_mft_matrix(n_out, n_in, dx, du, lam, A);
    mft_adjoint_with(A, n_in, n_out, G, out);
    free(A);
}

/* OPD = OPD_fixed + sum_j c_j Z_j + OPD_pix (BasisOptic and mask layers, Sec. 3). */
void orc_opd(const orc_problem *q, double *opd) {
    size_t npx = (size_t)q->n_pupil * q->n_pupil;
    for (size_t i = 0; i < npx; ++i) {
        double v = q->opd_fixed[i];
        for (int j = 0; j < q->n_zern; ++j) v += q->coeff[j] * q->basis[(size_t)j * npx + i];
        if (q->opd_pix) v += q->opd_pix[i];
        opd[i] = v;
    }
}

/* Pupil normalisation of BasisOptic(normalise=True): T_hat = T / sqrt(sum T^2). */
static double pupil_scale(const orc_problem *q) {
    size_t npx = (size_t)q->n_pupil * q->n_pupil;
    double s = 0;
    for (size_t i = 0; i < npx; ++i) s += q->transmission[i] * q->transmission[i];
    return 1.0 / sqrt(s);
}

/* Source position of (source s, exposure e): theta_s + dither_e. */
static void source_angle(const orc_problem *q, int s, int e, double *tx, double *ty) {
    *tx = q->pos[2 * s] + q->dither[2 * e];
    *ty = q->pos[2 * s + 1] + q->dither[2 * e + 1];
}

/* Pupil phasor of wavelength l, source s, exposure e:
 * P = T_hat exp(i 2 pi / lambda (OPD + x theta_x + y theta_y)). */
void orc_phasor(const orc_problem *q, const double *opd, int l, int s, int e, cplx *P) {
    int n = q->n_pupil;
    double dx = q->diameter / n, lam = q->lambdas[l], tx, ty, sc = pupil_scale(q);
    source_angle(q, s, e, &tx, &ty);
    for (int ny = 0; ny < n; ++ny)
        for (int nx = 0; nx < n; ++nx) {
            size_t i = (size_t)ny * n + nx;
            double path = opd[i] + coord(nx, n, dx) * tx + coord(ny, n, dx) * ty;
            double ph = TWO_PI * path / lam;
            P[i] = sc * q->transmission[i] * (cos(ph) + I * sin(ph));
        }
}

static double weight_norm(const orc_problem *q) {
    double s = 0;
    for (int l = 0; l < q->n_lambda; ++l) s += q->weights[l];
    return s;
}

/* Complex field E of one PSF (wavelength l, source s, exposure e), unit flux. */
void orc_psf_field(const orc_problem *q, int l, int s, int e, cplx *E) {
    int n = q->n_pupil, no = q->n_det * q->oversample;
    double *opd = (double *)malloc((size_t)n * n * sizeof(double));
    cplx *P = (cplx *)malloc((size_t)n * n * sizeof(cplx));
    orc_opd(q, opd);
    orc_phasor(q, opd, l, s, e, P);
    fresnel_pre(q, q->lambdas[l], 1, P);
    orc_mft(n, q->diameter / n, no, mft_du(q), q->lambdas[l], P, E);
    fresnel_post(q, q->lambdas[l], 1, E);
    free(opd);
    free(P);
}

/* Per-source polychromatic intensity at unit flux on the oversampled grid:
 * I_src[e][s][k] = sum_l w_l |E_{l,s,e}[k]|^2 with sum_l w_l = 1.
 * mats[l] (optional) are the MFT matrices per wavelength. */
static void intensity_src(const orc_problem *q, cplx **mats, double *I_src) {
    int n = q->n_pupil, no = q->n_det * q->oversample;
    size_t nq = (size_t)no * no, npx = (size_t)n * n;
    double wn = weight_norm(q);
    double *opd = (double *)malloc(npx * sizeof(double));
    cplx *P = (cplx *)malloc(npx * sizeof(cplx));
    cplx *E = (cplx *)malloc(nq * sizeof(cplx));
    orc_opd(q, opd);
    memset(I_src, 0, (size_t)q->n_exp * q->n_src * nq * sizeof(double));
    for (int e = 0; e < q->n_exp; ++e)
        for (int s = 0; s < q->n_src; ++s) {
            double *Ie = I_src + ((size_t)e * q->n_src + s) * nq;
            for (int l = 0; l < q->n_lambda; ++l) {
                orc_phasor(q, opd, l, s, e, P);
                fresnel_pre(q, q->lambdas[l], 1, P);
                mft_with(mats[l], n, no, P, E);
                fresnel_post(q, q->lambdas[l], 1, E);
                double w = q->weights[l] / wn;
                for (size_t k = 0; k < nq; ++k) Ie[k] += w * (creal(E[k]) * creal(E[k]) + cimag(E[k]) * cimag(E[k]));
            }
        }
    free(opd);
    free(P);
    free(E);
}

static cplx **make_mats(const orc_problem *q) {
    int n = q->n_pupil, no = q->n_det * q->oversample;
    cplx **mats = (cplx **)malloc((size_t)q->n_lambda * sizeof(cplx *));
    for (int l = 0; l < q->n_lambda; ++l) {
        mats[l] = (cplx *)malloc((size_t)no * n * sizeof(cplx));
        orc_mft_matrix(no, n, q->diameter / n, mft_du(q), q->lambdas[l], mats[l]);
    }
    return mats;
}

static void free_mats(const orc_problem *q, cplx **mats) {
    for (int l = 0; l < q->n_lambda; ++l) free(mats[l]);
    free(mats);
}

/* Bin the oversampled image by summing os x os blocks, then apply the pixel response. */
static void bin_flat(const orc_problem *q, const double *I_src, double *B_src, double *model) {
    int nd = q->n_det, os = q->oversample, no = nd * os;
    size_t nq = (size_t)no * no, np = (size_t)nd * nd;
    for (int e = 0; e < q->n_exp; ++e) {
        for (int s = 0; s < q->n_src; ++s) {
            const double *Ie = I_src + ((size_t)e * q->n_src + s) * nq;
            double *Be = B_src + ((size_t)e * q->n_src + s) * np;
            for (int py = 0; py < nd; ++py)
                for (int px = 0; px < nd; ++px) {
                    double acc = 0;
                    for (int a = 0; a < os; ++a)
                        for (int b = 0; b < os; ++b) acc += Ie[(size_t)(py * os + a) * no + (px * os + b)];
                    Be[(size_t)py * nd + px] = acc;
                }
        }
        for (size_t p = 0; p < np; ++p) {
            double b = 0;
            for (int s = 0; s < q->n_src; ++s) b += q->flux[s] * B_src[((size_t)e * q->n_src + s) * np + p];
            model[(size_t)e * np + p] = q->flat[p] * b;
        }
    }
}

/* Forward model: model[e][py][px] = FF * binned sum_s F_s I_src; psf_os (optional)
 * receives the flux-weighted oversampled intensity [e][ky][kx] before binning. */
void orc_forward(const orc_problem *q, double *model, double *psf_os) {
    int no = q->n_det * q->oversample;
    size_t nq = (size_t)no * no, np = (size_t)q->n_det * q->n_det;
    cplx **mats = make_mats(q);
    double *I_src = (double *)malloc((size_t)q->n_exp * q->n_src * nq * sizeof(double));
    double *B_src = (double *)malloc((size_t)q->n_exp * q->n_src * np * sizeof(double));
    intensity_src(q, mats, I_src);
    bin_flat(q, I_src, B_src, model);
    if (psf_os)
        for (int e = 0; e < q->n_exp; ++e)
            for (size_t k = 0; k < nq; ++k) {
                double v = 0;
                for (int s = 0; s < q->n_src; ++s) v += q->flux[s] * I_src[((size_t)e * q->n_src + s) * nq + k];
                psf_os[(size_t)e * nq + k] = v;
            }
    free(I_src);
    free(B_src);
    free_mats(q, mats);
}

/* Poisson negative log-likelihood (Sec. 4), dropping ln d!:
 * L = sum (m - d ln max(m, 1e-30)); returns the number of clamped pixels. */
static long poisson_nll(size_t n, const double *model, const int *data, double *loss, double *g_m) {
    long clamped = 0;
    double acc = 0;
    for (size_t i = 0; i < n; ++i) {
        double m = model[i], mc = m;
        if (mc < 1e-30) {
            mc = 1e-30;
            ++clamped;
        }
        acc += m - (double)data[i] * log(mc);
        if (g_m) g_m[i] = 1.0 - (double)data[i] / mc;
    }
    *loss = acc;
    return clamped;
}

/* chi^2 log prior on the pixel response (Sec. 4: mean 1, s.d. sigma):
 * sum_p (FF_p - 1)^2 / (2 sigma^2); adds its gradient (FF_p - 1) / sigma^2 to
 * g_flat when g_flat is not NULL.  Zero when sigma = 0. */
static double prf_prior(const orc_problem *q, double *g_flat) {
    if (!(q->prf_sigma > 0)) return 0.0;
    size_t np = (size_t)q->n_det * q->n_det;
    double acc = 0, s2 = q->prf_sigma * q->prf_sigma;
    for (size_t p = 0; p < np; ++p) {
        double dev = q->flat[p] - 1.0;
        acc += dev * dev / (2.0 * s2);
        if (g_flat) g_flat[p] += dev / s2;
    }
    return acc;
}

/* Loss only (used by the finite-difference pins). */
double orc_loss(const orc_problem *q, const int *data) {
    size_t np = (size_t)q->n_det * q->n_det * q->n_exp;
    double *model = (double *)malloc(np * sizeof(double)), L;
    orc_forward(q, model, NULL);
    poisson_nll(np, model, data, &L, NULL);
    free(model);
    return L + prf_prior(q, NULL);
}

/* Loss and its gradient by the analytic adjoint (reverse-mode chain rule of Sec. 4's loss).
 *   g_m      = dL/dm = 1 - d/m
 *   dL/dFF_p = sum_e g_m B_e[p]
 *   dL/dF_s  = sum_e sum_p FF_p g_m[e][p] B_{e,s}[p]
 *   G_E      = 2 w_l F_s FF[bin q] g_m[e][bin q] E_{l,s,e}[q]       (dL/dRe E + i dL/dIm E)
 *   G_P      = A^H G_E conj(A)                                       (adjoint MFT)
 *   g_phi    = Im(G_P conj(P))                                       (dL/dphase)
 *   g_OPD    = sum_{l,s,e} (2 pi/lambda_l) g_phi
 *   dL/dc_j  = <Z_j, g_OPD>,  dL/dOPD_pix = g_OPD
 *   dL/dtheta_x[s] = sum_{l,e,n} (2 pi/lambda_l) g_phi[n] x_n  (and y likewise)
 * Any gradient pointer may be NULL.  Returns the number of clamped model pixels. */
long orc_loss_grad(const orc_problem *q, const int *data, double *loss, double *model_out, double *g_coeff,
                   double *g_opd_pix, double *g_flat, double *g_flux, double *g_pos) {
    int n = q->n_pupil, nd = q->n_det, os = q->oversample, no = nd * os;
    size_t npx = (size_t)n * n, nq = (size_t)no * no, np = (size_t)nd * nd;
    double dx = q->diameter / n, wn = weight_norm(q);
    cplx **mats = make_mats(q);
    double *I_src = (double *)malloc((size_t)q->n_exp * q->n_src * nq * sizeof(double));
    double *B_src = (double *)malloc((size_t)q->n_exp * q->n_src * np * sizeof(double));
    double *model = (double *)malloc((size_t)q->n_exp * np * sizeof(double));
    double *g_m = (double *)malloc((size_t)q->n_exp * np * sizeof(double));
    intensity_src(q, mats, I_src);
    bin_flat(q, I_src, B_src, model);
    long clamped = poisson_nll((size_t)q->n_exp * np, model, data, loss, g_m);
    if (model_out) memcpy(model_out, model, (size_t)q->n_exp * np * sizeof(double));

    if (g_flat)
        for (size_t p = 0; p < np; ++p) {
            double acc = 0;
            for (int e = 0; e < q->n_exp; ++e) {
                double b = 0;
                for (int s = 0; s < q->n_src; ++s) b += q->flux[s] * B_src[((size_t)e * q->n_src + s) * np + p];
                acc += g_m[(size_t)e * np + p] * b;
            }
            g_flat[p] = acc;
        }
    *loss += prf_prior(q, g_flat);
    if (g_flux)
        for (int s = 0; s < q->n_src; ++s) {
            double acc = 0;
            for (int e = 0; e < q->n_exp; ++e)
                for (size_t p = 0; p < np; ++p)
                    acc += q->flat[p] * g_m[(size_t)e * np + p] * B_src[((size_t)e * q->n_src + s) * np + p];
            g_flux[s] = acc;
        }

    double *g_opd = (double *)calloc(npx, sizeof(double));
    double *opd = (double *)malloc(npx * sizeof(double));
    cplx *P = (cplx *)malloc(npx * sizeof(cplx));
    cplx *E = (cplx *)malloc(nq * sizeof(cplx));
    cplx *GP = (cplx *)malloc(npx * sizeof(cplx));
    cplx *PF = (cplx *)malloc(npx * sizeof(cplx));
    orc_opd(q, opd);
    if (g_pos) memset(g_pos, 0, (size_t)2 * q->n_src * sizeof(double));
    for (int e = 0; e < q->n_exp; ++e)
        for (int s = 0; s < q->n_src; ++s)
            for (int l = 0; l < q->n_lambda; ++l) {
                double lam = q->lambdas[l], c = 2.0 * (q->weights[l] / wn) * q->flux[s];
                orc_phasor(q, opd, l, s, e, P);
                memcpy(PF, P, npx * sizeof(cplx));
                fresnel_pre(q, lam, 1, PF);
                mft_with(mats[l], n, no, PF, E);
                fresnel_post(q, lam, 1, E);
                for (int ky = 0; ky < no; ++ky)
                    for (int kx = 0; kx < no; ++kx) {
                        size_t p = (size_t)(ky / os) * nd + (kx / os);
                        E[(size_t)ky * no + kx] *= c * q->flat[p] * g_m[(size_t)e * np + p];
                    }
                /* adjoints of the three linear steps, in reverse order */
                fresnel_post(q, lam, -1, E);
                mft_adjoint_with(mats[l], n, no, E, GP);
                fresnel_pre(q, lam, -1, GP);
                double k = TWO_PI / lam, sx = 0, sy = 0;
                for (int ny = 0; ny < n; ++ny)
                    for (int nx = 0; nx < n; ++nx) {
                        size_t i = (size_t)ny * n + nx;
                        double gphi = cimag(GP[i] * conj(P[i]));
                        g_opd[i] += k * gphi;
                        sx += k * gphi * coord(nx, n, dx);
                        sy += k * gphi * coord(ny, n, dx);
                    }
                if (g_pos) {
                    g_pos[2 * s] += sx;
                    g_pos[2 * s + 1] += sy;
                }
            }
    if (g_opd_pix) memcpy(g_opd_pix, g_opd, npx * sizeof(double));
    if (g_coeff)
        for (int j = 0; j < q->n_zern; ++j) {
            double acc = 0;
            for (size_t i = 0; i < npx; ++i) acc += q->basis[(size_t)j * npx + i] * g_opd[i];
            g_coeff[j] = acc;
        }
    free(g_opd);
    free(opd);
    free(P);
    free(E);
    free(GP);
    free(PF);
    free(I_src);
    free(B_src);
    free(model);
    free(g_m);
    free_mats(q, mats);
    return clamped;
}

/* The model at selected detector pixels only, for sizes where the full image
 * is out of reach: for exposure e_idx[i] and pixel p_idx[i],
 * out[i] = FF[p] sum_s F_s sum_l w_l sum_{q in the os x os block of p} |E_{l,s,e}[q]|^2,
 * with each E[q] a direct sum sum_ny A[ky][ny] sum_nx P[ny][nx] A[kx][nx]. */
void orc_model_at(const orc_problem *q, int n_pix, const int *e_idx, const int *p_idx, double *out) {
    int n = q->n_pupil, nd = q->n_det, os = q->oversample, no = nd * os;
    size_t npx = (size_t)n * n;
    double dx = q->diameter / n, du = mft_du(q), wn = weight_norm(q);
    double *opd = (double *)malloc(npx * sizeof(double));
    cplx *P = (cplx *)malloc(npx * sizeof(cplx));
    cplx *ax = (cplx *)malloc((size_t)n * sizeof(cplx)), *ay = (cplx *)malloc((size_t)n * sizeof(cplx));
    orc_opd(q, opd);
    for (int i = 0; i < n_pix; ++i) out[i] = 0;
    for (int e = 0; e < q->n_exp; ++e)
        for (int s = 0; s < q->n_src; ++s)
            for (int l = 0; l < q->n_lambda; ++l) {
                int any = 0;
                for (int i = 0; i < n_pix; ++i) any |= (e_idx[i] == e);
                if (!any) continue;
                double lam = q->lambdas[l], sc = sqrt(dx * du / lam), w = q->weights[l] / wn;
                orc_phasor(q, opd, l, s, e, P);
                fresnel_pre(q, lam, 1, P);
                for (int i = 0; i < n_pix; ++i) {
                    if (e_idx[i] != e) continue;
                    int py = p_idx[i] / nd, px = p_idx[i] % nd;
                    double acc = 0;
                    for (int a = 0; a < os; ++a)
                        for (int b = 0; b < os; ++b) {
                            int ky = py * os + a, kx = px * os + b;
                            for (int t = 0; t < n; ++t) {
                                double phx = -TWO_PI * coord(t, n, dx) * coord(kx, no, du) / lam;
                                double phy = -TWO_PI * coord(t, n, dx) * coord(ky, no, du) / lam;
                                ax[t] = sc * (cos(phx) + I * sin(phx));
                                ay[t] = sc * (cos(phy) + I * sin(phy));
                            }
                            cplx E = 0;
                            for (int ny = 0; ny < n; ++ny) {
                                cplx row = 0;
                                for (int nx = 0; nx < n; ++nx) row += P[(size_t)ny * n + nx] * ax[nx];
                                E += ay[ny] * row;
                            }
                            if (q->focal_length > 0) { /* the factor after the transform */
                                double f = q->focal_length, z = f + q->focal_shift, dr = q->pixscale * f / os;
                                double rx = coord(kx, no, dr), ry = coord(ky, no, dr);
                                double ph = (0.5 * TWO_PI) * (rx * rx + ry * ry) / (lam * z);
                                E *= cos(ph) + I * sin(ph);
                            }
                            acc += creal(E) * creal(E) + cimag(E) * cimag(E);
                        }
                    out[i] += q->flux[s] * w * acc;
                }
            }
    for (int i = 0; i < n_pix; ++i) out[i] *= q->flat[p_idx[i]];
    free(opd);
    free(P);
    free(ax);
    free(ay);
}
