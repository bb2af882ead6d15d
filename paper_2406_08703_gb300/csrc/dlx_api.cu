// C ABI entry points (include/dlx.h): plan creation, forward, loss + gradient,
// Adam, diagnostics.  Orchestration only; every step of the path is one of
// the kernels in k_elem.cu, k_gemm_simt.cu and k_gemm_tc.cu.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <initializer_list>
#include <string>

#include "dlx_common.cuh"
#include "s2_schedule.h"

static thread_local std::string g_last_error;

void dlx_set_error(const std::string &msg) { g_last_error = msg; }

namespace {

// Makes the plan's device current for the duration of a call and restores the caller's.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

int fail(int code, const std::string &msg) {
    dlx_set_error(msg);
    return code;
}

int cuda_fail(cudaError_t e, const char *where) {
    return fail(DLX_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define DLX_CU(call, where)                              \
    do {                                                 \
        cudaError_t _e = (call);                         \
        if (_e != cudaSuccess) return cuda_fail(_e, where); \
    } while (0)

template <class T>
cudaError_t plan_alloc(dlx_plan *p, T **ptr, size_t bytes) {
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, bytes ? bytes : 16);
    if (e != cudaSuccess) return e;
    p->allocs.push_back(q);
    p->workspace += bytes;
    *ptr = (T *)q;
    return cudaSuccess;
}

void plan_free(dlx_plan *p) {
    for (void *q : p->allocs) cudaFree(q);
    p->allocs.clear();
}

// Level-1 checks of a call's device arrays (list of pointer, bytes, alignment, name,
// optional), after those of its dlx_params; clears the plan's level-2 record.
struct Buf {
    const void *ptr;
    size_t bytes, align;
    const char *name;
    bool optional;
};
int check_call(dlx_plan *p, const dlx_params *prm, std::initializer_list<Buf> bufs,
               const dlx_grads *g = nullptr, const char *gname = "grads") {
    p->check_rc = 0;
    p->check_msg.clear();
    if (dlx::check_level() < 1) return DLX_OK;
    int rc = dlx::check_params(p, prm);
    for (const Buf &b : bufs)
        if (!rc) rc = dlx::check_buffer(b.ptr, b.bytes, b.align, p->device, b.name, b.optional);
    if (!rc) rc = dlx::check_grads(p, g, gname);
    return rc;
}

int validate_params(const dlx_plan *p, const dlx_params *prm) {
    if (!prm) return fail(DLX_ERR_INVALID_ARG, "params is NULL");
    if (!prm->transmission || !prm->weights || !prm->flux || !prm->pos || !prm->flat)
        return fail(DLX_ERR_INVALID_ARG, "transmission, weights, flux, pos and flat are required");
    if (p->nz > 0 && (!prm->zern_basis || !prm->zern_coeff))
        return fail(DLX_ERR_INVALID_ARG, "n_zern > 0 needs zern_basis and zern_coeff");
    return DLX_OK;
}

}  // namespace

namespace dlx {

static const char *kClassNames[KC_N] = {"mft_matrices", "prologue",      "stage1",          "stage2_intensity",
                                        "bin_nll",      "loss",          "adjoint_field",   "adjoint_stage2T",
                                        "adjoint_stage1T", "grad_reduce", "adam", "adjoint_field_scale"};

static cudaEvent_t pool_get(dlx_plan *p) {
    if (p->pool_next < p->pool.size()) return p->pool[p->pool_next++];
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    p->pool.push_back(e);
    p->pool_next++;
    return e;
}

KScope::KScope(dlx_plan *p_, int c, int n_, cudaStream_t s) : p(p_), cls(c), n(n_), st(s) {
    if ((p->timing >> cls) & 1u) {
        cudaEvent_t a = pool_get(p);
        b = pool_get(p);
        cudaEventRecord(a, st);
        p->recs.push_back({cls, a, b});
    }
}

KScope::~KScope() {
    p->launches[cls] += n;
    if (b) {
        cudaEventRecord(b, st);
        p->events[cls]++;
    }
    if (check_level() >= 2) class_check(p, cls, st);
}

const char *class_name(int cls) { return (cls >= 0 && cls < KC_N) ? kClassNames[cls] : "?"; }

void free_plan(dlx_plan *p) {
    if (!p) return;
    for (cudaEvent_t e : p->pool) cudaEventDestroy(e);
    p->pool.clear();
    plan_free(p);
    delete p;
}

int check_desc(const dlx_mft_desc *d, int *delta_out) {
    if (!d) return fail(DLX_ERR_INVALID_ARG, "desc is NULL");
    if (d->n_pupil < 2 || d->n_det < 1 || d->oversample < 1 || d->n_lambda < 1 || d->n_src < 1 || d->n_exp < 1 ||
        d->n_zern < 0)
        return fail(DLX_ERR_INVALID_ARG, "sizes must be positive (n_pupil >= 2)");
    if (!(d->diameter_m > 0) || !(d->pixscale_rad > 0)) return fail(DLX_ERR_INVALID_ARG, "diameter and pixscale > 0");
    if (!d->lambda_m) return fail(DLX_ERR_INVALID_ARG, "lambda_m is NULL");
    for (int l = 0; l < d->n_lambda; ++l)
        if (!(d->lambda_m[l] > 0) || !std::isfinite(d->lambda_m[l]))
            return fail(DLX_ERR_INVALID_ARG, "wavelengths must be finite and > 0");
    if (d->precision < DLX_FP32_SIMT || d->precision > DLX_BF16X3SA) return fail(DLX_ERR_INVALID_ARG, "bad precision");
    if (d->n_src > kMaxSrc) return fail(DLX_ERR_RANGE, "at most 32 sources per plan");
    if (!(d->prf_prior_sigma >= 0) || !std::isfinite(d->prf_prior_sigma))
        return fail(DLX_ERR_INVALID_ARG, "prf_prior_sigma must be finite and >= 0");
    if (!(d->focal_length_m >= 0) || !std::isfinite(d->focal_length_m) || !std::isfinite(d->focal_shift_m) ||
        (d->focal_length_m == 0 && d->focal_shift_m != 0) ||
        (d->focal_length_m > 0 && !(d->focal_length_m + d->focal_shift_m > 0)))
        return fail(DLX_ERR_INVALID_ARG, "focal_length_m >= 0 (0 with focal_shift_m 0) and focal_length_m + "
                                         "focal_shift_m > 0");
    // integer-pixel dithers: one MFT per source on a detector wide enough for every window
    int delta = 0;
    if (d->dither_px) {
        for (int k = 0; k < 2 * d->n_exp; ++k) {
            const int v = d->dither_px[k];
            if (v < -4096 || v > 4096) return fail(DLX_ERR_RANGE, "|dither_px| <= 4096");
            delta = std::max(delta, v < 0 ? -v : v);
        }
    }
    const long long nd_mft = (long long)d->n_det + 2LL * delta;
    const long long no_ll = nd_mft * d->oversample;
    if (d->n_pupil > 8192 || no_ll > 16384)
        return fail(DLX_ERR_RANGE, "n_pupil <= 8192 and (n_det + 2 max|dither_px|) * oversample <= 16384");
    // PSF and Zernike counts stay far inside the 32-bit index arithmetic
    if (d->n_zern > 4096 || (long long)d->n_lambda * d->n_src * d->n_exp > (1LL << 24))
        return fail(DLX_ERR_RANGE, "n_zern <= 4096 and n_lambda * n_src * n_exp <= 2^24");
    if (delta_out) *delta_out = delta;
    return DLX_OK;
}

int make_plan(const dlx_mft_desc *d, int device, int R_max, dlx_plan **out) {
    if (!d || !out) return fail(DLX_ERR_INVALID_ARG, "desc/out is NULL");
    *out = nullptr;
    if (R_max < 1) return fail(DLX_ERR_INVALID_ARG, "R_max must be >= 1");
    int delta = 0;
    if (int rc = check_desc(d, &delta)) return rc;
    const long long nd_mft = (long long)d->n_det + 2LL * delta;
    const long long no_ll = nd_mft * d->oversample;

    DeviceGuard guard(device);
    cudaDeviceProp prop;
    DLX_CU(cudaGetDeviceProperties(&prop, device), "cudaGetDeviceProperties");

    dlx_plan *p = new dlx_plan();
    p->desc = *d;
    p->lambdas.assign(d->lambda_m, d->lambda_m + d->n_lambda);
    p->desc.lambda_m = p->lambdas.data();
    if (d->dither_px) p->dither_px.assign(d->dither_px, d->dither_px + 2 * d->n_exp);
    p->desc.dither_px = d->dither_px ? p->dither_px.data() : nullptr;
    p->device = device;
    p->R_max = R_max;
    p->sm_count = prop.multiProcessorCount;
    p->cc_major = prop.major;
    p->cc_minor = prop.minor;
    p->ni = d->n_pupil;
    p->ndi = d->n_det;
    p->nei = d->n_exp;
    p->nd = (int)nd_mft;
    p->os = d->oversample;
    p->no = (int)no_ll;
    p->nl = d->n_lambda;
    p->ns = d->n_src;
    p->ne = d->dither_px ? 1 : d->n_exp;
    p->nz = d->n_zern;
    p->nse = p->ns * p->ne;
    p->B = p->nl * p->nse;
    p->ldi = dlx::operand_ld(p->ni);
    p->ldo = dlx::operand_ld(p->no);
    p->prec = d->precision;
    // a 16-bit split (hi + lo BF16 carry about 17 significant bits) leaves each operand a
    // representation error near 2^-17 that a contraction averages down only over its terms: with
    // fewer than 32 pupil samples the PSF misses 1e-5 of its peak (measured 1.0-3.2e-5 at 5 and
    // 17 samples), so those plans run the 22-bit FP16 split
    if (p->ni < kMinBf16Pupil && (p->prec == DLX_BF16X3 || p->prec == DLX_BF16X4 || p->prec == DLX_BF16X3SA))
        p->prec = DLX_F16X3;
    p->fmt = fmt_of_prec(p->prec);
    p->sr = (p->prec == DLX_BF16X3 || p->prec == DLX_BF16X3SA) ? 0x6d2b79f5u : 0u;  // stochastic split
    p->adj1 = (p->prec == DLX_BF16X3SA);
    // the FP16 split form runs the forward contractions mirror-paired (pair_layout)
    p->paired = (p->fmt == FMT_F16X4);
    if (p->paired) {
        p->hn = (p->ni + 1) / 2;
        p->hp = pair_half(p->ni);
        p->ldk = operand_ld(2 * p->hp);
    }
    p->prf_inv = d->prf_prior_sigma > 0 ? (float)(1.0 / (d->prf_prior_sigma * d->prf_prior_sigma)) : 0.f;
    p->planes = fmt_planes(p->fmt);
    p->esz = fmt_esize(p->fmt);
    p->dx = d->diameter_m / p->ni;
    double du_scale;
    fresnel_terms(d, &du_scale, &p->chirp);
    p->du = d->pixscale_rad / p->os * du_scale;

    if (p->prec != DLX_FP32_SIMT) {
        std::string why;
        if (!(p->cc_major == 10 && p->cc_minor == 3)) {
            delete p;
            return fail(DLX_ERR_UNSUPPORTED, "tensor-core forms are built for sm_103a only");
        }
        if (!tc_supported(p, &why)) {
            delete p;
            return fail(DLX_ERR_UNSUPPORTED, why);
        }
    }

    const int Bt = p->B * R_max;
    // adjoint chunk: the per-wavelength recomputation batch
    const size_t per_psf = (size_t)(p->adj1 ? 2 : p->planes) * p->esz * ((size_t)p->no * p->ldo + (size_t)p->ni * p->ldo);
    int chunk = Bt;
    if (d->psf_chunk > 0)
        chunk = std::min(d->psf_chunk, Bt);
    else if (d->workspace_limit_bytes > 0)
        chunk = (int)std::max<size_t>(1, std::min<size_t>(Bt, d->workspace_limit_bytes / per_psf));
    p->chunk = chunk;

    // partial-intensity planes.  CUDA-core form: wavelength groups, enough
    // independent 64-tiles to cover every SM twice.  Tensor-core forms: the
    // planes of the balanced split of (tile, wavelength) jobs, for every count of
    // active slots.
    std::vector<int> s2_host;
    std::vector<int> fold_host;
    std::vector<uint8_t> used_host;
    if (p->prec == DLX_FP32_SIMT) {
        long units = (long)((p->no + 63) / 64) * ((p->no + 63) / 64) * p->nse;
        p->G = (int)std::min<long>(p->nl, std::max<long>(1, (2L * p->sm_count + units - 1) / units));
    } else {
        const int tt = ((p->no + 127) / 128) * ((p->no + 127) / 128);
        p->G = 1;
        p->s2.resize(R_max);
        for (int R = 1; R <= R_max; ++R) {
            const int nseg = tt * R * p->nse;
            int nct = 0;
            std::vector<int> off;
            std::vector<S2Piece> pcs;
            const int planes = s2_schedule(nseg, p->nl, p->sm_count, nct, off, pcs);
            std::string why;
            if (!s2_check(nseg, p->nl, nct, off, pcs, planes, &why)) {
                free_plan(p);
                return fail(DLX_ERR_CUDA, why);
            }
            p->G = std::max(p->G, planes);
            dlx_plan::S2Split &sp = p->s2[R - 1];
            sp.off = (long)s2_host.size();
            s2_host.insert(s2_host.end(), off.begin(), off.end());
            while (s2_host.size() % 4) s2_host.push_back(0);
            sp.pcs = (long)s2_host.size();
            // the segments written in more than one plane are folded into plane 0 after the
            // contraction, so no piece clears the planes its segment leaves unwritten
            std::vector<int> used((size_t)nseg, 0);
            for (const S2Piece &q : pcs) {
                s2_host.insert(s2_host.end(), {q.seg, q.l0, q.l1, (q.pz & 0xffff) | (kS2None << 16)});
                used[q.seg] = std::max(used[q.seg], (q.pz & 0xffff) + 1);
            }
            sp.used = (long)used_host.size();
            for (int sg = 0; sg < nseg; ++sg) used_host.push_back((uint8_t)used[sg]);
            sp.fold = (long)fold_host.size() / 2;
            for (int sg = 0; sg < nseg; ++sg)
                if (used[sg] > 1) fold_host.insert(fold_host.end(), {sg, used[sg]});
            sp.nfold = (int)(fold_host.size() / 2 - sp.fold);
            sp.nct = nct;
            sp.npieces = (int)pcs.size();
        }
    }

    cudaError_t e = cudaSuccess;
    auto op_alloc = [&](Operand &o, int batch, int rows, int ld, int planes) {
        o.batch = batch;
        o.rows = rows;
        o.ld = ld;
        o.planes = planes;
        o.bytes = (size_t)batch * planes * rows * ld * p->esz;
        if (e == cudaSuccess) e = plan_alloc(p, &o.ptr, o.bytes);
        if (e == cudaSuccess) e = cudaMemset(o.ptr, 0, o.bytes);
    };
    // BF16x3sa: the adjoint-only operands (AH, GEt, GT1) hold the stochastic hi parts alone
    const int adj_planes = p->adj1 ? 2 : p->planes;
    // the fields stage 2 keeps for the adjoint (instead of its recomputation), when the adjoint
    // takes every PSF at once and a workspace limit leaves room for them
    const size_t ef_bytes = sizeof(float) * 2 * (size_t)Bt * p->no * p->ldo;
    const bool keep_e = field_kept(p->fmt, p->adj1, p->ni, p->chunk, Bt) &&
                        (d->workspace_limit_bytes == 0 || d->workspace_limit_bytes >= (size_t)Bt * per_psf + ef_bytes);
    p->padj = p->paired && keep_e;
    if (p->paired) {
        op_alloc(p->amat, p->nl, p->no, p->ldk, 2);
        op_alloc(p->Pp, Bt, 2 * p->hp, p->ldk, p->planes);
        op_alloc(p->T1t, Bt, p->no, p->ldk, p->planes);
    } else {
        op_alloc(p->amat, p->nl, p->no, p->ldi, p->planes);
        op_alloc(p->T1t, Bt, p->no, p->ldi, p->planes);
    }
    op_alloc(p->P, Bt, p->ni, p->ldi, p->planes);
    if (p->padj) {
        p->hno = (p->no + 1) / 2;
        p->hpo = pair_half(p->no);
        p->ldko = operand_ld(2 * p->hpo);
        op_alloc(p->amatH, p->nl, p->ni, p->ldko, 2);
        op_alloc(p->GEt, p->chunk, 2 * p->hpo, p->ldko, p->planes);
        op_alloc(p->GT1, p->chunk, p->ni, p->ldko, p->planes);
    } else {
        op_alloc(p->amatH, p->nl, p->ni, p->ldo, adj_planes);
        op_alloc(p->GEt, p->chunk, p->no, p->ldo, adj_planes);
        op_alloc(p->GT1, p->chunk, p->ni, p->ldo, adj_planes);
    }
    const size_t npx = (size_t)p->ni * p->ni, np = (size_t)p->nd * p->nd, nq = (size_t)p->no * p->no;
    const size_t npi = (size_t)p->ndi * p->ndi;
    // blocks of the one-pass binning: up to eight per SM, so that enough loads are in flight
    p->red_blocks = std::max(1, std::min((int)((npi + 255) / 256), std::max(1, p->sm_count * 8 / R_max)));
    if (e == cudaSuccess) e = plan_alloc(p, &p->lam_d, sizeof(double) * p->nl);
    if (e == cudaSuccess) e = plan_alloc(p, &p->wnorm, sizeof(float) * p->nl * R_max);
    if (e == cudaSuccess) e = plan_alloc(p, &p->pscale, sizeof(float) * 2 * R_max);
    if (e == cudaSuccess) e = plan_alloc(p, &p->tpart, sizeof(float) * kNormParts * R_max);
    if (p->fmt == FMT_F16X4) {
        // FP16 operand scales: alpha_l = 2^-ceil(log2 sqrt(dx du / lambda_l)); adjoint maxima
        std::vector<float> al(p->nl);
        for (int l = 0; l < p->nl; ++l) al[l] = inv_pow2_ceil((float)std::sqrt(p->dx * p->du / p->lambdas[l]));
        if (e == cudaSuccess) e = plan_alloc(p, &p->ascale, sizeof(float) * p->nl);
        if (e == cudaSuccess) e = cudaMemcpy(p->ascale, al.data(), sizeof(float) * p->nl, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = plan_alloc(p, &p->qmax, sizeof(unsigned int) * R_max * p->nse);
        if (e == cudaSuccess) e = plan_alloc(p, &p->gmax, sizeof(unsigned int) * Bt);
    }
    if (e == cudaSuccess) e = plan_alloc(p, &p->invlam, sizeof(float) * p->nl);
    if (e == cudaSuccess) e = plan_alloc(p, &p->tilt, sizeof(float2) * Bt * 2 * p->ni);
    if (e == cudaSuccess) e = plan_alloc(p, &p->opd, sizeof(float) * npx * R_max);
    if (e == cudaSuccess) e = plan_alloc(p, &p->Is, sizeof(float) * (size_t)p->G * p->nse * R_max * nq);
    if (e == cudaSuccess && keep_e) {
        e = plan_alloc(p, &p->Ef, ef_bytes);
        if (e == cudaSuccess) e = cudaMemset(p->Ef, 0, ef_bytes);
        if (e == cudaSuccess) e = plan_alloc(p, &p->GIt, sizeof(float) * p->ne * np * R_max);
    }
    if (e == cudaSuccess) e = plan_alloc(p, &p->GI, sizeof(float) * p->ne * np * R_max);
    if (e == cudaSuccess) e = plan_alloc(p, &p->model_tmp, sizeof(float) * p->nei * npi * R_max);
    if (d->dither_px) {
        // window of image e: big-detector pixel (x, y) = image pixel + (delta - dither_x, delta - dither_y)
        std::vector<int> off(2 * p->nei);
        for (int k = 0; k < p->nei; ++k) {
            off[2 * k] = delta - d->dither_px[2 * k];
            off[2 * k + 1] = delta - d->dither_px[2 * k + 1];
        }
        if (e == cudaSuccess) e = plan_alloc(p, &p->GIimg, sizeof(float) * p->nei * npi * R_max);
        if (e == cudaSuccess) e = plan_alloc(p, &p->Swin, sizeof(float) * np * R_max);
        if (e == cudaSuccess) e = plan_alloc(p, &p->crop, sizeof(int) * 2 * p->nei);
        if (e == cudaSuccess) e = cudaMemcpy(p->crop, off.data(), sizeof(int) * 2 * p->nei, cudaMemcpyHostToDevice);
    }
    if (p->prec != DLX_FP32_SIMT) {
        // split the long-K adjoint 1^T contraction only while its 128-tiles do not fill
        // the SMs once: every split adds a gphi plane and a re-read of the phasor tile
        // in the epilogue, which costs more than a partial last wave
        const long units = (long)p->chunk * ((p->ni + 127) / 128) * ((p->ni + 127) / 128);
        const int kblocks = (p->no + 31) / 32;
        int s = 1;
        while (s < 8 && units * s < (long)p->sm_count && kblocks / (2 * s) >= 4) s *= 2;
        p->gsplit = s;
    }
    if (e == cudaSuccess) e = plan_alloc(p, &p->gphi, sizeof(float) * Bt * npx * p->gsplit);
    if (e == cudaSuccess) e = plan_alloc(p, &p->gopd, sizeof(float2) * npx * R_max);
    if (e == cudaSuccess) e = plan_alloc(p, &p->red, sizeof(double) * p->red_blocks * (1 + kMaxSrc) * R_max);
    if (p->ns > 8 || d->dither_px) {
        // two-pass binning (and the window passes): one thread per pixel for the model pass, a
        // (blocks x source) grid for the flux gradients, each about 8 blocks of 256 threads per SM
        p->bin_a_blocks = (int)std::max<size_t>(1, std::min<size_t>((npi + 255) / 256, (size_t)p->sm_count * 8 / R_max));
        p->bin_b_blocks = (int)std::max<size_t>(
            1, std::min<size_t>((npi + 255) / 256, ((size_t)p->sm_count * 8 + (size_t)p->ns * R_max - 1) /
                                                      ((size_t)p->ns * R_max)));
        if (e == cudaSuccess) e = plan_alloc(p, &p->red_a, sizeof(double) * p->bin_a_blocks * R_max);
        // the window flux pass has (column blocks x row blocks) partials per source, most at R = 1
        const int nb_win = d->dither_px ? ((p->nd + 127) / 128) * win_flux_rows(p, 1) : 0;
        const size_t nb_flux = (size_t)std::max(p->bin_b_blocks, nb_win);
        if (e == cudaSuccess) e = plan_alloc(p, &p->red_b, sizeof(double) * nb_flux * kMaxSrc * R_max);
        if (e == cudaSuccess) e = plan_alloc(p, &p->fcount, sizeof(unsigned int) * kMaxSrc * R_max);
        if (e == cudaSuccess) e = cudaMemset(p->fcount, 0, sizeof(unsigned int) * kMaxSrc * R_max);
    }
    if (e == cudaSuccess && p->prec == DLX_FP32_SIMT)
        e = plan_alloc(p, &p->pos_part, sizeof(double) * 2 * Bt * p->gsplit);
    if (e == cudaSuccess) e = plan_alloc(p, &p->npart, sizeof(float2) * kNormParts * R_max);
    if (e == cudaSuccess) e = plan_alloc(p, &p->ncount, sizeof(unsigned int) * R_max);
    if (e == cudaSuccess) e = cudaMemset(p->ncount, 0, sizeof(unsigned int) * R_max);
    if (e == cudaSuccess && p->prec != DLX_FP32_SIMT) {
        const size_t tiles = (size_t)((p->ni + 127) / 128) * ((p->ni + 127) / 128);
        e = plan_alloc(p, &p->mom, sizeof(float) * 2 * 8 * tiles * Bt * p->gsplit);
    }
    if (e == cudaSuccess)
        e = plan_alloc(p, &p->zpart, sizeof(float2) * R_max * std::max(1, p->nz) * ((npx + 63) / 64));
    if (e == cudaSuccess) e = plan_alloc(p, &p->bcount, sizeof(unsigned int) * R_max);
    if (e == cudaSuccess) e = cudaMemset(p->bcount, 0, sizeof(unsigned int) * R_max);
    if (e == cudaSuccess && !s2_host.empty()) {
        e = plan_alloc(p, &p->s2_table, sizeof(int) * s2_host.size());
        if (e == cudaSuccess)
            e = cudaMemcpy(p->s2_table, s2_host.data(), sizeof(int) * s2_host.size(), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = plan_alloc(p, &p->s2_used, used_host.size());
        if (e == cudaSuccess) e = cudaMemcpy(p->s2_used, used_host.data(), used_host.size(), cudaMemcpyHostToDevice);
        if (e == cudaSuccess && !fold_host.empty()) {
            e = plan_alloc(p, &p->s2_fold, sizeof(int) * fold_host.size());
            if (e == cudaSuccess)
                e = cudaMemcpy(p->s2_fold, fold_host.data(), sizeof(int) * fold_host.size(), cudaMemcpyHostToDevice);
        }
    }
    if (e == cudaSuccess) e = plan_alloc(p, &p->err, sizeof(int32_t));
    if (e == cudaSuccess) e = plan_alloc(p, &p->clamped, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(p->err, 0, sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMemset(p->clamped, 0, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemcpy(p->lam_d, p->lambdas.data(), sizeof(double) * p->nl, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        std::vector<float> inv(p->nl);
        for (int l = 0; l < p->nl; ++l) inv[l] = (float)(1.0 / p->lambdas[l]);
        e = cudaMemcpy(p->invlam, inv.data(), sizeof(float) * p->nl, cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = launch_mft_matrices(p, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        int code = (e == cudaErrorMemoryAllocation) ? DLX_ERR_NOMEM : DLX_ERR_CUDA;
        std::string msg = std::string("plan setup: ") + cudaGetErrorString(e);
        cudaGetLastError();
        free_plan(p);
        return fail(code, msg);
    }
    if (p->prec != DLX_FP32_SIMT) {
        std::string why;
        if (!tc_make_maps(p, &why)) {
            free_plan(p);
            return fail(DLX_ERR_CUDA, "tensor maps: " + why);
        }
    }
    *out = p;
    return DLX_OK;
}

int eval_forward(dlx_plan *p, const DevParams &prm, int R, cudaStream_t st) {
    DLX_CU(launch_prologue(p, prm, R, st), "prologue");
    if (p->prec == DLX_FP32_SIMT) {
        DLX_CU(simt_forward(p, R, st), "simt forward");
    } else {
        DLX_CU(tc_forward(p, R, st), "tensor-core forward");
        if (folds_planes(p)) DLX_CU(launch_plane_fold(p, R, st), "plane fold");
    }
    return DLX_OK;
}

int eval_loss_grad(dlx_plan *p, const DevParams &prm, int R, const int32_t *data, size_t data_stride, double *loss,
                   const DevGrads *g, float *model, size_t model_stride, cudaStream_t st) {
    const bool pupil = g && (g->p[GZERN] || g->p[GPIX] || g->p[GPOS]);
    // stage 2 keeps each PSF's field for the adjoint when a pupil gradient is wanted and the
    // adjoint operand holds every PSF; the flag lives for this evaluation only
    struct KeepField {
        dlx_plan *p;
        ~KeepField() { p->keep_field = false; }
    } keep{p};
    p->keep_field = pupil && keeps_field(p, R);
    int rc = eval_forward(p, prm, R, st);
    if (rc) return rc;
    if (!model) {
        model = p->model_tmp;
        model_stride = (size_t)p->nei * p->ndi * p->ndi;
    }
    DLX_CU(launch_bin_nll(p, prm, R, data, data_stride, model, model_stride, g, loss, st), "bin+nll+loss");
    if (pupil) {
        const int Bt = R * p->B;
        for (int b0 = 0; b0 < Bt; b0 += p->chunk) {
            int nb = std::min(p->chunk, Bt - b0);
            if (p->prec == DLX_FP32_SIMT) {
                DLX_CU(simt_adjoint_chunk(p, prm, b0, nb, st), "simt adjoint");
            } else {
                DLX_CU(tc_adjoint_chunk(p, prm, b0, nb, st), "tensor-core adjoint");
            }
        }
        DLX_CU(launch_grad_reduce(p, prm, R, g, st), "gradient reductions");
    }
    return DLX_OK;
}

}  // namespace dlx

namespace {

dlx::DevParams dev_params(const dlx_plan *p, const dlx_params *q) {
    dlx::DevParams d{};
    d.p[dlx::PT] = q->transmission;
    d.p[dlx::POPDF] = q->opd_fixed;
    d.p[dlx::PBASIS] = q->zern_basis;
    d.p[dlx::PCOEFF] = q->zern_coeff;
    d.p[dlx::POPDPIX] = q->opd_pix;
    d.p[dlx::PW] = q->weights;
    d.p[dlx::PFLUX] = q->flux;
    d.p[dlx::PPOS] = q->pos;
    d.p[dlx::PDITHER] = p->crop ? nullptr : q->dither;  // integer dithers are windows, not tilts
    d.p[dlx::PFLAT] = q->flat;
    return d;
}

dlx::DevGrads dev_grads(const dlx_grads *g) {
    dlx::DevGrads d{};
    if (!g) return d;
    d.p[dlx::GZERN] = g->d_zern;
    d.p[dlx::GPIX] = g->d_opd_pix;
    d.p[dlx::GFLAT] = g->d_flat;
    d.p[dlx::GFLUX] = g->d_flux;
    d.p[dlx::GPOS] = g->d_pos;
    return d;
}

}  // namespace

extern "C" {

const char *dlx_last_error(void) { return g_last_error.c_str(); }

const char *dlx_version(void) { return "dlx 0.1 (sm_103a)"; }

int dlx_make_mft(const dlx_mft_desc *d, int device, dlx_plan **out) { return dlx::make_plan(d, device, 1, out); }

int dlx_destroy_plan(dlx_plan *p) {
    if (!p) return DLX_OK;
    DeviceGuard guard(p->device);
    cudaDeviceSynchronize();
    dlx::free_plan(p);
    return DLX_OK;
}

int dlx_plan_get_info(const dlx_plan *p, dlx_plan_info *o) {
    if (!p || !o) return fail(DLX_ERR_INVALID_ARG, "NULL argument");
    memset(o, 0, sizeof(*o));
    o->n_pupil = p->ni;
    o->n_det = p->ndi;
    o->oversample = p->os;
    o->n_out = p->ndi * p->os;
    o->n_mft_out = p->no;
    o->n_lambda = p->nl;
    o->n_src = p->ns;
    o->n_exp = p->nei;
    o->n_zern = p->nz;
    o->n_psf = p->B;
    o->precision = p->prec;
    o->psf_chunk = p->chunk;
    o->workspace_bytes = p->workspace;
    const double ni = p->ni, no = p->no;
    const double s1 = 8.0 * no * ni * ni, s2 = 8.0 * no * no * ni;
    o->flop_forward = p->B * (s1 + s2);
    // forward (s1 + s2) + adjoint stage 2^T (s2) + adjoint stage 1^T (s1), and the recomputed field
    // (s2) where the plan does not keep the fields of stage 2
    o->flop_loss_grad = p->B * (2 * s1 + (p->Ef ? 2 : 3) * s2);
    int t = (p->prec == DLX_FP32_SIMT) ? 64 : 128;
    o->gemm_tiles_stage2 = ((p->no + t - 1) / t) * ((p->no + t - 1) / t) * p->nse * p->G;
    return DLX_OK;
}

int dlx_forward(dlx_plan *p, const dlx_params *prm, float *model, void *stream) {
    if (!p || !model) return fail(DLX_ERR_INVALID_ARG, "plan/model is NULL");
    int rc = validate_params(p, prm);
    if (rc) return rc;
    if ((rc = check_call(p, prm, {{model, dlx::image_bytes(p), 4, "model", false}}))) return rc;
    DeviceGuard guard(p->device);
    cudaStream_t st = (cudaStream_t)stream;
    const dlx::DevParams d = dev_params(p, prm);
    if ((rc = dlx::eval_forward(p, d, 1, st))) return dlx::checked_status(p, rc);
    DLX_CU(dlx::launch_bin_nll(p, d, 1, nullptr, 0, model, 0, nullptr, nullptr, st), "bin");
    return dlx::checked_status(p, DLX_OK);
}

int dlx_model_jvp(dlx_plan *p, const dlx_params *prm, const float *t_map, uint32_t src_mask, double alpha, float *jvp,
                  float *work, void *stream) {
    if (!p || !t_map || !jvp || !work) return fail(DLX_ERR_INVALID_ARG, "plan/t_map/jvp/work is NULL");
    if (!(alpha > 0) || !std::isfinite(alpha)) return fail(DLX_ERR_INVALID_ARG, "alpha must be finite and > 0");
    int rc = validate_params(p, prm);
    if (rc) return rc;
    if ((rc = check_call(p, prm,
                         {{t_map, 4 * (size_t)p->ni * p->ni, 4, "t_map", false},
                          {jvp, dlx::image_bytes(p), 4, "jvp", false},
                          {work, dlx::image_bytes(p), 4, "work", false}})))
        return rc;
    DeviceGuard guard(p->device);
    cudaStream_t st = (cudaStream_t)stream;
    const dlx::DevParams d = dev_params(p, prm);
    // m(+alpha) into jvp, m(-alpha) into work; the model is quadratic in the phasor, so the
    // central difference over 2 alpha is the derivative itself
    p->tan_map = t_map;
    p->tan_mask = src_mask;
    for (int k = 0; k < 2 && rc == 0; ++k) {
        p->tan_coef = (float)(k == 0 ? alpha : -alpha);
        rc = dlx::eval_forward(p, d, 1, st);
        if (rc == 0) {
            cudaError_t e = dlx::launch_bin_nll(p, d, 1, nullptr, 0, k == 0 ? jvp : work, 0, nullptr, nullptr, st);
            if (e != cudaSuccess) rc = cuda_fail(e, "bin");
        }
    }
    p->tan_map = nullptr;
    p->tan_coef = 0.f;
    p->tan_mask = 0;
    if (rc) return dlx::checked_status(p, rc);
    DLX_CU(dlx::launch_scaled_diff(jvp, work, (size_t)p->nei * p->ndi * p->ndi, (float)(0.5 / alpha), st), "jvp");
    return dlx::checked_status(p, DLX_OK);
}

int dlx_model_vjp(dlx_plan *p, const dlx_params *prm, const float *cot, const dlx_grads *g, void *stream) {
    if (!p || !cot || !g) return fail(DLX_ERR_INVALID_ARG, "plan/cot/grads is NULL");
    int rc = validate_params(p, prm);
    if (rc) return rc;
    if ((rc = check_call(p, prm, {{cot, dlx::image_bytes(p), 4, "cot", false}}, g))) return rc;
    DeviceGuard guard(p->device);
    cudaStream_t st = (cudaStream_t)stream;
    const dlx::DevParams d = dev_params(p, prm);
    const dlx::DevGrads dg = dev_grads(g);
    p->cot = cot;
    rc = dlx::eval_loss_grad(p, d, 1, nullptr, 0, nullptr, &dg, nullptr, 0, st);
    p->cot = nullptr;
    return dlx::checked_status(p, rc);
}

int dlx_model_vjp_jvp(dlx_plan *p, const dlx_params *prm, const float *cot, const float *t_map, uint32_t src_mask,
                      double alpha, const dlx_grads *g, const dlx_grads *work, void *stream) {
    if (!p || !cot || !t_map || !g || !work) return fail(DLX_ERR_INVALID_ARG, "plan/cot/t_map/grads/work is NULL");
    if (!(alpha > 0) || !std::isfinite(alpha)) return fail(DLX_ERR_INVALID_ARG, "alpha must be finite and > 0");
    const float *gp[5] = {g->d_zern, g->d_opd_pix, g->d_flat, g->d_flux, g->d_pos};
    const float *wp[5] = {work->d_zern, work->d_opd_pix, work->d_flat, work->d_flux, work->d_pos};
    for (int k = 0; k < 5; ++k)
        if (gp[k] && !wp[k]) return fail(DLX_ERR_INVALID_ARG, "work lacks an array that grads has");
    int rc = validate_params(p, prm);
    if (rc) return rc;
    if ((rc = check_call(p, prm,
                         {{cot, dlx::image_bytes(p), 4, "cot", false},
                          {t_map, 4 * (size_t)p->ni * p->ni, 4, "t_map", false}},
                         g)) ||
        (dlx::check_level() >= 1 && (rc = dlx::check_grads(p, work, "work"))))
        return rc;
    DeviceGuard guard(p->device);
    cudaStream_t st = (cudaStream_t)stream;
    const dlx::DevParams d = dev_params(p, prm);
    // J^T cot at the phasors P (1 + i a) into g and P (1 - i a) into work; it is a quadratic
    // form of the phasor, so the central difference over 2 alpha is its derivative
    dlx_grads wk = *g;
    wk.d_zern = g->d_zern ? work->d_zern : nullptr;
    wk.d_opd_pix = g->d_opd_pix ? work->d_opd_pix : nullptr;
    wk.d_flat = g->d_flat ? work->d_flat : nullptr;
    wk.d_flux = g->d_flux ? work->d_flux : nullptr;
    wk.d_pos = g->d_pos ? work->d_pos : nullptr;
    p->cot = cot;
    p->tan_map = t_map;
    p->tan_mask = src_mask;
    for (int k = 0; k < 2 && rc == 0; ++k) {
        p->tan_coef = (float)(k == 0 ? alpha : -alpha);
        const dlx::DevGrads dg = dev_grads(k == 0 ? g : &wk);
        rc = dlx::eval_loss_grad(p, d, 1, nullptr, 0, nullptr, &dg, nullptr, 0, st);
    }
    p->cot = nullptr;
    p->tan_map = nullptr;
    p->tan_coef = 0.f;
    p->tan_mask = 0;
    if (rc) return dlx::checked_status(p, rc);
    const size_t n[5] = {(size_t)p->nz, (size_t)p->ni * p->ni, (size_t)p->ndi * p->ndi, (size_t)p->ns,
                         (size_t)2 * p->ns};
    for (int k = 0; k < 5; ++k)
        if (gp[k]) DLX_CU(dlx::launch_scaled_diff((float *)gp[k], wp[k], n[k], (float)(0.5 / alpha), st), "vjp_jvp");
    return dlx::checked_status(p, DLX_OK);
}

int dlx_nll_cotangent(const float *model, const int32_t *data, size_t n, float *cot, void *stream) {
    if (!model || !data || !cot) return fail(DLX_ERR_INVALID_ARG, "model/data/cot is NULL");
    if (dlx::check_level() >= 1) {
        int dev = 0, rc;
        cudaGetDevice(&dev);
        if ((rc = dlx::check_buffer(model, 4 * n, 4, dev, "model", false)) ||
            (rc = dlx::check_buffer(data, 4 * n, 4, dev, "data", false)) ||
            (rc = dlx::check_buffer(cot, 4 * n, 4, dev, "cot", false)))
            return rc;
    }
    DLX_CU(dlx::launch_nll_cotangent(model, data, n, cot, (cudaStream_t)stream), "nll_cotangent");
    return DLX_OK;
}

int dlx_fisher_gram(const float *J, int n_par, size_t n_pix, const float *model, const int32_t *data, double *F,
                    double *work, void *stream) {
    if (!J || !model || !F || !work) return fail(DLX_ERR_INVALID_ARG, "J/model/F/work is NULL");
    if (n_par < 1 || n_par > DLX_GRAM_MAX_PAR) return fail(DLX_ERR_RANGE, "n_par must be 1..DLX_GRAM_MAX_PAR");
    if (n_pix == 0) return fail(DLX_ERR_INVALID_ARG, "n_pix is 0");
    if (dlx::check_level() >= 1) {
        int dev = 0, rc;
        cudaGetDevice(&dev);
        const size_t np2 = (size_t)n_par * n_par, tri = (size_t)n_par * (n_par + 1) / 2;
        if ((rc = dlx::check_buffer(J, 4 * (size_t)n_par * n_pix, 4, dev, "J", false)) ||
            (rc = dlx::check_buffer(model, 4 * n_pix, 4, dev, "model", false)) ||
            (rc = dlx::check_buffer(data, 4 * n_pix, 4, dev, "data", true)) ||
            (rc = dlx::check_buffer(F, 8 * np2, 8, dev, "F", false)) ||
            (rc = dlx::check_buffer(work, 8 * DLX_GRAM_BLOCKS * tri, 8, dev, "work", false)))
            return rc;
    }
    DLX_CU(dlx::launch_fisher_gram(J, n_par, n_pix, model, data, F, work, (cudaStream_t)stream), "fisher_gram");
    return DLX_OK;
}

int dlx_psf(dlx_plan *p, const dlx_params *prm, float *psf_os, void *stream) {
    if (!p || !psf_os) return fail(DLX_ERR_INVALID_ARG, "plan/psf is NULL");
    int rc = validate_params(p, prm);
    if (rc) return rc;
    const size_t noi = (size_t)p->ndi * p->os;
    if ((rc = check_call(p, prm, {{psf_os, 4 * (size_t)p->nei * noi * noi, 4, "psf_os", false}}))) return rc;
    DeviceGuard guard(p->device);
    cudaStream_t st = (cudaStream_t)stream;
    const dlx::DevParams d = dev_params(p, prm);
    if ((rc = dlx::eval_forward(p, d, 1, st))) return dlx::checked_status(p, rc);
    DLX_CU(dlx::launch_psf_out(p, d, psf_os, st), "psf");
    return dlx::checked_status(p, DLX_OK);
}

int dlx_loss_grad(dlx_plan *p, const dlx_params *prm, const int32_t *data, double *loss, const dlx_grads *g,
                  float *model_opt, void *stream) {
    if (!p || !data || !loss) return fail(DLX_ERR_INVALID_ARG, "plan/data/loss is NULL");
    int rc = validate_params(p, prm);
    if (rc) return rc;
    if ((rc = check_call(p, prm,
                         {{data, dlx::image_bytes(p), 4, "data", false},
                          {loss, sizeof(double), 8, "loss", false},
                          {model_opt, dlx::image_bytes(p), 4, "model", true}},
                         g)))
        return rc;
    DeviceGuard guard(p->device);
    cudaStream_t st = (cudaStream_t)stream;
    DLX_CU(cudaMemsetAsync(p->clamped, 0, sizeof(unsigned long long), st), "memset");
    const dlx::DevParams d = dev_params(p, prm);
    const dlx::DevGrads dg = dev_grads(g);
    return dlx::checked_status(p, dlx::eval_loss_grad(p, d, 1, data, 0, loss, g ? &dg : nullptr, model_opt, 0, st));
}

int dlx_plan_diagnostics(dlx_plan *p, int64_t *clamped, int32_t *device_error) {
    if (!p) return fail(DLX_ERR_INVALID_ARG, "plan is NULL");
    DeviceGuard guard(p->device);
    DLX_CU(cudaDeviceSynchronize(), "synchronize");
    unsigned long long c = 0;
    int32_t err = 0;
    DLX_CU(cudaMemcpy(&c, p->clamped, sizeof(c), cudaMemcpyDeviceToHost), "copy");
    DLX_CU(cudaMemcpy(&err, p->err, sizeof(err), cudaMemcpyDeviceToHost), "copy");
    DLX_CU(cudaMemset(p->err, 0, sizeof(int32_t)), "memset");
    if (clamped) *clamped = (int64_t)c;
    if (device_error) *device_error = err;
    return DLX_OK;
}

int dlx_plan_set_timing(dlx_plan *p, int class_mask) {
    if (!p) return fail(DLX_ERR_INVALID_ARG, "plan is NULL");
    p->timing = (uint32_t)class_mask;
    return DLX_OK;
}

int dlx_plan_get_timing(dlx_plan *p, dlx_kernel_times *out) {
    if (!p || !out) return fail(DLX_ERR_INVALID_ARG, "NULL argument");
    DeviceGuard guard(p->device);
    DLX_CU(cudaDeviceSynchronize(), "synchronize");
    memset(out, 0, sizeof(*out));
    out->n_classes = dlx::KC_N;
    for (int c = 0; c < dlx::KC_N; ++c) {
        out->name[c] = dlx::kClassNames[c];
        out->launches[c] = p->launches[c];
        out->events[c] = p->events[c];
        out->total_launches += p->launches[c];
    }
    for (const auto &r : p->recs) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) out->ms[r.cls] += ms;
    }
    p->recs.clear();
    p->pool_next = 0;
    for (int c = 0; c < 16; ++c) p->launches[c] = p->events[c] = 0;
    return DLX_OK;
}

int dlx_adam(float *theta, const float *grad, float *m, float *v, size_t n, float lr, float beta1, float beta2,
             float eps, int t, void *stream) {
    if (n && (!theta || !grad || !m || !v)) return fail(DLX_ERR_INVALID_ARG, "NULL array");
    if (t < 1) return fail(DLX_ERR_INVALID_ARG, "Adam step t is 1-based");
    if (dlx::check_level() >= 1 && n) {
        int dev = 0, rc;
        cudaGetDevice(&dev);
        if ((rc = dlx::check_buffer(theta, 4 * n, 4, dev, "theta", false)) ||
            (rc = dlx::check_buffer(grad, 4 * n, 4, dev, "grad", false)) ||
            (rc = dlx::check_buffer(m, 4 * n, 4, dev, "m", false)) ||
            (rc = dlx::check_buffer(v, 4 * n, 4, dev, "v", false)))
            return rc;
    }
    DLX_CU(dlx::launch_adam(theta, grad, m, v, n, lr, beta1, beta2, eps, t, (cudaStream_t)stream), "adam");
    return DLX_OK;
}

}  // extern "C"
