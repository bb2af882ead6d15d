// dlx_forward_noalloc: the forward model of a small optical model, computed
// without allocating any device memory.
//
// Some callers cannot call cudaMalloc: a host application that reserves all
// of the GPU's memory through its own allocator at start-up and forbids any
// further allocation while it runs (for example an instrument-control or
// real-time data-reduction loop that must never stall or fail on an
// allocation).  They can still pass their own input and output buffers.  This
// entry point takes its working memory -- MFT matrices, phasors, first-stage
// products, intensity planes, reduction partials -- from one file-scope device
// array of fixed size that every GPU loading the library holds until the
// process exits, and runs the same kernels as dlx_forward in the FP32
// CUDA-core form.
#include <cmath>
#include <cstring>

#include "dlx_common.cuh"

namespace {

constexpr size_t kNoAllocScratchBytes = 16u << 20;  // 16 MiB per GPU
constexpr int kMaxLambdas = 256;

// Working memory shared by every call on a device.  In host code this name is
// only a stand-in for the device symbol; its device address comes from
// cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of the scratch array on the current device, looked up on every
// call (a lookup is cheap, and a cached address would go stale if the device's
// context were reset and the array reloaded elsewhere).
int scratch_address(void **out) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
        dlx_set_error(std::string("cudaGetSymbolAddress of the no-allocation scratch failed: ") +
                      cudaGetErrorString(e));
        return DLX_ERR_CUDA;
    }
    *out = p;
    return DLX_OK;
}

// The wavelength tables travel as a kernel argument (by value), so the call copies
// nothing from host memory with cudaMemcpy.
struct LamTable {
    double lam[kMaxLambdas];
    int n;
};

// lam_d[l] = lambda_l, invlam[l] = 1/lambda_l rounded to float (as a plan stores them),
// and the reset of the normalisation's block counter.
__global__ void k_noalloc_tables(const LamTable t, double *lam_d, float *invlam, unsigned int *ncount) {
    const int l = threadIdx.x;
    if (l < t.n) {
        lam_d[l] = t.lam[l];
        invlam[l] = (float)(1.0 / t.lam[l]);
    }
    if (l == 0) *ncount = 0u;
}

// Bump layout inside the scratch array, 256-byte aligned regions.
struct Carve {
    char *base;
    size_t off = 0;
    template <class T>
    T *take(size_t n) {
        off = (off + 255) / 256 * 256;
        T *p = (T *)(base + off);
        off += n * sizeof(T);
        return p;
    }
};

}  // namespace

extern "C" int dlx_forward_noalloc(const dlx_mft_desc *d, const dlx_params *prm, float *model, void *stream) {
    if (!d || !prm || !model) {
        dlx_set_error("desc, params and model are required");
        return DLX_ERR_INVALID_ARG;
    }
    // the plan's own checks: sizes, ranges, wavelengths, Fresnel terms
    if (int rc = dlx::check_desc(d, nullptr)) return rc;
    if (!prm->transmission || !prm->weights || !prm->flux || !prm->pos || !prm->flat ||
        (d->n_zern > 0 && (!prm->zern_basis || !prm->zern_coeff))) {
        dlx_set_error("transmission, weights, flux, pos, flat (and the Zernike arrays when n_zern > 0) are required");
        return DLX_ERR_INVALID_ARG;
    }
    if (d->dither_px) {
        dlx_set_error("dlx_forward_noalloc: integer-pixel dither windows (dither_px) need a plan");
        return DLX_ERR_UNSUPPORTED;
    }
    // the scratch holds at least 8 * Ni * Ni8 bytes of phasor per PSF, so more than 2^17 PSFs never fit
    const long long B_ll = (long long)d->n_lambda * d->n_src * d->n_exp;
    if (d->n_lambda > kMaxLambdas || B_ll > (1LL << 17)) {
        dlx_set_error("dlx_forward_noalloc: at most 256 wavelengths and 2^17 PSFs, and the working memory must fit "
                      "the fixed 16 MiB scratch");
        return DLX_ERR_RANGE;
    }

    // a plan that only points into the scratch array (no member allocates)
    dlx_plan p;
    p.desc = *d;
    p.R_max = 1;
    p.ni = d->n_pupil;
    p.nd = d->n_det;
    p.os = d->oversample;
    p.no = d->n_det * d->oversample;
    p.nl = d->n_lambda;
    p.ns = d->n_src;
    p.ne = d->n_exp;
    p.nz = d->n_zern;
    p.ndi = p.nd;
    p.nei = p.ne;
    p.nse = p.ns * p.ne;
    p.B = p.nl * p.nse;
    p.ldi = (p.ni + 7) / 8 * 8;
    p.ldo = (p.no + 7) / 8 * 8;
    p.prec = DLX_FP32_SIMT;
    p.fmt = dlx::FMT_F32;
    p.planes = 2;
    p.esz = 4;
    p.dx = d->diameter_m / p.ni;
    double du_scale;
    dlx::fresnel_terms(d, &du_scale, &p.chirp);
    p.du = d->pixscale_rad / p.os * du_scale;
    p.G = 1;
    p.chunk = 1;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        dlx_set_error("cudaGetDevice failed");
        return DLX_ERR_CUDA;
    }
    p.device = dev;
    if (cudaDeviceGetAttribute(&p.sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        dlx_set_error("cudaDeviceGetAttribute failed");
        return DLX_ERR_CUDA;
    }
    if (dlx::check_level() >= 1) {
        // checked mode: every array is device memory of this device, aligned, and large enough
        int rc = dlx::check_params(&p, prm);
        if (!rc) rc = dlx::check_buffer(model, sizeof(float) * (size_t)p.ne * p.nd * p.nd, 4, dev, "model", false);
        if (rc) return rc;
    }
    const size_t np = (size_t)p.nd * p.nd, nq = (size_t)p.no * p.no, npx = (size_t)p.ni * p.ni;
    p.red_blocks = std::max(1, std::min((int)((np + 255) / 256), p.sm_count * 2));
    // more than 8 sources: the model pass of the two-pass binning (no loss, no partials)
    p.bin_a_blocks = std::max(1, std::min((int)((np + 255) / 256), p.sm_count * 8));

    // bytes this call needs, with the same carve as below (alignment included)
    Carve need{nullptr};
    need.take<double>(p.nl);
    need.take<float>(p.nl);
    need.take<float>(p.nl);
    need.take<float>(2);
    need.take<float>(dlx::kNormParts);
    need.take<float2>((size_t)p.B * 2 * p.ni);
    need.take<float>(npx);
    need.take<float>((size_t)p.nl * 2 * p.no * p.ldi);
    need.take<float>((size_t)p.nl * 2 * p.ni * p.ldo);
    need.take<float>((size_t)p.B * 2 * p.ni * p.ldi);
    need.take<float>((size_t)p.B * 2 * p.no * p.ldi);
    need.take<float>((size_t)p.nse * nq);
    need.take<double>((size_t)p.red_blocks * (1 + dlx::kMaxSrc));
    need.take<unsigned long long>(1);
    need.take<float2>(dlx::kNormParts);
    need.take<unsigned int>(1);
    if (need.off > kNoAllocScratchBytes) {
        dlx_set_error("dlx_forward_noalloc: this shape needs " + std::to_string(need.off) +
                      " bytes of working memory, above the fixed 16 MiB scratch; use dlx_make_mft + dlx_forward");
        return DLX_ERR_RANGE;
    }

    void *base = nullptr;
    int rc = scratch_address(&base);
    if (rc) return rc;
    Carve c{(char *)base};
    p.lam_d = c.take<double>(p.nl);
    p.invlam = c.take<float>(p.nl);
    p.wnorm = c.take<float>(p.nl);
    p.pscale = c.take<float>(2);
    p.tpart = c.take<float>(dlx::kNormParts);
    p.tilt = c.take<float2>((size_t)p.B * 2 * p.ni);
    p.opd = c.take<float>(npx);
    p.amat.ptr = c.take<float>((size_t)p.nl * 2 * p.no * p.ldi);
    p.amatH.ptr = c.take<float>((size_t)p.nl * 2 * p.ni * p.ldo);
    p.P.ptr = c.take<float>((size_t)p.B * 2 * p.ni * p.ldi);
    p.T1t.ptr = c.take<float>((size_t)p.B * 2 * p.no * p.ldi);
    p.Is = c.take<float>((size_t)p.nse * nq);
    p.red = c.take<double>((size_t)p.red_blocks * (1 + dlx::kMaxSrc));
    p.clamped = c.take<unsigned long long>(1);
    p.npart = c.take<float2>(dlx::kNormParts);
    p.ncount = c.take<unsigned int>(1);

    // The FP32 contractions read operands only inside their true extents and every
    // region above is written before it is read in this call, so nothing has to be
    // cleared; the tables below are rewritten on every call because another call
    // may have left a different shape in the array.
    cudaStream_t st = (cudaStream_t)stream;
    LamTable tab{};
    tab.n = p.nl;
    for (int l = 0; l < p.nl; ++l) tab.lam[l] = d->lambda_m[l];
    k_noalloc_tables<<<1, kMaxLambdas, 0, st>>>(tab, p.lam_d, p.invlam, p.ncount);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = dlx::launch_mft_matrices(&p, st);
    if (e != cudaSuccess) {
        dlx_set_error(std::string("dlx_forward_noalloc: ") + cudaGetErrorString(e));
        return DLX_ERR_CUDA;
    }
    dlx::DevParams dp{};
    dp.p[dlx::PT] = prm->transmission;
    dp.p[dlx::POPDF] = prm->opd_fixed;
    dp.p[dlx::PBASIS] = prm->zern_basis;
    dp.p[dlx::PCOEFF] = prm->zern_coeff;
    dp.p[dlx::POPDPIX] = prm->opd_pix;
    dp.p[dlx::PW] = prm->weights;
    dp.p[dlx::PFLUX] = prm->flux;
    dp.p[dlx::PPOS] = prm->pos;
    dp.p[dlx::PDITHER] = prm->dither;
    dp.p[dlx::PFLAT] = prm->flat;
    rc = dlx::eval_forward(&p, dp, 1, st);
    if (rc) return rc;
    e = dlx::launch_bin_nll(&p, dp, 1, nullptr, 0, model, 0, nullptr, nullptr, st);
    if (e != cudaSuccess) {
        dlx_set_error(std::string("dlx_forward_noalloc: ") + cudaGetErrorString(e));
        return DLX_ERR_CUDA;
    }
    return DLX_OK;
}
