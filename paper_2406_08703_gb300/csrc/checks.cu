// Checked mode of the dlx library and its test hook for the bounded waits.
//
// The kernels cannot run under a memory checker here, so the library checks its
// own calls.  Level 1 checks, before any launch, every device array an entry
// point will read or write: it must be device memory of the plan's device (or
// managed memory), aligned for its element type, and -- where the driver reports
// the allocation that holds it -- lie inside that allocation for the full size the
// plan's shapes imply.  Level 2 also synchronises the stream after each kernel
// class and turns an error there, or a raised device error flag (a bounded wait
// that expired), into the call's status, naming the class.
#include <cudaTypedefs.h>

#include <atomic>
#include <cstdlib>
#include <string>

#include "dlx_common.cuh"

namespace dlx {
namespace {

std::atomic<int> g_level{-1};

int level_from_env() {
    const char *e = std::getenv("DLX_CHECKS");
    if (!e || !*e) return 0;
    const int v = std::atoi(e);
    return v < 0 ? 0 : (v > 2 ? 2 : v);
}

PFN_cuMemGetAddressRange_v3020 range_fn() {
    // looked up once per process (thread-safe static initialisation)
    static const PFN_cuMemGetAddressRange_v3020 fn = []() -> PFN_cuMemGetAddressRange_v3020 {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuMemGetAddressRange", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            return (PFN_cuMemGetAddressRange_v3020)p;
        return nullptr;
    }();
    return fn;
}

}  // namespace

int check_level() {
    int v = g_level.load(std::memory_order_relaxed);
    if (v < 0) {
        int want = -1;
        v = level_from_env();
        g_level.compare_exchange_strong(want, v);
        v = g_level.load(std::memory_order_relaxed);
    }
    return v;
}

// One device array: NULL passes when `optional`; otherwise the checks of level 1.
int check_buffer(const void *ptr, size_t bytes, size_t align, int device, const char *name, bool optional) {
    if (!ptr) {
        if (optional) return DLX_OK;
        dlx_set_error(std::string(name) + " is NULL");
        return DLX_ERR_INVALID_ARG;
    }
    if ((uintptr_t)ptr % align) {
        dlx_set_error(std::string(name) + " is not " + std::to_string(align) + "-byte aligned");
        return DLX_ERR_INVALID_ARG;
    }
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
        cudaGetLastError();
        dlx_set_error(std::string(name) + " is not a CUDA pointer");
        return DLX_ERR_INVALID_ARG;
    }
    if (at.type == cudaMemoryTypeDevice) {
        if (at.device != device) {
            dlx_set_error(std::string(name) + " is memory of device " + std::to_string(at.device) + ", the call's is " +
                          std::to_string(device));
            return DLX_ERR_INVALID_ARG;
        }
    } else if (at.type != cudaMemoryTypeManaged) {
        dlx_set_error(std::string(name) + (at.type == cudaMemoryTypeHost ? " is host (pinned) memory"
                                                                         : " is not device memory"));
        return DLX_ERR_INVALID_ARG;
    }
    if (bytes == 0) return DLX_OK;
    if (PFN_cuMemGetAddressRange_v3020 fn = range_fn()) {
        CUdeviceptr base = 0;
        size_t size = 0;
        if (fn(&base, &size, (CUdeviceptr)(uintptr_t)ptr) == CUDA_SUCCESS) {
            const size_t have = (size_t)(base + size - (CUdeviceptr)(uintptr_t)ptr);
            if (bytes > have) {
                dlx_set_error(std::string(name) + ": " + std::to_string(bytes) + " bytes needed, " +
                              std::to_string(have) + " left in its allocation");
                return DLX_ERR_INVALID_ARG;
            }
        }
    }
    return DLX_OK;
}

// The arrays of dlx_params for plan p.
int check_params(const dlx_plan *p, const dlx_params *q) {
    const size_t f = sizeof(float), npx = (size_t)p->ni * p->ni, nimg = (size_t)p->ndi * p->ndi;
    const int dev = p->device;
    int rc;
    if ((rc = check_buffer(q->transmission, f * npx, 4, dev, "params.transmission", false))) return rc;
    if ((rc = check_buffer(q->opd_fixed, f * npx, 4, dev, "params.opd_fixed", true))) return rc;
    if ((rc = check_buffer(q->zern_basis, f * p->nz * npx, 4, dev, "params.zern_basis", p->nz == 0))) return rc;
    if ((rc = check_buffer(q->zern_coeff, f * p->nz, 4, dev, "params.zern_coeff", p->nz == 0))) return rc;
    if ((rc = check_buffer(q->opd_pix, f * npx, 4, dev, "params.opd_pix", true))) return rc;
    if ((rc = check_buffer(q->weights, f * p->nl, 4, dev, "params.weights", false))) return rc;
    if ((rc = check_buffer(q->flux, f * p->ns, 4, dev, "params.flux", false))) return rc;
    if ((rc = check_buffer(q->pos, 2 * f * p->ns, 4, dev, "params.pos", false))) return rc;
    if (!p->crop && (rc = check_buffer(q->dither, 2 * f * p->nei, 4, dev, "params.dither", true))) return rc;
    return check_buffer(q->flat, f * nimg, 4, dev, "params.flat", false);
}

// The arrays of dlx_grads (each may be NULL: not computed).
int check_grads(const dlx_plan *p, const dlx_grads *g, const char *what) {
    if (!g) return DLX_OK;
    const size_t f = sizeof(float);
    const std::string w(what);
    const int dev = p->device;
    int rc;
    if ((rc = check_buffer(g->d_zern, f * p->nz, 4, dev, (w + ".d_zern").c_str(), true))) return rc;
    if ((rc = check_buffer(g->d_opd_pix, f * p->ni * p->ni, 4, dev, (w + ".d_opd_pix").c_str(), true))) return rc;
    if ((rc = check_buffer(g->d_flat, f * p->ndi * p->ndi, 4, dev, (w + ".d_flat").c_str(), true))) return rc;
    if ((rc = check_buffer(g->d_flux, f * p->ns, 4, dev, (w + ".d_flux").c_str(), true))) return rc;
    return check_buffer(g->d_pos, 2 * f * p->ns, 4, dev, (w + ".d_pos").c_str(), true);
}

// Bytes of one image set [nei][ndi][ndi] of 4-byte elements.
size_t image_bytes(const dlx_plan *p) { return 4 * (size_t)p->nei * p->ndi * p->ndi; }

void class_check(dlx_plan *p, int cls, cudaStream_t st) {
    if (p->check_rc) return;  // the first failure of the call is the one reported
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        p->check_rc = DLX_ERR_CUDA;
        p->check_msg = std::string("kernel class ") + class_name(cls) + ": " + cudaGetErrorString(e);
        return;
    }
    int32_t err = 0;
    if (cudaMemcpy(&err, p->err, sizeof(err), cudaMemcpyDeviceToHost) == cudaSuccess && err != 0) {
        cudaMemset(p->err, 0, sizeof(err));  // reported through the call's status
        p->check_rc = DLX_ERR_TIMEOUT;
        p->check_msg = std::string("kernel class ") + class_name(cls) +
                       ": a device-side bounded wait expired (code " + std::to_string(err) + ")";
    }
}

// The status of a call after its launches: a level-2 failure replaces OK.
int checked_status(dlx_plan *p, int rc) {
    if (p->check_rc) {
        const int c = p->check_rc;
        if (rc == DLX_OK) {
            dlx_set_error(p->check_msg);
            rc = c;
        }
        p->check_rc = 0;
        p->check_msg.clear();
    }
    return rc;
}

}  // namespace dlx

extern "C" {

int dlx_set_checks(int level) {
    if (level < 0 || level > 2) {
        dlx_set_error("checks level must be 0, 1 or 2");
        return DLX_ERR_INVALID_ARG;
    }
    dlx::g_level.store(level);
    return DLX_OK;
}

int dlx_get_checks(void) { return dlx::check_level(); }

int dlx_check_buffer(const void *ptr, size_t bytes, int device) {
    return dlx::check_buffer(ptr, bytes, 4, device, "buffer", false);
}

int dlx_check_loss_grad_args(dlx_plan *p, const dlx_params *prm, const int32_t *data, const double *loss,
                             const dlx_grads *g, const float *model_opt) {
    if (!p || !prm) {
        dlx_set_error("plan/params is NULL");
        return DLX_ERR_INVALID_ARG;
    }
    int rc;
    if ((rc = dlx::check_params(p, prm))) return rc;
    if ((rc = dlx::check_buffer(data, dlx::image_bytes(p), 4, p->device, "data", false))) return rc;
    if ((rc = dlx::check_buffer(loss, sizeof(double), 8, p->device, "loss", false))) return rc;
    if ((rc = dlx::check_grads(p, g, "grads"))) return rc;
    return dlx::check_buffer(model_opt, dlx::image_bytes(p), 4, p->device, "model", true);
}

int dlx_plan_inject_fault(dlx_plan *p, int kind) {
    if (!p) {
        dlx_set_error("plan is NULL");
        return DLX_ERR_INVALID_ARG;
    }
    if (kind != 1 || p->prec == DLX_FP32_SIMT) {
        dlx_set_error("kind 1 (a withheld operand copy) on a tensor-core plan is the only fault");
        return DLX_ERR_INVALID_ARG;
    }
    p->inject = kind;
    return DLX_OK;
}

}  // extern "C"
