// Continuous-batching fit server (dlx_server_create / dlx_submit / dlx_poll).
//
// Requests are fits of the optical model (K Adam steps of loss + gradient, or a
// single evaluation).  A scheduler thread owns the device work:
//   * admission: queued requests are admitted, in arrival order, as slots and
//     HBM budget free up; a request's fixed inputs, parameters, Adam state and
//     data stay resident on the device until it finishes;
//   * buckets: requests with the same shape, wavelength set and precision share
//     a bucket -- one plan with R_max slots -- so one grouped launch per kernel
//     advances every active slot of the bucket by one step; each bucket has its
//     own stream, so different buckets' work overlaps on the device;
//   * CUDA graphs: the step of a bucket with R active slots (prologue, the MFT
//     contractions, binning/NLL, adjoint, reductions, Adam) is captured once per
//     R and replayed;
//   * slots are kept contiguous: a finished slot is refilled by moving the
//     bucket's last active slot into it (device-to-device copies), so a launch
//     always covers slots [0, R).
// Every per-slot reduction in the kernels has a fixed order, so a request's
// results do not depend on which other requests share its launches.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "dlx_common.cuh"

namespace {

using clk = std::chrono::steady_clock;

double secs(clk::time_point a, clk::time_point b) { return std::chrono::duration<double>(b - a).count(); }

struct Bucket;

struct Req {
    uint64_t ticket = 0;
    dlx_mft_desc desc{};
    std::vector<double> lambdas;
    std::vector<int32_t> dither_px;  // integer-pixel dithers (windows), or empty
    bool has_pix = false;
    std::vector<float> T, opd_fixed, basis, weights, dither, coeff, pix, flux, pos, flat;
    std::vector<int32_t> data;
    int n_steps = 0;
    float lr[5] = {0, 0, 0, 0, 0};
    std::vector<float> m_in, v_in;  // resume state (empty = zeros)
    int step_in = 0;
    clk::time_point t_submit, t_admit, t_done;
    int status = DLX_PENDING;
    bool done = false;
    int steps_done = 0;
    Bucket *bucket = nullptr;
    int slot = -1;
    // results (copied out of the bucket, which may be released before the poll)
    double loss = 0;
    std::vector<float> theta_out, grad_out, m_out, v_out;
    int off[6] = {0};
};

__global__ void k_step_inc(int *step, int R) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < R) step[r] += 1;
}

struct Bucket {
    std::string key;
    dlx_plan *plan = nullptr;
    int cap = 0, active = 0;
    int ni = 0, nd = 0, nl = 0, ns = 0, ne = 0, nz = 0;
    bool has_pix = false;
    size_t n_theta = 0, bytes = 0;
    int off[6] = {0};  // parameter groups: zern, opd_pix, flat, flux, pos, end
    cudaStream_t stream = nullptr;
    // slot-major device arrays
    float *T = nullptr, *opd_fixed = nullptr, *basis = nullptr, *weights = nullptr, *dither = nullptr;
    float *theta = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr, *lr = nullptr;
    int32_t *data = nullptr;
    double *loss = nullptr;
    int *step = nullptr, *off_d = nullptr;
    std::vector<Req *> slot_req;
    std::map<int, cudaGraphExec_t> graphs;
    std::vector<void *> allocs;
    uint64_t launches = 0;

    size_t sz_T() const { return (size_t)ni * ni; }
    size_t sz_basis() const { return (size_t)nz * ni * ni; }
    size_t sz_data() const { return (size_t)ne * nd * nd; }

    dlx::DevParams params() const {
        dlx::DevParams d{};
        d.p[dlx::PT] = T;
        d.s[dlx::PT] = sz_T();
        d.p[dlx::POPDF] = opd_fixed;
        d.s[dlx::POPDF] = sz_T();
        d.p[dlx::PBASIS] = nz ? basis : nullptr;
        d.s[dlx::PBASIS] = sz_basis();
        d.p[dlx::PCOEFF] = nz ? theta + off[0] : nullptr;
        d.s[dlx::PCOEFF] = n_theta;
        d.p[dlx::POPDPIX] = has_pix ? theta + off[1] : nullptr;
        d.s[dlx::POPDPIX] = n_theta;
        d.p[dlx::PW] = weights;
        d.s[dlx::PW] = nl;
        d.p[dlx::PFLUX] = theta + off[3];
        d.s[dlx::PFLUX] = n_theta;
        d.p[dlx::PPOS] = theta + off[4];
        d.s[dlx::PPOS] = n_theta;
        d.p[dlx::PDITHER] = (plan && plan->crop) ? nullptr : dither;  // windows read no dither angles
        d.s[dlx::PDITHER] = 2 * (size_t)ne;
        d.p[dlx::PFLAT] = theta + off[2];
        d.s[dlx::PFLAT] = n_theta;
        return d;
    }
    dlx::DevGrads grads() const {
        dlx::DevGrads g{};
        g.p[dlx::GZERN] = nz ? grad + off[0] : nullptr;
        // the pixel-OPD gradient has a slot region only when the map is fitted (the
        // Zernike gradient is reduced from the plan's own g_OPD buffer either way)
        g.p[dlx::GPIX] = has_pix ? grad + off[1] : nullptr;
        g.p[dlx::GFLAT] = grad + off[2];
        g.p[dlx::GFLUX] = grad + off[3];
        g.p[dlx::GPOS] = grad + off[4];
        for (int k = 0; k < dlx::NGRAD; ++k) g.s[k] = n_theta;
        return g;
    }
};

}  // namespace

struct dlx_server {
    int device = 0;
    size_t budget = 0, in_use = 0;
    int max_slots = 1;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    bool stop = false;
    std::thread worker;
    uint64_t next_ticket = 1;
    std::unordered_map<uint64_t, std::unique_ptr<Req>> reqs;
    std::deque<Req *> queue;
    std::map<std::string, std::unique_ptr<Bucket>> buckets;
    dlx_server_stats stats{};
    int fault_next = 0;
};

namespace {

int fail(int code, const std::string &msg) {
    dlx_set_error(msg);
    return code;
}

std::string bucket_key(const Req &r) {
    std::string k;
    auto put = [&](const void *p, size_t n) { k.append((const char *)p, n); };
    const dlx_mft_desc &d = r.desc;
    put(&d.n_pupil, sizeof(int));
    put(&d.diameter_m, sizeof(double));
    put(&d.n_det, sizeof(int));
    put(&d.pixscale_rad, sizeof(double));
    put(&d.oversample, sizeof(int));
    put(&d.n_src, sizeof(int));
    put(&d.n_exp, sizeof(int));
    put(&d.n_zern, sizeof(int));
    put(&d.precision, sizeof(int));
    int hp = r.has_pix;
    put(&hp, sizeof(int));
    put(&d.prf_prior_sigma, sizeof(double));  // the plan's loss
    put(&d.focal_length_m, sizeof(double));    // Fresnel regime
    put(&d.focal_shift_m, sizeof(double));
    put(r.lambdas.data(), r.lambdas.size() * sizeof(double));
    const int nwin = (int)r.dither_px.size();
    put(&nwin, sizeof(int));
    put(r.dither_px.data(), r.dither_px.size() * sizeof(int32_t));
    return k;
}

size_t theta_size(const dlx_mft_desc &d, bool has_pix) {
    return (size_t)d.n_zern + (has_pix ? (size_t)d.n_pupil * d.n_pupil : 0) + (size_t)d.n_det * d.n_det +
           (size_t)d.n_src * 3;
}

// Device bytes of a bucket with `cap` slots: plan workspaces, operands, inputs,
// parameters, gradient and Adam state.  The same arithmetic as make_plan's
// allocations, used for admission before anything is allocated.
size_t bucket_bytes(const dlx_mft_desc &d, bool has_pix, int cap) {
    // integer-dither windows: the MFT runs once per source on a detector wider by 2 max|dither|
    size_t delta = 0;
    if (d.dither_px)
        for (int k = 0; k < 2 * d.n_exp; ++k) delta = std::max<size_t>(delta, (size_t)std::abs(d.dither_px[k]));
    const size_t ne_mft = d.dither_px ? 1 : (size_t)d.n_exp;
    const size_t ni = d.n_pupil, nd = d.n_det, no = ((size_t)d.n_det + 2 * delta) * d.oversample, nl = d.n_lambda;
    const size_t ldi = dlx::operand_ld((int)ni), ldo = dlx::operand_ld((int)no), B = nl * d.n_src * ne_mft, Bt = B * cap;
    const int fmt = dlx::fmt_of_prec(d.precision);
    const size_t pe = (size_t)dlx::fmt_planes(fmt) * dlx::fmt_esize(fmt);
    size_t b = pe * (nl * no * ldi + nl * ni * ldo + Bt * ni * ldi + Bt * no * ldi + Bt * no * ldo + Bt * ni * ldo);
    b += 4 * (Bt * ni * ni) + 8 * (Bt * 2 * ni) + 4 * (size_t)d.n_src * ne_mft * cap * no * no * 2;
    // the mirror-paired forward of the FP16 split form: the paired phasor, and first-stage rows of
    // ldk instead of ldi columns
    if (fmt == dlx::FMT_F16X4) {
        const size_t hp = (size_t)dlx::pair_half((int)ni), ldk = dlx::operand_ld((int)(2 * hp));
        b += pe * (Bt * 2 * hp * ldk + Bt * no * (ldk > ldi ? ldk - ldi : 0));
    }
    // the fields stage 2 keeps for the adjoint (the bucket's plan takes every PSF in one chunk)
    if (dlx::field_kept(fmt, d.precision == DLX_BF16X3SA, (int)ni, (int)Bt, (int)Bt))
        b += 8 * Bt * no * ldo + 4 * (size_t)cap * ne_mft * (no / d.oversample) * (no / d.oversample);
    b += 16 * (size_t)cap * ni * ni + 8 * (size_t)cap * d.n_exp * nd * nd;
    if (d.dither_px) b += 4 * (size_t)cap * (d.n_exp * nd * nd + 2 * (no / d.oversample) * (no / d.oversample));
    const size_t nth = theta_size(d, has_pix);
    b += (size_t)cap * 4 * (ni * ni * (1 + 1 + d.n_zern) + nl + 2 * d.n_exp + d.n_exp * nd * nd + 4 * nth + 5);
    return b + (64u << 20);  // reduction partials, tables, allocator rounding
}

template <class T>
cudaError_t balloc(Bucket *b, T **p, size_t n) {
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, std::max<size_t>(n, 1) * sizeof(T));
    if (e == cudaSuccess) {
        b->allocs.push_back(q);
        *p = (T *)q;
        cudaMemset(q, 0, std::max<size_t>(n, 1) * sizeof(T));
    }
    return e;
}

void destroy_bucket(Bucket *b) {
    if (b->stream) cudaStreamSynchronize(b->stream);
    for (auto &kv : b->graphs) cudaGraphExecDestroy(kv.second);
    b->graphs.clear();
    for (void *q : b->allocs) cudaFree(q);
    b->allocs.clear();
    if (b->plan) dlx_destroy_plan(b->plan);
    if (b->stream) cudaStreamDestroy(b->stream);
}

int create_bucket(dlx_server *s, const Req &r, Bucket **out) {
    auto b = std::make_unique<Bucket>();
    const dlx_mft_desc &d = r.desc;
    b->key = bucket_key(r);
    b->ni = d.n_pupil;
    b->nd = d.n_det;
    b->nl = d.n_lambda;
    b->ns = d.n_src;
    b->ne = d.n_exp;
    b->nz = d.n_zern;
    b->has_pix = r.has_pix;
    // slots: as many as the budget share of one bucket allows, up to max_slots
    const size_t one = bucket_bytes(d, r.has_pix, 1), two = bucket_bytes(d, r.has_pix, 2);
    const size_t per = two > one ? two - one : one;
    const size_t free_budget = s->budget > s->in_use ? s->budget - s->in_use : 0;
    int cap = (int)std::min<size_t>(s->max_slots, free_budget > one ? 1 + (free_budget - one) / per : 1);
    cap = std::max(1, std::min(cap, s->max_slots));
    b->cap = cap;
    b->bytes = bucket_bytes(d, r.has_pix, cap);
    if (b->bytes > free_budget) return DLX_ERR_NOMEM;
    dlx_mft_desc pd = d;
    pd.lambda_m = r.lambdas.data();
    pd.dither_px = r.dither_px.empty() ? nullptr : r.dither_px.data();
    pd.psf_chunk = 0;
    pd.workspace_limit_bytes = 0;
    int rc = dlx::make_plan(&pd, s->device, cap, &b->plan);
    if (rc) return rc;
    const size_t nth = theta_size(d, r.has_pix);
    b->n_theta = nth;
    b->off[0] = 0;
    b->off[1] = d.n_zern;
    b->off[2] = b->off[1] + (r.has_pix ? d.n_pupil * d.n_pupil : 0);
    b->off[3] = b->off[2] + d.n_det * d.n_det;
    b->off[4] = b->off[3] + d.n_src;
    b->off[5] = b->off[4] + 2 * d.n_src;
    cudaError_t e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = balloc(b.get(), &b->T, cap * b->sz_T());
    if (e == cudaSuccess) e = balloc(b.get(), &b->opd_fixed, cap * b->sz_T());
    if (e == cudaSuccess) e = balloc(b.get(), &b->basis, cap * b->sz_basis());
    if (e == cudaSuccess) e = balloc(b.get(), &b->weights, (size_t)cap * b->nl);
    if (e == cudaSuccess) e = balloc(b.get(), &b->dither, (size_t)cap * 2 * b->ne);
    if (e == cudaSuccess) e = balloc(b.get(), &b->theta, cap * nth);
    if (e == cudaSuccess) e = balloc(b.get(), &b->grad, cap * nth);
    if (e == cudaSuccess) e = balloc(b.get(), &b->m, cap * nth);
    if (e == cudaSuccess) e = balloc(b.get(), &b->v, cap * nth);
    if (e == cudaSuccess) e = balloc(b.get(), &b->lr, (size_t)cap * 5);
    if (e == cudaSuccess) e = balloc(b.get(), &b->data, cap * b->sz_data());
    if (e == cudaSuccess) e = balloc(b.get(), &b->loss, (size_t)cap);
    if (e == cudaSuccess) e = balloc(b.get(), &b->step, (size_t)cap);
    if (e == cudaSuccess) e = balloc(b.get(), &b->off_d, 6);
    if (e == cudaSuccess) e = cudaMemcpy(b->off_d, b->off, sizeof(b->off), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        destroy_bucket(b.get());
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? DLX_ERR_NOMEM : DLX_ERR_CUDA;
    }
    b->slot_req.assign(cap, nullptr);
    s->in_use += b->bytes;
    *out = b.get();
    s->buckets[b->key] = std::move(b);
    return DLX_OK;
}

// Upload a request's inputs into slot `r` of its bucket on the bucket stream; returns the
// first CUDA error of the copies (the slot is then not used).
cudaError_t upload(Bucket *b, int r, Req *q, bool poison) {
    cudaStream_t st = b->stream;
    cudaError_t err = cudaSuccess;
    auto keep = [&](cudaError_t e) {
        if (err == cudaSuccess) err = e;
    };
    auto h2d = [&](void *dst, const void *src, size_t bytes) {
        if (bytes) keep(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st));
    };
    h2d(b->T + r * b->sz_T(), q->T.data(), 4 * b->sz_T());
    if (!q->opd_fixed.empty()) h2d(b->opd_fixed + r * b->sz_T(), q->opd_fixed.data(), 4 * b->sz_T());
    else keep(cudaMemsetAsync(b->opd_fixed + r * b->sz_T(), 0, 4 * b->sz_T(), st));
    if (b->nz) h2d(b->basis + r * b->sz_basis(), q->basis.data(), 4 * b->sz_basis());
    h2d(b->weights + (size_t)r * b->nl, q->weights.data(), 4 * b->nl);
    if (!q->dither.empty()) h2d(b->dither + (size_t)r * 2 * b->ne, q->dither.data(), 8 * b->ne);
    else keep(cudaMemsetAsync(b->dither + (size_t)r * 2 * b->ne, 0, 8 * b->ne, st));
    std::vector<float> th(b->n_theta, 0.f);
    std::copy(q->coeff.begin(), q->coeff.end(), th.begin() + b->off[0]);
    if (b->has_pix) std::copy(q->pix.begin(), q->pix.end(), th.begin() + b->off[1]);
    std::copy(q->flat.begin(), q->flat.end(), th.begin() + b->off[2]);
    std::copy(q->flux.begin(), q->flux.end(), th.begin() + b->off[3]);
    std::copy(q->pos.begin(), q->pos.end(), th.begin() + b->off[4]);
    if (poison) th[b->off[3]] = NAN;  // host-side fault injection: a bad input, no device fault
    h2d(b->theta + r * b->n_theta, th.data(), 4 * b->n_theta);
    keep(cudaStreamSynchronize(st));  // th is a local buffer
    if (!q->m_in.empty()) h2d(b->m + r * b->n_theta, q->m_in.data(), 4 * b->n_theta);
    else keep(cudaMemsetAsync(b->m + r * b->n_theta, 0, 4 * b->n_theta, st));
    if (!q->v_in.empty()) h2d(b->v + r * b->n_theta, q->v_in.data(), 4 * b->n_theta);
    else keep(cudaMemsetAsync(b->v + r * b->n_theta, 0, 4 * b->n_theta, st));
    h2d(b->step + r, &q->step_in, sizeof(int));
    float lr[5];
    for (int k = 0; k < 5; ++k) lr[k] = q->n_steps > 0 ? q->lr[k] : 0.f;
    if (!b->has_pix) lr[1] = 0.f;
    h2d(b->lr + 5 * r, lr, sizeof(lr));
    h2d(b->data + r * b->sz_data(), q->data.data(), 4 * b->sz_data());
    keep(cudaStreamSynchronize(st));
    return err;
}

// Move slot `from` into slot `to` (device-to-device), keeping slots contiguous.
void move_slot(Bucket *b, int from, int to) {
    cudaStream_t st = b->stream;
    auto d2d = [&](void *base, size_t elems, size_t es) {
        cudaMemcpyAsync((char *)base + to * elems * es, (char *)base + from * elems * es, elems * es,
                        cudaMemcpyDeviceToDevice, st);
    };
    d2d(b->T, b->sz_T(), 4);
    d2d(b->opd_fixed, b->sz_T(), 4);
    if (b->nz) d2d(b->basis, b->sz_basis(), 4);
    d2d(b->weights, b->nl, 4);
    d2d(b->dither, 2 * b->ne, 4);
    d2d(b->theta, b->n_theta, 4);
    d2d(b->grad, b->n_theta, 4);
    d2d(b->m, b->n_theta, 4);
    d2d(b->v, b->n_theta, 4);
    d2d(b->lr, 5, 4);
    d2d(b->data, b->sz_data(), 4);
    d2d(b->loss, 1, 8);
    d2d(b->step, 1, 4);
    b->slot_req[to] = b->slot_req[from];
    b->slot_req[to]->slot = to;
    b->slot_req[from] = nullptr;
}

// Issue one step of a bucket with R active slots on its stream.
int issue_step(Bucket *b, int R) {
    const dlx::DevParams prm = b->params();
    const dlx::DevGrads g = b->grads();
    int rc = dlx::eval_loss_grad(b->plan, prm, R, b->data, b->sz_data(), b->loss, &g, nullptr, 0, b->stream);
    rc = dlx::checked_status(b->plan, rc);  // checked mode, level 2 (eager steps only)
    if (rc) return rc;
    k_step_inc<<<(R + 127) / 128, 128, 0, b->stream>>>(b->step, R);
    cudaError_t e = dlx::launch_adam_slots(b->theta, b->grad, b->m, b->v, b->n_theta, R, b->off_d, b->lr, b->step,
                                           0.9f, 0.999f, 1e-8f, b->stream);
    return e == cudaSuccess ? DLX_OK : DLX_ERR_CUDA;
}

// One step through a captured graph (captured on the first use of each R after
// an eager warm-up step).
int run_step(dlx_server *s, Bucket *b) {
    const int R = b->active;
    auto it = b->graphs.find(R);
    if (it == b->graphs.end()) {
        int rc = issue_step(b, R);  // eager: sets kernel attributes, warms the plan
        if (rc) return rc;
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        // the graph replays the same step (restart the step counters it advanced)
        if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
            int rc2 = issue_step(b, R);
            cudaError_t e = cudaStreamEndCapture(b->stream, &graph);
            if (rc2 == DLX_OK && e == cudaSuccess && cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess)
                b->graphs[R] = exec;
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
        }
        return DLX_OK;
    }
    cudaError_t e = cudaGraphLaunch(it->second, b->stream);
    s->stats.graph_launches++;
    return e == cudaSuccess ? DLX_OK : DLX_ERR_CUDA;
}

void finish(dlx_server *s, Req *q, int status) {
    q->status = status;
    q->done = true;
    q->t_done = clk::now();
    if (status == DLX_OK) s->stats.completed++;
}

void worker_loop(dlx_server *s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (!s->stop) {
        // ---- admission, in arrival order, as slots and budget allow
        for (auto it = s->queue.begin(); it != s->queue.end();) {
            Req *q = *it;
            if (s->fault_next == 1) {
                s->fault_next = 0;
                finish(s, q, DLX_ERR_NOMEM);
                s->stats.rejected++;
                it = s->queue.erase(it);
                continue;
            }
            const std::string key = bucket_key(*q);
            Bucket *b = nullptr;
            auto bi = s->buckets.find(key);
            if (bi != s->buckets.end()) b = bi->second.get();
            if (!b) {
                // keep idle buckets (their plans and graphs) cached; free them only when
                // the new bucket would not fit in the budget otherwise
                int rc = create_bucket(s, *q, &b);
                if (rc == DLX_ERR_NOMEM) {
                    bool freed = false;
                    for (auto e = s->buckets.begin(); e != s->buckets.end();) {
                        if (e->second->active == 0) {
                            s->in_use -= e->second->bytes;
                            destroy_bucket(e->second.get());
                            e = s->buckets.erase(e);
                            freed = true;
                        } else {
                            ++e;
                        }
                    }
                    if (freed) rc = create_bucket(s, *q, &b);
                }
                if (rc == DLX_ERR_NOMEM) {
                    ++it;  // wait for memory to free up
                    continue;
                }
                if (rc) {
                    finish(s, q, rc);
                    s->stats.rejected++;
                    it = s->queue.erase(it);
                    continue;
                }
            }
            if (b->active >= b->cap) {
                ++it;
                continue;
            }
            for (int k = 0; k < b->active; ++k)
                if (b->slot_req[k] && b->slot_req[k]->steps_done > 0) {
                    s->stats.midflight_admits++;
                    break;
                }
            const int r = b->active++;
            b->slot_req[r] = q;
            q->bucket = b;
            q->slot = r;
            q->t_admit = clk::now();
            const bool poison = s->fault_next == 2;
            if (poison) s->fault_next = 0;
            lk.unlock();
            const cudaError_t ue = upload(b, r, q, poison);
            lk.lock();
            it = s->queue.erase(it);
            if (ue != cudaSuccess) {  // the slot (the last one) is given back unused
                cudaGetLastError();
                b->slot_req[r] = nullptr;
                b->active--;
                finish(s, q, DLX_ERR_CUDA);
                continue;
            }
            s->stats.admitted++;
        }
        int active = 0;
        for (auto &kv : s->buckets) active += kv.second->active;
        s->stats.active = active;
        s->stats.queued = (int)s->queue.size();
        if (active == 0) {
            s->cv_work.wait_for(lk, std::chrono::milliseconds(50));
            continue;
        }
        // ---- one step of every active bucket (each on its own stream), then collect
        std::vector<Bucket *> live;
        for (auto &kv : s->buckets)
            if (kv.second->active > 0) live.push_back(kv.second.get());
        lk.unlock();
        std::vector<int> rcs(live.size());
        for (size_t i = 0; i < live.size(); ++i) rcs[i] = run_step(s, live[i]);
        std::vector<std::vector<double>> losses(live.size());
        for (size_t i = 0; i < live.size(); ++i) {
            Bucket *b = live[i];
            losses[i].resize(b->active);
            cudaMemcpyAsync(losses[i].data(), b->loss, 8 * b->active, cudaMemcpyDeviceToHost, b->stream);
        }
        for (Bucket *b : live) cudaStreamSynchronize(b->stream);
        int32_t derr = 0;
        lk.lock();
        for (size_t i = 0; i < live.size(); ++i) {
            Bucket *b = live[i];
            cudaError_t ce = cudaGetLastError();
            int32_t e = 0;
            cudaMemcpy(&e, b->plan->err, 4, cudaMemcpyDeviceToHost);
            derr |= e;
            s->stats.evals += b->active;
            if (b->active > 1) s->stats.grouped_launches++;
            for (int r = b->active - 1; r >= 0; --r) {
                Req *q = b->slot_req[r];
                q->steps_done++;
                int status = DLX_OK;
                if (rcs[i] != DLX_OK || ce != cudaSuccess) status = DLX_ERR_CUDA;
                else if (e) status = DLX_ERR_TIMEOUT;
                else if (!std::isfinite(losses[i][r])) status = DLX_ERR_NONFINITE;
                const int need = std::max(1, q->n_steps);
                if (status != DLX_OK || q->steps_done >= need) {
                    if (status == DLX_OK) {
                        q->loss = losses[i][r];
                        memcpy(q->off, b->off, sizeof(q->off));
                        // parameters, gradient and Adam moments of the slot to the request
                        const size_t o = r * b->n_theta, nb = 4 * b->n_theta;
                        std::vector<float> *dst[4] = {&q->theta_out, &q->grad_out, &q->m_out, &q->v_out};
                        const float *src[4] = {b->theta + o, b->grad + o, b->m + o, b->v + o};
                        cudaError_t ce2 = cudaSuccess;
                        for (int k = 0; k < 4 && ce2 == cudaSuccess; ++k) {
                            dst[k]->resize(b->n_theta);
                            ce2 = cudaMemcpy(dst[k]->data(), src[k], nb, cudaMemcpyDeviceToHost);
                        }
                        if (ce2 != cudaSuccess) {
                            status = DLX_ERR_CUDA;
                            for (auto *d : dst) d->clear();
                        }
                    }
                    finish(s, q, status);
                    const int last = b->active - 1;
                    if (r != last) {
                        move_slot(b, last, r);
                        s->stats.slot_moves++;
                    }
                    b->slot_req[last] = nullptr;
                    b->active--;
                    cudaStreamSynchronize(b->stream);
                }
            }
        }
        if (derr) cudaMemset(live[0]->plan->err, 0, 4);
        s->cv_done.notify_all();
    }
}

void copy_out(const Req *q, dlx_result *out) {
    out->loss = q->loss;
    out->queued_s = secs(q->t_submit, q->t_admit);
    out->latency_s = secs(q->t_submit, q->t_done);
    out->steps_done = q->steps_done;
    out->adam_step = q->step_in + q->n_steps;  // K = 0 evaluates with every rate at zero: no Adam step
    if (q->theta_out.empty()) return;
    if (out->adam_m) memcpy(out->adam_m, q->m_out.data(), 4 * q->m_out.size());
    if (out->adam_v) memcpy(out->adam_v, q->v_out.data(), 4 * q->v_out.size());
    const dlx_mft_desc &d = q->desc;
    const int *off = q->off;
    auto cp = [&](float *dst, const std::vector<float> &src, int o, size_t n) {
        if (dst && n) memcpy(dst, src.data() + o, 4 * n);
    };
    const size_t npx = (size_t)d.n_pupil * d.n_pupil, np = (size_t)d.n_det * d.n_det;
    cp(out->zern_coeff, q->theta_out, off[0], d.n_zern);
    if (q->has_pix) cp(out->opd_pix, q->theta_out, off[1], npx);
    cp(out->flat, q->theta_out, off[2], np);
    cp(out->flux, q->theta_out, off[3], d.n_src);
    cp(out->pos, q->theta_out, off[4], 2 * (size_t)d.n_src);
    cp(out->g_zern, q->grad_out, off[0], d.n_zern);
    if (q->has_pix) cp(out->g_opd_pix, q->grad_out, off[1], npx);
    cp(out->g_flat, q->grad_out, off[2], np);
    cp(out->g_flux, q->grad_out, off[3], d.n_src);
    cp(out->g_pos, q->grad_out, off[4], 2 * (size_t)d.n_src);
}

}  // namespace

extern "C" {

int dlx_server_create(int device, size_t hbm_budget, int max_slots, dlx_server **out) {
    if (!out || max_slots < 1) return fail(DLX_ERR_INVALID_ARG, "out is NULL or max_slots < 1");
    *out = nullptr;
    int prev = 0;
    cudaGetDevice(&prev);
    if (cudaSetDevice(device) != cudaSuccess) return fail(DLX_ERR_CUDA, "cudaSetDevice failed");
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
        cudaSetDevice(prev);
        return fail(DLX_ERR_CUDA, "cudaMemGetInfo failed");
    }
    cudaSetDevice(prev);
    auto *s = new dlx_server();
    s->device = device;
    s->budget = hbm_budget ? hbm_budget : (size_t)(0.9 * (double)fr);
    s->max_slots = max_slots;
    s->stats.hbm_budget = s->budget;
    s->worker = std::thread(worker_loop, s);
    *out = s;
    return DLX_OK;
}

int dlx_server_destroy(dlx_server *s) {
    if (!s) return DLX_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(s->device);
    for (auto &kv : s->buckets) destroy_bucket(kv.second.get());
    cudaSetDevice(prev);
    delete s;
    return DLX_OK;
}

int dlx_submit(dlx_server *s, const dlx_request *rq, uint64_t *ticket) {
    if (!s || !rq || !ticket) return fail(DLX_ERR_INVALID_ARG, "NULL argument");
    const dlx_mft_desc &d = rq->desc;
    if (d.n_pupil < 2 || d.n_det < 1 || d.oversample < 1 || d.n_lambda < 1 || d.n_src < 1 || d.n_exp < 1 ||
        d.n_zern < 0 || !d.lambda_m || d.precision < DLX_FP32_SIMT || d.precision > DLX_BF16X3SA)
        return fail(DLX_ERR_INVALID_ARG, "bad request shape");
    if (d.n_src > dlx::kMaxSrc) return fail(DLX_ERR_RANGE, "at most 32 sources");
    if (d.dither_px)
        for (int k = 0; k < 2 * d.n_exp; ++k)
            if (d.dither_px[k] < -4096 || d.dither_px[k] > 4096) return fail(DLX_ERR_RANGE, "|dither_px| <= 4096");
    if (!(d.focal_length_m >= 0) || !std::isfinite(d.focal_length_m) || !std::isfinite(d.focal_shift_m) ||
        (d.focal_length_m == 0 && d.focal_shift_m != 0) ||
        (d.focal_length_m > 0 && !(d.focal_length_m + d.focal_shift_m > 0)))
        return fail(DLX_ERR_INVALID_ARG, "bad focal_length_m / focal_shift_m");
    if (!rq->transmission || !rq->weights || !rq->flux || !rq->pos || !rq->flat || !rq->data ||
        (d.n_zern > 0 && (!rq->zern_basis || !rq->zern_coeff)) || rq->n_steps < 0)
        return fail(DLX_ERR_INVALID_ARG, "missing request input");
    if (rq->adam_step < 0 || rq->adam_step > (1 << 30) - rq->n_steps)
        return fail(DLX_ERR_INVALID_ARG, "adam_step must be >= 0 (and adam_step + n_steps < 2^30)");
    auto q = std::make_unique<Req>();
    q->desc = d;
    q->lambdas.assign(d.lambda_m, d.lambda_m + d.n_lambda);
    q->desc.lambda_m = nullptr;
    if (d.dither_px) q->dither_px.assign(d.dither_px, d.dither_px + 2 * (size_t)d.n_exp);
    q->desc.dither_px = q->dither_px.empty() ? nullptr : q->dither_px.data();  // the request's own copy
    q->has_pix = rq->opd_pix != nullptr;
    const size_t npx = (size_t)d.n_pupil * d.n_pupil, np = (size_t)d.n_det * d.n_det;
    auto cp = [](std::vector<float> &dst, const float *src, size_t n) {
        if (src) dst.assign(src, src + n);
    };
    cp(q->T, rq->transmission, npx);
    cp(q->opd_fixed, rq->opd_fixed, npx);
    cp(q->basis, rq->zern_basis, (size_t)d.n_zern * npx);
    cp(q->weights, rq->weights, d.n_lambda);
    cp(q->dither, rq->dither, 2 * (size_t)d.n_exp);
    cp(q->coeff, rq->zern_coeff, d.n_zern);
    cp(q->pix, rq->opd_pix, npx);
    cp(q->flux, rq->flux, d.n_src);
    cp(q->pos, rq->pos, 2 * (size_t)d.n_src);
    cp(q->flat, rq->flat, np);
    q->data.assign(rq->data, rq->data + (size_t)d.n_exp * np);
    q->n_steps = rq->n_steps;
    for (int k = 0; k < 5; ++k) q->lr[k] = rq->lr[k];
    const size_t nth = theta_size(d, q->has_pix);
    cp(q->m_in, rq->adam_m, nth);
    cp(q->v_in, rq->adam_v, nth);
    q->step_in = rq->adam_step;
    const size_t need = bucket_bytes(d, q->has_pix, 1);
    std::lock_guard<std::mutex> lk(s->mu);
    s->stats.submitted++;
    if (need > s->budget) {
        s->stats.rejected++;
        return fail(DLX_ERR_NOMEM, "request alone exceeds the server's HBM budget");
    }
    q->ticket = s->next_ticket++;
    q->t_submit = clk::now();
    *ticket = q->ticket;
    s->queue.push_back(q.get());
    s->reqs[q->ticket] = std::move(q);
    s->cv_work.notify_all();
    return DLX_OK;
}

int dlx_poll(dlx_server *s, uint64_t ticket, double timeout_s, dlx_result *out) {
    if (!s) return fail(DLX_ERR_INVALID_ARG, "server is NULL");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return fail(DLX_ERR_INVALID_ARG, "unknown or already released ticket");
    Req *q = it->second.get();
    if (!q->done && timeout_s > 0) {
        const auto deadline = clk::now() + std::chrono::duration<double>(timeout_s);
        s->cv_done.wait_until(lk, deadline, [&] { return q->done; });
        if (!q->done) return fail(DLX_ERR_TIMEOUT, "poll deadline passed");
    }
    if (!q->done) return DLX_PENDING;
    const int status = q->status;
    if (status == DLX_OK && out) copy_out(q, out);
    if (status != DLX_OK) dlx_set_error("request failed");
    s->reqs.erase(it);
    return status;
}

int dlx_server_get_stats(dlx_server *s, dlx_server_stats *out) {
    if (!s || !out) return fail(DLX_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    *out = s->stats;
    out->hbm_in_use = s->in_use;
    out->queued = (int)s->queue.size();
    return DLX_OK;
}

int dlx_server_inject_fault(dlx_server *s, int kind) {
    if (!s || kind < 1 || kind > 2) return fail(DLX_ERR_INVALID_ARG, "fault kind is 1 (admission NOMEM) or 2 (NaN input)");
    std::lock_guard<std::mutex> lk(s->mu);
    s->fault_next = kind;
    return DLX_OK;
}

}  // extern "C"
